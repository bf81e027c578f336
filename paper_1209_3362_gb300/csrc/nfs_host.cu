// Host side of the C ABI declared in include/nfs.h: context lifecycle, the frame pipeline
// (copy -> exact mean -> row FFT -> column FFT -> delay update), binning tables and timings.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "nfs_internal.cuh"
#include "roi.cuh"

using namespace nfs;

namespace {

constexpr int kDefaultBlock = kDelayBlock;  // K: frames per fused delay update
constexpr int kMaxBlock = kDelayBlock;      // largest K the fused kernel takes
constexpr int kMaxChunk = 64;       // largest FFT chunk (FP64 path)
constexpr int kMaxChunkF32 = 32;    // largest FFT chunk of the FP32 path (its scratch holds 32 frames)
constexpr int kDefaultChunkF32 = 32; // FFT chunk of the FP32 path (measured on 2048x2048 frames: row and
                                     // column passes 19.0 us per frame at 32 frames per launch pair,
                                     // 19.6 at 16, 24.0 at 4)
constexpr int kMaxDim = 4096;
// Frames a context takes between resets: the delay kernels index frames with 32-bit integers.
constexpr long long kMaxFrames = (1LL << 31) - 4096;
constexpr int kMaxDelay = 65536;

bool factors_2_3(int n)
{
    if (n <= 0) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

long long gcd_ll(long long a, long long b)
{
    while (b) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// floor(2 nq sqrt(r2) / L) = the largest b with (b L)^2 <= 4 nq^2 r2, exact in 128-bit integers
// (4 nq^2 r2 exceeds 64 bits once nq lcm(H, W) passes ~3e9).
unsigned long long radial_bin(unsigned long long r2, long long nq, long long L)
{
    typedef unsigned __int128 u128;
    const u128 a = (u128)4 * (u128)nq * (u128)nq * (u128)r2;
    unsigned long long b = (unsigned long long)(2.0 * (double)nq * std::sqrt((double)r2) / (double)L);
    auto sq = [L](unsigned long long x) { const u128 y = (u128)x * (u128)L; return y * y; };
    while (b > 0 && sq(b) > a) --b;
    while (sq(b + 1) <= a) ++b;
    return b;
}

struct TimedPair {
    int stage;
    cudaEvent_t a, b;
};

}  // namespace

struct nfs_ctx {
    Geometry g{};
    int path = NFS_PATH_FUSED_F32;
    int K = kDefaultBlock;
    int R = 0, nd = 0, nq = 0;
    int fft_chunk = 4;
    int stage_frames = 1;
    int delay_variant = 0;
    int fft_generic = 0;  // 1: generic FFT kernels even where specialised ones exist
    int stall_group = -1; // test hook of the bounded-wait path (NFS_OPT_TEST_STALL_GROUP)
    bool own_streams = true;   // false for members of a batch (the batch owns the streams)
    bool defer_delay = false;  // members of a batch: the batch runs the delay update of full blocks
    int device = 0;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    std::vector<int32_t> delays;
    int tau_max = 0;

    // Host-push staging: a device ring of n_slots copy chunks of copy_frames frames each, so the
    // copy stream can run up to about two delay blocks ahead of the kernels; pageable sources pass
    // through two pinned host chunks first.
    int copy_frames = 1, n_slots = 2;
    uint16_t *d_stage = nullptr;
    uint16_t *h_stage[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_filled, ev_free;
    cudaEvent_t ev_hcopied[2] = {nullptr, nullptr};
    long long stage_i = 0, hstage_i = 0;

    unsigned long long *d_sums = nullptr;
    float *d_ref = nullptr;
    void *d_ring = nullptr;
    void *d_acc = nullptr;
    int *d_delays = nullptr;
    void *d_tw_row = nullptr, *d_tw_post = nullptr, *d_tw_col = nullptr;
    float2 *d_tws_row = nullptr, *d_tws_col = nullptr;  // per-stage twiddles of the specialised FFTs
    float2 *d_scratch = nullptr;                         // FP32 row-pass output, kMaxChunkF32 frames
    FftPlan plan_row, plan_col;
    int *d_bin_off = nullptr, *d_bin_modes = nullptr;
    long long *d_pairs = nullptr, *d_counts = nullptr;
    double *d_D = nullptr, *d_export = nullptr;
    DelaySchedule *sched = nullptr;  // tiled-kernel schedule (host copy, passed by value); NULL if too long
    int *d_err = nullptr;
    // Cross pass (one band of the out-of-core mode): pairs (block frame of the "current" sequence,
    // older frame of the "old" sequence); the current sequence's spectra go to d_ring_cur (K slots),
    // the old sequence's to d_ring.  Both sequences advance together: frame u of each per step.
    bool cross = false;
    void *d_ring_cur = nullptr;
    long long transforms = 0;  // frames transformed (both sequences of a cross pass)

    std::vector<long long> counts, pairs_h;
    std::vector<double> qmean;
    long long nframes = 0, nprocessed = 0;
    bool have_ref = false;

    int err = NFS_OK;
    std::string errmsg;

    int timing = 0;  // 1: events around every launch; 2: around delay-update launches only
    std::vector<TimedPair> pending;
    std::vector<cudaEvent_t> pool;
    double stage_ms[NFS_N_STAGES] = {};
    long long stage_n[NFS_N_STAGES] = {};
    long long launches = 0;

    bool f32() const { return path == NFS_PATH_FUSED_F32; }
    size_t csize() const { return f32() ? sizeof(float2) : sizeof(double2); }
    size_t asize() const { return f32() ? sizeof(float2) : sizeof(double); }
    size_t frame_bytes() const { return g.HW * sizeof(uint16_t); }
};

namespace {

int set_cuda_error(nfs_ctx *c, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return NFS_OK;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    c->errmsg = buf;
    if (c->err == NFS_OK) c->err = NFS_ECUDA;
    return NFS_ECUDA;
}

#define CK(ctx, call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return set_cuda_error((ctx), _e, #call); \
    } while (0)

cudaEvent_t pool_get(nfs_ctx *c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Runs one launcher with optional event timing around it.
template <class F>
int timed(nfs_ctx *c, int stage, cudaStream_t s, F &&f, const char *what)
{
    cudaEvent_t a = nullptr, b = nullptr;
    const bool on = c->timing == 1 || (c->timing == 2 && stage == NFS_STAGE_DELAY);
    if (on) {
        a = pool_get(c);
        b = pool_get(c);
        if (!a || !b) return set_cuda_error(c, cudaErrorMemoryAllocation, "cudaEventCreate");
        CK(c, cudaEventRecord(a, s));
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return set_cuda_error(c, e, what);
    if (on) {
        CK(c, cudaEventRecord(b, s));
        c->pending.push_back({stage, a, b});
    }
    if (stage != NFS_STAGE_H2D) c->launches++;
    return NFS_OK;
}

int harvest(nfs_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0.f;
        CK(c, cudaEventSynchronize(p.b));
        CK(c, cudaEventElapsedTime(&ms, p.a, p.b));
        c->stage_ms[p.stage] += ms;
        c->stage_n[p.stage] += 1;
        c->pool.push_back(p.a);
        c->pool.push_back(p.b);
    }
    c->pending.clear();
    return NFS_OK;
}

template <typename T>
int upload_twiddles(nfs_ctx *c, int L, void **dst)
{
    using C = typename cplx_t<T>::type;
    std::vector<C> h((size_t)std::max(L, 1));
    for (int m = 0; m < L; ++m) {
        double a = 2.0 * M_PI * (double)m / (double)L;
        h[m].x = (T)std::cos(a);
        h[m].y = (T)(-std::sin(a));
    }
    CK(c, cudaMalloc(dst, sizeof(C) * h.size()));
    CK(c, cudaMemcpy(*dst, h.data(), sizeof(C) * h.size(), cudaMemcpyHostToDevice));
    return NFS_OK;
}

// r2c post-processing twiddles exp(-2 pi i k / W), k = 0..W/2.
template <typename T>
int upload_post(nfs_ctx *c, int W, void **dst)
{
    using C = typename cplx_t<T>::type;
    std::vector<C> h((size_t)(W / 2 + 1));
    for (int k = 0; k <= W / 2; ++k) {
        double a = 2.0 * M_PI * (double)k / (double)W;
        h[k].x = (T)std::cos(a);
        h[k].y = (T)(-std::sin(a));
    }
    CK(c, cudaMalloc(dst, sizeof(C) * h.size()));
    CK(c, cudaMemcpy(*dst, h.data(), sizeof(C) * h.size(), cudaMemcpyHostToDevice));
    return NFS_OK;
}

// Per-stage twiddles of the size-specialised FP32 kernels (FP64 on the host, rounded once).
int upload_stage_twiddles(nfs_ctx *c, int L, float2 **dst)
{
    const std::vector<double> t = ct_stage_twiddles(L);
    std::vector<float2> h(std::max<size_t>(t.size() / 2, 1));
    for (size_t i = 0; i < t.size() / 2; ++i) h[i] = {(float)t[2 * i], (float)t[2 * i + 1]};
    CK(c, cudaMalloc((void **)dst, sizeof(float2) * h.size()));
    CK(c, cudaMemcpy(*dst, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
    return NFS_OK;
}

// Radial bin of every half-plane mode (integer rule of the header): bin_of[ky * (W/2+1) + kx] is the
// bin or -1 (the DC mode and |f| >= 0.5), counts[b] = C_b (weights 1 or 2), qmean[b] the weighted
// mean of 2 pi |f| over the bin (0 for an empty bin).  Host arithmetic only.
void bin_table(int H, int W, int nq, std::vector<int> *bin_of, std::vector<long long> *counts,
               std::vector<double> *qmean)
{
    const int Wh = W / 2 + 1;
    const long long L = (long long)H / gcd_ll(H, W) * W;
    std::vector<double> qsum((size_t)nq, 0.0);
    bin_of->assign((size_t)H * Wh, -1);
    counts->assign((size_t)nq, 0);
    for (int ky = 0; ky < H; ++ky) {
        const long long kys = (ky <= H / 2) ? ky : ky - H;
        for (int kx = 0; kx < Wh; ++kx) {
            if (kx == 0 && ky == 0) continue;
            const long long m = (long long)kx * (L / W), n = kys * (L / H);
            const unsigned long long r2 = (unsigned long long)(m * m + n * n);
            const unsigned long long b = radial_bin(r2, nq, L);
            if (b >= (unsigned long long)nq) continue;
            const int w = (kx != 0 && kx != W / 2) ? 2 : 1;
            (*bin_of)[(size_t)ky * Wh + kx] = (int)b;
            (*counts)[b] += w;
            qsum[b] += (double)w * 2.0 * M_PI * std::sqrt((double)r2) / (double)L;
        }
    }
    qmean->assign((size_t)nq, 0.0);
    for (int b = 0; b < nq; ++b)
        if ((*counts)[b]) (*qmean)[b] = qsum[b] / (double)(*counts)[b];
}

// The bin table of the context as a CSR list of (mode index << 1 | weight-is-2) by bin, on the device.
int build_bins(nfs_ctx *c)
{
    const int H = c->g.H, W = c->g.W, Wh = c->g.Wh, nq = c->nq;
    std::vector<int> bin_of;
    bin_table(H, W, nq, &bin_of, &c->counts, &c->qmean);
    std::vector<std::vector<int>> lists((size_t)nq);
    for (int ky = 0; ky < H; ++ky)
        for (int kx = 0; kx < Wh; ++kx) {
            const int b = bin_of[(size_t)ky * Wh + kx];
            if (b < 0) continue;
            const int two = (kx != 0 && kx != W / 2) ? 1 : 0;
            lists[b].push_back((int)(((long long)c->g.mode(kx, ky) << 1) | two));
        }
    std::vector<int> off((size_t)nq + 1, 0), modes;
    for (int b = 0; b < nq; ++b) off[b + 1] = off[b] + (int)lists[b].size();
    modes.reserve((size_t)off[nq]);
    for (int b = 0; b < nq; ++b) modes.insert(modes.end(), lists[b].begin(), lists[b].end());
    CK(c, cudaMalloc(&c->d_bin_off, sizeof(int) * off.size()));
    CK(c, cudaMemcpy(c->d_bin_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    CK(c, cudaMalloc(&c->d_bin_modes, sizeof(int) * std::max<size_t>(modes.size(), 1)));
    if (!modes.empty())
        CK(c, cudaMemcpy(c->d_bin_modes, modes.data(), sizeof(int) * modes.size(), cudaMemcpyHostToDevice));
    CK(c, cudaMalloc(&c->d_counts, sizeof(long long) * (size_t)nq));
    CK(c, cudaMemcpy(c->d_counts, c->counts.data(), sizeof(long long) * (size_t)nq, cudaMemcpyHostToDevice));
    return NFS_OK;
}

void free_all(nfs_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    cudaFree(c->d_stage);
    for (auto e : c->ev_filled) cudaEventDestroy(e);
    for (auto e : c->ev_free) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
        if (c->h_stage[i]) cudaFreeHost(c->h_stage[i]);
        if (c->ev_hcopied[i]) cudaEventDestroy(c->ev_hcopied[i]);
    }
    cudaFree(c->d_sums);
    cudaFree(c->d_ref);
    cudaFree(c->d_ring);
    cudaFree(c->d_ring_cur);
    cudaFree(c->d_acc);
    cudaFree(c->d_delays);
    cudaFree(c->d_tw_row);
    cudaFree(c->d_tw_post);
    cudaFree(c->d_tw_col);
    cudaFree(c->d_tws_row);
    cudaFree(c->d_tws_col);
    cudaFree(c->d_scratch);
    cudaFree(c->d_bin_off);
    cudaFree(c->d_bin_modes);
    cudaFree(c->d_pairs);
    cudaFree(c->d_counts);
    cudaFree(c->d_D);
    cudaFree(c->d_export);
    delete c->sched;
    cudaFree(c->d_err);
    if (c->own_streams) {
        if (c->stream) cudaStreamDestroy(c->stream);
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    }
}

int alloc_dev(nfs_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return NFS_ENOMEM;
    }
    return set_cuda_error(c, e, "cudaMalloc");
}

int flush_block(nfs_ctx *c)
{
    const long long nb = c->nframes - c->nprocessed;
    if (nb <= 0 || !c->f32()) return NFS_OK;
    DelayArgs a;
    a.ring = (const float2 *)c->d_ring;
    a.R = c->R;
    a.M = c->g.M;
    a.t0 = c->nprocessed;
    a.nb = (int)nb;
    a.delays = c->d_delays;
    a.nd = c->nd;
    a.acc = (float2 *)c->d_acc;
    a.sched = c->sched;
    a.err = c->d_err;
    a.tau_max = c->tau_max;
    a.stall_group = c->stall_group;
    if (c->cross) {
        a.ring_cur = (const float2 *)c->d_ring_cur;
        a.R_cur = c->K;
    }
    int rc = timed(c, NFS_STAGE_DELAY, c->stream, [&] { return launch_delay_f32(a, c->delay_variant, c->stream); },
                   "delay_f32");
    if (rc) return rc;
    c->nprocessed = c->nframes;
    return NFS_OK;
}

// Exact spatial sums of n device-resident frames (n <= kMaxChunk) into sums[0 .. n), in one launch
// for a whole copy chunk; the reference image comes from the first group the context ever sees
// (its first frame that is not dark).
int frame_sums(nfs_ctx *c, const uint16_t *dsrc, int n, unsigned long long *sums)
{
    CK(c, cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * (size_t)n, c->stream));
    int rc = timed(c, NFS_STAGE_MEAN, c->stream, [&] { return launch_frame_sums(dsrc, n, c->g, sums, c->stream); },
                   "frame_sums");
    if (rc) return rc;
    if (!c->have_ref && c->f32()) {
        rc = timed(c, NFS_STAGE_MEAN, c->stream, [&] { return launch_reference(dsrc, sums, n, c->g, c->d_ref, c->stream); },
                   "reference");
        if (rc) return rc;
        c->have_ref = true;
    }
    return NFS_OK;
}

// Transform nf device-resident frames (nf <= fft chunk) whose sums are in sums[0 .. nf) and, when a
// block is complete, update.  A cross context takes the old sequence's frames first (old = true:
// into the ring at the slots of frames nframes .., no count, no update) and then the same number
// of the current sequence's frames (into the K-slot current ring; these count and trigger the
// update).
int process_chunk(nfs_ctx *c, const uint16_t *dsrc, int nf, bool old, const unsigned long long *sums)
{
    int rc = NFS_OK;
    c->transforms += nf;
    const bool to_cur = c->cross && !old;
    float2 *ring = (float2 *)(to_cur ? c->d_ring_cur : c->d_ring);
    const int R = to_cur ? c->K : c->R;
    const int slot0 = (int)(c->nframes % R);
    if (c->f32()) {
        rc = timed(c, NFS_STAGE_ROWFFT, c->stream, [&] {
            return launch_row_fft<float>(dsrc, nf, sums, c->d_ref, c->g, c->plan_row, (const float2 *)c->d_tw_row,
                                         (const float2 *)c->d_tw_post, ring, R, slot0, c->stream,
                                         c->d_scratch, c->fft_generic ? nullptr : c->d_tws_row);
        }, "row_fft_f32");
        if (rc) return rc;
        rc = timed(c, NFS_STAGE_COLFFT, c->stream, [&] {
            return launch_col_fft<float>(nf, c->g, c->plan_col, (const float2 *)c->d_tw_col, ring, R,
                                         slot0, c->stream, c->d_scratch, c->fft_generic ? nullptr : c->d_tws_col);
        }, "col_fft_f32");
        if (rc) return rc;
        if (old) return NFS_OK;
        c->nframes += nf;
        if (c->nframes - c->nprocessed >= c->K && !c->defer_delay) return flush_block(c);
        return NFS_OK;
    }
    rc = timed(c, NFS_STAGE_ROWFFT, c->stream, [&] {
        return launch_row_fft<double>(dsrc, nf, sums, nullptr, c->g, c->plan_row, (const double2 *)c->d_tw_row,
                                      (const double2 *)c->d_tw_post, (double2 *)c->d_ring, c->R, slot0, c->stream);
    }, "row_fft_f64");
    if (rc) return rc;
    rc = timed(c, NFS_STAGE_COLFFT, c->stream, [&] {
        return launch_col_fft<double>(nf, c->g, c->plan_col, (const double2 *)c->d_tw_col, (double2 *)c->d_ring, c->R,
                                      slot0, c->stream);
    }, "col_fft_f64");
    if (rc) return rc;
    for (int f = 0; f < nf; ++f) {
        const long long t = c->nframes + f;
        rc = timed(c, NFS_STAGE_DELAY, c->stream, [&] {
            return launch_delay_f64((const double2 *)c->d_ring, c->R, c->g.M, t, c->d_delays, c->nd, (double *)c->d_acc,
                                    c->stream);
        }, "delay_f64");
        if (rc) return rc;
    }
    c->nframes += nf;
    c->nprocessed = c->nframes;
    if (c->timing && c->pending.size() > 200000) return harvest(c);
    return NFS_OK;
}

// FFT launch-pair size (frames per row/column launch) chosen by measurement per frame shape:
// candidates 1, 2, 4, 8, 16, 32 each transform 32 zero frames from the staging ring; the fastest is
// kept for the process (a context's first transform of a shape pays for the measurement).
int autotune_fft_chunk(nfs_ctx *c)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    const std::pair<int, int> key(c->g.H, c->g.W);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            c->fft_chunk = it->second;
            return NFS_OK;
        }
    }
    const int nfr = kMaxChunkF32;
    const int cands[6] = {1, 2, 4, 8, 16, 32};
    CK(c, cudaMemsetAsync(c->d_sums, 0, sizeof(unsigned long long) * kMaxChunk, c->stream));
    CK(c, cudaMemsetAsync(c->d_ref, 0, sizeof(float) * c->g.HW, c->stream));
    CK(c, cudaMemsetAsync(c->d_stage, 0, c->frame_bytes() * nfr, c->stream));
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    int best = c->fft_chunk;
    float best_ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep)  // the first round warms up
        for (int cand : cands) {
            CK(c, cudaEventRecord(e0, c->stream));
            for (int o = 0; o < nfr; o += cand) {
                if (launch_row_fft<float>(c->d_stage + (size_t)o * c->g.HW, cand, c->d_sums, c->d_ref, c->g, c->plan_row,
                                          (const float2 *)c->d_tw_row, (const float2 *)c->d_tw_post, (float2 *)c->d_ring,
                                          c->R, o, c->stream, c->d_scratch, c->d_tws_row) != cudaSuccess ||
                    launch_col_fft<float>(cand, c->g, c->plan_col, (const float2 *)c->d_tw_col, (float2 *)c->d_ring, c->R,
                                          o, c->stream, c->d_scratch, c->d_tws_col) != cudaSuccess)
                    return set_cuda_error(c, cudaGetLastError(), "autotune");
                c->launches += 2;
            }
            CK(c, cudaEventRecord(e1, c->stream));
            CK(c, cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(c, cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->fft_chunk = best;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    return NFS_OK;
}


// Frames the next chunk may take so that a chunk never spans two delay blocks.
int next_chunk(const nfs_ctx *c, long long remaining, int cap)
{
    long long nf = std::min<long long>(remaining, cap);
    if (c->f32()) nf = std::min<long long>(nf, c->K - (c->nframes - c->nprocessed));
    return (int)std::max<long long>(nf, 1);
}

int enter(nfs_ctx *c)
{
    if (!c) return NFS_EINVAL;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return set_cuda_error(c, e, "cudaSetDevice");
    return c->err;
}

// The argument checks of nfs_create_ex, made before any CUDA call.
int check_args(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block)
{
    if (!delays || n_delays <= 0 || n_qbins <= 0 || n_qbins > 65536) return NFS_EINVAL;
    if (path != NFS_PATH_FUSED_F32 && path != NFS_PATH_PLAIN_F64) return NFS_EINVAL;
    if (block < 0 || block > kMaxBlock) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j) {
        if (delays[j] < 0 || delays[j] > kMaxDelay) return NFS_EINVAL;
        if (j && delays[j] <= delays[j - 1]) return NFS_EINVAL;
    }
    if (H < 2 || W < 2 || H > kMaxDim || W > kMaxDim || (H % 2) || (W % 2) || !factors_2_3(H) || !factors_2_3(W / 2))
        return NFS_EUNSUPPORTED;
    return NFS_OK;
}

int create_impl(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block, nfs_ctx **out,
                bool cross = false)
{
    if (!out) return NFS_EINVAL;
    if (cross && path != NFS_PATH_FUSED_F32) return NFS_EINVAL;
    *out = nullptr;
    const int rc_args = check_args(H, W, delays, n_delays, n_qbins, path, block);
    if (rc_args) return rc_args;

    nfs_ctx *c = new (std::nothrow) nfs_ctx();
    if (!c) return NFS_ENOMEM;
    cudaGetDevice(&c->device);
    c->path = path;
    c->K = block ? block : kDefaultBlock;
    c->cross = cross;
    c->nd = n_delays;
    c->nq = n_qbins;
    c->delays.assign(delays, delays + n_delays);
    c->tau_max = delays[n_delays - 1];
    c->g = make_geometry(H, W, c->f32());
    c->R = c->tau_max + (c->f32() ? c->K : kMaxChunk);
    c->stage_frames = (int)std::max<size_t>(
        1, std::min<size_t>(c->f32() ? kMaxChunkF32 : kMaxChunk, (64u << 20) / c->frame_bytes()));
    c->fft_chunk = c->f32() ? kDefaultChunkF32 : std::min(4, c->stage_frames);
    c->pairs_h.assign((size_t)n_delays, 0);

    int rc = NFS_OK;
    auto bail = [&](int r) {
        free_all(c);
        delete c;
        return r;
    };
    if (!make_plan(c->g.Lr, &c->plan_row) || !make_plan(H, &c->plan_col)) return bail(NFS_EUNSUPPORTED);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(NFS_ECUDA);
    // copy chunks of up to 256 MB; the device staging ring covers two delay blocks, at most 4 GB
    c->copy_frames = (int)std::max<size_t>(1, std::min<size_t>(64, (256u << 20) / c->frame_bytes()));
    {
        const size_t cap = std::max<size_t>(2, (size_t(4) << 30) / (c->frame_bytes() * (size_t)c->copy_frames));
        const size_t want = std::max<size_t>(2, (2 * (size_t)c->K + c->copy_frames - 1) / c->copy_frames);
        c->n_slots = (int)std::min(cap, want);
    }
    c->ev_filled.assign((size_t)c->n_slots, nullptr);
    c->ev_free.assign((size_t)c->n_slots, nullptr);
    for (int i = 0; i < c->n_slots; ++i)
        if (cudaEventCreateWithFlags(&c->ev_filled[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(NFS_ECUDA);
    for (int i = 0; i < 2; ++i)
        if (cudaEventCreateWithFlags(&c->ev_hcopied[i], cudaEventDisableTiming) != cudaSuccess) return bail(NFS_ECUDA);
    if ((rc = alloc_dev(c, (void **)&c->d_stage, c->frame_bytes() * (size_t)c->copy_frames * c->n_slots)))
        return bail(rc);
    const size_t ring_bytes = (size_t)c->R * c->g.M * c->csize();
    const size_t acc_bytes = (size_t)c->nd * c->g.M * c->asize();
    // sums of up to two copy chunks (a cross pass stages one of each sequence)
    if ((rc = alloc_dev(c, (void **)&c->d_sums, sizeof(unsigned long long) * 2 * kMaxChunk))) return bail(rc);
    if (c->f32() && (rc = alloc_dev(c, (void **)&c->d_ref, sizeof(float) * c->g.HW))) return bail(rc);
    if ((rc = alloc_dev(c, &c->d_ring, ring_bytes))) return bail(rc);
    if (cross && (rc = alloc_dev(c, &c->d_ring_cur, (size_t)c->K * c->g.M * c->csize()))) return bail(rc);
    if ((rc = alloc_dev(c, &c->d_acc, acc_bytes))) return bail(rc);
    if ((rc = alloc_dev(c, (void **)&c->d_delays, sizeof(int) * (size_t)c->nd))) return bail(rc);
    if ((rc = alloc_dev(c, (void **)&c->d_pairs, sizeof(long long) * (size_t)c->nd))) return bail(rc);
    if ((rc = alloc_dev(c, (void **)&c->d_D, sizeof(double) * (size_t)c->nd * c->nq))) return bail(rc);
    if (cudaMemcpy(c->d_delays, c->delays.data(), sizeof(int) * (size_t)c->nd, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(NFS_ECUDA);
    if (cudaMemset(c->d_acc, 0, acc_bytes) != cudaSuccess) return bail(NFS_ECUDA);
    if (c->f32()) {
        if (upload_twiddles<float>(c, c->g.Lr, &c->d_tw_row) || upload_twiddles<float>(c, H, &c->d_tw_col) ||
            upload_post<float>(c, W, &c->d_tw_post) || upload_stage_twiddles(c, c->g.Lr, &c->d_tws_row) ||
            upload_stage_twiddles(c, H, &c->d_tws_col))
            return bail(NFS_ECUDA);
        if ((rc = alloc_dev(c, (void **)&c->d_scratch, sizeof(float2) * (size_t)kMaxChunkF32 * H * c->g.Wp)))
            return bail(rc);
    } else {
        if (upload_twiddles<double>(c, c->g.Lr, &c->d_tw_row) || upload_twiddles<double>(c, H, &c->d_tw_col) ||
            upload_post<double>(c, W, &c->d_tw_post))
            return bail(NFS_ECUDA);
    }
    if (build_bins(c)) return bail(NFS_ECUDA);
    if ((rc = alloc_dev(c, (void **)&c->d_err, sizeof(int) * kDelayErrWords))) return bail(rc);
    if (cudaMemset(c->d_err, 0, sizeof(int) * kDelayErrWords) != cudaSuccess) return bail(NFS_ECUDA);
    if (c->f32()) {
        std::vector<SubRun> srs;
        std::vector<Stage> sts;
        if (!build_delay_schedule(c->delays.data(), c->nd, cross, &srs, &sts)) return bail(NFS_EUNSUPPORTED);
        // a delay list too long for the parameter-space schedule uses the one-thread-per-mode kernel
        if (srs.size() <= (size_t)kMaxSubRuns && sts.size() <= (size_t)kMaxSchedStages) {
            c->sched = new (std::nothrow) DelaySchedule();
            if (!c->sched) return bail(NFS_ENOMEM);
            c->sched->nsr = (int)srs.size();
            c->sched->nst = (int)sts.size();
            c->sched->nbatch = count_delay_batches(srs);
            std::copy(srs.begin(), srs.end(), c->sched->sr);
            std::copy(sts.begin(), sts.end(), c->sched->st);
        }
        if (cross && !c->sched) return bail(NFS_EUNSUPPORTED);  // cross passes run on the tiled kernel only
    }
    *out = c;
    return NFS_OK;
}

bool is_page_locked(const void *p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

int nfs_create(int H, int W, const int32_t *delays, int n_delays, int n_qbins, nfs_ctx **out)
{
    return create_impl(H, W, delays, n_delays, n_qbins, NFS_PATH_FUSED_F32, 0, out);
}

int nfs_create_ex(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block_frames,
                  nfs_ctx **out)
{
    return create_impl(H, W, delays, n_delays, n_qbins, path, block_frames, out);
}

int nfs_bin_table(int H, int W, int n_qbins, int32_t *bin_of_mode, int64_t *bin_counts, double *q_mean)
{
    if (!bin_counts || n_qbins <= 0 || n_qbins > 65536) return NFS_EINVAL;
    if (H < 2 || W < 2 || H > kMaxDim || W > kMaxDim || (H % 2) || (W % 2) || !factors_2_3(H) || !factors_2_3(W / 2))
        return NFS_EUNSUPPORTED;
    std::vector<int> bin_of;
    std::vector<long long> counts;
    std::vector<double> qmean;
    bin_table(H, W, n_qbins, &bin_of, &counts, &qmean);
    if (bin_of_mode) std::copy(bin_of.begin(), bin_of.end(), bin_of_mode);
    std::copy(counts.begin(), counts.end(), bin_counts);
    if (q_mean) std::copy(qmean.begin(), qmean.end(), q_mean);
    return NFS_OK;
}

int nfs_push_frames(nfs_ctx *c, const uint16_t *h, int n)
{
    int rc = enter(c);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !h)) return NFS_EINVAL;
    if (n == 0) return NFS_OK;
    if (c->nframes + n > kMaxFrames) return NFS_ESTATE;
    const bool locked = is_page_locked(h);
    if (!locked && !c->h_stage[0]) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaMallocHost((void **)&c->h_stage[i], c->frame_bytes() * (size_t)c->copy_frames);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return NFS_ENOMEM;
            }
        }
    }
    long long done = 0;
    int last = -1;
    while (done < n) {
        const int nc = (int)std::min<long long>(c->copy_frames, n - done);
        const int slot = (int)(c->stage_i++ % c->n_slots);
        const size_t bytes = c->frame_bytes() * (size_t)nc;
        uint16_t *dst = c->d_stage + (size_t)slot * c->copy_frames * c->g.HW;
        const uint16_t *src = h + (size_t)done * c->g.HW;
        // the kernels that read this slot last time must be done before it is overwritten
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[slot], 0));
        int hs = -1;
        if (!locked) {
            hs = (int)(c->hstage_i++ & 1);
            CK(c, cudaEventSynchronize(c->ev_hcopied[hs]));
            memcpy(c->h_stage[hs], src, bytes);
            src = c->h_stage[hs];
        }
        rc = timed(c, NFS_STAGE_H2D, c->copy_stream, [&] {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->copy_stream);
        }, "h2d");
        if (rc) return rc;
        if (hs >= 0) CK(c, cudaEventRecord(c->ev_hcopied[hs], c->copy_stream));
        CK(c, cudaEventRecord(c->ev_filled[slot], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_filled[slot], 0));
        if ((rc = frame_sums(c, dst, nc, c->d_sums))) return rc;
        for (int o = 0; o < nc;) {
            const int nf = next_chunk(c, nc - o, c->fft_chunk);
            rc = process_chunk(c, dst + (size_t)o * c->g.HW, nf, false, c->d_sums + o);
            if (rc) return rc;
            o += nf;
        }
        CK(c, cudaEventRecord(c->ev_free[slot], c->stream));
        done += nc;
        last = slot;
    }
    // copies run in order on the copy stream: when the last one is done the caller's buffer is free
    if (locked && last >= 0) CK(c, cudaEventSynchronize(c->ev_filled[last]));
    return c->err;
}

int nfs_push_frames_device(nfs_ctx *c, const uint16_t *d, int n)
{
    int rc = enter(c);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !d) || (reinterpret_cast<uintptr_t>(d) & 1)) return NFS_EINVAL;
    if (c->nframes + n > kMaxFrames) return NFS_ESTATE;
    long long done = 0;
    while (done < n) {
        const int ng = (int)std::min<long long>(kMaxChunk, n - done);
        const uint16_t *grp = d + (size_t)done * c->g.HW;
        if ((rc = frame_sums(c, grp, ng, c->d_sums))) return rc;
        for (int o = 0; o < ng;) {
            const int nf = next_chunk(c, ng - o, c->fft_chunk);
            if ((rc = process_chunk(c, grp + (size_t)o * c->g.HW, nf, false, c->d_sums + o))) return rc;
            o += nf;
        }
        done += ng;
    }
    return c->err;
}

int nfs_structure_function(nfs_ctx *c, double *D, int64_t *bin_counts, int64_t *pair_counts, double *q_mean)
{
    int rc = enter(c);
    if (rc) return rc;
    if (!D || !bin_counts || !pair_counts) return NFS_EINVAL;
    if ((rc = flush_block(c))) return rc;
    for (int j = 0; j < c->nd; ++j) c->pairs_h[j] = std::max<long long>(0, c->nframes - c->delays[j]);
    CK(c, cudaMemcpyAsync(c->d_pairs, c->pairs_h.data(), sizeof(long long) * (size_t)c->nd, cudaMemcpyHostToDevice,
                          c->stream));
    rc = timed(c, NFS_STAGE_BIN, c->stream, [&] {
        return c->f32() ? launch_bin<float2>((const float2 *)c->d_acc, c->g.M, c->nd, c->nq, c->d_bin_off,
                                             c->d_bin_modes, c->d_pairs, c->d_counts, c->d_D, c->stream)
                        : launch_bin<double>((const double *)c->d_acc, c->g.M, c->nd, c->nq, c->d_bin_off,
                                             c->d_bin_modes, c->d_pairs, c->d_counts, c->d_D, c->stream);
    }, "bin");
    if (rc) return rc;
    CK(c, cudaMemcpyAsync(D, c->d_D, sizeof(double) * (size_t)c->nd * c->nq, cudaMemcpyDeviceToHost, c->stream));
    int dev_err[kDelayErrWords] = {};
    CK(c, cudaMemcpyAsync(dev_err, c->d_err, sizeof(dev_err), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (dev_err[0]) {
        char buf[1024];
        int n = snprintf(buf, sizeof(buf),
                         "delay kernel: a bounded wait gave up (kind %d, cta %d, warp %d, index %d, polls %d, ns %d, "
                         "cycles %d, progress %d, drained %d; steps/batches per warp:",
                         dev_err[1], dev_err[2], dev_err[3], dev_err[4], dev_err[5], dev_err[6], dev_err[7],
                         dev_err[8], dev_err[9]);
        for (int w = 0; w < 16 && n > 0 && n < (int)sizeof(buf) - 16; ++w)
            n += snprintf(buf + n, sizeof(buf) - n, " %d/%d", dev_err[10 + w], dev_err[26 + w]);
        if (n > 0 && n < (int)sizeof(buf) - 2) snprintf(buf + n, sizeof(buf) - n, ")");
        c->errmsg = buf;
        if (c->err == NFS_OK) c->err = NFS_ETIMEOUT;
        return c->err;
    }
    for (int b = 0; b < c->nq; ++b) bin_counts[b] = c->counts[b];
    for (int j = 0; j < c->nd; ++j) pair_counts[j] = c->pairs_h[j];
    if (q_mean)
        for (int b = 0; b < c->nq; ++b) q_mean[b] = c->qmean[b];
    if (c->timing && (rc = harvest(c))) return rc;
    return c->err;
}

int nfs_export_spectrum(nfs_ctx *c, int j, double *out)
{
    int rc = enter(c);
    if (rc) return rc;
    if (!out || j < 0 || j >= c->nd) return NFS_EINVAL;
    if ((rc = flush_block(c))) return rc;
    const size_t n = (size_t)c->g.H * c->g.Wh;
    if (!c->d_export && (rc = alloc_dev(c, (void **)&c->d_export, sizeof(double) * n))) return rc;
    const long long pairs = std::max<long long>(0, c->nframes - c->delays[j]);
    cudaError_t e = c->f32() ? launch_export<float2>((const float2 *)c->d_acc + (size_t)j * c->g.M, c->g, pairs,
                                                     c->d_export, c->stream)
                             : launch_export<double>((const double *)c->d_acc + (size_t)j * c->g.M, c->g, pairs,
                                                     c->d_export, c->stream);
    CK(c, e);
    c->launches++;
    CK(c, cudaMemcpyAsync(out, c->d_export, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return c->err;
}

int nfs_reset(nfs_ctx *c)
{
    int rc = enter(c);
    if (rc) return rc;
    CK(c, cudaMemsetAsync(c->d_acc, 0, (size_t)c->nd * c->g.M * c->asize(), c->stream));
    c->nframes = 0;
    c->nprocessed = 0;
    c->have_ref = false;
    return NFS_OK;
}

int nfs_synchronize(nfs_ctx *c)
{
    int rc = enter(c);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(c->copy_stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (c->timing && (rc = harvest(c))) return rc;
    return c->err;
}

int64_t nfs_frame_count(const nfs_ctx *c) { return c ? c->nframes : -1; }

void nfs_destroy(nfs_ctx *c)
{
    if (!c) return;
    free_all(c);
    delete c;
}

const char *nfs_strerror(int s)
{
    switch (s) {
        case NFS_OK: return "ok";
        case NFS_EINVAL: return "invalid argument";
        case NFS_EUNSUPPORTED: return "unsupported frame shape";
        case NFS_ENOMEM: return "out of memory";
        case NFS_ECUDA: return "CUDA error";
        case NFS_ESTATE: return "call not allowed in this state";
        case NFS_ETOOBIG: return "problem too large for the no-allocation scratch";
        case NFS_ETIMEOUT: return "a device-side wait ran out of time";
        default: return "unknown status";
    }
}

const char *nfs_last_error(const nfs_ctx *c) { return c ? c->errmsg.c_str() : ""; }

void *nfs_get_stream(const nfs_ctx *c) { return c ? (void *)c->stream : nullptr; }

int nfs_set_option(nfs_ctx *c, int key, int64_t v)
{
    int rc = enter(c);
    if (rc) return rc;
    switch (key) {
        case NFS_OPT_TIMING:
            if (v < 0 || v > 2) return NFS_EINVAL;
            c->timing = (int)v;
            return NFS_OK;
        case NFS_OPT_FFT_CHUNK:
            if (v == 0 && c->f32()) {
                // the measurement transforms zero frames into the ring with a zero reference image
                if (c->nframes > 0 || c->have_ref) return NFS_ESTATE;
                return autotune_fft_chunk(c);
            }
            if (v < 1 || v > (c->f32() ? kMaxChunkF32 : kMaxChunk)) return NFS_EINVAL;
            c->fft_chunk = (int)v;
            return NFS_OK;
        case NFS_OPT_DELAY_VARIANT:
            if (v < 0 || v > 2) return NFS_EINVAL;
            c->delay_variant = (int)v;
            return NFS_OK;
        case NFS_OPT_FFT_GENERIC:
            if (v < 0 || v > 1) return NFS_EINVAL;
            c->fft_generic = (int)v;
            return NFS_OK;
        case NFS_OPT_TEST_STALL_GROUP:
            if (v < -1 || v > 1000000) return NFS_EINVAL;
            c->stall_group = (int)v;
            return NFS_OK;
        default: return NFS_EINVAL;
    }
}

int nfs_get_option(const nfs_ctx *c, int key, int64_t *v)
{
    if (!c || !v) return NFS_EINVAL;
    switch (key) {
        case NFS_OPT_TIMING: *v = c->timing; return NFS_OK;
        case NFS_OPT_BLOCK_FRAMES: *v = c->K; return NFS_OK;
        case NFS_OPT_RING_SLOTS: *v = c->R; return NFS_OK;
        case NFS_OPT_PITCH: *v = c->g.Wp; return NFS_OK;
        case NFS_OPT_PATH: *v = c->path; return NFS_OK;
        case NFS_OPT_FFT_CHUNK: *v = c->fft_chunk; return NFS_OK;
        case NFS_OPT_DELAY_VARIANT: *v = c->delay_variant; return NFS_OK;
        case NFS_OPT_FFT_GENERIC: *v = c->fft_generic; return NFS_OK;
        case NFS_OPT_TEST_STALL_GROUP: *v = c->stall_group; return NFS_OK;
        default: return NFS_EINVAL;
    }
}

int nfs_get_timings(nfs_ctx *c, double *ms, int64_t *launches)
{
    int rc = nfs_synchronize(c);
    if (rc) return rc;
    for (int s = 0; s < NFS_N_STAGES; ++s) {
        if (ms) ms[s] = c->stage_ms[s];
        if (launches) launches[s] = c->stage_n[s];
    }
    return NFS_OK;
}

int nfs_reset_timings(nfs_ctx *c)
{
    int rc = nfs_synchronize(c);
    if (rc) return rc;
    for (int s = 0; s < NFS_N_STAGES; ++s) {
        c->stage_ms[s] = 0.0;
        c->stage_n[s] = 0;
    }
    return NFS_OK;
}

int64_t nfs_launch_count(const nfs_ctx *c) { return c ? c->launches : -1; }

int nfs_fit(nfs_ctx *c, const double *D_in, float *A, float *B, float *Gamma, int iters, int method)
{
    int rc = enter(c);
    if (rc) return rc;
    if (!A || !B || !Gamma || iters < 0 || (method != NFS_FIT_GAUSS_NEWTON && method != NFS_FIT_ADAM)) return NFS_EINVAL;
    const int nd = c->nd, nq = c->nq;
    std::vector<double> Dh;
    std::vector<long long> pairs((size_t)nd);
    if (D_in) {
        for (int j = 0; j < nd; ++j) pairs[j] = std::max<long long>(0, c->nframes - c->delays[j]);
    } else {
        Dh.resize((size_t)nd * nq);
        std::vector<int64_t> bc((size_t)nq), pc((size_t)nd);
        if ((rc = nfs_structure_function(c, Dh.data(), bc.data(), pc.data(), nullptr))) return rc;
        for (int j = 0; j < nd; ++j) pairs[j] = pc[j];
        D_in = Dh.data();
    }
    // delays with pairs (a delay with none carries no data); tau = 0 carries no dynamics
    std::vector<float> Df, tf;
    for (int j = 0; j < nd; ++j) {
        if (pairs[j] <= 0 || c->delays[j] == 0) continue;
        tf.push_back((float)c->delays[j]);
        for (int b = 0; b < nq; ++b) Df.push_back((float)D_in[(size_t)j * nq + b]);
    }
    const int nu = (int)tf.size();
    if (nu == 0) return NFS_ESTATE;
    float *dD = nullptr, *dt = nullptr, *dp = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dD, sizeof(float) * Df.size(), c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dt, sizeof(float) * tf.size(), c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dp, sizeof(float) * 3 * (size_t)nq, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dD, Df.data(), sizeof(float) * Df.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, A, sizeof(float) * nq, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp + nq, B, sizeof(float) * nq, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp + 2 * nq, Gamma, sizeof(float) * nq, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        e = (method == NFS_FIT_GAUSS_NEWTON)
                ? launch_fit_gauss_newton(dD, dt, nu, nq, dp, dp + nq, dp + 2 * nq, iters, 1e-3f, c->stream)
                : launch_fit_adam(dD, dt, nu, nq, dp, dp + nq, dp + 2 * nq, iters, 1e-2f, c->stream);
        if (e == cudaSuccess) c->launches++;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(A, dp, sizeof(float) * nq, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B, dp + nq, sizeof(float) * nq, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Gamma, dp + 2 * nq, sizeof(float) * nq, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(dD, c->stream);
    cudaFreeAsync(dt, c->stream);
    cudaFreeAsync(dp, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? c->err : set_cuda_error(c, e, "nfs_fit");
}

// ---------------------------------------------------------------- ragged batch

struct nfs_batch {
    int n = 0, device = 0, n_sm = 0;
    std::vector<nfs_ctx *> seq;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    DelaySchedule *d_scheds = nullptr;  // one per sequence
    BatchItem *d_items = nullptr;       // work list of one launch
    int *d_err = nullptr;
    std::vector<BatchItem> items;
    int err = NFS_OK;
    std::string errmsg;
    long long launches = 0;
    // regions of interest (nfs_roi_create): windows of one H x W camera sequence
    int roi_H = 0, roi_W = 0;
    std::vector<RoiRect> rois;
    RoiRect *d_rois = nullptr;
    uint16_t *d_crop = nullptr;   // kRoiGroup frames of every window
    uint16_t *d_full = nullptr;   // kRoiGroup full frames (host pushes), allocated on first use
    long long roi_max_words = 0;  // 4-byte words of the largest window's group
};

static void batch_free(nfs_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    for (nfs_ctx *c : b->seq) nfs_destroy(c);
    cudaFree(b->d_scheds);
    cudaFree(b->d_items);
    cudaFree(b->d_err);
    cudaFree(b->d_rois);
    cudaFree(b->d_crop);
    cudaFree(b->d_full);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
    delete b;
}

static int batch_fail(nfs_batch *b, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return NFS_OK;
    b->errmsg = std::string(where) + ": " + cudaGetErrorString(e);
    if (b->err == NFS_OK) b->err = NFS_ECUDA;
    return NFS_ECUDA;
}

// One persistent launch over every member whose pending block is full (all = false) or non-empty
// (all = true).
static int batch_flush(nfs_batch *b, bool all)
{
    b->items.clear();
    long long total = 0;
    for (size_t s = 0; s < b->seq.size(); ++s) {
        nfs_ctx *c = b->seq[s];
        const long long pend = c->nframes - c->nprocessed;
        if (pend <= 0 || (!all && pend < c->K)) continue;
        int nst = 0, nbatch = 0;
        truncate_schedule(*c->sched, c->nframes - 1, &nst, &nbatch);
        if (nst > 0) {
            BatchItem it;
            it.ring = (const float2 *)c->d_ring;
            it.acc = (float2 *)c->d_acc;
            it.sched = b->d_scheds + s;
            it.t0 = c->nprocessed;
            it.first = total;
            it.M = c->g.M;
            it.R = c->R;
            it.nb = (int)pend;
            it.nd = c->nd;
            it.nst = nst;
            it.nbatch = nbatch;
            b->items.push_back(it);
            total += (long long)(c->g.M / kTile);
        }
        c->nprocessed = c->nframes;
    }
    if (b->items.empty()) return NFS_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BatchItem) * b->items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_delay_batched(b->d_items, (int)b->items.size(), total, b->d_err, b->n_sm, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batched delay update");
    b->launches++;
    return NFS_OK;
}

static int batch_enter(nfs_batch *b)
{
    if (!b) return NFS_EINVAL;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return batch_fail(b, e, "cudaSetDevice");
    return b->err;
}

// the device status of the batched launches (after a synchronisation)
static int batch_check(nfs_batch *b)
{
    int dev_err[kDelayErrWords] = {};
    cudaError_t e = cudaMemcpyAsync(dev_err, b->d_err, sizeof(dev_err), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch status");
    if (dev_err[0]) {
        char buf[160];
        snprintf(buf, sizeof(buf), "batched delay kernel: a bounded wait gave up (kind %d, cta %d, warp %d, index %d)",
                 dev_err[1], dev_err[2], dev_err[3], dev_err[4]);
        b->errmsg = buf;
        if (b->err == NFS_OK) b->err = NFS_ETIMEOUT;
    }
    return b->err;
}

int nfs_batch_create(int n_seq, const int *H, const int *W, const int32_t *delay_offsets, const int32_t *delays,
                     const int *n_qbins, nfs_batch **out)
{
    if (!out) return NFS_EINVAL;
    *out = nullptr;
    if (n_seq <= 0 || !H || !W || !delay_offsets || !delays || !n_qbins) return NFS_EINVAL;
    for (int s = 0; s < n_seq; ++s)
        if (delay_offsets[s + 1] <= delay_offsets[s]) return NFS_EINVAL;
    nfs_batch *b = new (std::nothrow) nfs_batch();
    if (!b) return NFS_ENOMEM;
    cudaGetDevice(&b->device);
    b->n = n_seq;
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    std::vector<DelaySchedule> scheds((size_t)n_seq);
    for (int s = 0; s < n_seq; ++s) {
        nfs_ctx *c = nullptr;
        const int rc = create_impl(H[s], W[s], delays + delay_offsets[s], delay_offsets[s + 1] - delay_offsets[s],
                                   n_qbins[s], NFS_PATH_FUSED_F32, 0, &c);
        if (rc) {
            batch_free(b);
            return rc;
        }
        b->seq.push_back(c);
        if (!c->sched) {  // delay list too long for the tiled kernel's schedule
            batch_free(b);
            return NFS_EUNSUPPORTED;
        }
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
        cudaStreamDestroy(c->copy_stream);
        c->stream = b->stream;
        c->copy_stream = b->copy_stream;
        c->own_streams = false;
        c->defer_delay = true;
        scheds[s] = *c->sched;
        if (autotune_fft_chunk(c)) {
            batch_free(b);
            return NFS_ECUDA;
        }
    }
    if (cudaMalloc(&b->d_scheds, sizeof(DelaySchedule) * (size_t)n_seq) != cudaSuccess ||
        cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)n_seq) != cudaSuccess ||
        cudaMalloc(&b->d_err, sizeof(int) * kDelayErrWords) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return NFS_ENOMEM;
    }
    if (cudaMemcpy(b->d_scheds, scheds.data(), sizeof(DelaySchedule) * (size_t)n_seq, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int) * kDelayErrWords) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    *out = b;
    return NFS_OK;
}

void nfs_batch_destroy(nfs_batch *b) { batch_free(b); }

int nfs_batch_push(nfs_batch *b, int seq, const uint16_t *host_frames, int n)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    if (seq < 0 || seq >= b->n || n < 0 || (n > 0 && !host_frames)) return NFS_EINVAL;
    nfs_ctx *c = b->seq[seq];
    long long done = 0;
    while (done < n) {
        const long long room = c->K - (c->nframes - c->nprocessed);
        if (room <= 0) {
            if ((rc = batch_flush(b, false))) return rc;
            continue;
        }
        const int m = (int)std::min<long long>(room, n - done);
        if ((rc = nfs_push_frames(c, host_frames + (size_t)done * c->g.HW, m))) return rc;
        done += m;
    }
    return b->err;
}

int nfs_batch_push_device(nfs_batch *b, const uint16_t *const *dev_frames, const int *n_frames)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    if (!dev_frames || !n_frames) return NFS_EINVAL;
    std::vector<long long> done((size_t)b->n, 0);
    for (int s = 0; s < b->n; ++s)
        if (n_frames[s] < 0 || (n_frames[s] > 0 && !dev_frames[s])) return NFS_EINVAL;
    for (;;) {
        bool left = false;
        for (int s = 0; s < b->n; ++s) {
            nfs_ctx *c = b->seq[s];
            const long long rem = n_frames[s] - done[s];
            if (rem <= 0) continue;
            left = true;
            const long long room = c->K - (c->nframes - c->nprocessed);
            if (room <= 0) continue;
            const int m = (int)std::min(room, rem);
            if ((rc = nfs_push_frames_device(c, dev_frames[s] + (size_t)done[s] * c->g.HW, m))) return rc;
            done[s] += m;
        }
        if (!left) break;
        // every member that still has frames now holds a full block: one launch for all of them
        if ((rc = batch_flush(b, false))) return rc;
    }
    return b->err;
}

int nfs_batch_structure_function(nfs_batch *b, int seq, double *D, int64_t *bin_counts, int64_t *pair_counts,
                                 double *q_mean)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    if (seq < 0 || seq >= b->n) return NFS_EINVAL;
    if ((rc = batch_flush(b, true))) return rc;
    if ((rc = batch_check(b))) return rc;
    return nfs_structure_function(b->seq[seq], D, bin_counts, pair_counts, q_mean);
}

int nfs_batch_reset(nfs_batch *b)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    for (nfs_ctx *c : b->seq)
        if ((rc = nfs_reset(c))) return rc;
    return NFS_OK;
}

int nfs_batch_synchronize(nfs_batch *b)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    return batch_check(b);
}

nfs_ctx *nfs_batch_member(nfs_batch *b, int seq) { return (b && seq >= 0 && seq < b->n) ? b->seq[seq] : nullptr; }

void *nfs_batch_get_stream(const nfs_batch *b) { return b ? (void *)b->stream : nullptr; }

int64_t nfs_batch_launch_count(const nfs_batch *b)
{
    if (!b) return -1;
    long long n = b->launches;
    for (nfs_ctx *c : b->seq) n += c->launches;
    return n;
}

const char *nfs_batch_last_error(const nfs_batch *b) { return b ? b->errmsg.c_str() : ""; }

// ---------------------------------------------------------------- regions of interest

// Frames cropped per launch: kRoiGroup frames of every window are cut from the full frames in one
// launch and pushed to the members as one device push.
constexpr int kRoiGroup = 64;

int nfs_roi_create(int H, int W, int n_roi, const int *y0, const int *x0, const int *h, const int *w,
                   const int32_t *delays, int n_delays, const int *n_qbins, nfs_batch **out)
{
    if (!out) return NFS_EINVAL;
    *out = nullptr;
    if (H <= 0 || W <= 0 || (W & 1) || n_roi <= 0 || !y0 || !x0 || !h || !w || !delays || n_delays <= 0 ||
        !n_qbins)
        return NFS_EINVAL;
    std::vector<RoiRect> rois((size_t)n_roi);
    long long off = 0, max_words = 0;
    for (int r = 0; r < n_roi; ++r) {
        if (y0[r] < 0 || x0[r] < 0 || h[r] <= 0 || w[r] <= 0 || (x0[r] & 1) || (w[r] & 1) || y0[r] > H - h[r] ||
            x0[r] > W - w[r])
            return NFS_EINVAL;
        const long long words = (long long)kRoiGroup * h[r] * (w[r] / 2);
        if (words >= (1LL << 31)) return NFS_EINVAL;  // the crop kernel's 32-bit indices
        const int rc_args = check_args(h[r], w[r], delays, n_delays, n_qbins[r], NFS_PATH_FUSED_F32, 0);
        if (rc_args) return rc_args;
        rois[(size_t)r] = RoiRect{y0[r], x0[r], h[r], w[r], off};
        off += (2 * words + 127) / 128 * 128;  // each window's frames start 256-byte aligned
        max_words = std::max(max_words, words);
    }
    std::vector<int> Hs((size_t)n_roi), Ws((size_t)n_roi), offs((size_t)n_roi + 1);
    std::vector<int32_t> dl((size_t)n_roi * n_delays);
    for (int r = 0; r < n_roi; ++r) {
        Hs[(size_t)r] = h[r];
        Ws[(size_t)r] = w[r];
        offs[(size_t)r] = r * n_delays;
        std::copy(delays, delays + n_delays, dl.begin() + (size_t)r * n_delays);
    }
    offs[(size_t)n_roi] = n_roi * n_delays;
    nfs_batch *b = nullptr;
    int rc = nfs_batch_create(n_roi, Hs.data(), Ws.data(), offs.data(), dl.data(), n_qbins, &b);
    if (rc) return rc;
    b->roi_H = H;
    b->roi_W = W;
    b->rois = rois;
    b->roi_max_words = max_words;
    if (cudaMalloc(&b->d_rois, sizeof(RoiRect) * rois.size()) != cudaSuccess ||
        cudaMalloc(&b->d_crop, sizeof(uint16_t) * (size_t)off) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return NFS_ENOMEM;
    }
    if (cudaMemcpy(b->d_rois, rois.data(), sizeof(RoiRect) * rois.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    *out = b;
    return NFS_OK;
}

int nfs_roi_push_device(nfs_batch *b, const uint16_t *d, int n)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    if (b->rois.empty() || n < 0 || (n > 0 && !d) || (reinterpret_cast<uintptr_t>(d) & 3)) return NFS_EINVAL;
    const size_t HW = (size_t)b->roi_H * b->roi_W;
    std::vector<const uint16_t *> ptrs(b->rois.size());
    std::vector<int> counts(b->rois.size());
    for (long long done = 0; done < n;) {
        const int nc = (int)std::min<long long>(kRoiGroup, n - done);
        cudaError_t e = launch_roi_crop(d + (size_t)done * HW, b->roi_H, b->roi_W, nc, b->d_rois,
                                        (int)b->rois.size(), b->roi_max_words, b->n_sm, b->d_crop, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest crop");
        b->launches++;
        // the members' kernels read the crop buffer on the batch's stream, before the next crop
        for (size_t r = 0; r < b->rois.size(); ++r) {
            ptrs[r] = b->d_crop + b->rois[r].dst;
            counts[r] = nc;
        }
        if ((rc = nfs_batch_push_device(b, ptrs.data(), counts.data()))) return rc;
        done += nc;
    }
    return b->err;
}

int nfs_roi_push(nfs_batch *b, const uint16_t *host, int n)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    if (b->rois.empty() || n < 0 || (n > 0 && !host)) return NFS_EINVAL;
    if (n == 0) return NFS_OK;
    const size_t HW = (size_t)b->roi_H * b->roi_W;
    if (!b->d_full && cudaMalloc(&b->d_full, sizeof(uint16_t) * HW * kRoiGroup) != cudaSuccess) {
        cudaGetLastError();
        return NFS_ENOMEM;
    }
    const bool locked = is_page_locked(host);
    for (long long done = 0; done < n;) {
        const int nc = (int)std::min<long long>(kRoiGroup, n - done);
        // stream-ordered after the previous group's crop, which reads d_full
        cudaError_t e = cudaMemcpyAsync(b->d_full, host + (size_t)done * HW, sizeof(uint16_t) * HW * nc,
                                        cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest upload");
        if ((rc = nfs_roi_push_device(b, b->d_full, nc))) return rc;
        done += nc;
    }
    // page-locked sources are copied asynchronously: the caller's buffer is free once they are done
    if (locked) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest upload");
    }
    return b->err;
}

}  // extern "C"

// ------------------------------------------------------------------ out-of-core bands
//
// When the ring for every delay does not fit, the delays are split into bands processed one after
// the other, each re-reading the frames from host memory (the paper's FIFO re-upload, organised
// by delay bands).  Band 0 is an ordinary pass over the delays d with d + K <= the slot budget.
// A later band with smallest delay lo takes the shift s = floor(lo / K) K and runs a cross pass:
// current sequence C_u = frame u + s (K-slot ring), old sequence O_u = frame u (ring of
// e_max + K slots), delays e = d - s, so the pair (C_u, O_{u-e}) is the pair (u + s, u + s - d).
// The block boundaries of C fall on multiples of K in the original frame index (s is a multiple
// of K), so every pair is added in the same block and warp as in one in-core pass.

namespace {

// One band: delays [first, last) of the list, shift s (s = 0: the ordinary pass).
struct Band {
    int first, last;
    long long shift;
};

// Does the tiled kernel's schedule of these (shifted) delays fit its parameter space?
bool schedule_fits(const std::vector<int> &d, bool cross)
{
    std::vector<SubRun> srs;
    std::vector<Stage> sts;
    if (!build_delay_schedule(d.data(), (int)d.size(), cross, &srs, &sts)) return false;
    return srs.size() <= (size_t)kMaxSubRuns && sts.size() <= (size_t)kMaxSchedStages;
}

int plan_bands(const int32_t *delays, int nd, long long N, long long max_slots, std::vector<Band> *bands,
               long long *n_transforms)
{
    bands->clear();
    *n_transforms = 0;
    const long long K = kDefaultBlock;
    int j = 0;
    while (j < nd) {
        const long long lo = delays[j];
        const bool first = bands->empty();
        // band 0 runs in place when its first delay fits; later bands are cross passes
        const bool in_place = first && lo + K <= max_slots;
        const long long s = in_place ? 0 : lo / K * K;
        const long long hi_max = in_place ? max_slots - K : max_slots - 2 * K + s;
        // a cross pass needs its first delay within the budget (always so for budgets of 3K slots)
        if (!in_place && (lo < K || lo > hi_max)) return NFS_EINVAL;
        int e = j;
        while (e < nd && delays[e] <= hi_max) ++e;
        // keep the band within the tiled kernel's schedule limits
        for (;;) {
            std::vector<int> d;
            for (int q = j; q < e; ++q) d.push_back((int)(delays[q] - s));
            if (schedule_fits(d, !in_place)) break;
            e = j + (e - j) / 2;
            if (e == j) return NFS_EUNSUPPORTED;
        }
        bands->push_back({j, e, s});
        if (in_place)
            *n_transforms += N;
        else if (N > s)
            *n_transforms += 2 * (N - s);
        j = e;
    }
    return NFS_OK;
}

// A cross pass over host frames: old sequence `old` and current sequence `cur`, n frames each
// (pinned or pageable; read before the call returns).
int cross_push(nfs_ctx *c, const uint16_t *cur, const uint16_t *old, long long n)
{
    const bool locked = is_page_locked(cur) && is_page_locked(old);
    if (!locked && !c->h_stage[0]) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaMallocHost((void **)&c->h_stage[i], c->frame_bytes() * (size_t)c->copy_frames);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return NFS_ENOMEM;
            }
        }
    }
    // copy nc frames from src into the next staging slot; returns the slot
    auto stage = [&](const uint16_t *src, int nc, int *slot_out) -> int {
        const int slot = (int)(c->stage_i++ % c->n_slots);
        uint16_t *dst = c->d_stage + (size_t)slot * c->copy_frames * c->g.HW;
        const size_t bytes = c->frame_bytes() * (size_t)nc;
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[slot], 0));
        int hs = -1;
        if (!locked) {
            hs = (int)(c->hstage_i++ & 1);
            CK(c, cudaEventSynchronize(c->ev_hcopied[hs]));
            memcpy(c->h_stage[hs], src, bytes);
            src = c->h_stage[hs];
        }
        const int rc = timed(c, NFS_STAGE_H2D, c->copy_stream, [&] {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->copy_stream);
        }, "h2d");
        if (rc) return rc;
        if (hs >= 0) CK(c, cudaEventRecord(c->ev_hcopied[hs], c->copy_stream));
        CK(c, cudaEventRecord(c->ev_filled[slot], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_filled[slot], 0));
        *slot_out = slot;
        return NFS_OK;
    };
    long long done = 0;
    int last = -1;
    while (done < n) {
        const int nc = (int)std::min<long long>(c->copy_frames, n - done);
        int so = 0, sc = 0, rc;
        if ((rc = stage(old + (size_t)done * c->g.HW, nc, &so))) return rc;
        if ((rc = stage(cur + (size_t)done * c->g.HW, nc, &sc))) return rc;
        const uint16_t *dold = c->d_stage + (size_t)so * c->copy_frames * c->g.HW;
        const uint16_t *dcur = c->d_stage + (size_t)sc * c->copy_frames * c->g.HW;
        // the old sequence's first frame (frame 0) gives the reference image
        if ((rc = frame_sums(c, dold, nc, c->d_sums))) return rc;
        if ((rc = frame_sums(c, dcur, nc, c->d_sums + kMaxChunk))) return rc;
        for (int o = 0; o < nc;) {
            const int nf = next_chunk(c, nc - o, c->fft_chunk);
            if ((rc = process_chunk(c, dold + (size_t)o * c->g.HW, nf, true, c->d_sums + o))) return rc;
            if ((rc = process_chunk(c, dcur + (size_t)o * c->g.HW, nf, false, c->d_sums + kMaxChunk + o))) return rc;
            o += nf;
        }
        CK(c, cudaEventRecord(c->ev_free[so], c->stream));
        CK(c, cudaEventRecord(c->ev_free[sc], c->stream));
        done += nc;
        last = sc;
    }
    if (locked && last >= 0) CK(c, cudaEventSynchronize(c->ev_filled[last]));
    return c->err;
}

}  // namespace

extern "C" {

int nfs_out_of_core_plan(const int32_t *delays, int n_delays, int64_t n_frames, int64_t max_ring_slots,
                         int32_t *band_first, int64_t *band_shift, int *n_bands, int64_t *n_transforms)
{
    if (!delays || n_delays <= 0 || n_frames < 0 || !n_bands || !n_transforms) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<Band> bands;
    long long nt = 0;
    const int rc = plan_bands(delays, n_delays, n_frames, max_ring_slots, &bands, &nt);
    if (rc) return rc;
    *n_bands = (int)bands.size();
    *n_transforms = nt;
    for (size_t b = 0; b < bands.size(); ++b) {
        if (band_first) band_first[b] = bands[b].first;
        if (band_shift) band_shift[b] = bands[b].shift;
    }
    if (band_first) band_first[bands.size()] = n_delays;
    return NFS_OK;
}

int nfs_structure_function_out_of_core(int H, int W, const int32_t *delays, int n_delays, int n_qbins,
                                       const uint16_t *frames, int64_t n_frames, int64_t max_ring_slots, double *D,
                                       int64_t *bin_counts, int64_t *pair_counts, double *q_mean,
                                       int64_t *n_transforms)
{
    if (!delays || n_delays <= 0 || n_qbins <= 0 || !D || !bin_counts || !pair_counts) return NFS_EINVAL;
    if (n_frames < 0 || n_frames > kMaxFrames || (n_frames > 0 && !frames)) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<Band> bands;
    long long planned = 0;
    int rc = plan_bands(delays, n_delays, n_frames, max_ring_slots, &bands, &planned);
    if (rc) return rc;
    const size_t HW = (size_t)H * W;
    long long done = 0;
    std::vector<double> Db;
    std::vector<int64_t> pc;
    for (const Band &b : bands) {
        const int nb = b.last - b.first;
        std::vector<int32_t> d(delays + b.first, delays + b.last);
        for (int32_t &x : d) x -= (int32_t)b.shift;
        nfs_ctx *c = nullptr;
        rc = create_impl(H, W, d.data(), nb, n_qbins, NFS_PATH_FUSED_F32, 0, &c, b.shift > 0);
        if (rc) return rc;
        Db.assign((size_t)nb * n_qbins, 0.0);
        pc.assign((size_t)nb, 0);
        if (b.shift == 0)
            rc = n_frames > 0 ? nfs_push_frames(c, frames, (int)n_frames) : NFS_OK;
        else if (n_frames > b.shift)
            rc = cross_push(c, frames + (size_t)b.shift * HW, frames, n_frames - b.shift);
        if (!rc) rc = nfs_structure_function(c, Db.data(), bin_counts, pc.data(), q_mean);
        done += c->transforms;
        nfs_destroy(c);
        if (rc) return rc;
        std::copy(Db.begin(), Db.end(), D + (size_t)b.first * n_qbins);
        for (int q = 0; q < nb; ++q) pair_counts[b.first + q] = n_frames > b.shift ? pc[q] : 0;
    }
    if (done != planned) return NFS_ESTATE;  // the passes transformed other frames than planned
    if (n_transforms) *n_transforms = done;
    return NFS_OK;
}

}  // extern "C"

extern "C" int nfs_delay_schedule(const int32_t *delays, int n_delays, int cross, int32_t *subruns, int32_t *stages,
                                  int max_entries, int *n_subruns, int *n_stages, int *block_frames,
                                  int *slot_rows, int *copy_barriers)
{
    if (!delays || n_delays <= 0 || !n_subruns || !n_stages) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<SubRun> srs;
    std::vector<Stage> sts;
    if (!build_delay_schedule(delays, n_delays, cross != 0, &srs, &sts)) return NFS_EUNSUPPORTED;
    *n_subruns = (int)srs.size();
    *n_stages = (int)sts.size();
    if (block_frames) *block_frames = kDelayBlock;
    if (slot_rows) *slot_rows = kSlotBuf;
    if (copy_barriers) *copy_barriers = kFullBars;
    if ((subruns && (int)srs.size() > max_entries) || (stages && (int)sts.size() > max_entries)) return NFS_ETOOBIG;
    for (size_t i = 0; subruns && i < srs.size(); ++i) {
        subruns[3 * i] = srs[i].j0;
        subruns[3 * i + 1] = srs[i].len;
        subruns[3 * i + 2] = srs[i].d0;
    }
    for (size_t i = 0; stages && i < sts.size(); ++i) {
        stages[5 * i] = sts[i].sr0;
        stages[5 * i + 1] = sts[i].nsr;
        stages[5 * i + 2] = sts[i].lo;
        stages[5 * i + 3] = sts[i].hi;
        stages[5 * i + 4] = sts[i].need;
    }
    return NFS_OK;
}
