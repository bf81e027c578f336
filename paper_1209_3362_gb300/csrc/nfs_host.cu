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

#include "nfs_host.cuh"

using namespace nfs;
using namespace nfs::host;

namespace {

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

}  // namespace

namespace nfs {
namespace host {

int set_cuda_error(nfs_ctx *c, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return NFS_OK;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    c->errmsg = buf;
    if (c->err == NFS_OK) c->err = NFS_ECUDA;
    return NFS_ECUDA;
}

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

int harvest(nfs_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0.f;
        CK(c, cudaEventSynchronize(p.b));
        CK(c, cudaEventElapsedTime(&ms, p.a, p.b));
        c->stage_ms[p.stage] += ms;
        c->stage_n[p.stage] += 1;
        if (c->timing == 3) {
            if (!c->tl_base) {
                c->tl_base = p.a;  // kept (not pooled) until the next reset of the timings
            }
            float t0 = 0.f, t1 = 0.f;
            CK(c, cudaEventElapsedTime(&t0, c->tl_base, p.a));
            CK(c, cudaEventElapsedTime(&t1, c->tl_base, p.b));
            c->timeline.push_back({p.stage, (double)t0, (double)t1});
        }
        if (p.a != c->tl_base) c->pool.push_back(p.a);
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
    std::vector<char> binned_tile(c->g.M / kTile, 0);
    for (int ky = 0; ky < H; ++ky)
        for (int kx = 0; kx < Wh; ++kx) {
            const int b = bin_of[(size_t)ky * Wh + kx];
            if (b < 0) continue;
            const long long kl = (long long)c->g.mode(kx, ky) - (long long)c->g.k0;  // slab-local index
            if (kl < 0 || kl >= (long long)c->g.M) continue;
            const int two = (kx != 0 && kx != W / 2) ? 1 : 0;
            lists[b].push_back((int)((kl << 1) | two));
            binned_tile[(size_t)kl / kTile] = 1;
        }
    std::vector<int> tiles;
    for (size_t t = 0; t < binned_tile.size(); ++t)
        if (binned_tile[t]) tiles.push_back((int)t);
    c->n_tiles_binned = (long long)tiles.size();
    CK(c, cudaMalloc(&c->d_tiles, sizeof(int) * std::max<size_t>(tiles.size(), 1)));
    if (!tiles.empty())
        CK(c, cudaMemcpy(c->d_tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice));
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
    if (c->tl_base) cudaEventDestroy(c->tl_base);
    cudaFree(c->d_stage);
    for (auto e : c->ev_filled) cudaEventDestroy(e);
    for (auto e : c->ev_free) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
        if (c->h_stage[i]) cudaFreeHost(c->h_stage[i]);
        if (c->ev_hcopied[i]) cudaEventDestroy(c->ev_hcopied[i]);
    }
    cudaFree(c->d_sums);
    cudaFree(c->d_slot_sums);
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
    cudaFree(c->d_tiles);
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

int release_slots(nfs_ctx *c)
{
    for (int s : c->free_pending) CK(c, cudaEventRecord(c->ev_free[s], c->stream));
    c->free_pending.clear();
    return NFS_OK;
}

int flush_block(nfs_ctx *c)
{
    const long long nb = c->nframes - c->nprocessed;
    if (nb <= 0 || !c->f32()) return NFS_OK;
    int rc = release_slots(c);  // recorded before the launch: the refills run beside it
    if (rc) return rc;
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
    if (!c->modes_all) {
        a.tiles = c->d_tiles;
        a.ntiles = (size_t)c->n_tiles_binned;
    }
    rc = timed(c, NFS_STAGE_DELAY, c->stream, [&] { return launch_delay_f32(a, c->delay_variant, c->stream); },
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
    return reference_once(c, dsrc, n, sums);
}

int reference_once(nfs_ctx *c, const uint16_t *dsrc, int n, const unsigned long long *sums)
{
    int rc = NFS_OK;
    if (!c->have_ref && c->f32()) {
        rc = timed(c, NFS_STAGE_MEAN, c->stream, [&] {
            char *base = reinterpret_cast<char *>(c->d_ref);
            return launch_reference(dsrc, sums, n, c->g, c->d_ref, c->stream,
                                    reinterpret_cast<uint16_t *>(base + ref_raw_offset(c->g.HW)),
                                    reinterpret_cast<float2 *>(base + ref_inv_offset(c->g.HW)));
        }, "reference");
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
    CK(c, cudaMemsetAsync(c->d_ref, 0, ref_buffer_bytes(c->g.HW), c->stream));
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

// The tiled kernel's schedule rebuilt with another stage span (NFS_EUNSUPPORTED, keeping the old
// one, if the span is out of range or the schedule would not fit the kernel parameters).
int set_delay_span(nfs_ctx *c, int span)
{
    if (!c->f32() || !c->sched) return NFS_EUNSUPPORTED;
    std::vector<SubRun> srs;
    std::vector<Stage> sts;
    if (!build_delay_schedule(c->delays.data(), c->nd, c->cross, &srs, &sts, span)) return NFS_EUNSUPPORTED;
    if (srs.size() > (size_t)kMaxSubRuns || sts.size() > (size_t)kMaxSchedStages) return NFS_EUNSUPPORTED;
    c->sched->nsr = (int)srs.size();
    c->sched->nst = (int)sts.size();
    c->sched->nbatch = count_delay_batches(srs);
    std::copy(srs.begin(), srs.end(), c->sched->sr);
    std::copy(sts.begin(), sts.end(), c->sched->st);
    c->span = span;
    return NFS_OK;
}

// Stage span chosen by measurement on this context's delay list: each candidate runs the tiled
// kernel in steady state (block t0 = tau_max, all stages active) over 8 tiles per SM of a zeroed
// ring, twice after one warm-up launch; the fastest is kept.  The accumulators are cleared
// afterwards (only before the first frame: the measurement uses the ring and the accumulators).
int autotune_delay_span(nfs_ctx *c)
{
    if (!c->f32() || !c->sched || c->cross) return NFS_EUNSUPPORTED;
    int n_sm = 0;
    CK(c, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    const size_t tiles = std::min<size_t>(c->g.M / kTile, (size_t)8 * (size_t)std::max(n_sm, 1));
    CK(c, cudaMemsetAsync(c->d_ring, 0, (size_t)c->R * c->g.M * c->csize(), c->stream));
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    const int cands[5] = {112, 176, 240, 320, 400};
    const int start = c->span;
    int best = start;
    float best_ms = 1e30f;
    int rc = NFS_OK;
    for (int cand : cands) {
        if (set_delay_span(c, cand) != NFS_OK) continue;
        DelayArgs a;
        a.ring = (const float2 *)c->d_ring;
        a.R = c->R;
        a.M = tiles * kTile;
        a.t0 = c->tau_max;
        a.nb = c->K;
        a.delays = c->d_delays;
        a.nd = c->nd;
        a.acc = (float2 *)c->d_acc;
        a.sched = c->sched;
        a.err = c->d_err;
        a.tau_max = c->tau_max;
        a.stall_group = -1;
        float tot = 0.f;
        for (int rep = 0; rep < 3 && rc == NFS_OK; ++rep) {
            if (cudaEventRecord(e0, c->stream) != cudaSuccess || launch_delay_f32(a, 0, c->stream) != cudaSuccess ||
                cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = set_cuda_error(c, cudaGetLastError(), "span autotune");
                break;
            }
            c->launches++;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) tot += ms;
        }
        if (rc) break;
        if (tot < best_ms) {
            best_ms = tot;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    int dev_err = 0;
    CK(c, cudaMemcpy(&dev_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_err) {
        c->errmsg = "span autotune: a bounded wait of the delay kernel gave up";
        if (c->err == NFS_OK) c->err = NFS_ETIMEOUT;
        return c->err;
    }
    CK(c, cudaMemsetAsync(c->d_acc, 0, (size_t)c->nd * c->g.M * c->asize(), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return set_delay_span(c, best);
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
    // n_delays is the binning launch's grid rows (at most 65535)
    if (!delays || n_delays <= 0 || n_delays > 65535 || n_qbins <= 0 || n_qbins > 65536) return NFS_EINVAL;
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
                bool cross, int slab, int n_slabs)
{
    if (!out) return NFS_EINVAL;
    if (cross && path != NFS_PATH_FUSED_F32) return NFS_EINVAL;
    if (n_slabs != 1 && (path != NFS_PATH_FUSED_F32 || cross)) return NFS_EINVAL;
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
    c->slab = slab;
    c->n_slabs = n_slabs;
    if (n_slabs != 1 && !make_slab(&c->g, slab, n_slabs)) {
        delete c;
        return NFS_EINVAL;
    }
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
        cudaStreamCreateWithPriority(&c->copy_stream, cudaStreamNonBlocking, copy_stream_priority()) != cudaSuccess)
        return bail(NFS_ECUDA);
    // copy chunks of up to 256 MB; the device staging ring covers two delay blocks, at most 9 GB
    // (the copies of block b + 2 then run beside the delay launch of block b)
    c->copy_frames = (int)std::max<size_t>(1, std::min<size_t>(64, (256u << 20) / c->frame_bytes()));
    {
        const size_t cap = std::max<size_t>(2, (size_t(9) << 30) / (c->frame_bytes() * (size_t)c->copy_frames));
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
    if ((rc = alloc_dev(c, (void **)&c->d_slot_sums, sizeof(unsigned long long) * (size_t)c->copy_frames * c->n_slots)))
        return bail(rc);
    if ((rc = alloc_dev(c, (void **)&c->d_stage, c->frame_bytes() * (size_t)c->copy_frames * c->n_slots)))
        return bail(rc);
    const size_t ring_bytes = (size_t)c->R * c->g.M * c->csize();
    const size_t acc_bytes = (size_t)c->nd * c->g.M * c->asize();
    // sums of up to two copy chunks (a cross pass stages one of each sequence)
    if ((rc = alloc_dev(c, (void **)&c->d_sums, sizeof(unsigned long long) * 2 * kMaxChunk))) return bail(rc);
    if (c->f32() && (rc = alloc_dev(c, (void **)&c->d_ref, ref_buffer_bytes(c->g.HW)))) return bail(rc);
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

int copy_stream_priority()
{
    // the greatest priority (numerically least): the copy kernel's CTAs are placed before the
    // compute stream's pending CTAs as SMs free up
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

const void *host_device_view(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

cudaError_t copy_h2d(void *dst, const void *src, size_t bytes, cudaStream_t s, bool sm_reads, long long *launches)
{
    if (sm_reads && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15) == 0) {
        if (const void *dev = host_device_view(src)) {
            const cudaError_t e = launch_gather_h2d(dev, dst, bytes, s);
            if (e == cudaSuccess && launches) ++*launches;
            return e;
        }
    }
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

}  // namespace host
}  // namespace nfs

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

int nfs_create_slab(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int slab, int n_slabs,
                    nfs_ctx **out)
{
    if (!out) return NFS_EINVAL;
    *out = nullptr;
    if (n_slabs < 1 || slab < 0 || slab >= n_slabs) return NFS_EINVAL;
    return create_impl(H, W, delays, n_delays, n_qbins, NFS_PATH_FUSED_F32, 0, out, false, slab, n_slabs);
}

int nfs_slab_range(int H, int W, int slab, int n_slabs, int64_t *first_mode, int64_t *n_modes)
{
    if (!first_mode || !n_modes) return NFS_EINVAL;
    if (H < 2 || W < 2 || H > kMaxDim || W > kMaxDim || (H % 2) || (W % 2) || !factors_2_3(H) || !factors_2_3(W / 2))
        return NFS_EUNSUPPORTED;
    Geometry g = make_geometry(H, W, true);
    if (!make_slab(&g, slab, n_slabs)) return NFS_EINVAL;
    *first_mode = (int64_t)g.k0;
    *n_modes = (int64_t)g.M;
    return NFS_OK;
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
    NvtxRange range("nfs_push_frames");
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
    // FP32 contexts that launch their own delay updates hold slot releases back to the next launch
    const bool hold = c->f32() && !c->defer_delay;
    while (done < n) {
        const int nc = (int)std::min<long long>(c->copy_frames, n - done);
        const int slot = (int)(c->stage_i++ % c->n_slots);
        const size_t bytes = c->frame_bytes() * (size_t)nc;
        uint16_t *dst = c->d_stage + (size_t)slot * c->copy_frames * c->g.HW;
        const uint16_t *src = h + (size_t)done * c->g.HW;
        // the kernels that read this slot last time must be done before it is overwritten (a slot
        // whose release is still held back is released now: the wait must see its latest use)
        if (std::find(c->free_pending.begin(), c->free_pending.end(), slot) != c->free_pending.end())
            if ((rc = release_slots(c))) return rc;
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[slot], 0));
        int hs = -1;
        if (!locked) {
            hs = (int)(c->hstage_i++ & 1);
            CK(c, cudaEventSynchronize(c->ev_hcopied[hs]));
            memcpy(c->h_stage[hs], src, bytes);
            src = c->h_stage[hs];
        }
        // The SM copy of whole page-locked frames also takes their sums (into the slot's own sums, which
        // the transforms of this slot read before it is handed back); otherwise a sum pass follows.
        unsigned long long *ssum = c->d_slot_sums + (size_t)slot * c->copy_frames;
        const void *dev = nullptr;
        const bool fused = c->h2d == 0 && (c->frame_bytes() & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 &&
                           (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (dev = host_device_view(src)) != nullptr;
        rc = timed(c, NFS_STAGE_H2D, c->copy_stream, [&] {
            if (!fused) return copy_h2d(dst, src, bytes, c->copy_stream, c->h2d == 0, &c->launches);
            cudaError_t e = cudaMemsetAsync(ssum, 0, sizeof(unsigned long long) * (size_t)nc, c->copy_stream);
            if (e == cudaSuccess) e = launch_gather_h2d_sums(dev, dst, nc, c->frame_bytes(), ssum, c->copy_stream);
            if (e == cudaSuccess) ++c->launches;
            return e;
        }, "h2d");
        if (rc) return rc;
        if (hs >= 0) CK(c, cudaEventRecord(c->ev_hcopied[hs], c->copy_stream));
        CK(c, cudaEventRecord(c->ev_filled[slot], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_filled[slot], 0));
        unsigned long long *sums = fused ? ssum : c->d_sums;
        if ((rc = fused ? reference_once(c, dst, nc, sums) : frame_sums(c, dst, nc, sums))) return rc;
        for (int o = 0; o < nc;) {
            const int nf = next_chunk(c, nc - o, c->fft_chunk);
            rc = process_chunk(c, dst + (size_t)o * c->g.HW, nf, false, sums + o);
            if (rc) return rc;
            o += nf;
        }
        if (hold)
            c->free_pending.push_back(slot);
        else
            CK(c, cudaEventRecord(c->ev_free[slot], c->stream));
        done += nc;
        last = slot;
    }
    if ((rc = release_slots(c))) return rc;
    // copies run in order on the copy stream: when the last one is done the caller's buffer is free
    if (locked && last >= 0) CK(c, cudaEventSynchronize(c->ev_filled[last]));
    return c->err;
}

int nfs_push_frames_device(nfs_ctx *c, const uint16_t *d, int n)
{
    NvtxRange range("nfs_push_frames_device");
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
    NvtxRange range("nfs_structure_function");
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
    NvtxRange range("nfs_export_spectrum");
    int rc = enter(c);
    if (rc) return rc;
    if (!out || j < 0 || j >= c->nd) return NFS_EINVAL;
    // the FP32 path updates only the tiles the bins read unless every mode was asked for
    if (c->f32() && !c->modes_all) {
        c->errmsg = "nfs_export_spectrum: the 2-D spectrum needs NFS_OPT_MODES = 1 before the first frame";
        return NFS_ESTATE;  // not sticky: the context stays usable
    }
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
            if (v < 0 || v > 3) return NFS_EINVAL;
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
        case NFS_OPT_H2D:
            if (v < 0 || v > 1) return NFS_EINVAL;
            c->h2d = (int)v;
            return NFS_OK;
        case NFS_OPT_MODES:
            if (v < 0 || v > 1) return NFS_EINVAL;
            if (c->nframes > 0) return NFS_ESTATE;  // earlier blocks would lack the other modes
            c->modes_all = (int)v;
            return NFS_OK;
        case NFS_OPT_DELAY_SPAN:
            if (v == 0) {
                if (c->nframes > 0 || c->have_ref) return NFS_ESTATE;
                return autotune_delay_span(c);
            }
            if (v < kMinSpan || v > kMaxSpan) return NFS_EINVAL;
            return set_delay_span(c, (int)v);
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
        case NFS_OPT_SLAB_FIRST_MODE: *v = (int64_t)c->g.k0; return NFS_OK;
        case NFS_OPT_SLAB_MODES: *v = (int64_t)c->g.M; return NFS_OK;
        case NFS_OPT_DELAY_SPAN: *v = c->span; return NFS_OK;
        case NFS_OPT_H2D: *v = c->h2d; return NFS_OK;
        case NFS_OPT_MODES: *v = c->modes_all; return NFS_OK;
        case NFS_OPT_DELAY_MODES:
            *v = (c->f32() && !c->modes_all) ? c->n_tiles_binned * kTile : (int64_t)c->g.M;
            return NFS_OK;
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
    if (c->tl_base) c->pool.push_back(c->tl_base);
    c->tl_base = nullptr;
    c->timeline.clear();
    return NFS_OK;
}

int nfs_get_timeline(nfs_ctx *c, int32_t *stage, double *start_ms, double *end_ms, int64_t cap, int64_t *n)
{
    if (!c || !n || cap < 0 || (cap > 0 && (!stage || !start_ms || !end_ms))) return NFS_EINVAL;
    int rc = nfs_synchronize(c);
    if (rc) return rc;
    const int64_t m = (int64_t)c->timeline.size();
    for (int64_t i = 0; i < std::min(m, cap); ++i) {
        stage[i] = c->timeline[(size_t)i].stage;
        start_ms[i] = c->timeline[(size_t)i].start_ms;
        end_ms[i] = c->timeline[(size_t)i].end_ms;
    }
    *n = m;
    return NFS_OK;
}

int64_t nfs_launch_count(const nfs_ctx *c) { return c ? c->launches : -1; }

int nfs_fit(nfs_ctx *c, const double *D_in, float *A, float *B, float *Gamma, int iters, int method)
{
    NvtxRange range("nfs_fit");
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

}  // extern "C"
