// nfs_structure_function_noalloc: a one-shot analysis that allocates nothing.
//
// Some callers cannot allocate device memory while they run: a process whose device memory is
// already owned by another allocator (a framework's memory pool holding the whole GPU), or an
// acquisition loop that must not take the device-wide synchronisation cudaMalloc and cudaFree
// can imply.  This entry point runs the steps of the context path (exact frame sums, the r2c FFT
// with the generic kernels, the one-thread-per-mode FP32 delay update in blocks of 32 frames, the
// CSR binning kernel) with all of its scratch -- spectrum ring, accumulators, tables, sums -- carved
// out of one file-scope __device__ array of NFS_NOALLOC_SCRATCH_BYTES.  Twiddles and the bin table
// are built on the device (the bin lists by a stable counting placement in mode order, so the
// binned sums do not depend on timing), so no host heap is used either.  The paper has no
// counterpart to this entry point.
#include <algorithm>

#include "nfs_internal.cuh"

namespace nfs {

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NFS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNaBlock = 32;  // K of the fused delay update (same default as a context)
constexpr int kNaChunk = 4;   // frames per FFT launch pair
// The array's device address on the current device, looked up on every call with that device
// current: host code must not pass the symbol itself to a kernel (on the host it names a host-side
// stand-in, not device memory), and an address kept from an earlier call could be stale after the
// device's context was torn down and created again (the module, and the array with it, reloads).
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

template <typename C>
__global__ void k_na_twiddles(C *tw, int L, int n)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m].x = (float)c;
        tw[m].y = (float)(-s);
    }
}

__device__ unsigned long long na_isqrt(unsigned long long v)
{
    unsigned long long r = (unsigned long long)sqrt((double)v);
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// bin_of[mode(kx, ky)] = (bin << 1) | (weight == 2), or -1 for excluded modes (padding modes are
// set to -1 beforehand).
__global__ void k_na_bin_index(int *bin_of, Geometry g, int nq, long long L)
{
    const size_t n = (size_t)g.H * g.Wh;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(i / g.Wh), kx = (int)(i - (size_t)ky * g.Wh);
        int code = -1;
        if (!(kx == 0 && ky == 0)) {
            const long long kys = (ky <= g.H / 2) ? ky : ky - g.H;
            const long long m = (long long)kx * (L / g.W), n = kys * (L / g.H);
            const unsigned long long r2 = (unsigned long long)(m * m + n * n);
            const unsigned long long b =
                na_isqrt(4ull * (unsigned long long)nq * (unsigned long long)nq * r2) / (unsigned long long)L;
            if (b < (unsigned long long)nq) code = (int)(b << 1) | ((kx != 0 && kx != g.W / 2) ? 1 : 0);
        }
        bin_of[g.mode(kx, ky)] = code;
    }
}

// counts[b] = sum of the weights of bin b, nmodes[b] = its number of modes (integer adds: exact in
// any order).
__global__ void k_na_bin_counts(const int *bin_of, size_t M, long long *counts, int *nmodes)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const int c = bin_of[i];
        if (c >= 0) {
            atomicAdd((unsigned long long *)&counts[c >> 1], (c & 1) ? 2ull : 1ull);
            atomicAdd(&nmodes[c >> 1], 1);
        }
    }
}

// off[b] = modes of bins 0 .. b-1 (exclusive prefix sum, off[nq] = total); cursor[b] = off[b].
__global__ void k_na_bin_offsets(const int *nmodes, int nq, int *off, int *cursor)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < nq; ++b) {
        off[b] = acc;
        cursor[b] = acc;
        acc += nmodes[b];
    }
    off[nq] = acc;
}

// The bin lists in CSR form, entries (mode << 1) | (weight == 2), each bin's modes in increasing
// mode order (a stable counting placement): one warp walks the modes 32 at a time, the lanes of one
// bin take consecutive places by their rank among that bin's lanes, and the lowest of them then
// advances the bin's cursor.
__global__ void k_na_bin_place(const int *__restrict__ bin_of, size_t M, int *cursor, int *modes)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    for (size_t base = 0; base < M; base += 32) {
        const size_t i = base + lane;
        const int c = i < M ? bin_of[i] : -1;
        const int b = c >= 0 ? (c >> 1) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        if (b >= 0) modes[cursor[b] + __popc(same & lt)] = (int)((i << 1) | (size_t)(c & 1));
        __syncwarp();
        if (b >= 0 && (same & lt) == 0) cursor[b] += __popc(same);
        __syncwarp();
    }
}

size_t carve(size_t *off, size_t bytes)
{
    const size_t o = *off;
    *off = (o + bytes + 255) / 256 * 256;
    return o;
}

bool factors_2_3_na(int n)
{
    if (n <= 0) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

long long gcd_na(long long a, long long b)
{
    while (b) {
        const long long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

#define NA_CK(call)                               \
    do {                                          \
        if ((call) != cudaSuccess) return NFS_ECUDA; \
    } while (0)

}  // namespace
}  // namespace nfs

using namespace nfs;

extern "C" int nfs_structure_function_noalloc(const uint16_t *dev_frames, int n_frames, int H, int W,
                                              const int32_t *delays, int n_delays, int n_qbins, void *stream,
                                              double *D, int64_t *bin_counts, int64_t *pair_counts)
{
    if (n_frames < 0 || n_frames > (1 << 30) || (n_frames > 0 && !dev_frames) || (reinterpret_cast<uintptr_t>(dev_frames) & 1) || !delays ||
        n_delays <= 0 || n_delays > 65535 || n_qbins <= 0 || n_qbins > 65536 || !D || !bin_counts || !pair_counts)
        return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > 65536 || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    if (H < 2 || W < 2 || H > 4096 || W > 4096 || (H % 2) || (W % 2) || !factors_2_3_na(H) || !factors_2_3_na(W / 2))
        return NFS_EUNSUPPORTED;
    // The device bin index evaluates 4 nq^2 r2 (r2 up to lcm(H, W)^2 / 2) in 64-bit integers.
    const double Lq = (double)n_qbins * (double)((long long)H / gcd_na(H, W) * W);
    if (2.0 * Lq * Lq >= 1.8e19) return NFS_EUNSUPPORTED;

    const Geometry g = make_geometry(H, W, true);
    FftPlan prow, pcol;
    if (!make_plan(g.Lr, &prow) || !make_plan(H, &pcol)) return NFS_EUNSUPPORTED;
    const int nd = n_delays, nq = n_qbins;
    const int R = delays[nd - 1] + kNaBlock;

    // Frames must be this device's memory (another device's would be read through a peer pointer).
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return NFS_ECUDA;
    if (n_frames > 0) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, dev_frames) != cudaSuccess) {
            cudaGetLastError();
            return NFS_EINVAL;
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != cur)
            return NFS_EINVAL;
    }
    // The call synchronises its stream before it returns, which stream capture does not allow.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return NFS_ESTATE;
    }
    if (cap != cudaStreamCaptureStatusNone) return NFS_ESTATE;

    // Scratch layout, every piece 256-byte aligned.
    size_t off = 0;
    const size_t o_ring = carve(&off, (size_t)R * g.M * sizeof(float2));
    const size_t o_acc = carve(&off, (size_t)nd * g.M * sizeof(float2));
    const size_t o_sums = carve(&off, sizeof(unsigned long long) * kNaChunk);
    const size_t o_ref = carve(&off, sizeof(float) * g.HW);
    const size_t o_scr = carve(&off, sizeof(float2) * (size_t)kNaChunk * H * g.Wp);
    const size_t o_twr = carve(&off, sizeof(float2) * (size_t)(g.Lr > 0 ? g.Lr : 1));
    const size_t o_twc = carve(&off, sizeof(float2) * (size_t)H);
    const size_t o_twp = carve(&off, sizeof(float2) * (size_t)g.Wh);
    const size_t o_bin = carve(&off, sizeof(int) * g.M);
    const size_t o_cnt = carve(&off, sizeof(long long) * (size_t)nq);
    const size_t o_nmodes = carve(&off, sizeof(int) * (size_t)nq);
    const size_t o_boff = carve(&off, sizeof(int) * ((size_t)nq + 1));
    const size_t o_cursor = carve(&off, sizeof(int) * (size_t)nq);
    const size_t o_bmodes = carve(&off, sizeof(int) * g.M);
    const size_t o_pairs = carve(&off, sizeof(long long) * (size_t)nd);
    const size_t o_del = carve(&off, sizeof(int) * (size_t)nd);
    const size_t o_D = carve(&off, sizeof(double) * (size_t)nd * nq);
    if (off > (size_t)NFS_NOALLOC_SCRATCH_BYTES) return NFS_ETOOBIG;

    void *base_v = nullptr;
    if (scratch_address(&base_v) != cudaSuccess) return NFS_ECUDA;
    unsigned char *base = (unsigned char *)base_v;
    cudaStream_t s = (cudaStream_t)stream;
    float2 *ring = (float2 *)(base + o_ring);
    float2 *acc = (float2 *)(base + o_acc);
    unsigned long long *sums = (unsigned long long *)(base + o_sums);
    float *ref = (float *)(base + o_ref);
    float2 *scr = (float2 *)(base + o_scr);
    float2 *twr = (float2 *)(base + o_twr), *twc = (float2 *)(base + o_twc), *twp = (float2 *)(base + o_twp);
    int *bin_of = (int *)(base + o_bin);
    long long *cnt = (long long *)(base + o_cnt), *pairs = (long long *)(base + o_pairs);
    int *nmodes = (int *)(base + o_nmodes), *boff = (int *)(base + o_boff), *cursor = (int *)(base + o_cursor);
    int *bmodes = (int *)(base + o_bmodes);
    int *dd = (int *)(base + o_del);
    double *Dd = (double *)(base + o_D);

    // The array keeps the previous call's contents: zero what accumulates.
    NA_CK(cudaMemsetAsync(acc, 0, (size_t)nd * g.M * sizeof(float2), s));
    NA_CK(cudaMemsetAsync(cnt, 0, sizeof(long long) * (size_t)nq, s));
    NA_CK(cudaMemsetAsync(nmodes, 0, sizeof(int) * (size_t)nq, s));
    for (int j = 0; j < nd; ++j) pair_counts[j] = n_frames > delays[j] ? n_frames - delays[j] : 0;
    NA_CK(cudaMemcpyAsync(dd, delays, sizeof(int) * (size_t)nd, cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(pairs, pair_counts, sizeof(long long) * (size_t)nd, cudaMemcpyHostToDevice, s));
    k_na_twiddles<float2><<<8, 256, 0, s>>>(twr, g.Lr, g.Lr);
    k_na_twiddles<float2><<<8, 256, 0, s>>>(twc, H, H);
    k_na_twiddles<float2><<<8, 256, 0, s>>>(twp, W, g.Wh);
    const long long L = (long long)H / gcd_na(H, W) * W;
    NA_CK(cudaMemsetAsync(bin_of, 0xff, sizeof(int) * g.M, s));
    k_na_bin_index<<<256, 256, 0, s>>>(bin_of, g, nq, L);
    k_na_bin_counts<<<256, 256, 0, s>>>(bin_of, g.M, cnt, nmodes);
    k_na_bin_offsets<<<1, 1, 0, s>>>(nmodes, nq, boff, cursor);
    k_na_bin_place<<<1, 32, 0, s>>>(bin_of, g.M, cursor, bmodes);
    NA_CK(cudaGetLastError());

    long long done = 0, processed = 0;
    while (done < n_frames) {
        const long long room = kNaBlock - (done - processed);
        const int nf = (int)std::min<long long>(std::min<long long>(kNaChunk, room), n_frames - done);
        const uint16_t *src = dev_frames + (size_t)done * g.HW;
        NA_CK(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * (size_t)nf, s));
        NA_CK(launch_frame_sums(src, nf, g, sums, s));
        if (done == 0) NA_CK(launch_reference(src, sums, nf, g, ref, s));
        const int slot0 = (int)(done % R);
        NA_CK(launch_row_fft<float>(src, nf, sums, ref, g, prow, twr, twp, ring, R, slot0, s, scr, nullptr));
        NA_CK(launch_col_fft<float>(nf, g, pcol, twc, ring, R, slot0, s, scr, nullptr));
        done += nf;
        if (done - processed == kNaBlock || done == n_frames) {
            DelayArgs a{ring, R, g.M, processed, (int)(done - processed), dd, nd, acc, nullptr, nullptr, delays[nd - 1],
                        -1};
            NA_CK(launch_delay_f32(a, 1, s));  // the one-thread-per-mode kernel: blocks of 32 frames
            processed = done;
        }
    }
    NA_CK(launch_bin<float2>(acc, g.M, nd, nq, boff, bmodes, pairs, cnt, Dd, s));
    NA_CK(cudaMemcpyAsync(D, Dd, sizeof(double) * (size_t)nd * nq, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(bin_counts, cnt, sizeof(long long) * (size_t)nq, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    return NFS_OK;
}
