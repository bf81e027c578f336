// Ingest kernels: the copy of pushed frames from page-locked host memory, the exact spatial sum of
// every frame (for the mean normalisation of the differential analysis: images are divided by their
// spatial average) and the FP32 reference image subtracted before the FP32 transform.
#include <algorithm>

#include "nfs_internal.cuh"
#include "roi.cuh"

namespace nfs {

// Host-to-device frame copy read by the SMs: page-locked host memory is addressed directly (unified
// addressing) and copied 16 bytes per thread per step into device memory.  Used instead of the
// copy engines for host pushes: on GB300 machines the copy engines read some page-locked buffers at
// 8-38 GB/s for their first gigabytes while loads from the SMs read the same pages at full speed
// (and a few dozen CTAs of this kernel reach the ~210 GB/s the copy engines reach at best).  It
// uses no shared memory and CTAs of 128 threads (4096 registers), so one fits beside a CTA of the
// delay kernel on every SM.
__global__ void __launch_bounds__(kGatherThreads) k_gather_h2d(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four independent 16-byte loads in flight per thread
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}

cudaError_t launch_gather_h2d(const void *host_src, void *dst, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    if (((reinterpret_cast<uintptr_t>(host_src) | reinterpret_cast<uintptr_t>(dst) | bytes) & 15) != 0)
        return cudaErrorInvalidValue;  // the caller falls back to the copy engines
    // the largest shared-memory carve-out, as the delay kernel's: an SM takes CTAs of a kernel
    // that prefers another carve-out only once it has drained
    // (set on every call: the attribute belongs to the current device)
    const cudaError_t carve =
        cudaFuncSetAttribute(k_gather_h2d, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (carve != cudaSuccess) return carve;
    const size_t n16 = bytes / 16;
    const size_t want = (n16 + 4 * kGatherThreads - 1) / (4 * kGatherThreads);
    const unsigned grid = (unsigned)std::min<size_t>(kGatherCtas, std::max<size_t>(want, 1));
    k_gather_h2d<<<grid, kGatherThreads, 0, s>>>(reinterpret_cast<const uint4 *>(host_src), reinterpret_cast<uint4 *>(dst), n16);
    return cudaGetLastError();
}

// Host-to-device copy of nf whole frames (f16 16-byte pieces each) read by the SMs, adding each
// frame's exact pixel sum into sums[f] on the way (the frames pass through the SMs anyway, so the
// separate sum pass over device memory is saved): cpf CTAs per frame, one 64-bit atomic per CTA.
__device__ __forceinline__ unsigned sum_u16x8(uint4 v)
{
    return (v.x & 0xffffu) + (v.x >> 16) + (v.y & 0xffffu) + (v.y >> 16) + (v.z & 0xffffu) + (v.z >> 16) +
           (v.w & 0xffffu) + (v.w >> 16);
}

__global__ void __launch_bounds__(kGatherThreads) k_gather_h2d_sums(const uint4 *__restrict__ src,
                                                                    uint4 *__restrict__ dst, size_t f16, int cpf,
                                                                    unsigned long long *__restrict__ sums)
{
    const int f = blockIdx.x / cpf, part = blockIdx.x % cpf;
    const uint4 *s = src + (size_t)f * f16;
    uint4 *d = dst + (size_t)f * f16;
    const size_t stride = (size_t)cpf * blockDim.x;
    size_t i = (size_t)part * blockDim.x + threadIdx.x;
    unsigned long long acc = 0;
    for (; i + 3 * stride < f16; i += 4 * stride) {
        const uint4 a = s[i], b = s[i + stride], c = s[i + 2 * stride], e = s[i + 3 * stride];
        d[i] = a;
        d[i + stride] = b;
        d[i + 2 * stride] = c;
        d[i + 3 * stride] = e;
        acc += (unsigned long long)(sum_u16x8(a) + sum_u16x8(b)) + (sum_u16x8(c) + sum_u16x8(e));
    }
    for (; i < f16; i += stride) {
        const uint4 a = s[i];
        d[i] = a;
        acc += sum_u16x8(a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ unsigned long long ws[kGatherThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
#pragma unroll
        for (int w = 0; w < kGatherThreads / 32; ++w) t += ws[w];
        atomicAdd(&sums[f], t);
    }
}

cudaError_t launch_gather_h2d_sums(const void *host_src, void *dst, int nf, size_t frame_bytes,
                                   unsigned long long *sums, cudaStream_t s)
{
    if (nf <= 0) return cudaSuccess;
    if (((reinterpret_cast<uintptr_t>(host_src) | reinterpret_cast<uintptr_t>(dst) | frame_bytes) & 15) != 0)
        return cudaErrorInvalidValue;
    const cudaError_t carve =
        cudaFuncSetAttribute(k_gather_h2d_sums, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (carve != cudaSuccess) return carve;
    const int cpf = std::max(1, kGatherCtas / nf);
    k_gather_h2d_sums<<<(unsigned)(nf * cpf), kGatherThreads, 0, s>>>(reinterpret_cast<const uint4 *>(host_src),
                                                                       reinterpret_cast<uint4 *>(dst), frame_bytes / 16,
                                                                       cpf, sums);
    return cudaGetLastError();
}

// sums[blockIdx.y] += sum of the frame's pixels.  Integer arithmetic, so the result is exact and
// independent of the order of the atomic adds.  VEC: 16-byte loads (frame start 16-byte aligned).
template <bool VEC>
__global__ void __launch_bounds__(256) k_frame_sums(const uint16_t *__restrict__ frames, size_t HW,
                                                    unsigned long long *__restrict__ sums)
{
    const uint16_t *f = frames + (size_t)blockIdx.y * HW;
    unsigned long long acc = 0;
    size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t nthr = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    if (VEC) {
        const uint4 *v = reinterpret_cast<const uint4 *>(f);
        const size_t n8 = HW / 8;
        auto sum8 = [](uint4 q) -> unsigned {
            return (q.x & 0xffffu) + (q.x >> 16) + (q.y & 0xffffu) + (q.y >> 16) + (q.z & 0xffffu) + (q.z >> 16) +
                   (q.w & 0xffffu) + (q.w >> 16);
        };
        size_t i = tid;
        // four independent 16-byte loads in flight per thread
        for (; i + 3 * nthr < n8; i += 4 * nthr) {
            const uint4 q0 = __ldg(v + i), q1 = __ldg(v + i + nthr), q2 = __ldg(v + i + 2 * nthr),
                        q3 = __ldg(v + i + 3 * nthr);
            acc += (unsigned long long)(sum8(q0) + sum8(q1)) + (unsigned long long)(sum8(q2) + sum8(q3));
        }
        for (; i < n8; i += nthr) acc += sum8(__ldg(v + i));
        done = n8 * 8;
    }
    for (size_t i = done + tid; i < HW; i += nthr) acc += f[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&sums[blockIdx.y], acc);
}

cudaError_t launch_frame_sums(const uint16_t *frames, int nf, const Geometry &g, unsigned long long *sums,
                              cudaStream_t s)
{
    if (nf <= 0) return cudaSuccess;
    bool vec = ((reinterpret_cast<uintptr_t>(frames) & 15) == 0) && ((g.HW * 2) % 16 == 0);
    size_t work = vec ? g.HW / 8 : g.HW;
    int bx = (int)((work + 255) / 256);
    int cap = (nf >= 8) ? 64 : 512 / nf;
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    dim3 grid(bx, nf);
    if (vec)
        k_frame_sums<true><<<grid, 256, 0, s>>>(frames, g.HW, sums);
    else
        k_frame_sums<false><<<grid, 256, 0, s>>>(frames, g.HW, sums);
    return cudaGetLastError();
}

// ref[x] = fl32(fl32(i_f(x)) * hi) for the first frame f < nf whose sum is not 0 (a dark frame
// normalises to the zero image, which would leave the static beam in every transform), with
// hi + lo = HW / sum(i_f) as a float pair; the zero image when all nf frames are dark.  Any fixed
// image would do (it cancels in every difference); this one removes the static beam before the
// FP32 transform.  raw (optional) receives i_f itself and inv (optional) {hi, lo}: a row pass that
// reads the 2-byte counts and forms the same product gets the same image bit for bit.
__global__ void k_reference(const uint16_t *__restrict__ frames, const unsigned long long *__restrict__ sums, int nf,
                            size_t HW, float *__restrict__ ref, uint16_t *__restrict__ raw, float2 *__restrict__ inv)
{
    int f = 0;
    while (f < nf && sums[f] == 0) ++f;
    const unsigned long long S = f < nf ? sums[f] : 0;
    const double invd = S ? (double)HW / (double)S : 0.0;
    const float hi = (float)invd, lo = (float)(invd - (double)hi);
    const uint16_t *frame = frames + (size_t)(f < nf ? f : 0) * HW;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const uint16_t n = f < nf ? frame[i] : (uint16_t)0;
        ref[i] = __fmul_rn((float)n, hi);
        if (raw) raw[i] = n;
    }
    if (inv && blockIdx.x == 0 && threadIdx.x == 0) *inv = make_float2(hi, lo);
}

cudaError_t launch_reference(const uint16_t *frames, const unsigned long long *sums, int nf, const Geometry &g,
                             float *ref, cudaStream_t s, uint16_t *raw, float2 *inv)
{
    if (nf <= 0) return cudaErrorInvalidValue;
    int bx = (int)((g.HW + 255) / 256);
    if (bx > 1216) bx = 1216;
    k_reference<<<bx, 256, 0, s>>>(frames, sums, nf, g.HW, ref, raw, inv);
    return cudaGetLastError();
}

// Regions of interest: window r of frame f goes to dst + roi[r].dst + f*h*w, row-major (a plain
// crop; every window is then analysed as a sequence of its own).  One grid row per window, 4-byte
// copies: W, x0 and w are even and src is 4-byte aligned, so every source and destination word is
// whole.  32-bit indices: n*h*(w/2) < 2^31 is checked by the host.
__global__ void __launch_bounds__(256) k_roi_crop(const uint16_t *__restrict__ src, int H, int W, int n,
                                                  const RoiRect *__restrict__ roi, uint16_t *__restrict__ dst)
{
    const RoiRect r = roi[blockIdx.y];
    const unsigned ww = (unsigned)r.w >> 1;  // words per window row
    const unsigned rows = (unsigned)n * (unsigned)r.h;
    const unsigned words = rows * ww;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst + r.dst);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) {
        const unsigned row = i / ww, xw = i - row * ww;
        const unsigned f = row / (unsigned)r.h, y = row - f * (unsigned)r.h;
        const size_t at = ((size_t)f * H + r.y0 + y) * (size_t)W + r.x0;  // even
        d32[i] = __ldg(s32 + at / 2 + xw);
    }
}

cudaError_t launch_roi_crop(const uint16_t *src, int H, int W, int n, const RoiRect *d_roi, int n_roi,
                            long long max_words, int n_sm, uint16_t *dst, cudaStream_t s)
{
    if (n <= 0 || n_roi <= 0) return cudaSuccess;
    long long bx = (max_words + 255) / 256;
    const long long cap = std::max(1LL, (long long)n_sm * 8 / n_roi);
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    k_roi_crop<<<dim3((unsigned)bx, (unsigned)n_roi), 256, 0, s>>>(src, H, W, n, d_roi, dst);
    return cudaGetLastError();
}

}  // namespace nfs
