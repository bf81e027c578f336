// Azimuthal (radial) average of the accumulated difference spectra into q bins (Fig. 1e,f):
//
//   D_b(tau_j) = sum_{k in b} w_k acc_j(k) / ((N - tau_j) C_b)
//
// in FP64.  The modes of each bin come from a host-built list sorted by bin; one CTA reduces one
// (bin, delay) entry in a fixed order (strided per-thread sums, then a fixed shuffle and shared
// memory tree), so the result does not change from run to run.
#include "nfs_internal.cuh"

namespace nfs {

__device__ __forceinline__ double acc_value(const float2 *a, size_t i)
{
    const float2 v = a[i];
    return (double)v.x - (double)v.y;  // Kahan pair: sum - compensation
}
__device__ __forceinline__ double acc_value(const double *a, size_t i) { return a[i]; }

template <typename Acc>
__global__ void __launch_bounds__(128) k_bin(const Acc *__restrict__ acc, size_t M, int nq,
                                             const int *__restrict__ off, const int *__restrict__ modes,
                                             const long long *__restrict__ pairs,
                                             const long long *__restrict__ counts, double *__restrict__ D)
{
    const int b = blockIdx.x;
    const int j = blockIdx.y;
    const Acc *aj = acc + (size_t)j * M;
    double s = 0.0;
    const int lo = off[b], hi = off[b + 1];
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int code = __ldg(modes + i);
        const double v = acc_value(aj, (size_t)(code >> 1));
        s += (code & 1) ? 2.0 * v : v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double part[4];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double tot = (part[0] + part[1]) + (part[2] + part[3]);
        const long long np = pairs[j], c = counts[b];
        D[(size_t)j * nq + b] = (np > 0 && c > 0) ? tot / ((double)np * (double)c) : 0.0;
    }
}

template <typename Acc>
cudaError_t launch_bin(const Acc *acc, size_t M, int nd, int nq, const int *bin_off, const int *bin_modes,
                       const long long *pairs, const long long *counts, double *D, cudaStream_t s)
{
    if (nd <= 0 || nq <= 0) return cudaSuccess;
    dim3 grid(nq, nd);
    k_bin<Acc><<<grid, 128, 0, s>>>(acc, M, nq, bin_off, bin_modes, pairs, counts, D);
    return cudaGetLastError();
}

template <typename Acc>
__global__ void k_export(const Acc *__restrict__ acc_j, Geometry g, long long pairs, double *__restrict__ out)
{
    const size_t n = (size_t)g.H * g.Wh;
    const double inv = pairs > 0 ? 1.0 / (double)pairs : 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t ky = i / g.Wh, kx = i - ky * g.Wh;
        const size_t kl = g.mode((int)kx, (int)ky) - g.k0;  // modes outside a slab read as 0
        out[i] = kl < g.M ? acc_value(acc_j, kl) * inv : 0.0;
    }
}

template <typename Acc>
cudaError_t launch_export(const Acc *acc_j, const Geometry &g, long long pairs, double *out, cudaStream_t s)
{
    const size_t n = (size_t)g.H * g.Wh;
    int bx = (int)((n + 255) / 256);
    if (bx > 4096) bx = 4096;
    k_export<Acc><<<bx, 256, 0, s>>>(acc_j, g, pairs, out);
    return cudaGetLastError();
}

template cudaError_t launch_bin<float2>(const float2 *, size_t, int, int, const int *, const int *,
                                        const long long *, const long long *, double *, cudaStream_t);
template cudaError_t launch_bin<double>(const double *, size_t, int, int, const int *, const int *,
                                        const long long *, const long long *, double *, cudaStream_t);
template cudaError_t launch_export<float2>(const float2 *, const Geometry &, long long, double *, cudaStream_t);
template cudaError_t launch_export<double>(const double *, const Geometry &, long long, double *, cudaStream_t);

}  // namespace nfs
