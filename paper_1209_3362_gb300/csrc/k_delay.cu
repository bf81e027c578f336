// Delay update of the difference power spectra, the left-hand side of Eq. 1:
//
//   acc[j][k] += sum over new frames t with t >= tau_j of |P_t(k) - P_{t - tau_j}(k)|^2
//
// where P_t is the spectrum of frame t held in ring slot t mod R.  By linearity P_t - P_s is the
// transform of the real-space difference n_t - n_s, so each pair costs one complex subtraction
// and a squared modulus per mode instead of a transform ("only the square moduli of FFT
// differences" of the processing paragraph).  Averaging over t at fixed tau is the time average
// that stands for the ensemble average of Eq. 1 for stationary dynamics.
#include "nfs_internal.cuh"

namespace nfs {

// Kahan step: (s, c) += p, value = s - c.
__device__ __forceinline__ float2 kahan_add(float2 a, float p)
{
    const float y = p - a.y;
    const float t = a.x + y;
    a.y = (t - a.x) - y;
    a.x = t;
    return a;
}

// Fused FP32 update for a block of nb <= KB new frames t0 .. t0+nb-1.  One thread per mode k: the
// block's spectra stay in registers, each delay adds a plain FP32 block partial into a Kahan pair.
template <int KB>
__global__ void __launch_bounds__(256) k_delay_f32_block(const float2 *__restrict__ ring, int R, size_t M,
                                                         int base_slot, long long t0, int nb,
                                                         const int *__restrict__ delays, int nd,
                                                         float2 *__restrict__ acc)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    float2 x[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) {
        if (i < nb) {
            int sl = base_slot + i;
            if (sl >= R) sl -= R;
            x[i] = ring[(size_t)sl * M + k];
        }
    }
    const long long tlast = t0 + nb - 1;
    for (int j = 0; j < nd; ++j) {
        const int tau = __ldg(delays + j);
        if ((long long)tau > tlast) break;
        float p = 0.0f;
#pragma unroll
        for (int i = 0; i < KB; ++i) {
            if (i < nb && t0 + i >= tau) {
                int sl = base_slot + i - tau;
                if (sl < 0) sl += R;
                if (sl >= R) sl -= R;
                const float2 y = ring[(size_t)sl * M + k];
                const float dr = x[i].x - y.x, di = x[i].y - y.y;
                p = fmaf(dr, dr, p);
                p = fmaf(di, di, p);
            }
        }
        float2 *a = acc + (size_t)j * M + k;
        *a = kahan_add(*a, p);
    }
}

constexpr int kBlockMax = 32;

cudaError_t launch_delay_f32(const DelayArgs &a, int variant, cudaStream_t s)
{
    (void)variant;
    if (a.nb <= 0) return cudaSuccess;
    if (a.nb > kBlockMax) return cudaErrorInvalidValue;
    const int base = (int)(a.t0 % a.R);
    const unsigned grid = (unsigned)((a.M + 255) / 256);
    k_delay_f32_block<kBlockMax><<<grid, 256, 0, s>>>(a.ring, a.R, a.M, base, a.t0, a.nb, a.delays, a.nd, a.acc);
    return cudaGetLastError();
}

// Plain FP64 path: one frame t per launch, FP64 accumulators, no blocking.
__global__ void __launch_bounds__(256) k_delay_f64(const double2 *__restrict__ ring, int R, size_t M, int tslot,
                                                   long long t, const int *__restrict__ delays, int nd,
                                                   double *__restrict__ acc)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const double2 x = ring[(size_t)tslot * M + k];
    for (int j = 0; j < nd; ++j) {
        const int tau = __ldg(delays + j);
        if ((long long)tau > t) break;
        int sl = tslot - tau;
        if (sl < 0) sl += R;
        const double2 y = ring[(size_t)sl * M + k];
        const double dr = x.x - y.x, di = x.y - y.y;
        acc[(size_t)j * M + k] += dr * dr + di * di;
    }
}

cudaError_t launch_delay_f64(const double2 *ring, int R, size_t M, long long t, const int *delays, int nd,
                             double *acc, cudaStream_t s)
{
    const int tslot = (int)(t % R);
    const unsigned grid = (unsigned)((M + 255) / 256);
    k_delay_f64<<<grid, 256, 0, s>>>(ring, R, M, tslot, t, delays, nd, acc);
    return cudaGetLastError();
}

}  // namespace nfs
