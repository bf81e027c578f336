// Per-bin fit of Eq. 1 with the intermediate scattering function f(q, tau) = exp(-Gamma(q) tau):
//
//   D_model(q, tau) = 2 A(q) [1 - exp(-Gamma(q) tau)] + 2 B(q)
//
// where A = a T I_s (static amplitude) and B = a B (noise background) of Eq. 1.  The loss of a
// bin is the unweighted least squares L = sum_j (D_model(tau_j) - D(tau_j))^2 over the delays.
// One thread per bin; D is [n_delays][n_bins] so a warp reads 32 consecutive bins per delay.
//
//   dL/dA = sum_j 2 r_j * 2 (1 - e_j)      dL/dB = sum_j 2 r_j * 2      dL/dGamma = sum_j 2 r_j * 2 A tau_j e_j
//
// with r_j = D_model(tau_j) - D(tau_j), e_j = exp(-Gamma tau_j).  The Gauss-Newton kernel solves
// (J^T J + lambda diag(J^T J)) delta = -J^T r per bin (Levenberg-Marquardt damping) for `iters`
// steps and clamps A, B >= 0 and Gamma > 0 after each step.
#include <cmath>

#include "nfs_internal.cuh"

namespace nfs {

__global__ void k_fit_loss_grad(const float *__restrict__ D, const float *__restrict__ tau, int nd, int nq,
                                const float *__restrict__ A, const float *__restrict__ B,
                                const float *__restrict__ G, float *__restrict__ loss, float *__restrict__ gA,
                                float *__restrict__ gB, float *__restrict__ gG)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nq) return;
    const float a = A[b], bb = B[b], g = G[b];
    float l = 0.f, da = 0.f, db = 0.f, dg = 0.f;
    for (int j = 0; j < nd; ++j) {
        const float t = __ldg(tau + j);
        const float e = expf(-g * t);
        const float r = 2.f * a * (1.f - e) + 2.f * bb - D[(size_t)j * nq + b];
        l = fmaf(r, r, l);
        da = fmaf(4.f * r, 1.f - e, da);
        db = fmaf(4.f, r, db);
        dg = fmaf(4.f * r * a * t, e, dg);
    }
    loss[b] = l;
    if (gA) gA[b] = da;
    if (gB) gB[b] = db;
    if (gG) gG[b] = dg;
}

// Solve the 3x3 symmetric system M x = v (Cramer's rule on the damped normal matrix); false if singular.
__device__ __forceinline__ bool solve3(const float M[3][3], const float v[3], float x[3])
{
    const float c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    const float c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    const float c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    const float det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    const float inv = 1.f / det;
    const float i00 = c00 * inv, i01 = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * inv,
                i02 = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * inv;
    const float i10 = c01 * inv, i11 = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * inv,
                i12 = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * inv;
    const float i20 = c02 * inv, i21 = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) * inv,
                i22 = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * inv;
    x[0] = i00 * v[0] + i01 * v[1] + i02 * v[2];
    x[1] = i10 * v[0] + i11 * v[1] + i12 * v[2];
    x[2] = i20 * v[0] + i21 * v[1] + i22 * v[2];
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

__device__ __forceinline__ float bin_loss(const float *D, const float *tau, int nd, int nq, int b, float a, float bb,
                                          float g)
{
    float l = 0.f;
    for (int j = 0; j < nd; ++j) {
        const float r = 2.f * a * (1.f - expf(-g * __ldg(tau + j))) + 2.f * bb - D[(size_t)j * nq + b];
        l = fmaf(r, r, l);
    }
    return l;
}

__global__ void k_fit_gauss_newton(const float *__restrict__ D, const float *__restrict__ tau, int nd, int nq,
                                   float *__restrict__ A, float *__restrict__ B, float *__restrict__ G, int iters,
                                   float lambda0)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nq) return;
    float a = A[b], bb = B[b], g = G[b];
    float lam = lambda0;
    float cur = bin_loss(D, tau, nd, nq, b, a, bb, g);
    // The normal equations are formed in scaled units: residuals divided by the bin's largest |D|
    // and each parameter's column multiplied by that parameter's current magnitude (Jacobi
    // scaling), so that A ~ 1e8 next to B ~ 1e2 and Gamma ~ 1e-2 still gives an FP32-solvable
    // 3x3 system; the step is scaled back afterwards.
    float dmax = 0.f;
    for (int j = 0; j < nd; ++j) dmax = fmaxf(dmax, fabsf(D[(size_t)j * nq + b]));
    const float rs = dmax > 0.f ? 1.f / dmax : 1.f;
    for (int it = 0; it < iters; ++it) {
        const float c[3] = {fmaxf(fabsf(a), 1e-6f * dmax + 1e-30f), fmaxf(fabsf(bb), 1e-6f * dmax + 1e-30f),
                            fmaxf(fabsf(g), 1e-12f)};
        float M[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        float v[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < nd; ++j) {
            const float t = __ldg(tau + j);
            const float e = expf(-g * t);
            const float r = (2.f * a * (1.f - e) + 2.f * bb - D[(size_t)j * nq + b]) * rs;
            const float J[3] = {2.f * (1.f - e) * c[0] * rs, 2.f * c[1] * rs, 2.f * a * t * e * c[2] * rs};
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                v[p] = fmaf(J[p], r, v[p]);
#pragma unroll
                for (int q = 0; q < 3; ++q) M[p][q] = fmaf(J[p], J[q], M[p][q]);
            }
        }
        // Levenberg-Marquardt: accept a step that lowers the loss, otherwise raise the damping
        bool stepped = false;
        for (int tries = 0; tries < 8 && !stepped; ++tries) {
            float Md[3][3];
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) Md[p][q] = M[p][q] + (p == q ? lam * M[p][p] : 0.f);
            const float rhs[3] = {-v[0], -v[1], -v[2]};
            float x[3];
            if (solve3(Md, rhs, x)) {
                const float na = fmaxf(a + x[0] * c[0], 0.f), nb = fmaxf(bb + x[1] * c[1], 0.f);
                const float ng = fmaxf(g + x[2] * c[2], 1e-12f);
                const float nl = bin_loss(D, tau, nd, nq, b, na, nb, ng);
                if (nl <= cur) {
                    a = na;
                    bb = nb;
                    g = ng;
                    cur = nl;
                    lam = fmaxf(lam * 0.3f, 1e-7f);
                    stepped = true;
                    break;
                }
            }
            lam *= 10.f;
        }
        if (!stepped) break;
    }
    A[b] = a;
    B[b] = bb;
    G[b] = g;
}

// Adam on u with theta = theta0 (1 + u) per parameter (a scale-free step for parameters whose
// magnitudes differ by orders), gradients from the same loss; positivity clamps as above.
__global__ void k_fit_adam(const float *__restrict__ D, const float *__restrict__ tau, int nd, int nq,
                           float *__restrict__ A, float *__restrict__ B, float *__restrict__ G, int iters, float lr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nq) return;
    const float s0[3] = {fmaxf(fabsf(A[b]), 1e-30f), fmaxf(fabsf(B[b]), 1e-30f), fmaxf(fabsf(G[b]), 1e-30f)};
    const float t0[3] = {A[b], B[b], G[b]};
    float u[3] = {0.f, 0.f, 0.f}, m1[3] = {0.f, 0.f, 0.f}, m2[3] = {0.f, 0.f, 0.f};
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-12f;
    float p1 = 1.f, p2 = 1.f;
    for (int it = 0; it < iters; ++it) {
        const float a = fmaxf(t0[0] * (1.f + u[0]), 0.f), bb = fmaxf(t0[1] * (1.f + u[1]), 0.f),
                    g = fmaxf(t0[2] * (1.f + u[2]), 1e-12f);
        float gr[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < nd; ++j) {
            const float t = __ldg(tau + j);
            const float e = expf(-g * t);
            const float r = 2.f * a * (1.f - e) + 2.f * bb - D[(size_t)j * nq + b];
            gr[0] = fmaf(4.f * r, 1.f - e, gr[0]);
            gr[1] = fmaf(4.f, r, gr[1]);
            gr[2] = fmaf(4.f * r * a * t, e, gr[2]);
        }
        p1 *= b1;
        p2 *= b2;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float gu = gr[p] * s0[p];
            m1[p] = b1 * m1[p] + (1.f - b1) * gu;
            m2[p] = b2 * m2[p] + (1.f - b2) * gu * gu;
            const float mh = m1[p] / (1.f - p1), vh = m2[p] / (1.f - p2);
            u[p] -= lr * mh / (sqrtf(vh) + eps);
        }
    }
    A[b] = fmaxf(t0[0] * (1.f + u[0]), 0.f);
    B[b] = fmaxf(t0[1] * (1.f + u[1]), 0.f);
    G[b] = fmaxf(t0[2] * (1.f + u[2]), 1e-12f);
}

cudaError_t launch_fit_adam(const float *D, const float *tau, int nd, int nq, float *A, float *B, float *G, int iters,
                            float lr, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    k_fit_adam<<<(nq + 127) / 128, 128, 0, s>>>(D, tau, nd, nq, A, B, G, iters, lr);
    return cudaGetLastError();
}

cudaError_t launch_fit_loss_grad(const float *D, const float *tau, int nd, int nq, const float *A, const float *B,
                                 const float *G, float *loss, float *gA, float *gB, float *gG, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    k_fit_loss_grad<<<(nq + 127) / 128, 128, 0, s>>>(D, tau, nd, nq, A, B, G, loss, gA, gB, gG);
    return cudaGetLastError();
}

cudaError_t launch_fit_gauss_newton(const float *D, const float *tau, int nd, int nq, float *A, float *B, float *G,
                                    int iters, float lambda, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    k_fit_gauss_newton<<<(nq + 127) / 128, 128, 0, s>>>(D, tau, nd, nq, A, B, G, iters, lambda);
    return cudaGetLastError();
}

}  // namespace nfs

using namespace nfs;

extern "C" int nfs_fit_loss_grad(const float *D, const float *tau, int n_delays, int n_bins, const float *A,
                                 const float *B, const float *Gamma, float *loss, float *gA, float *gB, float *gGamma,
                                 void *stream)
{
    if (!D || !tau || !A || !B || !Gamma || !loss || n_delays < 0 || n_bins < 0) return NFS_EINVAL;
    return launch_fit_loss_grad(D, tau, n_delays, n_bins, A, B, Gamma, loss, gA, gB, gGamma, (cudaStream_t)stream) ==
                   cudaSuccess
               ? NFS_OK
               : NFS_ECUDA;
}

extern "C" int nfs_fit_gauss_newton(const float *D, const float *tau, int n_delays, int n_bins, float *A, float *B,
                                    float *Gamma, int iters, float lambda, void *stream)
{
    if (!D || !tau || !A || !B || !Gamma || n_delays < 0 || n_bins < 0 || iters < 0 || !(lambda >= 0.f))
        return NFS_EINVAL;
    return launch_fit_gauss_newton(D, tau, n_delays, n_bins, A, B, Gamma, iters, lambda, (cudaStream_t)stream) ==
                   cudaSuccess
               ? NFS_OK
               : NFS_ECUDA;
}
