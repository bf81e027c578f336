// 2-D real-to-complex FFT of normalised frames into the spectrum ring.
//
// By the linearity of the Fourier transform (processing paragraph of the paper) every frame is
// transformed once; pairs are differenced in Fourier space afterwards.  The transform is the
// unscaled forward DFT exp(-2 pi i (k_x x / W + k_y y / H)), done in two shared-memory passes:
//
//   row pass     each real row of W samples is read as W/2 complex points z[m] = p[2m] + i p[2m+1],
//                transformed with a mixed-radix (4, 2, 3) Stockham FFT of length W/2, and split
//                into the W/2+1 non-redundant outputs X[k] = E[k] + exp(-2 pi i k / W) O[k] with
//                E = (Z[k] + conj Z[W/2-k]) / 2 and O = (Z[k] - conj Z[W/2-k]) / 2i.  The input
//                pixels are normalised on load: p = i / <i> (FP64 path), or
//                p = i / <i> - r with the FP32 reference image r, 1/<i> carried as a float pair and
//                the subtraction fused so that only p itself is rounded (FP32 path).
//   column pass  each group of CB adjacent columns of the slot is transformed along y in place.
//
// FP32: the row pass writes a column-pair scratch, the column pass writes the tile-major ring (see
// ring_index) in column-major mode order.  FP64: both passes work in place in the slot-major ring
// [R][M] in row-major mode order.
//
// Stockham stage of radix R on a length-L transform whose sub-transforms have length Ns so far:
// butterfly j < L/R reads x[j + r L/R] (r < R), twists input r by exp(-2 pi i (j mod Ns) r / (Ns R)),
// applies an R-point DFT and writes output r to (j / Ns) Ns R + (j mod Ns) + r Ns.
#include "nfs_internal.cuh"

namespace nfs {

template <typename C>
__device__ __forceinline__ C cadd(C a, C b)
{
    return {a.x + b.x, a.y + b.y};
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b)
{
    return {a.x - b.x, a.y - b.y};
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// -i * a
template <typename C>
__device__ __forceinline__ C cmi(C a)
{
    return {a.y, -a.x};
}

template <typename C, int R>
struct Dft;
template <typename C>
struct Dft<C, 2> {
    __device__ __forceinline__ static void run(C *v)
    {
        C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};
template <typename C>
struct Dft<C, 4> {
    __device__ __forceinline__ static void run(C *v)
    {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = cmi(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};
template <typename C>
struct Dft<C, 3> {
    __device__ __forceinline__ static void run(C *v)
    {
        using T = decltype(v[0].x);
        const T h = (T)0.5;
        const T s = (T)0.86602540378443864676;  // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = csub(v[1], v[2]);
        C m = {v[0].x - h * t1.x, v[0].y - h * t1.y};
        C r = {s * t2.y, -s * t2.x};  // -i s t2
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

// Elements of transform b at position i live at buf[b * bs + i * is].  BFAST: consecutive threads
// take consecutive transforms (column pass); otherwise consecutive butterflies of one transform.
template <typename C, int R, bool BFAST>
__device__ __forceinline__ void fft_stage(const C *__restrict__ in, C *__restrict__ out, int L, int Ns, int nb,
                                          int is, int bs, const C *__restrict__ tw)
{
    const int nbf = L / R;
    const int total = nb * nbf;
    const int tws = L / (Ns * R);
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        int b, j;
        if (BFAST) {
            b = g % nb;
            j = g / nb;
        } else {
            b = g / nbf;
            j = g - b * nbf;
        }
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[b * bs + (j + r * nbf) * is];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + k * r * tws));
        Dft<C, R>::run(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[b * bs + (base + r * Ns) * is] = v[r];
    }
}

// Runs all stages; returns the buffer holding the result (a or b).
template <typename C, bool BFAST>
__device__ C *fft_all(C *a, C *b, const FftPlan &plan, int nb, int is, int bs, const C *tw)
{
    int Ns = 1;
    for (int st = 0; st < plan.nstages; ++st) {
        const int R = plan.radix[st];
        if (R == 4)
            fft_stage<C, 4, BFAST>(a, b, plan.L, Ns, nb, is, bs, tw);
        else if (R == 2)
            fft_stage<C, 2, BFAST>(a, b, plan.L, Ns, nb, is, bs, tw);
        else
            fft_stage<C, 3, BFAST>(a, b, plan.L, Ns, nb, is, bs, tw);
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_fft(const uint16_t *__restrict__ frames,
                                                 const unsigned long long *__restrict__ sums,
                                                 const float *__restrict__ ref, Geometry g, FftPlan plan,
                                                 const typename cplx_t<T>::type *__restrict__ tw,
                                                 const typename cplx_t<T>::type *__restrict__ twp,
                                                 typename cplx_t<T>::type *__restrict__ ring, int R, int slot0,
                                                 int rpc, typename cplx_t<T>::type *__restrict__ scratch)
{
    using C = typename cplx_t<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = g.Lr;
    C *bufA = reinterpret_cast<C *>(smem_raw);
    C *bufB = bufA + (size_t)rpc * L;
    const int f = blockIdx.y;
    const int row0 = blockIdx.x * rpc;
    const unsigned long long S = sums[f];
    const double invd = S ? (double)g.HW / (double)S : 0.0;
    // 1/<i> as an unevaluated float pair hi + lo: rounding 1/<i> to one float would scale the frame
    // by (1 + d), d ~ 1e-8, and leak d times the beam's large low-q spectrum into the differences.
    const float inv_hi = (float)invd;
    const float inv_lo = (float)(invd - (double)inv_hi);
    const uint16_t *fr = frames + (size_t)f * g.HW;

    for (int e = threadIdx.x; e < rpc * L; e += blockDim.x) {
        const int r = e / L, m = e - r * L;
        const int y = row0 + r;
        C z = {(T)0, (T)0};
        if (y < g.H) {
            const size_t o = (size_t)y * g.W + 2 * m;
            const uint16_t a = fr[o], b = fr[o + 1];
            if (sizeof(T) == 4) {
                // p = i (hi + lo) - r with the subtraction inside the first fused multiply-add, so
                // only the small result p is rounded
                const float fa = (float)a, fb = (float)b;
                z.x = (T)__fmaf_rn(fa, inv_lo, __fmaf_rn(fa, inv_hi, -__ldg(ref + o)));
                z.y = (T)__fmaf_rn(fb, inv_lo, __fmaf_rn(fb, inv_hi, -__ldg(ref + o + 1)));
            } else {
                z.x = (T)((double)a * invd);
                z.y = (T)((double)b * invd);
            }
        }
        bufA[e] = z;
    }
    __syncthreads();
    C *Z = fft_all<C, false>(bufA, bufB, plan, rpc, 1, L, tw);

    const int slot = (slot0 + f) % R;
    const T half = (T)0.5;
    for (int e = threadIdx.x; e < rpc * g.Wp; e += blockDim.x) {
        const int r = e / g.Wp, k = e - r * g.Wp;
        const int y = row0 + r;
        if (y >= g.H) continue;
        C X = {(T)0, (T)0};
        if (k < g.Wh) {
            const C zk = Z[r * L + (k == L ? 0 : k)];
            C zc = Z[r * L + (k == 0 ? 0 : L - k)];
            zc.y = -zc.y;
            const C E = {half * (zk.x + zc.x), half * (zk.y + zc.y)};
            const C d = csub(zk, zc);
            const C O = {half * d.y, -half * d.x};  // (zk - zc) / 2i
            X = cadd(E, cmul(__ldg(twp + k), O));
        }
        if (sizeof(T) == 4)
            scratch[(size_t)f * g.H * g.Wp + g.scratch_index(k, y)] = X;
        else
            ring[(size_t)slot * g.M + (size_t)y * g.Wp + k] = X;
    }
}

// FP32: columns x0 .. x0+CB-1 read from the column-pair scratch, written to the tile-major ring in
// column-major mode order (columns >= W/2+1 are padding and are dropped).  FP64: in place in the
// slot-major ring.
template <typename T>
__global__ void __launch_bounds__(256) k_col_fft(Geometry g, FftPlan plan,
                                                 const typename cplx_t<T>::type *__restrict__ tw,
                                                 typename cplx_t<T>::type *__restrict__ ring, int R, int slot0,
                                                 int CB, const typename cplx_t<T>::type *__restrict__ scratch)
{
    using C = typename cplx_t<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g.H;
    C *bufA = reinterpret_cast<C *>(smem_raw);
    C *bufB = bufA + (size_t)H * CB;
    const int f = blockIdx.y;
    const int x0 = blockIdx.x * CB + 2 * g.kp0;
    const int slot = (slot0 + f) % R;
    const C *src = scratch + (size_t)f * g.H * g.Wp;
    for (int e = threadIdx.x; e < H * CB; e += blockDim.x) {
        const int y = e / CB, c = e - y * CB;
        const int x = x0 + c;
        C v = {(T)0, (T)0};
        if (x < g.Wp) v = (sizeof(T) == 4) ? src[g.scratch_index(x, y)] : ring[(size_t)slot * g.M + (size_t)y * g.Wp + x];
        bufA[e] = v;
    }
    __syncthreads();
    C *Y = fft_all<C, true>(bufA, bufB, plan, CB, CB, 1, tw);
    for (int e = threadIdx.x; e < H * CB; e += blockDim.x) {
        const int y = e / CB, c = e - y * CB;
        const int x = x0 + c;
        if (sizeof(T) == 4) {
            const size_t kl = g.mode(x, y) - g.k0;  // the slab's modes only (wraps above M below k0)
            if (x < g.Wh && kl < g.M) ring[ring_index(slot, kl, R)] = Y[e];
        } else if (x < g.Wp) {
            ring[(size_t)slot * g.M + (size_t)y * g.Wp + x] = Y[e];
        }
    }
}

static int row_rows_per_cta(const Geometry &g)
{
    int rpc = 512 / (g.Lr > 0 ? g.Lr : 1);
    if (rpc < 1) rpc = 1;
    if (rpc > 16) rpc = 16;
    return rpc;
}

template <typename T>
cudaError_t launch_row_fft(const uint16_t *frames, int nf, const unsigned long long *sums, const float *ref,
                           const Geometry &g, const FftPlan &plan, const typename cplx_t<T>::type *tw_row,
                           const typename cplx_t<T>::type *tw_post, typename cplx_t<T>::type *ring, int R,
                           int slot0, cudaStream_t s, typename cplx_t<T>::type *scratch, const float2 *tws_row)
{
    using C = typename cplx_t<T>::type;
    if (nf <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (tws_row) {
            cudaError_t e = launch_row_fft_ct(frames, nf, sums, ref, g, tws_row, tw_post, scratch, s, tw_row);
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();
        }
    }
    const int rpc = row_rows_per_cta(g);
    const size_t smem = 2 * (size_t)rpc * g.Lr * sizeof(C);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_row_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((g.H + rpc - 1) / rpc, nf);
    k_row_fft<T><<<grid, 256, smem, s>>>(frames, sums, ref, g, plan, tw_row, tw_post, ring, R, slot0, rpc, scratch);
    return cudaGetLastError();
}

static int col_block(const Geometry &g, size_t csize)
{
    const size_t elems = (64 * 1024) / csize;  // per buffer; two buffers
    int cb = (int)(elems / (size_t)g.H);
    if (cb < 1) cb = 1;
    if (cb > 64) cb = 64;
    return cb;
}

template <typename T>
cudaError_t launch_col_fft(int nf, const Geometry &g, const FftPlan &plan, const typename cplx_t<T>::type *tw_col,
                           typename cplx_t<T>::type *ring, int R, int slot0, cudaStream_t s,
                           const typename cplx_t<T>::type *scratch, const float2 *tws_col)
{
    using C = typename cplx_t<T>::type;
    if (nf <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        if (tws_col) {
            cudaError_t e = launch_col_fft_ct(nf, g, tws_col, scratch, ring, R, slot0, s);
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();
        }
    }
    int cb = col_block(g, sizeof(C));
    if (sizeof(T) == 4 && cb > 2) cb = 2;  // one scratch column pair per CTA
    const size_t smem = 2 * (size_t)g.H * cb * sizeof(C);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_col_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(sizeof(T) == 4 ? (unsigned)((2 * g.ncp + cb - 1) / cb) : (unsigned)((g.Wp + cb - 1) / cb), nf);
    k_col_fft<T><<<grid, 256, smem, s>>>(g, plan, tw_col, ring, R, slot0, cb, scratch);
    return cudaGetLastError();
}

template cudaError_t launch_row_fft<float>(const uint16_t *, int, const unsigned long long *, const float *,
                                           const Geometry &, const FftPlan &, const float2 *, const float2 *,
                                           float2 *, int, int, cudaStream_t, float2 *, const float2 *);
template cudaError_t launch_row_fft<double>(const uint16_t *, int, const unsigned long long *, const float *,
                                            const Geometry &, const FftPlan &, const double2 *, const double2 *,
                                            double2 *, int, int, cudaStream_t, double2 *, const float2 *);
template cudaError_t launch_col_fft<float>(int, const Geometry &, const FftPlan &, const float2 *, float2 *, int,
                                           int, cudaStream_t, const float2 *, const float2 *);
template cudaError_t launch_col_fft<double>(int, const Geometry &, const FftPlan &, const double2 *, double2 *,
                                            int, int, cudaStream_t, const double2 *, const float2 *);

Geometry make_geometry(int H, int W, bool colmajor)
{
    Geometry g;
    g.H = H;
    g.W = W;
    g.Lr = W / 2;
    g.Wh = W / 2 + 1;
    g.Wp = (g.Wh + 3) / 4 * 4;
    g.HW = (size_t)H * W;
    g.colmajor = colmajor ? 1 : 0;
    const size_t m = colmajor ? (size_t)g.Wh * H : (size_t)H * g.Wp;
    g.M = (m + kTile - 1) / kTile * kTile;
    g.k0 = 0;
    g.kp0 = 0;
    g.ncp = g.Wp / 2;
    return g;
}

bool make_slab(Geometry *g, int slab, int n_slabs)
{
    if (!g->colmajor || g->k0 != 0) return false;
    const long long T = (long long)(g->M / kTile);
    if (n_slabs < 1 || slab < 0 || slab >= n_slabs || n_slabs > T) return false;
    const long long tb = T * slab / n_slabs, te = T * (slab + 1) / n_slabs;
    g->k0 = (size_t)tb * kTile;
    g->M = (size_t)(te - tb) * kTile;
    const long long c0 = (long long)(g->k0 / (size_t)g->H);
    long long c1 = (long long)((g->k0 + g->M - 1) / (size_t)g->H);
    if (c1 > g->Wh - 1) c1 = g->Wh - 1;  // the last tile's padding modes belong to no column
    g->kp0 = (int)(c0 / 2);
    g->ncp = (int)(c1 / 2 - c0 / 2 + 1);
    return true;
}

bool make_plan(int L, FftPlan *plan)
{
    plan->L = L;
    plan->nstages = 0;
    int n = L;
    while (n % 4 == 0) {
        if (plan->nstages >= kMaxStages) return false;
        plan->radix[plan->nstages++] = 4;
        n /= 4;
    }
    while (n % 2 == 0) {
        if (plan->nstages >= kMaxStages) return false;
        plan->radix[plan->nstages++] = 2;
        n /= 2;
    }
    while (n % 3 == 0) {
        if (plan->nstages >= kMaxStages) return false;
        plan->radix[plan->nstages++] = 3;
        n /= 3;
    }
    return n == 1;
}

}  // namespace nfs
