// Compile-time-specialised FP32 FFT passes for the common frame sizes (the same transforms as the
// generic kernels in k_fft.cu: unscaled forward DFT, rows as half-length complex transforms plus
// the real-to-complex split, then columns).
//
// With the transform length, radices and batch known at compile time every index is a shift or
// a constant multiply and every per-thread loop unrolls.  Twiddles come from a per-stage table
// with one row per twiddle power, in which consecutive butterflies read consecutive entries (a
// warp's load is one contiguous run); shared memory is padded by one element in 16 so the
// strided stores of the early Stockham stages do not collide in banks.  The row pass
// writes the column-pair scratch, which the column pass reads as one contiguous run per CTA; the
// column pass (in place in one buffer) writes each column as whole 16-mode tile rows of the ring.
#include <cmath>

#include "nfs_internal.cuh"

namespace nfs {
namespace ct {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ float2 cmi(float2 a) { return {a.y, -a.x}; }  // -i a

template <int R>
struct Dft;
template <>
struct Dft<2> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        const float2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};
template <>
struct Dft<3> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        const float s = 0.86602540378443864676f;  // sin(2 pi / 3)
        const float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        const float2 m = {v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y};
        const float2 r = {s * t2.y, -s * t2.x};
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};
template <>
struct Dft<4> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = cmi(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};
template <>
struct Dft<8> {
    // two 4-point transforms of the even and odd inputs, joined with exp(-2 pi i k / 8)
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        const float h = 0.70710678118654752440f;
        const float2 o1 = {h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};   // (1 - i)/sqrt2 * o1
        const float2 o2 = cmi(o[2]);                                         // -i * o2
        const float2 o3 = {h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};  // (-1 - i)/sqrt2 * o3
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <>
struct Dft<16> {
    // 16 = 4 x 4: transforms of length 4 over the inputs n = 4 n1 + n2 (for each n2), twiddles
    // exp(-2 pi i n2 k1 / 16), transforms of length 4 over n2; output k1 + 4 k2
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
            Dft<4>::run(y[n2]);
        }
        const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;  // cos, sin (pi / 8)
        const float h = 0.70710678118654752440f;
        // n2 = 1: powers 0, 1, 2, 3; n2 = 2: powers 0, 2, 4, 6; n2 = 3: powers 0, 3, 6, 9
        y[1][1] = cmul(y[1][1], {c1, -s1});
        y[1][2] = cmul(y[1][2], {h, -h});
        y[1][3] = cmul(y[1][3], {s1, -c1});
        y[2][1] = cmul(y[2][1], {h, -h});
        y[2][2] = cmi(y[2][2]);
        y[2][3] = cmul(y[2][3], {-h, -h});
        y[3][1] = cmul(y[3][1], {s1, -c1});
        y[3][2] = cmul(y[3][2], {-h, -h});
        y[3][3] = cmul(y[3][3], {-c1, s1});
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<4>::run(z);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
        }
    }
};

// Stockham stages left for a remaining length (radices 16, 8, 4, 3, 2), by dynamic programming
// over the lengths up to rem (rem <= kMaxPlan; longer lengths take radix 8/4/2/3 greedily).
constexpr int kMaxPlan = 2048;
__host__ __device__ constexpr int radix_choice(int i) { return i == 0 ? 8 : (i == 1 ? 16 : (i == 2 ? 4 : (i == 3 ? 2 : 3))); }
__host__ __device__ constexpr int n_stages(int rem)
{
    if (rem <= 1) return 0;
    if (rem > kMaxPlan) return 1 << 20;
    int dp[kMaxPlan + 1] = {};
    for (int n = 2; n <= rem; ++n) {
        int best = 1 << 20;
        for (int i = 0; i < 5; ++i)
            if (n % radix_choice(i) == 0 && 1 + dp[n / radix_choice(i)] < best) best = 1 + dp[n / radix_choice(i)];
        dp[n] = best;
    }
    return dp[rem];
}
// Radix of the next stage of a length-L transform given the remaining length (also used on the
// host for the tables).  Transforms of 2048 points and more take the fewest stages (each one a
// round trip through shared memory; radix 16 pays off there), shorter ones radix 8 first (radix-16
// butterflies leave threads idle in their CTAs and measured slower).
__host__ __device__ constexpr int pick_radix(int L, int rem)
{
    if (L < 2048 || rem > kMaxPlan) return (rem % 8 == 0 && rem != 16) ? 8 : (rem % 4 == 0 ? 4 : (rem % 2 == 0 ? 2 : 3));
    const int best = n_stages(rem);
    for (int i = 0; i < 5; ++i)
        if (rem % radix_choice(i) == 0 && 1 + n_stages(rem / radix_choice(i)) == best) return radix_choice(i);
    return 2;
}
// Offset of the stage with sub-length NS in the per-stage twiddle table of length L.
__host__ __device__ constexpr int tw_offset(int L, int NS)
{
    int off = 0, ns = 1;
    while (ns < NS) {
        const int r = pick_radix(L, L / ns);
        off += ns * (r - 1);
        ns *= r;
    }
    return off;
}
__host__ __device__ constexpr int padded(int x) { return x + (x >> 4); }
// padded(x0 + r STEP) from xp0 = padded(x0): when STEP is a multiple of 16 the padding of the step
// is exact (STEP / 16 more), so only one index per thread is padded at run time.
template <int STEP>
__device__ __forceinline__ int padded_step(int x0, int xp0, int r)
{
    if constexpr (STEP % 16 == 0)
        return xp0 + r * (STEP + STEP / 16);
    else
        return padded(x0 + r * STEP);
}

// One Stockham stage on NB transforms of length L (element (b, i) at b*L + i, or i*NB + b when
// BFAST; padded), NT threads.  INPLACE: in == out, all inputs are read before a barrier.
template <int L, int R, int NS, int NB, bool BFAST, bool INPLACE, int NT>
__device__ __forceinline__ void stage(const float2 *in, float2 *out, const float2 *__restrict__ tws)
{
    constexpr int NBF = L / R;
    constexpr int TOT = NB * NBF;
    constexpr int PER = (TOT + NT - 1) / NT;
    constexpr int OFF = tw_offset(L, NS);
    float2 v[PER][R];
    int jj[PER], bb[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int g = threadIdx.x + p * NT;
        int b, j;
        if (BFAST) {
            b = g % NB;
            j = g / NB;
        } else {
            b = g / NBF;
            j = g % NBF;
        }
        jj[p] = j;
        bb[p] = b;
        if (TOT % NT == 0 || g < TOT) {
            // element i = j + r NBF sits at i NB + b (BFAST) or b L + i
            constexpr int STEP = BFAST ? NBF * NB : NBF;
            const int x0 = BFAST ? j * NB + b : b * L + j, xp0 = padded(x0);
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = in[padded_step<STEP>(x0, xp0, r)];
        }
    }
    if (INPLACE) __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int g = threadIdx.x + p * NT;
        if (TOT % NT == 0 || g < TOT) {
            const int j = jj[p], b = bb[p];
            const int k = j % NS;
            if (NS > 1) {
                // powers of two of the twiddle are read from the table, the others are their
                // products (w^3 = w^2 w, w^5 = w^4 w, ...): fewer L1 reads, a few roundings more
                float2 tw[R];
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    if ((r & (r - 1)) == 0) {
                        tw[r] = __ldg(tws + OFF + (r - 1) * NS + k);
                    } else {
                        int hb = 1;
                        while (2 * hb <= r) hb *= 2;
                        tw[r] = cmul(tw[hb], tw[r - hb]);
                    }
                }
#pragma unroll
                for (int r = 1; r < R; ++r) v[p][r] = cmul(v[p][r], tw[r]);
            }
            Dft<R>::run(v[p]);
            const int base = (j / NS) * NS * R + k;  // output i = base + r NS
            constexpr int STEP = BFAST ? NS * NB : NS;
            const int x0 = BFAST ? base * NB + b : b * L + base, xp0 = padded(x0);
#pragma unroll
            for (int r = 0; r < R; ++r) out[padded_step<STEP>(x0, xp0, r)] = v[p][r];
        }
    }
}

template <int L, int NS, int NB, bool BFAST, bool INPLACE, int NT>
__device__ __forceinline__ float2 *run_stages(float2 *a, float2 *b, const float2 *__restrict__ tws)
{
    if constexpr (NS >= L) {
        return a;
    } else {
        constexpr int R = pick_radix(L, L / NS);
        stage<L, R, NS, NB, BFAST, INPLACE, NT>(a, INPLACE ? a : b, tws);
        __syncthreads();
        if constexpr (INPLACE)
            return run_stages<L, NS * R, NB, BFAST, INPLACE, NT>(a, b, tws);
        else
            return run_stages<L, NS * R, NB, BFAST, INPLACE, NT>(b, a, tws);
    }
}

constexpr int kNT = 256;

// Rows per CTA: the largest power of two with RPC * L <= 2048 (a multiple of 256 for the sizes
// instantiated below).
__host__ __device__ constexpr int rows_per_cta(int L)
{
    int r = 1;
    while (2 * r * L <= 2048) r *= 2;
    return r;
}

// Row pass for frames of width W = 2L: RPC rows per CTA, 8 complex points per thread; output to
// the column-pair scratch of frame blockIdx.y.
// hw / S as an unevaluated float pair (hi + lo, about 46 bits), from FP32 arithmetic only: GB300's
// FP64 pipe is narrow, and a double division in every thread of a row pass kept it 20 % busy.
// Dekker's double-float reciprocal: S = s_hi + s_lo exactly (16-bit counts of at most 2^24
// pixels give S < 2^40, so S - s_hi fits in 16 bits); q0 = hw / s_hi correctly rounded, whose remainder hw - q0 s_hi a fused multiply-add
// gives exactly; one correction q1 = (hw - q0 S) / s_hi; (q0, q1) renormalised by a fast two-sum.
__device__ __forceinline__ void inv_mean_pair(unsigned long long S, int hw, float &hi, float &lo)
{
    if (S == 0ull) {
        hi = lo = 0.f;
        return;
    }
    const float s_hi = __ull2float_rn(S);
    const float s_lo = (float)((long long)S - (long long)s_hi);
    const float h = (float)hw;
    const float q0 = __fdiv_rn(h, s_hi);
    float r = __fmaf_rn(-q0, s_hi, h);
    r = __fmaf_rn(-q0, s_lo, r);
    const float q1 = __fdiv_rn(r, s_hi);
    hi = __fadd_rn(q0, q1);
    lo = __fsub_rn(q1, __fsub_rn(hi, q0));
}

template <int L>
__global__ void __launch_bounds__(kNT) k_row_fft_ct(const uint16_t *__restrict__ frames,
                                                    const unsigned long long *__restrict__ sums,
                                                    const float *__restrict__ ref, Geometry g,
                                                    const float2 *__restrict__ tws, const float2 *__restrict__ twp,
                                                    float2 *__restrict__ scratch)
{
    constexpr int RPC = rows_per_cta(L);
    constexpr int N = RPC * L;
    constexpr int PER = N / kNT;
    static_assert(N % kNT == 0, "row batch must fill the CTA");
    __shared__ __align__(16) float2 bufA[padded(N)];
    __shared__ __align__(16) float2 bufB[padded(N)];
    const int f = blockIdx.y;
    const int row0 = blockIdx.x * RPC;
    // 1/<i> as a float pair; the reference subtraction sits inside the first FMA (see k_fft.cu)
    float inv_hi, inv_lo;
    inv_mean_pair(sums[f], g.HW, inv_hi, inv_lo);
    const uint16_t *fr = frames + (size_t)f * g.HW;
    constexpr int W = 2 * L;
    unsigned raw[PER];
    float2 rf[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * kNT;
        const int r = e / L, m = e % L;
        const int y = row0 + r;
        if (y < g.H) {
            const size_t o = (size_t)y * W + 2 * m;
            raw[p] = __ldg(reinterpret_cast<const unsigned *>(fr + o));
            rf[p] = __ldg(reinterpret_cast<const float2 *>(ref + o));
        } else {
            raw[p] = 0u;
            rf[p] = {0.f, 0.f};
        }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * kNT;
        const float a = (float)(raw[p] & 0xffffu), b = (float)(raw[p] >> 16);
        bufA[padded(e)] = {__fmaf_rn(a, inv_lo, __fmaf_rn(a, inv_hi, -rf[p].x)),
                           __fmaf_rn(b, inv_lo, __fmaf_rn(b, inv_hi, -rf[p].y))};
    }
    __syncthreads();
    const float2 *Z = run_stages<L, 1, RPC, false, false, kNT>(bufA, bufB, tws);

    // outputs k < WP of each row, laid out so that a thread group covers the RPC rows of one
    // column pair (contiguous in the scratch)
    constexpr int WP = ((L + 1) + 3) / 4 * 4;
    float2 *out = scratch + (size_t)f * g.H * WP;
    for (int e = threadIdx.x; e < RPC * WP; e += kNT) {
        const int c = e & 1, r = (e >> 1) % RPC, kp = (e >> 1) / RPC;
        const int k = 2 * kp + c;
        const int y = row0 + r;
        if (y >= g.H) continue;
        float2 X = {0.f, 0.f};
        if (k <= L) {
            const float2 zk = Z[padded(r * L + (k == L ? 0 : k))];
            float2 zc = Z[padded(r * L + (k == 0 ? 0 : L - k))];
            zc.y = -zc.y;
            const float2 E = {0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y)};
            const float2 d = csub(zk, zc);
            const float2 O = {0.5f * d.y, -0.5f * d.x};
            X = cadd(E, cmul(__ldg(twp + k), O));
        }
        out[((size_t)kp * g.H + y) * 2 + c] = X;
    }
}

// Row pass of 2048-wide frames, one warp per row.  The packed row z[n] = p[2n] + i p[2n+1]
// (1024 points) is transformed as 32 x 32 (n = 32 n1 + n2, k = k1 + 32 k2):
//   lane n2 takes the 32-point DFT over n1 in registers and multiplies by W_1024^(n2 k1);
//   the 32 x 32 values pass once through shared memory (padded rows: both the store and the load
//   are two wavefronts per warp);
//   lane k1 takes the 32-point DFT over n2, giving Z[k1 + 32 k2] in its register k2.
// The real-to-complex split X[k] = E + W_2048^k O (E, O from Z[k] and conj Z[1024 - k]) finds
// Z[1024 - k] in lane (32 - k1) mod 32, register 31 - k2 (lane 0: its own register (32 - k2) mod
// 32), read with a warp shuffle.  One shared-memory round trip per row instead of one per radix
// stage.
constexpr int kRowWarpsW = 4;  // rows (warps) per CTA

// W_32^j = exp(-2 pi i j / 32), j < 22 (the twiddles of the 8 x 4 decomposition below)
__constant__ float2 kW32[22] = {
    {1.0f, 0.0f}, {0.98078528040323043f, -0.19509032201612825f}, {0.92387953251128674f, -0.38268343236508978f},
    {0.83146961230254524f, -0.55557023301960218f}, {0.70710678118654757f, -0.70710678118654746f}, {0.55557023301960229f, -0.83146961230254524f},
    {0.38268343236508984f, -0.92387953251128674f}, {0.19509032201612833f, -0.98078528040323043f}, {0.0f, -1.0f},
    {-0.19509032201612819f, -0.98078528040323043f}, {-0.38268343236508973f, -0.92387953251128674f}, {-0.55557023301960196f, -0.83146961230254546f},
    {-0.70710678118654746f, -0.70710678118654757f}, {-0.83146961230254535f, -0.55557023301960218f}, {-0.92387953251128674f, -0.38268343236508989f},
    {-0.98078528040323043f, -0.19509032201612861f}, {-1.0f, 0.0f}, {-0.98078528040323043f, 0.19509032201612836f},
    {-0.92387953251128685f, 0.38268343236508967f}, {-0.83146961230254546f, 0.55557023301960196f}, {-0.70710678118654768f, 0.70710678118654746f},
    {-0.55557023301960218f, 0.83146961230254524f}};

// W_64^k = W_2048^(32 k), k < 32: the real-to-complex split's twiddle steps between a lane's
// outputs, as float values of the same double cosines and sines as the post-processing table
// (warp-uniform indices: constant-bank operands instead of 31 loads per lane and row)
__constant__ float2 kW64[32] = {
    {1.0f, -0.0f}, {0.9951847195625305f, -0.0980171412229538f}, {0.9807852506637573f, -0.19509032368659973f}, {0.9569403529167175f, -0.290284663438797f},
    {0.9238795042037964f, -0.3826834261417389f}, {0.8819212913513184f, -0.4713967442512512f}, {0.8314695954322815f, -0.5555702447891235f}, {0.7730104327201843f, -0.6343932747840881f},
    {0.7071067690849304f, -0.7071067690849304f}, {0.6343932747840881f, -0.7730104327201843f}, {0.5555702447891235f, -0.8314695954322815f}, {0.4713967442512512f, -0.8819212913513184f},
    {0.3826834261417389f, -0.9238795042037964f}, {0.290284663438797f, -0.9569403529167175f}, {0.19509032368659973f, -0.9807852506637573f}, {0.0980171412229538f, -0.9951847195625305f},
    {6.123234262925839e-17f, -1.0f}, {-0.0980171412229538f, -0.9951847195625305f}, {-0.19509032368659973f, -0.9807852506637573f}, {-0.290284663438797f, -0.9569403529167175f},
    {-0.3826834261417389f, -0.9238795042037964f}, {-0.4713967442512512f, -0.8819212913513184f}, {-0.5555702447891235f, -0.8314695954322815f}, {-0.6343932747840881f, -0.7730104327201843f},
    {-0.7071067690849304f, -0.7071067690849304f}, {-0.7730104327201843f, -0.6343932747840881f}, {-0.8314695954322815f, -0.5555702447891235f}, {-0.8819212913513184f, -0.4713967442512512f},
    {-0.9238795042037964f, -0.3826834261417389f}, {-0.9569403529167175f, -0.290284663438797f}, {-0.9807852506637573f, -0.19509032368659973f}, {-0.9951847195625305f, -0.0980171412229538f}};

// In-register 32-point DFT, natural order in and out: 32 = 8 x 4 (n = 4 m + r, k = k' + 8 k''),
// eight-point transforms over m, twiddles W_32^(r k'), four-point transforms over r.
__device__ __forceinline__ void dft32(float2 (&v)[32])
{
    float2 y[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int m = 0; m < 8; ++m) y[r][m] = v[4 * m + r];
        Dft<8>::run(y[r]);
#pragma unroll
        for (int k = 1; k < 8; ++k)
            if (r) y[r][k] = cmul(y[r][k], kW32[r * k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float2 u[4] = {y[0][k], y[1][k], y[2][k], y[3][k]};
        Dft<4>::run(u);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[k + 8 * q] = u[q];
    }
}

// Output columns of a 2048-wide row (W/2 + 1 rounded up to 4) and the CTA-wide store of its rows to
// the column-pair scratch: element (kp, r, c) goes to ((kp H + y0 + r) 2 + c), so the CTA's four
// consecutive rows of one column pair are one 64-byte run (a row stored alone gives 16-byte runs).
constexpr int kRowPitchW = 1028;
static_assert(kRowWarpsW == 4, "store_rows indexes 4 rows x 2 columns per column pair");
static_assert(kRowWarpsW * kRowPitchW <= kRowWarpsW * 32 * 33, "output rows fit the transpose buffer");
__device__ __forceinline__ void store_rows(float2 (&tr)[kRowWarpsW][32][33], const Geometry &g, int y0,
                                           float2 *__restrict__ out)
{
    const float2 *rows = &tr[0][0][0];
    for (int e = threadIdx.x; e < kRowWarpsW * kRowPitchW; e += kRowWarpsW * 32) {
        const int c = e & 1, r = (e >> 1) & (kRowWarpsW - 1), kp = e >> 3;
        const int y = y0 + r;
        if (y < g.H) out[((size_t)kp * g.H + y) * 2 + c] = rows[r * kRowPitchW + 2 * kp + c];
    }
}

__global__ void __launch_bounds__(kRowWarpsW * 32, 4) k_row_fft_w1024(const uint16_t *__restrict__ frames,
                                                                       const unsigned long long *__restrict__ sums,
                                                                       const float *__restrict__ ref, Geometry g,
                                                                       const float2 *__restrict__ tw,
                                                                       const float2 *__restrict__ twp,
                                                                       float2 *__restrict__ scratch)
{
    __shared__ __align__(16) float2 tr[kRowWarpsW][32][33];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int f = blockIdx.y;
    const int y0 = blockIdx.x * kRowWarpsW;
    const int y = y0 + wq;
    if (y >= g.H) {  // rows past the frame: only the CTA's two barriers below
        __syncthreads();
        __syncthreads();
        store_rows(tr, g, y0, scratch + (size_t)f * g.H * g.Wp);
        return;
    }
    // 1/<i> as a float pair; the reference subtraction sits inside the first FMA (see k_fft.cu)
    float inv_hi, inv_lo;
    inv_mean_pair(sums[f], g.HW, inv_hi, inv_lo);
    const unsigned *fr = reinterpret_cast<const unsigned *>(frames + (size_t)f * g.HW + (size_t)y * 2048);
    // the reference image rebuilt from the reference frame's 2-byte counts: fl32(count) times its
    // reciprocal mean's high part, the product k_reference stored (half the bytes of the floats)
    const char *rb = reinterpret_cast<const char *>(ref);
    const unsigned *rr = reinterpret_cast<const unsigned *>(rb + ref_raw_offset(g.HW)) + (size_t)y * 1024;
    const float ref_hi = __ldg(reinterpret_cast<const float2 *>(rb + ref_inv_offset(g.HW))).x;
    float2 v[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
        const unsigned raw = __ldg(fr + 32 * n1 + lane);
        const unsigned rw = __ldg(rr + 32 * n1 + lane);
        const float rx = __fmul_rn((float)(rw & 0xffffu), ref_hi), ry = __fmul_rn((float)(rw >> 16), ref_hi);
        const float a = (float)(raw & 0xffffu), b = (float)(raw >> 16);
        v[n1] = {__fmaf_rn(a, inv_lo, __fmaf_rn(a, inv_hi, -rx)), __fmaf_rn(b, inv_lo, __fmaf_rn(b, inv_hi, -ry))};
    }
    dft32(v);
    // W_1024^(n2 k1) with k1 = k' + 8 k'': W_1024^(n2 k') W_1024^(8 n2 k'')
    float2 a8[8], b4[4];
#pragma unroll
    for (int k = 0; k < 8; ++k) a8[k] = __ldg(tw + lane * k);
#pragma unroll
    for (int q = 0; q < 4; ++q) b4[q] = __ldg(tw + ((8 * lane * q) & 1023));
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
        const float2 w = (k1 >> 3) ? cmul(a8[k1 & 7], b4[k1 >> 3]) : a8[k1];
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) tr[wq][k1][lane] = v[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = tr[wq][lane][n2];
    dft32(v);  // v[k2] = Z[lane + 32 k2]

    // every warp is done with its transpose tile: the CTA's buffer now takes its four output rows
    __syncthreads();
    float2 *row = &tr[0][0][0] + wq * kRowPitchW;
    const float2 p1 = __ldg(twp + lane);  // W_2048^lane
    const int src = (32 - lane) & 31;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
        float2 zc;
        zc.x = __shfl_sync(0xffffffffu, v[31 - k2].x, src);
        zc.y = __shfl_sync(0xffffffffu, v[31 - k2].y, src);
        if (lane == 0) zc = v[(32 - k2) & 31];
        zc.y = -zc.y;
        const float2 zk = v[k2];
        const float2 E = {0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y)};
        const float2 d = csub(zk, zc);
        const float2 O = {0.5f * d.y, -0.5f * d.x};
        const float2 w = k2 ? cmul(p1, kW64[k2]) : p1;  // W_2048^(lane + 32 k2)
        row[lane + 32 * k2] = cadd(E, cmul(w, O));
    }
    // k = 1024 (the Nyquist column, from Z[0]) and the zero padding columns 1025 .. Wp - 1
    if (lane == 0) {
        const float2 zk = v[0];
        const float2 zc = {zk.x, -zk.y};
        const float2 E = {0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y)};
        const float2 d = csub(zk, zc);
        const float2 O = {0.5f * d.y, -0.5f * d.x};
        row[1024] = cadd(E, cmul(__ldg(twp + 1024), O));
    } else if (1024 + lane < kRowPitchW) {
        row[1024 + lane] = {0.f, 0.f};
    }
    __syncthreads();
    store_rows(tr, g, y0, scratch + (size_t)f * g.H * g.Wp);
}

// Threads of the column pass: the largest of 256, 128, 64 that divides the 2H points of a pair.
__host__ __device__ constexpr int col_threads(int H)
{
    return (2 * H) % 256 == 0 ? 256 : ((2 * H) % 128 == 0 ? 128 : 64);
}

// Column pass for frames of height H: one column pair per CTA, read contiguously from the scratch,
// transformed in place, written as whole tile rows of the ring (column-major modes).
template <int H>
__global__ void __launch_bounds__(col_threads(H)) k_col_fft_ct(Geometry g, const float2 *__restrict__ tws,
                                                               const float2 *__restrict__ scratch,
                                                               float2 *__restrict__ ring, int R, int slot0)
{
    constexpr int NT = col_threads(H);
    constexpr int N = H * 2;
    constexpr int PER = N / NT;
    static_assert(N % NT == 0, "column batch must fill the CTA");
    __shared__ __align__(16) float2 buf[padded(N)];
    const int f = blockIdx.y;
    const int kp = blockIdx.x + g.kp0;
    const int slot = (slot0 + f) % R;
    const float2 *src = scratch + (size_t)f * H * g.Wp + (size_t)kp * H * 2;
    const int t = threadIdx.x;
#pragma unroll
    for (int p = 0; p < PER; ++p)  // e = y * 2 + c: the BFAST layout of two columns
        buf[padded_step<NT>(t, padded(t), p)] = __ldg(src + t + p * NT);
    __syncthreads();
    const float2 *Y = run_stages<H, 1, 2, true, true, NT>(buf, buf, tws);
    if constexpr (H % NT == 0 && NT % kTile == 0 && H % kTile == 0) {
        // element e = t + p NT is column c = p NT / H, row y = t + (p NT) mod H.  Its slab-local mode
        // kl = kl0[c] + yoff (signed: negative below the slab) has tile floor(kl / 16) = floor(kl0 / 16)
        // + yoff / 16 and lane kl mod 16 = t mod 16, because the column start and the slab's first
        // mode (always) are multiples of the tile: the ring index is a per-column base plus R yoff.
        if ((g.k0 & (kTile - 1)) == 0) {
            long long kl0[2], base[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                kl0[c] = (long long)(2 * kp + c) * H + t - (long long)g.k0;
                base[c] = ((kl0[c] >> kTileShift) * R + slot) * kTile + (t & (kTile - 1));
            }
            const int yp = padded(2 * t);
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                constexpr int CPER = H / NT;  // elements per column and thread
                const int c = p / CPER, yoff = (p % CPER) * NT;
                const long long kl = kl0[c] + yoff;
                if (2 * kp + c < g.Wh && kl >= 0 && kl < (long long)g.M)
                    ring[base[c] + (long long)R * yoff] = Y[padded_step<2 * NT>(2 * t, yp, p % CPER) + c];
            }
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = t + p * NT;
        const int c = e / H, y = e % H;
        const int kx = 2 * kp + c;
        const size_t kl = (size_t)kx * H + y - g.k0;  // the slab's modes only
        if (kx < g.Wh && kl < g.M) ring[ring_index(slot, kl, R)] = Y[padded(y * 2 + c)];
    }
}

}  // namespace ct

std::vector<double> ct_stage_twiddles(int L)
{
    std::vector<double> t;
    int ns = 1;
    while (ns < L) {
        const int r = ct::pick_radix(L, L / ns);
        for (int q = 1; q < r; ++q)  // q-major: consecutive butterflies k read consecutive entries
            for (int k = 0; k < ns; ++k) {
                const double a = 2.0 * M_PI * (double)k * q / ((double)ns * r);
                t.push_back(std::cos(a));
                t.push_back(-std::sin(a));
            }
        ns *= r;
    }
    return t;
}

template <int L>
static cudaError_t row_ct(const uint16_t *frames, int nf, const unsigned long long *sums, const float *ref,
                          const Geometry &g, const float2 *tws, const float2 *twp, float2 *scratch, cudaStream_t s)
{
    constexpr int RPC = ct::rows_per_cta(L);
    dim3 grid((g.H + RPC - 1) / RPC, nf);
    ct::k_row_fft_ct<L><<<grid, ct::kNT, 0, s>>>(frames, sums, ref, g, tws, twp, scratch);
    return cudaGetLastError();
}

template <int H>
static cudaError_t col_ct(int nf, const Geometry &g, const float2 *tws, const float2 *scratch, float2 *ring, int R,
                          int slot0, cudaStream_t s)
{
    dim3 grid(g.ncp, nf);
    ct::k_col_fft_ct<H><<<grid, ct::col_threads(H), 0, s>>>(g, tws, scratch, ring, R, slot0);
    return cudaGetLastError();
}

static bool ct_size(int n)
{
    switch (n) {
        case 64: case 128: case 192: case 256: case 384: case 512: case 768: case 1024: case 2048: return true;
        default: return false;
    }
}

cudaError_t launch_row_fft_ct(const uint16_t *frames, int nf, const unsigned long long *sums, const float *ref,
                              const Geometry &g, const float2 *tws, const float2 *twp, float2 *scratch, cudaStream_t s,
                              const float2 *tw)
{
    if (!tws || (reinterpret_cast<uintptr_t>(frames) & 3) || g.Wp != ((g.Lr + 1) + 3) / 4 * 4 || !ct_size(g.Lr))
        return cudaErrorNotSupported;
    if (g.Lr == 1024 && tw && g.Wp == ct::kRowPitchW) {  // one warp per row (the plan below: 4 shared-memory stages)
        dim3 grid((g.H + ct::kRowWarpsW - 1) / ct::kRowWarpsW, nf);
        ct::k_row_fft_w1024<<<grid, ct::kRowWarpsW * 32, 0, s>>>(frames, sums, ref, g, tw, twp, scratch);
        return cudaGetLastError();
    }
    switch (g.Lr) {
        case 64: return row_ct<64>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 128: return row_ct<128>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 192: return row_ct<192>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 256: return row_ct<256>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 384: return row_ct<384>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 512: return row_ct<512>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 768: return row_ct<768>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 1024: return row_ct<1024>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        case 2048: return row_ct<2048>(frames, nf, sums, ref, g, tws, twp, scratch, s);
        default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_col_fft_ct(int nf, const Geometry &g, const float2 *tws, const float2 *scratch, float2 *ring,
                              int R, int slot0, cudaStream_t s)
{
    if (!tws || !g.colmajor || !ct_size(g.H)) return cudaErrorNotSupported;
    switch (g.H) {
        case 64: return col_ct<64>(nf, g, tws, scratch, ring, R, slot0, s);
        case 128: return col_ct<128>(nf, g, tws, scratch, ring, R, slot0, s);
        case 192: return col_ct<192>(nf, g, tws, scratch, ring, R, slot0, s);
        case 256: return col_ct<256>(nf, g, tws, scratch, ring, R, slot0, s);
        case 384: return col_ct<384>(nf, g, tws, scratch, ring, R, slot0, s);
        case 512: return col_ct<512>(nf, g, tws, scratch, ring, R, slot0, s);
        case 768: return col_ct<768>(nf, g, tws, scratch, ring, R, slot0, s);
        case 1024: return col_ct<1024>(nf, g, tws, scratch, ring, R, slot0, s);
        case 2048: return col_ct<2048>(nf, g, tws, scratch, ring, R, slot0, s);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace nfs
