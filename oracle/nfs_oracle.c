/*
 * nfs_oracle.c -- plain FP64 CPU oracle for the double-frame differential analysis of dynamic
 * near-field-scattering (NFS) image sequences (Cerchiari et al., "Quasi-real-time analysis of
 * dynamic near field scattering data using a graphics processing unit", arXiv:1209.3362).
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA library and is used by the test suite,
 * the smoke check and the benchmark's CPU-baseline leg; the product path never calls it.  It
 * shares no code with the CUDA library.
 *
 * What it computes, written out from its definition (paragraph on the differential analysis and
 * Eq. 1, and the processing paragraph that averages "for any given Delta N"):
 *
 *   1. n_t(x) = i_t(x) / <i_t>_x                 each image divided by its spatial average
 *   2. for every delay tau_j and every t with t + tau_j < N:
 *        Delta i(x) = n_t(x) - n_{t+tau_j}(x)     the difference is formed in REAL space
 *        Delta I(k) = sum_x Delta i(x) exp(-2 pi i (k_x x / W + k_y y / H))   (own FFT, unscaled)
 *        P_j(k)    += |Delta I(k)|^2              for the half plane 0 <= k_x <= W/2
 *   3. D(k, tau_j) = P_j(k) / (N - tau_j)         the time average over all stationary pairs
 *   4. azimuthal average into n_q bins (Fig. 1e,f):  with k_y' = k_y or k_y - H (signed),
 *        L = lcm(H, W), m = k_x L/W, n = k_y' L/H, r2 = m^2 + n^2 (an integer),
 *        bin(k) = floor( isqrt(4 n_q^2 r2) / L )  ==  floor(2 n_q |f|) with |f| in cycles/px;
 *        a mode is kept when bin < n_q and k != 0; weight w_k = 1 on the k_x = 0 and k_x = W/2
 *        columns, 2 elsewhere (the half plane then sums like the full plane);
 *        C_b = sum of w_k over the bin,  D_b(tau_j) = sum_{k in b} w_k D(k, tau_j) / C_b.
 *
 * Readings where the paper is silent: the FFT sign and scale (e^{-i}, unscaled), the DC mode
 * (excluded: its difference is 0 in exact arithmetic), the binning rule above, mean
 * normalisation rather than division by the zero-frequency value (they differ by a constant), and
 * a frame whose spatial mean is 0 (a dark frame) normalising to the zero image.
 *
 * Parity pins (tests/test_oracle.py): the FFT against brute-force DFT sums, Parseval's identity,
 * exact zeros at tau = 0 and for identical frames, time-reversal and intensity-scale invariance,
 * the FFT-linearity route, a travelling-cosine closed form (also with dark frames), the
 * Ornstein-Uhlenbeck statistical closed form of Eq. 1, and the bin table against a brute-force
 * count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NFSOR_OK 0
#define NFSOR_EINVAL (-1)
#define NFSOR_ENOMEM (-3)

typedef struct {
    double re, im;
} cplx;

/* ---------------------------------------------------------------- 1-D DFT (recursive) ---- */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/* Table of exp(-2 pi i j / n), j = 0..n-1, from cos and sin of the reduced angle. */
static cplx *twiddle_table(int n)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w) return NULL;
    for (int j = 0; j < n; ++j) {
        double a = 2.0 * M_PI * (double)j / (double)n;
        w[j].re = cos(a);
        w[j].im = -sin(a);
    }
    return w;
}

/*
 * X[k] = sum_{q < len} x[q * stride] * exp(-2 pi i q k / len), k = 0..len-1, stored contiguously.
 * Decimation in time over the smallest prime factor p of len: the p interleaved subsequences are
 * transformed recursively (results in X[r*m .. r*m+m)), then combined with
 *     X[k + s m] = sum_{r < p} w_len^{r (k + s m)} Y_r[k].
 * tw is the table of the top-level length ntop; w_len^j = tw[j * (ntop / len)].
 */
static void dft_rec(int len, const cplx *x, int stride, cplx *X, cplx *scratch, const cplx *tw,
                    int ntop)
{
    if (len == 1) {
        X[0] = x[0];
        return;
    }
    int p = smallest_factor(len);
    int m = len / p;
    for (int r = 0; r < p; ++r) dft_rec(m, x + (size_t)r * stride, stride * p, X + (size_t)r * m, scratch, tw, ntop);
    int step = ntop / len;
    for (int k = 0; k < m; ++k) {
        for (int s = 0; s < p; ++s) {
            int kk = k + s * m;
            double ar = 0.0, ai = 0.0;
            long e = 0; /* (r * kk) mod len, advanced by kk per term */
            for (int r = 0; r < p; ++r) {
                cplx w = tw[e * step];
                cplx y = X[(size_t)r * m + k];
                ar += w.re * y.re - w.im * y.im;
                ai += w.re * y.im + w.im * y.re;
                e += kk;
                if (e >= len) e -= len;
            }
            scratch[kk].re = ar;
            scratch[kk].im = ai;
        }
    }
    memcpy(X, scratch, sizeof(cplx) * (size_t)len);
}

/* Workspace for 2-D transforms of one H x W shape. */
#define COLS_PER_GATHER 8 /* columns copied out together (whole cache lines per row) */
typedef struct {
    int H, W;
    cplx *twH, *twW;
    cplx *line_in, *line_out, *scratch;
    cplx *cols; /* COLS_PER_GATHER columns of H values each */
} fft2_plan;

static void fft2_free(fft2_plan *p)
{
    free(p->twH);
    free(p->twW);
    free(p->line_in);
    free(p->line_out);
    free(p->scratch);
    free(p->cols);
    memset(p, 0, sizeof(*p));
}

static int fft2_init(fft2_plan *p, int H, int W)
{
    memset(p, 0, sizeof(*p));
    p->H = H;
    p->W = W;
    int n = H > W ? H : W;
    p->twH = twiddle_table(H);
    p->twW = twiddle_table(W);
    p->line_in = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    p->line_out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    p->scratch = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    p->cols = (cplx *)malloc(sizeof(cplx) * (size_t)H * COLS_PER_GATHER);
    if (!p->twH || !p->twW || !p->line_in || !p->line_out || !p->scratch || !p->cols) {
        fft2_free(p);
        return NFSOR_ENOMEM;
    }
    return NFSOR_OK;
}

/* In-place unscaled forward 2-D DFT of a row-major H x W complex array: every row, then every
 * column (columns are copied out a few at a time, transformed one by one and copied back). */
static void fft2_forward(fft2_plan *p, cplx *a)
{
    int H = p->H, W = p->W;
    for (int y = 0; y < H; ++y) {
        dft_rec(W, a + (size_t)y * W, 1, p->line_out, p->scratch, p->twW, W);
        memcpy(a + (size_t)y * W, p->line_out, sizeof(cplx) * (size_t)W);
    }
    for (int x0 = 0; x0 < W; x0 += COLS_PER_GATHER) {
        int nc = W - x0 < COLS_PER_GATHER ? W - x0 : COLS_PER_GATHER;
        for (int y = 0; y < H; ++y)
            for (int c = 0; c < nc; ++c) p->cols[(size_t)c * H + y] = a[(size_t)y * W + x0 + c];
        for (int c = 0; c < nc; ++c) {
            dft_rec(H, p->cols + (size_t)c * H, 1, p->line_out, p->scratch, p->twH, H);
            memcpy(p->cols + (size_t)c * H, p->line_out, sizeof(cplx) * (size_t)H);
        }
        for (int y = 0; y < H; ++y)
            for (int c = 0; c < nc; ++c) a[(size_t)y * W + x0 + c] = p->cols[(size_t)c * H + y];
    }
}

/* Public: full-plane unscaled forward 2-D DFT (complex in, complex out; split re/im arrays). */
int nfsor_fft2(int H, int W, const double *in_re, const double *in_im, double *out_re, double *out_im)
{
    if (H <= 0 || W <= 0 || !in_re || !out_re || !out_im) return NFSOR_EINVAL;
    fft2_plan p;
    if (fft2_init(&p, H, W)) return NFSOR_ENOMEM;
    size_t n = (size_t)H * W;
    cplx *a = (cplx *)malloc(sizeof(cplx) * n);
    if (!a) {
        fft2_free(&p);
        return NFSOR_ENOMEM;
    }
    for (size_t i = 0; i < n; ++i) {
        a[i].re = in_re[i];
        a[i].im = in_im ? in_im[i] : 0.0;
    }
    fft2_forward(&p, a);
    for (size_t i = 0; i < n; ++i) {
        out_re[i] = a[i].re;
        out_im[i] = a[i].im;
    }
    free(a);
    fft2_free(&p);
    return NFSOR_OK;
}

/* ---------------------------------------------------------------- radial bins ------------ */

static int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* floor(sqrt(v)) of a 128-bit integer: 4 n_q^2 r2 exceeds 64 bits for large n_q and lcm(H, W). */
typedef unsigned __int128 u128;
static uint64_t isqrt_u128(u128 v)
{
    uint64_t s = (uint64_t)sqrt((double)v);
    while (s > 0 && (u128)s * s > v) --s;
    while ((u128)(s + 1) * (s + 1) <= v) ++s;
    return s;
}

/*
 * bin_of_mode[ky][kx] (kx = 0..W/2) gets the bin index or -1 (excluded), counts[b] = C_b (integer
 * weights 1 or 2), q_mean[b] = sum w_k 2 pi |f_k| / C_b in rad/px (0 for an empty bin).
 */
int nfsor_bins(int H, int W, int nq, int32_t *bin_of_mode, int64_t *counts, double *q_mean)
{
    if (H <= 0 || W <= 0 || (W % 2) || (H % 2) || nq <= 0 || !counts) return NFSOR_EINVAL;
    int64_t L = (int64_t)H / gcd64(H, W) * W;
    int Wh = W / 2 + 1;
    double *qsum = (double *)calloc((size_t)nq, sizeof(double));
    if (!qsum) return NFSOR_ENOMEM;
    for (int b = 0; b < nq; ++b) counts[b] = 0;
    for (int ky = 0; ky < H; ++ky) {
        int64_t kys = ky <= H / 2 ? ky : ky - H;
        for (int kx = 0; kx < Wh; ++kx) {
            int64_t m = (int64_t)kx * (L / W);
            int64_t n = kys * (L / H);
            uint64_t r2 = (uint64_t)(m * m + n * n);
            u128 a = (u128)4 * (u128)nq * (u128)nq * (u128)r2;
            int64_t b = (int64_t)(isqrt_u128(a) / (uint64_t)L);
            int keep = (b < nq) && !(kx == 0 && ky == 0);
            if (bin_of_mode) bin_of_mode[(size_t)ky * Wh + kx] = keep ? (int32_t)b : -1;
            if (!keep) continue;
            int w = (kx == 0 || kx == W / 2) ? 1 : 2;
            counts[b] += w;
            qsum[b] += w * 2.0 * M_PI * sqrt((double)r2) / (double)L;
        }
    }
    if (q_mean)
        for (int b = 0; b < nq; ++b) q_mean[b] = counts[b] ? qsum[b] / (double)counts[b] : 0.0;
    free(qsum);
    return NFSOR_OK;
}

/* ---------------------------------------------------------------- frames ----------------- */

/* Frames are either uint16 counts (f16 != NULL) or FP64 values (f64 != NULL). */
typedef struct {
    const uint16_t *f16;
    const double *f64;
    int N, H, W, normalize;
} frame_src;

/* dst = n_t: frame t divided by its spatial mean (or copied when normalize == 0).  A frame whose
 * spatial mean is 0 (a dark frame: every uint16 count 0) normalises to the zero image. */
static void load_frame(const frame_src *s, int t, double *dst)
{
    size_t n = (size_t)s->H * s->W;
    if (s->f16) {
        const uint16_t *src = s->f16 + (size_t)t * n;
        uint64_t sum = 0;
        for (size_t i = 0; i < n; ++i) sum += src[i];
        double mean = (double)sum / (double)n;
        for (size_t i = 0; i < n; ++i)
            dst[i] = !s->normalize ? (double)src[i] : (mean != 0.0 ? (double)src[i] / mean : 0.0);
    } else {
        const double *src = s->f64 + (size_t)t * n;
        double sum = 0.0;
        for (size_t i = 0; i < n; ++i) sum += src[i];
        double mean = sum / (double)n;
        for (size_t i = 0; i < n; ++i) dst[i] = !s->normalize ? src[i] : (mean != 0.0 ? src[i] / mean : 0.0);
    }
}

static int check_delays(const int32_t *delays, int nd)
{
    for (int j = 0; j < nd; ++j) {
        if (delays[j] < 0) return 0;
        if (j > 0 && delays[j] <= delays[j - 1]) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------------- structure function ----- */

/* Adds |DFT(n_t - n_{t+tau})|^2 over the half plane into acc (work buffers a, b, F). */
static void add_pair(const frame_src *s, fft2_plan *plan, int t, int tau, double *a, double *b, cplx *F, double *acc)
{
    int H = s->H, W = s->W, Wh = W / 2 + 1;
    size_t nfull = (size_t)H * W;
    load_frame(s, t, a);
    load_frame(s, t + tau, b);
    for (size_t i = 0; i < nfull; ++i) {
        F[i].re = a[i] - b[i];
        F[i].im = 0.0;
    }
    fft2_forward(plan, F);
    for (int ky = 0; ky < H; ++ky)
        for (int kx = 0; kx < Wh; ++kx) {
            cplx v = F[(size_t)ky * W + kx];
            acc[(size_t)ky * Wh + kx] += v.re * v.re + v.im * v.im;
        }
}

/*
 * Work is split over threads by pairs, not by delay: consecutive delays are grouped until the group
 * has at least 4 pairs per thread, the group's pairs are listed in order (delay, then t ascending)
 * and thread th takes the contiguous th-th share of the list.  A thread sums its pairs of one delay
 * into its own partial ("segment"); the partials of a delay are then added in thread order, so the
 * result does not depend on timing.  Pairs of one delay may be summed in any order (each is one
 * term of the time average).
 */
static int sf_core(const frame_src *s, const int32_t *delays, int nd, int nq, int nthreads, double *D,
                   int64_t *bin_counts, int64_t *pair_counts, double *q_mean, double *D2d)
{
    int N = s->N, H = s->H, W = s->W;
    if (N < 0 || H < 2 || W < 2 || (H % 2) || (W % 2) || nd < 0 || nq <= 0 || !delays || !D || !bin_counts ||
        !pair_counts)
        return NFSOR_EINVAL;
    if (!check_delays(delays, nd)) return NFSOR_EINVAL;
    int Wh = W / 2 + 1;
    size_t nhalf = (size_t)H * Wh, nfull = (size_t)H * W;
    int32_t *bin = (int32_t *)malloc(sizeof(int32_t) * nhalf);
    double *P = (double *)malloc(sizeof(double) * nhalf);
    if (!bin || !P) {
        free(bin);
        free(P);
        return NFSOR_ENOMEM;
    }
    int rc = nfsor_bins(H, W, nq, bin, bin_counts, q_mean);
    if (rc) {
        free(bin);
        free(P);
        return rc;
    }
#ifdef _OPENMP
    int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    int nth = 1;
    (void)nthreads;
#endif
    for (int j = 0; j < nd; ++j) pair_counts[j] = N - delays[j] > 0 ? N - delays[j] : 0;
    int err = 0;
    for (int j0 = 0; j0 < nd && !err;) {
        /* the group j0 .. j1-1 and the first pair index of each of its delays */
        long long tot = 0;
        int j1 = j0;
        while (j1 < nd && (tot < 4LL * nth || j1 == j0)) tot += pair_counts[j1++];
        int ng = j1 - j0;
        long long *first = (long long *)malloc(sizeof(long long) * (size_t)(ng + 1));
        int nseg = nth + ng - 1; /* segment of (thread th, delay j) = th + (j - j0) */
        double *seg = (double *)calloc((size_t)nseg * nhalf, sizeof(double));
        if (!first || !seg) {
            free(first);
            free(seg);
            err = 1;
            break;
        }
        first[0] = 0;
        for (int g = 0; g < ng; ++g) first[g + 1] = first[g] + pair_counts[j0 + g];
#pragma omp parallel num_threads(nth)
        {
#ifdef _OPENMP
            int tid = omp_get_thread_num();
#else
            int tid = 0;
#endif
            long long lo = tot * tid / nth, hi = tot * (tid + 1) / nth;
            double *a = (double *)malloc(sizeof(double) * nfull);
            double *b = (double *)malloc(sizeof(double) * nfull);
            cplx *F = (cplx *)malloc(sizeof(cplx) * nfull);
            fft2_plan plan;
            int ok = a && b && F && fft2_init(&plan, H, W) == NFSOR_OK;
            if (!ok) {
#pragma omp atomic write
                err = 1;
            }
            int g = 0;
            for (long long q = lo; ok && q < hi; ++q) {
                while (q >= first[g + 1]) ++g;
                int t = (int)(q - first[g]);
                add_pair(s, &plan, t, delays[j0 + g], a, b, F, seg + (size_t)(tid + g) * nhalf);
            }
            if (ok) fft2_free(&plan);
            free(a);
            free(b);
            free(F);
        }
        for (int g = 0; g < ng && !err; ++g) {
            int j = j0 + g;
            /* partials of delay j in thread order (threads whose share overlaps its pairs) */
            for (size_t i = 0; i < nhalf; ++i) P[i] = 0.0;
            for (int th = 0; th < nth; ++th) {
                long long lo = tot * th / nth, hi = tot * (th + 1) / nth;
                if (hi <= first[g] || lo >= first[g + 1]) continue;
                const double *sp = seg + (size_t)(th + g) * nhalf;
                for (size_t i = 0; i < nhalf; ++i) P[i] += sp[i];
            }
            long long npairs = pair_counts[j];
            double inv = npairs ? 1.0 / (double)npairs : 0.0;
            if (D2d)
                for (size_t i = 0; i < nhalf; ++i) D2d[(size_t)j * nhalf + i] = P[i] * inv;
            for (int q = 0; q < nq; ++q) D[(size_t)j * nq + q] = 0.0;
            for (int ky = 0; ky < H; ++ky)
                for (int kx = 0; kx < Wh; ++kx) {
                    int32_t bb = bin[(size_t)ky * Wh + kx];
                    if (bb < 0) continue;
                    int w = (kx == 0 || kx == W / 2) ? 1 : 2;
                    D[(size_t)j * nq + bb] += w * P[(size_t)ky * Wh + kx] * inv;
                }
            for (int q = 0; q < nq; ++q)
                D[(size_t)j * nq + q] = bin_counts[q] ? D[(size_t)j * nq + q] / (double)bin_counts[q] : 0.0;
        }
        free(first);
        free(seg);
        j0 = j1;
    }
    free(bin);
    free(P);
    return err ? NFSOR_ENOMEM : NFSOR_OK;
}

/*
 * Binned structure function D[nd][nq] of N uint16 frames [N][H][W] (row-major), with
 * bin_counts[nq] = C_b, pair_counts[nd] = N - tau_j (0 if negative), q_mean[nq] (may be NULL) and
 * optionally D2d[nd][H][W/2+1] = D(k, tau_j) before binning (may be NULL).
 */
int nfsor_structure_function_u16(const uint16_t *frames, int N, int H, int W, const int32_t *delays, int nd,
                                 int nq, int nthreads, double *D, int64_t *bin_counts, int64_t *pair_counts,
                                 double *q_mean, double *D2d)
{
    if (!frames && N > 0) return NFSOR_EINVAL;
    frame_src s = {frames, NULL, N, H, W, 1};
    return sf_core(&s, delays, nd, nq, nthreads, D, bin_counts, pair_counts, q_mean, D2d);
}

/* Same on FP64 frames; normalize = 0 treats the frames as already-normalised images n_t(x). */
int nfsor_structure_function_f64(const double *frames, int N, int H, int W, int normalize, const int32_t *delays,
                                 int nd, int nq, int nthreads, double *D, int64_t *bin_counts,
                                 int64_t *pair_counts, double *q_mean, double *D2d)
{
    if (!frames && N > 0) return NFSOR_EINVAL;
    frame_src s = {NULL, frames, N, H, W, normalize};
    return sf_core(&s, delays, nd, nq, nthreads, D, bin_counts, pair_counts, q_mean, D2d);
}

/*
 * D(k, tau) at a single mode (kx, ky), kx in [0, W/2], ky in [0, H): the same definition (real-space
 * difference of normalised frames, then its DFT at that one mode), for spot checks of outputs too
 * large for the full oracle.  uint16 frames.
 */
int nfsor_mode_power_u16(const uint16_t *frames, int N, int H, int W, int kx, int ky, int tau, int nthreads,
                         double *out)
{
    if (!frames || !out || H < 2 || W < 2 || kx < 0 || kx > W / 2 || ky < 0 || ky >= H || tau < 0) return NFSOR_EINVAL;
    int npairs = N - tau;
    *out = 0.0;
    if (npairs <= 0) return NFSOR_OK;
    size_t n = (size_t)H * W;
    cplx *ex = (cplx *)malloc(sizeof(cplx) * (size_t)W);
    cplx *ey = (cplx *)malloc(sizeof(cplx) * (size_t)H);
    double *mean = (double *)malloc(sizeof(double) * (size_t)N);
    if (!ex || !ey || !mean) {
        free(ex);
        free(ey);
        free(mean);
        return NFSOR_ENOMEM;
    }
    for (int x = 0; x < W; ++x) {
        double a = 2.0 * M_PI * (double)(((long)kx * x) % W) / (double)W;
        ex[x].re = cos(a);
        ex[x].im = -sin(a);
    }
    for (int y = 0; y < H; ++y) {
        double a = 2.0 * M_PI * (double)(((long)ky * y) % H) / (double)H;
        ey[y].re = cos(a);
        ey[y].im = -sin(a);
    }
    for (int t = 0; t < N; ++t) {
        uint64_t sum = 0;
        const uint16_t *f = frames + (size_t)t * n;
        for (size_t i = 0; i < n; ++i) sum += f[i];
        mean[t] = (double)sum / (double)n;
    }
#ifdef _OPENMP
    int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    int nth = 1;
    (void)nthreads;
#endif
    double *part = (double *)calloc((size_t)nth, sizeof(double));
    if (!part) {
        free(ex);
        free(ey);
        free(mean);
        return NFSOR_ENOMEM;
    }
#pragma omp parallel num_threads(nth)
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
#pragma omp for schedule(static)
        for (int t = 0; t < npairs; ++t) {
            const uint16_t *fa = frames + (size_t)t * n;
            const uint16_t *fb = frames + (size_t)(t + tau) * n;
            double ia = mean[t] != 0.0 ? 1.0 / mean[t] : 0.0;  /* a dark frame normalises to 0 */
            double ib = mean[t + tau] != 0.0 ? 1.0 / mean[t + tau] : 0.0;
            double sr = 0.0, si = 0.0;
            for (int y = 0; y < H; ++y) {
                double rr = 0.0, ri = 0.0;
                for (int x = 0; x < W; ++x) {
                    double d = (double)fa[(size_t)y * W + x] * ia - (double)fb[(size_t)y * W + x] * ib;
                    rr += d * ex[x].re;
                    ri += d * ex[x].im;
                }
                sr += rr * ey[y].re - ri * ey[y].im;
                si += rr * ey[y].im + ri * ey[y].re;
            }
            part[tid] += sr * sr + si * si;
        }
    }
    double acc = 0.0;
    for (int th = 0; th < nth; ++th) acc += part[th];
    *out = acc / (double)npairs;
    free(part);
    free(ex);
    free(ey);
    free(mean);
    return NFSOR_OK;
}

int nfsor_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
