// Delay update of the difference power spectra, the left-hand side of Eq. 1:
//
//   acc[j][k] += sum over new frames t with t >= tau_j of |P_t(k) - P_{t - tau_j}(k)|^2
//
// where P_t is the spectrum of frame t held in ring slot t mod R.  By linearity P_t - P_s is the
// transform of the real-space difference n_t - n_s, so each pair costs one complex subtraction
// and a squared modulus per mode instead of a transform ("only the square moduli of FFT
// differences" of the processing paragraph).  Averaging over t at fixed tau is the time average
// that stands for the ensemble average of Eq. 1 for stationary dynamics.
//
// Tiled kernel (variant 0).  One CTA owns a tile of 16 consecutive modes for a block of K = 512
// new frames; 16 warps each take 32 consecutive frames, a half-warp 16 of them (lane = mode + 16 x
// half), holding those 16 spectra in registers.  Delays are taken in order as runs of consecutive
// values ("sub-runs" of up to 16): for a run starting at d0 a lane keeps the 16 older values
// P_{t-d0} .. in a register window and slides it back one frame per delay, so one shared-memory
// load serves 16 pairs; an isolated delay costs one load per pair.  The tile's slots (128 bytes:
// 16 modes) stream newest-to-oldest through a 1024-slot ring in shared memory, filled by bulk
// asynchronous copies (TMA, cp.async.bulk) that complete on mbarriers, one copy group per stage,
// later stages' groups issued while earlier ones compute as far as the ring's rows allow (16-mode
// slots give twice the rows of 32-mode ones in the same memory, hence the deeper prefetch that the
// stages of sparse large delays need).  Per-lane partial sums go through shared memory, are added
// in a fixed order and then into the Kahan (sum, compensation) pair of the accumulator.
#include <algorithm>
#include <cmath>

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

// ------------------------------------------------------------------ schedule (host)

bool build_delay_schedule(const int *delays, int nd, bool cross, std::vector<SubRun> *srs, std::vector<Stage> *sts,
                          int span)
{
    if (span < kMinSpan || span > kMaxSpan) return false;
    srs->clear();
    sts->clear();
    int j = 0;
    // tau = 0 pairs a frame with itself: D = 0 exactly (in a cross pass it pairs two different frames)
    if (!cross)
        while (j < nd && delays[j] == 0) ++j;
    while (j < nd) {
        const int j0 = j, d0 = delays[j];
        int len = 1;
        while (j0 + len < nd && len < 16 && delays[j0 + len] == d0 + len) ++len;
        srs->push_back({j0, len, d0});
        j = j0 + len;
    }
    // SPAN: the widest delay range of one stage (measured on GB300 with K = 512 and 1024 slot
    // rows and one writer warp: 240 ran the 200 log delays 1..2000 2 % faster than 112 and sparse
    // delays 64 apart 9 % faster; 320 and more slowed both, their copy groups leaving too few free
    // rows to prefetch).  The default; a context may measure the best span for its own delay list
    // (NFS_OPT_DELAY_SPAN = 0).  The span groups sub-runs into copy stages only: the pair
    // arithmetic and the batches of partial sums, so the results, do not depend on it.
    const int K = kDelayBlock, SB = kSlotBuf, SPAN = span;
    // needed frame range of every consumer step, relative to t0: step 0 reads the block itself
    std::vector<int> need_lo(1, 0), need_hi(1, K - 1);
    // frames t0 + lo_prev .. are in the buffer after the block is loaded (a cross pass's block is
    // made of other frames than the older sequence it is paired with: none of those are loaded)
    int lo_prev = cross ? K : 0;
    size_t r = 0;
    while (r < srs->size()) {
        Stage st;
        st.sr0 = (int)r;
        const int dmin = (*srs)[r].d0;
        int dmax = dmin + (*srs)[r].len - 1;
        size_t e = r + 1;
        while (e < srs->size() && (*srs)[e].d0 + (*srs)[e].len - 1 - dmin <= SPAN) {
            dmax = (*srs)[e].d0 + (*srs)[e].len - 1;
            ++e;
        }
        st.nsr = (int)(e - r);
        // load only what this stage needs and is not loaded yet (a large first delay or a large gap
        // must not pull in unneeded frames: a group never exceeds K + SPAN slots)
        st.lo = -dmax;
        st.hi = std::min(lo_prev - 1, K - 1 - dmin);
        if (K + dmax - dmin > SB) return false;  // cannot happen: K + SPAN <= SB
        if (st.lo <= st.hi) lo_prev = st.lo;
        need_lo.push_back(-dmax);
        need_hi.push_back(K - 1 - dmin);
        sts->push_back(st);
        r = e;
    }
    // When may the group of stage s (group g = s + 1, consumed by step g) be issued?  Its rows of the
    // slot ring must no longer hold frames a pending step reads (a frame f sits in row f mod SB), and
    // the mbarrier it reuses (group g - kFullBars, consumed by step g - kFullBars) must have been
    // observed by every consumer.
    for (size_t s = 0; s < sts->size(); ++s) {
        Stage &st = (*sts)[s];
        const int g = (int)s + 1;
        int need = std::max(0, g - kFullBars + 1);
        if (st.lo <= st.hi) {
            for (int q = g - 1; q >= 0; --q) {  // latest earlier step that reads a row the group overwrites
                // frames f in [lo, hi] and h in [need_lo, need_hi] share a row iff h = f + k SB, k != 0
                // (k = 0 too against a cross pass's block: the same index there is another frame)
                bool clash = false;
                const int a = st.lo, b = st.hi, c = need_lo[q], d = need_hi[q];
                const int kmin = (int)std::floor((double)(c - b) / SB), kmax = (int)std::ceil((double)(d - a) / SB);
                for (int k = kmin; k <= kmax && !clash; ++k)
                    if ((k != 0 || (cross && q == 0)) && std::max(a, c - k * SB) <= std::min(b, d - k * SB)) clash = true;
                if (clash) {
                    need = std::max(need, q + 1);
                    break;
                }
            }
        }
        if (need > g) return false;  // the step that needs this group would wait for itself
        st.need = need;
    }
    return true;
}

// Sub-runs are packed into batches of at most 16 delays in schedule order (a sub-run never splits).
int count_delay_batches(const std::vector<SubRun> &srs)
{
    int n = 0, pend = 0;
    for (const SubRun &sr : srs) {
        if (pend + sr.len > 16) {
            ++n;
            pend = 0;
        }
        pend += sr.len;
    }
    return n + (pend ? 1 : 0);
}

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ cycle accounting (measuring build)

// With NFS_DELAY_PROFILE defined (buildlib.build(profile=True)) the tiled kernel adds each warp
// role's clock64 cycles by phase into g_delay_prof (lane 0 of each warp; read and cleared through
// nfs_delay_profile); otherwise the accounting compiles to nothing.
enum DelayProf {
    kProfConsumer,      // consumer warps: from the first copy-group wait to the last hand-over
    kProfConsWaitGroup, //   waiting for copy groups
    kProfConsWaitFree,  //   waiting for a free partial-sum buffer
    kProfConsCompute,   //   pair arithmetic of the sub-runs
    kProfConsHand,      //   step and batch hand-overs
    kProfWriter,        // writer warp: whole tile
    kProfWriterWait,    //   waiting for written batches
    kProfProducerWait,  // producer lane: waiting for free slot-ring rows
    kProfPrologue,      // thread 0: barrier set-up to the first synchronisation
    kProfEpilogue,      // thread 0: final synchronisation and barrier invalidation
    kProfTiles,         // tile passes counted
    kProfSlots
};
#ifdef NFS_DELAY_PROFILE
__device__ unsigned long long g_delay_prof[kProfSlots];
#define NFS_PROF(x) x
#else
#define NFS_PROF(x)
#endif

// ------------------------------------------------------------------ tiled kernel

constexpr int kWarps = 16;                       // consumer warps (32 frames each: 16 per half-warp)
constexpr int kTw = 16;                          // consecutive frames per lane (a half-warp's run)
constexpr int kProducer = kWarps;                // warp that issues the copy groups
constexpr int kWriter = kWarps + 1;              // first of the warps that reduce partial sums into the
constexpr int kWriters = 2;                      // accumulators (writer i takes the batches k = i mod 2)
constexpr int kThreads = (kWarps + 1 + kWriters) * 32;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
static_assert(kWarps * 2 * kTw == kDelayBlock, "block = warps x half-warps x frames per lane");
static_assert(kTile == 16, "a half-warp covers one tile: lane = mode + 16 x half");

constexpr int kRedBufs = 3;                      // partial-sum buffers: the writer may lag two batches
constexpr int kRedStride = kWarps * 32;          // words per delay slot of a buffer

struct TiledSmem {
    float2 buf[kSlotBuf][kTile];            // slot ring: frame s at row s mod kSlotBuf (128-byte rows)
    float red[kRedBufs][16][kRedStride];     // per-lane partial sums of a batch of up to 16 delays
    unsigned long long full[kFullBars];      // copy-group barriers (group g on full[g % kFullBars])
    unsigned long long red_full[kRedBufs];   // batch k (buffer k % 3) written by all consumer warps
    unsigned long long red_free[kRedBufs];   // batch k drained by the writer
    int done;                              // consumer-warp step completions, all warps (diagnostics)
    int abort;                             // set when a bounded wait gives up
    int wsteps[kWarps];                    // per consumer warp: steps completed (the producer waits for
                                           // the minimum: a sum would let fast warps count for a slow one)
    int wbatches[kWarps];                  // per consumer warp: batches handed over (diagnostics)
    int wdrained;                          // batches the writers have drained (diagnostics)
};

// err[0] = 1 once any wait of the launch gives up; the first thread to give up records in err[1..]
// which wait it was: kind (1 copy group, 2 batch written, 3 batch drained, 4 producer progress),
// CTA, warp, group or batch index, polls, globaltimer ns and clock64 cycles spent (low 31 bits
// of each, saturated), and the CTA's progress counter.
__device__ __forceinline__ void set_abort(TiledSmem &S, int *err, int kind, int index, long long polls,
                                          unsigned long long ns, long long cycles)
{
    *(volatile int *)&S.abort = 1;
    if (atomicCAS(err + 1, 0, kind) == 0) {
        err[2] = (int)blockIdx.x;
        err[3] = (int)(threadIdx.x >> 5);
        err[4] = index;
        err[5] = (int)(polls > 0x7fffffffLL ? 0x7fffffffLL : polls);
        err[6] = (int)(ns > 0x7fffffffull ? 0x7fffffffull : ns);
        err[7] = (int)(cycles > 0x7fffffffLL ? 0x7fffffffLL : cycles);
        err[8] = *(volatile int *)&S.done;
        err[9] = *(volatile int *)&S.wdrained;
        for (int w = 0; w < kWarps; ++w) {
            err[10 + w] = ((volatile int *)S.wsteps)[w];
            err[10 + kWarps + w] = ((volatile int *)S.wbatches)[w];
        }
    }
    __threadfence();
    atomicExch(err, 1);
}
constexpr long long kMinPolls = 100000;  // a wait gives up only after this many polls AND the time limit

// Wait for a phase of an mbarrier (bounded; returns at once once any thread of the launch has
// given up).
__device__ __forceinline__ bool wait_bar(TiledSmem &S, unsigned long long *bar, unsigned par, int *err, int kind,
                                         int index)
{
    if (mbar_try_wait(bar, par)) return true;
    const unsigned long long t0 = global_ns();
    const long long c0 = clock64();
    long long polls = 0;
    while (!mbar_try_wait(bar, par)) {
        // give up at once when this CTA or any other CTA of the launch has given up
        if (*(volatile int *)&S.abort || *(volatile int *)err) return false;
        ++polls;
        const unsigned long long dt = global_ns() - t0;
        if (polls > kMinPolls && dt > kWaitLimitNs) {
            set_abort(S, err, kind, index, polls, dt, clock64() - c0);
            return false;
        }
    }
    return true;
}

// Wait for copy group g.
__device__ __forceinline__ bool wait_group(TiledSmem &S, int g, int *err)
{
    return wait_bar(S, &S.full[g % kFullBars], (unsigned)((g / kFullBars) & 1), err, 1, g);
}

// Issue the bulk copies of frames t0+lo .. t0+hi of this tile into the slot ring (producer lane).
__device__ __forceinline__ void issue_group(TiledSmem &S, const float2 *__restrict__ ring, int R, size_t tile,
                                            long long t0, int lo, int hi, unsigned long long *bar)
{
    const long long a0 = t0 + lo, b = t0 + hi;
    const unsigned bytes = (lo <= hi) ? (unsigned)((hi - lo + 1) * kTile * sizeof(float2)) : 0u;
    mbar_expect_tx(bar, bytes);
    long long a = a0;
    while (a <= b) {
        const int rs = (int)(((a % R) + R) % R);
        const int bp = (int)(a & (kSlotBuf - 1));
        long long n = b - a + 1;
        n = n < (long long)(R - rs) ? n : (long long)(R - rs);
        n = n < (long long)(kSlotBuf - bp) ? n : (long long)(kSlotBuf - bp);
        bulk_g2s(&S.buf[bp][0], ring + ((tile * (size_t)R + (size_t)rs) * kTile), (unsigned)(n * kTile * sizeof(float2)),
                 bar);
        a += n;
    }
}

// A consumer warp has finished reading the slot ring for one step.
__device__ __forceinline__ void step_done(TiledSmem &S, int lane)
{
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        ++((volatile int *)S.wsteps)[threadIdx.x >> 5];
        atomicAdd(&S.done, 1);
    }
}

// Steps completed by every consumer warp.
__device__ __forceinline__ int min_steps(TiledSmem &S)
{
    int m = 0x7fffffff;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) m = min(m, ((volatile int *)S.wsteps)[w]);
    return m;
}

// Packed FP32 pairs (Blackwell f32x2 arithmetic): a complex value is one 64-bit register
// {re, im}; the difference and the squared-modulus accumulation are one instruction each.
typedef unsigned long long pk_t;
__device__ __forceinline__ pk_t psub(pk_t a, pk_t b)
{
    pk_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ pk_t psq_acc(pk_t d, pk_t acc)  // acc + {d.re^2, d.im^2}
{
    pk_t r;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(d), "l"(acc));
    return r;
}
__device__ __forceinline__ pk_t padd(pk_t a, pk_t b)
{
    pk_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ float phsum(pk_t a)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
    return lo + hi;
}

// One sub-run of consecutive delays d0 .. d0+len-1 for the warp's frames ta .. ta+15, with
// base = ta - d0: the pair (ta + i, d0 + u) reads frame base + i - u.  The window holds the 16
// older values of the current delay; moving to the next delay drops the newest and loads one
// older frame.  MASKED: drop pairs whose older frame is < 0 or whose new frame lies past the
// block (i >= hi_lim).  WRAP: the 31 slot rows touched wrap around the slot ring, so every
// address is taken modulo; otherwise they are immediate offsets from one base address.
__device__ __forceinline__ float2 unpk(pk_t a)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(a));
    return v;
}

// Where a consumer lane leaves its partial sum in a batch row: the two half-warps' values of one
// mode side by side, so the writer reads both with one 8-byte load.
__device__ __forceinline__ int red_slot(int warp, int lane) { return warp * 32 + 2 * (lane & (kTile - 1)) + (lane >> 4); }

template <bool MASKED, bool WRAP, bool PACKED>
__device__ __forceinline__ void subrun(TiledSmem &S, const pk_t (&xt)[kTw], int lane, int warp, int base, int len,
                                       float (*red)[kRedStride], int pend, int hi_lim)
{
    const float2 *col = &S.buf[0][lane & (kTile - 1)];
    const float2 *p0 = col + (size_t)((base & (kSlotBuf - 1)) * kTile);
    const int ri = red_slot(warp, lane);
    auto ldf = [&](int off) -> pk_t {  // the value of frame base + off
        const float2 *a = WRAP ? col + (size_t)(((base + off) & (kSlotBuf - 1)) * kTile) : p0 + off * kTile;
        return *reinterpret_cast<const pk_t *>(a);
    };
    pk_t w[kTw];
#pragma unroll
    for (int i = 0; i < kTw; ++i) w[i] = ldf(i);
#pragma unroll
    for (int uu = 0; uu < 16; ++uu) {
        if (uu >= len) break;
        if (PACKED) {
            pk_t a[2] = {0ull, 0ull};
#pragma unroll
            for (int i = 0; i < kTw; ++i) {
                pk_t d = psub(xt[i], w[(i - uu) & (kTw - 1)]);
                if (MASKED) {
                    const bool v = (i - uu >= -base) && (i < hi_lim);
                    d = v ? d : 0ull;
                }
                a[i & 1] = psq_acc(d, a[i & 1]);
            }
            red[pend + uu][ri] = phsum(padd(a[0], a[1]));
        } else {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < kTw; ++i) {
                const float2 x = unpk(xt[i]), y = unpk(w[(i - uu) & (kTw - 1)]);
                float dr = x.x - y.x, di = x.y - y.y;
                if (MASKED) {
                    const bool v = (i - uu >= -base) && (i < hi_lim);
                    dr = v ? dr : 0.f;
                    di = v ? di : 0.f;
                }
                a[i & 3] = fmaf(dr, dr, a[i & 3]);
                a[i & 3] = fmaf(di, di, a[i & 3]);
            }
            red[pend + uu][ri] = (a[0] + a[1]) + (a[2] + a[3]);
        }
        if (uu + 1 < len) w[(kTw - 1 - uu) & (kTw - 1)] = ldf(-uu - 1);
    }
}

// Picks the sub-run variant for this warp (the choice is uniform within the warp).  Half-warp h
// holds frames taw + 16 h .. taw + 16 h + 15 (ta: this lane's first frame, hi_lim: its count of
// new frames); the conditions below hold for both halves at once.
template <bool PACKED>
__device__ __forceinline__ void subrun_dispatch(TiledSmem &S, const pk_t (&xt)[kTw], int lane, int warp, int taw,
                                                int ta, int d0, int len, float (*red)[kRedStride], int pend,
                                                int hi_lim, int hi_lim_w)
{
    const int base = ta - d0, basew = taw - d0;
    if (hi_lim_w <= 0 || basew + 2 * kTw - 1 < 0) {  // no pair of this warp is valid
        for (int u = 0; u < len; ++u) red[pend + u][red_slot(warp, lane)] = 0.f;
        return;
    }
    if (basew - (len - 1) >= 0 && hi_lim_w >= 2 * kTw) {
        const int r0 = basew & (kSlotBuf - 1);  // rows r0 - 15 .. r0 + 31 of both halves, unwrapped
        if (r0 >= 16 && r0 + 2 * kTw - 1 < kSlotBuf)
            subrun<false, false, PACKED>(S, xt, lane, warp, base, len, red, pend, hi_lim);
        else
            subrun<false, true, PACKED>(S, xt, lane, warp, base, len, red, pend, hi_lim);
    } else {
        subrun<true, true, PACKED>(S, xt, lane, warp, base, len, red, pend, hi_lim);
    }
}

// Consumer side of a batch hand-over: this warp's partial sums of batch b are written.
__device__ __forceinline__ void hand_over(TiledSmem &S, int b, int lane)
{
    __syncwarp();
    if (lane == 0) {
        mbar_arrive(&S.red_full[b]);
        ++((volatile int *)S.wbatches)[threadIdx.x >> 5];
    }
}

__device__ __forceinline__ void mbar_inval(unsigned long long *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One CTA's pass over one 16-mode tile for a block of new frames t0 .. t0+nb-1 (all warps of the
// CTA take part; every role falls through to the final barrier, so a persistent caller can run
// several tiles in a row).  sched: the sequence's schedule (kernel parameters or global memory);
// nst, nbatch: its stages and batches for this block (early blocks leave late stages out).
template <bool PACKED>
__device__ __forceinline__ void tile_pass(TiledSmem &S, const float2 *__restrict__ ring, int R, size_t M,
                                          long long t0, int nb, const DelaySchedule &sched, int nst, int nbatch,
                                          float2 *__restrict__ acc, int nd, int *__restrict__ err, int stall_group,
                                          size_t tile, const float2 *__restrict__ ring_cur = nullptr, int R_cur = 0)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    NFS_PROF(long long pf_t0 = clock64(); long long pf[kProfSlots] = {};)

    if (tid == 0) {
        for (int b = 0; b < kFullBars; ++b) mbar_init(&S.full[b], 1);
        for (int b = 0; b < kRedBufs; ++b) {
            mbar_init(&S.red_full[b], kWarps);
            mbar_init(&S.red_free[b], 1);
        }
        S.done = 0;
        S.abort = 0;
        S.wdrained = 0;
        for (int w = 0; w < kWarps; ++w) S.wsteps[w] = S.wbatches[w] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    NFS_PROF(if (tid == 0) pf[kProfPrologue] += clock64() - pf_t0;)

    if (warp == kProducer) {
        // issue every copy group as soon as its rows are free and its barrier is reusable
        if (lane == 0) {
            int issued = 0;
            for (int g = 0; g <= nst; ++g) {
                // test hook: issue nothing from group stall_group on (every group issued before it
                // is consumed before the consumers reach it, so no copy is left in flight)
                if (g == stall_group) break;
                const int need = (g == 0) ? 0 : sched.st[g - 1].need;
                bool ok = true;
                NFS_PROF(const long long pw0 = clock64();)
                if (min_steps(S) < need) {
                    const unsigned long long tw = global_ns();
                    const long long c0 = clock64();
                    long long polls = 0;
                    while (min_steps(S) < need) {
                        if (*(volatile int *)&S.abort || *(volatile int *)err) {
                            ok = false;
                            break;
                        }
                        ++polls;
                        const unsigned long long dt = global_ns() - tw;
                        if (polls > kMinPolls && dt > kWaitLimitNs) {
                            set_abort(S, err, 4, g, polls, dt, clock64() - c0);
                            ok = false;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                NFS_PROF(pf[kProfProducerWait] += clock64() - pw0;)
                if (!ok) break;
                __threadfence_block();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (g == 0)  // the block's own frames (in a cross pass: from the other sequence's ring)
                    issue_group(S, ring_cur ? ring_cur : ring, ring_cur ? R_cur : R, tile, t0, 0, kDelayBlock - 1,
                                &S.full[0]);
                else
                    issue_group(S, ring, R, tile, t0, sched.st[g - 1].lo, sched.st[g - 1].hi, &S.full[g % kFullBars]);
                issued = g + 1;
            }
            if (*(volatile int *)&S.abort || *(volatile int *)err) {
                // let copies still in flight land (bounded) before the shared memory is reused
                for (int g = issued - 1; g >= 0 && g >= issued - kFullBars; --g) {
                    unsigned long long *bar = &S.full[g % kFullBars];
                    const unsigned par = (unsigned)((g / kFullBars) & 1);
                    const unsigned long long tw = global_ns();
                    while (!mbar_try_wait(bar, par) && global_ns() - tw < kWaitLimitNs / 20) {
                    }
                }
            }
        }
    } else if (warp >= kWriter) {
        // Reduce each batch over the consumer warps in a fixed order and add it to the Kahan pairs.
        // A batch is the longest run of consecutive sub-runs with at most 16 delays (the consumers'
        // rule), so the writers take every batch's delays from the schedule; writer wi handles the
        // batches k = wi mod kWriters (different delays: no two writers touch one accumulator).  A
        // writer waits for batch k only after its batch k - kWriters, so every batch before k - 1
        // is written and the buffer's mbarrier is in batch k's phase (no parity aliasing).  (Loading
        // the next batch's accumulators right after releasing a buffer measured slower on runs of
        // consecutive delays than loading them once the batch is written.)
        // lane = mode + 16 h: half h adds the batch's delays 8 h .. 8 h + 7 at its mode.
        const int wi = warp - kWriter;
        const int m = lane & (kTile - 1), jh = (lane >> 4) * 8;
        float2 *const base = acc + tile * kTile + m;
        const int nsr = nst > 0 ? sched.st[nst - 1].sr0 + sched.st[nst - 1].nsr : 0;
        int r = 0, jb = 0, n = 0;
        auto next_batch = [&]() {  // the delays jb .. jb+n-1 of the batch starting at sub-run r
            jb = sched.sr[r].j0;
            n = 0;
            while (r < nsr && n + sched.sr[r].len <= 16) n += sched.sr[r++].len;
        };
        float2 old[8];
        auto load_old = [&]() {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (jh + q < n && (unsigned)(jb + jh + q) < (unsigned)nd) old[q] = base[(size_t)(jb + jh + q) * M];
        };
        NFS_PROF(const long long pwr = clock64();)
        for (int k = 0; k < nbatch; ++k) {
            const int b = k % kRedBufs;
            if (r < nsr) next_batch();
            if (k % kWriters != wi) continue;
            // After a failed wait the batch may not be written yet: stop touching global memory
            // (the launch's results are void and the error word says so).
            NFS_PROF(const long long pww = clock64();)
            if (!wait_bar(S, &S.red_full[b], (unsigned)((k / kRedBufs) & 1), err, 2, k)) break;
            NFS_PROF(pf[kProfWriterWait] += clock64() - pww;)
            load_old();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (jh + q < n && (unsigned)(jb + jh + q) < (unsigned)nd) {
                    const pk_t *row = reinterpret_cast<const pk_t *>(S.red[b][jh + q]) + m;
                    pk_t s0 = 0ull, s1 = 0ull;  // {half 0, half 1} sums over even and odd warps
#pragma unroll
                    for (int w = 0; w < kWarps; w += 2) {
                        s0 = padd(s0, row[w * 16]);
                        s1 = padd(s1, row[w * 16 + 16]);
                    }
                    base[(size_t)(jb + jh + q) * M] = kahan_add(old[q], phsum(padd(s0, s1)));
                }
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&S.red_free[b]);
                *(volatile int *)&S.wdrained = k + 1;
            }
        }
        NFS_PROF(pf[kProfWriter] += clock64() - pwr;)
    } else {
        // consumers
        const int taw = (int)(t0 + (long long)warp * 2 * kTw);  // first frame of this warp (indices < 2^31)
        const int ta = taw + (lane >> 4) * kTw;                 // first frame of this lane's half-warp
        const int hi_lim = (int)(t0 + nb - ta);                 // frames ta + i are new frames for i < hi_lim
        const int hi_lim_w = (int)(t0 + nb - taw);
        NFS_PROF(const long long pc0 = clock64(); long long pq = pc0;)
        wait_group(S, 0, err);
        NFS_PROF(pf[kProfConsWaitGroup] += clock64() - pq;)
        pk_t xt[kTw];
#pragma unroll
        for (int i = 0; i < kTw; ++i)
            xt[i] = *reinterpret_cast<const pk_t *>(&S.buf[(ta + i) & (kSlotBuf - 1)][lane & (kTile - 1)]);
        step_done(S, lane);

        // After a failed wait the loop still runs to the end (every shared-memory index stays in
        // bounds, the numbers are wrong and the error word says so), so no barrier loses a warp.
        int pend = 0, batch = 0;
        auto open_batch = [&](int k) {  // before writing batch k: the writer has drained batch k - 3
            if (k >= kRedBufs)
                wait_bar(S, &S.red_free[k % kRedBufs], (unsigned)(((k - kRedBufs) / kRedBufs) & 1), err, 3, k);
        };
        open_batch(0);
        for (int s = 0; s < nst; ++s) {
            const Stage st = sched.st[s];
            NFS_PROF(pq = clock64();)
            wait_group(S, s + 1, err);
            NFS_PROF(pf[kProfConsWaitGroup] += clock64() - pq;)
            for (int r = st.sr0; r < st.sr0 + st.nsr; ++r) {
                const SubRun sr = sched.sr[r];
                if (pend + sr.len > 16) {
                    NFS_PROF(pq = clock64();)
                    hand_over(S, batch % kRedBufs, lane);
                    ++batch;
                    pend = 0;
                    NFS_PROF(long long pq2 = clock64(); pf[kProfConsHand] += pq2 - pq;)
                    open_batch(batch);
                    NFS_PROF(pf[kProfConsWaitFree] += clock64() - pq2;)
                }
                NFS_PROF(pq = clock64();)
                subrun_dispatch<PACKED>(S, xt, lane, warp, taw, ta, sr.d0, sr.len, S.red[batch % kRedBufs], pend, hi_lim,
                                        hi_lim_w);
                NFS_PROF(pf[kProfConsCompute] += clock64() - pq;)
                pend += sr.len;
            }
            NFS_PROF(pq = clock64();)
            step_done(S, lane);
            NFS_PROF(pf[kProfConsHand] += clock64() - pq;)
        }
        if (pend) {
            hand_over(S, batch % kRedBufs, lane);
        }
        NFS_PROF(pf[kProfConsumer] += clock64() - pc0;)
    }
    NFS_PROF(const long long pe0 = clock64();)
    __syncthreads();  // every role has finished this tile (all copies issued were consumed)
    if (tid == 0) {
        for (int b = 0; b < kFullBars; ++b) mbar_inval(&S.full[b]);
        for (int b = 0; b < kRedBufs; ++b) {
            mbar_inval(&S.red_full[b]);
            mbar_inval(&S.red_free[b]);
        }
    }
    __syncthreads();
#ifdef NFS_DELAY_PROFILE
    if (tid == 0) {
        pf[kProfEpilogue] += clock64() - pe0;
        pf[kProfTiles] += 1;
    }
    if (lane == 0)
        for (int q = 0; q < kProfSlots; ++q)
            if (pf[q]) atomicAdd(&g_delay_prof[q], (unsigned long long)pf[q]);
#endif
}

template <bool PACKED>
__global__ void __launch_bounds__(kThreads, 1) k_delay_f32_tiled(const float2 *__restrict__ ring, int R, size_t M,
                                                                 long long t0, int nb,
                                                                 const __grid_constant__ DelaySchedule sched,
                                                                 float2 *__restrict__ acc, int nd,
                                                                 int *__restrict__ err, int stall_group,
                                                                 const float2 *__restrict__ ring_cur, int R_cur,
                                                                 const int *__restrict__ tiles)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TiledSmem &S = *reinterpret_cast<TiledSmem *>(smem_raw);
    const size_t tile = tiles ? (size_t)tiles[blockIdx.x] : (size_t)blockIdx.x;
    tile_pass<PACKED>(S, ring, R, M, t0, nb, sched, sched.nst, sched.nbatch, acc, nd, err, stall_group, tile,
                      ring_cur, R_cur);
}

// Ragged batch: one persistent launch over the tiles of several sequences (each with its own frame
// shape, ring, accumulators and schedule); CTA b takes work items b, b + gridDim.x, ...
template <bool PACKED>
__global__ void __launch_bounds__(kThreads, 1) k_delay_f32_batched(const BatchItem *__restrict__ items, int nitems,
                                                                   long long total_tiles, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TiledSmem &S = *reinterpret_cast<TiledSmem *>(smem_raw);
    for (long long i = blockIdx.x; i < total_tiles; i += gridDim.x) {
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].first <= i)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchItem it = items[lo];
        const size_t tile = it.tiles ? (size_t)it.tiles[i - it.first] : (size_t)(i - it.first);
        tile_pass<PACKED>(S, it.ring, it.R, it.M, it.t0, it.nb, *it.sched, it.nst, it.nbatch, it.acc, it.nd, err, -1,
                          tile);
    }
}

cudaError_t launch_delay_batched(const BatchItem *d_items, int nitems, long long total_tiles, int *err, int n_sm,
                                 cudaStream_t s)
{
    if (nitems <= 0 || total_tiles <= 0) return cudaSuccess;
    const size_t smem = sizeof(TiledSmem);
    cudaError_t e = cudaFuncSetAttribute(k_delay_f32_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = total_tiles < (long long)n_sm ? total_tiles : (long long)n_sm;
    k_delay_f32_batched<true><<<(unsigned)grid, kThreads, smem, s>>>(d_items, nitems, total_tiles, err);
    return cudaGetLastError();
}

// Stages and batches of a block whose last frame is tlast (stages whose smallest delay exceeds it
// have no valid pair yet).
void truncate_schedule(const DelaySchedule &sc, long long tlast, int *nst_out, int *nbatch_out)
{
    int nst = 0;
    while (nst < sc.nst && (long long)sc.sr[sc.st[nst].sr0].d0 <= tlast) ++nst;
    int nb_batches = 0, pend = 0;
    if (nst > 0)
        for (int r = 0; r < sc.st[nst - 1].sr0 + sc.st[nst - 1].nsr; ++r) {
            if (pend + sc.sr[r].len > 16) {
                ++nb_batches;
                pend = 0;
            }
            pend += sc.sr[r].len;
        }
    *nst_out = nst;
    *nbatch_out = nb_batches + (pend ? 1 : 0);
}

// ------------------------------------------------------------------ simple block kernel (variant 1)

// One thread per mode: the block's spectra stay in registers, each delay adds a plain FP32 block
// partial into a Kahan pair.  Used for blocks of up to 32 frames and as a cross-check.
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
            x[i] = ring[ring_index(sl, k, R)];
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
                const float2 y = ring[ring_index(sl, k, R)];
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
    if (a.nb <= 0) return cudaSuccess;
    if (a.ring_cur && (variant == 1 || !a.sched)) return cudaErrorNotSupported;  // cross passes: tiled only
    if (variant == 1 || !a.sched) {
        // simple kernel, in sub-blocks of up to 32 frames (all frames of the block are in the ring)
        for (int o = 0; o < a.nb; o += kBlockMax) {
            const int nb = std::min(kBlockMax, a.nb - o);
            const long long t0 = a.t0 + o;
            const int base = (int)(t0 % a.R);
            const unsigned grid = (unsigned)((a.M + 255) / 256);
            k_delay_f32_block<kBlockMax><<<grid, 256, 0, s>>>(a.ring, a.R, a.M, base, t0, nb, a.delays, a.nd, a.acc);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (a.nb > kDelayBlock || (a.M % kTile) != 0) return cudaErrorInvalidValue;
    // Stages whose smallest delay exceeds the block's last frame have no valid pair yet (early
    // blocks of a sequence): leave them out of this launch, with the batches they would fill.
    DelaySchedule sc = *a.sched;
    int nst = 0, nbatch = 0;
    truncate_schedule(sc, a.t0 + a.nb - 1, &nst, &nbatch);
    if (nst == 0) return cudaSuccess;  // nothing to add (or only tau = 0 in the list)
    sc.nst = nst;
    sc.nbatch = nbatch;
    const size_t smem = sizeof(TiledSmem);
    const unsigned grid = (unsigned)(a.tiles ? a.ntiles : a.M / kTile);
    if (grid == 0) return cudaSuccess;
    if (variant == 2) {
        cudaError_t e = cudaFuncSetAttribute(k_delay_f32_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_delay_f32_tiled<false><<<grid, kThreads, smem, s>>>(a.ring, a.R, a.M, a.t0, a.nb, sc, a.acc, a.nd, a.err,
                                                               a.stall_group, a.ring_cur, a.R_cur, a.tiles);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_delay_f32_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_delay_f32_tiled<true><<<grid, kThreads, smem, s>>>(a.ring, a.R, a.M, a.t0, a.nb, sc, a.acc, a.nd, a.err,
                                                              a.stall_group, a.ring_cur, a.R_cur, a.tiles);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ plain FP64 path

// One frame t per launch, FP64 accumulators, no blocking; slot-major ring [R][M].
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

// The delay kernel's cycle accounting (a measuring build only): out[0 .. n) = the kProfSlots sums
// (see DelayProf), cleared afterwards when reset != 0.
extern "C" int nfs_delay_profile(unsigned long long *out, int n, int reset)
{
#ifdef NFS_DELAY_PROFILE
    if (!out || n < 0) return NFS_EINVAL;
    unsigned long long h[nfs::kProfSlots] = {};
    if (cudaMemcpyFromSymbol(h, nfs::g_delay_prof, sizeof(h)) != cudaSuccess) return NFS_ECUDA;
    for (int i = 0; i < n && i < nfs::kProfSlots; ++i) out[i] = h[i];
    if (reset) {
        const unsigned long long z[nfs::kProfSlots] = {};
        if (cudaMemcpyToSymbol(nfs::g_delay_prof, z, sizeof(z)) != cudaSuccess) return NFS_ECUDA;
    }
    return nfs::kProfSlots;
#else
    (void)out;
    (void)n;
    (void)reset;
    return NFS_EUNSUPPORTED;
#endif
}
