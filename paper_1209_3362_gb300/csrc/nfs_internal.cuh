// Internal declarations shared by the CUDA translation units of the NFS library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nfs.h"

namespace nfs {

template <typename T>
struct cplx_t;
template <>
struct cplx_t<float> {
    using type = float2;
};
template <>
struct cplx_t<double> {
    using type = double2;
};

// FFT plan of one transform length: radices in stage order and the twiddle table
// tw[m] = exp(-2 pi i m / L), m < L (built in FP64 on the host).
constexpr int kMaxStages = 16;
struct FftPlan {
    int L = 0;
    int nstages = 0;
    int radix[kMaxStages] = {};
};

bool make_plan(int L, FftPlan *plan);  // false if L has a prime factor other than 2 or 3

// One device-side description of the frame geometry.
//
// Mode order of a spectrum in HBM (the flat index k the delay update and the binning use):
//   column-major (FP32 path):  k = kx * H + ky,  kx < W/2+1, ky < H   (M = H (W/2+1) rounded up to 32)
//   row-major    (FP64 path):  k = ky * Wp + kx, kx < Wp (pitch)      (M = H Wp rounded up to 32)
// The FP32 row pass writes a column-pair scratch [kx/2][ky][kx%2] (Wp columns) that the column
// pass reads as contiguous runs of 2 columns.
struct Geometry {
    int H, W;      // frame size
    int Lr;        // row transform length W/2
    int Wh;        // W/2 + 1 non-redundant columns
    int Wp;        // W/2 + 1 rounded up to a multiple of 4 (row pitch / scratch columns)
    size_t M;      // complex values per spectrum held (multiple of 16; a slab's share, see k0)
    size_t HW;     // pixels per frame
    int colmajor;  // 1: column-major mode order (FP32), 0: row-major with pitch Wp (FP64)
    // Mode slab (FP32 path): the spectrum ring and accumulators hold modes k0 .. k0+M-1 of the
    // column-major order, at local index k - k0; the column pass transforms column pairs
    // kp0 .. kp0+ncp-1 only.  The whole spectrum: k0 = 0, kp0 = 0, ncp = Wp/2.
    size_t k0;
    int kp0, ncp;
    __host__ __device__ size_t mode(int kx, int ky) const
    {
        return colmajor ? (size_t)kx * H + ky : (size_t)ky * Wp + kx;
    }
    __host__ __device__ size_t scratch_index(int kx, int ky) const  // FP32 column-pair scratch
    {
        return ((size_t)(kx >> 1) * H + ky) * 2 + (kx & 1);
    }
};
Geometry make_geometry(int H, int W, bool colmajor);
// Slab `slab` of n_slabs of the FP32 geometry g (its 16-mode tiles split evenly, in order): sets k0,
// M, kp0 and ncp.  False if n_slabs < 1, slab out of range or more slabs than tiles.
bool make_slab(Geometry *g, int slab, int n_slabs);

// --------------------------------------------------------------- launchers (stream-ordered)

// Copy bytes from page-locked host memory to device memory with loads issued by the SMs (at most
// kGatherCtas CTAs of kGatherThreads threads on stream s).  cudaErrorInvalidValue (nothing
// launched) unless both addresses and the size are multiples of 16 bytes.
constexpr int kGatherCtas = 128, kGatherThreads = 128;
cudaError_t launch_gather_h2d(const void *host_src, void *dst, size_t bytes, cudaStream_t s);

// sums[f] = sum of the pixels of frame f (exact, uint64) for f < nf.  sums must be zeroed.
cudaError_t launch_frame_sums(const uint16_t *frames, int nf, const Geometry &g, unsigned long long *sums,
                              cudaStream_t s);

// ref[x] = fl32(fl32(i_f(x)) * hi), hi + lo = HW / sum(i_f) as a float pair: the FP32 normalised first
// frame f < nf whose sum is not 0 (zero if all nf frames are dark).  A context's reference buffer
// (ref_buffer_bytes) also keeps that frame's raw counts (raw, at ref_raw_offset) and {hi, lo} (inv, at
// ref_inv_offset), so a row pass may rebuild the same image from 2-byte counts; raw and inv may be
// NULL (the image alone).
cudaError_t launch_reference(const uint16_t *frames, const unsigned long long *sums, int nf, const Geometry &g,
                             float *ref, cudaStream_t s, uint16_t *raw = nullptr, float2 *inv = nullptr);
__host__ __device__ inline size_t ref_raw_offset(size_t HW) { return 4 * HW; }
__host__ __device__ inline size_t ref_inv_offset(size_t HW) { return (6 * HW + 15) / 16 * 16; }
__host__ __device__ inline size_t ref_buffer_bytes(size_t HW) { return ref_inv_offset(HW) + 16; }

// Row pass: for nf frames, normalise (and subtract ref when T = float) and transform every row.
// FP32: writes the column-group scratch of frame f at scratch + f * H * Wp.  FP64: writes the
// row transforms [H][Wp] into ring slot (slot0 + f) % R (slot-major ring).
// tws_row: per-stage twiddles of the size-specialised FP32 kernels (NULL: generic kernels only).
template <typename T>
cudaError_t launch_row_fft(const uint16_t *frames, int nf, const unsigned long long *sums, const float *ref,
                           const Geometry &g, const FftPlan &plan, const typename cplx_t<T>::type *tw_row,
                           const typename cplx_t<T>::type *tw_post, typename cplx_t<T>::type *ring, int R,
                           int slot0, cudaStream_t s, typename cplx_t<T>::type *scratch = nullptr,
                           const float2 *tws_row = nullptr);

// Compile-time-specialised FP32 passes; cudaErrorNotSupported for sizes without one.
// tw: the W_L table of the generic kernels (the 2048-wide row pass, one warp per row, uses it;
// NULL: the shared-memory Stockham kernels for every size).
cudaError_t launch_row_fft_ct(const uint16_t *frames, int nf, const unsigned long long *sums, const float *ref,
                              const Geometry &g, const float2 *tws, const float2 *twp, float2 *scratch,
                              cudaStream_t s, const float2 *tw = nullptr);
cudaError_t launch_col_fft_ct(int nf, const Geometry &g, const float2 *tws, const float2 *scratch, float2 *ring,
                              int R, int slot0, cudaStream_t s);
// Per-stage twiddle table of the specialised kernels for length L (stage s with sub-length NS and
// radix R holds exp(-2 pi i k r / (NS R)) at offset(s) + k (R - 1) + r - 1); empty if none.
std::vector<double> ct_stage_twiddles(int L);

// Column pass: length-H transforms of the nf frames of the row pass.  FP32: reads the scratch,
// writes ring slots (slot0 + f) % R (tile-major ring, column-major modes).  FP64: in place in the
// slot-major ring.
template <typename T>
cudaError_t launch_col_fft(int nf, const Geometry &g, const FftPlan &plan, const typename cplx_t<T>::type *tw_col,
                           typename cplx_t<T>::type *ring, int R, int slot0, cudaStream_t s,
                           const typename cplx_t<T>::type *scratch = nullptr, const float2 *tws_col = nullptr);

// Layout of the FP32 spectrum ring: tiles of 16 consecutive modes (flat k in column-major mode
// order), each tile holding its R slots contiguously, [tile][slot][16] float2 (128-byte slots), so
// the time series of a tile is one contiguous run of memory (a slot range is one bulk copy).
constexpr int kTile = 16;
constexpr int kTileShift = 4;
static_assert((1 << kTileShift) == kTile, "tile shift");
__host__ __device__ __forceinline__ size_t ring_index(int slot, size_t k, int R)
{
    return ((k >> kTileShift) * (size_t)R + (size_t)slot) * kTile + (k & (kTile - 1));
}

// Schedule of the tiled delay kernel (built on the host from the delay list, fixed per context).
// A sub-run is up to 16 consecutive delays d0 .. d0+len-1 (delay indices j0 .. j0+len-1); a stage
// is a group of sub-runs whose ring slots are loaded together.  Slot offsets are relative to the
// first frame t0 of the block: stage s loads frames t0+lo .. t0+hi (hi < the previous stage's lo).
struct SubRun {
    int j0, len, d0;
};
struct Stage {
    int sr0, nsr;    // sub-runs sr0 .. sr0+nsr-1
    int lo, hi;      // frames t0+lo .. t0+hi to load (lo > hi: nothing new)
    int need;        // the copy group of this stage may be issued once the consumers have finished
                     // this many steps (step 0 = reading the block's own frames, step s+1 = stage s):
                     // its slot-ring rows are then free and its mbarrier has been observed
};
constexpr int kFullBars = 8;       // copy-group mbarriers of the tiled kernel (group g uses g % 8)
constexpr int kDelayErrWords = 48; // status words of the tiled kernel
constexpr int kDelayBlock = 512;   // K of the tiled kernel: 16 warps x 2 half-warps x 16 frames
constexpr int kSlotBuf = 1024;     // shared-memory slot ring of the tiled kernel (128-byte slots)
// cross: a cross pass (the block's frames belong to one sequence, the older frames of every pair
// to another, indexed alike; delay 0 is a real pair), see DelayArgs::ring_cur
constexpr int kDefaultSpan = 240;           // widest delay range of one copy stage (default)
constexpr int kMinSpan = 16;
constexpr int kMaxSpan = kSlotBuf - kDelayBlock;  // a stage's group must fit the slot ring with the block
bool build_delay_schedule(const int *delays, int nd, bool cross, std::vector<SubRun> *subruns,
                          std::vector<Stage> *stages, int span = kDefaultSpan);
int count_delay_batches(const std::vector<SubRun> &subruns);  // batches the consumers hand to the writer

// The schedule travels by value in the kernel parameters (constant bank): uniform, cached reads.
constexpr int kMaxSubRuns = 256;
constexpr int kMaxSchedStages = 128;
struct DelaySchedule {
    int nsr, nst;
    int nbatch;  // batches of up to 16 delays whose partial sums are reduced together
    SubRun sr[kMaxSubRuns];
    Stage st[kMaxSchedStages];
};

// Fused FP32 delay update for new frames t0 .. t0+nb-1 (all already in the ring).
struct DelayArgs {
    const float2 *ring;  // tile-major, see ring_index
    int R;
    size_t M;            // modes per spectrum (multiple of 32) = accumulator row stride
    long long t0;
    int nb;
    const int *delays;
    int nd;
    float2 *acc;  // [nd][M] (Kahan sum, compensation)
    const DelaySchedule *sched;  // host copy; NULL = no tiled schedule (one-thread-per-mode kernel)
    int *err;     // device status words (kDelayErrWords): [0] set when a bounded wait gives up, [1..] where
    int tau_max;
    int stall_group;  // test hook: the producer stops before this copy group (-1: off)
    // Cross pass (out-of-core bands): the block's new frames t0 .. t0+nb-1 come from ring_cur
    // (R_cur slots, frame t in slot t mod R_cur) and every older frame of a pair from ring; a pair
    // at delay d is (block frame t, ring frame t - d), d = 0 included.  NULL: one ring for both.
    const float2 *ring_cur = nullptr;
    int R_cur = 0;
    // Tiles to update (16-mode tile indices, ascending; the tiled kernels only): NULL = every tile.
    // A context lists the tiles that hold a binned mode, so the corner modes beyond the Nyquist
    // circle, which no bin reads, are not updated.
    const int *tiles = nullptr;
    size_t ntiles = 0;
};
cudaError_t launch_delay_f32(const DelayArgs &a, int variant, cudaStream_t s);

// One work item of the ragged batch: the block t0 .. t0+nb-1 of one sequence, work tiles
// first .. first+ntiles-1 of the launch (its tiles[0 .. ntiles), or tiles 0 .. ntiles-1).
struct BatchItem {
    const float2 *ring;
    float2 *acc;
    const DelaySchedule *sched;  // device copy
    const int *tiles;            // the tiles to update (NULL: tiles 0 .. ntiles-1)
    long long t0;
    long long first;
    long long ntiles;
    size_t M;
    int R, nb, nd, nst, nbatch;
};
void truncate_schedule(const DelaySchedule &sc, long long tlast, int *nst, int *nbatch);
cudaError_t launch_delay_batched(const BatchItem *d_items, int nitems, long long total_tiles, int *err, int n_sm,
                                 cudaStream_t s);

// Plain FP64 update of one frame t.
cudaError_t launch_delay_f64(const double2 *ring, int R, size_t M, long long t, const int *delays, int nd,
                             double *acc, cudaStream_t s);

// Binning: D[j][b] = sum_{i in bin b} w_i value_j(i) / (pairs_j * C_b).
// modes: CSR by bin, entries (flat index << 1) | (weight == 2).
template <typename Acc>
cudaError_t launch_bin(const Acc *acc, size_t M, int nd, int nq, const int *bin_off, const int *bin_modes,
                       const long long *pairs, const long long *counts, double *D, cudaStream_t s);

// 2-D export: out[ky][kx] (kx < Wh) = value_j(ky*Wp + kx) / pairs.
template <typename Acc>
cudaError_t launch_export(const Acc *acc_j, const Geometry &g, long long pairs, double *out, cudaStream_t s);

// Eq. 1 fit (k_fit.cu); all pointers device, D [nd][nq], tau [nd], parameters [nq].
cudaError_t launch_fit_loss_grad(const float *D, const float *tau, int nd, int nq, const float *A, const float *B,
                                 const float *G, float *loss, float *gA, float *gB, float *gG, cudaStream_t s);
cudaError_t launch_fit_gauss_newton(const float *D, const float *tau, int nd, int nq, float *A, float *B, float *G,
                                    int iters, float lambda, cudaStream_t s);
cudaError_t launch_fit_adam(const float *D, const float *tau, int nd, int nq, float *A, float *B, float *G, int iters,
                            float lr, cudaStream_t s);

}  // namespace nfs
