/*
 * nfs.h -- C ABI of the GB300 library for the double-frame differential analysis of dynamic
 * near-field-scattering (shadowgraph, Schlieren, DDM) image sequences, after Cerchiari, Croccolo,
 * Cardinaux and Scheffold, arXiv:1209.3362.
 *
 * The library computes, for a stream of camera frames i_t(x) (uint16, H x W, row-major):
 *
 *   n_t(x)        = i_t(x) / <i_t>_x                 (frames normalised by their spatial average)
 *   Delta I(k, t, tau) = FT[n_t - n_{t+tau}](k)        (spatial Fourier transform of a difference)
 *   D(k, tau)     = < |Delta I(k, t, tau)|^2 >_t        (left-hand side of Eq. 1, averaged over every
 *                                                      pair t, t+tau of a stationary sequence)
 *   D_b(tau)      = azimuthal average of D(k, tau) over the radial bin b   (Fig. 1e,f)
 *
 * The Fourier transform is the unscaled forward DFT, exp(-2 pi i (k_x x / W + k_y y / H)).  By
 * linearity (processing paragraph of the paper) each frame is transformed once and pairs differ
 * in Fourier space.  Radial bins: with |f| the mode frequency in cycles/px, bin b holds the modes
 * with b <= 2 n_q |f| < b + 1 (integer-exact rule: L = lcm(H, W), m = k_x L / W, n = k_y' L / H with
 * k_y' the signed row frequency, bin = floor(isqrt(4 n_q^2 (m^2 + n^2)) / L)); the DC mode and
 * |f| >= 0.5 are left out; half-plane modes count twice except on the k_x = 0 and k_x = W/2
 * columns, so bin sums equal full-plane sums.  q = 2 pi |f| rad/px.
 *
 * Conventions for every call:
 *   - Return value: NFS_OK (0) or a negative status below.  nfs_strerror() names it; the context
 *     keeps the text of its last CUDA error (nfs_last_error()).
 *   - A CUDA error inside asynchronous work is sticky: every later call on that context returns
 *     NFS_ECUDA until nfs_destroy().
 *   - All device memory and streams belong to the context.  Host pointers passed in are only
 *     read or written during the call.
 *   - A context is used by one host thread at a time; contexts are independent of each other.
 *   - The device current at nfs_create() is the context's device; every call makes it current.
 */
#ifndef NFS_H
#define NFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NFS_OK 0
#define NFS_EINVAL (-1)       /* bad argument (NULL pointer, non-increasing delays, n < 0, ...) */
#define NFS_EUNSUPPORTED (-2) /* frame shape outside what the kernels handle */
#define NFS_ENOMEM (-3)       /* device or pinned host allocation failed */
#define NFS_ECUDA (-4)        /* a CUDA call or kernel failed (sticky) */
#define NFS_ESTATE (-5)       /* call not allowed in the context's current state */
#define NFS_ETOOBIG (-6)      /* problem needs more than the no-allocation scratch (see below) */
#define NFS_ETIMEOUT (-7)     /* a bounded wait inside a kernel gave up (sticky, like NFS_ECUDA) */

/* Arithmetic of the analysis path. */
#define NFS_PATH_FUSED_F32 0 /* FP32 frames and spectra, blocked fused delay update, Kahan-FP32
                                accumulators, FP64 mean and bin sums (the fast path) */
#define NFS_PATH_PLAIN_F64 1 /* FP64 everywhere, one frame per delay update, unfused (comparator) */

typedef struct nfs_ctx nfs_ctx;

/*
 * Create an analysis context (Eq. 1 for a single image sequence).
 *   H, W      frame height and width in pixels: even, 2 <= H, W <= 4096, prime factors 2 and 3
 *             only; otherwise NFS_EUNSUPPORTED.
 *   delays    n_delays (1..65535) frame delays tau_j, strictly increasing, tau_0 >= 0 (tau = 0 is
 *             allowed and gives D = 0 exactly), tau_max <= 65536.  Copied by the call.
 *   n_qbins   number of radial bins, 1..65536; bins span 0 <= |f| < 0.5 cycles/px evenly.
 *   *out      receives the context; NULL on failure.
 * Allocates the spectrum ring (tau_max + K slots of H x (W/2+1) complex values), the
 * accumulators (n_delays x H x (W/2+1)) and the staging buffers (copy chunks of up to 256 MB
 * covering two delay blocks, at most 9 GB) on the current device.
 * Uses NFS_PATH_FUSED_F32.
 */
int nfs_create(int H, int W, const int32_t *delays, int n_delays, int n_qbins, nfs_ctx **out);

/*
 * Same as nfs_create with an explicit path (NFS_PATH_*) and block size K (frames per fused delay
 * update, 1..512; 0 = the default 512).  The plain FP64 path ignores K (it updates once per frame).
 */
int nfs_create_ex(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block_frames,
                  nfs_ctx **out);

/*
 * ---------------------------------------------------------------- mode slabs (several GPUs)
 * Eq. 1 is evaluated independently at every wave vector q, so the spectrum can be split by mode:
 * a slab context takes every frame (mean, reference image and row transforms of whole frames, as
 * any context) but keeps only its slab's share of the modes -- the column transforms of the
 * column pairs that hold them, their ring slots, their accumulators and their terms of every bin.
 * The bin counts C_b stay those of the whole plane, so each slab's D_b(tau) is its share of the
 * azimuthal average and the results of the n_slabs slabs of one frame sequence ADD UP to the
 * whole context's D (up to FP64 rounding of the sum; pair counts, bin counts and q_mean are
 * those of the whole spectrum).  One context per GPU with a sum over GPUs of D (n_delays x n_qbins
 * doubles) is the only exchange.  The paper runs one GPU; the split is this library's.
 *
 * nfs_create_slab(): as nfs_create (fused FP32 path, K = 512) for slab `slab` of n_slabs, the
 * 16-mode tiles of the column-major mode order split evenly and in order.  nfs_export_spectrum on a
 * slab context writes 0 at the modes of other slabs (the exports of all slabs also add up).
 * Errors: NFS_EINVAL also for n_slabs < 1, slab outside [0, n_slabs) or more slabs than tiles.
 *
 * nfs_slab_range(): host only; first_mode and n_modes of the slab in the column-major order
 * k = k_x H + k_y (n_modes a multiple of 16; the last slab may end in padding modes past H(W/2+1)).
 * Errors: NFS_EINVAL (NULL outputs, bad slab), NFS_EUNSUPPORTED (shape).
 */
int nfs_create_slab(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int slab, int n_slabs,
                    nfs_ctx **out);
int nfs_slab_range(int H, int W, int slab, int n_slabs, int64_t *first_mode, int64_t *n_modes);

/*
 * The radial bin table of an H x W frame with n_qbins bins (the rule above; Fig. 1e,f's azimuthal
 * average), computed on the host with no device call.  Caller-owned outputs:
 *   bin_of_mode  [H][W/2+1] int32, row-major over (k_y, k_x): the bin of each half-plane mode or -1
 *                (the DC mode and |f| >= 0.5); may be NULL
 *   bin_counts   [n_qbins] C_b, the weighted mode count of each bin (weights 1 or 2)
 *   q_mean       [n_qbins] weighted mean of q = 2 pi |f| over the bin (0 if empty); may be NULL
 * NFS_EINVAL for bin_counts NULL or n_qbins outside 1..65536; NFS_EUNSUPPORTED for a shape
 * nfs_create rejects.  The bins of every context are exactly this table.
 */
int nfs_bin_table(int H, int W, int n_qbins, int32_t *bin_of_mode, int64_t *bin_counts, double *q_mean);

/*
 * Append n_frames frames from HOST memory, contiguous [n_frames][H][W] uint16, row-major.
 * Counts above 4095 are allowed (no clipping).  The frames are copied to the device before the
 * call returns, so the caller may reuse the buffer at once; the analysis itself runs
 * asynchronously on the context's stream.  Page-locked buffers are read directly (by the SMs or
 * the copy engines: NFS_OPT_H2D); pageable ones pass through the context's pinned staging buffers.
 * Read by the SMs, whole frames also have their exact sums taken during the copy (no separate sum
 * pass).  The copies run on a stream of the device's greatest priority, chunks of up to 256 MB into a
 * device staging ring of two delay blocks; a slot transformed into the spectrum ring is handed
 * back just before the next delay launch, so that its refill runs beside that launch.
 * A frame whose pixels sum to 0 has no mean: its normalised image is taken as 0.
 * A context takes at most 2^31 - 4096 frames between nfs_create/nfs_reset (frame indices in the
 * kernels are 32-bit): a push beyond that returns NFS_ESTATE and changes nothing.
 * Returns the status of earlier asynchronous work as well (sticky error).
 */
int nfs_push_frames(nfs_ctx *ctx, const uint16_t *host_frames, int n_frames);

/*
 * Append n_frames frames already in DEVICE memory of the context's device (same layout as
 * nfs_push_frames).  The call enqueues the reads on the context's stream (nfs_get_stream) and
 * returns: the frames must be completely written before that stream reaches them (finish the
 * writing work first, or make that stream wait for it, e.g. cudaStreamWaitEvent), and the buffer
 * must stay valid and unchanged until the context's stream has passed the work
 * (nfs_synchronize() or any call that returns results).  The address must be 2-byte aligned;
 * 16-byte alignment with W a multiple of 8 takes the vectorised loads.
 */
int nfs_push_frames_device(nfs_ctx *ctx, const uint16_t *dev_frames, int n_frames);

/*
 * Finish the frames pushed so far (including a partial block) and return the binned structure
 * function.  Caller-owned host outputs:
 *   D           [n_delays][n_qbins]  D_b(tau_j) = sum_{k in b} w_k D(k, tau_j) / C_b
 *   bin_counts  [n_qbins]            C_b (integer mode weights; exact)
 *   pair_counts [n_delays]           number of frame pairs averaged at tau_j: max(0, N - tau_j)
 *   q_mean      [n_qbins] or NULL    mean q (rad/px) of the bin
 * An entry with no pairs or an empty bin is 0 (its count tells it apart).  May be called
 * repeatedly while frames keep coming (a running result).  Synchronises the stream.
 */
int nfs_structure_function(nfs_ctx *ctx, double *D, int64_t *bin_counts, int64_t *pair_counts, double *q_mean);

/*
 * The 2-D spectrum D(k, tau_j) for one delay index j before binning, as FP64 [H][W/2+1]
 * (k_x fastest, k_y = 0..H-1 in FFT order).  Flushes pending frames and synchronises.  On the FP32
 * path it needs NFS_OPT_MODES = 1, set before the first frame (otherwise NFS_ESTATE, not sticky:
 * the delay update then keeps only the tiles the bins read).
 */
int nfs_export_spectrum(nfs_ctx *ctx, int delay_index, double *out);

/* Forget all frames (accumulators to zero, frame count to 0); keeps allocations and options. */
int nfs_reset(nfs_ctx *ctx);

/* Wait for all work queued on the context; returns the sticky status. */
int nfs_synchronize(nfs_ctx *ctx);

/* Frames pushed so far. */
int64_t nfs_frame_count(const nfs_ctx *ctx);

/* Destroy the context and free everything it owns; NULL is accepted. */
void nfs_destroy(nfs_ctx *ctx);

/* Static text for a status code. */
const char *nfs_strerror(int status);

/* Text of the context's last CUDA error ("" if none). */
const char *nfs_last_error(const nfs_ctx *ctx);

/* The cudaStream_t the context launches on, as void*. */
void *nfs_get_stream(const nfs_ctx *ctx);

/* Option keys for nfs_set_option / nfs_get_option. */
#define NFS_OPT_TIMING 1      /* 1 = record CUDA events around every kernel launch; 2 = around the
                                  delay-update launches only (the least overhead); 3 = as 1, and
                                  also keep each launch's start and end for nfs_get_timeline;
                                  default 0 */
#define NFS_OPT_BLOCK_FRAMES 2 /* read-only: K */
#define NFS_OPT_RING_SLOTS 3   /* read-only: ring slots R = tau_max + K (FP32) or tau_max + 64 (FP64) */
#define NFS_OPT_PITCH 4        /* read-only: complex values per spectrum row in HBM (>= W/2+1) */
#define NFS_OPT_PATH 5         /* read-only: NFS_PATH_* */
#define NFS_OPT_FFT_CHUNK 6    /* frames transformed per launch pair (1..32 FP32, 1..64 FP64; default 32
                                  FP32, 4 FP64; 0 = choose by measurement, FP32 path, only before the
                                  first frame: the measurement uses the ring and the reference image,
                                  so NFS_ESTATE once frames were pushed) */
#define NFS_OPT_DELAY_VARIANT 7 /* fused delay kernel: 0 = tiled, packed f32x2 math (default);
                                   1 = one thread per mode; 2 = tiled, scalar FP32 math */
#define NFS_OPT_FFT_GENERIC 8   /* 1 = generic FFT kernels even where size-specialised ones exist */
#define NFS_OPT_TEST_STALL_GROUP 9 /* test hook (default -1 = off): the tiled delay kernel's producer
                                      stops issuing copies from this group on, so a consumer's bounded
                                      wait runs out (~2 s) and the call returns NFS_ETIMEOUT; checks
                                      the failure path without faulting the GPU */
#define NFS_OPT_DELAY_SPAN 12   /* fused delay kernel: widest delay range of one copy stage, 16..512
                                   (default 240); 0 = choose by measurement among 112, 176, 240,
                                   320 and 400 on this context's own delay list (FP32 path, only
                                   before the first frame: the measurement runs the kernel on the
                                   ring and clears the accumulators afterwards, NFS_ESTATE once frames
                                   were pushed).  The span regroups copy stages only: results are
                                   bit-identical for every span */
#define NFS_OPT_H2D 13           /* how host pushes reach the device: 0 = the SMs read page-locked
                                    sources directly (a copy kernel on the copy stream, counted as a
                                    launch; default); 1 = the copy engines (cudaMemcpyAsync).  Sources
                                    that are not page-locked, or whose address or size is not a
                                    multiple of 16 bytes, always go through the copy engines.  Both
                                    move the same bytes: results are identical.  The SMs read at full
                                    speed whatever state the host pages are in; the copy engines were
                                    measured at 8-38 GB/s on the first gigabytes of some freshly
                                    pinned buffers */
#define NFS_OPT_MODES 14         /* which modes the FP32 delay update keeps: 0 = the 16-mode tiles that
                                    hold a binned mode (default: the corner modes beyond the Nyquist
                                    circle, |f| >= 1/2 cycle per pixel in the half-plane, which no bin
                                    reads, are left out; about 21 % of the modes); 1 = every mode
                                    (needed for nfs_export_spectrum).  Only before the first frame
                                    (NFS_ESTATE after); binned results are bit-identical either way */
#define NFS_OPT_DELAY_MODES 15   /* read-only: modes the delay update keeps (16 x tiles; all modes M of
                                    the context when NFS_OPT_MODES = 1 or on the FP64 path) */
#define NFS_OPT_SLAB_FIRST_MODE 10 /* read-only: first mode (column-major order) of a slab context */
#define NFS_OPT_SLAB_MODES 11      /* read-only: modes held (the slab's share, a multiple of 16) */
int nfs_set_option(nfs_ctx *ctx, int key, int64_t value);
int nfs_get_option(const nfs_ctx *ctx, int key, int64_t *value);

/* Stages reported by nfs_get_timings. */
#define NFS_STAGE_H2D 0   /* host-to-device frame copies */
#define NFS_STAGE_MEAN 1  /* per-frame exact integer sums (spatial mean) */
#define NFS_STAGE_ROWFFT 2 /* normalisation + row r2c FFTs */
#define NFS_STAGE_COLFFT 3 /* column FFTs into the spectrum ring */
#define NFS_STAGE_DELAY 4 /* delay update of the accumulators */
#define NFS_STAGE_BIN 5   /* radial binning */
#define NFS_N_STAGES 6

/*
 * Per-stage totals since the last nfs_reset_timings(): ms[s] = summed device time of the launches
 * of stage s (CUDA events on the context's stream), launches[s] = their number.  Needs
 * NFS_OPT_TIMING = 1; synchronises.  Arrays have NFS_N_STAGES entries.
 */
int nfs_get_timings(nfs_ctx *ctx, double *ms, int64_t *launches);
int nfs_reset_timings(nfs_ctx *ctx);

/*
 * Timeline of the launches and host-to-device copies recorded with NFS_OPT_TIMING = 3 since the
 * last nfs_reset_timings(), in issue order: stage[i] (NFS_STAGE_*), start_ms[i] and end_ms[i] in
 * milliseconds from the first recorded launch (copies run on the context's copy stream, kernels on
 * its compute stream; the times of both come from CUDA events on one device clock, so gaps and
 * overlaps between the two streams can be read off).  Up to cap entries are written (any pointer
 * may be NULL when cap is 0); *n receives the number recorded.  Synchronises.  Library tracing: the
 * paper has no counterpart.  Errors: NFS_EINVAL (ctx or n NULL, cap < 0), sticky errors.
 */
int nfs_get_timeline(nfs_ctx *ctx, int32_t *stage, double *start_ms, double *end_ms, int64_t cap, int64_t *n);

/*
 * Measuring hook of the fused delay kernel: in a library built with NFS_DELAY_PROFILE
 * (buildlib.build(profile=True)), the clock cycles its warp roles spent by phase, summed over every
 * launch since the last reset (consumer total, copy-group waits, partial-buffer waits, pair
 * arithmetic, hand-overs, writer total, writer waits, producer waits, prologue, epilogue, tile
 * passes): out[0 .. n) are written and the count of values is returned; reset != 0 clears them.
 * A normal build returns NFS_EUNSUPPORTED.  Library tracing: the paper has no counterpart.
 */
int nfs_delay_profile(unsigned long long *out, int n, int reset);

/*
 * Number of kernel launches the context has issued since creation (all stages, both paths).
 */
int64_t nfs_launch_count(const nfs_ctx *ctx);

/*
 * ---------------------------------------------------------------- ragged batch
 * Many independent sequences (regions of interest, cameras, experiments) of uneven frame shapes
 * and delay lists analysed together: each member is a context of its own, all members share one
 * stream, and the delay update of every member whose block of K frames is complete runs in ONE
 * persistent launch over a ragged work list of (sequence, 16-mode tile) items.  The FFT launch
 * size of each frame shape is chosen by a measuring autotuner when the batch is created.
 */
typedef struct nfs_batch nfs_batch;

/*
 * n_seq sequences; sequence s has frames H[s] x W[s] (as nfs_create), delays
 * delays[delay_offsets[s] .. delay_offsets[s+1]) (strictly increasing) and n_qbins[s] bins.
 * NFS_EUNSUPPORTED also for a delay list too long for the tiled kernel's schedule.
 */
int nfs_batch_create(int n_seq, const int *H, const int *W, const int32_t *delay_offsets, const int32_t *delays,
                     const int *n_qbins, nfs_batch **out);
void nfs_batch_destroy(nfs_batch *b);
/* Append host frames to one sequence (as nfs_push_frames). */
int nfs_batch_push(nfs_batch *b, int seq, const uint16_t *host_frames, int n_frames);
/* Append device frames to every sequence at once: dev_frames[s] holds n_frames[s] frames. */
int nfs_batch_push_device(nfs_batch *b, const uint16_t *const *dev_frames, const int *n_frames);
/* Finish every member's pending frames and return sequence seq's result (as nfs_structure_function). */
int nfs_batch_structure_function(nfs_batch *b, int seq, double *D, int64_t *bin_counts, int64_t *pair_counts,
                                 double *q_mean);
int nfs_batch_reset(nfs_batch *b);
int nfs_batch_synchronize(nfs_batch *b);
/* The member context of sequence seq (owned by the batch: do not destroy it). */
nfs_ctx *nfs_batch_member(nfs_batch *b, int seq);
void *nfs_batch_get_stream(const nfs_batch *b);
int64_t nfs_batch_launch_count(const nfs_batch *b);
const char *nfs_batch_last_error(const nfs_batch *b);

/*
 * ---------------------------------------------------------------- regions of interest
 * Spatially resolved analysis (near-field scattering lends itself to experiments that resolve the
 * sample in space; paper, introduction).  Each frame of
 * one H x W camera sequence is cut into n_roi windows, and window r (rows y0[r] .. y0[r]+h[r],
 * columns x0[r] .. x0[r]+w[r]) is analysed as a sequence of its own: normalised by its own spatial
 * mean, transformed at h[r] x w[r], binned into n_qbins[r] bins, with the same delay list for every
 * window.  Windows may overlap.  The result is a batch (above) with one member per window:
 * read window r with nfs_batch_structure_function(b, r, ...); nfs_batch_reset and
 * nfs_batch_destroy apply.  Window r's result equals nfs_create(h[r], w[r], ...) fed the cropped
 * frames, bit for bit.
 *
 * nfs_roi_create: NFS_EINVAL for a window outside the frame, an odd W, x0 or w (the crop moves
 * 4-byte words), an empty list or more than 65535 windows, a NULL pointer or a delay list or bin
 * count nfs_create rejects;
 * NFS_EUNSUPPORTED for a window shape nfs_create rejects (all checked before any CUDA call);
 * NFS_ENOMEM.
 * nfs_roi_push: n_frames full frames [n][H][W] from host memory; the buffer may be reused on
 * return.  nfs_roi_push_device: full frames already on the device, 4-byte aligned, read by
 * stream-ordered kernels on the batch's stream (keep them alive until nfs_batch_synchronize).
 * Both: NFS_EINVAL for a batch not made by nfs_roi_create; sticky errors as nfs_push_frames.
 */
int nfs_roi_create(int H, int W, int n_roi, const int *y0, const int *x0, const int *h, const int *w,
                   const int32_t *delays, int n_delays, const int *n_qbins, nfs_batch **out);
int nfs_roi_push(nfs_batch *b, const uint16_t *host_frames, int n_frames);
int nfs_roi_push_device(nfs_batch *b, const uint16_t *dev_frames, int n_frames);

/*
 * ---------------------------------------------------------------- Eq. 1 fit
 * Per radial bin b, fit D_b(tau) = 2 A_b [1 - exp(-Gamma_b tau)] + 2 B_b to the structure function,
 * i.e. Eq. 1 with the intermediate scattering function f = exp(-Gamma tau), A = a T I_s (static
 * amplitude), B = a B (noise background).  Loss per bin: sum over delays of the squared residual.
 */
#define NFS_FIT_GAUSS_NEWTON 0 /* Levenberg-Marquardt-damped Gauss-Newton, A, B >= 0, Gamma > 0 */
#define NFS_FIT_ADAM 1         /* Adam on theta = theta_0 (1 + u), step 1e-2 in u */

/*
 * Fit every bin of the context's structure function (D = NULL: the current result, as
 * nfs_structure_function gives it; else a caller-owned HOST array [n_delays][n_qbins]).  Delays
 * with no pair and tau = 0 are left out.  A, B, Gamma: HOST arrays [n_qbins], initial values in,
 * fitted values out.  iters: Gauss-Newton or Adam steps.  Synchronises; NFS_ESTATE if no delay
 * has data.
 */
int nfs_fit(nfs_ctx *ctx, const double *D, float *A, float *B, float *Gamma, int iters, int method);

/*
 * Device-level pieces for autograd drivers.  All pointers DEVICE memory, D [n_delays][n_bins]
 * (bins fastest), tau [n_delays], parameters and outputs [n_bins]; stream = cudaStream_t or NULL.
 * nfs_fit_loss_grad: loss[b] = sum_j r_j^2 and its gradients (gA, gB, gGamma may be NULL).
 * nfs_fit_gauss_newton: iters damped Gauss-Newton steps in place (lambda: initial damping).
 * Asynchronous on the stream; NFS_EINVAL for bad arguments, NFS_ECUDA if the launch fails.
 */
int nfs_fit_loss_grad(const float *D, const float *tau, int n_delays, int n_bins, const float *A, const float *B,
                      const float *Gamma, float *loss, float *gA, float *gB, float *gGamma, void *stream);
int nfs_fit_gauss_newton(const float *D, const float *tau, int n_delays, int n_bins, float *A, float *B,
                         float *Gamma, int iters, float lambda, void *stream);

/*
 * ---------------------------------------------------------------- out-of-core bands
 * The processing paragraph's case of a sequence whose spectra do not fit in device memory: the
 * memory holds only part of them and the frames are transferred to the GPU several times (the
 * paper re-uploads images through a FIFO, diagonal by diagonal).  Here the delays are split into
 * bands that each fit a budget of max_ring_slots spectra, and every band is one pass over the
 * frames, which stay in host memory:
 *   - band 0: an ordinary pass over the delays d with d + K <= max_ring_slots, K = 512 the block
 *     of the fused update (one transform per frame);
 *   - a later band with smallest delay lo: a pass with shift s = K floor(lo / K) that pairs
 *     frame u + s (as the newer frame) with frame u + s - d, holding the frames u + s in a
 *     K-slot ring and the frames u in a ring of (largest d - s) + K slots (two transforms per
 *     frame index: N - s each); its delays d satisfy (d - s) + 2 K <= max_ring_slots.
 * Every pair is added in the same K-frame block and in the same order as in one in-core pass,
 * so the results equal those of nfs_create + nfs_push_frames + nfs_structure_function.
 *
 * nfs_out_of_core_plan() gives the bands without touching the GPU (host logic only):
 *   band_first   [n_bands + 1] index of every band's first delay, then n_delays (may be NULL)
 *   band_shift   [n_bands] the shift s of every band (0 for band 0) (may be NULL)
 *   n_bands, n_transforms   out: the number of bands and of frame transforms all passes make
 *                (N per ordinary band, 2 (N - s) per shifted band; the paper's FIFO scheme makes
 *                N (2 alpha - 3 + 2 / alpha) for N - 1 = alpha N* frames and a memory of N*)
 * Arrays sized for n_delays bands suffice.  NFS_EINVAL for budgets below 3 K = 1536 slots (a band
 * must hold its first delay) or bad delays; NFS_EUNSUPPORTED if one delay alone exceeds the
 * schedule.
 *
 * nfs_structure_function_out_of_core() runs the bands and returns, for the whole delay list, what
 * nfs_structure_function returns (FP32 fused path).  frames: HOST memory [n_frames][H][W] uint16
 * (pinned or pageable), read n_bands (or twice as many) times, not kept after the call.  The
 * device memory a band holds (its rings, accumulators, staging) is freed before the next band.
 * n_transforms (may be NULL) receives the frame transforms made.  Errors as nfs_create and
 * nfs_structure_function; NFS_ESTATE if the passes did not transform the planned frames.
 */
int nfs_out_of_core_plan(const int32_t *delays, int n_delays, int64_t n_frames, int64_t max_ring_slots,
                         int32_t *band_first, int64_t *band_shift, int *n_bands, int64_t *n_transforms);
int nfs_structure_function_out_of_core(int H, int W, const int32_t *delays, int n_delays, int n_qbins,
                                       const uint16_t *frames, int64_t n_frames, int64_t max_ring_slots, double *D,
                                       int64_t *bin_counts, int64_t *pair_counts, double *q_mean,
                                       int64_t *n_transforms);

/*
 * ---------------------------------------------------------------- delay-kernel schedule (host logic)
 * nfs_delay_schedule() returns the copy schedule the fused delay kernel follows for a delay list,
 * so that its safety can be checked without a GPU.  The kernel takes a block of block_frames new
 * frames t0 .. per launch and streams older frames through a ring of slot_rows shared-memory rows
 * (frame f in row f mod slot_rows) in copy groups: group 0 brings the block itself, group s + 1 the
 * frames of stage s not yet present.  Step 0 reads the block; step s + 1 reads stage s's frames.
 *   delays, n_delays   as for nfs_create (strictly increasing, >= 0)
 *   cross        nonzero: the schedule of a shifted out-of-core pass (the block's frames and the
 *                older frames are two different sequences indexed alike; delay 0 is a real pair)
 *   subruns      [3 * max_entries] or NULL: per sub-run (j0, len, d0): delays j0 .. j0+len-1 are
 *                d0 .. d0+len-1 (runs of consecutive delays, at most 16)
 *   stages       [5 * max_entries] or NULL: per stage (first sub-run, sub-runs, lo, hi, need): its
 *                copy group loads frames t0+lo .. t0+hi (none when lo > hi) and may be issued once
 *                steps 0 .. need-1 are finished by every warp; the stage reads frames
 *                t0 - (largest delay) .. t0 + block_frames - 1 - (smallest delay)
 *   n_subruns, n_stages, block_frames, slot_rows, copy_barriers   out (copy group g waits on
 *                barrier g mod copy_barriers; the last three may be NULL)
 *   span         widest delay range of one stage, 16 .. 512 (0 = the default 240; see
 *                NFS_OPT_DELAY_SPAN)
 * NFS_ETOOBIG if an array would need more than max_entries entries (the counts are still set).
 * NFS_EINVAL also for a span outside 16 .. 512.
 */
int nfs_delay_schedule(const int32_t *delays, int n_delays, int cross, int32_t *subruns, int32_t *stages,
                       int max_entries, int *n_subruns, int *n_stages, int *block_frames, int *slot_rows,
                       int *copy_barriers, int span);

/*
 * ---------------------------------------------------------------- analysis without allocation
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory while they run: a process whose device memory is owned by another allocator
 * (a framework's pool that has reserved the GPU), or an acquisition loop that must not take the
 * device-wide synchronisation that cudaMalloc / cudaFree can imply.
 *
 * nfs_structure_function_noalloc() computes, in one call, the result nfs_create +
 * nfs_push_frames_device + nfs_structure_function give for the fused FP32 path, but takes all of its
 * scratch (spectrum ring, accumulators, twiddles, bin lists, sums) from one static device array of
 * NFS_NOALLOC_SCRATCH_BYTES, and calls no cudaMalloc, cudaFree or other allocating routine.  Its
 * steps differ from a context's in ways that change only FP32 rounding: the generic FFT kernels, the
 * one-thread-per-mode delay update in blocks of 32 frames, and a reference image taken from the
 * first 4 frames (a context takes it from its first copy chunk); the integer counts are identical.
 *   dev_frames   n_frames (at most 2^30) frames in DEVICE memory of the CURRENT device,
 *                [n_frames][H][W] uint16, 2-byte aligned
 *   H, W, delays, n_delays, n_qbins   as for nfs_create (delays and outputs are HOST memory)
 *   stream       cudaStream_t to run on (NULL = the legacy default stream); the call synchronises it
 *                before returning
 *   D, bin_counts, pair_counts        as for nfs_structure_function
 * Returns NFS_EINVAL, before any GPU work, for the argument errors of nfs_create and when dev_frames
 * is not device memory of the current device.
 * Returns NFS_ESTATE, before any GPU work, when the stream is being captured (the call ends by
 * synchronising its stream).
 * Returns NFS_EUNSUPPORTED, before any GPU work, also when 2 (n_qbins lcm(H, W))^2 >= 1.8e19 (its
 * device-side bin index works in 64-bit integers; nfs_create has no such limit).
 * Returns NFS_ETOOBIG, before any GPU work, when the sizes need more scratch than the array holds:
 * about 8 (tau_max + 32 + n_delays + 1) H (W/2 + 1) bytes plus small tables (for example 128 x 128
 * frames with tau_max = 50 and 50 delays need about 9 MB).
 * Notes for callers:
 *   - The array is a file-scope __device__ variable: every GPU that loads this library holds
 *     NFS_NOALLOC_SCRATCH_BYTES of device memory for it until the process exits.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress) with the current
 *     device, so an address is never reused after the device's context was created again.
 *   - Every call shares the one array and it keeps the previous call's contents (the call clears
 *     what must start at zero).  Calls that overlap on the GPU -- two host threads, or two
 *     streams -- race on it and give wrong results; serialise them.
 */
#define NFS_NOALLOC_SCRATCH_BYTES (64ull << 20)
int nfs_structure_function_noalloc(const uint16_t *dev_frames, int n_frames, int H, int W, const int32_t *delays,
                                   int n_delays, int n_qbins, void *stream, double *D, int64_t *bin_counts,
                                   int64_t *pair_counts);

#ifdef __cplusplus
}
#endif

#endif /* NFS_H */
