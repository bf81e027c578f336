// Host-side internals shared by the library's translation units: the analysis context and its
// constants, and the steps of the frame pipeline (defined in nfs_host.cu) that the batch and
// region-of-interest entry points (nfs_batch.cu) and the out-of-core driver (nfs_ooc.cu) reuse.
#pragma once
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nfs_internal.cuh"

namespace nfs {
// Copy of nf whole frames of frame_bytes each from page-locked host memory, read by the SMs like
// launch_gather_h2d, adding frame f's exact pixel sum into sums[f] (zeroed by the caller);
// cudaErrorInvalidValue (nothing launched) unless both addresses and frame_bytes are multiples of
// 16 bytes.  (k_ingest.cu)
cudaError_t launch_gather_h2d_sums(const void *host_src, void *dst, int nf, size_t frame_bytes,
                                   unsigned long long *sums, cudaStream_t s);

namespace host {

// A named NVTX range over a scope: the C ABI's entry points appear as ranges in a profiler's
// timeline (and can filter ncu captures); without a profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kDefaultBlock = kDelayBlock;  // K: frames per fused delay update
constexpr int kMaxBlock = kDelayBlock;      // largest K the fused kernel takes
constexpr int kMaxChunk = 64;       // largest FFT chunk (FP64 path)
constexpr int kMaxChunkF32 = 32;    // largest FFT chunk of the FP32 path (its scratch holds 32 frames)
constexpr int kDefaultChunkF32 = 32; // FFT chunk of the FP32 path (measured on 2048x2048 frames: row and
                                     // column passes 19.0 us per frame at 32 frames per launch pair,
                                     // 19.6 at 16, 24.0 at 4)
constexpr int kMaxDim = 4096;
// Frames a context takes between resets: the delay kernels index frames with 32-bit integers.
constexpr long long kMaxFrames = (1LL << 31) - 4096;
constexpr int kMaxDelay = 65536;

inline bool factors_2_3(int n)
{
    if (n <= 0) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

struct TimedPair {
    int stage;
    cudaEvent_t a, b;
};

}  // namespace host
}  // namespace nfs

// One analysis context (the opaque nfs_ctx of the C ABI).
struct nfs_ctx {
    nfs::Geometry g{};
    int path = NFS_PATH_FUSED_F32;
    int K = nfs::host::kDefaultBlock;
    int R = 0, nd = 0, nq = 0;
    int fft_chunk = 4;
    int stage_frames = 1;
    int delay_variant = 0;
    int span = nfs::kDefaultSpan;  // widest delay range of one copy stage of the tiled schedule
    int fft_generic = 0;  // 1: generic FFT kernels even where specialised ones exist
    int stall_group = -1; // test hook of the bounded-wait path (NFS_OPT_TEST_STALL_GROUP)
    int h2d = 0;          // host pushes: 0 = the SMs read page-locked sources, 1 = copy engines
    bool own_streams = true;   // false for members of a batch (the batch owns the streams)
    bool defer_delay = false;  // members of a batch: the batch runs the delay update of full blocks
    int device = 0;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    std::vector<int32_t> delays;
    int tau_max = 0;

    // Host-push staging: a device ring of n_slots copy chunks of copy_frames frames each, so the
    // copy stream can run up to about two delay blocks ahead of the kernels; pageable sources pass
    // through two pinned host chunks first.
    int copy_frames = 1, n_slots = 2;
    uint16_t *d_stage = nullptr;
    unsigned long long *d_slot_sums = nullptr;  // per staging slot: its frames' sums (host pushes)
    // Staging slots whose frames are transformed but whose release (ev_free) is held back until
    // just before the next delay launch, so that the copies refilling them overlap that launch
    // (where one copy CTA fits beside each delay CTA) instead of the transforms of the next block.
    std::vector<int> free_pending;
    uint16_t *h_stage[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_filled, ev_free;
    cudaEvent_t ev_hcopied[2] = {nullptr, nullptr};
    long long stage_i = 0, hstage_i = 0;

    unsigned long long *d_sums = nullptr;
    float *d_ref = nullptr;
    void *d_ring = nullptr;
    void *d_acc = nullptr;
    int *d_delays = nullptr;
    void *d_tw_row = nullptr, *d_tw_post = nullptr, *d_tw_col = nullptr;
    float2 *d_tws_row = nullptr, *d_tws_col = nullptr;  // per-stage twiddles of the specialised FFTs
    float2 *d_scratch = nullptr;                         // FP32 row-pass output, kMaxChunkF32 frames
    nfs::FftPlan plan_row, plan_col;
    int *d_bin_off = nullptr, *d_bin_modes = nullptr;
    // The 16-mode tiles that hold a binned mode (ascending): the FP32 delay update runs on these
    // only unless every mode is asked for (NFS_OPT_MODES = 1, which the 2-D export needs).
    int *d_tiles = nullptr;
    long long n_tiles_binned = 0;
    int modes_all = 0;
    long long *d_pairs = nullptr, *d_counts = nullptr;
    double *d_D = nullptr, *d_export = nullptr;
    nfs::DelaySchedule *sched = nullptr;  // tiled-kernel schedule (host copy, passed by value); NULL if too long
    int *d_err = nullptr;
    // Cross pass (one band of the out-of-core mode): pairs (block frame of the "current" sequence,
    // older frame of the "old" sequence); the current sequence's spectra go to d_ring_cur (K slots),
    // the old sequence's to d_ring.  Both sequences advance together: frame u of each per step.
    bool cross = false;
    void *d_ring_cur = nullptr;
    int slab = 0, n_slabs = 1;  // mode slab of this context (g.k0, g.M); 0 of 1 = the whole spectrum
    long long transforms = 0;  // frames transformed (both sequences of a cross pass)

    std::vector<long long> counts, pairs_h;
    std::vector<double> qmean;
    long long nframes = 0, nprocessed = 0;
    bool have_ref = false;

    int err = NFS_OK;
    std::string errmsg;

    int timing = 0;  // 1: events around every launch; 2: around delay-update launches only; 3: as 1 + timeline
    std::vector<nfs::host::TimedPair> pending;
    cudaEvent_t tl_base = nullptr;  // timeline origin: the first event recorded since the last reset
    struct TimelineEntry {
        int stage;
        double start_ms, end_ms;
    };
    std::vector<TimelineEntry> timeline;
    std::vector<cudaEvent_t> pool;
    double stage_ms[NFS_N_STAGES] = {};
    long long stage_n[NFS_N_STAGES] = {};
    long long launches = 0;

    bool f32() const { return path == NFS_PATH_FUSED_F32; }
    size_t csize() const { return f32() ? sizeof(float2) : sizeof(double2); }
    size_t asize() const { return f32() ? sizeof(float2) : sizeof(double); }
    size_t frame_bytes() const { return g.HW * sizeof(uint16_t); }
};

namespace nfs {
namespace host {

// Records a CUDA error on the context (sticky) and returns NFS_ECUDA.
int set_cuda_error(nfs_ctx *c, cudaError_t e, const char *where);

#define CK(ctx, call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return set_cuda_error((ctx), _e, #call); \
    } while (0)

cudaEvent_t pool_get(nfs_ctx *c);
int harvest(nfs_ctx *c);

// Runs one launcher with optional event timing around it.
template <class F>
int timed(nfs_ctx *c, int stage, cudaStream_t s, F &&f, const char *what)
{
    cudaEvent_t a = nullptr, b = nullptr;
    const bool on = c->timing == 1 || c->timing == 3 || (c->timing == 2 && stage == NFS_STAGE_DELAY);
    if (on) {
        a = pool_get(c);
        b = pool_get(c);
        if (!a || !b) return set_cuda_error(c, cudaErrorMemoryAllocation, "cudaEventCreate");
        CK(c, cudaEventRecord(a, s));
    }
    cudaError_t e = f();
    if (e != cudaSuccess) return set_cuda_error(c, e, what);
    if (on) {
        CK(c, cudaEventRecord(b, s));
        c->pending.push_back({stage, a, b});
    }
    if (stage != NFS_STAGE_H2D) c->launches++;
    return NFS_OK;
}

int flush_block(nfs_ctx *c);
int release_slots(nfs_ctx *c);
int frame_sums(nfs_ctx *c, const uint16_t *dsrc, int n, unsigned long long *sums);
// The reference image from n device frames with known sums, the first time a context sees frames.
int reference_once(nfs_ctx *c, const uint16_t *dsrc, int n, const unsigned long long *sums);
int process_chunk(nfs_ctx *c, const uint16_t *dsrc, int nf, bool old, const unsigned long long *sums);
int autotune_fft_chunk(nfs_ctx *c);
int set_delay_span(nfs_ctx *c, int span);
int autotune_delay_span(nfs_ctx *c);
int next_chunk(const nfs_ctx *c, long long remaining, int cap);
int enter(nfs_ctx *c);
int check_args(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block);
int create_impl(int H, int W, const int32_t *delays, int n_delays, int n_qbins, int path, int block, nfs_ctx **out,
                bool cross = false, int slab = 0, int n_slabs = 1);
bool is_page_locked(const void *p);
// Priority of the copy streams: the device's greatest.
int copy_stream_priority();
// The device-side address of page-locked host memory p, nullptr if p is not page-locked.
const void *host_device_view(const void *p);
// One host-to-device copy of a frame push on stream s.  With sm_reads, a page-locked source and
// 16-byte aligned addresses and size, the SMs read the host memory (launch_gather_h2d; ++*launches);
// otherwise the copy engines copy it (cudaMemcpyAsync).
cudaError_t copy_h2d(void *dst, const void *src, size_t bytes, cudaStream_t s, bool sm_reads, long long *launches);

}  // namespace host
}  // namespace nfs
