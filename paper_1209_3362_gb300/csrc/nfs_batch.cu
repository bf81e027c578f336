// Ragged batches of sequences (nfs_batch_*) and regions of interest of one camera sequence
// (nfs_roi_*): member contexts share one stream, and the delay update of every member with a full
// block runs in one persistent launch.
#include <algorithm>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "nfs_host.cuh"
#include "roi.cuh"

using namespace nfs;
using namespace nfs::host;

extern "C" {

// ---------------------------------------------------------------- ragged batch

struct nfs_batch {
    int n = 0, device = 0, n_sm = 0;
    std::vector<nfs_ctx *> seq;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    DelaySchedule *d_scheds = nullptr;  // one per sequence
    BatchItem *d_items = nullptr;       // work list of one launch
    int *d_err = nullptr;
    std::vector<BatchItem> items;
    int err = NFS_OK;
    std::string errmsg;
    long long launches = 0;
    // regions of interest (nfs_roi_create): windows of one H x W camera sequence
    int roi_H = 0, roi_W = 0;
    std::vector<RoiRect> rois;
    RoiRect *d_rois = nullptr;
    uint16_t *d_crop = nullptr;   // kRoiGroup frames of every window
    uint16_t *d_full = nullptr;   // kRoiGroup full frames (host pushes), allocated on first use
    long long roi_max_words = 0;  // 4-byte words of the largest window's group
};

static void batch_free(nfs_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    for (nfs_ctx *c : b->seq) nfs_destroy(c);
    cudaFree(b->d_scheds);
    cudaFree(b->d_items);
    cudaFree(b->d_err);
    cudaFree(b->d_rois);
    cudaFree(b->d_crop);
    cudaFree(b->d_full);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
    delete b;
}

static int batch_fail(nfs_batch *b, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return NFS_OK;
    b->errmsg = std::string(where) + ": " + cudaGetErrorString(e);
    if (b->err == NFS_OK) b->err = NFS_ECUDA;
    return NFS_ECUDA;
}

// One persistent launch over every member whose pending block is full (all = false) or non-empty
// (all = true).
static int batch_flush(nfs_batch *b, bool all)
{
    b->items.clear();
    long long total = 0;
    for (size_t s = 0; s < b->seq.size(); ++s) {
        nfs_ctx *c = b->seq[s];
        const long long pend = c->nframes - c->nprocessed;
        if (pend <= 0 || (!all && pend < c->K)) continue;
        int nst = 0, nbatch = 0;
        truncate_schedule(*c->sched, c->nframes - 1, &nst, &nbatch);
        if (nst > 0) {
            BatchItem it;
            it.ring = (const float2 *)c->d_ring;
            it.acc = (float2 *)c->d_acc;
            it.sched = b->d_scheds + s;
            it.tiles = c->modes_all ? nullptr : c->d_tiles;
            it.ntiles = c->modes_all ? (long long)(c->g.M / kTile) : c->n_tiles_binned;
            it.t0 = c->nprocessed;
            it.first = total;
            it.M = c->g.M;
            it.R = c->R;
            it.nb = (int)pend;
            it.nd = c->nd;
            it.nst = nst;
            it.nbatch = nbatch;
            if (it.ntiles > 0) b->items.push_back(it);
            total += it.ntiles;
        }
        c->nprocessed = c->nframes;
    }
    if (b->items.empty()) return NFS_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BatchItem) * b->items.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_delay_batched(b->d_items, (int)b->items.size(), total, b->d_err, b->n_sm, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batched delay update");
    b->launches++;
    return NFS_OK;
}

static int batch_enter(nfs_batch *b)
{
    if (!b) return NFS_EINVAL;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return batch_fail(b, e, "cudaSetDevice");
    return b->err;
}

// the device status of the batched launches (after a synchronisation)
static int batch_check(nfs_batch *b)
{
    int dev_err[kDelayErrWords] = {};
    cudaError_t e = cudaMemcpyAsync(dev_err, b->d_err, sizeof(dev_err), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch status");
    if (dev_err[0]) {
        char buf[160];
        snprintf(buf, sizeof(buf), "batched delay kernel: a bounded wait gave up (kind %d, cta %d, warp %d, index %d)",
                 dev_err[1], dev_err[2], dev_err[3], dev_err[4]);
        b->errmsg = buf;
        if (b->err == NFS_OK) b->err = NFS_ETIMEOUT;
    }
    return b->err;
}

int nfs_batch_create(int n_seq, const int *H, const int *W, const int32_t *delay_offsets, const int32_t *delays,
                     const int *n_qbins, nfs_batch **out)
{
    if (!out) return NFS_EINVAL;
    *out = nullptr;
    if (n_seq <= 0 || !H || !W || !delay_offsets || !delays || !n_qbins) return NFS_EINVAL;
    for (int s = 0; s < n_seq; ++s)
        if (delay_offsets[s + 1] <= delay_offsets[s]) return NFS_EINVAL;
    nfs_batch *b = new (std::nothrow) nfs_batch();
    if (!b) return NFS_ENOMEM;
    cudaGetDevice(&b->device);
    b->n = n_seq;
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&b->copy_stream, cudaStreamNonBlocking, copy_stream_priority()) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    std::vector<DelaySchedule> scheds((size_t)n_seq);
    for (int s = 0; s < n_seq; ++s) {
        nfs_ctx *c = nullptr;
        const int rc = create_impl(H[s], W[s], delays + delay_offsets[s], delay_offsets[s + 1] - delay_offsets[s],
                                   n_qbins[s], NFS_PATH_FUSED_F32, 0, &c);
        if (rc) {
            batch_free(b);
            return rc;
        }
        b->seq.push_back(c);
        if (!c->sched) {  // delay list too long for the tiled kernel's schedule
            batch_free(b);
            return NFS_EUNSUPPORTED;
        }
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
        cudaStreamDestroy(c->copy_stream);
        c->stream = b->stream;
        c->copy_stream = b->copy_stream;
        c->own_streams = false;
        c->defer_delay = true;
        scheds[s] = *c->sched;
        if (autotune_fft_chunk(c)) {
            batch_free(b);
            return NFS_ECUDA;
        }
    }
    if (cudaMalloc(&b->d_scheds, sizeof(DelaySchedule) * (size_t)n_seq) != cudaSuccess ||
        cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)n_seq) != cudaSuccess ||
        cudaMalloc(&b->d_err, sizeof(int) * kDelayErrWords) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return NFS_ENOMEM;
    }
    if (cudaMemcpy(b->d_scheds, scheds.data(), sizeof(DelaySchedule) * (size_t)n_seq, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int) * kDelayErrWords) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    *out = b;
    return NFS_OK;
}

void nfs_batch_destroy(nfs_batch *b) { batch_free(b); }

int nfs_batch_push(nfs_batch *b, int seq, const uint16_t *host_frames, int n)
{
    NvtxRange range("nfs_batch_push");
    int rc = batch_enter(b);
    if (rc) return rc;
    if (seq < 0 || seq >= b->n || n < 0 || (n > 0 && !host_frames)) return NFS_EINVAL;
    nfs_ctx *c = b->seq[seq];
    long long done = 0;
    while (done < n) {
        const long long room = c->K - (c->nframes - c->nprocessed);
        if (room <= 0) {
            if ((rc = batch_flush(b, false))) return rc;
            continue;
        }
        const int m = (int)std::min<long long>(room, n - done);
        if ((rc = nfs_push_frames(c, host_frames + (size_t)done * c->g.HW, m))) return rc;
        done += m;
    }
    return b->err;
}

int nfs_batch_push_device(nfs_batch *b, const uint16_t *const *dev_frames, const int *n_frames)
{
    NvtxRange range("nfs_batch_push_device");
    int rc = batch_enter(b);
    if (rc) return rc;
    if (!dev_frames || !n_frames) return NFS_EINVAL;
    std::vector<long long> done((size_t)b->n, 0);
    for (int s = 0; s < b->n; ++s)
        if (n_frames[s] < 0 || (n_frames[s] > 0 && !dev_frames[s])) return NFS_EINVAL;
    for (;;) {
        bool left = false;
        for (int s = 0; s < b->n; ++s) {
            nfs_ctx *c = b->seq[s];
            const long long rem = n_frames[s] - done[s];
            if (rem <= 0) continue;
            left = true;
            const long long room = c->K - (c->nframes - c->nprocessed);
            if (room <= 0) continue;
            const int m = (int)std::min(room, rem);
            if ((rc = nfs_push_frames_device(c, dev_frames[s] + (size_t)done[s] * c->g.HW, m))) return rc;
            done[s] += m;
        }
        if (!left) break;
        // every member that still has frames now holds a full block: one launch for all of them
        if ((rc = batch_flush(b, false))) return rc;
    }
    return b->err;
}

int nfs_batch_structure_function(nfs_batch *b, int seq, double *D, int64_t *bin_counts, int64_t *pair_counts,
                                 double *q_mean)
{
    NvtxRange range("nfs_batch_structure_function");
    int rc = batch_enter(b);
    if (rc) return rc;
    if (seq < 0 || seq >= b->n) return NFS_EINVAL;
    if ((rc = batch_flush(b, true))) return rc;
    if ((rc = batch_check(b))) return rc;
    return nfs_structure_function(b->seq[seq], D, bin_counts, pair_counts, q_mean);
}

int nfs_batch_reset(nfs_batch *b)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    for (nfs_ctx *c : b->seq)
        if ((rc = nfs_reset(c))) return rc;
    return NFS_OK;
}

int nfs_batch_synchronize(nfs_batch *b)
{
    int rc = batch_enter(b);
    if (rc) return rc;
    return batch_check(b);
}

nfs_ctx *nfs_batch_member(nfs_batch *b, int seq) { return (b && seq >= 0 && seq < b->n) ? b->seq[seq] : nullptr; }

void *nfs_batch_get_stream(const nfs_batch *b) { return b ? (void *)b->stream : nullptr; }

int64_t nfs_batch_launch_count(const nfs_batch *b)
{
    if (!b) return -1;
    long long n = b->launches;
    for (nfs_ctx *c : b->seq) n += c->launches;
    return n;
}

const char *nfs_batch_last_error(const nfs_batch *b) { return b ? b->errmsg.c_str() : ""; }

// ---------------------------------------------------------------- regions of interest

// Frames cropped per launch: kRoiGroup frames of every window are cut from the full frames in one
// launch and pushed to the members as one device push.
constexpr int kRoiGroup = 64;

int nfs_roi_create(int H, int W, int n_roi, const int *y0, const int *x0, const int *h, const int *w,
                   const int32_t *delays, int n_delays, const int *n_qbins, nfs_batch **out)
{
    if (!out) return NFS_EINVAL;
    *out = nullptr;
    // n_roi bounds the crop launch's grid rows (65535)
    if (H <= 0 || W <= 0 || (W & 1) || n_roi <= 0 || n_roi > 65535 || !y0 || !x0 || !h || !w || !delays ||
        n_delays <= 0 || !n_qbins)
        return NFS_EINVAL;
    std::vector<RoiRect> rois((size_t)n_roi);
    long long off = 0, max_words = 0;
    for (int r = 0; r < n_roi; ++r) {
        if (y0[r] < 0 || x0[r] < 0 || h[r] <= 0 || w[r] <= 0 || (x0[r] & 1) || (w[r] & 1) || y0[r] > H - h[r] ||
            x0[r] > W - w[r])
            return NFS_EINVAL;
        const long long words = (long long)kRoiGroup * h[r] * (w[r] / 2);
        if (words >= (1LL << 31)) return NFS_EINVAL;  // the crop kernel's 32-bit indices
        const int rc_args = check_args(h[r], w[r], delays, n_delays, n_qbins[r], NFS_PATH_FUSED_F32, 0);
        if (rc_args) return rc_args;
        rois[(size_t)r] = RoiRect{y0[r], x0[r], h[r], w[r], off};
        off += (2 * words + 127) / 128 * 128;  // each window's frames start 256-byte aligned
        max_words = std::max(max_words, words);
    }
    std::vector<int> Hs((size_t)n_roi), Ws((size_t)n_roi), offs((size_t)n_roi + 1);
    std::vector<int32_t> dl((size_t)n_roi * n_delays);
    for (int r = 0; r < n_roi; ++r) {
        Hs[(size_t)r] = h[r];
        Ws[(size_t)r] = w[r];
        offs[(size_t)r] = r * n_delays;
        std::copy(delays, delays + n_delays, dl.begin() + (size_t)r * n_delays);
    }
    offs[(size_t)n_roi] = n_roi * n_delays;
    nfs_batch *b = nullptr;
    int rc = nfs_batch_create(n_roi, Hs.data(), Ws.data(), offs.data(), dl.data(), n_qbins, &b);
    if (rc) return rc;
    b->roi_H = H;
    b->roi_W = W;
    b->rois = rois;
    b->roi_max_words = max_words;
    if (cudaMalloc(&b->d_rois, sizeof(RoiRect) * rois.size()) != cudaSuccess ||
        cudaMalloc(&b->d_crop, sizeof(uint16_t) * (size_t)off) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return NFS_ENOMEM;
    }
    if (cudaMemcpy(b->d_rois, rois.data(), sizeof(RoiRect) * rois.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        batch_free(b);
        return NFS_ECUDA;
    }
    *out = b;
    return NFS_OK;
}

int nfs_roi_push_device(nfs_batch *b, const uint16_t *d, int n)
{
    NvtxRange range("nfs_roi_push_device");
    int rc = batch_enter(b);
    if (rc) return rc;
    if (b->rois.empty() || n < 0 || (n > 0 && !d) || (reinterpret_cast<uintptr_t>(d) & 3)) return NFS_EINVAL;
    const size_t HW = (size_t)b->roi_H * b->roi_W;
    std::vector<const uint16_t *> ptrs(b->rois.size());
    std::vector<int> counts(b->rois.size());
    for (long long done = 0; done < n;) {
        const int nc = (int)std::min<long long>(kRoiGroup, n - done);
        cudaError_t e = launch_roi_crop(d + (size_t)done * HW, b->roi_H, b->roi_W, nc, b->d_rois,
                                        (int)b->rois.size(), b->roi_max_words, b->n_sm, b->d_crop, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest crop");
        b->launches++;
        // the members' kernels read the crop buffer on the batch's stream, before the next crop
        for (size_t r = 0; r < b->rois.size(); ++r) {
            ptrs[r] = b->d_crop + b->rois[r].dst;
            counts[r] = nc;
        }
        if ((rc = nfs_batch_push_device(b, ptrs.data(), counts.data()))) return rc;
        done += nc;
    }
    return b->err;
}

int nfs_roi_push(nfs_batch *b, const uint16_t *host, int n)
{
    NvtxRange range("nfs_roi_push");
    int rc = batch_enter(b);
    if (rc) return rc;
    if (b->rois.empty() || n < 0 || (n > 0 && !host)) return NFS_EINVAL;
    if (n == 0) return NFS_OK;
    const size_t HW = (size_t)b->roi_H * b->roi_W;
    if (!b->d_full && cudaMalloc(&b->d_full, sizeof(uint16_t) * HW * kRoiGroup) != cudaSuccess) {
        cudaGetLastError();
        return NFS_ENOMEM;
    }
    const bool locked = is_page_locked(host);
    for (long long done = 0; done < n;) {
        const int nc = (int)std::min<long long>(kRoiGroup, n - done);
        // stream-ordered after the previous group's crop, which reads d_full
        cudaError_t e = copy_h2d(b->d_full, host + (size_t)done * HW, sizeof(uint16_t) * HW * nc, b->stream,
                                 locked, &b->launches);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest upload");
        if ((rc = nfs_roi_push_device(b, b->d_full, nc))) return rc;
        done += nc;
    }
    // page-locked sources are copied asynchronously: the caller's buffer is free once they are done
    if (locked) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "region-of-interest upload");
    }
    return b->err;
}

}  // extern "C"
