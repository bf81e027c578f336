// Out-of-core delay bands (nfs_out_of_core_plan, nfs_structure_function_out_of_core) and the
// export of the fused delay kernel's copy schedule (nfs_delay_schedule).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "nfs_host.cuh"

using namespace nfs;
using namespace nfs::host;

// ------------------------------------------------------------------ out-of-core bands
//
// When the ring for every delay does not fit, the delays are split into bands processed one after
// the other, each re-reading the frames from host memory (the paper's FIFO re-upload, organised
// by delay bands).  Band 0 is an ordinary pass over the delays d with d + K <= the slot budget.
// A later band with smallest delay lo takes the shift s = floor(lo / K) K and runs a cross pass:
// current sequence C_u = frame u + s (K-slot ring), old sequence O_u = frame u (ring of
// e_max + K slots), delays e = d - s, so the pair (C_u, O_{u-e}) is the pair (u + s, u + s - d).
// The block boundaries of C fall on multiples of K in the original frame index (s is a multiple
// of K), so every pair is added in the same block and warp as in one in-core pass.

namespace {

// One band: delays [first, last) of the list, shift s (s = 0: the ordinary pass).
struct Band {
    int first, last;
    long long shift;
};

// Does the tiled kernel's schedule of these (shifted) delays fit its parameter space?
bool schedule_fits(const std::vector<int> &d, bool cross)
{
    std::vector<SubRun> srs;
    std::vector<Stage> sts;
    if (!build_delay_schedule(d.data(), (int)d.size(), cross, &srs, &sts)) return false;
    return srs.size() <= (size_t)kMaxSubRuns && sts.size() <= (size_t)kMaxSchedStages;
}

int plan_bands(const int32_t *delays, int nd, long long N, long long max_slots, std::vector<Band> *bands,
               long long *n_transforms)
{
    bands->clear();
    *n_transforms = 0;
    const long long K = kDefaultBlock;
    int j = 0;
    while (j < nd) {
        const long long lo = delays[j];
        const bool first = bands->empty();
        // band 0 runs in place when its first delay fits; later bands are cross passes
        const bool in_place = first && lo + K <= max_slots;
        const long long s = in_place ? 0 : lo / K * K;
        const long long hi_max = in_place ? max_slots - K : max_slots - 2 * K + s;
        // a cross pass needs its first delay within the budget (always so for budgets of 3K slots)
        if (!in_place && (lo < K || lo > hi_max)) return NFS_EINVAL;
        int e = j;
        while (e < nd && delays[e] <= hi_max) ++e;
        // keep the band within the tiled kernel's schedule limits
        for (;;) {
            std::vector<int> d;
            for (int q = j; q < e; ++q) d.push_back((int)(delays[q] - s));
            if (schedule_fits(d, !in_place)) break;
            e = j + (e - j) / 2;
            if (e == j) return NFS_EUNSUPPORTED;
        }
        bands->push_back({j, e, s});
        if (in_place)
            *n_transforms += N;
        else if (N > s)
            *n_transforms += 2 * (N - s);
        j = e;
    }
    return NFS_OK;
}

// A cross pass over host frames: old sequence `old` and current sequence `cur`, n frames each
// (pinned or pageable; read before the call returns).
int cross_push(nfs_ctx *c, const uint16_t *cur, const uint16_t *old, long long n)
{
    const bool locked = is_page_locked(cur) && is_page_locked(old);
    if (!locked && !c->h_stage[0]) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaMallocHost((void **)&c->h_stage[i], c->frame_bytes() * (size_t)c->copy_frames);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return NFS_ENOMEM;
            }
        }
    }
    // copy nc frames from src into the next staging slot; returns the slot
    auto stage = [&](const uint16_t *src, int nc, int *slot_out) -> int {
        const int slot = (int)(c->stage_i++ % c->n_slots);
        uint16_t *dst = c->d_stage + (size_t)slot * c->copy_frames * c->g.HW;
        const size_t bytes = c->frame_bytes() * (size_t)nc;
        CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[slot], 0));
        int hs = -1;
        if (!locked) {
            hs = (int)(c->hstage_i++ & 1);
            CK(c, cudaEventSynchronize(c->ev_hcopied[hs]));
            memcpy(c->h_stage[hs], src, bytes);
            src = c->h_stage[hs];
        }
        const int rc = timed(c, NFS_STAGE_H2D, c->copy_stream, [&] {
            return copy_h2d(dst, src, bytes, c->copy_stream, c->h2d == 0, &c->launches);
        }, "h2d");
        if (rc) return rc;
        if (hs >= 0) CK(c, cudaEventRecord(c->ev_hcopied[hs], c->copy_stream));
        CK(c, cudaEventRecord(c->ev_filled[slot], c->copy_stream));
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_filled[slot], 0));
        *slot_out = slot;
        return NFS_OK;
    };
    long long done = 0;
    int last = -1;
    while (done < n) {
        const int nc = (int)std::min<long long>(c->copy_frames, n - done);
        int so = 0, sc = 0, rc;
        if ((rc = stage(old + (size_t)done * c->g.HW, nc, &so))) return rc;
        if ((rc = stage(cur + (size_t)done * c->g.HW, nc, &sc))) return rc;
        const uint16_t *dold = c->d_stage + (size_t)so * c->copy_frames * c->g.HW;
        const uint16_t *dcur = c->d_stage + (size_t)sc * c->copy_frames * c->g.HW;
        // the old sequence's first frame (frame 0) gives the reference image
        if ((rc = frame_sums(c, dold, nc, c->d_sums))) return rc;
        if ((rc = frame_sums(c, dcur, nc, c->d_sums + kMaxChunk))) return rc;
        for (int o = 0; o < nc;) {
            const int nf = next_chunk(c, nc - o, c->fft_chunk);
            if ((rc = process_chunk(c, dold + (size_t)o * c->g.HW, nf, true, c->d_sums + o))) return rc;
            if ((rc = process_chunk(c, dcur + (size_t)o * c->g.HW, nf, false, c->d_sums + kMaxChunk + o))) return rc;
            o += nf;
        }
        CK(c, cudaEventRecord(c->ev_free[so], c->stream));
        CK(c, cudaEventRecord(c->ev_free[sc], c->stream));
        done += nc;
        last = sc;
    }
    if (locked && last >= 0) CK(c, cudaEventSynchronize(c->ev_filled[last]));
    return c->err;
}

}  // namespace

extern "C" {

int nfs_out_of_core_plan(const int32_t *delays, int n_delays, int64_t n_frames, int64_t max_ring_slots,
                         int32_t *band_first, int64_t *band_shift, int *n_bands, int64_t *n_transforms)
{
    if (!delays || n_delays <= 0 || n_frames < 0 || !n_bands || !n_transforms) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<Band> bands;
    long long nt = 0;
    const int rc = plan_bands(delays, n_delays, n_frames, max_ring_slots, &bands, &nt);
    if (rc) return rc;
    *n_bands = (int)bands.size();
    *n_transforms = nt;
    for (size_t b = 0; b < bands.size(); ++b) {
        if (band_first) band_first[b] = bands[b].first;
        if (band_shift) band_shift[b] = bands[b].shift;
    }
    if (band_first) band_first[bands.size()] = n_delays;
    return NFS_OK;
}

int nfs_structure_function_out_of_core(int H, int W, const int32_t *delays, int n_delays, int n_qbins,
                                       const uint16_t *frames, int64_t n_frames, int64_t max_ring_slots, double *D,
                                       int64_t *bin_counts, int64_t *pair_counts, double *q_mean,
                                       int64_t *n_transforms)
{
    NvtxRange range("nfs_structure_function_out_of_core");
    if (!delays || n_delays <= 0 || n_qbins <= 0 || !D || !bin_counts || !pair_counts) return NFS_EINVAL;
    if (n_frames < 0 || n_frames > kMaxFrames || (n_frames > 0 && !frames)) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<Band> bands;
    long long planned = 0;
    int rc = plan_bands(delays, n_delays, n_frames, max_ring_slots, &bands, &planned);
    if (rc) return rc;
    const size_t HW = (size_t)H * W;
    long long done = 0;
    std::vector<double> Db;
    std::vector<int64_t> pc;
    for (const Band &b : bands) {
        const int nb = b.last - b.first;
        std::vector<int32_t> d(delays + b.first, delays + b.last);
        for (int32_t &x : d) x -= (int32_t)b.shift;
        nfs_ctx *c = nullptr;
        rc = create_impl(H, W, d.data(), nb, n_qbins, NFS_PATH_FUSED_F32, 0, &c, b.shift > 0);
        if (rc) return rc;
        Db.assign((size_t)nb * n_qbins, 0.0);
        pc.assign((size_t)nb, 0);
        if (b.shift == 0)
            rc = n_frames > 0 ? nfs_push_frames(c, frames, (int)n_frames) : NFS_OK;
        else if (n_frames > b.shift)
            rc = cross_push(c, frames + (size_t)b.shift * HW, frames, n_frames - b.shift);
        if (!rc) rc = nfs_structure_function(c, Db.data(), bin_counts, pc.data(), q_mean);
        done += c->transforms;
        nfs_destroy(c);
        if (rc) return rc;
        std::copy(Db.begin(), Db.end(), D + (size_t)b.first * n_qbins);
        for (int q = 0; q < nb; ++q) pair_counts[b.first + q] = n_frames > b.shift ? pc[q] : 0;
    }
    if (done != planned) return NFS_ESTATE;  // the passes transformed other frames than planned
    if (n_transforms) *n_transforms = done;
    return NFS_OK;
}

}  // extern "C"

extern "C" int nfs_delay_schedule(const int32_t *delays, int n_delays, int cross, int32_t *subruns, int32_t *stages,
                                  int max_entries, int *n_subruns, int *n_stages, int *block_frames,
                                  int *slot_rows, int *copy_barriers, int span)
{
    if (!delays || n_delays <= 0 || !n_subruns || !n_stages) return NFS_EINVAL;
    if (span != 0 && (span < kMinSpan || span > kMaxSpan)) return NFS_EINVAL;
    for (int j = 0; j < n_delays; ++j)
        if (delays[j] < 0 || delays[j] > kMaxDelay || (j && delays[j] <= delays[j - 1])) return NFS_EINVAL;
    std::vector<SubRun> srs;
    std::vector<Stage> sts;
    if (!build_delay_schedule(delays, n_delays, cross != 0, &srs, &sts, span ? span : kDefaultSpan))
        return NFS_EUNSUPPORTED;
    *n_subruns = (int)srs.size();
    *n_stages = (int)sts.size();
    if (block_frames) *block_frames = kDelayBlock;
    if (slot_rows) *slot_rows = kSlotBuf;
    if (copy_barriers) *copy_barriers = kFullBars;
    if ((subruns && (int)srs.size() > max_entries) || (stages && (int)sts.size() > max_entries)) return NFS_ETOOBIG;
    for (size_t i = 0; subruns && i < srs.size(); ++i) {
        subruns[3 * i] = srs[i].j0;
        subruns[3 * i + 1] = srs[i].len;
        subruns[3 * i + 2] = srs[i].d0;
    }
    for (size_t i = 0; stages && i < sts.size(); ++i) {
        stages[5 * i] = sts[i].sr0;
        stages[5 * i + 1] = sts[i].nsr;
        stages[5 * i + 2] = sts[i].lo;
        stages[5 * i + 3] = sts[i].hi;
        stages[5 * i + 4] = sts[i].need;
    }
    return NFS_OK;
}
