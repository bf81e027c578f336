// Regions of interest: the crop of full camera frames into per-window frame sequences.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nfs {

// one region of interest of a frame: rows y0 .. y0+h, columns x0 .. x0+w; its frames start at
// element dst of the crop buffer
struct RoiRect {
    int y0, x0, h, w;
    long long dst;
};

// Window r of frame f (f < n) of the H x W frames src goes to dst + roi[r].dst + f*h*w.  W, x0 and
// w even, src 4-byte aligned, n*h*w/2 < 2^31 per window; max_words = the largest n*h*w/2.
cudaError_t launch_roi_crop(const uint16_t *src, int H, int W, int n, const RoiRect *d_roi, int n_roi,
                            long long max_words, int n_sm, uint16_t *dst, cudaStream_t s);

}  // namespace nfs
