"""Command-line analysis of a frame sequence stored on disk.

    python -m paper_1209_3362_gb300 FRAMES --delays log:1:2000:200 --bins 1024 --out result.npz

FRAMES is a .npy file of uint16 [N][H][W] (memory-mapped) or a raw uint16 file with --shape H W.
Delays: ``log:LO:HI:N`` (N log-spaced integer delays from LO to HI), ``range:LO:HI`` (every delay
LO..HI) or a comma-separated list.  ``--roi Y0 X0 H W`` (repeatable) analyses windows of the frames
instead of the whole frame; ``--max-ring-slots S`` runs the out-of-core bands when the ring for the
largest delay would not fit.  The output .npz holds, per analysed sequence, D [n_delays][n_bins],
q_mean (rad/px), tau, bin_counts and pair_counts.  Every step of the analysis runs in the CUDA
library; this module only reads the file and marshals arguments.
"""
from __future__ import annotations

import argparse
import sys
from typing import List

import numpy as np


def parse_delays(spec: str) -> List[int]:
    """``log:LO:HI:N``, ``range:LO:HI`` or ``d1,d2,...`` -> a strictly increasing list."""
    if spec.startswith("log:"):
        lo, hi, n = (int(v) for v in spec[4:].split(":"))
        out, prev = [], 0
        for j in range(n):
            v = lo * (hi / lo) ** (j / (n - 1)) if n > 1 else hi
            d = max(prev + 1, int(np.floor(v + 0.5)))
            out.append(d)
            prev = d
        return out
    if spec.startswith("range:"):
        lo, hi = (int(v) for v in spec[6:].split(":"))
        return list(range(lo, hi + 1))
    d = [int(v) for v in spec.split(",") if v.strip()]
    if not d or any(b <= a for a, b in zip(d, d[1:])):
        raise ValueError("delays must be a strictly increasing list")
    return d


def load_frames(path: str, shape=None) -> np.ndarray:
    if path.endswith(".npy"):
        a = np.load(path, mmap_mode="r")
    else:
        if not shape:
            raise ValueError("raw files need --shape H W")
        H, W = shape
        a = np.memmap(path, dtype=np.uint16, mode="r")
        if a.size % (H * W):
            raise ValueError("file size is not a whole number of H x W uint16 frames")
        a = a.reshape(-1, H, W)
    if a.dtype != np.uint16 or a.ndim != 3:
        raise ValueError("frames must be uint16 [N][H][W]")
    return a


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1209_3362_gb300", description=__doc__.split("\n\n")[0])
    ap.add_argument("frames")
    ap.add_argument("--shape", type=int, nargs=2, metavar=("H", "W"))
    ap.add_argument("--delays", required=True)
    ap.add_argument("--bins", type=int, required=True)
    ap.add_argument("--roi", type=int, nargs=4, action="append", metavar=("Y0", "X0", "H", "W"))
    ap.add_argument("--max-ring-slots", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=256, help="frames per push")
    ap.add_argument("--out", default="structure_function.npz")
    args = ap.parse_args(argv)

    import paper_1209_3362_gb300 as P

    frames = load_frames(args.frames, args.shape)
    N, H, W = frames.shape
    delays = parse_delays(args.delays)
    out = {"tau": np.asarray(delays, np.int64)}
    if args.roi:
        with P.NFSRoi(H, W, args.roi, delays, args.bins) as b:
            for o in range(0, N, args.chunk):
                b.push_frames(np.ascontiguousarray(frames[o:o + args.chunk]))
            for i in range(len(args.roi)):
                r = b.structure_function(i)
                for k in ("D", "q_mean", "bin_counts", "pair_counts"):
                    out[f"roi{i}_{k}"] = r[k]
    elif args.max_ring_slots:
        r = P.structure_function_out_of_core(np.ascontiguousarray(frames), delays, args.bins, args.max_ring_slots)
        for k in ("D", "q_mean", "bin_counts", "pair_counts"):
            out[k] = r[k]
    else:
        with P.NFS(H, W, delays, args.bins) as ctx:
            for o in range(0, N, args.chunk):
                ctx.push_frames(np.ascontiguousarray(frames[o:o + args.chunk]))
            r = ctx.structure_function()
        for k in ("D", "q_mean", "bin_counts", "pair_counts"):
            out[k] = r[k]
    np.savez(args.out, **out)
    print(f"{N} frames of {H}x{W}, {len(delays)} delays, {args.bins} bins -> {args.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
