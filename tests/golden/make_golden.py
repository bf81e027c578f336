#!/usr/bin/env python3
"""Writes the FP64 oracle's binned structure function of a full-size named workload (test
infrastructure: it calls only the oracle in ``oracle/`` and the seeded generator ``nfs_synth``).

The frames are the workload's own (``nfs_synth.workload_source``: counter-based draws, FP64, the
same frames on any device), generated on the CPU.  For every delay of the chosen subset the oracle
forms every real-space difference n_t - n_{t+tau} (t + tau < N), transforms it and bins
|Delta I|^2 (Eq. 1 averaged over all pairs at that delay, azimuthal average of Fig. 1e,f).  The
output ``<workload>_oracle.npz`` holds the delays and their indices in the workload's list, D
[n_subset][n_q], the bin and pair counts, q_mean, per-frame checksums of the generated frames (the
GPU test regenerates the frames and compares these first) and how the file was made.

  python tests/golden/make_golden.py ddm1024                # every delay
  python tests/golden/make_golden.py ddm2048 --every 10     # every 10th delay and the last

--checkpoint DIR keeps one file per finished delay so that an interrupted run resumes.
"""
from __future__ import annotations

import argparse
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import nfs_synth as S  # noqa: E402
import oracle  # noqa: E402


def subset_indices(nd: int, every: int):
    """Indices 0, every, 2 every, ... of a list of nd delays, and always the last one."""
    idx = list(range(0, nd, every))
    if idx[-1] != nd - 1:
        idx.append(nd - 1)
    return idx


def generate(w, batch: int = 16):
    """The workload's frames [N][H][W] uint16 on the CPU and their checksums [N][2]."""
    frames = np.empty((w.N, w.H, w.W), np.uint16)
    sums = np.empty((w.N, 2), np.int64)
    src = S.workload_source(w, device="cpu")
    t0 = time.time()
    for o in range(0, w.N, batch):
        n = min(batch, w.N - o)
        f = src.next_frames(n)
        frames[o:o + n] = f.numpy().view(np.uint16)
        sums[o:o + n] = S.frame_checksums(f)
        if (o // batch) % 25 == 0:
            print(f"  frames {o + n}/{w.N} ({time.time() - t0:.0f} s)", flush=True)
    return frames, sums


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(S.WORKLOADS))
    ap.add_argument("--every", type=int, default=1, help="take every n-th delay (and the last)")
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: every core of this process)")
    ap.add_argument("--checkpoint", default="", help="directory for per-delay partial results")
    ap.add_argument("--out", default="", help="output file (default tests/golden/<workload>_oracle.npz)")
    args = ap.parse_args()
    w = S.WORKLOADS[args.workload]
    idx = subset_indices(len(w.delays), max(1, args.every))
    delays = [w.delays[j] for j in idx]
    threads = args.threads or len(os.sched_getaffinity(0))
    oracle.build()
    print(f"{w.describe()}: {len(idx)} delays, {sum(max(0, w.N - d) for d in delays)} pairs, "
          f"{threads} threads", flush=True)
    t_gen = time.time()
    frames, sums = generate(w)
    t_gen = time.time() - t_gen
    if args.checkpoint:
        os.makedirs(args.checkpoint, exist_ok=True)
    D = np.zeros((len(idx), w.n_qbins), np.float64)
    pairs = np.zeros(len(idx), np.int64)
    counts = qmean = None
    t_or = time.time()
    for i, (j, tau) in enumerate(zip(idx, delays)):
        ck = os.path.join(args.checkpoint, f"{w.name}_j{j}.npz") if args.checkpoint else ""
        if ck and os.path.exists(ck):
            z = np.load(ck)
            if np.array_equal(z["sums"], sums):
                D[i], pairs[i], counts, qmean = z["D"], int(z["pairs"]), z["bin_counts"], z["q_mean"]
                print(f"  delay {tau} (index {j}): from checkpoint", flush=True)
                continue
        t = time.time()
        r = oracle.structure_function(frames, [tau], w.n_qbins, nthreads=threads)
        D[i], pairs[i], counts, qmean = r["D"][0], r["pair_counts"][0], r["bin_counts"], r["q_mean"]
        if ck:
            np.savez(ck + ".tmp.npz", D=D[i], pairs=pairs[i], bin_counts=counts, q_mean=qmean, sums=sums)
            os.replace(ck + ".tmp.npz", ck)
        print(f"  delay {tau} (index {j}): {pairs[i]} pairs in {time.time() - t:.0f} s", flush=True)
    t_or = time.time() - t_or
    out = args.out or os.path.join(HERE, f"{w.name}_oracle.npz")
    np.savez_compressed(
        out, workload=w.name, N=w.N, H=w.H, W=w.W, seed=w.seed, Dc=w.Dc, gamma0=w.gamma0, eps=w.eps,
        n_qbins=w.n_qbins, delays_all=np.asarray(w.delays, np.int32), delay_index=np.asarray(idx, np.int32),
        delays=np.asarray(delays, np.int32), D=D, bin_counts=counts, pair_counts=pairs, q_mean=qmean,
        frame_checksums=sums,
        made_by=(f"tests/golden/make_golden.py {w.name} --every {args.every}: FP64 oracle (real-space "
                 f"differences), {threads} threads on {platform.machine()}; frames {t_gen:.0f} s, "
                 f"oracle {t_or:.0f} s"))
    print(f"wrote {out}", flush=True)


if __name__ == "__main__":
    main()
