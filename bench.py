#!/usr/bin/env python3
"""Benchmark: frames/s of the structure-function analysis of a synthetic NFS image sequence.

Default workload: 4000 frames of 2048x2048 uint16 (12-bit counts from the seeded OU beam model),
200 log-spaced delays 1..2000, 1024 radial q bins -- one "step" is the whole job: every frame
through the exact mean, the r2c FFT into the spectrum ring, the fused delay update of Eq. 1 and the
radial binning, ending with the binned D(q, tau) copied to the host.

  value     frames/s with the frames already resident in HBM (nfs_push_frames_device)
  e2e       frames/s through nfs_push_frames from pinned host memory (H2D inside the timed region)
  roofline  the fused delay kernel: algorithmic bytes per launch / its mean CUDA-event duration
  plain_f64 the plain unfused FP64 GPU path on the same frames (one pass), and the largest
            relative difference of its binned D from the fused FP32 path's
  cpu_baseline  the FP64 CPU oracle on a bounded sample of pairs of the same frames, extrapolated
            to the whole job by pair count
  stage_gbs, hbm_bound, pass_bound  each stage's algorithmic DRAM bytes over its time, and the
            frames/s of a pass bound by HBM alone or by the delay update's FP32 arithmetic plus
            the other stages' HBM traffic

--workload ragged48 (48 sequences of uneven shapes, one batch) and --workload roi2048 (2048x2048
frames cut into 16 regions of interest) time the batch paths with frames resident in HBM.
--impl reference times the FP64 CPU oracle alone (rank 0 only), each step a bounded sample.
Multi-GPU (torchrun, N > 1): the mode-slab split -- every rank takes all frames of the one sequence
but holds 1/N of the spectrum's modes (nfs_create_slab); the ranks' shares of the binned D are
summed by one all-reduce of n_delays x n_qbins doubles (gloo, host memory) inside the timed step:
strong scaling, value = frames of the sequence per second; the timing is the max over ranks.
--replicas instead runs an independent sequence per rank with no collective (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nfs_synth as S  # noqa: E402

METRIC = "frames/s at 2048²,200 delays (fused FP32 vs plain FP64, err≤2e-5); HBM % of peak"


def load_peaks():
    """(HBM GB/s, SM max MHz, source) from MEASURED_PEAKS.json, else the recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


FP32_LANES_PER_SM = 128      # FP32 lanes of a Blackwell SM
FLOPS_PER_PAIR_MODE = 6      # |P_t - P_s|^2 accumulated: 2 subtractions, 2 squares, 2 additions

# DRAM traffic of the fused delay kernel per algorithmic byte, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of a steady-state launch; see profiles/).  It
# applies only to the kernel source it was measured on: any change to these files voids it.
DELAY_KERNEL_SOURCES = ("paper_1209_3362_gb300/csrc/k_delay.cu", "paper_1209_3362_gb300/csrc/nfs_internal.cuh")
NCU_DELAY_CALIBRATION = {"sha256": "977ae1a322a26a3cc567a51471d406befaa099aa1c79e8ffe88099503fee14cc",
                         "dram_bytes_per_alg_byte": 0.9950}


def delay_kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for f in DELAY_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def delay_block_bytes(delays, N, K, M):
    """Algorithmic bytes of every fused delay launch of one pass over N frames in blocks of K:
    each distinct ring slot read once (8 B per mode), each active accumulator read and written once
    (2 x 8 B per mode).  Returns (total bytes, launches, pairs)."""
    d = np.asarray(delays, np.int64)
    total = 0
    launches = 0
    pairs = 0
    for t0 in range(0, N, K):
        nb = min(K, N - t0)
        t = np.arange(t0, t0 + nb)
        act = d[d <= t0 + nb - 1]
        slots = set(t.tolist())
        for tau in act:
            s = t[t >= tau] - tau
            slots.update(s.tolist())
            pairs += int(s.size)
        total += 8 * M * len(slots) + 16 * M * int(act.size)
        launches += 1
    return total, launches, pairs


def binned_modes(P, H, W, n_qbins, first=0, count=None):
    """Half-plane modes that fall in a radial bin (the modes whose D the job needs), among the
    column-major modes first .. first+count-1 (a slab's share; default all)."""
    b = P.bin_table(H, W, n_qbins)["bin_of_mode"].T.reshape(-1)  # mode kx * H + ky
    count = b.size if count is None else count
    return int(np.count_nonzero(b[first:first + count] >= 0))


def sample_shape(job_delays, target_pairs, n_max):
    """A bounded sample of the job for the oracle: its first n frames with the job's own delays
    below n (a prefix of its list), n the largest with at most target_pairs pairs (at least 2)."""
    n = 2
    while n < n_max:
        m = n + 1
        if sum(m - d for d in job_delays if d < m) > target_pairs:
            break
        n = m
    delays = [d for d in job_delays if d < n] or [1]
    return n, delays, sum(max(0, n - d) for d in delays)


def oracle_sample(frames_host, job_delays, budget_s, cores, repeats=1, warmup=0):
    """Time the FP64 oracle (all cores; its threads split the sample's pairs across delays) on a
    sample sized from a one-pair probe to about budget_s; returns (n, delays, pairs, seconds per run)."""
    import oracle
    oracle.build()
    t = time.perf_counter()
    oracle.structure_function(frames_host[:2], [1], 8, nthreads=1)
    per_pair = time.perf_counter() - t
    n, delays, pairs = sample_shape(job_delays, max(3, int(budget_s * cores / max(per_pair, 1e-6))),
                                    frames_host.shape[0])
    for _ in range(warmup):
        oracle.structure_function(frames_host[:n], delays, 8, nthreads=cores)
    times = []
    for _ in range(max(1, repeats)):
        t = time.perf_counter()
        oracle.structure_function(frames_host[:n], delays, 8, nthreads=cores)
        times.append(time.perf_counter() - t)
    return n, delays, pairs, times


def golden_parity(w, D, pair_counts, bin_counts, checksums):
    """Largest relative difference of D from the FP64 oracle's stored values for this workload
    (tests/golden/<workload>_oracle.npz, written by tests/golden/make_golden.py from the same
    seeded frames), or None when there is no fixture or the frames differ from it."""
    p = os.path.join(ROOT, "tests", "golden", f"{w.name}_oracle.npz")
    if not os.path.exists(p):
        return None
    z = np.load(p)
    if int(z["N"]) != w.N or int(z["H"]) != w.H or int(z["W"]) != w.W or int(z["seed"]) != w.seed:
        return None
    diff = int(np.count_nonzero(np.any(z["frame_checksums"] != checksums, axis=1)))
    idx = z["delay_index"]
    ref, got = z["D"], D[idx]
    m = (z["bin_counts"][None, :] > 0) & (z["pair_counts"][:, None] > 0)
    exact = bool(np.array_equal(bin_counts, z["bin_counts"]) and np.array_equal(pair_counts[idx], z["pair_counts"]))
    return {"max_rel_err": float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))), "delays_checked": int(idx.size),
            "counts_exact": exact, "frames_differing": diff, "fixture": os.path.relpath(p, ROOT)}


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest x over all ranks (every rank gets it); x itself on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, frames_per_rank: int, step_ms: float) -> float:
    """Whole-job frames/s: the frames all ranks processed over the slowest rank's step time."""
    return world * frames_per_rank / (step_ms / 1000.0)


def run_reference(args, w):
    """The FP64 CPU oracle alone, each step a bounded sample of the job (its first frames and its
    own delays below that count); rank 0 prints."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    src = S.workload_source(w, device="cpu")
    fr = src.frames_numpy(min(w.N, 40))
    n, delays, pairs, times = oracle_sample(fr, w.delays, args.ref_budget, cores, repeats=args.steps,
                                            warmup=max(args.warmup, 0))
    per_pair = sum(times) / (len(times) * pairs)
    value = w.N / (per_pair * w.pair_total)
    ms = 1000.0 * sum(times) / len(times)
    sample = (f"first {n} frames of {w.H}x{w.W} with the job's delays below {n} ({len(delays)} delays, {pairs} "
              f"pair FFTs) per step; extrapolated by pair count to the job's {w.pair_total} pairs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "frames": w.N, "H": w.H, "W": w.W, "delays": len(w.delays),
                       "tau_max": w.delays[-1], "n_qbins": w.n_qbins},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ddm2048", choices=sorted(S.WORKLOADS) + sorted(S.RAGGED_WORKLOADS) + sorted(S.ROI_WORKLOADS))
    ap.add_argument("--frames", type=int, default=0, help="override N (smaller runs; not a bench value)")
    ap.add_argument("--H", type=int, default=0, help="override frame height (profiling cases; not a bench value)")
    ap.add_argument("--W", type=int, default=0, help="override frame width (profiling cases; not a bench value)")
    ap.add_argument("--delays", type=int, default=0, help="use delays 1..n (profiling cases; not a bench value)")
    ap.add_argument("--delay-step", type=int, default=1,
                    help="with --delays n: delays step, 2 step, .., n step (isolated delays; profiling cases)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--delay-variant", type=int, default=0, help="fused delay kernel variant (0 = default)")
    ap.add_argument("--span", type=int, default=0, help="delay-kernel stage span (0 = choose by measurement)")
    ap.add_argument("--fft-chunk", type=int, default=0, help="frames per FFT launch (0 = choose by measurement)")
    ap.add_argument("--replicas", action="store_true", help="N > 1: independent sequences per rank (weak scaling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--h2d", choices=("sm", "ce"), default="sm",
                    help="end-to-end host pushes: read by the SMs (library default) or by the copy engines")
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=4.0, help="seconds of oracle work per reference step")
    args = ap.parse_args()
    if args.workload in S.RAGGED_WORKLOADS:
        return run_ragged(args, S.RAGGED_WORKLOADS[args.workload])
    if args.workload in S.ROI_WORKLOADS:
        return run_roi(args, S.ROI_WORKLOADS[args.workload])
    w = S.WORKLOADS[args.workload]
    if args.frames or args.H or args.W or args.delays:
        import dataclasses
        w = dataclasses.replace(w, N=args.frames or w.N, H=args.H or w.H, W=args.W or w.W,
                                delays=tuple(range(args.delay_step, args.delays * args.delay_step + 1, args.delay_step))
                                if args.delays else w.delays)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_1209_3362_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    gloo = None
    slabs = world > 1 and not args.replicas
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if slabs:
            gloo = dist.new_group(backend="gloo")  # the one exchange: bin shares in host memory

    def barrier():
        if dist is not None:
            dist.barrier()

    def ranks_max(x: float) -> float:
        return max_over_ranks(x, dist, "cuda")

    P.build()
    P.load_library()
    hbm_peak, sm_mhz, peak_src = load_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s

    # ---- inputs: the rank's own sequence, generated on its GPU, resident in HBM.  Rank 0 analyses
    # the workload's own seeded frames (the counter-based generator gives the same frames on the
    # CPU, where the oracle's stored values were computed); other ranks take other seeds.
    seed = w.seed if (slabs or rank == 0) else w.seed + 7919 * rank
    src = S.OUFrameSource(w.H, w.W, w.Dc, w.gamma0, eps=w.eps, seed=seed, device="cuda")
    frames = torch.empty((w.N, w.H, w.W), dtype=torch.int16, device="cuda")
    checksums = np.zeros((w.N, 2), np.int64)
    gb = 16
    t_gen = time.perf_counter()
    for o in range(0, w.N, gb):
        n = min(gb, w.N - o)
        frames[o:o + n] = src.next_frames(n)
        checksums[o:o + n] = S.frame_checksums(frames[o:o + n])
    del src
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    if slabs:
        ctx = P.NFS(w.H, w.W, w.delays, w.n_qbins, slab=rank, n_slabs=world)
    else:
        ctx = P.NFS(w.H, w.W, w.delays, w.n_qbins, path="f32", block_frames=args.block)
    if args.delay_variant:
        ctx.set_option(P.OPT_DELAY_VARIANT, args.delay_variant)
    if not args.delay_variant:
        ctx.set_option(P.OPT_DELAY_SPAN, args.span)  # 0: measured on this delay list (results do not change)
    ctx.set_option(P.OPT_FFT_CHUNK, args.fft_chunk)  # 0: frames per FFT launch measured for this shape
    K = ctx.get_option(P.OPT_BLOCK_FRAMES)
    ctx_span = ctx.get_option(P.OPT_DELAY_SPAN)
    ctx_chunk = ctx.get_option(P.OPT_FFT_CHUNK)
    M = ctx.get_option(P.OPT_SLAB_MODES)  # modes held (column-major, padded to 16-mode tiles; a slab's share)
    # modes the delay update keeps: the 16-mode tiles holding a binned mode (the corner modes beyond
    # the Nyquist circle are in no bin); its flops and bytes are counted on these
    M_delay = ctx.get_option(P.OPT_DELAY_MODES)
    # algorithmic flops count the binned modes (of this rank's slab) only; the kernel also updates
    # the corner modes that share a 16-mode tile with a binned one, which are not counted
    modes = binned_modes(P, w.H, w.W, w.n_qbins, ctx.get_option(P.OPT_SLAB_FIRST_MODE), M)
    # the pinned host copy for the end-to-end run, written by the CPU (as an acquisition program
    # writes frames into its buffer) through a small page-locked staging buffer.  The library's
    # host push reads it with the SMs (NFS_OPT_H2D = 0): the copy engines read the first ~4.6 GB of
    # such a 33.5 GB buffer 6-25x slower than the rest on every pass, wherever it was allocated,
    # while loads from the SMs read the same pages at full speed.
    host = None
    if not args.no_e2e:
        host = torch.empty((w.N, w.H, w.W), dtype=torch.int16, pin_memory=True)
        stg = torch.empty((64, w.H, w.W), dtype=torch.int16, pin_memory=True)
        for o in range(0, w.N, 64):
            n = min(64, w.N - o)
            stg[:n].copy_(frames[o:o + n])
            torch.cuda.synchronize()
            host[o:o + n].copy_(stg[:n])
        del stg
    stream = torch.cuda.ExternalStream(ctx.stream)

    def finish():
        r = ctx.structure_function()
        return P.reduce_slabs(r, group=gloo) if slabs else r

    def step():
        ctx.reset()
        ctx.push_frames_device(frames)
        return finish()

    for _ in range(max(args.warmup, 0)):
        step()
    # events around the delay-update launches only (the roofline's kernel); events around all
    # ~3000 launches of a pass would cost several per cent of the step
    ctx.set_option(P.OPT_TIMING, 2)
    ctx.reset_timings()
    l0 = ctx.launch_count
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        ev1.synchronize()
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launch_count - l0
    dev_ms = ev0.elapsed_time(ev1)
    step_ms = ranks_max(max(dev_ms, 1000.0 * wall) / args.steps)
    value = job_value(1 if slabs else world, w.N, step_ms)
    tim = ctx.timings()
    D32 = res["D"]

    # ---- roofline of the fused delay kernel (the dominant kernel)
    # Its arithmetic intensity (6 flops per pair and mode against each ring value and accumulator
    # moved once per block) lies above the FP32 ridge point, so the roofline that bounds it is the
    # FP32 ALU peak; the HBM fraction the metric asks for is reported beside it.
    alg_bytes, n_launch, pairs = delay_block_bytes(w.delays, w.N, K, M_delay)
    alg_flops = FLOPS_PER_PAIR_MODE * pairs * modes
    delay_ms, delay_n = tim["delay"]
    per_launch_ms = delay_ms / max(delay_n, 1)
    per_launch_s = per_launch_ms / 1000.0
    achieved = (alg_flops / n_launch) / per_launch_s / 1e12
    hbm_achieved = (alg_bytes / n_launch) / per_launch_s / 1e9
    cal = NCU_DELAY_CALIBRATION
    traffic = None
    if cal["sha256"] and cal["sha256"] == delay_kernel_sha():
        traffic = cal["dram_bytes_per_alg_byte"] * alg_bytes / n_launch
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic, "kernel": "k_delay_f32_tiled",
                "peak_source": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                "flops_per_launch": alg_flops / n_launch, "bytes_per_launch": alg_bytes / n_launch,
                "launch_ms": per_launch_ms, "launches": n_launch,
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                        "peak_source": f"{peak_src} hbm_gbs"}}
    # per-stage breakdown: one more pass with events around every launch (not part of the timed region)
    ctx.set_option(P.OPT_TIMING, 1)
    ctx.reset_timings()
    step()
    stage_ms = {k: v[0] for k, v in ctx.timings().items()}
    ctx.set_option(P.OPT_TIMING, 0)
    # Algorithmic DRAM bytes of every stage of a pass (frames read once by the sums and once by the
    # row pass, the row pass's half-spectrum scratch written once and read once by the column pass,
    # ring spectra written once, the delay update's ring slots and accumulators, the accumulators
    # read once by the binning; the reference image stays in L2), each stage's rate, and the frames/s
    # a pass moving only these bytes at the measured HBM peak would reach.
    scratch = w.H * (((w.W // 2 + 1) + 3) // 4 * 4) * 8
    stage_bytes = {"mean": w.N * w.H * w.W * 2, "rowfft": w.N * (w.H * w.W * 2 + scratch),
                   "colfft": w.N * (scratch + M * 8), "delay": alg_bytes, "bin": len(w.delays) * M_delay * 8}
    stage_gbs = {k: b / (stage_ms[k] / 1e3) / 1e9 for k, b in stage_bytes.items() if stage_ms.get(k)}
    pass_bytes = sum(stage_bytes.values())
    hbm_bound = {"bytes_per_step": pass_bytes, "frames_per_s": w.N / (pass_bytes / (hbm_peak * 1e9)),
                 "peak_gbs": hbm_peak}
    # the pass's own bound: the delay update at the FP32 peak, every other stage at the HBM peak
    bound_s = alg_flops / (fp32_peak * 1e12) + (pass_bytes - alg_bytes) / (hbm_peak * 1e9)
    pass_bound = {"ms_per_step": 1e3 * bound_s, "frames_per_s": w.N / bound_s}

    # ---- end to end from pinned host memory
    e2e = None
    if not args.no_e2e:
        del frames
        torch.cuda.empty_cache()
        frames = None
        ctx.set_option(P.OPT_TIMING, 0)
        ctx.set_option(P.OPT_H2D, 0 if args.h2d == "sm" else 1)

        def step_host():
            ctx.reset()
            ctx.push_frames(host)
            return finish()

        step_host()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        e2e_s = ranks_max((time.perf_counter() - t0) / args.steps)
        # one more (untimed) pass with the timeline trace: how the copies ran against the kernels
        ctx.set_option(P.OPT_TIMING, 3)
        ctx.reset_timings()
        step_host()
        tl = ctx.timeline()
        ctx.set_option(P.OPT_TIMING, 0)
        cp = [(a, b) for s_, a, b in tl if s_ == "h2d"]
        chunk_bytes = w.N * w.H * w.W * 2 / max(len(cp), 1)
        slow = [b - a for a, b in cp if chunk_bytes / ((b - a) / 1e3) / 1e9 < 100.0]
        e2e_trace = {"copies": len(cp), "copies_below_100gbs": len(slow),
                     "slow_copy_gb": round(len(slow) * chunk_bytes / 1e9, 2),
                     "median_copy_gbs": float(np.median([chunk_bytes / ((b - a) / 1e3) / 1e9 for a, b in cp])) if cp else None,
                     "first_delay_launch_ms": next((a for s_, a, b in tl if s_ == "delay"), None),
                     "last_copy_end_ms": max((b for a, b in cp), default=None),
                     "pass_end_ms": max((b for s_, a, b in tl), default=None)}
        e2e = {"value": job_value(1 if slabs else world, w.N, 1000.0 * e2e_s), "unit": "frames/s",
               "h2d_bytes_per_step": int(w.N * w.H * w.W * 2), "h2d": args.h2d, "trace": e2e_trace,
               "d2h_bytes_per_step": int(len(w.delays) * w.n_qbins * 8)}
        # the copy engines' rate from this process's page-locked buffer (1 GiB, alone on the GPU):
        # the end-to-end rate depends on it, and it varies with the box's state
        probe = host.view(-1)[: 1 << 29]
        dev = torch.empty_like(probe, device="cuda")
        dev.copy_(probe, non_blocking=True)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        dev.copy_(probe, non_blocking=True)
        p1.record()
        p1.synchronize()
        e2e["h2d_probe_gbs"] = probe.numel() * 2 / (p0.elapsed_time(p1) / 1e3) / 1e9
        del dev
    ctx.close()

    # ---- the plain unfused FP64 GPU path, one pass on the same frames
    plain = None
    if not args.no_f64 and rank == 0:
        if frames is None:
            frames = host.cuda() if e2e is not None else None
        c64 = P.NFS(w.H, w.W, w.delays, w.n_qbins, path="f64")
        s64 = torch.cuda.ExternalStream(c64.stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s64)
        c64.push_frames_device(frames)
        r64 = c64.structure_function()
        e1.record(s64)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        m = (r64["bin_counts"][None, :] > 0) & (r64["pair_counts"][:, None] > 0)
        err = float(np.max(np.abs(D32[m] - r64["D"][m]) / np.abs(r64["D"][m])))
        plain = {"value": job_value(1, w.N, ms64), "unit": "frames/s", "ms_per_pass": ms64,
                 "max_rel_err_f32_vs_f64": err}
        c64.close()

    # ---- CPU baseline: the FP64 oracle on a bounded sample of the same frames (rank 0)
    cpu = None
    if not args.no_cpu and rank == 0:
        if frames is None:
            frames = host.cuda()
        fh = frames[:64].cpu().numpy().view(np.uint16)
        cores = len(os.sched_getaffinity(0))
        n_s, d_s, p_s, ts = oracle_sample(fh, w.delays, args.cpu_budget, cores)
        dt = ts[0]
        cpu = {"value": w.N / (dt / p_s * w.pair_total), "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"first {n_s} frames with the job's delays below {n_s} ({len(d_s)} delays): {p_s} pair "
                         f"FFTs of {w.H}x{w.W} in {dt:.1f} s, extrapolated by pair count to {w.pair_total} pairs"}
    parity = golden_parity(w, D32, res["pair_counts"], res["bin_counts"], checksums) if rank == 0 else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
                "scaling": "strong" if slabs else ("weak" if world > 1 else "strong"),
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "frames": w.N, "H": w.H, "W": w.W, "delays": len(w.delays),
                           "tau_max": w.delays[-1], "n_qbins": w.n_qbins, "block_frames": K,
                           "delay_span": ctx_span, "fft_chunk": ctx_chunk,
                           "delay_modes": int(M_delay), "binned_modes": int(modes),
                           "parallelism": (f"mode-slabs{world}" if slabs else f"replicas{world}"),
                           "l2": "inputs larger than L2 (frames "
                           f"{w.N * w.H * w.W * 2 / 1e9:.1f} GB, ring "
                           f"{ctx_bytes(w, K, M) / 1e9:.1f} GB per rank)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk.summary(), "plain_f64_gpu": plain, "stage_ms_per_step": stage_ms,
                "stage_gbs": stage_gbs, "hbm_bound": hbm_bound, "pass_bound": pass_bound,
                "delay_pairs_per_step": pairs, "parity_vs_oracle": parity, "input_generation_s": t_gen}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_ragged(args, rw):
    """Ragged batch: every sequence's frames resident in HBM, one pass of all sequences per step
    through nfs_batch_push_device (one persistent delay launch per frame block for all members)."""
    import torch
    import paper_1209_3362_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    P.build()
    P.load_library()
    mem = rw.members()
    frames = []
    for (H, W, Dc, d, nq, seed) in mem:
        src = S.OUFrameSource(H, W, Dc, seed=seed, device="cuda", dtype=torch.float32)
        f = torch.empty((rw.N, H, W), dtype=torch.int16, device="cuda")
        for o in range(0, rw.N, 50):
            f[o:o + 50] = src.next_frames(min(50, rw.N - o))
        frames.append(f)
    torch.cuda.synchronize()
    b = P.NFSBatch([(m[0], m[1]) for m in mem], [m[3] for m in mem], [m[4] for m in mem])
    stream = torch.cuda.ExternalStream(b.stream)

    def step():
        b.reset()
        b.push_frames_device(frames)
        return [b.structure_function(s) for s in range(len(mem))]

    for _ in range(max(args.warmup, 0)):
        step()
    l0 = b.launch_count
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        wall = time.perf_counter() - t0
    step_ms = max(ev0.elapsed_time(ev1), 1000.0 * wall) / args.steps
    total = rw.n_seq * rw.N
    shapes = {}
    for m in mem:
        shapes[f"{m[0]}x{m[1]}"] = shapes.get(f"{m[0]}x{m[1]}", 0) + 1
    line = {"metric": f"frames/s, ragged batch of {rw.n_seq} sequences x {rw.N} frames (uneven shapes)",
            "value": total / (step_ms / 1000.0), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rw.name, "sequences": rw.n_seq, "frames_per_sequence": rw.N, "shapes": shapes,
                       "delays": 64, "tau_max": rw.N // 2},
            "gpu_launches": int(b.launch_count - l0), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    b.close()


def run_roi(args, rw):
    """Regions of interest: full camera frames resident in HBM, cut into a grid of windows by the
    library (nfs_roi_push_device), every window analysed as a sequence of its own."""
    import torch
    import paper_1209_3362_gb300 as P
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    P.build()
    P.load_library()
    src = S.OUFrameSource(rw.H, rw.W, rw.Dc, seed=rw.seed, device="cuda", dtype=torch.float32)
    frames = torch.empty((rw.N, rw.H, rw.W), dtype=torch.int16, device="cuda")
    for o in range(0, rw.N, 50):
        frames[o:o + 50] = src.next_frames(min(50, rw.N - o))
    torch.cuda.synchronize()
    rois = rw.rois()
    b = P.NFSRoi(rw.H, rw.W, rois, rw.delays, rw.n_qbins)
    stream = torch.cuda.ExternalStream(b.stream)

    def step():
        b.reset()
        b.push_frames_device(frames)
        return [b.structure_function(r) for r in range(len(rois))]

    for _ in range(max(args.warmup, 0)):
        step()
    l0 = b.launch_count
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        wall = time.perf_counter() - t0
    step_ms = max(ev0.elapsed_time(ev1), 1000.0 * wall) / args.steps
    h, w = rois[0][2], rois[0][3]
    line = {"metric": f"frames/s, {rw.H}x{rw.W} frames cut into {len(rois)} regions of interest of {h}x{w}",
            "value": rw.N / (step_ms / 1000.0), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rw.name, "frames": rw.N, "H": rw.H, "W": rw.W, "rois": len(rois),
                       "roi_shape": [h, w], "delays": len(rw.delays), "tau_max": rw.delays[-1],
                       "n_qbins": rw.n_qbins},
            "gpu_launches": int(b.launch_count - l0), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    b.close()


def ctx_bytes(w, K, M):
    return (w.delays[-1] + K) * M * 8


if __name__ == "__main__":
    main()
