"""Seeded synthetic inputs for dynamic near-field-scattering (shadowgraph / DDM) sequences.

This module is shared by the oracle tests, the CUDA parity tests and the benchmark.  It only
*produces inputs* (camera frames, delay lists, workload shapes); it holds none of the analysis
arithmetic (no normalisation, no Fourier analysis of frames, no pair differences, no q binning).

Frame model (the test experiment of the paper: a static beam profile with a time-dependent
scattering contribution on top, recorded by a 12-bit CCD):

    i_t(x) = Poisson( P(x) * (1 + eps * phi_t(x)) ),  clipped to [0, 4095]

* P(x) is a Gaussian beam of peak P0 = 2000 counts and width sigma = 40 * min(H, W) / 128 px
  (40 px at 128x128), centred on the frame.  ``flat=True`` replaces it by the constant P0.
* phi_t is a real random field with unit spatial variance.  Its Fourier modes c_k(t) (half plane
  k_x >= 0) follow exact discrete Ornstein-Uhlenbeck steps

      c_k(t+1) = exp(-Gamma_k) c_k(t) + sqrt(S_k (1 - exp(-2 Gamma_k))) xi,   xi ~ CN(0, 1),

  started from the stationary law, with static spectrum S_k = 1 / (1 + (q/q0)^4) and relaxation
  rate Gamma_k = Dc q^2 + Gamma0, where q = 2 pi |f| rad/px and f is the mode frequency in
  cycles/px.  The DC mode is 0.  The k_x = 0 and k_x = W/2 columns are made Hermitian so the
  field is real; self-conjugate modes are real with variance S_k.  phi is the inverse transform
  scaled by the constant 1/sqrt(sum over the full plane of S_k), which gives unit variance in
  expectation (the scale does not change from frame to frame).

Random numbers are counter-based: every draw is a function of (seed, frame, stream, index) through
the Philox4x32-10 generator (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC 2011), written here in integer torch operations that are exact on every device.  A
source therefore gives the same frames on the CPU and on a GPU, and on x86 and Arm hosts: the
integer streams are identical, and the floating-point steps (Box-Muller normals, the OU update,
the inverse FFT, the Poisson sampler) differ between devices only in last-place rounding, which
changes a count only when a rate lands within ~1e-13 of a rounding edge (about one pixel in 1e12).
Shot noise is drawn with Hormann's transformed-rejection sampler PTRS (Insurance: Mathematics and
Economics 12, 1993) for rates of 10 and more, and by inversion of the CDF below that; every attempt
of every pixel has its own counter.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import torch

__all__ = [
    "log_delays",
    "Workload",
    "WORKLOADS",
    "RaggedWorkload",
    "RAGGED_WORKLOADS",
    "RoiWorkload",
    "ROI_WORKLOADS",
    "OUFrameSource",
    "uniform_frames",
    "travelling_cosine_frames",
    "beam_sigma",
    "ragged_shapes",
    "workload_source",
    "philox4x32",
    "complex_normals",
    "poisson_counts",
    "frame_checksums",
]


def log_delays(lo: int, hi: int, n: int) -> List[int]:
    """n strictly increasing integer delays spaced evenly on a log scale from lo to hi.

    d_j = max(d_{j-1} + 1, round_half_up(lo * (hi/lo)^(j/(n-1)))), d_{-1} = 0.  Small delays, where
    the log grid is denser than the integers, become consecutive integers; the list ends at hi.
    """
    if n <= 0:
        return []
    if n == 1:
        return [int(hi)]
    out: List[int] = []
    prev = 0
    for j in range(n):
        v = lo * (hi / lo) ** (j / (n - 1))
        d = max(prev + 1, int(math.floor(v + 0.5)))
        out.append(d)
        prev = d
    return out


def beam_sigma(H: int, W: int) -> float:
    """Beam width in px: 40 px at 128x128, scaled with the smaller frame side."""
    return 40.0 * min(H, W) / 128.0


@dataclasses.dataclass(frozen=True)
class Workload:
    """One analysis problem: N frames of H x W uint16, a delay list and n_qbins radial bins."""

    name: str
    N: int
    H: int
    W: int
    delays: tuple
    n_qbins: int
    Dc: float  # diffusion coefficient, px^2 / frame
    gamma0: float = 0.0  # q-independent rate, 1 / frame
    eps: float = 0.05  # fluctuation amplitude
    seed: int = 0

    @property
    def pair_total(self) -> int:
        return sum(max(0, self.N - t) for t in self.delays)

    def describe(self) -> str:
        return (f"{self.N} frames of {self.H}x{self.W} uint16, {len(self.delays)} delays "
                f"{self.delays[0]}..{self.delays[-1]}, {self.n_qbins} q bins")


WORKLOADS = {
    # 200 frames of 128x128, every delay 1..50, 64 bins, D = 0.5 px^2/frame.
    "ddm128": Workload("ddm128", 200, 128, 128, tuple(range(1, 51)), 64, 0.5, 0.0, 0.05, 12093363),
    # 1000 frames of 1024x1024, 100 log delays 1..500, 512 bins, D = 2 px^2/frame.
    "ddm1024": Workload("ddm1024", 1000, 1024, 1024, tuple(log_delays(1, 500, 100)), 512, 2.0, 0.0, 0.05,
                        12093364),
    # 4000 frames of 2048x2048, 200 log delays 1..2000, 1024 bins, Gamma = q^2 + 0.01.
    "ddm2048": Workload("ddm2048", 4000, 2048, 2048, tuple(log_delays(1, 2000, 200)), 1024, 1.0, 0.01, 0.05,
                        12093365),
    # The paper's largest-speed-up case: 2048 frames of 512x512 and every delay 1..2047 (all N - 1
    # delays, as the paper's program computes them), 256 bins, D = 1 px^2/frame.
    "paper512": Workload("paper512", 2048, 512, 512, tuple(range(1, 2048)), 256, 1.0, 0.0, 0.05, 12093368),
}


def _freq_grid(H: int, W: int, half: bool, dtype, device):
    fy = torch.fft.fftfreq(H, d=1.0, dtype=dtype, device=device)
    fx = (torch.fft.rfftfreq(W, d=1.0, dtype=dtype, device=device) if half
          else torch.fft.fftfreq(W, d=1.0, dtype=dtype, device=device))
    return torch.sqrt(fy[:, None] ** 2 + fx[None, :] ** 2)


# ------------------------------------------------------------------ counter-based random numbers

_MASK32 = 0xFFFFFFFF
_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57  # round multipliers of Philox4x32
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85  # Weyl key increments (golden ratio, sqrt(3) - 1)

# stream identifiers (third counter word; Poisson attempts add attempt << 8)
STREAM_INIT, STREAM_STEP, STREAM_SHOT = 0, 1, 2


def _mulhilo32(m: int, x: torch.Tensor):
    """(hi, lo) 32-bit halves of the 64-bit product m * x for uint32 values held in int64 tensors.

    x is split into 16-bit halves so that no partial product passes 2^49: int64 arithmetic stays
    exact (no overflow) on every device."""
    pl = (x & 0xFFFF) * m
    ph = (x >> 16) * m
    mid = pl + ((ph & 0xFFFF) << 16)
    return (ph >> 16) + (mid >> 32), mid & _MASK32


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Philox4x32 (10 rounds by default) of the counter (c0, c1, c2, c3) under the key (k0, k1).

    Counter words are int64 tensors (or ints) holding uint32 values, broadcast together; returns
    the four output words as int64 tensors in [0, 2^32).  Round: (hi0, lo0) = M0 c0, (hi1, lo1) =
    M1 c2, c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), then the key advances by (W0, W1)."""
    dev = next((v.device for v in (c0, c1, c2, c3) if isinstance(v, torch.Tensor)), torch.device("cpu"))
    c0, c1, c2, c3 = (v if isinstance(v, torch.Tensor) else torch.tensor(v, dtype=torch.int64, device=dev)
                      for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = torch.broadcast_tensors(c0, c1, c2, c3)
    shape = c0.shape
    k0 &= _MASK32
    k1 &= _MASK32

    def rounds_of(c0, c1, c2, c3):
        q0, q1 = k0, k1
        for r in range(rounds):
            if r:
                q0 = (q0 + _PHILOX_W0) & _MASK32
                q1 = (q1 + _PHILOX_W1) & _MASK32
            hi0, lo0 = _mulhilo32(_PHILOX_M0, c0)
            hi1, lo1 = _mulhilo32(_PHILOX_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ q0, lo1, hi0 ^ c3 ^ q1, lo0
        return c0, c1, c2, c3

    n = c0.numel()
    chunk = 1 << 18  # on the CPU, pieces that stay in cache across the ~300 element-wise steps
    if dev.type != "cpu" or n <= chunk:
        return rounds_of(c0, c1, c2, c3)
    flat = [v.reshape(-1) for v in (c0, c1, c2, c3)]
    outs = [torch.empty(n, dtype=torch.int64) for _ in range(4)]
    for o in range(0, n, chunk):
        res = rounds_of(*(v[o:o + chunk] for v in flat))
        for dst, r in zip(outs, res):
            dst[o:o + chunk] = r
    return tuple(v.reshape(shape) for v in outs)


def _unit(w: torch.Tensor, dtype) -> torch.Tensor:
    """(w + 1/2) / 2^32: a uint32 word as a uniform number strictly inside (0, 1) (exact in FP64)."""
    return (w.to(dtype) + 0.5) * (1.0 / 4294967296.0)


def _box_muller(w0, w1, dtype):
    """Two standard normal numbers from two uint32 words (Box and Muller, 1958)."""
    r = torch.sqrt(-2.0 * torch.log(_unit(w0, dtype)))
    th = (2.0 * math.pi) * _unit(w1, dtype)
    return r * torch.cos(th), r * torch.sin(th)


def complex_normals(n: int, t, stream: int, key: tuple, dtype, device) -> torch.Tensor:
    """n standard complex normal numbers CN(0, 1) (independent real and imaginary parts of
    variance 1/2) for each frame index in t (an int or a 1-D int64 tensor): [len(t), n] or [n].

    Element i comes from block i // 2 of the counter (block, t, stream, 0): words 0, 1 (even i) or
    2, 3 (odd i) through Box-Muller give its real and imaginary parts."""
    scalar = not isinstance(t, torch.Tensor)
    tt = torch.tensor([t], dtype=torch.int64, device=device) if scalar else t.to(device)
    blocks = torch.arange((n + 1) // 2, dtype=torch.int64, device=device)
    w0, w1, w2, w3 = philox4x32(blocks[None, :], tt[:, None], stream, 0, key[0], key[1])
    a0, a1 = _box_muller(w0, w1, dtype)
    b0, b1 = _box_muller(w2, w3, dtype)
    re = torch.stack((a0, b0), dim=-1).reshape(tt.numel(), -1)[:, :n]
    im = torch.stack((a1, b1), dim=-1).reshape(tt.numel(), -1)[:, :n]
    out = torch.complex(re, im) * math.sqrt(0.5)
    return out[0] if scalar else out


def _shot_words(pix: torch.Tensor, t: torch.Tensor, attempt: int, key: tuple):
    """Two uint32 words per (pixel, frame, attempt): pixels 2i and 2i+1 share the counter block
    (i, frame, STREAM_SHOT + (attempt << 8), 0) and take its words (0, 1) and (2, 3)."""
    w0, w1, w2, w3 = philox4x32(pix >> 1, t, STREAM_SHOT + (attempt << 8), 0, key[0], key[1])
    odd = (pix & 1).bool()
    return torch.where(odd, w2, w0), torch.where(odd, w3, w1)


def _shot_words_all(n: int, npix: int, t0: int, key: tuple, device):
    """The first attempt's two words of every pixel of frames t0 .. t0+n-1 (flat order), one
    counter block per pixel pair: the same values as _shot_words at attempt 0."""
    blocks = torch.arange(npix // 2, dtype=torch.int64, device=device)
    tt = torch.arange(t0, t0 + n, dtype=torch.int64, device=device)
    w0, w1, w2, w3 = philox4x32(blocks[None, :], tt[:, None], STREAM_SHOT, 0, key[0], key[1])
    wu = torch.stack((w0, w2), dim=-1).reshape(-1)
    wv = torch.stack((w1, w3), dim=-1).reshape(-1)
    return wu, wv


def poisson_counts(rate: torch.Tensor, t0: int, key: tuple) -> torch.Tensor:
    """Poisson samples of rate [n, H, W] (frames t0 .. t0+n-1), counter-based, as float values.

    Rates of 10 or more: PTRS, the transformed rejection with squeeze of Hormann (1993): with
    U uniform on (-1/2, 1/2), V uniform on (0, 1), us = 1/2 - |U|, b = 0.931 + 2.53 sqrt(lam),
    a = -0.059 + 0.02483 b, alpha = 1.1239 + 1.1328 / (b - 3.4), v_r = 0.9277 - 3.6224 / (b - 2):
    k = floor((2a/us + b) U + lam + 0.43) is accepted at once when us >= 0.07 and V <= v_r, rejected
    when k < 0 or (us < 0.013 and V > us), and otherwise accepted when
    log(V alpha / (a/us^2 + b)) <= -lam + k log(lam) - log(k!).  Rejected pixels draw again with the
    next attempt's counter.  Rates below 10: inversion of the CDF with one uniform.  Rate 0: 0."""
    n, H, W = rate.shape
    dev, dt = rate.device, rate.dtype
    lam = rate.reshape(-1)
    npix = H * W
    out = torch.zeros_like(lam)
    wu_all, wv_all = _shot_words_all(n, npix, t0, key, dev)
    big_mask = lam >= 10.0
    small = torch.nonzero((lam > 0.0) & ~big_mask).reshape(-1)
    everything = bool(big_mask.all())
    big = None if everything else torch.nonzero(big_mask).reshape(-1)
    attempt = 0
    while True:
        if attempt == 0:
            L = lam if everything else lam[big]
            wu = wu_all if everything else wu_all[big]
            wv = wv_all if everything else wv_all[big]
        else:
            if big.numel() == 0:
                break
            L = lam[big]
            wu, wv = _shot_words(big % npix, big // npix + t0, attempt, key)
        U = _unit(wu, dt) - 0.5
        V = _unit(wv, dt)
        us = 0.5 - torch.abs(U)
        b = 0.931 + 2.53 * torch.sqrt(L)
        a = -0.059 + 0.02483 * b
        k = torch.floor((2.0 * a / us + b) * U + L + 0.43)
        vr = 0.9277 - 3.6224 / (b - 2.0)
        acc = (us >= 0.07) & (V <= vr)
        # the full test only where the squeeze did not decide
        slow = torch.nonzero(~acc & ~((k < 0) | ((us < 0.013) & (V > us)))).reshape(-1)
        if slow.numel():
            Ls, ks, uss, bs, as_ = L[slow], k[slow], us[slow], b[slow], a[slow]
            alpha = 1.1239 + 1.1328 / (bs - 3.4)
            lhs = torch.log(V[slow] * alpha / (as_ / (uss * uss) + bs))
            rhs = -Ls + ks * torch.log(Ls) - torch.lgamma(ks + 1.0)
            acc[slow] = lhs <= rhs
        if attempt == 0 and everything:
            out = torch.where(acc, k, out)
            big = torch.nonzero(~acc).reshape(-1)
        else:
            idx = big
            out[idx[acc]] = k[acc]
            big = idx[~acc]
        attempt += 1
        if attempt > 200:
            raise RuntimeError("Poisson sampler did not converge")
    if small.numel():
        L = lam[small]
        u = _unit(wu_all[small], dt)
        k = torch.zeros_like(L)
        p = torch.exp(-L)
        F = p.clone()
        for i in range(1, 200):
            more = u > F
            if not bool(more.any()):
                break
            k = torch.where(more, k + 1.0, k)
            p = p * L / i
            F = torch.where(more, F + p, F)
        out[small] = k
    return out.reshape(n, H, W)


class OUFrameSource:
    """Sequential generator of frames following the model in the module docstring."""

    def __init__(self, H: int, W: int, Dc: float, gamma0: float = 0.0, q0: float = 0.1,
                 eps: float = 0.05, P0: float = 2000.0, sigma: Optional[float] = None,
                 flat: bool = False, shot_noise: bool = True, seed: int = 0,
                 device: str | torch.device = "cpu", dtype=torch.float64):
        if H % 2 or W % 2:
            raise ValueError("H and W must be even")
        self.H, self.W = H, W
        self.eps = float(eps)
        self.shot_noise = shot_noise
        self.device = torch.device(device)
        self.dtype = dtype
        cdtype = torch.complex128 if dtype == torch.float64 else torch.complex64
        self.cdtype = cdtype
        self.key = (int(seed) & _MASK32, (int(seed) >> 32) & _MASK32)

        q = 2.0 * math.pi * _freq_grid(H, W, True, dtype, self.device)
        S = 1.0 / (1.0 + (q / q0) ** 4)
        S[0, 0] = 0.0
        gamma = Dc * q * q + gamma0
        self.S = S
        self.gamma = gamma
        self.a = torch.exp(-gamma)
        self.b = torch.sqrt(S * (-torch.expm1(-2.0 * gamma)))
        qf = 2.0 * math.pi * _freq_grid(H, W, False, dtype, self.device)
        Sf = 1.0 / (1.0 + (qf / q0) ** 4)
        Sf[0, 0] = 0.0
        self.field_scale = 1.0 / math.sqrt(float(Sf.sum()))

        if flat:
            prof = torch.full((H, W), float(P0), dtype=dtype, device=self.device)
        else:
            s = beam_sigma(H, W) if sigma is None else float(sigma)
            y = torch.arange(H, dtype=dtype, device=self.device) - (H - 1) / 2.0
            x = torch.arange(W, dtype=dtype, device=self.device) - (W - 1) / 2.0
            prof = P0 * torch.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / (2.0 * s * s))
        self.profile = prof
        self.c = torch.sqrt(S) * self._cn(0, STREAM_INIT)[0]
        self.t = 0

    def _cn(self, t, stream: int) -> torch.Tensor:
        """CN(0, 1) values of every half-plane mode for frame index t (int or 1-D tensor): [n, H, W/2+1]."""
        shape = self.S.shape
        n = shape[0] * shape[1]
        v = complex_normals(n, t if isinstance(t, torch.Tensor) else torch.tensor([t], dtype=torch.int64),
                            stream, self.key, self.dtype, self.device)
        return v.reshape(-1, *shape).to(self.cdtype)

    def _hermitian(self, F: torch.Tensor) -> torch.Tensor:
        H, W = self.H, self.W
        F = F.clone()
        for col in (0, W // 2):
            c = F[..., :, col]
            lo = c[..., 1:H // 2]
            c[..., H // 2 + 1:] = torch.flip(lo, dims=[-1]).conj()
            for row in (0, H // 2):
                c[..., row] = math.sqrt(2.0) * c[..., row].real
        F[..., 0, 0] = 0
        return F

    def fields(self, n: int) -> torch.Tensor:
        """The next n unit-variance fields phi_t, shape [n, H, W] (advances the sequence).  The
        innovation of the step t -> t+1 is the STREAM_STEP draw of frame index t."""
        xi = self._cn(torch.arange(self.t, self.t + n, dtype=torch.int64), STREAM_STEP)
        cs = []
        for i in range(n):
            cs.append(self.c)
            self.c = self.a * self.c + self.b * xi[i]
            self.t += 1
        F = self._hermitian(torch.stack(cs))
        phi = torch.fft.irfft2(F, s=(self.H, self.W), norm="forward")
        return phi * self.field_scale

    def next_frames(self, n: int) -> torch.Tensor:
        """The next n frames as an int16-storage tensor [n, H, W] holding 12-bit counts (made a few
        frames at a time: the integer draws need ~150 bytes of temporaries per pixel)."""
        cap = (1 << 26) if self.device.type == "cuda" else (1 << 23)  # pixels per group (device memory is ample)
        g = max(1, cap // (self.H * self.W))
        if n > g:
            return torch.cat([self.next_frames(min(g, n - o)) for o in range(0, n, g)])
        t0 = self.t
        phi = self.fields(n)
        rate = self.profile * (1.0 + self.eps * phi)
        rate = torch.clamp(rate, min=0.0)
        if self.shot_noise:
            counts = poisson_counts(rate, t0, self.key)
        else:
            counts = torch.round(rate)
        counts = torch.clamp(counts, 0, 4095)
        return counts.to(torch.int16)

    def frames_numpy(self, n: int) -> np.ndarray:
        """The next n frames as a host uint16 array [n, H, W]."""
        return self.next_frames(n).cpu().numpy().view(np.uint16)


def uniform_frames(N: int, H: int, W: int, seed: int, lo: int = 1, hi: int = 4095) -> np.ndarray:
    """N frames of independent uniform integer counts in [lo, hi] (host uint16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=(N, H, W), dtype=np.uint16)


def travelling_cosine_frames(N: int, H: int, W: int, kx0: int, ky0: int, eps: float,
                             omega: float) -> np.ndarray:
    """Already-normalised FP64 frames n_t(x) = 1 + eps cos(2 pi (kx0 x / W + ky0 y / H) + omega t)."""
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    ph = 2.0 * np.pi * (kx0 * x / W + ky0 * y / H)
    return np.stack([1.0 + eps * np.cos(ph + omega * t) for t in range(N)])


def workload_source(w: Workload, device: str | torch.device = "cpu", dtype=torch.float64) -> OUFrameSource:
    """The frame source of a named workload (beam profile, shot noise, its own seed): the same frames
    on every device in FP64 (the default)."""
    return OUFrameSource(w.H, w.W, w.Dc, w.gamma0, eps=w.eps, seed=w.seed, device=device, dtype=dtype)


@dataclasses.dataclass(frozen=True)
class RaggedWorkload:
    """Many independent sequences of uneven frame shapes (regions of interest or cameras)."""

    name: str
    n_seq: int
    N: int  # frames per sequence
    seed: int

    def members(self):
        """[(H, W, Dc, delays, n_qbins, seed)] per sequence: shapes drawn uniformly from the six
        camera ROI shapes, D uniform in [0.1, 5] px^2/frame, 64 log delays 1..N/2, n_q = min(H, W)/2."""
        rng = np.random.Generator(np.random.PCG64(self.seed))
        shapes = ragged_shapes(self.n_seq, self.seed + 1)
        Ds = rng.uniform(0.1, 5.0, self.n_seq)
        d = tuple(log_delays(1, self.N // 2, 64))
        return [(h, w, float(Ds[i]), d, min(h, w) // 2, self.seed + 100 + i) for i, (h, w) in enumerate(shapes)]


RAGGED_WORKLOADS = {"ragged48": RaggedWorkload("ragged48", 48, 500, 12093367)}


@dataclasses.dataclass(frozen=True)
class RoiWorkload:
    """One camera sequence cut into a grid of equal regions of interest (spatially resolved
    analysis): every window is analysed as a sequence of its own, with one delay list."""

    name: str
    H: int
    W: int
    N: int
    grid: tuple  # (rows, cols) of windows
    delays: tuple
    n_qbins: int  # per window
    Dc: float
    seed: int

    def rois(self):
        """[(y0, x0, h, w)] row by row."""
        h, w = self.H // self.grid[0], self.W // self.grid[1]
        return [(r * h, c * w, h, w) for r in range(self.grid[0]) for c in range(self.grid[1])]


ROI_WORKLOADS = {"roi2048": RoiWorkload("roi2048", 2048, 2048, 1000, (4, 4), tuple(log_delays(1, 500, 100)), 256,
                                        2.0, 12093369)}


def ragged_shapes(n_seq: int, seed: int) -> Sequence[tuple]:
    """Frame shapes for a ragged batch, drawn uniformly from the six camera ROI shapes."""
    shapes = [(128, 128), (256, 256), (384, 512), (512, 512), (768, 1024), (1024, 1024)]
    rng = np.random.Generator(np.random.PCG64(seed))
    return [shapes[i] for i in rng.integers(0, len(shapes), size=n_seq)]


def frame_checksums(frames) -> np.ndarray:
    """Per-frame checksums of uint16 frames [n, H, W] (numpy or torch on any device): the sum of
    the counts and the sum of count x (pixel index mod 65521 + 1), as int64 [n, 2]; frames generated
    on two devices are compared with these instead of shipping the frames."""
    f = torch.as_tensor(frames) if not isinstance(frames, torch.Tensor) else frames
    n = f.shape[0]
    v = f.reshape(n, -1).to(torch.int64) & 0xFFFF
    wgt = (torch.arange(v.shape[1], dtype=torch.int64, device=v.device) % 65521) + 1
    return torch.stack((v.sum(dim=1), (v * wgt).sum(dim=1)), dim=1).cpu().numpy()
