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

Random numbers come from ``torch.Generator`` seeded per source, so a source gives the same frames
on every run on the same device type.  The same code runs on CPU and on CUDA (different streams).
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
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(int(seed))

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
        self.c = torch.sqrt(S) * self._cn(S.shape)
        self.t = 0

    def _cn(self, shape):
        return torch.randn(shape, dtype=self.cdtype, generator=self.gen, device=self.device)

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
        """The next n unit-variance fields phi_t, shape [n, H, W] (advances the sequence)."""
        cs = []
        for _ in range(n):
            cs.append(self.c)
            self.c = self.a * self.c + self.b * self._cn(self.c.shape)
            self.t += 1
        F = self._hermitian(torch.stack(cs))
        phi = torch.fft.irfft2(F, s=(self.H, self.W), norm="forward")
        return phi * self.field_scale

    def next_frames(self, n: int) -> torch.Tensor:
        """The next n frames as an int16-storage tensor [n, H, W] holding 12-bit counts."""
        phi = self.fields(n)
        rate = self.profile * (1.0 + self.eps * phi)
        rate = torch.clamp(rate, min=0.0)
        if self.shot_noise:
            counts = torch.poisson(rate, generator=self.gen)
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


def workload_source(w: Workload, device: str | torch.device = "cpu", dtype=None) -> OUFrameSource:
    """The frame source of a named workload (beam profile, shot noise, its own seed)."""
    if dtype is None:
        dtype = torch.float64 if torch.device(device).type == "cpu" else torch.float32
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
