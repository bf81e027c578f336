"""Differentiable per-bin fit of Eq. 1, D(q, tau) = 2 A(q) [1 - exp(-Gamma(q) tau)] + 2 B(q).

The loss and its gradient come from the library's CUDA kernel (nfs_fit_loss_grad); this module
only wraps it as a torch.autograd.Function and drives it with Adam or with the library's
Gauss-Newton kernel.  All tensors are CUDA float32: D [n_delays, n_bins], tau [n_delays],
parameters [n_bins].
"""
from __future__ import annotations

import ctypes

import torch

from . import NFS_OK, NFSError, load_library


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or None)


def _check_inputs(D, tau, *params):
    for t in (D, tau) + params:
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    nd, nq = D.shape
    assert tau.shape == (nd,) and all(p.shape == (nq,) for p in params)
    return nd, nq


def loss_and_grad(A, B, Gamma, D, tau):
    """Per-bin loss sum_j r_j^2 and its gradients (a single kernel launch)."""
    nd, nq = _check_inputs(D, tau, A, B, Gamma)
    loss = torch.empty_like(A)
    gA, gB, gG = torch.empty_like(A), torch.empty_like(A), torch.empty_like(A)
    rc = load_library().nfs_fit_loss_grad(_p(D), _p(tau), nd, nq, _p(A), _p(B), _p(Gamma), _p(loss), _p(gA),
                                          _p(gB), _p(gG), _stream())
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_fit_loss_grad")
    return loss, gA, gB, gG


class NFSFit(torch.autograd.Function):
    """loss[b] of Eq. 1's fit for parameters (A, B, Gamma); backward from the kernel's gradients."""

    @staticmethod
    def forward(ctx, A, B, Gamma, D, tau):
        loss, gA, gB, gG = loss_and_grad(A.detach().contiguous(), B.detach().contiguous(),
                                         Gamma.detach().contiguous(), D, tau)
        ctx.save_for_backward(gA, gB, gG)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        gA, gB, gG = ctx.saved_tensors
        return grad_loss * gA, grad_loss * gB, grad_loss * gG, None, None


def fit_gauss_newton(D, tau, A, B, Gamma, iters: int = 50, damping: float = 1e-3):
    """Damped Gauss-Newton in place on clones of A, B, Gamma; returns the fitted tensors."""
    A, B, Gamma = A.clone(), B.clone(), Gamma.clone()
    nd, nq = _check_inputs(D, tau, A, B, Gamma)
    rc = load_library().nfs_fit_gauss_newton(_p(D), _p(tau), nd, nq, _p(A), _p(B), _p(Gamma), int(iters),
                                             ctypes.c_float(damping), _stream())
    if rc != NFS_OK:
        raise NFSError(rc, "nfs_fit_gauss_newton")
    return A, B, Gamma


def fit_adam(D, tau, A0, B0, Gamma0, steps: int = 500, lr: float = 1e-2):
    """Adam through NFSFit on u with theta = theta0 (1 + u) (scale-free steps); clamps A, B >= 0,
    Gamma > 0.  Returns the fitted tensors and the final per-bin loss."""
    u = torch.zeros((3,) + A0.shape, device=A0.device, dtype=torch.float32, requires_grad=True)
    opt = torch.optim.Adam([u], lr=lr)
    base = torch.stack([A0, B0, Gamma0])
    for _ in range(steps):
        opt.zero_grad()
        th = base * (1.0 + u)
        loss = NFSFit.apply(th[0].clamp(min=0), th[1].clamp(min=0), th[2].clamp(min=1e-12), D, tau)
        loss.sum().backward()
        opt.step()
    with torch.no_grad():
        th = base * (1.0 + u)
        A, B, G = th[0].clamp(min=0), th[1].clamp(min=0), th[2].clamp(min=1e-12)
        loss, *_ = loss_and_grad(A.contiguous(), B.contiguous(), G.contiguous(), D, tau)
    return A, B, G, loss
