"""FP64 reference of the Eq. 1 fit's loss and gradient (test infrastructure), and the closed-form
fit workload: 1024 bins x 200 log-spaced delays 1..500, known A, B, Gamma, 1 % multiplicative
noise, initial guesses at +-50 % of the truth."""
import numpy as np

import nfs_synth as S


def model(A, B, G, tau):
    return 2.0 * A[None, :] * (1.0 - np.exp(-G[None, :] * tau[:, None])) + 2.0 * B[None, :]


def loss_grad_fp64(A, B, G, D, tau):
    A, B, G, D, tau = (np.asarray(x, np.float64) for x in (A, B, G, D, tau))
    e = np.exp(-G[None, :] * tau[:, None])
    r = 2.0 * A[None, :] * (1.0 - e) + 2.0 * B[None, :] - D
    loss = np.sum(r * r, axis=0)
    gA = np.sum(4.0 * r * (1.0 - e), axis=0)
    gB = np.sum(4.0 * r, axis=0)
    gG = np.sum(4.0 * r * A[None, :] * tau[:, None] * e, axis=0)
    return loss, gA, gB, gG


def fit_workload(nq=1024, nd=200, seed=12093366, noise=0.01):
    rng = np.random.default_rng(seed)
    tau = np.asarray(S.log_delays(1, 500, nd), np.float64)
    A = 10.0 ** rng.uniform(2, 5, nq)
    B = A * 10.0 ** rng.uniform(-3, -1, nq)
    G = 10.0 ** rng.uniform(np.log10(0.01), np.log10(0.5), nq)
    D = model(A, B, G, tau) * (1.0 + noise * rng.standard_normal((nd, nq)))
    A0 = A * rng.uniform(0.5, 1.5, nq)
    B0 = B * rng.uniform(0.5, 1.5, nq)
    G0 = G * rng.uniform(0.5, 1.5, nq)
    return dict(tau=tau, A=A, B=B, G=G, D=D, A0=A0, B0=B0, G0=G0)
