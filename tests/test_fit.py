"""The Eq. 1 fit: the FP64 reference gradient is pinned to finite differences on the CPU; the CUDA
loss/gradient kernel is checked against it and against central finite differences (h = 1e-3,
relative), Gauss-Newton must recover the known parameters from +-50 % starts, and Adam through
the autograd Function must reduce the loss."""
import numpy as np
import pytest

from fit_reference import fit_workload, loss_grad_fp64


def test_fp64_reference_gradient_matches_finite_differences():
    w = fit_workload(nq=16, nd=40)
    A, B, G = w["A0"], w["B0"], w["G0"]
    l0, gA, gB, gG = loss_grad_fp64(A, B, G, w["D"], w["tau"])
    for name, g, idx in (("A", gA, 0), ("B", gB, 1), ("G", gG, 2)):
        p = [A.copy(), B.copy(), G.copy()]
        h = 1e-6 * p[idx]
        p_hi = [x.copy() for x in p]
        p_lo = [x.copy() for x in p]
        p_hi[idx] += h
        p_lo[idx] -= h
        fd = (loss_grad_fp64(*p_hi, w["D"], w["tau"])[0] - loss_grad_fp64(*p_lo, w["D"], w["tau"])[0]) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9 * np.abs(g).max(), err_msg=name)


@pytest.mark.gpu
def test_fit_kernel_gradients():
    import torch
    import paper_1209_3362_gb300 as P
    from paper_1209_3362_gb300 import fit as F
    P.build()
    w = fit_workload()
    dev = lambda x: torch.tensor(np.asarray(x, np.float32), device="cuda").contiguous()
    D, tau = dev(w["D"]), dev(w["tau"])
    A, B, G = dev(w["A0"]), dev(w["B0"]), dev(w["G0"])
    loss, gA, gB, gG = F.loss_and_grad(A, B, G, D, tau)
    rl, rA, rB, rG = loss_grad_fp64(A.cpu().numpy(), B.cpu().numpy(), G.cpu().numpy(), D.cpu().numpy().astype(np.float64),
                                    tau.cpu().numpy())
    for got, ref in ((loss, rl), (gA, rA), (gB, rB), (gG, rG)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref) / (np.abs(ref) + 1e-6 * np.abs(ref).max())) < 2e-3
    # central finite differences (h = 1e-3 relative) of the loss, evaluated in FP64 so that the
    # difference quotient is not swamped by FP32 rounding of a large loss
    Dn, tn = D.cpu().numpy().astype(np.float64), tau.cpu().numpy().astype(np.float64)
    p = [x.cpu().numpy().astype(np.float64) for x in (A, B, G)]
    for idx, g in enumerate((gA, gB, gG)):
        h = 1e-3 * p[idx]
        hi = [x.copy() for x in p]
        lo = [x.copy() for x in p]
        hi[idx] += h
        lo[idx] -= h
        fd = (loss_grad_fp64(*hi, Dn, tn)[0] - loss_grad_fp64(*lo, Dn, tn)[0]) / (2 * h)
        g = g.cpu().numpy().astype(np.float64)
        rel = np.abs(fd - g) / (np.abs(g) + 1e-4 * np.abs(g).max())
        assert np.quantile(rel, 0.99) < 1e-3 and rel.max() < 1e-2, (idx, np.quantile(rel, 0.99), rel.max())
    # the autograd Function returns the same gradients
    Ar, Br, Gr = (x.clone().requires_grad_() for x in (A, B, G))
    F.NFSFit.apply(Ar, Br, Gr, D, tau).sum().backward()
    assert torch.equal(Ar.grad, gA) and torch.equal(Br.grad, gB) and torch.equal(Gr.grad, gG)


@pytest.mark.gpu
def test_gauss_newton_and_adam_recover_the_truth():
    import torch
    import paper_1209_3362_gb300 as P
    from paper_1209_3362_gb300 import fit as F
    P.build()
    w = fit_workload()
    dev = lambda x: torch.tensor(np.asarray(x, np.float32), device="cuda").contiguous()
    D, tau = dev(w["D"]), dev(w["tau"])
    A, B, G = F.fit_gauss_newton(D, tau, dev(w["A0"]), dev(w["B0"]), dev(w["G0"]), iters=100)
    for got, truth, tol in ((A, w["A"], 0.02), (G, w["G"], 0.03)):
        rel = np.abs(got.cpu().numpy() / truth - 1.0)
        assert np.median(rel) < tol / 4 and np.quantile(rel, 0.95) < tol, (np.median(rel), np.quantile(rel, 0.95))
    l0 = F.loss_and_grad(dev(w["A0"]), dev(w["B0"]), dev(w["G0"]), D, tau)[0]
    A2, B2, G2, l2 = F.fit_adam(D, tau, dev(w["A0"]), dev(w["B0"]), dev(w["G0"]), steps=400)
    assert float(torch.median(l2 / l0)) < 0.05


@pytest.mark.gpu
def test_context_fit_recovers_the_relaxation_rate():
    """nfs_fit on the structure function of the 128x128 OU sequence: the fitted Gamma(q) follows
    the generator's D q^2 (statistical, so the tolerance is loose)."""
    import paper_1209_3362_gb300 as P
    import nfs_synth as S
    P.build()
    w = S.WORKLOADS["ddm128"]
    fr = S.workload_source(w).frames_numpy(w.N)
    with P.NFS(w.H, w.W, w.delays, w.n_qbins) as ctx:
        ctx.push_frames(fr)
        r = ctx.structure_function()
        q = r["q_mean"]
        Dm = r["D"]
        G0 = 1.3 * w.Dc * q * q + 1e-3
        A0 = np.maximum(Dm[-1] / 2.0, 1e-3)
        B0 = np.maximum(Dm[0] / 4.0, 1e-3)
        A, B, G = ctx.fit(A0, B0, G0, iters=200)
    sel = (q * q * w.Dc > 0.04) & (q * q * w.Dc < 0.8)
    rel = np.abs(G[sel] / (w.Dc * q[sel] ** 2) - 1.0)
    assert sel.sum() > 10 and np.median(rel) < 0.2, (sel.sum(), np.median(rel))


@pytest.mark.gpu
def test_fit_of_the_pipelines_own_structure_function():
    """Eq. 1's fit on the library's own D(q, tau) (the pipeline half of the fit workload): 1000 frames
    of 1024x1024 from the 1024x1024 workload's generator (Gamma = D q^2, D = 2 px^2/frame), 1024 q bins,
    200 log delays 1..500 (consecutive up to 164).  Gamma starts at +-50 % of the generator's D q^2,
    A and B from the data; Gauss-Newton (nfs_fit) and Adam through the autograd Function must recover
    Gamma(q) over the bins these delays resolve, 0.1 <= q < 0.5 rad/px (Gamma tau from 0.02-0.5 at
    tau = 1 to a plateau well before tau = 500).  Statistical: tolerances from the sequence's noise."""
    import torch
    import nfs_synth as S
    import paper_1209_3362_gb300 as P
    from paper_1209_3362_gb300 import fit as F
    P.build()
    w = S.WORKLOADS["ddm1024"]
    delays = S.log_delays(1, 500, 200)
    nq = 1024
    src = S.workload_source(w, device="cuda")
    with P.NFS(w.H, w.W, delays, nq) as ctx:
        for o in range(0, w.N, 100):
            ctx.push_frames_device(src.next_frames(min(100, w.N - o)))
        r = ctx.structure_function()
        q, D = r["q_mean"], r["D"]
        truth = w.Dc * q * q
        rng = np.random.default_rng(5)
        G0 = truth * (1.0 + rng.uniform(-0.5, 0.5, nq)) + 1e-9
        A0 = np.maximum((D[-1] - D[0]) / 2.0, 1e-9) * (1.0 + rng.uniform(-0.5, 0.5, nq))
        B0 = np.maximum(D[0] / 4.0, 1e-9)
        A, B, G = ctx.fit(A0, B0, G0, iters=200)
    sel = (q >= 0.1) & (q < 0.5)
    rel = np.abs(G[sel] / truth[sel] - 1.0)
    assert sel.sum() > 100 and np.median(rel) < 0.05 and np.quantile(rel, 0.9) < 0.12, (np.median(rel), np.quantile(rel, 0.9))
    dev = lambda x: torch.tensor(np.asarray(x, np.float32), device="cuda").contiguous()  # noqa: E731
    Dt, tau = dev(D), dev(delays)
    l0 = F.loss_and_grad(dev(A0), dev(B0), dev(G0), Dt, tau)[0]
    A2, B2, G2, l2 = F.fit_adam(Dt, tau, dev(A0), dev(B0), dev(G0), steps=600)
    assert float(torch.median(l2 / l0)) < 1e-3
    rel2 = np.abs(G2.cpu().numpy()[sel] / truth[sel] - 1.0)
    assert np.median(rel2) < 0.12 and np.quantile(rel2, 0.9) < 0.3, (np.median(rel2), np.quantile(rel2, 0.9))
