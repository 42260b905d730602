"""Full-size parity checks of each workload in the launch configuration bench.py uses (GPU).

512^3 warm-started sequence (device buffers, and host buffers through the sequence entry
point), 256^3 differentiable flat solve, 256^3 moving-mesh solve with its adjoint, and the
48-problem batch.  The oracle computes what it can at these
sizes in seconds (FFT solves, one application of the FP64 curvilinear operator and of
its transpose, the psi-bar cotangent chain given the GPU's phi and lam); the rest is
checked through properties that hold at any size (residual of the FP64 operator,
central finite differences of the GPU forward map).
"""
import numpy as np
import pytest
import torch

from oracle import curv, flat, grad
from synth import grf, smoothed_grf, vector_noise

pytestmark = pytest.mark.gpu


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_warm_sequence_512(gb):
    n = 512
    d0, eta = grf(n, 2), grf(n, 3)
    s = gb.Solver(n)                     # the benchmark's configuration: mixed, fused, V(3,3)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    cycles = []
    for t in range(10):
        F = d0 + (0.05 * t) * eta
        _, st = s.solve(to_dev(F), phi, tol=1e-6, max_vcycles=40)
        assert st.status == 0 and st.rel_res <= 1e-6
        cycles.append(st.cycles)
    assert max(cycles[1:]) < cycles[0]   # warm starts save cycles (Eq. kwarm)
    ref = flat.fft_solve(F)
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-6


def test_host_sequence_512(gb):
    # the e2e path of the bench: page-locked sources in, page-locked solutions out, warm
    # starts on the device; equal to device-buffer solves of the same sequence, and the
    # last solution matches the FFT solve
    n, T = 512, 3
    d0, eta = grf(n, 2), grf(n, 3)
    Fs = [d0 + (0.05 * t) * eta for t in range(T)]
    s = gb.Solver(n)
    src = [torch.from_numpy(F).pin_memory() for F in Fs]
    outs = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(T)]
    sts = s.solve_host_sequence(src, outs, tol=1e-6, max_vcycles=40)
    assert all(st.status == 0 and st.rel_res <= 1e-6 for st in sts)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    for t in range(T):
        _, st = s.solve(src[t].cuda(), phi, tol=1e-6, max_vcycles=40)
        assert st.cycles == sts[t].cycles
        assert torch.equal(phi.cpu(), outs[t])
    assert rel_l2(outs[-1].numpy(), flat.fft_solve(Fs[-1])) < 1e-6


def test_differentiable_flat_256(gb):
    n = 256
    F = grf(n, 4)
    w = to_dev(vector_noise(n, 5), torch.float32)
    s = gb.Solver(n)
    Fd = to_dev(F).requires_grad_(True)
    phi = gb.MGSolve.apply(Fd, s, 1e-10, 60)
    loss = gb.GradDotLoss.apply(phi, w, s, 4)
    loss.backward()
    g = Fd.grad.cpu().numpy()
    ref = flat.fft_solve(grad.grad4_T(w.cpu().numpy().astype(np.float64)))
    ref -= ref.mean()
    assert rel_l2(g, ref) < 1e-6
    # central differences in 32 random source directions (the loss is linear in F)
    def L(FF):
        ph, _ = s.solve(FF, tol=1e-10, max_vcycles=60)
        return float(s.grad_dot(ph, w, 4))
    gd = to_dev(g)
    for seed in range(100, 132):
        v = to_dev(np.random.default_rng(seed).standard_normal((n, n, n)))
        fd = (L(to_dev(F) + 1e-3 * v) - L(to_dev(F) - 1e-3 * v)) / 2e-3
        assert abs(fd - float((gd * v).sum())) <= 1e-5 * max(1.0, abs(fd))


def test_moving_mesh_256(gb):
    n = 256
    psi = smoothed_grf(n, 6, 4.0, 0.5)
    delta = grf(n, 7)
    s = gb.Solver(n, op="curv")
    psid = to_dev(psi)
    phi, st = s.solve(to_dev(delta), tol=1e-6, max_vcycles=100, psi=psid)
    assert st.status == 0
    J, _ = s.curv_geometry(0)
    assert float(J.min()) > 0.0
    # residual of the GPU solution under the oracle's FP64 operator
    lev = curv.Level(psi, 1.0)
    f = curv.weighted_projection(delta, lev.J)
    res = np.linalg.norm(f - lev.L(phi.cpu().numpy())) / np.linalg.norm(f)
    assert res < 2e-6
    # adjoint of <w, grad2 phi> against central differences of the GPU forward map
    w = vector_noise(n, 8).astype(np.float64)
    phi_t, _ = s.solve(to_dev(delta), tol=1e-10, max_vcycles=200, psi=psid)
    pbar = to_dev(grad.grad2_T(w))
    dbar, psibar, st = s.solve_adjoint(pbar, phi=phi_t, source=to_dev(delta), want_psi_bar=True, tol=1e-10,
                                       max_vcycles=200)
    assert st.status == 0
    # psi_bar element by element: the oracle's cotangent chain (Sec. 4.8, Eq. adj_op:
    # B-cotangent of <lam, M phi>, triad cotangents of B = J A^-2 and of J, transposed
    # Hessian) fed with the GPU's phi and the GPU's lam.  source_bar = J (lam - <lam>_J)
    # with the GPU's FP32 J gives lam up to a constant, which neither cotangent sees.
    J32 = J.double().cpu().numpy()
    lam = dbar.cpu().numpy() / J32
    lam -= lam.mean()
    ph = phi_t.cpu().numpy()
    A = curv.triad(psi, 1.0)
    f = curv.weighted_projection(delta, lev.J)
    Jbar = f * (lam - float((lam * lev.J).sum() / lev.J.sum()))
    Abar = curv.Abar_from_J(A, Jbar) - curv.Abar_from_B(A, curv.Bbar_from_operator(lam, ph, 1.0))
    del A
    ref_psibar = curv.hessian_T(Abar, 1.0)
    del Abar
    assert rel_l2(psibar.cpu().numpy(), ref_psibar) < 1e-5
    # and lam solves the transposed system under the oracle's FP64 operator
    g = pbar.cpu().numpy() - float(pbar.mean())
    res = np.linalg.norm((g - curv.apply_MT(lam, lev.B, 1.0)) / lev.J) / np.linalg.norm(g / lev.J)
    assert res < 2e-6
    wd = to_dev(w)

    def L(d, p):
        ph, _ = s.solve(to_dev(d), tol=1e-10, max_vcycles=200, psi=to_dev(p))
        return float((wd * s.grad(ph, 2)).sum())

    for k in range(3):
        v = np.random.default_rng(300 + k).standard_normal((n, n, n))
        fd = (L(delta + 1e-3 * v, psi) - L(delta - 1e-3 * v, psi)) / 2e-3
        assert abs(fd - float((dbar * to_dev(v)).sum())) <= 1e-5 * max(1.0, abs(fd))
    # psi directions: the forward map rounds its geometry to FP32, whose noise in the loss
    # (~1e-7 relative) would dominate a difference quotient with eps = 1e-3 at this size;
    # eps = 1e-2 keeps that noise and the O(eps^2) truncation both near 1e-4
    for k in range(2):
        dpsi = smoothed_grf(n, 400 + k, 4.0, 0.5)
        fd = (L(delta, psi + 1e-2 * dpsi) - L(delta, psi - 1e-2 * dpsi)) / 2e-2
        assert abs(fd - float((psibar * to_dev(dpsi)).sum())) <= 1e-3 * max(1.0, abs(fd))


def test_batched_48(gb):
    shapes = [(64,) * 3] * 16 + [(96,) * 3] * 16 + [(128,) * 3] * 16
    srcs = [grf(s, 1000 + i) for i, s in enumerate(shapes)]
    F = [to_dev(a) for a in srcs]
    phis = [torch.zeros_like(f) for f in F]
    batch = gb.Batch(shapes)
    stats, times = batch.solve(F, phis, tol=1e-6, max_vcycles=40)
    for i, st in enumerate(stats):
        assert st.status == 0 and st.rel_res <= 1e-6
        assert rel_l2(phis[i].cpu().numpy(), flat.fft_solve(srcs[i])) < 1e-6
    for i in (0, 17, 40):
        ref, st = gb.Solver(shapes[i], fused=False).solve(F[i], tol=1e-6, max_vcycles=40)
        assert st.cycles == stats[i].cycles
        assert float((ref - phis[i]).abs().max()) <= 1e-12 * float(ref.abs().max())
    batch.close()
