"""Parity of the CUDA moving-mesh path and the adjoints with the FP64 oracle (GPU)."""
import numpy as np
import pytest
import torch

from oracle import curv, flat, grad
from synth import grf, smoothed_grf

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(gb, shape, psi):
    s = gb.Solver(shape, op="curv")
    s.set_geometry(to_dev(psi))
    return s


def psi_field(shape, seed, sigma=2.0, rowsum=0.5):
    return smoothed_grf(shape, seed, sigma, rowsum)


@pytest.mark.parametrize("shape", [(16, 16, 16), (16, 24, 32)])
def test_geometry_matches_oracle(gb, shape):
    psi = psi_field(shape, 6)
    s = make(gb, shape, psi)
    hier = curv.hierarchy(psi)
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for level in range(s.levels):
        J, B = s.curv_geometry(level)
        J, B = J.double().cpu().numpy(), B.double().cpu().numpy()
        lev = hier[level]
        np.testing.assert_allclose(J, lev.J, rtol=2e-7, atol=0)
        for k, (a, b) in enumerate(order):
            np.testing.assert_allclose(B[k], lev.B[a, b], rtol=0, atol=3e-7 * np.abs(lev.B[a, a]).max())


@pytest.mark.parametrize("transpose", [False, True])
def test_operator_matches_oracle_stencil(gb, transpose):
    # FP64 application with the GPU's own (FP32) coefficients vs the oracle stencil on the same coefficients
    shape = (16, 24, 32)
    psi = psi_field(shape, 7)
    s = make(gb, shape, psi)
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    rng = np.random.default_rng(1)
    for level in range(2):
        shp = s.level_shape(level)
        h = 2.0 ** level
        J, B6 = s.curv_geometry(level)
        J, B6 = J.double().cpu().numpy(), B6.double().cpu().numpy()
        B = np.empty((3, 3) + shp)
        for k, (a, b) in enumerate(order):
            B[a, b] = B6[k]
            B[b, a] = B6[k]
        u = rng.standard_normal(shp)
        got = s.curv_apply(level, to_dev(u), transpose=transpose, divide_by_J=True).cpu().numpy()
        ref = (curv.apply_MT(u, B, h) if transpose else curv.apply_M(u, B, h)) / J
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
        got32 = s.curv_apply(level, to_dev(u, torch.float32), transpose=transpose).double().cpu().numpy()
        assert np.abs(got32 - ref).max() < 2e-5 * np.abs(ref).max()


def test_transpose_dot_product_on_gpu(gb):
    shape = (24, 24, 24)
    s = make(gb, shape, psi_field(shape, 8))
    rng = np.random.default_rng(2)
    x, y = to_dev(rng.standard_normal(shape)), to_dev(rng.standard_normal(shape))
    Mx = s.curv_apply(0, x, transpose=False, divide_by_J=False)
    MTy = s.curv_apply(0, y, transpose=True, divide_by_J=False)
    lhs, rhs = float((y * Mx).sum()), float((x * MTy).sum())
    assert abs(lhs - rhs) < 1e-11 * float((y * Mx).abs().sum())
    assert float(s.curv_apply(0, torch.ones_like(x), divide_by_J=False).abs().max()) < 1e-12


def test_vcycle_matches_oracle(gb):
    shape = (32, 32, 32)
    psi = psi_field(shape, 9)
    s = make(gb, shape, psi)
    hier = curv.hierarchy(psi)
    r = grf(shape, 10)
    rd = to_dev(r, torch.float32)
    for tr in (False, True):
        got = s.curv_vcycle(rd, transpose=tr).double().cpu().numpy()
        ref = curv.vcycle(0, np.zeros(shape), rd.double().cpu().numpy(), hier, transpose=tr, cache={})
        assert rel_l2(got, ref) < 2e-5


@pytest.mark.parametrize("shape", [(16, 16, 16), (32, 32, 32), (16, 24, 32)])
def test_curvilinear_solve_matches_oracle(gb, shape):
    psi = psi_field(shape, 11)
    delta = grf(shape, 12)
    s = make(gb, shape, psi)
    ref, hist = curv.solve(delta, psi, tol=1e-12, max_cycles=300)
    phi, st = s.solve(to_dev(delta), tol=1e-6, max_vcycles=100)
    assert st.status == 0 and st.rel_res <= 1e-6
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-6
    phi, st = s.solve(to_dev(delta), tol=1e-10, max_vcycles=200)
    assert st.status == 0
    # the remaining difference is the FP32 rounding of the geometry coefficients
    assert rel_l2(phi.cpu().numpy(), ref) < 3e-7
    # convergence factor comparable with the oracle's cycle
    rho_gpu = (st.history[-1] / st.history[0]) ** (1.0 / max(1, len(st.history) - 1))
    rho_ora = (hist[-1] / hist[1]) ** (1.0 / (len(hist) - 2))
    assert rho_gpu < 1.2 * rho_ora + 0.02


def test_psi_zero_reduces_to_flat(gb):
    shape = (32, 32, 32)
    F = grf(shape, 13)
    s = make(gb, shape, np.zeros(shape))
    phi, st = s.solve(to_dev(F), tol=1e-10, max_vcycles=100)
    assert rel_l2(phi.cpu().numpy(), flat.fft_solve(F)) < 1e-9


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("shape", [(16, 24, 32), (32, 32, 32)])
def test_double_float_residual_is_the_fp64_residual(gb, shape, sym, monkeypatch):
    # Solved to 1e-12, the solution's residual under the GPU's own FP32 coefficients,
    # evaluated here in FP64 by the oracle stencil, is the residual the double-float
    # kernel reported.  That kernel forms each face (and edge) mean of the FP32 cell
    # coefficients in FP32 and everything else in double-float, so the stencil here
    # takes the same FP32 means; the rest of its arithmetic is FP64.
    def face32(B, a, b):
        c = B[a, b].astype(np.float32)
        return (np.float32(0.5) * (c + curv.at(c, a, 1))).astype(np.float64)

    def edge32(B, a, b):
        c = B[a, b].astype(np.float32)
        return (np.float32(0.25) * ((c + curv.at(c, a, 1)) + (curv.at(c, b, 1) + curv.at2(c, a, 1, b, 1)))
                ).astype(np.float64)

    psi = psi_field(shape, 17)
    delta = grf(shape, 18)
    s = gb.Solver(shape, op="curv", curv_sym=sym)
    s.set_geometry(to_dev(psi))
    phi, st = s.solve(to_dev(delta), tol=1e-12, max_vcycles=300)
    assert st.status == 0 and st.rel_res <= 1e-12
    J, B6 = s.curv_geometry(0)
    J, B6 = J.double().cpu().numpy(), B6.double().cpu().numpy()
    B = np.empty((3, 3) + shape)
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        B[a, b] = B6[k]
        B[b, a] = B6[k]
    f = delta - (delta * J).sum() / J.sum()
    monkeypatch.setattr(curv, "face_coeff", face32)
    monkeypatch.setattr(curv, "edge_coeff", edge32)
    Mphi = (curv.apply_M_sym if sym else curv.apply_M)(phi.cpu().numpy(), B, 1.0)
    rel = float(np.linalg.norm(f - Mphi / J) / np.linalg.norm(f))
    assert rel < 2e-12
    assert abs(rel - st.rel_res) < 0.05 * st.rel_res + 1e-14


@pytest.mark.parametrize("shape", [(16, 24, 32), (32, 32, 32)])
def test_transposed_double_float_residual_is_the_fp64_residual(gb, shape, monkeypatch):
    # The adjoint's transposed solve M^T lam = phi_bar - mean(phi_bar) to 1e-12: its
    # residual, evaluated in FP64 by the oracle's exact transpose with the GPU's FP32
    # coefficients and FP32 face means, is the one the double-float kernel reported.
    # lam is recovered up to a constant (which M^T annihilates) from source_bar = J (lam - s).
    def face32(B, a, b):
        c = B[a, b].astype(np.float32)
        return (np.float32(0.5) * (c + curv.at(c, a, 1))).astype(np.float64)

    psi = psi_field(shape, 19)
    pbar = grf(shape, 20)
    s = make(gb, shape, psi)
    dbar, _, st = s.solve_adjoint(to_dev(pbar), tol=1e-12, max_vcycles=300)
    assert st.status == 0 and st.rel_res <= 1e-12
    J, B6 = s.curv_geometry(0)
    J, B6 = J.double().cpu().numpy(), B6.double().cpu().numpy()
    B = np.empty((3, 3) + shape)
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        B[a, b] = B6[k]
        B[b, a] = B6[k]
    lam = dbar.cpu().numpy() / J
    g = pbar - pbar.mean()
    monkeypatch.setattr(curv, "face_coeff", face32)
    res = (g - curv.apply_MT(lam, B, 1.0)) / J
    rel = float(np.linalg.norm(res) / np.linalg.norm(g / J))
    assert rel < 2e-12
    assert abs(rel - st.rel_res) < 0.05 * st.rel_res + 1e-14


def test_adjoint_matches_oracle(gb):
    shape = (16, 16, 16)
    psi = psi_field(shape, 14, 1.5, 0.4)
    delta = grf(shape, 15)
    pbar = np.random.default_rng(3).standard_normal(shape)
    s = make(gb, shape, psi)
    phi, _ = s.solve(to_dev(delta), tol=1e-11, max_vcycles=200)
    dbar, psibar, st = s.solve_adjoint(to_dev(pbar), phi=phi, source=to_dev(delta), want_psi_bar=True,
                                       tol=1e-11, max_vcycles=200)
    assert st.status == 0
    ref_phi, _ = curv.solve(delta, psi, tol=1e-13, max_cycles=400)
    rd, rp = curv.solve_vjp(delta, psi, ref_phi, pbar, tol=1e-13, max_cycles=400)
    assert rel_l2(dbar.cpu().numpy(), rd) < 1e-6
    assert rel_l2(psibar.cpu().numpy(), rp) < 1e-5


def test_adjoint_against_gpu_central_differences(gb):
    # directional derivatives of <w, grad2 phi> by central differences of the GPU forward solve
    shape = (16, 16, 16)
    psi = psi_field(shape, 16, 2.0, 0.5)
    delta = grf(shape, 17)
    w = np.random.default_rng(4).standard_normal((3,) + shape)
    s = make(gb, shape, psi)

    def loss(d, p):
        phi, _ = s.solve(to_dev(d), tol=1e-12, max_vcycles=300, psi=to_dev(p))
        return float((w * grad.grad2(phi.cpu().numpy())).sum())

    phi, _ = s.solve(to_dev(delta), tol=1e-12, max_vcycles=300, psi=to_dev(psi))
    pbar = grad.grad2_T(w)
    dbar, psibar, _ = s.solve_adjoint(to_dev(pbar), phi=phi, source=to_dev(delta), want_psi_bar=True,
                                      tol=1e-12, max_vcycles=300)
    dbar, psibar = dbar.cpu().numpy(), psibar.cpu().numpy()
    rng = np.random.default_rng(5)
    for k in range(3):
        v = rng.standard_normal(shape)
        fd = (loss(delta + 1e-3 * v, psi) - loss(delta - 1e-3 * v, psi)) / 2e-3
        assert abs(fd - float((dbar * v).sum())) < 1e-6 * max(1.0, abs(fd))
        dpsi = psi_field(shape, 200 + k, 2.0, 0.5)
        eps = 1e-3
        fd = (loss(delta, psi + eps * dpsi) - loss(delta, psi - eps * dpsi)) / (2 * eps)
        # the forward map rounds its geometry coefficients to FP32, which puts ~1e-4
        # relative noise into this difference quotient; the adjoint itself matches the
        # FP64 oracle to 1e-5 (test_adjoint_matches_oracle)
        assert abs(fd - float((psibar * dpsi).sum())) < 1e-3 * max(1.0, abs(fd))


def test_flat_adjoint_and_autograd(gb):
    n = 32
    F = to_dev(grf(n, 18)).requires_grad_(True)
    w = to_dev(np.random.default_rng(6).standard_normal((3, n, n, n)))
    s = gb.Solver(n)
    phi = gb.MGSolve.apply(F, s, 1e-10, 60)
    # 4th-order gradient loss from the oracle's definition, written with torch.roll here
    def g4(u, ax):
        return (-torch.roll(u, -2, ax) + 8 * torch.roll(u, -1, ax) - 8 * torch.roll(u, 1, ax) + torch.roll(u, 2, ax)) / 12
    loss = sum((w[c] * g4(phi, ax)).sum() for c, ax in enumerate((2, 1, 0)))
    loss.backward()
    ref = flat.fft_solve(grad.grad4_T(w.cpu().numpy()))
    ref -= ref.mean()
    assert rel_l2(F.grad.cpu().numpy(), ref) < 1e-9


def test_curvilinear_autograd(gb):
    shape = (16, 16, 16)
    psi = to_dev(psi_field(shape, 19, 2.0, 0.4)).requires_grad_(True)
    delta = to_dev(grf(shape, 20)).requires_grad_(True)
    pbar = np.random.default_rng(7).standard_normal(shape)
    s = gb.Solver(shape, op="curv")
    phi = gb.CurvMGSolve.apply(delta, psi, s, 1e-11, 200)
    (phi * to_dev(pbar)).sum().backward()
    ref_phi, _ = curv.solve(delta.detach().cpu().numpy(), psi.detach().cpu().numpy(), tol=1e-13, max_cycles=400)
    rd, rp = curv.solve_vjp(delta.detach().cpu().numpy(), psi.detach().cpu().numpy(), ref_phi, pbar,
                            tol=1e-13, max_cycles=400)
    assert rel_l2(delta.grad.cpu().numpy(), rd) < 1e-6
    assert rel_l2(psi.grad.cpu().numpy(), rp) < 1e-5


def test_curvilinear_errors(gb):
    s = gb.Solver(16, op="curv")
    with pytest.raises(gb.GbmgError):
        s.solve(to_dev(grf(16, 1)))           # no geometry yet
    with pytest.raises(gb.GbmgError):
        gb.Solver(16, op="curv", smoother="chebyshev")
    with pytest.raises(gb.GbmgError):
        gb.Solver(16, op="curv", prec="fp64")


@pytest.mark.parametrize("shape,passes", [((16, 16, 16), 2), ((16, 24, 32), 1)])
def test_mesh_motion_matches_oracle(gb, shape, passes):
    """One mesh-motion step (Sec. 4.4, Eq. calcdefp and Eq. defadvance) against the oracle:
    psidot and the advanced psi, then a second step warm-started from the first psidot."""
    psi = psi_field(shape, 21, rowsum=0.3)
    rho = 1.0 + 0.3 * grf(shape, 22)
    kappa, m_init, dtau = 0.8, 1.0, 0.25
    ref_psi, ref_dot = curv.mesh_motion_step(psi, rho, kappa, m_init, dtau, passes=passes, tol=1e-12)
    s = gb.Solver(shape, op="curv")
    p = to_dev(psi)
    p, dot, st = s.mesh_motion(to_dev(rho), p, kappa, m_init, dtau, smooth_passes=passes, tol=1e-10,
                               max_vcycles=200)
    assert st.status == 0 and st.rel_res <= 1e-10
    # the remaining difference is the FP32 rounding of J in the source and of the coefficients
    assert rel_l2(dot.cpu().numpy(), ref_dot) < 1e-6
    assert rel_l2(p.cpu().numpy(), ref_psi) < 1e-6
    assert abs(float(p.mean())) < 1e-12 * float(p.abs().max())
    ref2_psi, ref2_dot = curv.mesh_motion_step(ref_psi, rho, kappa, m_init, dtau, passes=passes, tol=1e-12)
    p, dot2, st2 = s.mesh_motion(to_dev(rho), p, kappa, m_init, dtau, psidot=dot.clone(), smooth_passes=passes,
                                 tol=1e-10, max_vcycles=200)
    assert st2.status == 0 and st2.rel_res0 < st.rel_res0   # warm start from the previous psidot
    assert rel_l2(dot2.cpu().numpy(), ref2_dot) < 2e-6
    assert rel_l2(p.cpu().numpy(), ref2_psi) < 2e-6
    # the context needs its geometry again before the next solve
    with pytest.raises(gb.GbmgError):
        s.solve(to_dev(rho))
    with pytest.raises(gb.GbmgError):
        gb.Solver(shape).mesh_motion(to_dev(rho), to_dev(psi), kappa, m_init, dtau)


# ---------------------------------------------------------------- symmetric variant


def make_sym(gb, shape, psi):
    s = gb.Solver(shape, op="curv", curv_sym=True)
    s.set_geometry(to_dev(psi))
    return s


def test_sym_operator_matches_oracle_stencil(gb):
    shape = (16, 24, 32)
    psi = psi_field(shape, 30)
    s = make_sym(gb, shape, psi)
    order = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    rng = np.random.default_rng(31)
    for level in range(2):
        shp = s.level_shape(level)
        h = 2.0 ** level
        J, B6 = s.curv_geometry(level)
        J, B6 = J.double().cpu().numpy(), B6.double().cpu().numpy()
        B = np.empty((3, 3) + shp)
        for k, (a, b) in enumerate(order):
            B[a, b] = B6[k]
            B[b, a] = B6[k]
        u = rng.standard_normal(shp)
        ref = curv.apply_M_sym(u, B, h) / J
        for tr in (False, True):           # S is its own transpose
            got = s.curv_apply(level, to_dev(u), transpose=tr, divide_by_J=True).cpu().numpy()
            assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
        got32 = s.curv_apply(level, to_dev(u, torch.float32)).double().cpu().numpy()
        assert np.abs(got32 - ref).max() < 2e-5 * np.abs(ref).max()
        # and it differs from the literal scheme on the same geometry
        lit = curv.apply_M(u, B, h) / J
        assert np.abs(lit - ref).max() > 1e-3 * np.abs(ref).max()


def test_sym_operator_is_symmetric_on_gpu(gb):
    shape = (24, 24, 24)
    s = make_sym(gb, shape, psi_field(shape, 32))
    rng = np.random.default_rng(33)
    x, y = to_dev(rng.standard_normal(shape)), to_dev(rng.standard_normal(shape))
    Sx = s.curv_apply(0, x, divide_by_J=False)
    Sy = s.curv_apply(0, y, divide_by_J=False)
    lhs, rhs = float((y * Sx).sum()), float((x * Sy).sum())
    assert abs(lhs - rhs) < 1e-11 * float((y * Sx).abs().sum())
    assert float(s.curv_apply(0, torch.ones_like(x), divide_by_J=False).abs().max()) < 1e-12


def test_sym_vcycle_and_solve_match_oracle(gb):
    shape = (32, 32, 32)
    psi = psi_field(shape, 34)
    s = make_sym(gb, shape, psi)
    hier = curv.hierarchy(psi, sym=True)
    r = grf(shape, 35)
    rd = to_dev(r, torch.float32)
    got = s.curv_vcycle(rd).double().cpu().numpy()
    ref = curv.vcycle(0, np.zeros(shape), rd.double().cpu().numpy(), hier, cache={})
    assert rel_l2(got, ref) < 2e-5
    for shp in [(16, 16, 16), (16, 24, 32)]:
        psi = psi_field(shp, 36)
        delta = grf(shp, 37)
        s = make_sym(gb, shp, psi)
        ref, hist = curv.solve(delta, psi, tol=1e-12, max_cycles=300, sym=True)
        phi, st = s.solve(to_dev(delta), tol=1e-10, max_vcycles=200)
        assert st.status == 0
        assert rel_l2(phi.cpu().numpy(), ref) < 3e-7
        rho_gpu = (st.history[-1] / st.history[0]) ** (1.0 / max(1, len(st.history) - 1))
        rho_ora = (hist[-1] / hist[1]) ** (1.0 / (len(hist) - 2))
        assert rho_gpu < 1.2 * rho_ora + 0.02
        lit, _ = curv.solve(delta, psi, tol=1e-12, max_cycles=300)
        assert rel_l2(lit, ref) > 1e-4             # the two discretisations differ


def test_sym_adjoint_matches_oracle(gb):
    shape = (16, 16, 16)
    psi = psi_field(shape, 38, 1.5, 0.4)
    delta = grf(shape, 39)
    pbar = np.random.default_rng(40).standard_normal(shape)
    s = make_sym(gb, shape, psi)
    phi, _ = s.solve(to_dev(delta), tol=1e-11, max_vcycles=200)
    dbar, psibar, st = s.solve_adjoint(to_dev(pbar), phi=phi, source=to_dev(delta), want_psi_bar=True,
                                       tol=1e-11, max_vcycles=200)
    assert st.status == 0
    ref_phi, _ = curv.solve(delta, psi, tol=1e-13, max_cycles=400, sym=True)
    rd, rp = curv.solve_vjp(delta, psi, ref_phi, pbar, tol=1e-13, max_cycles=400, sym=True)
    assert rel_l2(dbar.cpu().numpy(), rd) < 1e-6
    assert rel_l2(psibar.cpu().numpy(), rp) < 1e-5


def test_sym_option_needs_the_curvilinear_operator(gb):
    with pytest.raises(gb.GbmgError):
        gb.Solver((16, 16, 16), curv_sym=True)


def test_curvilinear_host_buffer_entry_points(gb):
    # mg_solve_host (page-locked buffers read in place by the conversion kernels) and
    # mg_solve_host_sequence (copies overlapped, warm start on the device) on the
    # curvilinear operator equal the device-buffer solves
    shape = (16, 16, 16)
    psi = psi_field(shape, 41)
    s = make(gb, shape, psi)
    d0, d1 = grf(shape, 42), grf(shape, 43)
    ref0, st0 = s.solve(to_dev(d0), tol=1e-9, max_vcycles=100)
    ref1, st1 = s.solve(to_dev(d1), ref0.clone(), tol=1e-9, max_vcycles=100)
    src = torch.from_numpy(d0.copy()).pin_memory()
    out = torch.zeros(shape, dtype=torch.float64).pin_memory()
    _, st = s.solve_host(src, out, tol=1e-9, max_vcycles=100)
    assert st.cycles == st0.cycles
    np.testing.assert_array_equal(out.numpy(), ref0.cpu().numpy())
    outs = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    sts = s.solve_host_sequence([src, torch.from_numpy(d1.copy()).pin_memory()], outs, tol=1e-9, max_vcycles=100)
    assert [x.cycles for x in sts] == [st0.cycles, st1.cycles]
    np.testing.assert_array_equal(outs[0].numpy(), ref0.cpu().numpy())
    np.testing.assert_array_equal(outs[1].numpy(), ref1.cpu().numpy())
