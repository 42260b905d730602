"""Pins of the curvilinear oracle (CPU): closed forms, invariants, consistency, FD gradients."""
import math

import numpy as np
import pytest

from oracle import curv, flat
from synth import grf, smoothed_grf


def coords(shape):
    nz, ny, nx = shape
    return np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float),
                       np.arange(nx, dtype=float), indexing="ij")   # z, y, x


def test_psi_zero_reduces_to_seven_point():
    # Sec. 4.3: psi = 0 gives sqrt(g) = 1, g^ab = delta^ab and the standard 7-point operator
    rng = np.random.default_rng(0)
    u = rng.standard_normal((8, 12, 16))
    for h in (1.0, 2.0):
        J, B = curv.geometry(np.zeros(u.shape), h)
        np.testing.assert_array_equal(J, 1.0)
        np.testing.assert_allclose(curv.apply_M(u, B, h), flat.apply_A(u, h), atol=1e-13)
        np.testing.assert_allclose(curv.diag_M(B, h), -6.0 / h ** 2, atol=1e-15)


def test_triad_plane_wave_closed_form():
    # second differences of cos(k.x): -4 sin^2(k_a/2) cos ; mixed four-point stencil: -sin k_a sin k_b cos
    shape = (16, 12, 8)
    z, y, x = coords(shape)
    k = (2 * np.pi * 1 / 8, 2 * np.pi * 2 / 12, 2 * np.pi * 3 / 16)       # (kx, ky, kz)
    amp = 0.2
    c = np.cos(k[0] * x + k[1] * y + k[2] * z)
    A = curv.triad(amp * c)
    for a in range(3):
        for b in range(3):
            if a == b:
                exact = (a == b) - amp * 4 * math.sin(k[a] / 2) ** 2 * c
            else:
                exact = -amp * math.sin(k[a]) * math.sin(k[b]) * c
            np.testing.assert_allclose(A[a, b], exact, atol=1e-13)


def test_geometry_against_linalg():
    psi = smoothed_grf(16, 6, 2.0, 0.5)
    J, B = curv.geometry(psi)
    A = np.moveaxis(curv.triad(psi), (0, 1), (-2, -1))
    ev = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(J, ev.prod(axis=-1), rtol=1e-12)
    Bm = np.moveaxis(B, (0, 1), (-2, -1))
    np.testing.assert_allclose(Bm @ A @ A, J[..., None, None] * np.eye(3), atol=1e-12)
    # Gershgorin-scaled recipe: lambda(A) in [0.5, 1.5] up to the spectral/discrete Hessian gap, J > 0
    assert ev.min() > 0.45 and J.min() > 0.1


def test_constant_B_symbol():
    # M on exp(i k.x) with constant B: -sum_a 4 B_aa sin^2(k_a/2) - 2 sum_{a<b} B_ab sin k_a sin k_b
    shape = (8, 12, 16)
    Bc = np.array([[1.3, 0.2, -0.15], [0.2, 0.9, 0.1], [-0.15, 0.1, 1.1]])
    B = np.broadcast_to(Bc[:, :, None, None, None], (3, 3) + shape).copy()
    z, y, x = coords(shape)
    for n in [(1, 2, 1), (3, 1, 2), (8, 6, 4), (5, 5, 3)]:
        k = (2 * np.pi * n[0] / shape[2], 2 * np.pi * n[1] / shape[1], 2 * np.pi * n[2] / shape[0])
        u = np.cos(k[0] * x + k[1] * y + k[2] * z + 0.4)
        sym = -sum(4 * Bc[a, a] * math.sin(k[a] / 2) ** 2 for a in range(3))
        sym -= 2 * sum(Bc[a, b] * math.sin(k[a]) * math.sin(k[b]) for a in range(3) for b in range(a + 1, 3))
        np.testing.assert_allclose(curv.apply_M(u, B), sym * u, atol=1e-12)
        np.testing.assert_allclose(curv.apply_MT(u, B), sym * u, atol=1e-12)


def test_conservation_and_null_space():
    psi = smoothed_grf(16, 9, 2.0, 0.5)
    J, B = curv.geometry(psi)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(psi.shape)
    assert np.abs(curv.apply_M(np.ones_like(u), B)).max() < 1e-13          # M 1 = 0
    assert abs(curv.apply_M(u, B).sum()) < 1e-11 * np.abs(u).sum()         # 1^T M = 0 (flux form)
    assert np.abs(curv.apply_MT(np.ones_like(u), B)).max() < 1e-13


def test_transpose_dot_product():
    psi = smoothed_grf((8, 12, 16), 10, 2.0, 0.5)
    _, B = curv.geometry(psi, 2.0)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(psi.shape), rng.standard_normal(psi.shape)
    lhs = float((y * curv.apply_M(x, B, 2.0)).sum())
    rhs = float((x * curv.apply_MT(y, B, 2.0)).sum())
    assert abs(lhs - rhs) < 1e-13 * abs(lhs) * 100
    # and the dense transpose at 4^3 x 6
    lev = curv.Level(smoothed_grf((4, 4, 6), 3, 1.0, 0.3), 1.0)
    np.testing.assert_allclose(curv.dense_L(lev, True) * lev.J.ravel()[:, None],
                               (curv.dense_L(lev) * lev.J.ravel()[:, None]).T, atol=1e-13)


def test_second_order_consistency_with_continuum():
    sp = pytest.importorskip("sympy")
    X, Y, Z, N = sp.symbols("X Y Z N")
    w = 2 * sp.pi / N
    Bs = {(0, 0): 1 + sp.Rational(3, 10) * sp.sin(w * X), (1, 1): 1 + sp.Rational(1, 5) * sp.cos(w * Y),
          (2, 2): 1 + sp.Rational(1, 10) * sp.sin(w * (Z + X)), (0, 1): sp.Rational(1, 10) * sp.cos(w * (X + Y)),
          (0, 2): sp.Rational(1, 20) * sp.sin(w * Z), (1, 2): sp.Rational(2, 25) * sp.cos(w * (Y - Z))}
    for (a, b) in list(Bs):
        Bs[(b, a)] = Bs[(a, b)]
    us = sp.sin(w * X) * sp.cos(w * Y) + sp.Rational(1, 2) * sp.sin(w * (2 * Z + Y))
    var = (X, Y, Z)
    cont = sum(sp.diff(Bs[(a, b)] * sp.diff(us, var[b]), var[a]) for a in range(3) for b in range(3))
    fB = {k: sp.lambdify((X, Y, Z, N), v, "numpy") for k, v in Bs.items()}
    fu = sp.lambdify((X, Y, Z, N), us, "numpy")
    fc = sp.lambdify((X, Y, Z, N), cont, "numpy")
    errs = []
    for n in (16, 32, 64):
        z, y, x = coords((n, n, n))
        B = np.empty((3, 3, n, n, n))
        for a in range(3):
            for b in range(3):
                B[a, b] = fB[(a, b)](x, y, z, n) * np.ones_like(x)
        num = curv.apply_M(fu(x, y, z, n), B)
        ref = fc(x, y, z, n)
        errs.append(np.abs(num - ref).max() / np.abs(ref).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_psi_zero_solve_equals_flat_jacobi_cycle():
    F = grf(16, 40)
    a, ha = curv.solve(F, np.zeros(F.shape), fixed_cycles=3)
    b, hb = flat.mg_solve(F, fixed_cycles=3, smoother="jacobi")
    np.testing.assert_allclose(a, b, atol=1e-11 * np.abs(b).max())
    np.testing.assert_allclose(ha, hb, rtol=1e-9)


def test_solve_matches_dense_pinv_8():
    psi = smoothed_grf(8, 12, 1.5, 0.4)
    delta = grf(8, 13)
    phi, hist = curv.solve(delta, psi, tol=1e-13, max_cycles=300)
    lev = curv.hierarchy(psi)[0]
    f = curv.weighted_projection(delta, lev.J)
    assert abs(float((f * lev.J).sum())) < 1e-12
    ref = (np.linalg.pinv(curv.dense_L(lev), rcond=1e-10) @ f.ravel()).reshape(f.shape)
    ref -= ref.mean()
    np.testing.assert_allclose(phi, ref, atol=1e-10 * np.abs(ref).max())


def test_manufactured_solution_16():
    psi = smoothed_grf(16, 14, 2.0, 0.5)
    lev = curv.hierarchy(psi)[0]
    rng = np.random.default_rng(3)
    phi_star = flat.fft_solve(rng.standard_normal(psi.shape))       # smooth, zero mean
    f = lev.L(phi_star)
    phi, hist = curv.solve(f, psi, tol=1e-12, max_cycles=200)
    assert hist[-1] <= 1e-12
    np.testing.assert_allclose(phi, phi_star, atol=1e-9 * np.abs(phi_star).max())
    rho = (hist[-1] / hist[1]) ** (1 / (len(hist) - 2))
    assert rho < 0.6


def test_vjp_against_central_differences():
    n = 8
    psi = smoothed_grf(n, 6, 1.5, 0.4)
    delta = grf(n, 7)
    rng = np.random.default_rng(1)
    pbar = rng.standard_normal((n, n, n))
    kw = dict(tol=1e-13, max_cycles=300)
    phi, _ = curv.solve(delta, psi, **kw)
    dbar, psibar = curv.solve_vjp(delta, psi, phi, pbar, **kw)

    def loss(d, p):
        return float((curv.solve(d, p, **kw)[0] * pbar).sum())

    for trial in range(2):
        v = rng.standard_normal((n, n, n))
        eps = 1e-4
        fd = (loss(delta + eps * v, psi) - loss(delta - eps * v, psi)) / (2 * eps)
        assert abs(fd - float((dbar * v).sum())) < 1e-6 * max(1.0, abs(fd))
        wdir = smoothed_grf(n, 100 + trial, 1.5, 0.4)
        eps = 1e-3
        fd = (loss(delta, psi + eps * wdir) - loss(delta, psi - eps * wdir)) / (2 * eps)
        assert abs(fd - float((psibar * wdir).sum())) < 1e-5 * max(1.0, abs(fd))


def test_binomial_smoothing_plane_wave_factor():
    """[1/4, 1/2, 1/4] per axis has the symbol cos^2(k/2); p passes over three axes multiply
    a plane wave by prod_a cos^2(k_a / 2)^p."""
    n = (8, 12, 16)
    kk = [2 * math.pi * m / s for m, s in zip((1, 2, 3), n)]   # (kz, ky, kx)
    z, y, x = np.meshgrid(*[np.arange(s) for s in n], indexing="ij")
    u = np.cos(kk[0] * z + kk[1] * y + kk[2] * x)
    for p in (1, 2):
        factor = np.prod([math.cos(k / 2) ** 2 for k in kk]) ** p
        np.testing.assert_allclose(curv.smooth_binomial(u, p), factor * u, rtol=0, atol=1e-13)


def test_mesh_motion_flat_mesh_is_spectral_solve():
    """psi = 0 (sqrt g = 1): the deformation-rate potential is the flat Poisson solution of
    the smoothed kappa (m_init - rho), and psi_new = dtau psidot (zero mean)."""
    n = 16
    rho = 1.0 + 0.3 * grf(n, 31)
    psi0 = np.zeros((n, n, n))
    kappa, m_init, dtau = 0.7, 1.0, 0.2
    new, psidot = curv.mesh_motion_step(psi0, rho, kappa, m_init, dtau, passes=2, tol=1e-12)
    ref = flat.fft_solve(curv.smooth_binomial(kappa * (m_init - rho), 2))
    ref -= ref.mean()
    np.testing.assert_allclose(psidot, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(new, dtau * ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_mesh_motion_equal_mass_per_cell_is_stationary():
    """m = sqrt(g) rho equal to m_init in every cell gives a zero source: psidot = 0 and psi
    only loses its mean (Eq. defadvance gauge)."""
    n = 16
    psi = smoothed_grf(n, 32, 2.0, 0.3) + 0.5
    J = curv.geometry(psi, 1.0)[0]
    rho = 1.3 / J
    new, psidot = curv.mesh_motion_step(psi, rho, 2.0, 1.3, 0.5, passes=1)
    assert np.abs(psidot).max() < 1e-12
    np.testing.assert_allclose(new, psi - psi.mean(), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- symmetric variant


def test_sym_psi_zero_and_constant_B_symbol():
    # psi = 0: the 7-point operator; constant B: the same symbol as the literal scheme,
    # -sum_a 4 B_aa sin^2(k_a/2) - 2 sum_{a<b} B_ab sin k_a sin k_b (edge differences of
    # cos(k.x): E_a E_b products give sin k_a sin k_b)
    rng = np.random.default_rng(20)
    u = rng.standard_normal((8, 12, 16))
    for h in (1.0, 2.0):
        _, B = curv.geometry(np.zeros(u.shape), h)
        np.testing.assert_allclose(curv.apply_M_sym(u, B, h), flat.apply_A(u, h), atol=1e-13)
        np.testing.assert_allclose(curv.diag_M_sym(B, h), -6.0 / h ** 2, atol=1e-15)
    shape = (8, 12, 16)
    Bc = np.array([[1.3, 0.2, -0.15], [0.2, 0.9, 0.1], [-0.15, 0.1, 1.1]])
    B = np.broadcast_to(Bc[:, :, None, None, None], (3, 3) + shape).copy()
    z, y, x = coords(shape)
    for n in [(1, 2, 1), (3, 1, 2), (8, 6, 4), (5, 5, 3)]:
        k = (2 * np.pi * n[0] / shape[2], 2 * np.pi * n[1] / shape[1], 2 * np.pi * n[2] / shape[0])
        u = np.cos(k[0] * x + k[1] * y + k[2] * z + 0.4)
        sym = -sum(4 * Bc[a, a] * math.sin(k[a] / 2) ** 2 for a in range(3))
        sym -= 2 * sum(Bc[a, b] * math.sin(k[a]) * math.sin(k[b]) for a in range(3) for b in range(a + 1, 3))
        np.testing.assert_allclose(curv.apply_M_sym(u, B), sym * u, atol=1e-12)


def test_sym_operator_is_symmetric_with_19_points():
    lev = curv.Level(smoothed_grf((4, 6, 6), 21, 1.0, 0.4), 1.0, sym=True)
    M = curv.dense_L(lev) * lev.J.ravel()[:, None]            # M = J L
    np.testing.assert_allclose(M, M.T, atol=1e-14 * np.abs(M).max())
    np.testing.assert_allclose(np.diag(M), curv.diag_M_sym(lev.B).ravel(), atol=1e-13)
    np.testing.assert_allclose(M.sum(axis=0), 0.0, atol=1e-13)   # 1^T M = 0
    np.testing.assert_allclose(M.sum(axis=1), 0.0, atol=1e-13)   # M 1 = 0
    # the stencil: the centre, 6 face and 12 edge neighbours, no corners
    shape = (4, 6, 6)
    i = np.ravel_multi_index((1, 2, 3), shape)
    nz = {tuple(int(v) for v in np.subtract(np.unravel_index(j, shape), (1, 2, 3)))
          for j in np.nonzero(np.abs(M[i]) > 1e-15)[0]}
    assert len(nz) == 19 and all(sum(abs(c) for c in o) <= 2 for o in nz)
    # the literal scheme is not symmetric on the same geometry
    Ml = curv.dense_L(curv.Level(lev.psi, 1.0)) * lev.J.ravel()[:, None]
    assert np.abs(Ml - Ml.T).max() > 1e-4 * np.abs(Ml).max()


def test_sym_second_order_consistency_and_agreement_with_literal():
    sp = pytest.importorskip("sympy")
    X, Y, Z, N = sp.symbols("X Y Z N")
    w = 2 * sp.pi / N
    Bs = {(0, 0): 1 + sp.Rational(3, 10) * sp.sin(w * X), (1, 1): 1 + sp.Rational(1, 5) * sp.cos(w * Y),
          (2, 2): 1 + sp.Rational(1, 10) * sp.sin(w * (Z + X)), (0, 1): sp.Rational(1, 10) * sp.cos(w * (X + Y)),
          (0, 2): sp.Rational(1, 20) * sp.sin(w * Z), (1, 2): sp.Rational(2, 25) * sp.cos(w * (Y - Z))}
    for (a, b) in list(Bs):
        Bs[(b, a)] = Bs[(a, b)]
    us = sp.sin(w * X) * sp.cos(w * Y) + sp.Rational(1, 2) * sp.sin(w * (2 * Z + Y))
    var = (X, Y, Z)
    cont = sum(sp.diff(Bs[(a, b)] * sp.diff(us, var[b]), var[a]) for a in range(3) for b in range(3))
    fB = {k: sp.lambdify((X, Y, Z, N), v, "numpy") for k, v in Bs.items()}
    fu = sp.lambdify((X, Y, Z, N), us, "numpy")
    fc = sp.lambdify((X, Y, Z, N), cont, "numpy")
    errs, gaps = [], []
    for n in (16, 32, 64):
        z, y, x = coords((n, n, n))
        B = np.empty((3, 3, n, n, n))
        for a in range(3):
            for b in range(3):
                B[a, b] = fB[(a, b)](x, y, z, n) * np.ones_like(x)
        u = fu(x, y, z, n)
        num = curv.apply_M_sym(u, B)
        ref = fc(x, y, z, n)
        errs.append(np.abs(num - ref).max() / np.abs(ref).max())
        gaps.append(np.abs(num - curv.apply_M(u, B)).max() / np.abs(ref).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert gaps[0] / gaps[1] > 3.5 and gaps[1] / gaps[2] > 3.5, gaps   # the schemes differ at O(h^2)


def test_sym_Bbar_is_the_derivative_of_the_bilinear_form():
    # <lam, M_sym(B) phi> is linear in B: <Bbar, dB> = <lam, M_sym(dB) phi> exactly
    shape = (6, 8, 10)
    rng = np.random.default_rng(22)
    lam, phi = rng.standard_normal(shape), rng.standard_normal(shape)
    Bbar = curv.Bbar_from_operator_sym(lam, phi, 2.0)
    for trial in range(3):
        dB = rng.standard_normal((3, 3) + shape)
        dB = 0.5 * (dB + dB.transpose(1, 0, 2, 3, 4))
        lhs = float((Bbar * dB).sum())
        rhs = float((lam * curv.apply_M_sym(phi, dB, 2.0)).sum())
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


def test_sym_solve_dense_pinv_and_vjp_central_differences():
    n = 8
    psi = smoothed_grf(n, 23, 1.5, 0.4)
    delta = grf(n, 24)
    kw = dict(tol=1e-13, max_cycles=300, sym=True)
    phi, hist = curv.solve(delta, psi, **kw)
    lev = curv.hierarchy(psi, sym=True)[0]
    f = curv.weighted_projection(delta, lev.J)
    ref = (np.linalg.pinv(curv.dense_L(lev), rcond=1e-10) @ f.ravel()).reshape(f.shape)
    np.testing.assert_allclose(phi, ref - ref.mean(), atol=1e-10 * np.abs(ref).max())
    rng = np.random.default_rng(25)
    pbar = rng.standard_normal((n, n, n))
    dbar, psibar = curv.solve_vjp(delta, psi, phi, pbar, **kw)

    def loss(d, p):
        return float((curv.solve(d, p, **kw)[0] * pbar).sum())

    v = rng.standard_normal((n, n, n))
    eps = 1e-4
    fd = (loss(delta + eps * v, psi) - loss(delta - eps * v, psi)) / (2 * eps)
    assert abs(fd - float((dbar * v).sum())) < 1e-6 * max(1.0, abs(fd))
    wdir = smoothed_grf(n, 26, 1.5, 0.4)
    eps = 1e-3
    fd = (loss(delta, psi + eps * wdir) - loss(delta, psi - eps * wdir)) / (2 * eps)
    assert abs(fd - float((psibar * wdir).sum())) < 1e-5 * max(1.0, abs(fd))
