"""Pins of the flat oracle against closed forms, brute force and library routines (CPU)."""
import itertools
import math
import os

import numpy as np
import numpy.polynomial.chebyshev as npcheb
import pytest

from oracle import flat
from synth import grf


def load_constants(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "paper_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def plane_wave(shape, n, phase=0.3):
    """cos(k.x + phase) with k_i = 2 pi n_i / N_i; returns (field, (kx, ky, kz))."""
    nz, ny, nx = shape
    kx, ky, kz = (2 * np.pi * n[0] / nx, 2 * np.pi * n[1] / ny, 2 * np.pi * n[2] / nz)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.cos(kx * x + ky * y + kz * z + phase), (kx, ky, kz)


def dense_laplacian(shape, h=1.0):
    """Dense 7-point periodic matrix built by explicit loops over cells and neighbours."""
    nz, ny, nx = shape
    n = nx * ny * nz
    M = np.zeros((n, n))
    idx = lambda z, y, x: ((z % nz) * ny + (y % ny)) * nx + (x % nx)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(z, y, x)
                M[i, i] += -6.0 / h ** 2
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    M[i, idx(z + dz, y + dy, x + dx)] += 1.0 / h ** 2
    return M


@pytest.mark.parametrize("shape", [(8, 12, 16), (16, 16, 16)])
def test_plane_wave_eigenvalue(shape):
    # Sec. 2.2 symbol lambda = -(4/h^2) sum sin^2(k_i h / 2); Sec. 4.3.1 symbol (2cos kx + 2cos ky + 2cos kz - 6)/dx^2
    for n in [(1, 0, 0), (2, 3, 1), (shape[2] // 2, shape[1] // 2, shape[0] // 2), (3, 1, 2)]:
        u, (kx, ky, kz) = plane_wave(shape, n)
        for h in (1.0, 2.0):
            lam_sin = -4.0 / h ** 2 * (math.sin(kx / 2) ** 2 + math.sin(ky / 2) ** 2 + math.sin(kz / 2) ** 2)
            lam_cos = (2 * math.cos(kx) + 2 * math.cos(ky) + 2 * math.cos(kz) - 6) / h ** 2
            assert abs(lam_sin - lam_cos) < 1e-13
            np.testing.assert_allclose(flat.apply_A(u, h), lam_sin * u, atol=1e-12)
    lam = flat.eigenvalues(shape, rfft=False)
    assert lam.shape == shape and abs(lam[0, 0, 0]) == 0.0


def test_checkerboard_is_top_of_jacobi_spectrum(golden_dir):
    c = load_constants(golden_dir)
    u, _ = plane_wave((8, 8, 8), (4, 4, 4), phase=0.0)     # (-1)^(x+y+z)
    mu = flat.apply_A(u) / (-6.0) / u
    np.testing.assert_allclose(mu, c["chebyshev_upper"], rtol=1e-14)


def test_fft_solve_matches_dense_pinv_8():
    shape = (8, 8, 8)
    F = grf(shape, 11)
    F = F + 0.7          # a non-zero mean must be projected out
    P = np.linalg.pinv(dense_laplacian(shape), rcond=1e-10)
    ref = (P @ F.ravel()).reshape(shape)
    np.testing.assert_allclose(flat.fft_solve(F), ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 8, 32)])
def test_fft_solve_residual_and_gauge(shape):
    F = grf(shape, 3)
    phi = flat.fft_solve(F)
    assert abs(phi.mean()) < 1e-14 * np.abs(phi).max()
    r = flat.project_mean(F) - flat.apply_A(phi)
    assert np.linalg.norm(r) / np.linalg.norm(F) < 1e-13


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5])
def test_chebyshev_plane_wave_factor(degree, golden_dir):
    c = load_constants(golden_dir)
    a, b = 2.0 / c["chebyshev_alpha"], c["chebyshev_upper"]
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    shape = (16, 16, 16)
    coef = np.zeros(degree + 1)
    coef[-1] = 1.0
    for n in [(1, 0, 0), (3, 2, 1), (8, 8, 8), (5, 0, 7), (8, 0, 0)]:
        e0, (kx, ky, kz) = plane_wave(shape, n)
        mu = 1.0 - (math.cos(kx) + math.cos(ky) + math.cos(kz)) / 3.0
        factor = npcheb.chebval((theta - mu) / delta, coef) / npcheb.chebval(theta / delta, coef)
        for h in (1.0, 4.0):
            e = flat.smooth_chebyshev(e0, np.zeros(shape), h, degree, c["chebyshev_alpha"])
            np.testing.assert_allclose(e, factor * e0, atol=1e-12)


def test_jacobi_plane_wave_factor(golden_dir):
    omega = load_constants(golden_dir)["jacobi_omega"]
    shape = (16, 16, 16)
    for n in [(1, 0, 0), (3, 2, 1), (8, 8, 8)]:
        e0, (kx, ky, kz) = plane_wave(shape, n)
        mu = 1.0 - (math.cos(kx) + math.cos(ky) + math.cos(kz)) / 3.0
        for sweeps in (1, 2, 3):
            e = flat.smooth_jacobi(e0, np.zeros(shape), 2.0, sweeps, omega)
            np.testing.assert_allclose(e, (1 - omega * mu) ** sweeps * e0, atol=1e-13)


def _matrix_of(fun, in_shape):
    n = int(np.prod(in_shape))
    cols = []
    for j in range(n):
        v = np.zeros(n)
        v[j] = 1.0
        cols.append(fun(v.reshape(in_shape)).ravel())
    return np.stack(cols, axis=1)


def test_restriction_is_prolongation_transpose_over_8():
    fine, coarse = (8, 8, 12), (4, 4, 6)
    R = _matrix_of(flat.restrict_fw, fine)
    P = _matrix_of(flat.prolong, coarse)
    assert R.shape == (np.prod(coarse), np.prod(fine))
    np.testing.assert_array_equal(R, P.T / 8.0)
    np.testing.assert_allclose(R @ np.ones(R.shape[1]), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(P @ np.ones(P.shape[1]), 1.0, rtol=0, atol=1e-15)


def test_restriction_is_27_tap_tensor_weights():
    # "27-tap" full weighting with the 1-D weights [1/4, 1/2, 1/4] (Sec. 3.4; Appendix B)
    fine = (8, 8, 8)
    w = {-1: 0.25, 0: 0.5, 1: 0.25}
    for (a, b, c) in itertools.product((-1, 0, 1), repeat=3):
        r = np.zeros(fine)
        r[(2 + c) % 8, (4 + b) % 8, (6 + a) % 8] = 1.0          # fine node 2I + (a,b,c), I = (3,2,1) in (x,y,z)
        rc = flat.restrict_fw(r)
        assert rc[1, 2, 3] == w[a] * w[b] * w[c]
        # an odd fine index along an axis is shared by two coarse nodes on that axis
        assert np.count_nonzero(rc) == 2 ** (abs(a) + abs(b) + abs(c))


def test_prolongation_exact_on_linear_functions():
    coarse = (6, 6, 6)
    z, y, x = np.meshgrid(*(np.arange(s, dtype=float) for s in coarse), indexing="ij")
    ec = 1.5 * x - 0.25 * y + 2.0 * z + 0.5
    ef = flat.prolong(ec)
    Z, Y, X = np.meshgrid(*(np.arange(2 * s, dtype=float) for s in coarse), indexing="ij")
    exact = 1.5 * X / 2 - 0.25 * Y / 2 + 2.0 * Z / 2 + 0.5
    interior = (slice(0, 2 * coarse[0] - 1),) * 3           # no periodic wrap
    np.testing.assert_allclose(ef[interior], exact[interior], atol=1e-13)


@pytest.mark.parametrize("shape,h", [((4, 4, 4), 8.0), ((6, 6, 6), 16.0), ((4, 6, 8), 2.0)])
def test_coarse_solve_is_pseudo_inverse(shape, h):
    r = grf(shape, 5) + 0.3
    P = np.linalg.pinv(dense_laplacian(shape, h), rcond=1e-10)
    np.testing.assert_allclose(flat.coarse_solve(r, h), (P @ r.ravel()).reshape(shape),
                               atol=1e-12 * np.abs(r).max() * h * h)


def test_levels_golden(golden_dir):
    with open(os.path.join(golden_dir, "levels.txt")) as fh:
        rows = [tuple(int(v) for v in l.split()) for l in fh if l.strip() and not l.startswith("#")]
    for n, L in rows:
        assert len(flat.level_shapes((n, n, n))) == L
    assert flat.level_shapes((96, 96, 96))[-1] == (6, 6, 6)
    assert flat.level_shapes((32, 32, 32), levels=2) == [(32, 32, 32), (16, 16, 16)]


def test_hierarchy_work_bound(golden_dir):
    c = load_constants(golden_dir)
    shapes = flat.level_shapes((1024,) * 3)
    ratio = sum(np.prod(s) for s in shapes) / 1024 ** 3
    assert ratio < c["hierarchy_work"] and abs(ratio - c["hierarchy_work"]) < 1e-3


def test_plain_method_32_converges_to_fft():
    # plain-method workload: 32^3, FP64, 4 levels, V(3,3) Chebyshev, phi = 0, tol 1e-10
    F = grf(32, 1)
    phi, hist = flat.mg_solve(F, tol=1e-10, max_cycles=50)
    assert len(flat.level_shapes(F.shape)) == 4
    assert hist[-1] <= 1e-10 and len(hist) - 1 <= 15
    ref = flat.fft_solve(F)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-10


def test_convergence_factor_mesh_independent(golden_dir):
    c = load_constants(golden_dir)
    rhos = []
    for n in (16, 32, 64):
        F = grf(n, 21)
        _, hist = flat.mg_solve(F, fixed_cycles=5)
        rhos.append((hist[5] / hist[2]) ** (1 / 3))
    assert all(0.3 * c["vcycle_rho_order"] < r < 2 * c["vcycle_rho_order"] for r in rhos), rhos
    assert max(rhos) / min(rhos) < 1.5


def test_jacobi_cycle_weaker_than_chebyshev():
    F = grf(32, 22)
    _, hc = flat.mg_solve(F, fixed_cycles=4)
    _, hj = flat.mg_solve(F, fixed_cycles=4, smoother="jacobi")
    assert hc[-1] < hj[-1]


def test_defect_correction_equals_vcycles_on_phi():
    F = grf(16, 31)
    phi0 = flat.fft_solve(F) + 0.01 * grf(16, 32)
    a, _ = flat.mg_solve(F, phi0=phi0, fixed_cycles=3)
    b = flat.defect_correction_solve(F, phi0, 3)
    np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())


def test_warm_start_cycle_saving():
    # Eq. (kwarm): k_warm ~ k_cold - log(1/eps)/log(1/rho)
    n, tol = 32, 1e-8
    d0, eta = grf(n, 2), grf(n, 3)
    F1 = d0 + 0.05 * eta
    phi0, _ = flat.mg_solve(d0, tol=1e-12)
    _, hc = flat.mg_solve(F1, tol=tol)
    _, hw = flat.mg_solve(F1, phi0=phi0, tol=tol)
    k_cold, k_warm = len(hc) - 1, len(hw) - 1
    rho = (hc[-1] / hc[1]) ** (1.0 / (k_cold - 1))
    exact1 = flat.fft_solve(F1)
    eps = np.linalg.norm(exact1 - phi0) / np.linalg.norm(exact1)
    predicted = k_cold - math.log(1 / eps) / math.log(1 / rho)
    assert k_warm < k_cold
    assert abs(k_warm - predicted) <= 1.5, (k_cold, k_warm, predicted)


def test_predictors_exact_on_their_sequences():
    """Sec. 3.2 predictors: growth scaling is exact on a pure-growth sequence, linear
    (quadratic) extrapolation on sequences linear (quadratic) in the step index, and
    linear extrapolation of a quadratic sequence misses by exactly twice its t^2 term."""
    rng = np.random.default_rng(11)
    a, b, c = (rng.standard_normal((4, 5, 6)) for _ in range(3))
    g = 1.25
    grow = [a]
    for _ in range(3):
        grow.append(g * grow[-1])
    assert np.array_equal(flat.predict([grow[2]], 0, g), grow[3])
    assert np.array_equal(flat.predict([grow[2]], 0), grow[2])
    lin = [a + t * b for t in range(4)]
    np.testing.assert_allclose(flat.predict([lin[2], lin[1]], 1), lin[3], rtol=0, atol=1e-14)
    quad = [a + t * b + t * t * c for t in range(5)]
    np.testing.assert_allclose(flat.predict([quad[3], quad[2], quad[1]], 2), quad[4], rtol=0, atol=1e-13)
    np.testing.assert_allclose(quad[4] - flat.predict([quad[3], quad[2]], 1), 2.0 * c, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        flat.predict([a], 3)


def test_extrapolation_saves_cycles_on_a_smooth_sequence():
    """Eq. kwarm with the predictors: on sources drifting smoothly (here linearly) in
    the step index, linear extrapolation starts orders of magnitude closer than
    recycling and needs fewer cycles to the same tolerance."""
    from synth import grf
    n = 16
    d0, eta = grf(n, 2), grf(n, 3)
    F = [d0 + 0.05 * t * eta for t in range(4)]
    sols = []
    for t in range(3):
        phi, _ = flat.mg_solve(F[t], phi0=sols[-1] if sols else None, tol=1e-12)
        sols.append(phi)
    _, rec = flat.mg_solve(F[3], phi0=sols[2], tol=1e-8)
    _, lin = flat.mg_solve(F[3], phi0=flat.predict([sols[2], sols[1]], 1), tol=1e-8)
    _, quad = flat.mg_solve(F[3], phi0=flat.predict([sols[2], sols[1], sols[0]], 2), tol=1e-8)
    assert lin[0] < 1e-3 * rec[0] and quad[0] < 1e-3 * rec[0]
    assert len(lin) < len(rec) and len(quad) < len(rec)


def test_pcg_exact_preconditioner_converges_in_one_step():
    """With the exact inverse on the zero-mean subspace as preconditioner, alpha = 1 and one
    PCG step is the solution."""
    r = flat.project_mean(grf(8, 41))
    e, _ = flat.pcg(r, 1, lambda v: flat.fft_solve(v), flat.apply_A)
    np.testing.assert_allclose(e, flat.fft_solve(r), rtol=0, atol=1e-12 * np.abs(e).max())


def test_pcg_terminates_within_the_distinct_eigenvalues():
    """Unpreconditioned CG on the 4^3 periodic Laplacian: the symbol 2(cos kx + cos ky + cos kz) - 6
    with cos in {1, 0, -1} takes 6 distinct nonzero values, so CG (exact arithmetic) ends
    within 6 steps on a zero-mean right-hand side."""
    r = flat.project_mean(np.random.default_rng(42).standard_normal((4, 4, 4)))
    lam = np.unique(np.round(flat.eigenvalues((4, 4, 4), rfft=False), 12))
    assert len(lam[lam != 0]) == 6
    e, its = flat.pcg(r, 6, lambda v: v, flat.apply_A)
    assert np.linalg.norm(flat.apply_A(e) - r) < 1e-12 * np.linalg.norm(r)
    e5, _ = flat.pcg(r, 5, lambda v: v, flat.apply_A)
    assert np.linalg.norm(flat.apply_A(e5) - r) > 1e-8 * np.linalg.norm(r)


def test_pcg_energy_decreases_and_first_step_is_scaled_vcycle():
    """MG-preconditioned CG: the error energy (e - e*, -A (e - e*)) decreases at every step,
    and the first step is the V-cycle correction scaled by alpha = (r, z) / (z, A z)."""
    n = 16
    r = flat.project_mean(grf(n, 43))
    nlev = len(flat.level_shapes((n, n, n)))
    M = lambda v: flat.vcycle(0, np.zeros_like(v), v, nlev)
    exact = flat.fft_solve(r)
    _, its = flat.pcg(r, 4, M, flat.apply_A)
    energy = [float(np.vdot(x - exact, -flat.apply_A(x - exact))) for x in its]
    assert all(b < a for a, b in zip(energy, energy[1:]))
    z = M(r)
    alpha = float(np.vdot(r, z)) / float(np.vdot(z, flat.apply_A(z)))
    np.testing.assert_allclose(its[0], alpha * z, rtol=0, atol=1e-13 * np.abs(z).max())


def test_mg_pcg_solve_converges_faster_than_vcycles():
    n = 32
    F = grf(n, 44)
    phi, hist = flat.mg_pcg_solve(F, inner_steps=2, tol=1e-10)
    np.testing.assert_allclose(phi, flat.fft_solve(F), rtol=0, atol=1e-9 * np.abs(phi).max())
    _, plain = flat.mg_solve(F, tol=1e-10)
    # two preconditioned steps per outer step beat two plain cycles per outer step
    assert 2 * (len(hist) - 1) <= len(plain) - 1
