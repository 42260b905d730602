"""Pins of the C FP64 V-cycle oracle (oracle/mg_fp64.c) on the CPU.

The C oracle restates oracle/flat.py (Sec. 2.1-2.3, Appendix B) so that a full 512^3
solve can be timed on the host cores.  It is pinned here to closed forms (plane-wave
eigenvalues of the 7-point operator, the Chebyshev error factor, the pseudo-inverse of
the coarsest operator) and to the NumPy oracle's V-cycle iterates, which are pinned in
tests/test_oracle_flat.py.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

from oracle import cmg, flat
from synth import grf

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def plane_wave(shape, n):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = [2 * np.pi * n[0] / nx, 2 * np.pi * n[1] / ny, 2 * np.pi * n[2] / nz]
    return np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3), k


@pytest.mark.parametrize("h", [1.0, 4.0])
def test_operator_plane_wave_eigenvalues(h):
    # Eq. (fftsolve): A cos(k.x) = (2 cos kx + 2 cos ky + 2 cos kz - 6) / h^2 cos(k.x)
    shape = (8, 12, 16)
    for n in [(1, 0, 0), (0, 2, 0), (3, 5, 1), (8, 6, 4), (5, 1, 3)]:
        u, k = plane_wave(shape, n)
        lam = (2 * np.cos(k[0]) + 2 * np.cos(k[1]) + 2 * np.cos(k[2]) - 6) / h ** 2
        np.testing.assert_allclose(cmg.apply_A(u, h), lam * u, rtol=0, atol=1e-13 / h ** 2)


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_plane_wave_factor(degree):
    # e <- p(D^-1 A) e on A e = 0: factor T_v((theta - mu)/delta) / T_v(theta/delta), mu the
    # eigenvalue of D^-1 A on the wave, [a, b] = [2/alpha, 2] (Sec. 2.3)
    shape = (8, 8, 16)
    a, b = 0.25, 2.0
    theta, delta = (a + b) / 2, (b - a) / 2
    Tv = [0] * degree + [1]
    for n in [(1, 0, 0), (2, 3, 1), (8, 4, 4), (5, 2, 3)]:
        u, k = plane_wave(shape, n)
        mu = 1 - (np.cos(k[0]) + np.cos(k[1]) + np.cos(k[2])) / 3
        f = C.chebval((theta - mu) / delta, Tv) / C.chebval(theta / delta, Tv)
        got = cmg.smooth_chebyshev(u, np.zeros(shape), 2.0, degree)
        np.testing.assert_allclose(got, f * u, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape,levels,h", [((4, 4, 4), 1, 1.0), ((8, 8, 8), 2, 2.0), ((4, 6, 8), 1, 1.0)])
def test_coarsest_solve_is_the_pseudo_inverse(shape, levels, h):
    # the coarsest level's solve is the minimum-norm solve: numpy's dense pinv of the
    # operator of that level (spacing h), applied to a random right-hand side
    s = cmg.Solver(shape, levels=levels)
    assert s.levels == levels
    cshape = tuple(v // 2 ** (levels - 1) for v in shape)
    n = int(np.prod(cshape))
    Adense = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Adense[:, j] = flat.apply_A(e.reshape(cshape), h).ravel()
    G = np.linalg.pinv(Adense, rcond=1e-10)
    if levels == 1:
        r = np.random.default_rng(1).standard_normal(shape)
        np.testing.assert_allclose(s.vcycle(r).ravel(), G @ r.ravel(), rtol=0, atol=1e-12 * np.abs(G @ r.ravel()).max())
    else:
        # through one V-cycle: the same cycle in the NumPy oracle, whose coarsest solve is the FFT
        r = np.random.default_rng(2).standard_normal(shape)
        ref = flat.vcycle(0, np.zeros(shape), r, levels)
        np.testing.assert_allclose(s.vcycle(r), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 32), (24, 24, 24)])
def test_vcycle_iterates_match_numpy_oracle(shape):
    s = cmg.Solver(shape)
    assert s.levels == len(flat.level_shapes(shape))
    r = grf(shape, 3)
    ref = flat.vcycle(0, np.zeros(shape), r, s.levels)
    got = s.vcycle(r)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # solves: cold and warm, the residual histories and the results
    F = grf(shape, 4) + 0.25
    p_ref, h_ref = flat.mg_solve(F, tol=1e-10, max_cycles=40)
    p, h = s.solve(F, tol=1e-10, max_cycles=40)
    assert len(h) == len(h_ref)
    np.testing.assert_allclose(h, h_ref, rtol=1e-6, atol=1e-15)
    assert np.abs(p - p_ref).max() <= 1e-12 * np.abs(p_ref).max()
    F2 = F + 0.05 * grf(shape, 5)
    p2_ref, h2_ref = flat.mg_solve(F2, phi0=p_ref, tol=1e-10, max_cycles=40)
    p2, h2 = s.solve(F2, phi0=p, tol=1e-10, max_cycles=40)
    np.testing.assert_allclose(h2, h2_ref, rtol=1e-6, atol=1e-15)
    assert np.abs(p2 - p2_ref).max() <= 1e-12 * np.abs(p2_ref).max()


def test_c1_solve_reaches_the_fft_solution():
    # configuration 1: 32^3, V(3,3) Chebyshev, 4 levels, phi = 0, tol 1e-10
    F = grf(32, 1)
    s = cmg.Solver(32)
    assert s.levels == 4
    phi, h = s.solve(F, tol=1e-10, max_cycles=50)
    assert h[-1] <= 1e-10 and len(h) - 1 <= 15
    ref = flat.fft_solve(F)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-9
    # the convergence factor is the multigrid one (~0.1 per cycle, Sec. 2.3)
    rho = (h[-1] / h[1]) ** (1.0 / (len(h) - 2))
    assert rho < 0.2


def test_stepwise_solve_equals_solve():
    F = grf(16, 6)
    s = cmg.Solver(16)
    phi, h = s.solve(F, tol=1e-9, max_cycles=30)
    rel = [s.begin(F, np.zeros_like(F))]
    while rel[-1] > 1e-9:
        rel.append(s.cycle())
    assert rel == h
    np.testing.assert_array_equal(s.end(), phi)


def test_results_do_not_depend_on_thread_count():
    F = grf((16, 24, 32), 7)
    out = []
    orig = cmg.threads()
    for t in (1, 3):
        cmg.set_threads(t)
        out.append(cmg.Solver((16, 24, 32)).solve(F, tol=1e-8, max_cycles=20))
    cmg.set_threads(orig)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_unsupported_meshes_are_rejected():
    with pytest.raises(ValueError):
        cmg.Solver((2, 8, 8))
    with pytest.raises(ValueError):
        cmg.Solver((34, 34, 34))     # coarsest 17^3 cells: above the 4096 the dense solve takes
