"""Moving-mesh kernels against the FP64 oracle across CTA tile seams (GPU).

The tiled curvilinear kernels (geometry, FP32 sweep and residual, double-float
residual, the psi-bar cotangent) work on 32 x 8 (x, y) tiles and chunks of z
planes.  These meshes span several tiles in x and y, end on ragged tiles on the
coarser levels (nx = 48 and ny = 20 at level 1 of 32 x 40 x 96), and split z into
several chunks, so a halo, periodic-wrap or tile-origin error at a seam shows up
element by element here.  Operators follow Sec. 4.3.1 (face-flux form), the
adjoint Sec. 4.8 (Eq. adj_rhs, adj_op) in its exact-transpose reading.
"""
import numpy as np
import pytest
import torch

from oracle import curv
from synth import grf, smoothed_grf

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPES = [(32, 40, 96), (64, 64, 64)]           # (nz, ny, nx)
ORDER = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def host(t):
    return t.double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver(gb, shape, psi, sym=False):
    s = gb.Solver(shape, op="curv", curv_sym=sym)
    s.set_geometry(to_dev(psi))
    return s


def gpu_coefficients(s, level):
    """The level's FP32 geometry as the oracle's FP64 (J, B[3, 3]) arrays."""
    J, B6 = s.curv_geometry(level)
    J, B6 = host(J), host(B6)
    B = np.empty((3, 3) + J.shape)
    for k, (a, b) in enumerate(ORDER):
        B[a, b] = B6[k]
        B[b, a] = B6[k]
    return J, B


def oracle_op(u, B, h, form):
    return {0: curv.apply_M, 1: curv.apply_MT, 2: curv.apply_M_sym}[form](u, B, h)


def oracle_diag(B, h, form):
    return curv.diag_M_sym(B, h) if form == 2 else curv.diag_M(B, h)


def forms(sym):
    # (transpose flag, oracle operator): M and M^T for the paper's scheme, S for either flag
    return [(False, 2), (True, 2)] if sym else [(False, 0), (True, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_geometry_every_level_across_tiles(gb, shape):
    psi = smoothed_grf(shape, 60, 2.0, 0.5)
    s = solver(gb, shape, psi)
    hier = curv.hierarchy(psi)
    assert s.levels == len(hier)
    for level in range(s.levels):
        J, B = gpu_coefficients(s, level)
        lev = hier[level]
        np.testing.assert_allclose(J, lev.J, rtol=2e-7, atol=0)
        for a, b in ORDER:
            np.testing.assert_allclose(B[a, b], lev.B[a, b], rtol=0, atol=3e-7 * np.abs(lev.B[a, a]).max())


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_operators_and_level_kernels_across_tiles(gb, shape, sym):
    # M, M^T (or S) through mg_curv_apply in FP64 and FP32, and the V-cycle's tiled FP32
    # residual and weighted-Jacobi sweep, all with the GPU's own FP32 coefficients,
    # on the two finest levels
    psi = smoothed_grf(shape, 61, 2.0, 0.5)
    s = solver(gb, shape, psi, sym)
    rng = np.random.default_rng(62)
    omega = 2.0 / 3.0
    for level in range(2):
        shp = s.level_shape(level)
        h = 2.0 ** level
        J, B = gpu_coefficients(s, level)
        u = rng.standard_normal(shp)
        r = rng.standard_normal(shp) / (h * h)
        u32, r32 = to_dev(u, torch.float32), to_dev(r, torch.float32)
        u3, r3 = host(u32), host(r32)
        for tr, form in forms(sym):
            ref = oracle_op(u, B, h, form) / J
            got = host(s.curv_apply(level, to_dev(u), transpose=tr, divide_by_J=True))
            assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
            got = host(s.curv_apply(level, u32, transpose=tr, divide_by_J=True))
            ref3 = oracle_op(u3, B, h, form) / J
            assert np.abs(got - ref3).max() < 2e-5 * np.abs(ref3).max()
            # tiled FP32 residual r - op(u) / (h^2 J)
            got = host(s.curv_residual(level, r32, u32, transpose=tr))
            ref = r3 - oracle_op(u3, B, h, form) / J
            assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()
            # tiled FP32 Jacobi sweep e + omega (J r - op(e)) / diag
            got = host(s.curv_smooth(level, u32, r32, transpose=tr))
            ref = u3 + omega * (J * r3 - oracle_op(u3, B, h, form)) / oracle_diag(B, h, form)
            assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_vcycle_across_tiles(gb, shape, sym):
    psi = smoothed_grf(shape, 63, 2.0, 0.5)
    s = solver(gb, shape, psi, sym)
    hier = curv.hierarchy(psi, sym=sym)
    rd = to_dev(grf(shape, 64), torch.float32)
    for tr in (False, True):
        got = host(s.curv_vcycle(rd, transpose=tr))
        ref = curv.vcycle(0, np.zeros(shape), host(rd), hier, transpose=tr, cache={})
        assert rel_l2(got, ref) < 2e-5


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_solve_across_tiles(gb, shape, sym):
    psi = smoothed_grf(shape, 65, 2.0, 0.5)
    delta = grf(shape, 66)
    s = solver(gb, shape, psi, sym)
    ref, _ = curv.solve(delta, psi, tol=1e-12, max_cycles=300, sym=sym)
    phi, st = s.solve(to_dev(delta), tol=1e-6, max_vcycles=100)
    assert st.status == 0 and st.rel_res <= 1e-6
    assert rel_l2(host(phi), ref) < 1e-6
    phi, st = s.solve(to_dev(delta), tol=1e-10, max_vcycles=200)
    assert st.status == 0
    # the remaining difference is the FP32 rounding of the geometry coefficients
    assert rel_l2(host(phi), ref) < 3e-7


@pytest.mark.parametrize("sym", [False, True])
def test_adjoint_across_tiles(gb, sym):
    shape = SHAPES[0]
    psi = smoothed_grf(shape, 67, 1.5, 0.4)
    delta = grf(shape, 68)
    pbar = np.random.default_rng(69).standard_normal(shape)
    s = solver(gb, shape, psi, sym)
    phi, _ = s.solve(to_dev(delta), tol=1e-11, max_vcycles=200)
    dbar, psibar, st = s.solve_adjoint(to_dev(pbar), phi=phi, source=to_dev(delta), want_psi_bar=True,
                                       tol=1e-11, max_vcycles=200)
    assert st.status == 0
    ref_phi, _ = curv.solve(delta, psi, tol=1e-13, max_cycles=400, sym=sym)
    rd, rp = curv.solve_vjp(delta, psi, ref_phi, pbar, tol=1e-13, max_cycles=400, sym=sym)
    assert rel_l2(host(dbar), rd) < 1e-6
    assert rel_l2(host(psibar), rp) < 1e-5


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_zero_iterate_sweep_equals_full_sweep(gb, shape, sym):
    # the V-cycle's first pre-smoothing sweep starts from e = 0 and runs pointwise; it must
    # give exactly the values of the full tiled sweep applied to a zero array
    psi = smoothed_grf(shape, 72, 2.0, 0.5)
    s = solver(gb, shape, psi, sym)
    rng = np.random.default_rng(73)
    for level in range(s.levels - 1):
        shp = s.level_shape(level)
        r = to_dev(rng.standard_normal(shp), torch.float32)
        for tr in (False, True):
            full = s.curv_smooth(level, torch.zeros_like(r), r, transpose=tr)
            point = s.curv_smooth(level, None, r, transpose=tr)
            assert torch.equal(full.view(torch.int32), point.view(torch.int32))   # bit for bit


@pytest.mark.parametrize("sym", [False, True])
def test_cycle_graphs_match_eager_cycles(gb, sym):
    # the curvilinear cycles run as CUDA graphs (one per orientation) unless switched
    # off: same iterates, cycles and histories for forward and adjoint solves, also after
    # the geometry has changed in place (a second psi), and the same timed launches
    shape = SHAPES[0]
    g = gb.Solver(shape, op="curv", curv_sym=sym)
    e = gb.Solver(shape, op="curv", curv_sym=sym)
    e.set_cycle_graphs(False)
    g.profile_begin(["curv0", "df0"])
    e.profile_begin(["curv0", "df0"])
    pbar = to_dev(np.random.default_rng(71).standard_normal(shape))
    for k in range(2):
        psi = to_dev(smoothed_grf(shape, 72 + k, 1.5, 0.4))
        delta = to_dev(grf(shape, 74 + k))
        pg, sg = g.solve(delta, tol=1e-9, max_vcycles=200, psi=psi)
        pe, se = e.solve(delta, tol=1e-9, max_vcycles=200, psi=psi)
        assert sg.cycles == se.cycles and sg.history == se.history
        assert torch.equal(pg, pe)
        dg, qg, ag = g.solve_adjoint(pbar, phi=pg, source=delta, want_psi_bar=True, tol=1e-9, max_vcycles=200)
        de, qe, ae = e.solve_adjoint(pbar, phi=pe, source=delta, want_psi_bar=True, tol=1e-9, max_vcycles=200)
        assert ag.cycles == ae.cycles and ag.history == ae.history
        assert torch.equal(dg, de) and torch.equal(qg, qe)
    for fam in ("curv0", "df0"):
        (cg, tg), (ce, te) = g.profile_read(fam), e.profile_read(fam)
        assert cg == ce > 0 and tg > 0.0 and te > 0.0
    g.profile_end()
    e.profile_end()
