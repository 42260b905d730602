"""Parity of the CUDA flat path with the FP64 oracle, through the C ABI (GPU)."""
import numpy as np
import pytest
import torch

from oracle import flat
from synth import grf

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPES = [(32, 32, 32), (16, 8, 32), (24, 24, 24), (12, 12, 12)]


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 2e-6)])
def test_apply_and_residual(gb, shape, dtype, tol):
    s = gb.Solver(shape, prec="fp64")
    for level in range(min(2, s.levels)):
        shp = s.level_shape(level)
        h = 2.0 ** level
        u, f = rand(shp, 1), rand(shp, 2)
        ud = to_dev(u, dtype)
        u32 = ud.double().cpu().numpy()
        f32 = to_dev(f, dtype).double().cpu().numpy()
        got = s.apply(level, ud).double().cpu().numpy()
        ref = flat.apply_A(u32, h)
        assert rel_max(got, ref) < tol * 12
        got = s.residual(level, to_dev(f, dtype), ud).double().cpu().numpy()
        assert rel_max(got, flat.residual(f32, u32, h)) < tol * 12


@pytest.mark.parametrize("smoother", ["chebyshev", "jacobi"])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_smoothers(gb, smoother, dtype, tol):
    s = gb.Solver((16, 8, 32), prec="fp64", smoother=smoother, degree=4, nu1=3)
    for level in range(s.levels):
        shp = s.level_shape(level)
        h = 2.0 ** level
        e, r = rand(shp, 3), rand(shp, 4)
        ed, rd = to_dev(e, dtype), to_dev(r, dtype)
        e_in, r_in = ed.double().cpu().numpy(), rd.double().cpu().numpy()
        got = s.smooth(level, ed, rd).double().cpu().numpy()
        if smoother == "chebyshev":
            ref = flat.smooth_chebyshev(e_in, r_in, h, 4, 8.0)
        else:
            ref = flat.smooth_jacobi(e_in, r_in, h, 3, 2.0 / 3.0)
        assert rel_max(got, ref) < tol


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-15), (torch.float32, 1e-6)])
def test_transfers(gb, shape, dtype, tol):
    s = gb.Solver(shape, prec="fp64")
    for level in range(s.levels - 1):
        fine = rand(s.level_shape(level), 5)
        fd = to_dev(fine, dtype)
        got = s.restrict(level, fd).double().cpu().numpy()
        assert rel_max(got, flat.restrict_fw(fd.double().cpu().numpy())) < tol
        coarse = rand(s.level_shape(level + 1), 6)
        cd = to_dev(coarse, dtype)
        base = rand(s.level_shape(level), 7)
        bd = to_dev(base, dtype)
        ref = bd.double().cpu().numpy() + flat.prolong(cd.double().cpu().numpy())
        got = s.prolong_add(level, cd, bd).double().cpu().numpy()
        assert rel_max(got, ref) < tol * 4


@pytest.mark.parametrize("shape", [(32, 48, 64), (24, 24, 24), (16, 8, 32), (24, 20, 40), (20, 20, 20)])
def test_prolong_add_fp32_forms_agree_bit_for_bit(gb, shape):
    # FP32 prolongation into an 8-byte-aligned buffer runs one thread per coarse cell with
    # x-pair accesses; into a view that starts one float further it runs one thread per
    # fine cell: the same midpoints in the same order, so the same bits
    s = gb.Solver(shape, prec="mixed")
    for level in range(s.levels - 1):
        fshape = s.level_shape(level)
        base = to_dev(rand(fshape, 7), torch.float32)
        coarse = to_dev(rand(s.level_shape(level + 1), 6), torch.float32)
        aligned = base.clone()
        buf = torch.empty(base.numel() + 1, dtype=torch.float32, device=DEV)
        shifted = buf[1:].view(fshape)
        shifted.copy_(base)
        s.prolong_add(level, coarse, aligned)
        s.prolong_add(level, coarse, shifted)
        torch.cuda.synchronize()
        assert aligned.data_ptr() % 8 == 0 and shifted.data_ptr() % 8 == 4
        assert torch.equal(aligned, shifted)


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 24, 24), (16, 8, 32), (8, 8, 8)])
def test_coarse_solve(gb, shape):
    s = gb.Solver(shape, prec="fp64")
    cshape = s.level_shape(s.levels - 1)
    h = 2.0 ** (s.levels - 1)
    r = rand(cshape, 8) + 0.25
    ref = flat.coarse_solve(r, h)
    got = s.coarse_solve(to_dev(r)).cpu().numpy()
    assert rel_max(got, ref) < 1e-12
    got32 = s.coarse_solve(to_dev(r, torch.float32)).double().cpu().numpy()
    assert rel_max(got32, ref) < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 8, 32), (24, 24, 24)])
def test_vcycle_matches_oracle(gb, prec, tol, shape):
    s = gb.Solver(shape, prec=prec, fused=False)
    r = grf(shape, 9)
    rd = to_dev(r, s.work_dtype)
    got = s.vcycle(rd).double().cpu().numpy()
    ref = flat.vcycle(0, np.zeros(shape), rd.double().cpu().numpy(), s.levels)
    assert rel_max(got, ref) < tol


def test_df_conversions_bit_exact(gb):
    rng = np.random.default_rng(10)
    x = np.concatenate([
        rng.standard_normal(100000) * 10.0 ** rng.integers(-30, 30, 100000),
        np.array([0.0, -0.0, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -24 + 2.0 ** -50,
                  2.0 ** -126, 3.4e38, -3.0e38, 1e-300, 123456789.123456789, np.pi * 1e20]),
    ])
    s = gb.Solver(8, prec="mixed")
    df = s.f64_to_df(to_dev(x)).cpu().numpy()
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    normal = np.abs(x) >= 2.0 ** -126
    np.testing.assert_array_equal(df[normal, 0], hi[normal])
    np.testing.assert_array_equal(df[normal, 1], lo[normal])
    assert np.all(df[~normal, 0] == 0.0)
    back = s.df_to_f64(to_dev(df, torch.float32)).cpu().numpy()
    big = np.abs(x) >= 2.0 ** -100
    err = np.abs(back[big] - x[big]) / np.abs(x[big])
    assert err.max() < 2.0 ** -46
    special = s.f64_to_df(to_dev(np.array([np.inf, -np.inf, np.nan]))).cpu().numpy()
    assert np.isposinf(special[0, 0]) and np.isneginf(special[1, 0]) and np.isnan(special[2, 0])
    # 8-byte-aligned views take the one-element kernels; same values
    xd = to_dev(x)
    np.testing.assert_array_equal(s.f64_to_df(xd[1:]).cpu().numpy(), df[1:])
    dd = to_dev(df, torch.float32)
    np.testing.assert_array_equal(s.df_to_f64(dd[1:]).cpu().numpy(), back[1:])


@pytest.mark.parametrize("n", [32, 64])
def test_df_residual_matches_fp64(gb, n):
    F = grf(n, 11) + 0.3
    phi = flat.fft_solve(F) * (1 + 1e-4) + 1e-3 * grf(n, 12)
    m = float(F.mean())
    s = gb.Solver(n, prec="mixed")
    r = s.df_residual(s.f64_to_df(to_dev(F)), m, s.f64_to_df(to_dev(phi))).double().cpu().numpy()
    ref = flat.residual(F - m, phi)
    tol = 1e-7 * np.abs(ref) + 1e-12 * np.abs(phi).max()
    assert np.all(np.abs(r - ref) <= tol), float(np.abs(r - ref).max())


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 8, 32)])
def test_plain_fp64_solve_plain_method(gb, shape):
    # plain-method workload: FP64, V(3,3) Chebyshev, 4 levels at 32^3, phi = 0, tol 1e-10
    F = grf(shape, 1)
    s = gb.Solver(shape, prec="fp64")
    phi, st = s.solve(to_dev(F), tol=1e-10, max_vcycles=50)
    assert st.status == 0 and st.rel_res <= 1e-10
    ref = flat.fft_solve(F)
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10
    _, hist = flat.mg_solve(F, tol=1e-10)
    assert st.cycles == len(hist) - 1
    np.testing.assert_allclose(st.history, hist[1:], rtol=1e-3)


def test_fixed_cycle_iterates_match_oracle(gb):
    F = grf(32, 13)
    phi0 = flat.fft_solve(grf(32, 14))
    ref, _ = flat.mg_solve(F, phi0=phi0, fixed_cycles=3)
    s = gb.Solver(32, prec="fp64")
    # tol 0 never converges, so exactly max_vcycles cycles run
    phi, st = s.solve(to_dev(F), to_dev(phi0), tol=0.0, max_vcycles=3)
    assert st.cycles == 3 and st.status == 4
    assert rel_max(phi.cpu().numpy(), ref) < 1e-12
    sm = gb.Solver(32, prec="mixed", fused=False)
    phim, _ = sm.solve(to_dev(F), to_dev(phi0), tol=0.0, max_vcycles=3)
    assert np.linalg.norm(phim.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("fused", [0, 2])
@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (16, 8, 32), (48, 48, 48), (56, 40, 112)])
def test_mixed_solve_to_1e6(gb, shape, fused):
    F = grf(shape, 15)
    s = gb.Solver(shape, prec="mixed", fused=fused)
    phi, st = s.solve(to_dev(F), tol=1e-6, max_vcycles=40)
    assert st.status == 0 and st.rel_res <= 1e-6
    ref = flat.fft_solve(F)
    err = np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-6
    # the mixed solve can go far below FP32 accuracy thanks to the double-float outer loop
    phi, st = s.solve(to_dev(F), tol=1e-11, max_vcycles=60)
    assert st.status == 0
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_warm_start_saves_cycles(gb):
    n = 64
    d0, eta = grf(n, 2), grf(n, 3)
    s = gb.Solver(n, prec="mixed")
    phi, st0 = s.solve(to_dev(d0), tol=1e-6)
    F1 = d0 + 0.05 * eta
    _, cold = s.solve(to_dev(F1), tol=1e-6)
    warm_phi, warm = s.solve(to_dev(F1), phi.clone(), tol=1e-6)
    assert warm.cycles < cold.cycles
    assert abs(warm.rel_res0 - 0.05 * np.linalg.norm(eta) / np.linalg.norm(F1)) < 0.01
    ref = flat.fft_solve(F1)
    assert np.linalg.norm(warm_phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-6


def test_host_buffer_solve_matches_device(gb):
    n = 32
    F = grf(n, 16)
    s = gb.Solver(n, prec="mixed")
    phi_d, st_d = s.solve(to_dev(F), tol=1e-8)
    # pageable numpy buffers: staged through device copies
    phi_h = np.zeros_like(F)
    _, st_h = s.solve_host(F, phi_h, tol=1e-8)
    assert st_h.cycles == st_d.cycles
    np.testing.assert_array_equal(phi_h, phi_d.cpu().numpy())
    # page-locked buffers, read and written in place by the conversion kernels, from a
    # nonzero initial guess (the initial phi is read from host memory too)
    phi0 = grf(n, 19)
    phi_d2, st_d2 = s.solve(to_dev(F), to_dev(phi0), tol=1e-8)
    Fp = torch.from_numpy(F.copy()).pin_memory()
    phi_p = torch.from_numpy(phi0.copy()).pin_memory()
    _, st_p = s.solve_host(Fp, phi_p, tol=1e-8)
    assert st_p.cycles == st_d2.cycles
    np.testing.assert_array_equal(phi_p.numpy(), phi_d2.cpu().numpy())
    np.testing.assert_array_equal(Fp.numpy(), F)   # the source is not written
    # FP64 precision with page-locked buffers takes the staged path
    s64 = gb.Solver(n, prec="fp64")
    phi_d3, st_d3 = s64.solve(to_dev(F), tol=1e-10)
    phi_p3 = torch.zeros((n, n, n), dtype=torch.float64).pin_memory()
    _, st_p3 = s64.solve_host(Fp, phi_p3, tol=1e-10)
    assert st_p3.cycles == st_d3.cycles
    np.testing.assert_array_equal(phi_p3.numpy(), phi_d3.cpu().numpy())


def _device_chain(s, Fs, phi0, tol):
    phi = to_dev(phi0) if phi0 is not None else torch.zeros((s.shape), dtype=torch.float64, device="cuda")
    out, stats = [], []
    for F in Fs:
        phi = phi.clone()
        phi, st = s.solve(to_dev(F), phi, tol=tol)
        out.append(phi.cpu().numpy())
        stats.append(st)
    return out, stats


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_host_sequence_matches_chained_device_solves(gb, prec):
    n, T = 32, 5
    tol = 1e-8 if prec == "mixed" else 1e-10
    rng = np.random.default_rng(3)
    base = grf(n, 40)
    Fs = [base + 0.05 * t * grf(n, 41) + 0.01 * rng.standard_normal(base.shape) for t in range(T)]
    s = gb.Solver(n, prec=prec)
    # page-locked buffers, zero start
    ref, ref_st = _device_chain(s, Fs, None, tol)
    src = [torch.from_numpy(F.copy()).pin_memory() for F in Fs]
    outs = [torch.full((n, n, n), 7.0, dtype=torch.float64).pin_memory() for _ in Fs]
    sts = s.solve_host_sequence(src, outs, tol=tol)
    assert [st.cycles for st in sts] == [st.cycles for st in ref_st]
    assert sts[1].cycles < sts[0].cycles          # warm start from the previous solution
    for t in range(T):
        np.testing.assert_array_equal(outs[t].numpy(), ref[t])
        np.testing.assert_array_equal(src[t].numpy(), Fs[t])
    # pageable buffers and an initial guess for the first solve
    phi0 = grf(n, 42)
    ref, ref_st = _device_chain(s, Fs[:3], phi0, tol)
    outs = [np.empty((n, n, n)) for _ in range(3)]
    sts = s.solve_host_sequence(Fs[:3], outs, phi0=phi0, tol=tol)
    assert [st.cycles for st in sts] == [st.cycles for st in ref_st]
    for t in range(3):
        np.testing.assert_array_equal(outs[t], ref[t])
    # one solve, then an empty sequence
    ref, _ = _device_chain(s, Fs[:1], None, tol)
    one = [np.empty((n, n, n))]
    s.solve_host_sequence(Fs[:1], one, tol=tol)
    np.testing.assert_array_equal(one[0], ref[0])
    assert s.solve_host_sequence([], []) == []
    with pytest.raises(ValueError):
        s.solve_host_sequence(Fs[:2], one)


def test_host_sequence_reports_nonconvergence(gb):
    n = 16
    s = gb.Solver(n, prec="mixed")
    Fs = [grf(n, 60), grf(n, 61)]
    outs = [np.empty((n, n, n)) for _ in Fs]
    sts = s.solve_host_sequence(Fs, outs, tol=1e-30, max_vcycles=2)
    assert [st.status for st in sts] == [4, 4] and [st.cycles for st in sts] == [2, 2]
    assert np.isfinite(outs[1]).all()


def test_results_do_not_depend_on_buffer_alignment(gb):
    # 16-byte-aligned F and phi take the pair conversion kernels, 8-byte-offset views the
    # one-element kernels; both visit the elements in the same order for the mean of F,
    # so copies, residuals and iterates are identical.
    n = 32
    F, phi0 = grf(n, 70), grf(n, 71)
    s = gb.Solver(n, prec="mixed")
    phi_a, st_a = s.solve(to_dev(F), to_dev(phi0), tol=1e-10)
    bf = torch.empty(n ** 3 + 1, dtype=torch.float64, device=DEV)
    bp = torch.empty(n ** 3 + 1, dtype=torch.float64, device=DEV)
    Fb, pb = bf[1:].view(n, n, n), bp[1:].view(n, n, n)
    Fb.copy_(to_dev(F))
    pb.copy_(to_dev(phi0))
    phi_b, st_b = s.solve(Fb, pb, tol=1e-10)
    assert st_a.cycles == st_b.cycles and st_a.history == st_b.history
    np.testing.assert_array_equal(phi_a.cpu().numpy(), phi_b.cpu().numpy())


def test_error_statuses(gb):
    n = 16
    s = gb.Solver(n, prec="mixed")
    F = grf(n, 17)
    bad = F.copy()
    bad[3, 4, 5] = np.nan
    phi, st = s.solve(to_dev(bad), tol=1e-6)
    assert st.status == 5
    phi0 = to_dev(grf(n, 18))
    phi, st = s.solve(to_dev(F), phi0.clone(), tol=1e-6, max_vcycles=0)
    assert st.status == 4 and st.cycles == 0
    # phi written with the gauge applied even when no cycle ran
    np.testing.assert_allclose(phi.cpu().numpy(), phi0.cpu().numpy() - phi0.cpu().numpy().mean(), atol=1e-12)
    with pytest.raises(gb.GbmgError):
        s.solve(to_dev(F), tol=1e-30, max_vcycles=2, raise_on_nonconvergence=True)
    with pytest.raises(ValueError):
        s.solve(to_dev(F).float())
    with pytest.raises(gb.GbmgError):
        gb.Solver((4, 4, 2))


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (32, 48, 64), (96, 96, 96)])
@pytest.mark.parametrize("degree", [1, 2, 3, 4])
@pytest.mark.parametrize("fused", [1, 2])
def test_fused_vcycle_bit_identical_to_unfused(gb, shape, degree, fused):
    # the temporally blocked kernels and the single-CTA bottom cycle round exactly like
    # the one-kernel-per-operation chain (fused 1: blocked from 2^18 cells, the bottom
    # cycle from the first level of at most 16^3; fused 2: blocked on every level of at
    # least 16^3)
    r = to_dev(grf(shape, 19), torch.float32)
    a = gb.Solver(shape, prec="mixed", fused=fused, degree=degree).vcycle(r)
    b = gb.Solver(shape, prec="mixed", fused=False, degree=degree).vcycle(r)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(112, 80, 144), (64, 112, 160), (56, 40, 112)])
@pytest.mark.parametrize("degree", [2, 3])
def test_fused_vcycle_bit_identical_on_ragged_tiles(gb, shape, degree):
    # x and y sides that are not multiples of the 64 x 32 leg tiles (the last tile of each
    # row and column hangs over the mesh) and odd coarse sides, blocked on every level of
    # at least 16^3
    g = torch.Generator(device="cuda").manual_seed(29)
    r = torch.randn(shape, generator=g, device="cuda", dtype=torch.float32)
    a = gb.Solver(shape, prec="mixed", fused=2, degree=degree).vcycle(r)
    b = gb.Solver(shape, prec="mixed", fused=False, degree=degree).vcycle(r)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_fused_vcycle_bit_identical_with_more_tiles_than_ctas(gb):
    # nx, ny, nz = 640, 512, 256: 160 tiles of 64 x 32 cells on the finest level, more than
    # the 152 CTAs of the persistent legs, so some CTAs run whole tiles (whose z streams
    # start at plane 0) and the others start at each tile's phase; the coarser levels have
    # fewer tiles than CTAs, with runs that cross tile ends
    shape = (256, 512, 640)
    g = torch.Generator(device="cuda").manual_seed(23)
    r = torch.randn(shape, generator=g, device="cuda", dtype=torch.float32)
    a = gb.Solver(shape, prec="mixed", fused=1, degree=3).vcycle(r)
    b = gb.Solver(shape, prec="mixed", fused=False, degree=3).vcycle(r)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 48, 64)])
def test_fused_solve_iterates_match_unfused(gb, shape):
    F = to_dev(grf(shape, 20))
    pa, sa = gb.Solver(shape, prec="mixed", fused=2).solve(F, tol=0.0, max_vcycles=4)
    pb, sb = gb.Solver(shape, prec="mixed", fused=False).solve(F, tol=0.0, max_vcycles=4)
    assert sa.cycles == sb.cycles == 4
    diff = (pa - pb).abs().max().item()
    assert diff <= 1e-14 * pb.abs().max().item()
    np.testing.assert_allclose(sa.history, sb.history, rtol=1e-5)


@pytest.mark.parametrize("order,growth", [(0, 1.0), (0, 1.3), (1, 1.0), (2, 1.0)])
def test_predict_matches_oracle_bit_for_bit(gb, order, growth):
    shape = (24, 16, 32)
    hist = [np.random.default_rng(70 + k).standard_normal(shape) for k in range(3)]
    s = gb.Solver(shape)
    got = s.predict([to_dev(h) for h in hist], order=order, growth=growth).cpu().numpy()
    assert np.array_equal(got, flat.predict(hist, order, growth))
    # in place on the most recent solution
    h0 = to_dev(hist[0])
    s.predict([h0, to_dev(hist[1]), to_dev(hist[2])], order=order, growth=growth, out=h0)
    assert np.array_equal(h0.cpu().numpy(), flat.predict(hist, order, growth))
    with pytest.raises(gb.GbmgError):
        s.predict([to_dev(hist[0])], order=2)


def test_predictors_save_cycles_in_a_warm_sequence(gb):
    """Eq. kwarm with the predictors on the GPU: sources drifting linearly in the step
    index; extrapolated starts need fewer cycles than recycling and reach the same
    solution (FFT oracle)."""
    n = 32
    d0, eta = grf(n, 2), grf(n, 3)
    F = [d0 + 0.05 * t * eta for t in range(5)]
    s = gb.Solver(n)
    sols = []
    for t in range(4):
        phi = sols[-1].clone() if sols else torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        s.solve(to_dev(F[t]), phi, tol=1e-10, max_vcycles=40)
        sols.append(phi)
    _, rec = s.solve(to_dev(F[4]), sols[3].clone(), tol=1e-8, max_vcycles=40)
    lin_phi = s.predict([sols[3], sols[2]], order=1)
    _, lin = s.solve(to_dev(F[4]), lin_phi, tol=1e-8, max_vcycles=40)
    quad_phi = s.predict([sols[3], sols[2], sols[1]], order=2)
    _, quad = s.solve(to_dev(F[4]), quad_phi, tol=1e-8, max_vcycles=40)
    assert lin.rel_res0 < 1e-3 * rec.rel_res0 and quad.rel_res0 < 1e-3 * rec.rel_res0
    assert lin.cycles < rec.cycles and quad.cycles < rec.cycles
    ref = flat.fft_solve(F[4])
    for p in (lin_phi, quad_phi):
        assert np.linalg.norm(p.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.parametrize("fused", [0, 2])
def test_krylov_solve_matches_oracle(gb, fused):
    """Defect correction with V-cycle-preconditioned CG steps (Sec. 3.2): same solution as
    the FFT oracle, residual history close to the oracle's mg_pcg_solve, and fewer
    outer steps than plain V-cycles."""
    shape = (32, 32, 32)
    F = grf(shape, 51)
    s = gb.Solver(shape, krylov=2, fused=fused)
    phi, st = s.solve(to_dev(F), tol=1e-10, max_vcycles=40)
    assert st.status == 0 and st.rel_res <= 1e-10
    ref = flat.fft_solve(F)
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-9
    _, hist = flat.mg_pcg_solve(F, inner_steps=2, tol=1e-10)
    m = min(len(st.history), len(hist) - 1, 4)
    np.testing.assert_allclose(st.history[:m], hist[1:m + 1], rtol=2e-2)
    _, plain = gb.Solver(shape, fused=fused).solve(to_dev(F), tol=1e-10, max_vcycles=40)
    assert 2 * st.cycles <= plain.cycles + 1


def test_krylov_option_validation(gb):
    with pytest.raises(gb.GbmgError):
        gb.Solver(32, krylov=17)
    with pytest.raises(gb.GbmgError):
        gb.Solver(32, krylov=2, prec="fp64")
    with pytest.raises(gb.GbmgError):
        gb.Solver(16, op="curv", krylov=1)


def test_solves_on_side_streams_match_default_stream(gb):
    # every call runs on torch's current stream: two contexts solving on two side streams
    # give the same bits as on the default stream
    shape = (32, 48, 64)
    F1, F2 = to_dev(grf(shape, 31)), to_dev(grf(shape, 32))
    a = gb.Solver(shape, prec="mixed")
    b = gb.Solver(shape, prec="mixed")
    ref1, st1 = a.solve(F1, tol=1e-8)
    ref2, st2 = b.solve(F2, tol=1e-8)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s1):
        p1, t1 = a.solve(F1, tol=1e-8)
    with torch.cuda.stream(s2):
        p2, t2 = b.solve(F2, tol=1e-8)
        q2, _ = b.solve(F1, p2.clone(), tol=1e-8)
    torch.cuda.synchronize()
    assert (t1.cycles, t2.cycles) == (st1.cycles, st2.cycles)
    assert torch.equal(p1, ref1) and torch.equal(p2, ref2)
    ref = flat.fft_solve(grf(shape, 31))
    assert np.linalg.norm(q2.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-7


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 48, 64), (56, 40, 112)])
def test_cycle_graphs_match_eager_cycles(gb, shape):
    # mixed fused solves run their cycles as CUDA graphs unless switched off: same
    # iterates, cycles and residual histories on a warm sequence of three sources, the
    # graph replays counted as kernel launches, and the timed families (event nodes inside
    # the graphs) timed at the same launches
    F = [to_dev(grf(shape, 60 + k)) for k in range(3)]
    g = gb.Solver(shape, prec="mixed")
    eager = gb.Solver(shape, prec="mixed")
    eager.set_cycle_graphs(False)
    fams = ["down0", "up0", "df0"]
    g.profile_begin(fams)
    eager.profile_begin(fams)
    pg = torch.zeros_like(F[0])
    pe = torch.zeros_like(F[0])
    for f in F:
        n0 = gb.launch_count()
        _, sg = g.solve(f, pg, tol=1e-9)
        ng = gb.launch_count() - n0
        n0 = gb.launch_count()
        _, se = eager.solve(f, pe, tol=1e-9)
        ne = gb.launch_count() - n0
        assert sg.cycles == se.cycles and sg.history == se.history
        assert torch.equal(pg, pe)
        assert ng == ne
    for fam in fams:  # (meshes below 2^18 cells have no fused legs on level 0)
        (cg, tg), (ce, te) = g.profile_read(fam), eager.profile_read(fam)
        assert cg == ce and (cg == 0 or (tg > 0.0 and te > 0.0))
    assert g.profile_read("df0")[0] > 0
    g.profile_end()
    eager.profile_end()
    ref = flat.fft_solve(grf(shape, 62))
    assert np.linalg.norm(pg.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-8


def test_krylov_cycle_graphs_match_eager_cycles(gb):
    # the MG-preconditioned CG corrections keep their scalars on the device, so their
    # cycles are graph launches too: the same bits as launched one by one
    shape = (64, 64, 64)
    F = to_dev(grf(shape, 63))
    g = gb.Solver(shape, prec="mixed", krylov=2)
    e = gb.Solver(shape, prec="mixed", krylov=2)
    e.set_cycle_graphs(False)
    for _ in range(2):
        pg, sg = g.solve(F, tol=1e-9)
        pe, se = e.solve(F, tol=1e-9)
        assert sg.cycles == se.cycles and sg.history == se.history
        assert torch.equal(pg, pe)
