"""The curvilinear operator from raw coefficients (mg_set_coefficients), checked on the GPU.

With J and B given directly (coarse levels restrict them), the GPU operator is pinned to
the closed-form Fourier symbol of the Sec. 4.3.1 stencil for constant B,
    sigma(k) = -(sum_a B^aa 4 sin^2(k_a / 2) + 2 sum_{a<b} B^ab sin k_a sin k_b) / h^2,
(the same symbol for the symmetric variant), a constant-B solve is pinned to the spectral
solution with that symbol, and a variable-coefficient solve to a manufactured solution of
the oracle's FP64 stencil on the same coefficients.
"""
import numpy as np
import pytest
import torch

from oracle import curv
from synth import grf, smoothed_grf

pytestmark = pytest.mark.gpu

ORDER = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
BCONST = np.array([[1.2, 0.15, -0.1], [0.15, 0.9, 0.2], [-0.1, 0.2, 1.1]])


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def const_coeffs(shape, J=1.0):
    B32 = BCONST.astype(np.float32).astype(np.float64)
    B6 = np.stack([np.full(shape, B32[a, b]) for a, b in ORDER])
    return np.full(shape, J), B6, B32


def symbol(theta, B, h):
    """theta: per-index phases (x, y, z) of the mode; B the 3x3 constant coefficients."""
    s = sum(B[a, a] * 4.0 * np.sin(theta[a] / 2) ** 2 for a in range(3))
    s += 2.0 * sum(B[a, b] * np.sin(theta[a]) * np.sin(theta[b]) for a in range(3) for b in range(a + 1, 3))
    return -s / (h * h)


def phases(shape):
    nz, ny, nx = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    return np.meshgrid(kx, ky, kz, indexing="ij")


@pytest.mark.parametrize("sym", [False, True])
def test_constant_coefficient_operator_matches_fourier_symbol(gb, sym):
    shape = (16, 24, 32)
    J, B6, B = const_coeffs(shape)
    s = gb.Solver(shape, op="curv", curv_sym=sym)
    s.set_coefficients(to_dev(J, torch.float32), to_dev(B6, torch.float32))
    for level in range(2):
        shp = s.level_shape(level)
        h = 2.0 ** level
        Jl, B6l = s.curv_geometry(level)
        Bl = np.empty((3, 3))
        for k, (a, b) in enumerate(ORDER):
            vals = B6l[k].double().cpu().numpy()
            # the restriction of a constant is that constant up to FP32 rounding of the sums
            assert np.abs(vals - vals.mean()).max() <= 2e-7 * abs(vals.mean())
            Bl[a, b] = Bl[b, a] = vals.mean()
        nz, ny, nx = shp
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        for n in [(1, 0, 0), (0, 1, 2), (3, 2, 1), (5, 4, 3), (nx // 2, ny // 2, nz // 2)]:
            theta = [2 * np.pi * n[0] / nx, 2 * np.pi * n[1] / ny, 2 * np.pi * n[2] / nz]
            u = np.cos(theta[0] * x + theta[1] * y + theta[2] * z + 0.3)
            lam = symbol(theta, Bl, h)
            for tr in (False, True):
                got = s.curv_apply(level, to_dev(u), transpose=tr, divide_by_J=False).cpu().numpy()
                tol = (1e-12 if level == 0 else 1e-6) * max(1.0, abs(lam))
                assert np.abs(got - lam * u).max() <= tol, (level, n, tr)


@pytest.mark.parametrize("sym", [False, True])
def test_constant_coefficient_solve_matches_spectral_solution(gb, sym):
    shape = (32, 32, 32)
    J, B6, B = const_coeffs(shape)
    f = grf(shape, 80)
    f -= f.mean()
    s = gb.Solver(shape, op="curv", curv_sym=sym)
    s.set_coefficients(to_dev(J, torch.float32), to_dev(B6, torch.float32))
    phi, st = s.solve(to_dev(f), tol=1e-11, max_vcycles=300)
    assert st.status == 0
    # spectral solution of the same discrete operator: phi_hat = f_hat / sigma(k), k = 0 removed
    tx, ty, tz = phases(shape)
    lam = np.transpose(symbol([tx, ty, tz], B, 1.0), (2, 1, 0))
    lam[0, 0, 0] = 1.0
    ph = np.fft.fftn(f) / lam
    ph[0, 0, 0] = 0.0
    ref = np.real(np.fft.ifftn(ph))
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-9


def test_variable_coefficients_manufactured_solution(gb, monkeypatch):
    shape = (16, 24, 32)
    psi = smoothed_grf(shape, 81, 2.0, 0.5)
    g = gb.Solver(shape, op="curv")
    g.set_geometry(to_dev(psi))
    J32, B632 = g.curv_geometry(0)
    s = gb.Solver(shape, op="curv")
    s.set_coefficients(J32, B632)
    J, B6 = J32.double().cpu().numpy(), B632.double().cpu().numpy()
    B = np.empty((3, 3) + shape)
    for k, (a, b) in enumerate(ORDER):
        B[a, b] = B[b, a] = B6[k]
    phis = grf(shape, 82)
    phis -= phis.mean()

    # the solver's double-float residual forms each face mean of two FP32 cell coefficients
    # in FP32 (the rest in double-float): the manufactured source uses the same means
    def face32(Bm, a, b):
        c = Bm[a, b].astype(np.float32)
        return (np.float32(0.5) * (c + curv.at(c, a, 1))).astype(np.float64)

    monkeypatch.setattr(curv, "face_coeff", face32)
    f = curv.apply_M(phis, B, 1.0) / J           # J-weighted mean zero: 1^T M = 0
    monkeypatch.undo()
    phi, st = s.solve(to_dev(f), tol=1e-11, max_vcycles=300)
    assert st.status == 0
    assert rel_l2(phi.cpu().numpy(), phis) < 1e-8
    # the same finest operator as the psi path: the same solution
    phi_g, st_g = g.solve(to_dev(f), tol=1e-11, max_vcycles=300)
    assert st_g.status == 0
    assert rel_l2(phi.cpu().numpy(), phi_g.cpu().numpy()) < 1e-9
    # the adjoint gives source_bar, but psi_bar needs psi
    pbar = to_dev(np.random.default_rng(83).standard_normal(shape))
    dbar, _, st = s.solve_adjoint(pbar, tol=1e-10, max_vcycles=300)
    dbar_g, _, _ = g.solve_adjoint(pbar, tol=1e-10, max_vcycles=300)
    assert st.status == 0 and rel_l2(dbar.cpu().numpy(), dbar_g.cpu().numpy()) < 1e-8
    with pytest.raises(gb.GbmgError):
        s.solve_adjoint(pbar, phi=phi, source=to_dev(f), want_psi_bar=True, tol=1e-10, max_vcycles=300)
    with pytest.raises(gb.GbmgError):
        gb.Solver(shape).set_coefficients(J32, B632)      # flat context
