"""The allocation-free residual entry point (GPU).

mg_rel_residual_noalloc serves callers that must not allocate device memory; its
reduction scratch is a fixed array inside the library.  Its result is checked
against the oracle's FP64 relative residual and against the solver's own
evaluation (mg_solve with no cycles), on two calls in a row with nonzero
potentials, so that the second call reuses the scratch the first one left.
Collected last on purpose.
"""
import numpy as np
import pytest
import torch

from oracle import flat
from synth import grf

pytestmark = pytest.mark.gpu


def _call(L, F, phi, out):
    nz, ny, nx = F.shape
    stream = torch.cuda.current_stream().cuda_stream
    assert L.mg_rel_residual_noalloc(nx, ny, nz, F.data_ptr(), phi.data_ptr(), out.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    return out.item()


def _potentials(shape, F, seed):
    """Two nonzero potentials: a small random one (residual ratio near 1) and the exact
    solution perturbed by 1e-7 relative noise (ratio ~1e-3: F and A phi cancel)."""
    sol = flat.fft_solve(F)
    noise = np.random.default_rng(seed).standard_normal(shape)
    return [0.01 * grf(shape, seed + 10), sol * (1.0 + 1e-7 * noise)]


def test_noalloc_relative_residual_matches_oracle_and_solver_on_two_calls(gb):
    L = gb.lib()
    shape = (32, 48, 64)            # (nz, ny, nx)
    solver = gb.Solver(shape)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    Fh = grf(shape, 1) + 0.3
    F = torch.from_numpy(Fh).cuda()
    for phih in _potentials(shape, Fh, 2):
        phi = torch.from_numpy(phih).cuda()
        got = _call(L, F, phi, out)
        ref = flat.rel_residual(flat.project_mean(Fh), phih)
        assert abs(got - ref) <= 1e-6 * ref, (got, ref)
        # the existing entry point: a solve with no cycles only evaluates the residual
        _, st = solver.solve(F, phi.clone(), tol=0.0, max_vcycles=0)
        assert st.cycles == 0
        assert abs(got - st.rel_res0) <= 1e-6 * st.rel_res0, (got, st.rel_res0)
    # a mesh with more planes than the fixed scratch holds is rejected before any launch
    stream = torch.cuda.current_stream().cuda_stream
    assert L.mg_rel_residual_noalloc(4, 4, 4097, F.data_ptr(), phi.data_ptr(), out.data_ptr(), stream) == 1
    assert b"4096" in L.mg_last_error()


def test_noalloc_relative_residual_on_large_planes(gb):
    # 512 x 512 planes: about 1024 cells per thread in each plane's sums
    L = gb.lib()
    shape = (8, 512, 512)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    Fh = grf(shape, 3) - 0.2
    F = torch.from_numpy(Fh).cuda()
    for phih in _potentials(shape, Fh, 4):
        got = _call(L, F, torch.from_numpy(phih).cuda(), out)
        ref = flat.rel_residual(flat.project_mean(Fh), phih)
        assert abs(got - ref) <= 1e-6 * ref, (got, ref)
