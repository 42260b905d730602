"""The allocation-free residual entry point (GPU).

mg_rel_residual_noalloc serves callers that must not allocate device memory; its
reduction scratch is a fixed array inside the library.  It must give the same
relative residual as the solver's own evaluation (mg_solve with no cycles), also
on a second call in a row, which reuses the same scratch.  Collected last on
purpose.
"""
import numpy as np
import pytest
import torch

from synth import grf

pytestmark = pytest.mark.gpu


def test_noalloc_relative_residual_matches_solver_on_two_calls(gb):
    L = gb.lib()
    shape = (32, 48, 64)            # (nz, ny, nx)
    nz, ny, nx = shape
    solver = gb.Solver(shape)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for seed, scale in ((1, 0.0), (2, 0.01)):
        F = torch.from_numpy(grf(shape, seed) + 0.3).cuda()
        phi = torch.from_numpy(scale * grf(shape, seed + 10)).cuda()
        assert L.mg_rel_residual_noalloc(nx, ny, nz, F.data_ptr(), phi.data_ptr(), out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        got = out.item()
        # the existing entry point: a solve with no cycles only evaluates the residual
        _, st = solver.solve(F, phi.clone(), tol=0.0, max_vcycles=0)
        assert st.cycles == 0
        assert abs(got - st.rel_res0) <= 1e-5 * st.rel_res0, (got, st.rel_res0)
    # a mesh with more planes than the fixed scratch holds is rejected before any launch
    assert L.mg_rel_residual_noalloc(4, 4, 4097, F.data_ptr(), phi.data_ptr(), out.data_ptr(), stream) == 1
    assert b"4096" in L.mg_last_error()
