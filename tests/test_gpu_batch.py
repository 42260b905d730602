"""Batched persistent solves of uneven problems vs one-at-a-time solves (GPU)."""
import numpy as np
import pytest
import torch

from oracle import flat
from synth import grf

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 32), (24, 24, 24), (16, 32, 48), (32, 32, 32), (48, 48, 48), (16, 16, 16)]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batched_matches_individual_solves(gb):
    srcs = [grf(s, 1000 + i) for i, s in enumerate(SHAPES)]
    batch = gb.Batch(SHAPES)
    F = [to_dev(a) for a in srcs]
    phis = [torch.zeros_like(f) for f in F]
    stats, times = batch.solve(F, phis, tol=1e-8, max_vcycles=40)
    assert all(st.status == 0 for st in stats)
    for i, shape in enumerate(SHAPES):
        s = gb.Solver(shape, fused=False)
        ref, st = s.solve(F[i], tol=1e-8, max_vcycles=40)
        assert stats[i].cycles == st.cycles
        np.testing.assert_allclose(stats[i].history, st.history, rtol=1e-5)
        diff = float((phis[i] - ref).abs().max())
        assert diff <= 1e-12 * float(ref.abs().max())
        exact = flat.fft_solve(srcs[i])
        assert np.linalg.norm(phis[i].cpu().numpy() - exact) / np.linalg.norm(exact) < 1e-7
    # completion times: positive, and a problem needing more cycles does not finish earlier
    assert all(t > 0 for t in times)
    order = sorted(range(len(SHAPES)), key=lambda i: stats[i].cycles)
    assert times[order[-1]] >= times[order[0]]
    batch.close()


def test_batched_warm_start_and_statuses(gb):
    shapes = [(32, 32, 32), (24, 24, 24)]
    batch = gb.Batch(shapes)
    F = [to_dev(grf(s, 7 + i)) for i, s in enumerate(shapes)]
    phis = [torch.zeros_like(f) for f in F]
    stats, _ = batch.solve(F, phis, tol=1e-10, max_vcycles=40)
    assert all(st.status == 0 for st in stats)
    # warm start from the solution: already converged, no cycle
    stats, _ = batch.solve(F, phis, tol=1e-6, max_vcycles=40)
    assert all(st.cycles == 0 and st.status == 0 for st in stats)
    # an unreachable tolerance runs out of cycles
    cold = [torch.zeros_like(f) for f in F]
    stats, _ = batch.solve(F, cold, tol=0.0, max_vcycles=3)
    assert all(st.status == 4 and st.cycles == 3 for st in stats)
    blocks = batch.autotune(F, [torch.zeros_like(f) for f in F], tol=1e-6)
    assert blocks > 0
    batch.close()


def test_batch_rejects_unsupported_contexts(gb):
    with pytest.raises(gb.GbmgError):
        s = gb.Solver(32, fused=True)
        import ctypes
        arr = (ctypes.c_void_p * 1)(s._ctx)
        b = ctypes.c_void_p()
        gb._check(gb.lib().mg_batch_create(ctypes.byref(b), arr, 1, None))
