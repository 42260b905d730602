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
    guess = [torch.zeros_like(f) for f in F]
    blocks, tiles = batch.autotune(F, guess, tol=1e-6)
    assert blocks > 0 and len(tiles) == 4 and all(t >= 1024 for t in tiles)
    assert batch.tiles() == tiles
    # the autotuner leaves the solution from the given guesses (a cold solve, not a warm one)
    ref, st = gb.Solver(shapes[0], fused=False).solve(F[0], tol=1e-6, max_vcycles=40)
    assert float((guess[0] - ref).abs().max()) <= 1e-12 * float(ref.abs().max())
    batch.close()


def test_batched_tile_sizes_do_not_change_results(gb):
    shapes = [(32, 32, 32), (48, 48, 48), (16, 32, 48)]
    F = [to_dev(grf(s, 20 + i)) for i, s in enumerate(shapes)]
    batch = gb.Batch(shapes)
    base = [torch.zeros_like(f) for f in F]
    st0, _ = batch.solve(F, base, tol=1e-8, max_vcycles=40)
    for tiles in ([1024] * 5, [65536, 1024, 2048, 8192, 1024], [2048, 16384, 1024, 1024, 4096]):
        batch.set_tiles(tiles)
        phis = [torch.zeros_like(f) for f in F]
        st, _ = batch.solve(F, phis, tol=1e-8, max_vcycles=40)
        for a, b_, s0, s1 in zip(phis, base, st0, st):
            assert s0.cycles == s1.cycles
            assert float((a - b_).abs().max()) <= 1e-13 * float(b_.abs().max())
    with pytest.raises(gb.GbmgError):
        batch.set_tiles([1000])
    batch.close()


def test_batch_rejects_unsupported_contexts(gb):
    with pytest.raises(gb.GbmgError):
        s = gb.Solver(32, fused=True)
        import ctypes
        arr = (ctypes.c_void_p * 1)(s._ctx)
        b = ctypes.c_void_p()
        gb._check(gb.lib().mg_batch_create(ctypes.byref(b), arr, 1, None))


def test_batched_graph_replay_matches_direct_launch(gb):
    shapes = [(32, 32, 32), (24, 24, 24), (16, 32, 48)]
    F = [to_dev(grf(s, 40 + i)) for i, s in enumerate(shapes)]
    batch = gb.Batch(shapes)
    direct = [torch.zeros_like(f) for f in F]
    st0, _ = batch.solve(F, direct, tol=1e-8, max_vcycles=40)
    batch.use_graph(True)
    for tol in (1e-8, 1e-8, 1e-6, 1e-8):       # capture, replay, re-capture, re-capture
        phis = [torch.zeros_like(f) for f in F]
        st, times = batch.solve(F, phis, tol=tol, max_vcycles=40)
        assert all(x.status == 0 and x.rel_res <= tol for x in st)
        if tol == 1e-8:
            for a, b_, s0, s1 in zip(phis, direct, st0, st):
                assert s0.cycles == s1.cycles
                assert torch.equal(a, b_)
    # new source values through the same pointers are picked up by the replay
    for f in F:
        f.mul_(2.0)
    phis = [torch.zeros_like(f) for f in F]
    batch.solve(F, phis, tol=1e-8, max_vcycles=40)
    for a, b_ in zip(phis, direct):
        assert float((a - 2.0 * b_).abs().max()) <= 1e-12 * float(b_.abs().max())
    batch.close()
