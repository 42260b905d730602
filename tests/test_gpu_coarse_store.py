"""Coarse-level corrections stored in BF16 / FP16 (opts.coarse_store), against the oracle (GPU).

A precision option of the mixed solve: the correction a level of fewer than 128^3 cells
hands up to the next finer level is held in a 16-bit format.  Inside the double-float defect
correction (Sec. 3.2) the converged solution must still be the FP64 oracle's FFT solution;
the tests check that, the cycle cost, and that the rounding really takes place.
"""
import numpy as np
import pytest
import torch

from oracle import flat
from synth import grf

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("store", ["bf16", "fp16"])
def test_coarse_store_converges_to_the_oracle(gb, n, store):
    F = grf(n, 70)
    ref = flat.fft_solve(F)
    Fd = torch.from_numpy(F).cuda()
    phi32, st32 = gb.Solver(n).solve(Fd, tol=1e-10, max_vcycles=60)
    s = gb.Solver(n, coarse_store=store)
    phi, st = s.solve(Fd, tol=1e-10, max_vcycles=60)
    assert st.status == 0 and st.rel_res <= 1e-10
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-9
    if store == "bf16":
        # BF16 keeps FP32's exponent range: the coarse correction's 8-bit significand costs
        # at most a couple of cycles
        assert st.cycles <= st32.cycles + 2
    else:
        # FP16: the inner problem is scaled to a unit 2-norm residual, so per-cell coarse
        # corrections fall towards FP16's subnormal range and the cycle loses accuracy;
        # the defect correction still reaches the FP64 solution
        assert st.cycles >= st32.cycles
    # one V-cycle of the error equation: rounded, so not the FP32 cycle, but close to it
    r = torch.from_numpy(grf(n, 71)).cuda().float()
    e16 = s.vcycle(r).double().cpu().numpy()
    e32 = gb.Solver(n).vcycle(r).double().cpu().numpy()
    d = rel_l2(e16, e32)
    assert 0.0 < d < (2e-2 if store == "bf16" else 3e-3), d


def test_coarse_store_options_are_checked(gb):
    with pytest.raises(gb.GbmgError):
        gb.Solver(32, prec="fp64", coarse_store="bf16")
    with pytest.raises(gb.GbmgError):
        gb.Solver(32, op="curv", coarse_store="fp16")
    with pytest.raises(gb.GbmgError):
        gb.Batch([(32, 32, 32)], coarse_store="bf16")
