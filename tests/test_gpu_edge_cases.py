"""Degenerate inputs and the smallest meshes, against the oracle (GPU).

The method's degenerate cases (Sec. 2.1: the periodic operator's null space is the
constants, so a constant source projects to zero; a solve started from the exact
solution has nothing to do) and the mesh that is its own coarsest level (Sec. 2.3: the
coarsest level is solved directly).
"""
import numpy as np
import pytest
import torch

from oracle import flat
from synth import grf

pytestmark = pytest.mark.gpu


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("value", [0.0, 3.25])
def test_constant_source_gives_zero_potential(gb, prec, value):
    # F - mean(F) = 0: the zero-mean solution is zero; a cold start has nothing to do
    shape = (16, 24, 32)
    s = gb.Solver(shape, prec=prec)
    phi, st = s.solve(to_dev(np.full(shape, value)), tol=1e-10, max_vcycles=20)
    assert st.status == 0 and st.cycles == 0
    assert float(phi.abs().max()) == 0.0


def test_constant_source_from_a_nonzero_guess(gb):
    # the guess's own residual is all there is; the solve removes it and the gauge its mean
    shape = (32, 32, 32)
    guess = grf(shape, 90)
    s = gb.Solver(shape)
    # ||F - mean|| = 0, so the tolerance applies to ||A phi|| itself
    phi, st = s.solve(to_dev(np.full(shape, -1.5)), to_dev(guess), tol=1e-10, max_vcycles=40)
    assert st.status == 0 and st.rel_res <= 1e-10
    assert float(phi.abs().max()) <= 1e-8 * np.abs(guess).max()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_warm_start_from_the_solution_runs_no_cycle(gb, prec):
    shape = (32, 32, 32)
    F = grf(shape, 91)
    ref = flat.fft_solve(F)
    s = gb.Solver(shape, prec=prec)
    phi, st = s.solve(to_dev(F), to_dev(ref + 0.75), tol=1e-8, max_vcycles=20)
    assert st.status == 0 and st.cycles == 0 and st.rel_res0 <= 1e-8
    # the gauge removes the constant the guess carried
    assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(4, 4, 4), (8, 4, 4), (4, 6, 8)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_single_level_mesh_is_solved_directly(gb, shape, prec):
    # no level can be coarsened: the finest level is the coarsest and its pseudo-inverse is
    # the whole solver
    F = grf(shape, 92)
    s = gb.Solver(shape, prec=prec)
    assert s.levels == 1
    phi, st = s.solve(to_dev(F), tol=1e-12, max_vcycles=10)
    assert st.status == 0
    assert st.cycles <= (1 if prec == "fp64" else 4)
    ref = flat.fft_solve(F)
    assert np.linalg.norm(phi.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_curvilinear_constant_source_gives_zero_potential(gb):
    # L phi = f - <f>_J: a constant source is its own weighted mean
    shape = (16, 16, 16)
    psi = 0.2 * grf(shape, 93) / 10.0
    s = gb.Solver(shape, op="curv")
    s.set_geometry(to_dev(psi))
    phi, st = s.solve(to_dev(np.full(shape, 2.0)), tol=1e-10, max_vcycles=20)
    assert st.status == 0 and st.cycles == 0
    assert float(phi.abs().max()) == 0.0


def test_too_coarse_a_hierarchy_is_rejected(gb):
    # the coarsest level is inverted densely: more than 512 cells there is an argument error
    with pytest.raises(gb.GbmgError):
        gb.Solver((32, 32, 32), levels=2)
    with pytest.raises(gb.GbmgError):
        gb.Solver((8, 8, 256))
