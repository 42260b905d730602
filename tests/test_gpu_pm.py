"""Cloud-in-cell paint/read and the static PM force evaluation against the oracle (GPU)."""
import numpy as np
import pytest
import torch

from oracle import pm
from synth import lattice_particles

pytestmark = pytest.mark.gpu


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


@pytest.mark.parametrize("shape", [(16, 16, 16), (16, 24, 32)])
def test_paint_matches_oracle(gb, shape):
    rng = np.random.default_rng(1)
    pos = (rng.random((5000, 3)) * np.array(shape[::-1]) * 1.5 - 3.0).astype(np.float32)   # wraps both ways
    mass = rng.random(5000).astype(np.float32)
    s = gb.Solver(shape)
    got = s.cic_paint(to_dev(pos), to_dev(mass)).cpu().numpy()
    ref = pm.cic_paint(pos.astype(np.float64), mass.astype(np.float64), shape)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    got1 = s.cic_paint(to_dev(pos), 0.5).cpu().numpy()
    np.testing.assert_allclose(got1, pm.cic_paint(pos.astype(np.float64), 0.5, shape), rtol=1e-13, atol=1e-13)
    empty = s.cic_paint(torch.zeros((0, 3), dtype=torch.float32, device="cuda"))
    assert float(empty.abs().max()) == 0.0


@pytest.mark.parametrize("ncomp", [1, 3])
def test_read_matches_oracle_bit_for_bit(gb, ncomp):
    shape = (16, 24, 32)
    rng = np.random.default_rng(2)
    pos = (rng.random((3000, 3)) * np.array(shape[::-1])).astype(np.float32)
    field = rng.standard_normal((ncomp,) + shape)
    s = gb.Solver(shape)
    f = to_dev(field if ncomp > 1 else field[0])
    got = s.cic_read(f, to_dev(pos)).cpu().numpy()
    assert np.array_equal(got, pm.cic_read(field, pos.astype(np.float64)))


def test_force_evaluation_matches_oracle(gb):
    """paint -> solve -> fourth-order gradient -> read on displaced lattice particles."""
    n = 32
    pos = lattice_particles(32, n, 7, rms_displacement=1.5)
    s = gb.Solver(n)
    p = to_dev(pos)
    rho = s.cic_paint(p, 1.0)
    phi, st = s.solve(rho, tol=1e-11, max_vcycles=60)
    assert st.status == 0
    force = -s.cic_read(s.grad(phi, 4), p)
    _, ref = pm.pm_force(pos.astype(np.float64), 1.0, (n, n, n))
    got = force.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8


def test_single_precision_force_path(gb):
    """mg_force (FP32 gradient and read) against the FP64 oracle force: the FP32 rounding of
    phi, amplified by the cancellation of the differences, bounds the error."""
    n = 32
    pos = lattice_particles(32, n, 8, rms_displacement=1.5)
    s = gb.Solver(n)
    p = to_dev(pos)
    rho = s.cic_paint(p, 1.0)
    phi, _ = s.solve(rho, tol=1e-11, max_vcycles=60)
    got = s.force(phi, p).double().cpu().numpy()
    _, ref = pm.pm_force(pos.astype(np.float64), 1.0, (n, n, n))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-5
    assert s.force(phi, torch.zeros((0, 3), dtype=torch.float32, device="cuda")).shape == (0, 3)
