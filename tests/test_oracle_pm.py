"""Pins of the particle-mesh oracle (CPU): conservation, lattice uniformity, the
paint/read transpose identity, exact interpolation of linear fields and the force of
a single particle pair."""
import numpy as np
import pytest

from oracle import flat, grad, pm


def particles(n, shape, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * np.array(shape[::-1], dtype=np.float64)


def test_paint_conserves_mass_and_hits_nodes():
    shape = (6, 7, 8)
    pos = particles(500, shape, 1)
    m = np.random.default_rng(2).random(500)
    assert np.isclose(pm.cic_paint(pos, m, shape).sum(), m.sum(), rtol=1e-14)
    # a particle on a node deposits all its mass there, also across the periodic edge
    rho = pm.cic_paint(np.array([[3.0, 6.0, 5.0], [8.0, 0.0, 0.0]]), [2.0, 1.0], shape)
    assert rho[5, 6, 3] == 2.0 and rho[0, 0, 0] == 1.0 and rho.sum() == 3.0


def test_lattice_paints_uniform_density():
    shape = (4, 6, 8)
    g = np.stack(np.meshgrid(np.arange(8) + 0.5, np.arange(6) + 0.5, np.arange(4) + 0.5, indexing="ij"),
                 -1).reshape(-1, 3)
    np.testing.assert_allclose(pm.cic_paint(g, 1.0, shape), np.ones(shape), rtol=0, atol=1e-14)


def test_read_is_transpose_of_paint():
    shape = (5, 6, 7)
    pos = particles(300, shape, 3)
    m = np.random.default_rng(4).standard_normal(300)
    f = np.random.default_rng(5).standard_normal(shape)
    lhs = float((pm.cic_paint(pos, m, shape) * f).sum())
    rhs = float((m * pm.cic_read(f, pos)[:, 0]).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_read_interpolates_linear_fields_exactly():
    shape = (8, 8, 8)
    z, y, x = np.meshgrid(*[np.arange(8.0)] * 3, indexing="ij")
    lin = 0.5 + 2.0 * x - 1.5 * y + 0.25 * z
    pos = 1.0 + np.random.default_rng(6).random((200, 3)) * 6.0   # away from the periodic seam
    want = 0.5 + 2.0 * pos[:, 0] - 1.5 * pos[:, 1] + 0.25 * pos[:, 2]
    np.testing.assert_allclose(pm.cic_read(lin, pos)[:, 0], want, rtol=0, atol=1e-12)


def test_force_pipeline_is_antisymmetric_for_a_pair():
    """Two equal particles placed symmetrically about the box centre feel opposite forces
    along their separation (momentum conservation of the mesh force for this symmetric
    configuration), and the force points from one particle to the other."""
    shape = (16, 16, 16)
    pos = np.array([[5.0, 8.0, 8.0], [11.0, 8.0, 8.0]])
    _, F = pm.pm_force(pos, 1.0, shape)
    np.testing.assert_allclose(F[0], -F[1], rtol=0, atol=1e-12)
    # nabla^2 phi = rho - mean gives phi minima at the masses, so -grad phi is attractive:
    # particle 0 (x = 5) is pulled towards its nearer neighbour at x = 11 (the periodic image
    # at x = -5 is farther)
    assert abs(F[0, 1]) < 1e-12 and abs(F[0, 2]) < 1e-12 and F[0, 0] > 0.0
    phi = flat.fft_solve(pm.cic_paint(pos, 1.0, shape))
    np.testing.assert_allclose(-pm.cic_read(grad.grad4(phi), pos), F, rtol=0, atol=0)
