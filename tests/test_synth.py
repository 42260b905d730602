"""CPU checks that the seeded input generators (synth/) produce the documented recipe:
Gaussian random fields with zero mean, unit variance and a k^-2 power spectrum, the
smoothed deformation potential scaled to its Hessian row-sum bound, warm-start
sequences exactly linear in t, and lattice particles with the requested rms
displacement; every generator is deterministic in its seed."""
import numpy as np
import pytest

from synth import grf, lattice_particles, smoothed_grf, vector_noise, warm_sequence, white_noise


def test_seeds_are_deterministic_and_distinct():
    np.testing.assert_array_equal(white_noise(8, 3), white_noise(8, 3))
    assert not np.array_equal(white_noise(8, 3), white_noise(8, 4))
    np.testing.assert_array_equal(grf((8, 12, 16), 5), grf((8, 12, 16), 5))
    np.testing.assert_array_equal(vector_noise(8, 2), vector_noise(8, 2))
    assert vector_noise(8, 2).shape == (3, 8, 8, 8) and vector_noise(8, 2).dtype == np.float32


@pytest.mark.parametrize("index", [-2.0, -1.0])
def test_grf_moments_and_power_law(index):
    n = 64
    f = grf(n, 11, spectral_index=index)
    assert f.shape == (n, n, n) and f.dtype == np.float64
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12
    # shell-averaged |f_k|^2 against |k| on the continuum wavenumber: slope = index
    fk = np.abs(np.fft.rfftn(f)) ** 2
    k1 = 2 * np.pi * np.fft.fftfreq(n)
    kx = 2 * np.pi * np.fft.rfftfreq(n)
    k = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kx[None, None, :] ** 2)
    edges = np.geomspace(4 * 2 * np.pi / n, 0.5 * np.pi, 9)
    kc, pc = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (k >= lo) & (k < hi)
        kc.append(k[sel].mean())
        pc.append(fk[sel].mean())
    slope = np.polyfit(np.log(kc), np.log(pc), 1)[0]
    assert abs(slope - index) < 0.1


def test_smoothed_potential_meets_its_hessian_bound():
    # the recipe scales the spectral Hessian's largest row sum to the bound; the
    # second-order central-difference Hessian of a field smoothed over 4 cells agrees
    # with it to a few percent
    n, bound = 48, 0.5
    psi = smoothed_grf(n, 6, 4.0, bound)
    assert abs(psi.mean()) < 1e-14
    H = np.empty((3, 3, n, n, n))
    for a in range(3):
        ax = 2 - a
        H[a, a] = np.roll(psi, -1, ax) - 2 * psi + np.roll(psi, 1, ax)
        for b in range(a + 1, 3):
            bx = 2 - b
            v = (np.roll(np.roll(psi, -1, ax), -1, bx) - np.roll(np.roll(psi, -1, ax), 1, bx)
                 - np.roll(np.roll(psi, 1, ax), -1, bx) + np.roll(np.roll(psi, 1, ax), 1, bx)) / 4
            H[a, b] = H[b, a] = v
    rowsum = np.abs(H).sum(axis=1).max(axis=0)
    assert abs(rowsum.max() / bound - 1.0) < 0.05


def test_warm_sequence_is_linear_in_t():
    seq = list(warm_sequence(16, 1, 2, 4, rate=0.05))
    assert len(seq) == 4
    d0, eta = grf(16, 1), grf(16, 2)
    for t, s in enumerate(seq):
        np.testing.assert_allclose(s, d0 + 0.05 * t * eta, rtol=0, atol=1e-14)


def test_lattice_particles_displacement():
    n_side, n_mesh, rms = 16, 32, 0.7
    pos = lattice_particles(n_side, n_mesh, 9, rms_displacement=rms)
    assert pos.shape == (n_side ** 3, 3) and pos.dtype == np.float32
    assert pos.min() >= 0.0 and pos.max() < n_mesh
    spacing = n_mesh / n_side
    g = (np.arange(n_side) + 0.5) * spacing
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)[..., ::-1].reshape(-1, 3)
    d = (pos - q + n_mesh / 2) % n_mesh - n_mesh / 2
    assert abs(np.sqrt((d.astype(np.float64) ** 2).sum(-1).mean()) / (rms * spacing) - 1.0) < 1e-5
