"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds input generation only: seeded white noise, Gaussian random
fields with a power-law spectrum, a Gaussian-smoothed deformation potential and
the sequence of sources used for warm-started solves.  It contains none of the
solver's arithmetic (no stencil, no smoother, no transfer operator), so that the
oracle and the CUDA path receive bit-identical inputs without sharing any of
the method.

Conventions: arrays are float64 with shape (nz, ny, nx), x the fastest index;
mesh spacing is one cell.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

__all__ = ["white_noise", "grf", "smoothed_grf", "warm_sequence", "vector_noise", "lattice_particles", "workers"]


def workers() -> int:
    import os
    return max(1, os.cpu_count() or 1)


def _shape3(n) -> tuple[int, int, int]:
    if isinstance(n, int):
        return (n, n, n)
    n = tuple(int(v) for v in n)
    assert len(n) == 3
    return n


def white_noise(shape, seed: int) -> np.ndarray:
    """Standard-normal float64 field from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(_shape3(shape))


def _kmag(shape) -> np.ndarray:
    """|k| on the rfftn grid of `shape`, k_i = 2 pi n_i / N_i (continuum wavenumber)."""
    nz, ny, nx = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.rfftfreq(nx)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    return np.sqrt(k2)


def grf(shape, seed: int, spectral_index: float = -2.0) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field with P(k) proportional to k^n.

    White noise is multiplied by |k|^(n/2) in Fourier space (k = 0 removed),
    transformed back, then the sample mean is subtracted and the field divided
    by its sample standard deviation.
    """
    shape = _shape3(shape)
    w = white_noise(shape, seed)
    wk = sfft.rfftn(w, workers=workers())
    k = _kmag(shape)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (spectral_index / 2.0)
    wk *= amp
    f = sfft.irfftn(wk, s=shape, workers=workers())
    f -= f.mean()
    f /= f.std()
    return f


def smoothed_grf(shape, seed: int, sigma_cells: float, max_hessian_rowsum: float,
                 spectral_index: float = -2.0) -> np.ndarray:
    """Deformation potential psi: a GRF smoothed by exp(-k^2 sigma^2 / 2), then scaled.

    The scale is set so that max over cells of max_a sum_b |H_ab| equals
    `max_hessian_rowsum`, where H is the continuum (spectral, -k_a k_b) Hessian
    of the smoothed field.  This is an input recipe, not the method's Hessian.
    """
    shape = _shape3(shape)
    base = grf(shape, seed, spectral_index)
    bk = sfft.rfftn(base, workers=workers())
    nz_, ny_, nx_ = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz_)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(ny_)[None, :, None]
    kx = 2 * np.pi * np.fft.rfftfreq(nx_)[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    bk *= np.exp(-0.5 * k2 * sigma_cells ** 2)
    ks = (kx, ky, kz)
    rowsum = None
    for a in range(3):
        acc = None
        for b in range(3):
            hab = sfft.irfftn(-ks[a] * ks[b] * bk, s=shape, workers=workers())
            acc = np.abs(hab) if acc is None else acc + np.abs(hab)
        rowsum = acc if rowsum is None else np.maximum(rowsum, acc)
    smooth = sfft.irfftn(bk, s=shape, workers=workers())
    scale = max_hessian_rowsum / float(rowsum.max())
    psi = smooth * scale
    psi -= psi.mean()
    return psi


def vector_noise(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Three-component standard-normal field, shape (3, nz, ny, nx)."""
    shape = _shape3(shape)
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((3,) + shape).astype(dtype)


def warm_sequence(shape, seed0: int, seed_eta: int, steps: int, rate: float = 0.05):
    """Sources delta_t = delta_0 + rate * t * eta for t = 0..steps-1 (generator of arrays)."""
    d0 = grf(shape, seed0)
    eta = grf(shape, seed_eta)
    for t in range(steps):
        yield d0 + (rate * t) * eta


def lattice_particles(n_side: int, n_mesh: int, seed: int, rms_displacement: float = 1.0) -> np.ndarray:
    """Particles (n_side^3, 3) float32, columns x, y, z in mesh cell units on an n_mesh^3
    mesh: a cubic lattice (spacing n_mesh / n_side, offset half a spacing) displaced along
    the gradient of a seeded potential (a P(k) ~ k^-2 field divided by k^2, i.e. a
    Zel'dovich-like displacement), scaled to the requested rms displacement in cells and
    wrapped into [0, n_mesh).  Input generation only."""
    shape = (n_side,) * 3
    d = white_noise(shape, seed)
    dk = sfft.rfftn(d, workers=workers())
    nz_, ny_, nx_ = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz_)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(ny_)[None, :, None]
    kx = 2 * np.pi * np.fft.rfftfreq(nx_)[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[0, 0, 0] = 1.0
    pk = dk * k2 ** (-0.5) / k2          # delta_k ~ k^-1 white noise, potential delta_k / k^2
    pk[0, 0, 0] = 0.0
    disp = np.stack([sfft.irfftn(1j * kk * pk, s=shape, workers=workers()) for kk in (kx, ky, kz)], -1)
    disp *= rms_displacement / np.sqrt((disp ** 2).sum(-1).mean())
    spacing = n_mesh / n_side
    g = (np.arange(n_side) + 0.5) * spacing
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)[..., ::-1]   # (z, y, x) grid -> columns x, y, z
    pos = (q.reshape(-1, 3) + disp.reshape(-1, 3) * spacing) % n_mesh
    return pos.astype(np.float32)
