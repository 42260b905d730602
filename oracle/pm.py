"""Particle-mesh steps around the Poisson solve (oracle, test infrastructure).

Plain float64 NumPy, written from the paper:

* Sec. 2.1 ("The PM gravity solve"): particles are deposited by cloud-in-cell
  interpolation to form the density; the source of the Poisson equation is the
  density contrast (mean-density normalisation absorbed into F).
* Sec. 3.4 implementation list and the force-evaluation cost table: a static PM
  force evaluation is paint, solve, fourth-order gradient, read.

Conventions (readings, the paper fixes none of them): positions are in cell units,
mesh node (i, j, k) sits at position (i, j, k), the mesh is periodic; cloud-in-cell
gives node floor(x) the weight 1 - f and node floor(x) + 1 the weight f per axis,
f = x - floor(x); reading uses the same weights (paint and read are transposes).
Fields are (nz, ny, nx) arrays; positions are (n, 3) with columns x, y, z.
"""
from __future__ import annotations

import numpy as np

from . import flat, grad


def _stencil(pos: np.ndarray, shape):
    """Nodes and weights of the 8 CIC corners: list of (iz, iy, ix, w), corner order
    dz, dy, dx in {0, 1} with dx fastest."""
    nz, ny, nx = shape
    p = np.asarray(pos, dtype=np.float64)
    i0 = np.floor(p).astype(np.int64)
    f = p - i0
    out = []
    for dz in (0, 1):
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dx in (0, 1):
                wx = f[:, 0] if dx else 1.0 - f[:, 0]
                out.append(((i0[:, 2] + dz) % nz, (i0[:, 1] + dy) % ny, (i0[:, 0] + dx) % nx, (wx * wy) * wz))
    return out


def cic_paint(pos: np.ndarray, mass, shape) -> np.ndarray:
    """Mass deposited per node: sum over particles of m_p times the CIC weight."""
    rho = np.zeros(shape, dtype=np.float64)
    m = np.broadcast_to(np.asarray(mass, dtype=np.float64), (len(pos),))
    for iz, iy, ix, w in _stencil(pos, shape):
        np.add.at(rho, (iz, iy, ix), m * w)
    return rho


def cic_read(field: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """Field components interpolated at the particles: field (ncomp, nz, ny, nx) or (nz, ny, nx);
    returns (n, ncomp), corners summed in the stencil order."""
    f = np.asarray(field, dtype=np.float64)
    if f.ndim == 3:
        f = f[None]
    out = np.zeros((len(pos), f.shape[0]))
    for iz, iy, ix, w in _stencil(pos, f.shape[1:]):
        out += w[:, None] * f[:, iz, iy, ix].T
    return out


def pm_force(pos: np.ndarray, mass, shape) -> tuple[np.ndarray, np.ndarray]:
    """Static PM force evaluation: rho = paint, A phi = rho (mean projected, so the constant
    normalisation of the contrast drops out), force = -grad4 phi read at the particles.
    Returns (phi, force (n, 3))."""
    rho = cic_paint(pos, mass, shape)
    phi = flat.fft_solve(rho)
    return phi, -cic_read(grad.grad4(phi), pos)
