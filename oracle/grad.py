"""Periodic finite-difference gradients and their transposes (oracle, test infrastructure).

* 4th-order centred first derivative from a width-2 halo (Sec. 3.4 implementation
  list, "one-exchange finite-difference gradient"):
  (D4 u)_i = (-u_{i+2} + 8 u_{i+1} - 8 u_{i-1} + u_{i-2}) / (12 h).
* 2nd-order central difference (Sec. 4.1): (D2 u)_i = (u_{i+1} - u_{i-1}) / (2 h).

Both stencils are antisymmetric on the periodic mesh, so the transpose of the
gradient is minus the matching divergence.  Output layout: (3, nz, ny, nx) with
component 0 = x, 1 = y, 2 = z.

Parity pins: plane-wave symbols (i sin k (8 - 2cos k)/6 and i sin k) and the
dot-product identity <D u, w> = <u, D^T w>, in tests/test_oracle_grad.py.
"""
from __future__ import annotations

import numpy as np

# array axis of each Cartesian component: x is the last (fastest) axis
AXIS = (2, 1, 0)


def _at(u: np.ndarray, comp: int, s: int) -> np.ndarray:
    """u evaluated at i + s e_comp (periodic)."""
    return np.roll(u, -s, axis=AXIS[comp])


def grad4(u: np.ndarray, h: float = 1.0) -> np.ndarray:
    return np.stack([(-_at(u, a, 2) + 8 * _at(u, a, 1) - 8 * _at(u, a, -1) + _at(u, a, -2)) / (12 * h)
                     for a in range(3)])


def grad4_T(w: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Transpose of grad4 applied to a vector field w of shape (3, nz, ny, nx)."""
    out = np.zeros(w.shape[1:], dtype=np.float64)
    for a in range(3):
        wa = w[a].astype(np.float64)
        out += (-_at(wa, a, -2) + 8 * _at(wa, a, -1) - 8 * _at(wa, a, 1) + _at(wa, a, 2)) / (12 * h)
    return out


def grad2(u: np.ndarray, h: float = 1.0) -> np.ndarray:
    return np.stack([(_at(u, a, 1) - _at(u, a, -1)) / (2 * h) for a in range(3)])


def grad2_T(w: np.ndarray, h: float = 1.0) -> np.ndarray:
    out = np.zeros(w.shape[1:], dtype=np.float64)
    for a in range(3):
        wa = w[a].astype(np.float64)
        out += (_at(wa, a, -1) - _at(wa, a, 1)) / (2 * h)
    return out
