"""Flat-mesh oracle: periodic 7-point Poisson problem and its geometric multigrid.

TEST INFRASTRUCTURE.  Plain float64 NumPy/SciPy, written from the paper:

* Sec. 2.1, Eq. (linsys): A phi = F with the second-order seven-point Laplacian,
  periodic, symmetric negative semidefinite, null space = constants; F has its
  mean projected out and phi is fixed to zero mean.
* Sec. 2.2, Eq. (fftsolve): phi = F^-1[F_hat / lambda(k)],
  lambda(k) = -(4/h^2) sum_i sin^2(k_i h / 2) = (2cos kx + 2cos ky + 2cos kz - 6)/h^2.
* Sec. 2.3: Chebyshev-accelerated Jacobi smoother, Eq. (flat_chebyshev), on the
  interval [2/alpha, 2] of the spectrum of D^-1 A; weighted Jacobi,
  Eq. (flat_jacobi), omega = 2/3; residual, Eq. (flat_residual); full-weighting
  restriction; error equation on the coarse level, Eq. (coarse_error); trilinear
  prolongation and correction, Eq. (coarse_correction); the seven-point operator
  rediscretised on each level.
* Appendix B: restriction is the 1-D stencil [1/4, 1/2, 1/4] applied along each
  axis followed by decimation.
* Sec. 3.2: warm start as defect correction, phi = phi0 + e with A e = F - A phi0.

Readings taken where the paper is silent or ambiguous:
* Chebyshev degree v means v applications of the operator per smoothing pass
  (the standard Chebyshev semi-iteration on D^-1 A), not degree v+1 in the error.
* Restriction and prolongation are vertex-centred: coarse node I sits on fine
  node 2I.  Prolongation is the transpose of restriction times 8.
* Levels: coarsen while every side is even and half of it is at least 4.
* Coarsest level: exact solve on the zero-mean subspace (pseudo-inverse), done
  here with the FFT of the coarse operator.

Array layout: (nz, ny, nx), x fastest; spacing h = 2**level in fine-cell units.

Parity pins (tests/test_oracle_flat.py): plane-wave eigenvalues, dense
pseudo-inverse at 8^3, Chebyshev and Jacobi plane-wave factors, R = P^T / 8
from unit vectors, exact prolongation of linear functions, V-cycle convergence
to the FFT solution, mesh-independent convergence factor.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def _workers() -> int:
    import os
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- operator


def apply_A(u: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Seven-point periodic Laplacian: (A u)_i = (sum of the 6 face neighbours - 6 u_i) / h^2.

    Sec. 2.1, Eq. (linsys).
    """
    out = -6.0 * u
    for axis in range(3):
        out = out + np.roll(u, 1, axis=axis) + np.roll(u, -1, axis=axis)
    return out / (h * h)


def residual(F: np.ndarray, u: np.ndarray, h: float = 1.0) -> np.ndarray:
    """r = F - A u.  Sec. 2.3, Eq. (flat_residual)."""
    return F - apply_A(u, h)


def eigenvalues(shape, h: float = 1.0, rfft: bool = True) -> np.ndarray:
    """lambda(k) = -(4/h^2) sum_i sin^2(k_i/2), k_i = 2 pi n_i / N_i.  Sec. 2.2.

    Returned on the rfftn grid (last axis halved) when rfft is True.
    """
    nz, ny, nx = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * (np.fft.rfftfreq(nx) if rfft else np.fft.fftfreq(nx))
    s = (np.sin(kz / 2)[:, None, None] ** 2 + np.sin(ky / 2)[None, :, None] ** 2
         + np.sin(kx / 2)[None, None, :] ** 2)
    return -4.0 * s / (h * h)


def project_mean(F: np.ndarray) -> np.ndarray:
    """F - mean(F): the solvability projection of Sec. 2.1."""
    return F - F.mean()


def fft_solve(F: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Exact zero-mean solution of A phi = F - mean(F) by Eq. (fftsolve), k = 0 set to zero."""
    shape = F.shape
    Fk = sfft.rfftn(F, workers=_workers())
    lam = eigenvalues(shape, h)
    lam[0, 0, 0] = 1.0
    Fk = Fk / lam
    Fk[0, 0, 0] = 0.0
    return sfft.irfftn(Fk, s=shape, workers=_workers())


# ---------------------------------------------------------------- transfers


def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full weighting: [1/4, 1/2, 1/4] along each axis, then keep even nodes.  Appendix B."""
    t = r
    for axis in range(3):
        t = 0.5 * t + 0.25 * (np.roll(t, 1, axis=axis) + np.roll(t, -1, axis=axis))
    return t[::2, ::2, ::2].copy()


def prolong(ec: np.ndarray) -> np.ndarray:
    """Trilinear (vertex-centred) interpolation to the mesh twice as fine.  Sec. 2.3.

    Along each axis, fine node 2I copies coarse node I and fine node 2I+1 is the
    mean of coarse nodes I and I+1 (periodic).
    """
    t = ec
    for axis in range(3):
        n = t.shape[axis]
        shape = list(t.shape)
        shape[axis] = 2 * n
        out = np.empty(shape, dtype=t.dtype)
        even = [slice(None)] * 3
        odd = [slice(None)] * 3
        even[axis] = slice(0, 2 * n, 2)
        odd[axis] = slice(1, 2 * n, 2)
        out[tuple(even)] = t
        out[tuple(odd)] = 0.5 * (t + np.roll(t, -1, axis=axis))
        t = out
    return t


# ---------------------------------------------------------------- smoothers


def chebyshev_interval(alpha: float = 8.0) -> tuple[float, float]:
    """Target interval [2/alpha, 2] of the spectrum of D^-1 A.  Sec. 2.3."""
    return 2.0 / alpha, 2.0


def smooth_chebyshev(e: np.ndarray, r: np.ndarray, h: float, degree: int = 3,
                     alpha: float = 8.0) -> np.ndarray:
    """Degree-v Chebyshev-accelerated Jacobi smoothing of A e = r.  Sec. 2.3, Eq. (flat_chebyshev).

    Chebyshev semi-iteration on the Jacobi-preconditioned operator D^-1 A,
    D = diag(A) = -6/h^2, with the interval [a, b] = [2/alpha, 2]:
    theta = (a+b)/2, delta = (b-a)/2, sigma = theta/delta.  Uses `degree`
    operator applications; the error is multiplied by
    T_v((theta - mu)/delta) / T_v(theta/delta) on an eigenvector of D^-1 A with
    eigenvalue mu.
    """
    a, b = chebyshev_interval(alpha)
    theta = 0.5 * (a + b)
    delta = 0.5 * (b - a)
    sigma = theta / delta
    Dinv = -(h * h) / 6.0
    e = e.copy()
    z = Dinv * residual(r, e, h)
    d = z / theta
    rho = 1.0 / sigma
    for i in range(1, degree + 1):
        e = e + d
        if i < degree:
            z = Dinv * residual(r, e, h)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = (rho_new * rho) * d + (2.0 * rho_new / delta) * z
            rho = rho_new
    return e


def smooth_jacobi(e: np.ndarray, r: np.ndarray, h: float, sweeps: int = 2,
                  omega: float = 2.0 / 3.0) -> np.ndarray:
    """Weighted Jacobi sweeps e += omega D^-1 (r - A e), D = -6/h^2.  Sec. 2.3, Eq. (flat_jacobi)."""
    Dinv = -(h * h) / 6.0
    for _ in range(sweeps):
        e = e + omega * Dinv * residual(r, e, h)
    return e


# ---------------------------------------------------------------- hierarchy


def level_shapes(shape, levels: int = 0) -> list[tuple[int, int, int]]:
    """Mesh sides of each level: halve while all sides are even and half is >= 4.

    `levels` > 0 caps the count.  For n^3 with n a power of two this gives
    log2(n) - 1 levels (Sec. 4.3: L = log2 n_g - 1).
    """
    shapes = [tuple(int(v) for v in shape)]
    while True:
        if levels and len(shapes) >= levels:
            break
        s = shapes[-1]
        if all(v % 2 == 0 and v // 2 >= 4 for v in s):
            shapes.append(tuple(v // 2 for v in s))
        else:
            break
    return shapes


def coarse_solve(r: np.ndarray, h: float) -> np.ndarray:
    """Exact solve of the coarsest error equation on the zero-mean subspace (pseudo-inverse)."""
    return fft_solve(r, h)


def vcycle(level: int, e: np.ndarray, r: np.ndarray, nlevels: int, smoother: str = "cheb",
           degree: int = 3, alpha: float = 8.0, nu1: int = 2, nu2: int = 2,
           omega: float = 2.0 / 3.0) -> np.ndarray:
    """One V-cycle (mu = 1) for A_l e = r on level `level`.  Sec. 2.3.

    pre-smooth; r_c = R (r - A_l e); e_c = V-cycle on level+1 from zero (or the
    exact coarsest solve); e += P e_c; post-smooth.  A_l is the 7-point
    operator with spacing h_l = 2^l (rediscretised).
    """
    h = float(2 ** level)
    if level == nlevels - 1:
        return coarse_solve(r, h)

    if smoother == "cheb":
        e = smooth_chebyshev(e, r, h, degree, alpha)
    else:
        e = smooth_jacobi(e, r, h, nu1, omega)
    rc = restrict_fw(residual(r, e, h))
    ec = vcycle(level + 1, np.zeros_like(rc), rc, nlevels, smoother, degree, alpha, nu1, nu2, omega)
    e = e + prolong(ec)
    if smoother == "cheb":
        e = smooth_chebyshev(e, r, h, degree, alpha)
    else:
        e = smooth_jacobi(e, r, h, nu2, omega)
    return e


def rel_residual(F: np.ndarray, phi: np.ndarray) -> float:
    """||F - A phi||_2 / ||F||_2 with F already mean-projected (Sec. 3.1 convergence figure)."""
    return float(np.linalg.norm(residual(F, phi)) / np.linalg.norm(F))


def mg_solve(F: np.ndarray, phi0: np.ndarray | None = None, tol: float = 1e-10,
             max_cycles: int = 50, levels: int = 0, smoother: str = "cheb", degree: int = 3,
             alpha: float = 8.0, nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0,
             fixed_cycles: int | None = None):
    """Multigrid solve of A phi = F on the periodic mesh.

    F is mean-projected first (Sec. 2.1).  Starting from phi0 (cold start:
    zeros; warm start: the previous potential, Sec. 3.2), V-cycles are applied
    until ||F - A phi|| / ||F|| <= tol or max_cycles is reached
    (`fixed_cycles` forces an exact cycle count).  The result is returned with
    its mean removed (the gauge of Sec. 2.3).  Returns (phi, history) with the
    relative residual before the first and after every cycle.
    """
    F = project_mean(np.asarray(F, dtype=np.float64))
    nlev = len(level_shapes(F.shape, levels))
    phi = np.zeros_like(F) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    normF = float(np.linalg.norm(F))
    hist = [float(np.linalg.norm(residual(F, phi))) / normF]
    ncyc = fixed_cycles if fixed_cycles is not None else max_cycles
    for _ in range(ncyc):
        if fixed_cycles is None and hist[-1] <= tol:
            break
        phi = vcycle(0, phi, F, nlev, smoother, degree, alpha, nu1, nu2, omega)
        hist.append(float(np.linalg.norm(residual(F, phi))) / normF)
    phi = phi - phi.mean()
    return phi, hist


def defect_correction_solve(F: np.ndarray, phi0: np.ndarray, cycles: int, **kw):
    """Warm start as defect correction (Sec. 3.2): phi = phi0 + e, A e = F - A phi0.

    Each cycle applies one V-cycle to the error equation from e = 0 and adds the
    correction; identical in exact arithmetic to V-cycles on phi itself.
    """
    F = project_mean(np.asarray(F, dtype=np.float64))
    nlev = len(level_shapes(F.shape, kw.pop("levels", 0)))
    phi = np.array(phi0, dtype=np.float64, copy=True)
    for _ in range(cycles):
        r = residual(F, phi)
        phi = phi + vcycle(0, np.zeros_like(r), r, nlev, **kw)
    return phi - phi.mean()


def predict(history, order: int, growth: float = 1.0) -> np.ndarray:
    """Initial guess of the next solve from earlier solutions (Sec. 3.2, "Predictors").

    history[0] is the most recent solution phi_{n-1}, history[1] is phi_{n-2}, ...
      order 0: growth * phi_{n-1}  (recycling for growth = 1; the growth-scaled
               predictor, Eq. growth, with growth = D(a_n) / D(a_{n-1}))
      order 1: 2 phi_{n-1} - phi_{n-2}                 (linear extrapolation)
      order 2: 3 phi_{n-1} - 3 phi_{n-2} + phi_{n-3}   (quadratic extrapolation)
    Each product and sum is one IEEE operation, left to right as written.
    """
    h = [np.asarray(x, dtype=np.float64) for x in history]
    if order == 0:
        return growth * h[0]
    if order == 1:
        return 2.0 * h[0] - h[1]
    if order == 2:
        return 3.0 * h[0] - 3.0 * h[1] + h[2]
    raise ValueError("order must be 0, 1 or 2")


def pcg(r: np.ndarray, steps: int, precond, apply) -> tuple[np.ndarray, list[float]]:
    """`steps` iterations of preconditioned conjugate gradients for apply(e) = r from e = 0
    (Sec. 3.2: multigrid as the preconditioner of a conjugate-gradient iteration).
    Standard PCG: z = M r, p = z; alpha = (r, z) / (p, A p); e += alpha p; r -= alpha A p;
    beta = (r', z') / (r, z); p = z' + beta p.  A and M may both be negative definite (the
    periodic Laplacian and its V-cycle on zero-mean fields): the iterates are those of CG
    on -A with the preconditioner -M.  Returns (e, iterates) with the iterate after each step."""
    e = np.zeros_like(r)
    rr = np.array(r, dtype=np.float64, copy=True)
    z = precond(rr)
    p = z.copy()
    rz = float(np.vdot(rr, z))
    its = []
    for j in range(steps):
        q = apply(p)
        alpha = rz / float(np.vdot(p, q))
        e = e + alpha * p
        its.append(e)
        rr = rr - alpha * q
        if j == steps - 1:
            break
        z = precond(rr)
        rz_new = float(np.vdot(rr, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return e, its


def mg_pcg_solve(F: np.ndarray, phi0: np.ndarray | None = None, inner_steps: int = 2, tol: float = 1e-10,
                 max_outer: int = 50, levels: int = 0, degree: int = 3, alpha: float = 8.0):
    """Defect correction whose correction is `inner_steps` steps of PCG on A e = r with one
    V-cycle from zero (Chebyshev smoother) as the preconditioner.  Returns (phi, history)
    with the relative residual before the first and after every outer step."""
    F = project_mean(np.asarray(F, dtype=np.float64))
    nlev = len(level_shapes(F.shape, levels))
    phi = np.zeros_like(F) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    nF = float(np.linalg.norm(F))
    hist = [float(np.linalg.norm(residual(F, phi))) / nF]
    M = lambda v: vcycle(0, np.zeros_like(v), v, nlev, "cheb", degree, alpha)
    for _ in range(max_outer):
        if hist[-1] <= tol:
            break
        e, _ = pcg(residual(F, phi), inner_steps, M, apply_A)
        phi = phi + e
        hist.append(float(np.linalg.norm(residual(F, phi))) / nF)
    return phi - phi.mean(), hist
