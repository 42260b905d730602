"""Moving-mesh (curvilinear) oracle: geometry, 19-point operator, V-cycle, adjoint.

TEST INFRASTRUCTURE.  Plain float64 NumPy/SciPy written from the paper:

* Sec. 4.1, Eq. (map): x = xi + grad psi(xi), cell units, periodic.
* Sec. 4.2, Eq. (triad): A = I + Hess psi, second derivatives by 2nd-order
  central stencils, mixed terms with a 1/(4 dx^2) four-point stencil;
  Eq. (metric): g = A^T A, sqrt(g) = det A.
* Sec. 4.3, Eq. (LB) and (curv_linsys): L_psi[u] = (1/sqrt g) d_a(sqrt g g^ab d_b u).
* Sec. 4.3.1: conservative finite volume form with B = sqrt(g) g^-1; normal
  derivative by the two-point difference across the face; tangential
  derivatives central at cell centres and averaged onto the face; divergence
  of the face fluxes divided by sqrt(g) dx.
* Sec. 4.3.2, Eq. (solvability): f <- f - sum(f sqrt g)/sum(sqrt g); gauge:
  plain mean removed from the solution.
* Sec. 4.3.3: weighted Jacobi nu1 = nu2 = 2, V-cycle, L = log2 n_g - 1 levels.
* Appendix B, Eq. (jacobi): u <- u + omega (f - L u)/D, omega = 2/3, with D
  assembled from the face-averaged diagonal coefficients; psi restricted to
  each coarse level by full weighting and the coarse operator rebuilt.
* Sec. 4.8 adjoint, Eq. (curv_operator), (adj_rhs), (adj_op): A = W^-1 M with
  W = diag(sqrt g); F_bar = A^-T phi_bar; s_bar = -[d_s(A phi)]^T F_bar.

Readings taken where the paper is silent or ambiguous:
* Face coefficient B_{i+1/2} = (B_i + B_{i+1})/2 (arithmetic mean).
* The V-cycle works on L = M/J (the paper's A_psi): the residual f - L u is
  restricted, the coarse problem is L_c e = R r.
* With variable B the literal discretisation is not exactly symmetric, so the
  adjoint uses the exact discrete transpose M^T rather than the paper's
  sqrt(g)-conjugation shortcut (which assumes M = M^T); the two coincide when
  M = M^T.
* The adjoint is written in M-form: M phi~ = b, b = J (delta - <delta>_J),
  phi = phi~ - mean(phi~); M^T lambda = g with g the mean-free cotangent.
* Coarsest level: exact least-squares minimum-norm solve (dense pseudo-inverse).
* Symmetric variant (sym=True; not the paper's scheme, which is the literal one
  above): the same face terms B^{aa}, and the cross terms a != b moved to the cell
  edges, -sum_{a != b} E_a^T C_ab E_b with C_ab the mean of B^{ab} over the four cells
  around the edge and E_a the a-difference averaged over the two b-positions of the
  edge.  M = M^T exactly; for constant B both schemes have the same Fourier symbol.

Parity pins (tests/test_oracle_curv.py): psi = 0 reduces to the 7-point
operator; constant-B Fourier symbol; M 1 = 0 and 1^T M = 0; second-order
consistency with the continuum divergence on smooth fields; dot-product test of
the transpose; triad/determinant against closed forms and numpy.linalg;
central finite differences of the full solve for the delta- and psi-gradients;
dense pseudo-inverse solves at 8^3.  Symmetric variant: psi = 0 and constant-B
symbol, dense M = M^T with its diagonal and a 19-point stencil, second-order
consistency (and an O(h^2) gap to the literal scheme), the B-cotangent as the exact
derivative of the bilinear form, dense pseudo-inverse solve and FD gradients.
"""
from __future__ import annotations

import numpy as np

from . import flat

AXIS = (2, 1, 0)  # array axis of Cartesian component x, y, z


def at(u: np.ndarray, comp: int, s: int) -> np.ndarray:
    """u evaluated at i + s e_comp on the periodic mesh."""
    return np.roll(u, -s, axis=AXIS[comp])


def at2(u: np.ndarray, a: int, sa: int, b: int, sb: int) -> np.ndarray:
    return at(at(u, a, sa), b, sb)


# ---------------------------------------------------------------- geometry


def hessian(psi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Hess psi by second-order central stencils (Sec. 4.2).  Shape (3, 3, nz, ny, nx)."""
    H = np.empty((3, 3) + psi.shape)
    for a in range(3):
        H[a, a] = (at(psi, a, 1) - 2.0 * psi + at(psi, a, -1)) / (h * h)
        for b in range(a + 1, 3):
            v = (at2(psi, a, 1, b, 1) - at2(psi, a, 1, b, -1)
                 - at2(psi, a, -1, b, 1) + at2(psi, a, -1, b, -1)) / (4.0 * h * h)
            H[a, b] = v
            H[b, a] = v
    return H


def triad(psi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """A = I + Hess psi, Eq. (triad).  Shape (3, 3, ...)."""
    A = hessian(psi, h)
    for a in range(3):
        A[a, a] += 1.0
    return A


def geometry(psi: np.ndarray, h: float = 1.0):
    """Volume element J = sqrt(g) = det A and B = sqrt(g) g^-1 = J A^-2 per cell.

    Eq. (metric) with g = A^T A = A^2 for the symmetric triad.  Returns (J, B)
    with B of shape (3, 3, nz, ny, nx).
    """
    A = triad(psi, h)
    Am = np.moveaxis(A, (0, 1), (-2, -1))           # (..., 3, 3)
    J = np.linalg.det(Am)
    Ainv = np.linalg.inv(Am)
    B = J[..., None, None] * (Ainv @ Ainv)
    return J, np.moveaxis(B, (-2, -1), (0, 1)).copy()


# ---------------------------------------------------------------- operator


def face_coeff(B: np.ndarray, a: int, b: int) -> np.ndarray:
    """B^{ab} on the a-face i+1/2: arithmetic mean of the two adjacent cells."""
    return 0.5 * (B[a, b] + at(B[a, b], a, 1))


def face_gradients(u: np.ndarray, a: int, h: float):
    """Components of grad u on the a-face i+1/2, index b = 0..2.

    b == a: two-point normal difference (u_{i+a} - u_i)/h.
    b != a: central difference at the two adjacent cell centres, averaged.
    """
    G = []
    for b in range(3):
        if b == a:
            G.append((at(u, a, 1) - u) / h)
        else:
            Db = (at(u, b, 1) - at(u, b, -1)) / (2.0 * h)
            G.append(0.5 * (Db + at(Db, a, 1)))
    return G


def apply_M(u: np.ndarray, B: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Flux-divergence M u = sum_a (F^a_{i+1/2} - F^a_{i-1/2}) / h with F^a = sum_b B^{ab}_face G_b.

    Sec. 4.3.1.  L_psi = M / sqrt(g).
    """
    out = np.zeros_like(u, dtype=np.float64)
    for a in range(3):
        G = face_gradients(u, a, h)
        Fa = sum(face_coeff(B, a, b) * G[b] for b in range(3))
        out += (Fa - at(Fa, a, -1)) / h
    return out


def apply_MT(y: np.ndarray, B: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Exact transpose M^T y, by summation by parts of apply_M.

    <y, M x> = sum_a sum_i F^a[x]_i (y_i - y_{i+a})/h, so with
    q_ab = B^{ab}_face (y_i - y_{i+a})/h, M^T y = sum_ab G_ab^T q_ab, where
    G_aa^T q = (q_{i-a} - q_i)/h and, for b != a,
    G_ab^T q = [(q_{i-b} - q_{i+b}) + (q_{i-a-b} - q_{i-a+b})] / (4h).
    """
    out = np.zeros_like(y, dtype=np.float64)
    for a in range(3):
        lam = (y - at(y, a, 1)) / h
        for b in range(3):
            q = face_coeff(B, a, b) * lam
            if b == a:
                out += (at(q, a, -1) - q) / h
            else:
                out += ((at(q, b, -1) - at(q, b, 1))
                        + (at2(q, a, -1, b, -1) - at2(q, a, -1, b, 1))) / (4.0 * h)
    return out


def diag_M(B: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Diagonal of M: -(1/h^2) sum_a (B^{aa}_{a-face,+} + B^{aa}_{a-face,-}).  Appendix B."""
    d = np.zeros(B.shape[2:])
    for a in range(3):
        fa = face_coeff(B, a, a)
        d -= (fa + at(fa, a, -1)) / (h * h)
    return d


# ---------------------------------------------------------------- symmetric variant


def edge_coeff(B: np.ndarray, a: int, b: int) -> np.ndarray:
    """C_ab on the edge e + (e_a + e_b)/2 (array index e): mean of B^{ab} over its four cells."""
    c = B[a, b]
    return 0.25 * (c + at(c, a, 1) + at(c, b, 1) + at2(c, a, 1, b, 1))


def edge_grad(u: np.ndarray, a: int, b: int, h: float) -> np.ndarray:
    """E_a u on the ab-edges: the a-difference averaged over the edge's two b-positions."""
    return 0.5 * ((at(u, a, 1) - u) + (at2(u, a, 1, b, 1) - at(u, b, 1))) / h


def edge_grad_T(q: np.ndarray, a: int, b: int, h: float) -> np.ndarray:
    """Transpose of edge_grad(., a, b): cells from ab-edge values."""
    return 0.5 * ((at(q, a, -1) - q) + (at2(q, a, -1, b, -1) - at(q, b, -1))) / h


def apply_M_sym(u: np.ndarray, B: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Symmetric variant: sum_a (face flux differences of B^{aa}) - sum_{a != b} E_a^T C_ab E_b u."""
    out = np.zeros_like(u, dtype=np.float64)
    for a in range(3):
        Fa = face_coeff(B, a, a) * (at(u, a, 1) - u) / h
        out += (Fa - at(Fa, a, -1)) / h
        for b in range(3):
            if b == a:
                continue
            lo, hi = min(a, b), max(a, b)           # the edge set of the unordered pair
            C = edge_coeff(B, lo, hi)
            out -= edge_grad_T(C * edge_grad(u, b, a, h), a, b, h)
    return out


def diag_M_sym(B: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Diagonal of apply_M_sym: the face part of diag_M plus, per pair a < b,
    (1/2h^2)(-C(e) + C(e-a) + C(e-b) - C(e-a-b)) from the four edges around the cell."""
    d = diag_M(B, h)
    for a in range(3):
        for b in range(a + 1, 3):
            C = edge_coeff(B, a, b)
            d += 0.5 * (-C + at(C, a, -1) + at(C, b, -1) - at2(C, a, -1, b, -1)) / (h * h)
    return d


def Bbar_from_operator_sym(lam: np.ndarray, phi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Cotangent of B for <lam, M_sym(B) phi>: the face part as Bbar_from_operator's
    b == a terms; per pair a < b, dC(e) = -[(E_a lam)(E_b phi) + (E_b lam)(E_a phi)](e),
    spread as 1/4 onto the edge's four cells (all of it in Bbar[a, b], none in Bbar[b, a])."""
    Bbar = np.zeros((3, 3) + phi.shape)
    for a in range(3):
        Lam = (lam - at(lam, a, 1)) / h
        fbar = (at(phi, a, 1) - phi) / h * Lam
        Bbar[a, a] += 0.5 * (fbar + at(fbar, a, -1))
        for b in range(a + 1, 3):
            cbar = -(edge_grad(lam, a, b, h) * edge_grad(phi, b, a, h)
                     + edge_grad(lam, b, a, h) * edge_grad(phi, a, b, h))
            Bbar[a, b] += 0.25 * (cbar + at(cbar, a, -1) + at(cbar, b, -1) + at2(cbar, a, -1, b, -1))
    return Bbar


# ---------------------------------------------------------------- hierarchy


class Level:
    def __init__(self, psi: np.ndarray, h: float, sym: bool = False):
        self.psi = psi
        self.h = h
        self.sym = sym
        self.J, self.B = geometry(psi, h)
        # diagonal of M (same for M^T)
        self.D = diag_M_sym(self.B, h) if sym else diag_M(self.B, h)

    def L(self, u, transpose=False):
        """L u = M u / J (forward) or M^T u / J (operator of the transposed solve)."""
        if self.sym:
            Mu = apply_M_sym(u, self.B, self.h)
        else:
            Mu = apply_MT(u, self.B, self.h) if transpose else apply_M(u, self.B, self.h)
        return Mu / self.J


def hierarchy(psi: np.ndarray, levels: int = 0, sym: bool = False) -> list[Level]:
    """psi_{l+1} = R psi_l (full weighting), geometry rebuilt with h_l = 2^l (Appendix B, Sec. 4.3)."""
    shapes = flat.level_shapes(psi.shape, levels)
    out = []
    p = np.asarray(psi, dtype=np.float64)
    for l in range(len(shapes)):
        out.append(Level(p, float(2 ** l), sym))
        if l + 1 < len(shapes):
            p = flat.restrict_fw(p)
    return out


def dense_L(level: Level, transpose: bool = False) -> np.ndarray:
    """Dense matrix of L (or the transposed-solve operator) built column by column from unit vectors."""
    n = level.psi.size
    shape = level.psi.shape
    Mat = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        Mat[:, j] = level.L(e.reshape(shape), transpose).ravel()
        e[j] = 0.0
    return Mat


def coarse_solve(level: Level, r: np.ndarray, transpose: bool = False, cache: dict | None = None):
    """Minimum-norm least-squares solve with the dense pseudo-inverse of the coarsest operator."""
    key = (id(level), transpose)
    if cache is not None and key in cache:
        P = cache[key]
    else:
        # relative cutoff 1e-10 drops the constant null mode (its singular value is at rounding level)
        P = np.linalg.pinv(dense_L(level, transpose), rcond=1e-10)
        if cache is not None:
            cache[key] = P
    return (P @ r.ravel()).reshape(r.shape)


def vcycle(l: int, e: np.ndarray, r: np.ndarray, hier: list[Level], nu1: int = 2, nu2: int = 2,
           omega: float = 2.0 / 3.0, transpose: bool = False, cache: dict | None = None):
    """Curvilinear V-cycle for L_l e = r (Sec. 4.3, Eq. (curv_error); Appendix B).

    Weighted Jacobi u += omega (r - L u)/D_L with D_L = diag(M)/J; residual
    restricted by full weighting; coarse operator rebuilt from the restricted
    psi; trilinear prolongation.
    """
    lev = hier[l]
    if l == len(hier) - 1:
        return coarse_solve(lev, r, transpose, cache)
    DL = lev.D / lev.J
    for _ in range(nu1):
        e = e + omega * (r - lev.L(e, transpose)) / DL
    rc = flat.restrict_fw(r - lev.L(e, transpose))
    ec = vcycle(l + 1, np.zeros_like(rc), rc, hier, nu1, nu2, omega, transpose, cache)
    e = e + flat.prolong(ec)
    for _ in range(nu2):
        e = e + omega * (r - lev.L(e, transpose)) / DL
    return e


def weighted_projection(delta: np.ndarray, J: np.ndarray) -> np.ndarray:
    """f = delta - sum(delta sqrt g)/sum(sqrt g), Eq. (solvability)."""
    return delta - float((delta * J).sum() / J.sum())


def solve(delta: np.ndarray, psi: np.ndarray, tol: float = 1e-10, max_cycles: int = 100,
          levels: int = 0, nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0,
          phi0: np.ndarray | None = None, fixed_cycles: int | None = None,
          hier: list[Level] | None = None, sym: bool = False):
    """Curvilinear Poisson solve L_psi phi = f with f the volume-weighted projection of delta.

    V-cycles until ||f - L phi|| / ||f|| <= tol; the mean of phi is removed at
    the end (Sec. 4.3.2 gauge).  Returns (phi, history).
    """
    hier = hierarchy(psi, levels, sym) if hier is None else hier
    f = weighted_projection(np.asarray(delta, dtype=np.float64), hier[0].J)
    phi = np.zeros_like(f) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    nf = float(np.linalg.norm(f))
    hist = [float(np.linalg.norm(f - hier[0].L(phi))) / nf]
    cache: dict = {}
    ncyc = fixed_cycles if fixed_cycles is not None else max_cycles
    for _ in range(ncyc):
        if fixed_cycles is None and hist[-1] <= tol:
            break
        phi = vcycle(0, phi, f, hier, nu1, nu2, omega, False, cache)
        hist.append(float(np.linalg.norm(f - hier[0].L(phi))) / nf)
    return phi - phi.mean(), hist


def solve_transposed(g: np.ndarray, hier: list[Level], tol: float = 1e-10, max_cycles: int = 100,
                     nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0):
    """Solve M^T lam = g (g mean-free) with V-cycles on L~ = W^-1 M^T and source g / J.

    Returns lam with its mean removed (the constant null space of M^T does not
    affect either gradient).
    """
    J = hier[0].J
    s = g / J
    lam = np.zeros_like(g)
    ns = float(np.linalg.norm(s))
    cache: dict = {}
    for _ in range(max_cycles):
        if float(np.linalg.norm(s - hier[0].L(lam, True))) / ns <= tol:
            break
        lam = vcycle(0, lam, s, hier, nu1, nu2, omega, True, cache)
    return lam - lam.mean()


# ---------------------------------------------------------------- adjoint


def hessian_T(Hbar: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Transpose of psi -> H (all nine entries): sum_ab D_ab^T Hbar_ab; each stencil is self-adjoint."""
    out = np.zeros(Hbar.shape[2:])
    for a in range(3):
        out += (at(Hbar[a, a], a, 1) - 2.0 * Hbar[a, a] + at(Hbar[a, a], a, -1)) / (h * h)
        for b in range(3):
            if b == a:
                continue
            q = Hbar[a, b]
            out += (at2(q, a, 1, b, 1) - at2(q, a, 1, b, -1)
                    - at2(q, a, -1, b, 1) + at2(q, a, -1, b, -1)) / (4.0 * h * h)
    return out


def Bbar_from_operator(lam: np.ndarray, phi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Cotangent of the cell coefficients B for the scalar <lam, M(B) phi>.

    <lam, M phi> = sum_a sum_i sum_b B^{ab}_face(i) G_b^a[phi](i) (lam_i - lam_{i+a})/h,
    and B^{ab}_face(i) = (B^{ab}_i + B^{ab}_{i+a})/2.
    """
    Bbar = np.zeros((3, 3) + phi.shape)
    for a in range(3):
        Lam = (lam - at(lam, a, 1)) / h
        G = face_gradients(phi, a, h)
        for b in range(3):
            fbar = G[b] * Lam
            Bbar[a, b] += 0.5 * (fbar + at(fbar, a, -1))
    return Bbar


def Abar_from_B(A: np.ndarray, Bbar: np.ndarray) -> np.ndarray:
    """Cotangent of the triad for B = J A^-2, J = det A (symmetric A, full-matrix cotangent).

    dJ = J tr(A^-1 dA); d(A^-2) = -A^-1 dA A^-2 - A^-2 dA A^-1.
    """
    Am = np.moveaxis(A, (0, 1), (-2, -1))
    Bb = np.moveaxis(Bbar, (0, 1), (-2, -1))
    J = np.linalg.det(Am)
    Ai = np.linalg.inv(Am)
    Ai2 = Ai @ Ai
    inner = np.sum(Bb * Ai2, axis=(-2, -1))
    Ab = (J * inner)[..., None, None] * np.swapaxes(Ai, -1, -2)
    Ab -= J[..., None, None] * (np.swapaxes(Ai, -1, -2) @ Bb @ np.swapaxes(Ai2, -1, -2)
                                + np.swapaxes(Ai2, -1, -2) @ Bb @ np.swapaxes(Ai, -1, -2))
    return np.moveaxis(Ab, (-2, -1), (0, 1))


def Abar_from_J(A: np.ndarray, Jbar: np.ndarray) -> np.ndarray:
    """Cotangent of the triad for J = det A: Jbar J A^-T."""
    Am = np.moveaxis(A, (0, 1), (-2, -1))
    J = np.linalg.det(Am)
    Ai = np.linalg.inv(Am)
    Ab = (Jbar * J)[..., None, None] * np.swapaxes(Ai, -1, -2)
    return np.moveaxis(Ab, (-2, -1), (0, 1))


def solve_vjp(delta: np.ndarray, psi: np.ndarray, phi: np.ndarray, phi_bar: np.ndarray,
              tol: float = 1e-11, max_cycles: int = 200, levels: int = 0,
              nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0, sym: bool = False):
    """Gradients of <phi_bar, phi> for phi = solve(delta, psi): returns (delta_bar, psi_bar).

    M-form of Eq. (adj_rhs) and (adj_op): M phi~ = b with b = J (delta - <delta>_J)
    and phi = phi~ - mean(phi~).  With g = phi_bar - mean(phi_bar) and
    M^T lam = g,
      delta_bar = J lam - J sum(J lam)/sum(J),
      psi_bar   = Hess^T[ Abar_J(Jbar) - Abar_B(Bbar) ],
    where Jbar = (delta - <delta>_J)(lam - sum(J lam)/sum(J)) is the source's
    dependence on J and Bbar is the operator's dependence on B contracted with
    lam and phi.  `phi` is the converged forward solution.
    """
    hier = hierarchy(psi, levels, sym)
    lev0 = hier[0]
    J = lev0.J
    g = phi_bar - phi_bar.mean()
    lam = solve_transposed(g, hier, tol, max_cycles, nu1, nu2, omega)
    T = J.sum()
    lamJ = float((lam * J).sum()) / T
    delta_bar = J * lam - J * lamJ
    f = weighted_projection(delta, J)
    Jbar = f * (lam - lamJ)
    A = triad(psi, lev0.h)
    Bbar = Bbar_from_operator_sym(lam, phi, lev0.h) if sym else Bbar_from_operator(lam, phi, lev0.h)
    Abar = Abar_from_J(A, Jbar) - Abar_from_B(A, Bbar)
    psi_bar = hessian_T(Abar, lev0.h)
    return delta_bar, psi_bar


# ---------------------------------------------------------------- mesh motion


def smooth_binomial(u: np.ndarray, passes: int) -> np.ndarray:
    """passes of the separable [1/4, 1/2, 1/4] filter, periodic (the one-axis weights of the
    full-weighting restriction, Appendix B, without decimation; the paper smooths the
    mesh-motion source without naming the filter)."""
    u = np.asarray(u, dtype=np.float64)
    for _ in range(passes):
        for ax in range(3):
            u = 0.25 * (np.roll(u, 1, axis=ax) + np.roll(u, -1, axis=ax)) + 0.5 * u
    return u


def mesh_motion_step(psi: np.ndarray, rho: np.ndarray, kappa: float, m_init: float, dtau: float,
                     passes: int = 2, tol: float = 1e-10):
    """One mesh-motion step (Sec. 4.4): L_psi[psidot] = kappa (m_init - sqrt(g) rho), Eq. calcdefp,
    with the smoothed source, solved by the curvilinear solver (weighted projection, zero-mean
    gauge); then psi <- Z[psi + dtau psidot], Eq. defadvance.  Returns (psi_new, psidot)."""
    J = geometry(np.asarray(psi, dtype=np.float64), 1.0)[0]
    src = smooth_binomial(kappa * (m_init - J * rho), passes)
    psidot, _ = solve(src, psi, tol=tol)
    new = psi + dtau * psidot
    return new - new.mean(), psidot
