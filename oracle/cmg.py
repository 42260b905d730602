"""ctypes wrapper of the C FP64 V-cycle (oracle/mg_fp64.c).

TEST INFRASTRUCTURE: the CPU oracle in C, used where the NumPy oracle is too slow (a
full 512^3 solve on the host cores for the CPU baseline and the reference arm of the
benchmark).  It follows the same steps as oracle/flat.py (Sec. 2.1-2.3, Appendix B;
see the C file's header) and shares no code with the CUDA library.

Parity pins (tests/test_oracle_cmg.py): the operator on plane waves against the
eigenvalues of Eq. (fftsolve); the Chebyshev pass on a plane wave against the factor
T_v((theta - mu)/delta) / T_v(theta/delta); the coarsest solve against numpy's dense
pseudo-inverse; V-cycle iterates against oracle/flat.py's at 1e-12; convergence to the
FFT solution; results independent of the thread count.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mg_fp64.c")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libora_mg.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/_build/libora_mg.so with the host C compiler (OpenMP if available)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle")
    tmp = LIB + ".tmp"
    base = [cc, "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle C build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.ora_create.restype = P
        L.ora_create.argtypes = [I, I, I, I, I, D]
        L.ora_destroy.argtypes = [P]
        L.ora_levels.restype = I
        L.ora_levels.argtypes = [P]
        L.ora_threads.restype = I
        L.ora_set_threads.argtypes = [I]
        L.ora_vcycle.argtypes = [P, P, P]
        L.ora_solve.restype = I
        L.ora_solve.argtypes = [P, P, P, D, I, P]
        L.ora_begin.restype = D
        L.ora_begin.argtypes = [P, P, P]
        L.ora_cycle.restype = D
        L.ora_cycle.argtypes = [P]
        L.ora_end.argtypes = [P, P]
        L.ora_apply.argtypes = [I, I, I, D, P, P]
        L.ora_smooth_cheb.restype = I
        L.ora_smooth_cheb.argtypes = [I, I, I, D, I, D, P, P]
        _lib = L
    return _lib


def threads() -> int:
    """Threads the C oracle runs on (OpenMP's default: the host's cores)."""
    return int(lib().ora_threads())


def set_threads(n: int) -> None:
    """Run the C oracle's loops on n threads."""
    lib().ora_set_threads(int(n))


def _f64(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def apply_A(u: np.ndarray, h: float = 1.0) -> np.ndarray:
    """7-point periodic Laplacian of u at spacing h."""
    u = _f64(u)
    out = np.empty_like(u)
    nz, ny, nx = u.shape
    lib().ora_apply(nx, ny, nz, float(h), u.ctypes.data, out.ctypes.data)
    return out


def smooth_chebyshev(e: np.ndarray, r: np.ndarray, h: float, degree: int = 3, alpha: float = 8.0) -> np.ndarray:
    """One Chebyshev smoothing pass of A e = r (returns the new e)."""
    e = np.array(e, dtype=np.float64, copy=True, order="C")
    r = _f64(r)
    nz, ny, nx = e.shape
    if lib().ora_smooth_cheb(nx, ny, nz, float(h), int(degree), float(alpha), e.ctypes.data, r.ctypes.data):
        raise MemoryError("oracle C smoother")
    return e


class Solver:
    """FP64 V(degree, degree) Chebyshev multigrid on an (nz, ny, nx) periodic mesh."""

    def __init__(self, shape, levels: int = 0, degree: int = 3, alpha: float = 8.0):
        nz, ny, nx = (shape,) * 3 if isinstance(shape, int) else tuple(int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self._c = lib().ora_create(nx, ny, nz, levels, degree, alpha)
        if not self._c:
            raise ValueError(f"oracle C solver: unsupported mesh {self.shape}")
        self.levels = int(lib().ora_levels(self._c))

    def close(self):
        if self._c:
            lib().ora_destroy(self._c)
            self._c = None

    def __del__(self):
        self.close()

    def vcycle(self, r: np.ndarray) -> np.ndarray:
        """One V-cycle on A e = r from e = 0."""
        r = _f64(r)
        assert r.shape == self.shape
        e = np.empty_like(r)
        lib().ora_vcycle(self._c, r.ctypes.data, e.ctypes.data)
        return e

    def begin(self, F: np.ndarray, phi0: np.ndarray) -> float:
        """Start a solve of A phi = F - mean(F) from phi0; returns the relative residual.
        F and phi0 are read now (the solver keeps its own copies)."""
        F, phi0 = _f64(F), _f64(phi0)
        assert F.shape == self.shape and phi0.shape == self.shape
        return float(lib().ora_begin(self._c, F.ctypes.data, phi0.ctypes.data))

    def cycle(self) -> float:
        """One V-cycle of the solve in progress; returns the new relative residual."""
        return float(lib().ora_cycle(self._c))

    def end(self, out: np.ndarray | None = None) -> np.ndarray:
        """The solve's iterate with its mean removed."""
        out = np.empty(self.shape) if out is None else out
        assert out.shape == self.shape and out.dtype == np.float64 and out.flags.c_contiguous
        lib().ora_end(self._c, out.ctypes.data)
        return out

    def solve(self, F: np.ndarray, phi0: np.ndarray | None = None, tol: float = 1e-10, max_cycles: int = 50):
        """Returns (phi, history) like oracle.flat.mg_solve."""
        F = _f64(F)
        assert F.shape == self.shape
        phi = np.zeros_like(F) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True, order="C")
        hist = np.zeros(max_cycles + 1)
        k = lib().ora_solve(self._c, F.ctypes.data, phi.ctypes.data, float(tol), int(max_cycles), hist.ctypes.data)
        return phi, [float(v) for v in hist[:k + 1]]
