"""GB300-native geometric multigrid for the particle-mesh Poisson equation.

Thin ctypes binding of the C ABI in include/gbmg.h (libgbmg.so, built in-tree by
`_build.build()`).  This module only marshals arguments: every step of a solve
runs in the library's CUDA kernels.  Tensors are torch CUDA tensors, contiguous,
shaped (nz, ny, nx) with x fastest; torch's current stream is used for each call.

If libgbmg.so is missing the import still succeeds but every call raises
RuntimeError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

__all__ = ["Solver", "GbmgError", "Stats", "lib", "library_path", "launch_count", "F32", "F64"]

F32, F64 = 0, 1
OP_FLAT7, OP_CURV19 = 0, 1
FP64, MIXED = 0, 1
CHEBYSHEV, JACOBI = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "not converged",
          5: "non-finite residual", 6: "diverged", 7: "invalid state"}
CONVERGENCE_STATUSES = (4, 5, 6)


class GbmgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("prec", ctypes.c_int), ("smoother", ctypes.c_int),
                ("degree", ctypes.c_int), ("alpha", ctypes.c_double), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("fused", ctypes.c_int),
                ("krylov", ctypes.c_int), ("curv_sym", ctypes.c_int),
                ("coarse_store", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("rel_res0", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("res_hist", ctypes.c_double * 64)]


@dataclass
class Stats:
    cycles: int
    status: int
    rel_res0: float
    rel_res: float
    history: list

    @classmethod
    def from_c(cls, s: _Stats) -> "Stats":
        return cls(s.cycles, s.status, s.rel_res0, s.rel_res, [s.res_hist[i] for i in range(min(s.cycles, 64))])


_LIB = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong
_S = ctypes.c_int  # gbmg_status

# name -> (restype, argtypes)
_SIGS = {
    "gbmg_default_opts": (None, [ctypes.POINTER(_Opts)]),
    "mg_setup": (_S, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, ctypes.POINTER(_Opts), _P]),
    "mg_destroy": (None, [_P]),
    "mg_set_stream": (_S, [_P, _P]),
    "mg_set_cycle_graphs": (_S, [_P, ctypes.c_int]),
    "mg_solve": (_S, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(_Stats)]),
    "mg_solve_host": (_S, [_P, _P, _P, _D, _I, ctypes.POINTER(_Stats)]),
    "mg_solve_host_sequence": (_S, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P, _D, _I,
                                    ctypes.POINTER(_Stats)]),
    "mg_last_stats": (_S, [_P, ctypes.POINTER(_Stats)]),
    "mg_num_levels": (_I, [_P]),
    "mg_level_dims": (_S, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mg_status_string": (ctypes.c_char_p, [_S]),
    "mg_last_error": (ctypes.c_char_p, []),
    "mg_apply": (_S, [_P, _I, _I, _P, _P]),
    "mg_residual": (_S, [_P, _I, _I, _P, _P, _P]),
    "mg_smooth": (_S, [_P, _I, _I, _P, _P]),
    "mg_restrict": (_S, [_P, _I, _I, _P, _P]),
    "mg_prolong_add": (_S, [_P, _I, _I, _P, _P]),
    "mg_coarse_solve": (_S, [_P, _I, _P, _P]),
    "mg_vcycle": (_S, [_P, _P, _P]),
    "mg_f64_to_df": (_S, [_P, _LL, _P, _P]),
    "mg_df_to_f64": (_S, [_P, _LL, _P, _P]),
    "mg_df_residual": (_S, [_P, _P, _D, _P, _P]),
    "mg_set_geometry": (_S, [_P, _P]),
    "mg_set_coefficients": (_S, [_P, _P, _P]),
    "mg_solve_adjoint": (_S, [_P, _P, _P, _P, _P, _P, _D, _I, ctypes.POINTER(_Stats)]),
    "mg_curv_apply": (_S, [_P, _I, _I, _I, _I, _P, _P]),
    "mg_curv_geometry": (_S, [_P, _I, _P, _P]),
    "mg_curv_vcycle": (_S, [_P, _I, _P, _P]),
    "mg_curv_residual": (_S, [_P, _I, _I, _P, _P, _P]),
    "mg_curv_smooth": (_S, [_P, _I, _I, _P, _P, _P]),
    "mg_profile_begin": (_S, [_P, _I]),
    "mg_profile_read": (_S, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "mg_profile_end": (_S, [_P]),
    "mg_launch_count": (_LL, []),
    "mg_rel_residual_noalloc": (_S, [_I, _I, _I, _P, _P, _P, _P]),
    "mg_grad": (_S, [_P, _I, _I, _P, _P]),
    "mg_grad_dot": (_S, [_P, _I, _P, _P, _P]),
    "mg_predict": (_S, [_P, _I, _D, ctypes.POINTER(_P), _I, _P]),
    "mg_cic_paint": (_S, [_P, _P, _P, _D, ctypes.c_longlong, _P]),
    "mg_cic_read": (_S, [_P, _P, _I, _P, ctypes.c_longlong, _P]),
    "mg_force": (_S, [_P, _P, _P, ctypes.c_longlong, _P]),
    "mg_mesh_motion": (_S, [_P, _P, _D, _D, _I, _D, _P, _P, _D, _I, ctypes.POINTER(_Stats)]),
    "mg_batch_create": (_S, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _P]),
    "mg_batch_destroy": (None, [_P]),
    "mg_batch_set_blocks": (_S, [_P, _I]),
    "mg_batch_set_tiles": (_S, [_P, ctypes.POINTER(_I), _I]),
    "mg_batch_get_tiles": (_S, [_P, ctypes.POINTER(_I), _I]),
    "mg_batch_num_levels": (_I, [_P]),
    "mg_batch_use_graph": (_S, [_P, _I]),
    "mg_batch_autotune": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(_I),
                               ctypes.POINTER(_I)]),
    "mg_batch_solve": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(_Stats),
                            ctypes.POINTER(_D)]),
}

PROF = {"down0": 1, "up0": 2, "df0": 3, "smooth0": 4, "curv0": 5}


def launch_count() -> int:
    """Kernels launched by libgbmg.so in this process so far."""
    return int(lib().mg_launch_count())


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgbmg.so (built by `_build.build()`); raises if it is not there."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgbmg.so is not built ({path}); run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, allow_convergence: bool = False):
    if status == 0 or (allow_convergence and status in CONVERGENCE_STATUSES):
        return
    raise GbmgError(status, lib().mg_last_error().decode())


def _ptr(t: torch.Tensor | None, dtype=None, shape=None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise ValueError("expected float32 or float64")


def _shape3(n) -> tuple[int, int, int]:
    if isinstance(n, int):
        return (n, n, n)
    return tuple(int(v) for v in n)


class Solver:
    """One multigrid hierarchy for a periodic (nz, ny, nx) mesh on the current CUDA device."""

    def __init__(self, shape, levels: int = 0, degree: int = 3, prec: str = "mixed",
                 smoother: str | None = None, fused: bool = True, alpha: float = 8.0,
                 nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0, op: str = "flat", krylov: int = 0,
                 curv_sym: bool = False, coarse_store: str = "fp32"):
        L = lib()
        if smoother is None:
            smoother = "jacobi" if op == "curv" else "chebyshev"
        self.op = op
        self.shape = _shape3(shape)
        o = _Opts()
        L.gbmg_default_opts(ctypes.byref(o))
        o.op = {"flat": OP_FLAT7, "curv": OP_CURV19}[op]
        o.prec = {"fp64": FP64, "mixed": MIXED}[prec]
        o.smoother = {"chebyshev": CHEBYSHEV, "jacobi": JACOBI}[smoother]
        o.degree, o.alpha, o.nu1, o.nu2, o.omega, o.fused = degree, alpha, nu1, nu2, omega, int(fused)
        o.krylov = int(krylov)
        o.curv_sym = int(curv_sym)
        o.coarse_store = {"fp32": 0, "bf16": 1, "fp16": 2}[coarse_store]
        self.prec = prec
        self.work_dtype = torch.float64 if prec == "fp64" else torch.float32
        ctx = _P()
        nz, ny, nx = self.shape
        _check(L.mg_setup(ctypes.byref(ctx), nx, ny, nz, levels, degree, ctypes.byref(o),
                          torch.cuda.current_stream().cuda_stream))
        self._ctx = ctx
        self.levels = L.mg_num_levels(ctx)

    # -- lifetime
    def close(self):
        if getattr(self, "_ctx", None):
            lib().mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self):
        if not self._ctx:
            raise RuntimeError("solver is closed")
        _check(lib().mg_set_stream(self._ctx, torch.cuda.current_stream().cuda_stream))
        return self._ctx

    def level_shape(self, level: int) -> tuple[int, int, int]:
        x, y, z = _I(), _I(), _I()
        _check(lib().mg_level_dims(self._ctx, level, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z)))
        return (z.value, y.value, x.value)

    # -- solves
    def set_geometry(self, psi: torch.Tensor):
        """Curvilinear contexts: set the deformation potential psi (float64, mesh shape)."""
        _check(lib().mg_set_geometry(self._c(), _ptr(psi, torch.float64, self.shape)))

    def set_coefficients(self, J: torch.Tensor, B: torch.Tensor):
        """Curvilinear contexts: set J (float32, mesh shape) and B (float32, (6,) + mesh shape,
        packed xx, yy, zz, xy, xz, yz) directly; coarse levels restrict them."""
        _check(lib().mg_set_coefficients(self._c(), _ptr(J, torch.float32, self.shape),
                                         _ptr(B, torch.float32, (6,) + self.shape)))

    def solve(self, F: torch.Tensor, phi: torch.Tensor | None = None, tol: float = 1e-6,
              max_vcycles: int = 50, raise_on_nonconvergence: bool = False, psi: torch.Tensor | None = None):
        """Solve A phi = F (or L_psi phi = F); phi (float64) is the warm start and is overwritten.

        Returns (phi, Stats).  Non-convergence is reported in Stats.status unless
        raise_on_nonconvergence is set.  psi (curvilinear only) sets the geometry first.
        """
        ctx = self._c()
        if phi is None:
            phi = torch.zeros_like(F)
        st = _Stats()
        s = lib().mg_solve(ctx, _ptr(F, torch.float64, self.shape), _ptr(psi, torch.float64, self.shape),
                           _ptr(phi, torch.float64, self.shape), float(tol), int(max_vcycles), ctypes.byref(st))
        _check(s, allow_convergence=not raise_on_nonconvergence)
        return phi, Stats.from_c(st)

    def solve_adjoint(self, phi_bar: torch.Tensor, phi: torch.Tensor | None = None,
                      source: torch.Tensor | None = None, want_psi_bar: bool = False, tol: float = 1e-6,
                      max_vcycles: int = 50):
        """Vector-Jacobian product of the solve: returns (source_bar, psi_bar or None, Stats)."""
        src_bar = torch.empty_like(phi_bar)
        psi_bar = torch.empty_like(phi_bar) if want_psi_bar else None
        st = _Stats()
        s = lib().mg_solve_adjoint(self._c(), _ptr(phi_bar, torch.float64, self.shape), _ptr(src_bar),
                                   _ptr(psi_bar), _ptr(phi, torch.float64, self.shape),
                                   _ptr(source, torch.float64, self.shape), float(tol), int(max_vcycles),
                                   ctypes.byref(st))
        _check(s, allow_convergence=True)
        return src_bar, psi_bar, Stats.from_c(st)

    def curv_apply(self, level: int, u: torch.Tensor, transpose: bool = False, divide_by_J: bool = True):
        out = torch.empty_like(u)
        _check(lib().mg_curv_apply(self._c(), level, _dtype_code(u), int(transpose), int(divide_by_J),
                                   _ptr(u, shape=self.level_shape(level)), _ptr(out)))
        return out

    def curv_geometry(self, level: int):
        """(J, B) of a level as float32 tensors, B packed xx, yy, zz, xy, xz, yz."""
        shp = self.level_shape(level)
        dev = torch.device("cuda", torch.cuda.current_device())
        J = torch.empty(shp, dtype=torch.float32, device=dev)
        B = torch.empty((6,) + shp, dtype=torch.float32, device=dev)
        _check(lib().mg_curv_geometry(self._c(), level, _ptr(J), _ptr(B)))
        return J, B

    def curv_residual(self, level: int, r: torch.Tensor, u: torch.Tensor, transpose: bool = False):
        """FP32 residual r - op(u) / (h^2 J) of a level (the V-cycle's tiled kernel)."""
        shp = self.level_shape(level)
        out = torch.empty_like(r)
        _check(lib().mg_curv_residual(self._c(), level, int(transpose), _ptr(r, torch.float32, shp),
                                      _ptr(u, torch.float32, shp), _ptr(out)))
        return out

    def curv_smooth(self, level: int, e: torch.Tensor | None, r: torch.Tensor, transpose: bool = False):
        """One FP32 weighted-Jacobi sweep of a level (the V-cycle's tiled kernel); returns the new e.
        e None: sweep of a zero iterate (the pointwise first sweep of the V-cycle)."""
        shp = self.level_shape(level)
        out = torch.empty_like(r)
        _check(lib().mg_curv_smooth(self._c(), level, int(transpose), _ptr(e, torch.float32, shp),
                                    _ptr(r, torch.float32, shp), _ptr(out)))
        return out

    def curv_vcycle(self, r: torch.Tensor, transpose: bool = False):
        out = torch.empty_like(r)
        _check(lib().mg_curv_vcycle(self._c(), int(transpose), _ptr(r, torch.float32, self.shape), _ptr(out)))
        return out

    def predict(self, history, order: int = 1, growth: float = 1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """Warm-start predictor (mg_predict): history[0] is the most recent solution.
        order 0: growth * phi_{n-1}; 1: 2 phi_{n-1} - phi_{n-2}; 2: 3 phi_{n-1} - 3 phi_{n-2} + phi_{n-3}."""
        if out is None:
            out = torch.empty_like(history[0])
        arr = (_P * len(history))(*[_ptr(h, torch.float64, self.shape) for h in history])
        _check(lib().mg_predict(self._c(), int(order), float(growth), arr, len(history),
                                _ptr(out, torch.float64, self.shape)))
        return out

    def mesh_motion(self, rho: torch.Tensor, psi: torch.Tensor, kappa: float, m_init: float, dtau: float,
                    psidot: torch.Tensor | None = None, smooth_passes: int = 2, tol: float = 1e-6,
                    max_vcycles: int = 100):
        """One mesh-motion step (mg_mesh_motion): psi (float64) advanced in place; returns (psi, psidot, Stats)."""
        if psidot is None:
            psidot = torch.zeros_like(psi)
        st = _Stats()
        s = lib().mg_mesh_motion(self._c(), _ptr(rho, torch.float64, self.shape), float(kappa), float(m_init),
                                 int(smooth_passes), float(dtau), _ptr(psi, torch.float64, self.shape),
                                 _ptr(psidot, torch.float64, self.shape), float(tol), int(max_vcycles), ctypes.byref(st))
        _check(s, allow_convergence=True)
        return psi, psidot, Stats.from_c(st)

    def cic_paint(self, pos: torch.Tensor, mass=1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """Cloud-in-cell density (float64, mesh shape) of particles pos (n, 3) float32 in cell units;
        mass: scalar or float32 tensor (n,)."""
        if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous float32 (n, 3) tensor")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=pos.device)
        mptr, m0 = (None, float(mass)) if not torch.is_tensor(mass) else (_ptr(mass, torch.float32, (pos.shape[0],)), 0.0)
        _check(lib().mg_cic_paint(self._c(), _ptr(pos, torch.float32), mptr, m0, int(pos.shape[0]),
                                  _ptr(out, torch.float64, self.shape)))
        return out

    def cic_read(self, field: torch.Tensor, pos: torch.Tensor) -> torch.Tensor:
        """Field (ncomp, *mesh) or mesh-shaped, float64, interpolated at pos (n, 3) float32: (n, ncomp)."""
        if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 3 or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous float32 (n, 3) tensor")
        nc = 1 if field.dim() == 3 else field.shape[0]
        out = torch.empty((pos.shape[0], nc), dtype=torch.float64, device=pos.device)
        shp = self.shape if nc == 1 and field.dim() == 3 else (nc,) + self.shape
        _check(lib().mg_cic_read(self._c(), _ptr(field, torch.float64, shp), nc, _ptr(pos, torch.float32),
                                 int(pos.shape[0]), _ptr(out)))
        return out

    def force(self, phi: torch.Tensor, pos: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """FP32 force -grad4 phi at the particles (mg_force): (n, 3) float32."""
        if out is None:
            out = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=pos.device)
        _check(lib().mg_force(self._c(), _ptr(phi, torch.float64, self.shape), _ptr(pos, torch.float32),
                              int(pos.shape[0]), _ptr(out, torch.float32, (pos.shape[0], 3))))
        return out

    def solve_host(self, F, phi, tol: float = 1e-6, max_vcycles: int = 50):
        """Same solve on host float64 arrays (numpy or CPU tensors); phi is overwritten."""
        import numpy as np
        Fa = F.numpy() if isinstance(F, torch.Tensor) else F
        Pa = phi.numpy() if isinstance(phi, torch.Tensor) else phi
        for a in (Fa, Pa):
            if a.dtype != np.float64 or not a.flags.c_contiguous or tuple(a.shape) != self.shape:
                raise ValueError("expected C-contiguous float64 arrays of the solver's shape")
        st = _Stats()
        s = lib().mg_solve_host(self._c(), Fa.ctypes.data, Pa.ctypes.data, float(tol), int(max_vcycles),
                                ctypes.byref(st))
        _check(s, allow_convergence=True)
        return phi, Stats.from_c(st)

    def solve_host_sequence(self, sources, phis, phi0=None, tol: float = 1e-6, max_vcycles: int = 50):
        """Warm-started sequence on host float64 arrays: phis[t] receives the solution for
        sources[t], each solve starting from the previous one (phi0, or zero, for the first).
        Copies overlap the neighbouring solves; page-locked buffers (pinned tensors) make
        them asynchronous.  Returns the per-solve Stats."""
        import numpy as np

        def host(a):
            a = a.numpy() if isinstance(a, torch.Tensor) else a
            if a.dtype != np.float64 or not a.flags.c_contiguous or tuple(a.shape) != self.shape:
                raise ValueError("expected C-contiguous float64 arrays of the solver's shape")
            return a
        if len(sources) != len(phis):
            raise ValueError("sources and phis differ in length")
        src = [host(a) for a in sources]
        out = [host(a) for a in phis]
        count = len(src)
        sp = (_P * max(count, 1))(*[a.ctypes.data for a in src])
        op = (_P * max(count, 1))(*[a.ctypes.data for a in out])
        p0 = host(phi0).ctypes.data if phi0 is not None else None
        st = (_Stats * max(count, 1))()
        s = lib().mg_solve_host_sequence(self._c(), count, sp, op, p0, float(tol), int(max_vcycles), st)
        _check(s, allow_convergence=True)
        return [Stats.from_c(st[t]) for t in range(count)]

    # -- measurement
    def set_cycle_graphs(self, enable: bool):
        """Run each V-cycle as one CUDA graph launch (default) or launch every kernel eagerly."""
        _check(lib().mg_set_cycle_graphs(self._c(), 1 if enable else 0))

    def profile_begin(self, families):
        """Time every launch of the named kernel families (see PROF) with CUDA events."""
        mask = 0
        for f in families:
            mask |= 1 << PROF[f]
        _check(lib().mg_profile_begin(self._c(), mask))

    def profile_read(self, family: str) -> tuple[int, float]:
        """(launches, total device milliseconds) of a timed family since profile_begin."""
        n, ms = _I(), _D()
        _check(lib().mg_profile_read(self._c(), PROF[family], ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def profile_end(self):
        _check(lib().mg_profile_end(self._c()))

    # -- components (each runs one kernel family of the V-cycle)
    def apply(self, level: int, u: torch.Tensor, out: torch.Tensor | None = None):
        out = torch.empty_like(u) if out is None else out
        _check(lib().mg_apply(self._c(), level, _dtype_code(u), _ptr(u, shape=self.level_shape(level)), _ptr(out)))
        return out

    def residual(self, level: int, f: torch.Tensor, u: torch.Tensor, out: torch.Tensor | None = None):
        out = torch.empty_like(u) if out is None else out
        shp = self.level_shape(level)
        _check(lib().mg_residual(self._c(), level, _dtype_code(u), _ptr(f, u.dtype, shp), _ptr(u, shape=shp),
                                 _ptr(out, u.dtype, shp)))
        return out

    def smooth(self, level: int, e: torch.Tensor, r: torch.Tensor):
        shp = self.level_shape(level)
        _check(lib().mg_smooth(self._c(), level, _dtype_code(e), _ptr(e, shape=shp), _ptr(r, e.dtype, shp)))
        return e

    def restrict(self, level: int, fine: torch.Tensor, out: torch.Tensor | None = None):
        shp = self.level_shape(level + 1)
        out = torch.empty(shp, dtype=fine.dtype, device=fine.device) if out is None else out
        _check(lib().mg_restrict(self._c(), level, _dtype_code(fine), _ptr(fine, shape=self.level_shape(level)),
                                 _ptr(out, fine.dtype, shp)))
        return out

    def prolong_add(self, level: int, coarse: torch.Tensor, fine: torch.Tensor):
        _check(lib().mg_prolong_add(self._c(), level, _dtype_code(fine), _ptr(coarse, fine.dtype, self.level_shape(level + 1)),
                                    _ptr(fine, shape=self.level_shape(level))))
        return fine

    def coarse_solve(self, r: torch.Tensor, out: torch.Tensor | None = None):
        out = torch.empty_like(r) if out is None else out
        shp = self.level_shape(self.levels - 1)
        _check(lib().mg_coarse_solve(self._c(), _dtype_code(r), _ptr(r, shape=shp), _ptr(out, r.dtype, shp)))
        return out

    def vcycle(self, r: torch.Tensor, out: torch.Tensor | None = None):
        out = torch.empty_like(r) if out is None else out
        _check(lib().mg_vcycle(self._c(), _ptr(r, self.work_dtype, self.shape), _ptr(out, self.work_dtype, self.shape)))
        return out

    def grad(self, u: torch.Tensor, order: int = 4) -> torch.Tensor:
        out = torch.empty((3,) + self.shape, dtype=torch.float64, device=u.device)
        _check(lib().mg_grad(self._c(), order, 0, _ptr(u, torch.float64, self.shape), _ptr(out)))
        return out

    def grad_T(self, w: torch.Tensor, order: int = 4) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float64, device=w.device)
        _check(lib().mg_grad(self._c(), order, 1, _ptr(w, torch.float32, (3,) + self.shape), _ptr(out)))
        return out

    def grad_dot(self, u: torch.Tensor, w: torch.Tensor, order: int = 4) -> torch.Tensor:
        out = torch.empty(1, dtype=torch.float64, device=u.device)
        _check(lib().mg_grad_dot(self._c(), order, _ptr(u, torch.float64, self.shape),
                                 _ptr(w, torch.float32, (3,) + self.shape), _ptr(out)))
        return out[0]

    def f64_to_df(self, x: torch.Tensor) -> torch.Tensor:
        out = torch.empty(x.shape + (2,), dtype=torch.float32, device=x.device)
        _check(lib().mg_f64_to_df(self._c(), x.numel(), _ptr(x, torch.float64), _ptr(out)))
        return out

    def df_to_f64(self, df: torch.Tensor) -> torch.Tensor:
        out = torch.empty(df.shape[:-1], dtype=torch.float64, device=df.device)
        _check(lib().mg_df_to_f64(self._c(), out.numel(), _ptr(df, torch.float32), _ptr(out)))
        return out

    def df_residual(self, F_df: torch.Tensor, m: float, phi_df: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.shape, dtype=torch.float32, device=F_df.device)
        _check(lib().mg_df_residual(self._c(), _ptr(F_df, torch.float32), float(m), _ptr(phi_df, torch.float32), _ptr(out)))
        return out


class Batch:
    """Independent flat solves of uneven sizes in one persistent launch (mg_batch_*)."""

    def __init__(self, shapes, degree: int = 3, levels: int = 0, coarse_store: str = "fp32"):
        self.solvers = [Solver(s, levels=levels, degree=degree, prec="mixed", fused=False, coarse_store=coarse_store)
                        for s in shapes]
        arr = (_P * len(self.solvers))(*[sv._ctx for sv in self.solvers])
        b = _P()
        _check(lib().mg_batch_create(ctypes.byref(b), arr, len(self.solvers),
                                     torch.cuda.current_stream().cuda_stream))
        self._b = b

    def _ptrs(self, fields, dtype=torch.float64):
        if len(fields) != len(self.solvers):
            raise ValueError("one field per problem expected")
        return (_P * len(fields))(*[_ptr(f, dtype, sv.shape) for f, sv in zip(fields, self.solvers)])

    def autotune(self, sources, phis, tol=1e-6, max_vcycles=50) -> tuple[int, list[int]]:
        """Pick the grid size and the per-level tile sizes by timing solves from the guesses in phis
        (which end up holding the solutions).  Returns (blocks, tiles)."""
        blocks = _I()
        nl = lib().mg_batch_num_levels(self._b)
        tiles = (_I * nl)()
        _check(lib().mg_batch_autotune(self._b, self._ptrs(sources), self._ptrs(phis), float(tol), int(max_vcycles),
                                       ctypes.byref(blocks), tiles))
        return blocks.value, list(tiles)

    def set_blocks(self, blocks: int):
        _check(lib().mg_batch_set_blocks(self._b, int(blocks)))

    def use_graph(self, on: bool = True):
        _check(lib().mg_batch_use_graph(self._b, 1 if on else 0))

    def tiles(self) -> list[int]:
        nl = lib().mg_batch_num_levels(self._b)
        t = (_I * nl)()
        _check(lib().mg_batch_get_tiles(self._b, t, nl))
        return list(t)

    def set_tiles(self, tiles):
        t = (_I * len(tiles))(*[int(x) for x in tiles])
        _check(lib().mg_batch_set_tiles(self._b, t, len(tiles)))

    def solve(self, sources, phis, tol=1e-6, max_vcycles=50):
        """Solve all problems; phis are initial guesses in, solutions out.  Returns (stats, times_ms)."""
        n = len(self.solvers)
        st = (_Stats * n)()
        times = (_D * n)()
        s = lib().mg_batch_solve(self._b, self._ptrs(sources), self._ptrs(phis), float(tol), int(max_vcycles), st, times)
        _check(s, allow_convergence=True)
        return [Stats.from_c(x) for x in st], list(times)

    def close(self):
        if getattr(self, "_b", None):
            lib().mg_batch_destroy(self._b)
            self._b = None
        for sv in getattr(self, "solvers", []):
            sv.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autograd


class MGSolve(torch.autograd.Function):
    """phi = solve(F) for the flat operator; backward: the adjoint solve (same operator)."""

    @staticmethod
    def forward(ctx, F, solver, tol, max_vcycles):
        phi, st = solver.solve(F.detach().contiguous(), tol=tol, max_vcycles=max_vcycles)
        ctx.solver, ctx.tol, ctx.maxv = solver, tol, max_vcycles
        return phi

    @staticmethod
    def backward(ctx, phi_bar):
        src_bar, _, _ = ctx.solver.solve_adjoint(phi_bar.contiguous(), tol=ctx.tol, max_vcycles=ctx.maxv)
        return src_bar, None, None, None


class CurvMGSolve(torch.autograd.Function):
    """phi = solve(delta, psi) for the moving-mesh operator; backward: adjoint solve on
    the exact transpose and the gradient through the geometry (recomputed from psi)."""

    @staticmethod
    def forward(ctx, delta, psi, solver, tol, max_vcycles):
        delta = delta.detach().contiguous()
        psi = psi.detach().contiguous()
        phi, st = solver.solve(delta, tol=tol, max_vcycles=max_vcycles, psi=psi)
        ctx.save_for_backward(delta, psi, phi)
        ctx.solver, ctx.tol, ctx.maxv = solver, tol, max_vcycles
        return phi.clone()

    @staticmethod
    def backward(ctx, phi_bar):
        delta, psi, phi = ctx.saved_tensors
        ctx.solver.set_geometry(psi)
        d_bar, p_bar, _ = ctx.solver.solve_adjoint(phi_bar.contiguous(), phi=phi, source=delta,
                                                   want_psi_bar=ctx.needs_input_grad[1], tol=ctx.tol,
                                                   max_vcycles=ctx.maxv)
        return d_bar, p_bar, None, None, None


class GradDotLoss(torch.autograd.Function):
    """loss = sum(w . grad_h phi) with the library's finite-difference gradient; d loss / d phi = grad_h^T w."""

    @staticmethod
    def forward(ctx, phi, w, solver, order):
        ctx.solver, ctx.order = solver, order
        ctx.save_for_backward(w)
        return solver.grad_dot(phi.detach().contiguous(), w.contiguous(), order)

    @staticmethod
    def backward(ctx, g):
        (w,) = ctx.saved_tensors
        return g * ctx.solver.grad_T(w, ctx.order), None, None, None
