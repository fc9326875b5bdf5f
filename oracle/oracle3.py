"""CPU oracle for the three-dimensional WaveHoltz hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It wraps the plain C implementation in ``waveholtz_oracle3.c`` (one
WaveHoltz iteration on a 3D overset grid at second or fourth order, FP64, single
thread).  The
fixed-point iteration, GMRES and the filter functions of ``oracle.oracle`` apply to it
unchanged (they only call ``iterate``).  It shares no code with the CUDA library; inputs
come from ``paper_2504_03074_gb300.grids3``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .oracle import TimeSetup

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "waveholtz_oracle3.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle3.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle3_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

# coefficient arrays returned by coef(): c^2 a00, a11, a22, a01, a02, a12, b0, b1, b2
COEF_NAMES = ("a00", "a11", "a22", "a01", "a02", "a12", "b0", "b1", "b2")


def build(force=False, openmp=False):
    """Compile the C oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if openmp else _LIB
    extra = ["-fopenmp"] if openmp else []
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib(openmp=False):
    """The oracle library; openmp=True loads the same source built with OpenMP over its
    point loops (the all-cores CPU baseline: same arithmetic per point, same results)."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            L = C.CDLL(build(openmp=openmp))
            vp, dp, cp = C.c_void_p, C.POINTER(C.c_double), C.c_char_p
            L.o3_new.restype = vp
            L.o3_new.argtypes = []
            L.o3_new_order.restype = vp
            L.o3_new_order.argtypes = [C.c_int]
            L.o3_error.restype = cp
            L.o3_error.argtypes = [vp]
            L.o3_add_grid.restype = C.c_int
            L.o3_add_grid.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int,
                                      C.c_double, C.c_double, C.c_double, vp, vp, vp]
            L.o3_set_forcing.argtypes = [vp, C.c_int, vp]
            L.o3_set_boundary.argtypes = [vp, C.c_int, vp]
            L.o3_set_interp.argtypes = [vp, C.c_long] + [vp] * 11
            L.o3_prepare.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, dp]
            L.o3_iterate.restype = C.c_int
            L.o3_iterate.argtypes = [vp, C.c_int, vp, vp]
            L.o3_apply_lap.argtypes = [vp, C.c_int, vp, vp]
            L.o3_apply_bc.argtypes = [vp, C.c_int, vp]
            L.o3_apply_bc_forced.argtypes = [vp, C.c_int, vp, C.c_double]
            L.o3_set_neumann.argtypes = [vp, C.c_int, vp]
            L.o3_set_dissipation.restype = C.c_int
            L.o3_set_dissipation.argtypes = [vp, C.c_double]
            L.o3_get_coef.restype = C.c_int
            L.o3_get_coef.argtypes = [vp, C.c_int, C.c_int, vp]
            L.o3_interpolate.argtypes = [vp, vp]
            L.o3_free.argtypes = [vp]
            if openmp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if openmp else _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle3:
    """One three-dimensional overset Helmholtz problem held by the C oracle."""

    def __init__(self, problem, omega=None, cfl=0.9, periods=1, alpha_mode=0, openmp=False,
                 nu=0.0):
        """nu > 0 turns on the dissipative march (the upwind-dissipation variant: the
        deviation of the march from the iterate's periodic motion is damped, so that the
        discrete Helmholtz solution stays the fixed point)."""
        self.problem = problem
        self.L = lib(openmp)
        self.order = int(getattr(problem, "order", 2))
        self.h = self.L.o3_new_order(self.order)
        if not self.h:
            raise ValueError(f"order {self.order}: the 3D oracle takes 2 or 4")
        if self.L.o3_set_dissipation(self.h, float(nu)) != 0:
            raise ValueError("the dissipation coefficient must be >= 0")
        self._keep = []
        for gi, g in enumerate(problem.grids):
            bc = (C.c_int * 6)(*g.bc)
            mask = np.ascontiguousarray(g.mask, dtype=np.int8)
            rx = None if g.rx is None else np.ascontiguousarray(g.rx, dtype=np.float64)
            c2 = None if problem.c2 is None else np.ascontiguousarray(problem.c2[gi], np.float64)
            self._keep += [mask, rx, c2]
            r = self.L.o3_add_grid(self.h, g.n[0], g.n[1], g.n[2], g.kind, bc, int(g.ortho),
                                   g.h[0], g.h[1], g.h[2], _p(mask), _p(rx), _p(c2))
            if r < 0:
                raise ValueError(self.L.o3_error(self.h).decode())
            f = np.ascontiguousarray(problem.f[gi], np.float64)
            self.L.o3_set_forcing(self.h, gi, _p(f))
            gb = getattr(problem, "g", None)
            if gb is not None and gb[gi] is not None:
                ga = np.ascontiguousarray(gb[gi], np.float64)
                self._keep.append(ga)
                self.L.o3_set_boundary(self.h, gi, _p(ga))
            gnn = getattr(problem, "gn", None)
            if gnn is not None and gnn[gi] is not None:
                ga = np.ascontiguousarray(gnn[gi], np.float64)
                self._keep.append(ga)
                self.L.o3_set_neumann(self.h, gi, _p(ga))
        it = problem.interp
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (it.recv_grid, it.recv_i, it.recv_j, it.recv_k, it.donor_grid, it.donor_i0,
                 it.donor_j0, it.donor_k0)]
        ws = [np.ascontiguousarray(a, np.float64) for a in (it.wx, it.wy, it.wz)]
        self._keep += arrs + ws
        self.L.o3_set_interp(self.h, it.n, *[_p(a) for a in arrs + ws])
        self.prepare(problem.omega if omega is None else omega, cfl, periods, alpha_mode)

    def prepare(self, omega, cfl=0.9, periods=1, alpha_mode=0):
        out = (C.c_double * 7)()
        if self.L.o3_prepare(self.h, omega, cfl, periods, alpha_mode, out) != 0:
            raise ValueError(self.L.o3_error(self.h).decode())
        self.omega = omega
        self.time = TimeSetup(list(out))
        return self.time

    def __del__(self):
        try:
            self.L.o3_free(self.h)
        except Exception:
            pass

    def iterate(self, v, forcing=True):
        v = np.ascontiguousarray(v, np.float64)
        out = np.empty_like(v)
        if self.L.o3_iterate(self.h, 1 if forcing else 0, _p(v), _p(out)) != 0:
            raise RuntimeError("oracle not prepared")
        return out

    def zeros(self):
        return np.zeros(self.problem.n_total)

    def active(self):
        return np.concatenate([(g.mask != 0).ravel() for g in self.problem.grids])

    # --- pieces for pin tests (extended arrays, shape (e2, e1, e0)) ---
    def ext_shape(self, gi):
        g = self.problem.grids[gi]
        gh = g.ghosts(self.order)
        return tuple(g.n[a] + 2 * gh[a] for a in (2, 1, 0))

    def apply_lap(self, gi, u_ext):
        u = np.ascontiguousarray(u_ext, np.float64)
        out = np.zeros_like(u)
        self.L.o3_apply_lap(self.h, gi, _p(u), _p(out))
        return out

    def apply_bc(self, gi, u_ext, fcos=0.0):
        """The ghost rules of grid gi on a copy of u_ext, with forcing factor fcos."""
        u = np.array(u_ext, np.float64, order="C")
        self.L.o3_apply_bc_forced(self.h, gi, _p(u), float(fcos))
        return u

    def coef(self, gi, which):
        out = np.zeros(self.ext_shape(gi))
        w = COEF_NAMES.index(which) if isinstance(which, str) else which
        if self.L.o3_get_coef(self.h, gi, w, _p(out)) != 0:
            raise ValueError("no coefficients on a Cartesian grid")
        return out

    def interpolate(self, us_ext):
        us = [np.array(u, np.float64, order="C") for u in us_ext]
        ptrs = (C.c_void_p * len(us))(*[u.ctypes.data for u in us])
        self.L.o3_interpolate(self.h, ptrs)
        return us
