"""CPU oracle for the WaveHoltz hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It wraps the plain C implementation in ``waveholtz_oracle.c``
(one WaveHoltz iteration, FP64, single thread) and adds, in plain numpy:

* the fixed-point iteration of Algorithm 1 (Sec. 2.2) with the scaled residual
  ||r||_2 / sqrt(N) (Sec. 6.1);
* GMRES on A v = b with A v = v - W_h(v, 0) and b = W_h(0, f) (Eqs. WaveHoltzLinearSystem
  and MevalII, Sec. 4.3), restarted, classical Gram-Schmidt applied twice, Givens
  rotations;
* the discrete filter function beta_d by its definition, the trapezoid sum
  (Eq. betad, App. B.3), its three-sinc_d form (Eqs. discreteBetaThreeSincs, sincd) and
  the adjusted alpha_d (Eq. alphadII).

It shares no code with the CUDA library; inputs come from
``paper_2504_03074_gb300.grids`` (which holds none of the method's arithmetic).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "waveholtz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def build(force=False, openmp=False):
    """Compile the C oracle with gcc (plain -O2, no fast-math, no vectorisation flags)."""
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
            vp, ip, dp, cp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_char_p
            L.or_new.restype = vp
            L.or_new.argtypes = [C.c_int]
            L.or_error.restype = cp
            L.or_error.argtypes = [vp]
            L.or_add_grid.restype = C.c_int
            L.or_add_grid.argtypes = [vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, C.c_double,
                                      C.c_double, vp, vp, vp]
            L.or_set_forcing.argtypes = [vp, C.c_int, vp]
            L.or_set_boundary.argtypes = [vp, C.c_int, vp]
            L.or_set_neumann.argtypes = [vp, C.c_int, vp]
            L.or_set_dissipation.restype = C.c_int
            L.or_set_dissipation.argtypes = [vp, C.c_double]
            L.or_set_interp.argtypes = [vp, C.c_long] + [vp] * 8
            L.or_prepare.argtypes = [vp, C.c_double, C.c_double, C.c_int, C.c_int, dp]
            L.or_iterate.restype = C.c_int
            L.or_iterate.argtypes = [vp, C.c_int, vp, vp]
            L.or_apply_lap.argtypes = [vp, C.c_int, vp, vp]
            L.or_apply_bc.argtypes = [vp, C.c_int, vp, C.c_double]
            L.or_get_coef.restype = C.c_int
            L.or_get_coef.argtypes = [vp, C.c_int, C.c_int, vp]
            L.or_interpolate.argtypes = [vp, vp]
            L.or_b_mu.restype = C.c_double
            L.or_b_mu.argtypes = [C.c_int]
            L.or_free.argtypes = [vp]
            if openmp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if openmp else _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class TimeSetup:
    def __init__(self, arr):
        self.dt, self.omega_e, self.alpha = float(arr[0]), float(arr[1]), float(arr[2])
        self.Nt, self.M = int(arr[3]), int(arr[4])
        self.dt_max, self.Tbar = float(arr[5]), float(arr[6])

    def __repr__(self):
        return (f"TimeSetup(dt={self.dt:.8g}, omega_e={self.omega_e:.10g}, "
                f"alpha={self.alpha:.8g}, Nt={self.Nt}, M={self.M})")


class Oracle:
    """One overset Helmholtz problem held by the C oracle."""

    def __init__(self, problem, omega=None, cfl=0.9, periods=1, alpha_mode=0, openmp=False,
                 nu=0.0):
        self.problem = problem
        self.L = lib(openmp)
        self.h = self.L.or_new(problem.order)
        if self.L.or_set_dissipation(self.h, float(nu)) != 0:
            raise ValueError("the dissipation coefficient must be >= 0")
        self._keep = []
        for gi, g in enumerate(problem.grids):
            bc = (C.c_int * 4)(*g.bc)
            mask = np.ascontiguousarray(g.mask, dtype=np.int8)
            rx = None if g.rx is None else np.ascontiguousarray(g.rx, dtype=np.float64)
            c2 = None if problem.c2 is None else np.ascontiguousarray(problem.c2[gi], np.float64)
            self._keep += [mask, rx, c2]
            r = self.L.or_add_grid(self.h, g.n[0], g.n[1], g.kind, bc, int(g.orthogonal),
                                   g.h[0], g.h[1], _p(mask), _p(rx), _p(c2))
            if r < 0:
                raise ValueError(self.L.or_error(self.h).decode())
            f = np.ascontiguousarray(problem.f[gi], np.float64)
            self.L.or_set_forcing(self.h, gi, _p(f))
            gb = getattr(problem, "g", None)
            if gb is not None and gb[gi] is not None:
                ga = np.ascontiguousarray(gb[gi], np.float64)
                self._keep.append(ga)
                self.L.or_set_boundary(self.h, gi, _p(ga))
            gn = getattr(problem, "gn", None)
            if gn is not None and gn[gi] is not None:
                gna = np.ascontiguousarray(gn[gi], np.float64)
                self._keep.append(gna)
                self.L.or_set_neumann(self.h, gi, _p(gna))
        it = problem.interp
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (it.recv_grid, it.recv_i, it.recv_j, it.donor_grid, it.donor_i0, it.donor_j0)]
        ws = [np.ascontiguousarray(a, np.float64) for a in (it.wx, it.wy)]
        self._keep += arrs + ws
        self.L.or_set_interp(self.h, it.n, *[_p(a) for a in arrs + ws])
        self.prepare(problem.omega if omega is None else omega, cfl, periods, alpha_mode)

    def prepare(self, omega, cfl=0.9, periods=1, alpha_mode=0):
        out = (C.c_double * 7)()
        if self.L.or_prepare(self.h, omega, cfl, periods, alpha_mode, out) != 0:
            raise ValueError(self.L.or_error(self.h).decode())
        self.omega = omega
        self.time = TimeSetup(list(out))
        return self.time

    def __del__(self):
        try:
            self.L.or_free(self.h)
        except Exception:
            pass

    # --- the iteration map W_h (Algorithm 1 body) ---
    def iterate(self, v, forcing=True):
        v = np.ascontiguousarray(v, np.float64)
        out = np.empty_like(v)
        if self.L.or_iterate(self.h, 1 if forcing else 0, _p(v), _p(out)) != 0:
            raise RuntimeError("oracle not prepared")
        return out

    def zeros(self):
        return np.zeros(self.problem.n_total)

    def active(self):
        return np.concatenate([(g.mask != 0).ravel() for g in self.problem.grids])

    # --- pieces for pin tests ---
    def ext_shape(self, gi):
        g = self.problem.grids[gi]
        gh = g.ghosts(self.problem.order)
        return (g.n[1] + 2 * gh[1], g.n[0] + 2 * gh[0])

    def apply_lap(self, gi, u_ext):
        u = np.ascontiguousarray(u_ext, np.float64)
        out = np.zeros_like(u)
        self.L.or_apply_lap(self.h, gi, _p(u), _p(out))
        return out

    def apply_bc(self, gi, u_ext, fcos):
        u = np.array(u_ext, np.float64, order="C")
        self.L.or_apply_bc(self.h, gi, _p(u), fcos)
        return u

    def coef(self, gi, which):
        out = np.zeros(self.ext_shape(gi))
        if self.L.or_get_coef(self.h, gi, which, _p(out)) != 0:
            raise ValueError("no coefficients on a Cartesian grid")
        return out

    def interpolate(self, us_ext):
        us = [np.array(u, np.float64, order="C") for u in us_ext]
        ptrs = (C.c_void_p * len(us))(*[u.ctypes.data for u in us])
        self.L.or_interpolate(self.h, ptrs)
        return us


def scaled_norm(r, n_active):
    """||r||_2 / sqrt(N) (Sec. 6.1)."""
    return float(np.linalg.norm(r) / math.sqrt(n_active))


def fpi(orc, iters, v0=None, forcing=True):
    """Algorithm 1: v^{k+1} = W_h(v^k, f); returns the iterates' history."""
    v = orc.zeros() if v0 is None else np.array(v0, np.float64)
    hist, res = [v.copy()], []
    na = orc.problem.n_active
    for _ in range(iters):
        vn = orc.iterate(v, forcing)
        res.append(scaled_norm(vn - v, na))
        v = vn
        hist.append(v.copy())
    return v, hist, res


def gmres(orc, tol=1e-10, restart=60, max_it=400, v0=None):
    """GMRES on (I - S) v = b (Sec. 4.3): b = W_h(0, f), A q = q - W_h(q, 0).

    Stops when ||b - A v||_2 / ||b||_2 <= tol (the residual is recomputed at each
    restart, so the reported value is the true residual at exit).
    """
    b = orc.iterate(orc.zeros(), True)
    v = orc.zeros() if v0 is None else np.array(v0, np.float64)

    def A(q):
        return q - orc.iterate(q, False)

    bnorm = np.linalg.norm(b)
    its, hist = 0, []
    while True:
        r = b - A(v) if np.any(v) else b.copy()
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol or its >= max_it:
            return v, its, hist
        m = restart
        Q = np.zeros((m + 1, r.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[0] = r / beta
        k = 0
        for k in range(m):
            w = A(Q[k])
            its += 1
            for _ in range(2):  # classical Gram-Schmidt, twice
                h = Q[:k + 1] @ w
                w = w - Q[:k + 1].T @ h
                H[:k + 1, k] += h
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                Q[k + 1] = w / H[k + 1, k]
            for i in range(k):  # apply earlier rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) / bnorm <= tol or its >= max_it:
                break
        kk = k + 1
        y = np.zeros(kk)
        for i in range(kk - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:kk] @ y[i + 1:kk]) / H[i, i]
        v = v + Q[:kk].T @ y


# ---------------------------------------------------------------- filter functions

def beta_d_sum(lam, omega, dt, Nt, alpha, periods=1):
    """beta_d(lambda) by the trapezoid sum (Eq. betad), T-bar = periods * Nt * dt."""
    M = periods * Nt
    n = np.arange(M + 1)
    sig = np.ones(M + 1)
    sig[0] = sig[-1] = 0.5
    t = n * dt
    lam = np.atleast_1d(np.asarray(lam, np.float64))
    terms = (np.cos(omega * t) - alpha / 2.0)[None, :] * np.cos(lam[:, None] * t[None, :])
    return (2.0 / (M * dt)) * (terms * sig[None, :]).sum(axis=1) * dt


def sinc_d(z, T, dt):
    """sinc_d(z, T) = sin(z T) / (T tan(z dt/2)/(dt/2)) (Eq. sincd); 1 at z = 0."""
    z = np.asarray(z, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.sin(z * T) / (T * np.tan(z * dt / 2.0) / (dt / 2.0))
    return np.where(z == 0.0, 1.0, out)


def beta_d_sincs(lam, omega, dt, Nt, alpha, periods=1):
    """Three-sinc_d form (Eq. discreteBetaThreeSincs)."""
    T = periods * Nt * dt
    return (sinc_d(omega + lam, T, dt) + sinc_d(omega - lam, T, dt)
            - alpha * sinc_d(lam, T, dt))


def beta_continuous(lam, omega, T, alpha=0.5):
    """Continuous filter function, three-sinc form (Eq. filterThreeSincs)."""
    def sinc(x):
        return np.sinc(np.asarray(x) / np.pi)
    return sinc((omega - lam) * T) + sinc((omega + lam) * T) - alpha * sinc(lam * T)


def alpha_d(omega_e, dt):
    """alpha_d = tan(omega_e dt / 2) / tan(omega_e dt) (Eq. alphad)."""
    return math.tan(omega_e * dt / 2.0) / math.tan(omega_e * dt)


def lambda_tilde(lam_h, dt):
    """Explicit-scheme frequency of a discrete eigenmode (Eq. discreteExplicitLambdaTilde)."""
    return 2.0 / dt * np.arcsin(np.asarray(lam_h) * dt / 2.0)
