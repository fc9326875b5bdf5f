"""Thin ctypes binding to libwaveholtz (C ABI: ``include/waveholtz.h``).

Argument marshalling only: every step of a WaveHoltz iteration runs in the library's
CUDA kernels.  PyTorch provides device memory and the stream.  There is no CPU path:
if the shared library cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import grids as G

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libwaveholtz.so")
_lib = None

WH_OK = 0
STATUS = {0: "WH_OK", -1: "WH_ERR_ARG", -2: "WH_ERR_CUDA", -3: "WH_ERR_STATE",
          -4: "WH_ERR_DIVERGED", -5: "WH_ERR_TIMEOUT", -6: "WH_ERR_NOT_CONVERGED",
          -7: "WH_ERR_GRID", -8: "WH_ERR_NOMEM"}
FP64, FP32 = 0, 1
FPI, GMRES = 0, 1
PERSISTENT, GRAPH = 0, 1


class WHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("order", C.c_int32), ("periods", C.c_int32), ("cfl", C.c_double),
                ("alpha_mode", C.c_int32), ("precision", C.c_int32), ("launch_mode", C.c_int32),
                ("barrier_spin_limit", C.c_uint64), ("trajectory_bytes", C.c_uint64),
                ("resident_blocks", C.c_int32)]


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int32 * 2), ("kind", C.c_int32), ("bc", C.c_int32 * 4),
                ("orthogonal", C.c_int32), ("instance", C.c_int32), ("h", C.c_double * 2),
                ("mask", C.c_void_p),
                ("rx", C.c_void_p), ("c2", C.c_void_p)]


class InterpDesc(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in
                                     ("recv_grid", "recv_i", "recv_j", "donor_grid", "donor_i0",
                                      "donor_j0", "wx", "wy")]


class Grid3Desc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("kind", C.c_int32), ("bc", C.c_int32 * 6),
                ("ortho", C.c_int32), ("instance", C.c_int32), ("h", C.c_double * 3),
                ("mask", C.c_void_p), ("rx", C.c_void_p), ("c2", C.c_void_p)]


class Interp3Desc(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in
                                     ("recv_grid", "recv_i", "recv_j", "recv_k", "donor_grid",
                                      "donor_i0", "donor_j0", "donor_k0", "wx", "wy", "wz")]


class TimeInfo(C.Structure):
    _fields_ = [("omega", C.c_double), ("dt", C.c_double), ("omega_e", C.c_double),
                ("alpha", C.c_double), ("dt_max", C.c_double), ("Tbar", C.c_double),
                ("Nt", C.c_int32), ("M", C.c_int32), ("n_active", C.c_int64),
                ("n_total", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("launch_mode", C.c_int32), ("fold_gather", C.c_int32),
                ("tile_tickets", C.c_int32), ("tma", C.c_int32), ("pdl", C.c_int32),
                ("ms_per_iteration", C.c_double), ("candidates", C.c_int32),
                ("temporal_depth", C.c_int32), ("unit_depth", C.c_int32),
                ("blocked_points", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("residual", C.c_double),
                ("seconds", C.c_double), ("n_history", C.c_int32), ("products_fp64", C.c_int32),
                ("products_fp32", C.c_int32)]


EXPORTS = ["wh_options_default", "wh_create", "wh_destroy", "wh_last_error", "wh_set_stream",
           "wh_add_grid", "wh_set_interp", "wh_set_forcing", "wh_set_boundary_data",
           "wh_prepare", "wh_iterate",
           "wh_iterate_host", "wh_solve", "wh_dot", "wh_get_time_info", "wh_last_launch_count",
           "wh_profile_kernels", "wh_multidot_noalloc", "wh_prepare_batch", "wh_solve_batch", "wh_apply_adjoint", "wh_adjoint",
           "wh_set_coefficient", "wh_set_tuning", "wh_autotune", "wh_add_grid3",
           "wh_set_interp3", "wh_set_deflation", "wh_widen_f32", "wh_probe_fp64",
           "wh_get_tuning", "wh_set_deflation_basis", "wh_eigs", "wh_dense_eig",
           "wh_dense_invariant", "wh_get_state", "wh_set_state"]


def lib_path():
    return _LIB_PATH


def lib():
    """Load libwaveholtz.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libwaveholtz.so not built ({_LIB_PATH}); run "
                           "paper_2504_03074_gb300.build.build() -- there is no CPU fallback")
    L = C.CDLL(_LIB_PATH)
    vp, st = C.c_void_p, C.c_int
    L.wh_options_default.argtypes = [C.POINTER(Options)]
    L.wh_create.argtypes = [C.POINTER(Options), C.POINTER(vp)]
    L.wh_destroy.argtypes = [vp]
    L.wh_destroy.restype = None
    L.wh_last_error.argtypes = [vp]
    L.wh_last_error.restype = C.c_char_p
    L.wh_set_stream.argtypes = [vp, vp]
    L.wh_add_grid.argtypes = [vp, C.POINTER(GridDesc), C.POINTER(C.c_int32)]
    L.wh_set_interp.argtypes = [vp, C.POINTER(InterpDesc)]
    L.wh_add_grid3.argtypes = [vp, C.POINTER(Grid3Desc), C.POINTER(C.c_int32)]
    L.wh_set_interp3.argtypes = [vp, C.POINTER(Interp3Desc)]
    L.wh_set_deflation.argtypes = [vp, C.c_int32, vp, vp]
    L.wh_set_forcing.argtypes = [vp, C.c_int32, vp]
    L.wh_set_boundary_data.argtypes = [vp, C.c_int32, vp]
    L.wh_prepare.argtypes = [vp, C.c_double, C.POINTER(TimeInfo)]
    L.wh_prepare_batch.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(TimeInfo)]
    L.wh_iterate.argtypes = [vp, C.c_int32, vp, vp]
    L.wh_iterate_host.argtypes = [vp, C.c_int32, vp, vp]
    L.wh_solve.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, vp,
                           C.POINTER(Stats), vp, C.c_int32]
    L.wh_dot.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(C.c_double)]
    L.wh_solve_batch.argtypes = [vp, C.c_double, C.c_int32, C.c_int32, vp, C.POINTER(Stats)]
    L.wh_apply_adjoint.argtypes = [vp, vp, vp]
    L.wh_adjoint.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32, vp, vp, vp,
                             C.POINTER(Stats)]
    L.wh_set_coefficient.argtypes = [vp, C.c_int32, vp]
    L.wh_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.wh_autotune.argtypes = [vp, C.c_int32, C.POINTER(Tuning)]
    L.wh_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.wh_set_deflation_basis.argtypes = [vp, C.c_int32, vp, vp]
    L.wh_eigs.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                          C.c_uint64, vp, vp, vp, vp, C.POINTER(Stats)]
    L.wh_dense_eig.argtypes = [C.c_int32, vp, vp, vp]
    L.wh_dense_invariant.argtypes = [C.c_int32, vp, C.c_int32, vp, C.POINTER(C.c_int32)]
    L.wh_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.wh_set_state.argtypes = [vp, vp, C.c_size_t]
    L.wh_get_time_info.argtypes = [vp, C.POINTER(TimeInfo)]
    L.wh_multidot_noalloc.argtypes = [vp, C.c_int64, C.c_int32, vp, C.c_int64, vp, vp]
    L.wh_profile_kernels.argtypes = [vp, C.c_int32, C.POINTER(C.c_double),
                                     C.POINTER(C.c_int32)]
    L.wh_widen_f32.argtypes = [vp, vp, C.c_int64, vp]
    L.wh_probe_fp64.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wh_last_launch_count.argtypes = [vp]
    L.wh_last_launch_count.restype = C.c_int64
    for name in EXPORTS:
        if name not in ("wh_destroy", "wh_last_error", "wh_last_launch_count"):
            getattr(L, name).restype = st
    _lib = L
    return L


def probe_fp64(reps=5):
    """The device's FP64 FMA throughput (TFLOP/s, FMA = 2 FLOP) and the best launch's ms."""
    t, ms = C.c_double(), C.c_double()
    st = lib().wh_probe_fp64(reps, C.byref(t), C.byref(ms))
    if st != WH_OK:
        raise WHError(st, "wh_probe_fp64 failed")
    return t.value, ms.value


def widen_f32(x, out, stream=None):
    """out = FP64 of the float32 device tensor x by the library's integer widening."""
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().wh_widen_f32(_ptr(x), _ptr(out), x.numel(), C.c_void_p(raw))
    if st != WH_OK:
        raise WHError(st, "wh_widen_f32 failed")
    return out


def dense_eig(A):
    """Eigenvalues and unit eigenvectors (columns) of a small real matrix by the library's
    host routine (the one wh_eigs uses): (w, V) complex numpy arrays."""
    A = np.ascontiguousarray(A, np.float64)
    m = A.shape[0]
    w = np.zeros(2 * m)
    V = np.zeros(2 * m * m)
    st = lib().wh_dense_eig(m, _ptr(A), _ptr(w), _ptr(V))
    if st != WH_OK:
        raise WHError(st, "wh_dense_eig failed")
    return w[0::2] + 1j * w[1::2], (V[0::2] + 1j * V[1::2]).reshape(m, m)


def invariant_basis(A, want):
    """Real orthonormal basis (columns) of the invariant subspace of the `want` eigenvalues
    of largest modulus of a small real matrix, by the library's host routine; returns
    (Q, p)."""
    A = np.ascontiguousarray(A, np.float64)
    m = A.shape[0]
    Q = np.zeros(m * (want + 1))
    p = C.c_int32()
    st = lib().wh_dense_invariant(m, _ptr(A), want, _ptr(Q), C.byref(p))
    if st != WH_OK:
        raise WHError(st, "wh_dense_invariant failed")
    return Q[:m * p.value].reshape(p.value, m).T.copy(), p.value


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


class Solver:
    """One overset Helmholtz problem in libwaveholtz (one context)."""

    def __init__(self, problem, periods=1, cfl=0.9, alpha_mode=0, precision=FP64, stream=None,
                 launch_mode=GRAPH, barrier_spin_limit=0, trajectory_bytes=0,
                 resident_blocks=0):
        gn = getattr(problem, "gn", None)
        if gn is not None and any(x is not None and np.any(x != 0) for x in gn):
            raise ValueError("the library takes no Neumann data (dU/dn != 0)")
        self.L = lib()
        self.problem = problem
        opt = Options()
        self.L.wh_options_default(C.byref(opt))
        opt.order, opt.periods, opt.cfl = problem.order, periods, cfl
        opt.alpha_mode, opt.precision = alpha_mode, precision
        opt.launch_mode, opt.barrier_spin_limit = launch_mode, barrier_spin_limit
        opt.trajectory_bytes = trajectory_bytes
        opt.resident_blocks = resident_blocks
        h = C.c_void_p()
        self._check(self.L.wh_create(C.byref(opt), C.byref(h)), None)
        self.h = h
        # The library works on one CUDA stream: a dedicated torch stream unless the caller
        # names one.  Each call is ordered after the caller's current stream and the
        # caller's stream is ordered after the call (no host synchronisation).
        import torch
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.set_stream(self.stream)
        if getattr(problem, "dim", 2) == 3:
            self._add_3d(problem)
            self.info = None
            return
        for gi, g in enumerate(problem.grids):
            mask = np.ascontiguousarray(g.mask, np.int8)
            rx = None if g.rx is None else np.ascontiguousarray(g.rx, np.float64)
            c2 = None if problem.c2 is None else np.ascontiguousarray(problem.c2[gi], np.float64)
            d = GridDesc()
            d.n[0], d.n[1] = g.n
            d.kind = g.kind
            for s in range(4):
                d.bc[s] = g.bc[s]
            d.orthogonal = int(g.orthogonal)
            d.instance = int(getattr(g, "instance", 0))
            d.h[0], d.h[1] = g.h
            d.mask, d.rx, d.c2 = _ptr(mask), _ptr(rx), _ptr(c2)
            gid = C.c_int32()
            self._check(self.L.wh_add_grid(self.h, C.byref(d), C.byref(gid)))
            f = np.ascontiguousarray(problem.f[gi], np.float64)
            self._check(self.L.wh_set_forcing(self.h, gid.value, _ptr(f)))
            gb = getattr(problem, "g", None)
            if gb is not None and gb[gi] is not None:
                ga = np.ascontiguousarray(gb[gi], np.float64)
                self._check(self.L.wh_set_boundary_data(self.h, gid.value, _ptr(ga)))
        it = problem.interp
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (it.recv_grid, it.recv_i, it.recv_j, it.donor_grid, it.donor_i0, it.donor_j0)]
        ws = [np.ascontiguousarray(a, np.float64) for a in (it.wx, it.wy)]
        d = InterpDesc(it.n, *[_ptr(a) for a in arrs + ws])
        self._check(self.L.wh_set_interp(self.h, C.byref(d)))
        self.info = None

    def _add_3d(self, problem):
        """Three-dimensional grids and interpolation (``grids3.Problem3``)."""
        for gi, g in enumerate(problem.grids):
            mask = np.ascontiguousarray(g.mask, np.int8)
            rx = None if g.rx is None else np.ascontiguousarray(g.rx, np.float64)
            c2 = None if problem.c2 is None else np.ascontiguousarray(problem.c2[gi], np.float64)
            d = Grid3Desc()
            for a in range(3):
                d.n[a] = g.n[a]
                d.h[a] = g.h[a]
            for s in range(6):
                d.bc[s] = g.bc[s]
            d.kind, d.ortho, d.instance = g.kind, int(g.ortho), 0
            d.mask, d.rx, d.c2 = _ptr(mask), _ptr(rx), _ptr(c2)
            gid = C.c_int32()
            self._check(self.L.wh_add_grid3(self.h, C.byref(d), C.byref(gid)))
            f = np.ascontiguousarray(problem.f[gi], np.float64)
            self._check(self.L.wh_set_forcing(self.h, gid.value, _ptr(f)))
            gb = getattr(problem, "g", None)
            if gb is not None and gb[gi] is not None:
                ga = np.ascontiguousarray(gb[gi], np.float64)
                self._check(self.L.wh_set_boundary_data(self.h, gid.value, _ptr(ga)))
        it = problem.interp
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (it.recv_grid, it.recv_i, it.recv_j, it.recv_k, it.donor_grid, it.donor_i0,
                 it.donor_j0, it.donor_k0)]
        ws = [np.ascontiguousarray(a, np.float64) for a in (it.wx, it.wy, it.wz)]
        d = Interp3Desc(it.n, *[_ptr(a) for a in arrs + ws])
        self._check(self.L.wh_set_interp3(self.h, C.byref(d)))

    def _check(self, status, h=0):
        if status != WH_OK:
            msg = "" if h is None else self.L.wh_last_error(self.h).decode()
            raise WHError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.wh_destroy(self.h)
            self.h = None

    __del__ = close

    def set_stream(self, stream):
        """Issue work on a torch.cuda.Stream."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.L.wh_set_stream(self.h, C.c_void_p(raw)))
        self.stream = stream

    def _enter(self):
        self.stream.wait_stream(self._torch.cuda.current_stream())

    def _leave(self):
        self._torch.cuda.current_stream().wait_stream(self.stream)

    def prepare(self, omega=None):
        """Prepare one frequency (a list: one per instance of a batch); returns the time
        setup (a list of them for a batch)."""
        om = self.problem.omega if omega is None else omega
        if isinstance(om, (list, tuple, np.ndarray)):
            k = len(om)
            arr = (C.c_double * k)(*[float(x) for x in om])
            infos = (TimeInfo * k)()
            self._check(self.L.wh_prepare_batch(self.h, arr, infos))
            self.infos = list(infos)
            self.info = self.infos[0]
            return self.infos
        ti = TimeInfo()
        self._check(self.L.wh_prepare(self.h, om, C.byref(ti)))
        self.info = ti
        self.infos = [ti]
        return ti

    @property
    def n_total(self):
        return self.problem.n_total

    def iterate(self, v_in, v_out, forcing=True):
        """v_out = W_h(v_in, f or 0): device tensors (float64, n_total, contiguous)."""
        self._enter()
        self._check(self.L.wh_iterate(self.h, 1 if forcing else 0, _ptr(v_in), _ptr(v_out)))
        self._leave()
        return v_out

    def iterate_host(self, v_in, forcing=True):
        """Host numpy in, host numpy out (copies inside the call)."""
        v = np.ascontiguousarray(v_in, np.float64)
        out = np.empty_like(v)
        self._enter()
        self._check(self.L.wh_iterate_host(self.h, 1 if forcing else 0, _ptr(v), _ptr(out)))
        return out

    def iterate_host_buffers(self, v_in, v_out, forcing=True):
        """Same with caller-owned (e.g. pinned torch CPU) buffers."""
        self._enter()
        self._check(self.L.wh_iterate_host(self.h, 1 if forcing else 0, _ptr(v_in), _ptr(v_out)))
        return v_out

    def solve(self, u, method=GMRES, tol=1e-8, max_it=500, restart=50, history_cap=2000):
        """Solve in place on device tensor u (initial guess in, solution out)."""
        st = Stats()
        hist = np.zeros(max(history_cap, 1))
        self._enter()
        status = self.L.wh_solve(self.h, method, tol, max_it, restart, _ptr(u), C.byref(st),
                                 _ptr(hist), history_cap)
        self._leave()
        if status not in (WH_OK, -6):
            self._check(status)
        st.history = hist[:st.n_history].copy()
        st.status = STATUS.get(status, status)
        return st

    def set_deflation(self, phi=None, lam2=None):
        """Deflation set of FPI solves (Algorithm 3): phi a contiguous float64 CUDA tensor of
        shape (k, n_total) with orthonormal rows (kept by reference: keep it alive and
        unchanged), lam2 the k eigenvalues lambda_m^2; None removes the set."""
        if phi is None:
            self._check(self.L.wh_set_deflation(self.h, 0, None, None))
            self._defl = None
            return
        lam = np.ascontiguousarray(lam2, np.float64)
        assert phi.is_cuda and phi.is_contiguous() and phi.shape[0] == lam.size
        self._check(self.L.wh_set_deflation(self.h, int(lam.size), _ptr(phi), _ptr(lam)))
        self._defl = (phi, lam)

    def get_state(self):
        """The state of the last solve that stopped at max_it, as bytes (wh_get_state)."""
        n = C.c_size_t(0)
        self._check(self.L.wh_get_state(self.h, None, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        self._check(self.L.wh_get_state(self.h, _ptr(buf), C.byref(n)))
        return buf.tobytes()

    def set_state(self, state):
        """Load a saved solve (bytes from get_state); the next solve() continues it."""
        buf = np.frombuffer(state, np.uint8).copy()
        self._check(self.L.wh_set_state(self.h, _ptr(buf), buf.size))

    def set_deflation_basis(self, Q, T):
        """Deflation with an S-invariant orthonormal basis Q (contiguous float64 CUDA tensor
        (k, n_total), kept by reference) and its Rayleigh matrix T = Q S Q^T (k x k host
        array): the exact inflation of wh_set_deflation_basis."""
        Tm = np.ascontiguousarray(T, np.float64)
        assert Q.is_cuda and Q.is_contiguous() and Q.shape[0] == Tm.shape[0] == Tm.shape[1]
        self._check(self.L.wh_set_deflation_basis(self.h, int(Q.shape[0]), _ptr(Q), _ptr(Tm)))
        self._defl = (Q, Tm)

    def eigs(self, k, m=0, tol=1e-10, max_products=5000, passes=2, seed=0):
        """Deflation eigenpairs on the GPU (wh_eigs): returns (Q, T, beta, lambda2, stats);
        Q a (k, n_total) CUDA tensor.  A run that ends at max_products returns with
        stats.converged == 0 instead of raising."""
        torch = self._torch
        Q = torch.zeros((k, self.problem.n_total), dtype=torch.float64, device="cuda")
        T = np.zeros((k, k))
        beta = np.zeros(k)
        lam2 = np.zeros(k)
        st = Stats()
        self._enter()
        status = self.L.wh_eigs(self.h, k, m, tol, max_products, passes, seed, _ptr(Q), _ptr(T),
                                _ptr(beta), _ptr(lam2), C.byref(st))
        self._leave()
        if status not in (WH_OK, -6):
            self._check(status)
        st.status = STATUS.get(status, status)
        return Q, T, beta, lam2, st

    def solve_batch(self, u, tol=1e-8, max_it=500, restart=50):
        """Batched solve of every instance in place on device tensor u; list of Stats."""
        k = len(self.infos)
        st = (Stats * k)()
        self._enter()
        status = self.L.wh_solve_batch(self.h, tol, max_it, restart, _ptr(u), st)
        self._leave()
        if status not in (WH_OK, -6):
            self._check(status)
        out = list(st)
        for x in out:
            x.status = STATUS.get(status, status)
        return out

    def apply_adjoint(self, w_in, w_out):
        """w_out = S^T w_in (device tensors)."""
        self._enter()
        self._check(self.L.wh_apply_adjoint(self.h, _ptr(w_in), _ptr(w_out)))
        self._leave()
        return w_out

    def adjoint(self, u, g, tol=1e-10, max_it=1000, restart=200):
        """Adjoint solve and gradients for dJ/du = g at solution u (device tensors):
        returns (lam, grad_c2, grad_f, stats).  Like solve(), an adjoint GMRES that stops
        above tol returns with stats.converged == 0 (the gradients are then those of the
        last lam) instead of raising."""
        torch = self._torch
        lam = torch.zeros_like(u)
        gc2 = torch.zeros_like(u)
        gf = torch.zeros_like(u)
        st = Stats()
        self._enter()
        status = self.L.wh_adjoint(self.h, _ptr(u), _ptr(g), tol, max_it, restart, _ptr(lam),
                                   _ptr(gc2), _ptr(gf), C.byref(st))
        self._leave()
        if status not in (WH_OK, -6):
            self._check(status)
        st.status = STATUS.get(status, status)
        return lam, gc2, gf, st

    def set_coefficient(self, gid, c2):
        """Replace c(x)^2 of one grid (host array or None); re-run prepare() afterwards."""
        arr = None if c2 is None else np.ascontiguousarray(c2, np.float64)
        self._check(self.L.wh_set_coefficient(self.h, gid, _ptr(arr)))

    def set_forcing(self, gid, f):
        """Replace the forcing of one grid (host array); re-run prepare() afterwards."""
        arr = np.ascontiguousarray(f, np.float64)
        self._check(self.L.wh_set_forcing(self.h, gid, _ptr(arr)))

    def set_boundary_data(self, gid, g):
        """Dirichlet data of one grid (host array, or None to remove); re-run prepare()."""
        arr = None if g is None else np.ascontiguousarray(g, np.float64)
        self._check(self.L.wh_set_boundary_data(self.h, gid, _ptr(arr)))

    def dot(self, x, y):
        out = C.c_double()
        self._enter()
        self._check(self.L.wh_dot(self.h, _ptr(x), _ptr(y), x.numel(), C.byref(out)))
        return out.value

    def set_tuning(self, launch_mode=-1, fold_gather=-1, tile_tickets=-1, tma=-1, pdl=-1,
                   temporal_depth=-1, unit_depth=-1):
        """Fix the launch layout (-1: the library's choice); see wh_tuning."""
        t = Tuning(launch_mode, fold_gather, tile_tickets, tma, pdl, 0.0, 0, temporal_depth,
                   unit_depth, 0)
        self._check(self.L.wh_set_tuning(self.h, C.byref(t)))

    def get_tuning(self):
        """The launch layout in use (after prepare) as a dict."""
        t = Tuning()
        self._check(self.L.wh_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def autotune(self, reps=3):
        """Time every valid launch layout on the prepared problem and keep the fastest;
        returns it as a dict (launch_mode, fold_gather, tile_tickets, tma, pdl,
        ms_per_iteration, candidates)."""
        t = Tuning()
        self._enter()
        status = self.L.wh_autotune(self.h, reps, C.byref(t))
        self._leave()
        self._check(status)
        return t.as_dict()

    def profile_kernels(self, reps=50):
        """Average device ms per launch and launches per iteration of each kernel:
        dict(march=(ms, n), bc_gather=(ms, n), init=(ms, n), finish=(ms, n))."""
        ms = (C.c_double * 4)()
        cnt = (C.c_int32 * 4)()
        self._enter()
        self._check(self.L.wh_profile_kernels(self.h, reps, ms, cnt))
        names = ("march", "bc_gather", "init", "finish")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(names)}

    def last_launch_count(self):
        return int(self.L.wh_last_launch_count(self.h))


_autograd_fn = None


def _waveholtz_fn():
    """torch.autograd.Function for u = WaveHoltz fixed point of (c^2, f) (built on first use)."""
    global _autograd_fn
    if _autograd_fn is not None:
        return _autograd_fn
    import torch

    class WaveHoltzFixedPoint(torch.autograd.Function):
        @staticmethod
        def forward(fctx, c2, f, owner):
            owner._load(c2, f)
            u = torch.zeros(owner.problem.n_total, dtype=torch.float64, device=c2.device)
            st = owner.solver.solve(u, GMRES, owner.tol, owner.max_it, owner.restart)
            if not st.converged:
                raise WHError(-6, f"forward solve stopped at residual {st.residual:.3e}")
            owner.forward_stats = st
            fctx.owner = owner
            fctx.save_for_backward(c2, f, u)
            return u

        @staticmethod
        def backward(fctx, gu):
            owner = fctx.owner
            c2, f, u = fctx.saved_tensors
            owner._load(c2, f)
            g = gu.detach().to(torch.float64).contiguous()
            _, gc2, gf, st = owner.solver.adjoint(u, g, owner.adj_tol, owner.max_it,
                                                  owner.restart)
            if not st.converged:
                raise WHError(-6, f"adjoint solve stopped at residual {st.residual:.3e}")
            owner.adjoint_stats = st
            return (gc2 if fctx.needs_input_grad[0] else None,
                    gf if fctx.needs_input_grad[1] else None, None)

    _autograd_fn = WaveHoltzFixedPoint
    return _autograd_fn


class DifferentiableSolve:
    """u(c^2, f): the converged WaveHoltz solution as a differentiable torch function.

    ``c2`` and ``f`` are compact float64 device tensors (n_total, every grid point, the
    values at non-discretization points are ignored).  The forward pass loads them into one
    library context, prepares the time setup and runs GMRES on (I - S) v = b; the backward
    pass runs the adjoint GMRES on (I - S^T) lam = dJ/du and the checkpointed reverse sweep
    (``wh_adjoint``), which returns dJ/dc^2 and dJ/df of the discrete map.  The fixed point
    is the discrete Helmholtz solution at omega whatever the time step (the explicit
    omega-tilde recipe makes 4/dt^2 sin^2(omega-tilde dt/2) = omega^2), so the gradient is
    that of the discrete Helmholtz solution, although dt itself moves with max c^2."""

    def __init__(self, problem, tol=1e-12, adj_tol=None, max_it=1000, restart=200, **solver_kw):
        self.problem = problem
        self.solver = Solver(problem, **solver_kw)
        self.tol, self.max_it, self.restart = tol, max_it, restart
        self.adj_tol = tol if adj_tol is None else adj_tol
        self._loaded = None
        self.forward_stats = self.adjoint_stats = None

    def _load(self, c2, f):
        key = (c2.data_ptr(), c2._version, f.data_ptr(), f._version)
        if key == self._loaded:
            return
        c2h = c2.detach().to("cpu", self.solver._torch.float64).numpy()
        fh = f.detach().to("cpu", self.solver._torch.float64).numpy()
        for gi, (cg, fg) in enumerate(zip(self.problem.split(c2h), self.problem.split(fh))):
            self.solver.set_coefficient(gi, cg)
            self.solver.set_forcing(gi, fg)
        self.solver.prepare()
        self._loaded = key

    def __call__(self, c2, f):
        return _waveholtz_fn().apply(c2, f, self)

    def close(self):
        self.solver.close()
