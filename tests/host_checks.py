"""Feeds a 2D problem's grid descriptions and interpolation data through the library's
host-side validation (wh_create, wh_add_grid, wh_set_interp) without device work."""
import ctypes as C

import numpy as np


def library_takes(problem):
    """Asserts that the library's host checks take every grid and the interpolation data
    of ``problem`` (a 2D grids.Problem)."""
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    L = W.lib()
    opt = W.Options()
    L.wh_options_default(C.byref(opt))
    opt.order = problem.order
    h = C.c_void_p()
    assert L.wh_create(C.byref(opt), C.byref(h)) == 0
    try:
        keep, gid = [], C.c_int32()
        for g in problem.grids:
            d = W.GridDesc()
            d.n[0], d.n[1] = g.n
            d.kind = g.kind
            for s in range(4):
                d.bc[s] = g.bc[s]
            d.orthogonal, d.instance = int(g.orthogonal), 0
            d.h[0], d.h[1] = g.h
            keep.append(np.ascontiguousarray(g.mask, np.int8))
            d.mask = keep[-1].ctypes.data
            if g.rx is not None:
                keep.append(np.ascontiguousarray(g.rx))
                d.rx = keep[-1].ctypes.data
            assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == 0, L.wh_last_error(h)
        it = problem.interp
        arrs = [np.ascontiguousarray(a, np.int32) for a in
                (it.recv_grid, it.recv_i, it.recv_j, it.donor_grid, it.donor_i0, it.donor_j0)]
        arrs += [np.ascontiguousarray(a) for a in (it.wx, it.wy)]
        desc = W.InterpDesc(it.n, *[a.ctypes.data for a in arrs])
        assert L.wh_set_interp(h, C.byref(desc)) == 0, L.wh_last_error(h)
    finally:
        L.wh_destroy(h)


def library_status3(problem):
    """Feeds a 3D problem (grids3.Problem3) through wh_add_grid3 and wh_set_interp3;
    returns the first nonzero status with its message, or (0, "")."""
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    L = W.lib()
    opt = W.Options()
    L.wh_options_default(C.byref(opt))
    opt.order = problem.order
    h = C.c_void_p()
    assert L.wh_create(C.byref(opt), C.byref(h)) == 0
    try:
        keep, gid = [], C.c_int32()
        for g in problem.grids:
            d = W.Grid3Desc()
            for a in range(3):
                d.n[a] = g.n[a]
                d.h[a] = g.h[a]
            for s in range(6):
                d.bc[s] = g.bc[s]
            d.kind, d.ortho, d.instance = g.kind, int(g.ortho), 0
            keep.append(np.ascontiguousarray(g.mask, np.int8))
            d.mask = keep[-1].ctypes.data
            if g.rx is not None:
                keep.append(np.ascontiguousarray(g.rx))
                d.rx = keep[-1].ctypes.data
            st = L.wh_add_grid3(h, C.byref(d), C.byref(gid))
            if st != 0:
                return st, L.wh_last_error(h)
        it = problem.interp
        cols = [np.ascontiguousarray(getattr(it, k), np.int32) for k in
                ("recv_grid", "recv_i", "recv_j", "recv_k", "donor_grid", "donor_i0",
                 "donor_j0", "donor_k0")]
        cols += [np.ascontiguousarray(getattr(it, k)) for k in ("wx", "wy", "wz")]
        desc = W.Interp3Desc(it.n, *[a.ctypes.data for a in cols])
        st = L.wh_set_interp3(h, C.byref(desc))
        return (st, L.wh_last_error(h)) if st != 0 else (0, "")
    finally:
        L.wh_destroy(h)
