"""The C ABI library builds, loads and exports every declared symbol; host-side
validation of grid descriptions works without a GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz
    waveholtz.lib()
    return waveholtz


def _declared():
    hdr = open(os.path.join(ROOT, "include", "waveholtz.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(wh_[a-z_0-9]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(W):
    names = _declared()
    assert len(names) >= 15
    L = C.CDLL(W.lib_path())
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(W.EXPORTS)


def _ctx(W, order=4):
    opt = W.Options()
    W.lib().wh_options_default(C.byref(opt))
    opt.order = order
    h = C.c_void_p()
    assert W.lib().wh_create(C.byref(opt), C.byref(h)) == 0
    return h


def _desc(W, g):
    d = W.GridDesc()
    d.n[0], d.n[1] = g.n
    d.kind = g.kind
    for s in range(4):
        d.bc[s] = g.bc[s]
    d.orthogonal = int(g.orthogonal)
    d.instance = int(getattr(g, "instance", 0))
    d.h[0], d.h[1] = g.h
    keep = [np.ascontiguousarray(g.mask, np.int8)]
    d.mask = keep[0].ctypes.data
    if g.rx is not None:
        keep.append(np.ascontiguousarray(g.rx))
        d.rx = keep[-1].ctypes.data
    return d, keep


def test_options_and_create(W):
    L = W.lib()
    opt = W.Options()
    assert L.wh_options_default(C.byref(opt)) == 0
    assert (opt.order, opt.periods, opt.cfl, opt.alpha_mode, opt.precision) == (4, 1, 0.9, 0, 0)
    h = C.c_void_p()
    opt.order = 3
    assert L.wh_create(C.byref(opt), C.byref(h)) == -1
    opt.order, opt.cfl = 4, 1.5
    assert L.wh_create(C.byref(opt), C.byref(h)) == -1
    assert L.wh_create(None, None) == -1
    L.wh_destroy(None)


def test_tuning_validation_on_host(W):
    """wh_set_tuning checks its fields without touching the device; wh_autotune needs a
    prepared context."""
    L = W.lib()
    opt = W.Options()
    L.wh_options_default(C.byref(opt))
    h = C.c_void_p()
    assert L.wh_create(C.byref(opt), C.byref(h)) == 0
    ok = W.Tuning(-1, 1, 0, -1, 1, 0.0, 0)
    assert L.wh_set_tuning(h, C.byref(ok)) == 0
    for bad in (W.Tuning(-1, 2, 0, 0, 0, 0.0, 0), W.Tuning(-1, 0, -2, 0, 0, 0.0, 0),
                W.Tuning(7, 0, 0, 0, 0, 0.0, 0), W.Tuning(-1, 0, 0, 0, 3, 0.0, 0)):
        assert L.wh_set_tuning(h, C.byref(bad)) == -1
    assert L.wh_set_tuning(h, None) == -1
    out = W.Tuning()
    assert L.wh_autotune(h, 3, C.byref(out)) == -3  # WH_ERR_STATE before wh_prepare
    assert L.wh_autotune(h, 0, C.byref(out)) == -1
    L.wh_destroy(h)


def test_grid_validation_on_host(W):
    L = W.lib()
    h = _ctx(W)
    gid = C.c_int32()
    # Neumann side meeting Dirichlet sides: rejected
    g = G.cartesian_grid("c", 16, 16, 0, 1, 0, 1, [1, 1, 2, 2], 4)
    d, keep = _desc(W, g)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -7
    assert b"Neumann" in L.wh_last_error(h)
    # non-orthogonal grid with a physical side: rejected
    t = G.sheared_torus_grid("t", 16, 16, 0.1, 0.1, 4)
    t.bc = [1, 1, 3, 3]
    d, keep = _desc(W, t)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -7
    # unpaired periodic sides
    g = G.cartesian_grid("c", 16, 16, 0, 1, 0, 1, [3, 1, 1, 1], 4)
    d, keep = _desc(W, g)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -7
    # too small
    g = G.cartesian_grid("c", 6, 16, 0, 1, 0, 1, [1, 1, 1, 1], 4)
    d, keep = _desc(W, g)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -1
    # bad mask value
    g = G.cartesian_grid("c", 16, 16, 0, 1, 0, 1, [1, 1, 1, 1], 4)
    g.mask[3, 3] = 9
    d, keep = _desc(W, g)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -7
    # a valid overset grid
    prob = G.disk_problem(nb=64, nth=128, nr=12, order=4, omega=5.0, width=0.8, r_cut=0.75)
    for g in prob.grids:
        d, keep = _desc(W, g)
        assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == 0
    assert gid.value == 1
    # instance ids must start at 0 and be contiguous
    g = G.cartesian_grid("c", 16, 16, 0, 1, 0, 1, [1, 1, 1, 1], 4)
    g.instance = 3
    d, keep = _desc(W, g)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == -1
    # interpolation with an out-of-range grid index: rejected on the host
    it = prob.interp
    rg = np.ascontiguousarray(it.recv_grid, np.int32).copy()
    rg[0] = 7
    arrs = [rg] + [np.ascontiguousarray(a, np.int32) for a in
                   (it.recv_i, it.recv_j, it.donor_grid, it.donor_i0, it.donor_j0)]
    ws = [np.ascontiguousarray(a) for a in (it.wx, it.wy)]
    desc = W.InterpDesc(it.n, *[a.ctypes.data for a in arrs + ws])
    assert L.wh_set_interp(h, C.byref(desc)) == -7
    # iterate before prepare: state error, no device work
    assert L.wh_iterate(h, 1, C.c_void_p(16), C.c_void_p(32)) == -3
    ti = W.TimeInfo()
    assert L.wh_get_time_info(h, C.byref(ti)) == -3
    L.wh_destroy(h)
