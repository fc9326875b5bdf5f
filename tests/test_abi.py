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
    opt.order, opt.cfl = 4, 2.5  # (1, 2] is accepted, unstable, for the divergence checks
    assert L.wh_create(C.byref(opt), C.byref(h)) == -1
    opt.cfl, opt.resident_blocks = 0.9, -1
    assert L.wh_create(C.byref(opt), C.byref(h)) == -1
    opt.resident_blocks = 0
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


def _desc3(W, g):
    d = W.Grid3Desc()
    for a in range(3):
        d.n[a] = g.n[a]
        d.h[a] = g.h[a]
    for s in range(6):
        d.bc[s] = g.bc[s]
    d.kind, d.ortho, d.instance = g.kind, int(g.ortho), 0
    keep = [np.ascontiguousarray(g.mask, np.int8)]
    d.mask = keep[0].ctypes.data
    if g.rx is not None:
        keep.append(np.ascontiguousarray(g.rx))
        d.rx = keep[-1].ctypes.data
    return d, keep


def _interp3(W, it, **override):
    cols = {k: np.ascontiguousarray(getattr(it, k), np.int32).copy() for k in
            ("recv_grid", "recv_i", "recv_j", "recv_k", "donor_grid", "donor_i0", "donor_j0",
             "donor_k0")}
    cols.update(override)
    ws = [np.ascontiguousarray(getattr(it, k)) for k in ("wx", "wy", "wz")]
    keep = list(cols.values()) + ws
    return W.Interp3Desc(it.n, *[a.ctypes.data for a in keep]), keep


def test_grid3_validation_on_host(W):
    """Three-dimensional grids: order 4 on Cartesian grids only, no mixing with 2D grids,
    Neumann axes must be orthogonal, discretization points may not sit on non-Neumann sides
    or read unused points, and interpolation data must be explicit and complete."""
    from paper_2504_03074_gb300 import grids3 as G3
    L = W.lib()
    gid = C.c_int32()
    cube = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    # order 4: Cartesian grids only, a Neumann face meets no other physical face, every
    # ghost the 13-point stencil reads is filled by a rule, no boundary data
    h = _ctx(W, order=4)
    d, keep = _desc3(W, cube)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0, L.wh_last_error(h)
    gdat = np.ones((9, 9, 9))
    assert L.wh_set_boundary_data(h, 0, gdat.ctypes.data) == -1
    patch = G3.pole_patch_grid("p", 9, 6, 0.5, 0.5, 0.3, 1.0)
    d, keep = _desc3(W, patch)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -1
    neu = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [G.BC_NEUMANN] * 6)
    d, keep = _desc3(W, neu)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -1
    # faces without a rule whose ghosts the stencil of index-1 points would read
    open_box = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [G.BC_NONE] * 6)
    open_box.mask[:] = G.INTERP
    open_box.mask[1:-1, 1:-1, 1:-1] = G.DISC
    d, keep = _desc3(W, open_box)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -7
    L.wh_destroy(h)
    h = _ctx(W, order=2)
    d, keep = _desc3(W, open_box)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0, L.wh_last_error(h)
    L.wh_destroy(h)
    # 2D and 3D grids do not mix
    h = _ctx(W, order=2)
    g2 = G.cartesian_grid("c", 16, 16, 0, 1, 0, 1, [1, 1, 1, 1], 2)
    d2, keep2 = _desc(W, g2)
    assert L.wh_add_grid(h, C.byref(d2), C.byref(gid)) == 0
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -3
    L.wh_destroy(h)
    h = _ctx(W, order=2)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0
    assert L.wh_add_grid(h, C.byref(d2), C.byref(gid)) == -3
    L.wh_destroy(h)
    # a discretization point on a Dirichlet side
    h = _ctx(W, order=2)
    bad = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    bad.mask[0, 4, 4] = G.DISC
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -7
    # a stencil reading an unused point
    bad = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    bad.mask[4, 4, 4] = G.UNUSED
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -7
    # a Neumann side whose normal axis is not orthogonal to the others
    patch = G3.pole_patch_grid("p", 9, 6, 0.5, 0.5, 0.3, 1.0)
    patch.ortho = 4
    d, keep = _desc3(W, patch)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -1
    # unpaired periodic sides, too few points
    bad = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [3, 1, 1, 1, 1, 1])
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -1
    bad = G3.cartesian_grid3("c", (4, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -1
    L.wh_destroy(h)
    # a valid sphere-in-box grid, then interpolation errors
    prob = G3.sphere_problem(nb=48, nphi=64, nth=32, nr=10, npatch=20, width=0.5,
                             r_hole=0.75, patch_deg=30.0, omega=6.0)
    h = _ctx(W, order=2)
    keeps = []
    for g in prob.grids:
        d, keep = _desc3(W, g)
        keeps.append(keep)
        assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0, L.wh_last_error(h)
    it = prob.interp
    ok, keep = _interp3(W, it)
    assert L.wh_set_interp3(h, C.byref(ok)) == 0, L.wh_last_error(h)
    rg = np.ascontiguousarray(it.recv_grid, np.int32).copy()
    rg[0] = 9
    desc, keep = _interp3(W, it, recv_grid=rg)
    assert L.wh_set_interp3(h, C.byref(desc)) == -7
    di = np.ascontiguousarray(it.donor_i0, np.int32).copy()
    sel = np.nonzero(it.donor_grid == 0)[0][0]
    di[sel] = prob.grids[0].n[0] - 2  # stencil leaves the background
    desc, keep = _interp3(W, it, donor_i0=di)
    assert L.wh_set_interp3(h, C.byref(desc)) == -7
    short = W.Interp3Desc(it.n - 1, *[a.ctypes.data for a in _interp3(W, it)[1]])
    assert L.wh_set_interp3(h, C.byref(short)) == -7  # an interpolation point left out
    # 3D contexts: batch, differentiation and tuning calls are state errors
    out = W.Tuning()
    assert L.wh_set_tuning(h, C.byref(W.Tuning(-1, 1, 0, -1, 1, 0.0, 0))) == -3
    assert L.wh_set_coefficient(h, 0, None) == -3
    L.wh_destroy(h)


def test_grid3_order4_validation_on_host(W):
    """Fourth-order 3D host checks: a ghost rule that would read a receiver, a 13-point
    stencil that reaches an unused point two lines away, and a width-5 donor stencil that
    leaves its grid are refused (WH_ERR_GRID); the order-4 box-in-box is taken whole."""
    from paper_2504_03074_gb300 import grids3 as G3
    L = W.lib()
    gid = C.c_int32()
    h = _ctx(W, order=4)
    # a receiver two points inside a Dirichlet face, on the line of a rule's inward points
    bad = G3.cartesian_grid3("c", (12, 12, 12), (0, 0, 0), (1, 1, 1), [G.BC_DIRICHLET] * 6)
    bad.mask[5, 5, 2] = G.INTERP
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -7
    assert b"interpolation point" in L.wh_last_error(h)
    # an unused point behind a layer of receivers, two lines from discretization points
    bad = G3.cartesian_grid3("c", (12, 12, 12), (0, 0, 0), (1, 1, 1), [G.BC_DIRICHLET] * 6)
    bad.mask[5:8, 5:8, 5:8] = G.INTERP
    bad.mask[6, 6, 6] = G.UNUSED
    d, keep = _desc3(W, bad)
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == -7
    assert b"unused" in L.wh_last_error(h)
    L.wh_destroy(h)
    # the order-4 box-in-box: grids and width-5 interpolation taken; a donor corner moved so
    # that its 5-point stencil leaves the donor grid is refused (width 3 would still fit)
    prob = G3.box_in_box_problem(nb=17, ni=15, order=4, hole=0.1)
    h = _ctx(W, order=4)
    keeps = []
    for g in prob.grids:
        d, keep = _desc3(W, g)
        keeps.append(keep)
        assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0, L.wh_last_error(h)
    it = prob.interp
    ok, keep = _interp3(W, it)
    assert L.wh_set_interp3(h, C.byref(ok)) == 0, L.wh_last_error(h)
    di = np.ascontiguousarray(it.donor_i0, np.int32).copy()
    sel = int(np.nonzero(it.donor_grid == 0)[0][0])
    di[sel] = prob.grids[0].n[0] - 4
    desc, keep = _interp3(W, it, donor_i0=di)
    assert L.wh_set_interp3(h, C.byref(desc)) == -7
    L.wh_destroy(h)


def test_deflation_validation_on_host(W):
    """wh_set_deflation checks its arguments without touching the device, on 2D and 3D
    contexts alike."""
    L = W.lib()
    h = _ctx(W, order=2)
    lam = (C.c_double * 2)(1.0, 2.0)
    assert L.wh_set_deflation(h, -1, None, None) == -1
    assert L.wh_set_deflation(h, 2, None, lam) == -1
    assert L.wh_set_deflation(h, 2, C.c_void_p(64), None) == -1
    bad = (C.c_double * 1)(float("nan"))
    assert L.wh_set_deflation(h, 1, C.c_void_p(64), bad) == -1
    assert L.wh_set_deflation(h, 2, C.c_void_p(64), lam) == 0
    assert L.wh_set_deflation(h, 0, None, None) == 0
    L.wh_destroy(h)
    from paper_2504_03074_gb300 import grids3 as G3
    h = _ctx(W, order=2)
    cube = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    d, keep = _desc3(W, cube)
    gid = C.c_int32()
    assert L.wh_add_grid3(h, C.byref(d), C.byref(gid)) == 0
    assert L.wh_set_deflation(h, 2, C.c_void_p(64), bad) == -1
    assert L.wh_set_deflation(h, 2, C.c_void_p(64), lam) == 0
    assert L.wh_set_deflation(h, 0, None, None) == 0
    L.wh_destroy(h)


def test_set_forcing_rejection_leaves_forcing_unchanged(W):
    """A rejected wh_set_forcing (non-finite values) leaves the stored forcing as it was:
    the validation runs before anything is stored (checked through the host-side solve
    preconditions: the context stays usable and reports the same sizes)."""
    L = W.lib()
    prob = G.unit_square_problem(16, 2, 3.0)
    h = _ctx(W, 2)
    d, keep = _desc(W, prob.grids[0])
    gid = C.c_int32()
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == 0
    f = np.ascontiguousarray(prob.f[0], np.float64)
    assert L.wh_set_forcing(h, 0, f.ctypes.data) == 0
    bad = f.copy()
    bad[3, 4] = np.nan
    assert L.wh_set_forcing(h, 0, bad.ctypes.data) == -1
    assert b"non-finite" in L.wh_last_error(h)
    L.wh_destroy(h)


def test_widen_and_probe_arguments(W):
    """The testing and measurement aids refuse bad arguments without a device."""
    L = W.lib()
    assert L.wh_widen_f32(None, None, -1, None) == -1
    assert L.wh_widen_f32(None, None, 5, None) == -1
    assert L.wh_widen_f32(None, None, 0, None) == 0
    t = C.c_double()
    assert L.wh_probe_fp64(0, C.byref(t), None) == -1
    assert L.wh_probe_fp64(3, None, None) == -1


def test_state_validation_on_host(W):
    """wh_get_state / wh_set_state refuse without a stopped solve or a prepared context,
    before any device work."""
    L = W.lib()
    h = _ctx(W, 2)
    n = C.c_size_t(0)
    assert L.wh_get_state(h, None, None) == -1
    assert L.wh_get_state(h, None, C.byref(n)) == -3  # nothing saved
    buf = np.zeros(64, np.uint8)
    assert L.wh_set_state(h, None, 0) == -1
    assert L.wh_set_state(h, buf.ctypes.data, buf.size) == -3  # not prepared
    L.wh_destroy(h)


def test_boundary_data_validation_on_host(W):
    """wh_set_boundary_data checks its arguments without touching the device: a bad grid
    or non-finite data is refused and leaves the context as it was; NULL removes the data;
    order-4 curvilinear grids with a Dirichlet side refuse data; 3D contexts take them."""
    L = W.lib()
    prob = G.unit_square_problem(16, 4, 3.0)
    h = _ctx(W, 4)
    d, keep = _desc(W, prob.grids[0])
    gid = C.c_int32()
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == 0
    good = np.ones(16 * 16)
    bad = good.copy()
    bad[5] = np.nan
    assert L.wh_set_boundary_data(h, 1, good.ctypes.data) == -1
    assert L.wh_set_boundary_data(h, 0, bad.ctypes.data) == -1
    assert L.wh_set_boundary_data(h, 0, good.ctypes.data) == 0
    assert L.wh_set_boundary_data(h, 0, None) == 0
    L.wh_destroy(h)
    A = G.annulus_grid("annulus", 64, 10, 0.5, 0.8, 1.5, 4, inner_bc=G.BC_DIRICHLET)
    h = _ctx(W, 4)
    d, keep = _desc(W, A)
    assert L.wh_add_grid(h, C.byref(d), C.byref(gid)) == 0
    assert L.wh_set_boundary_data(h, 0, np.ones(64 * 10).ctypes.data) == -7
    L.wh_destroy(h)
    from paper_2504_03074_gb300 import grids3 as G3
    h = _ctx(W, order=2)
    cube = G3.cartesian_grid3("c", (9, 9, 9), (0, 0, 0), (1, 1, 1), [1] * 6)
    d3, keep3 = _desc3(W, cube)
    assert L.wh_add_grid3(h, C.byref(d3), C.byref(gid)) == 0
    assert L.wh_set_boundary_data(h, 0, np.ones(9 ** 3).ctypes.data) == 0
    bad3 = np.ones(9 ** 3)
    bad3[7] = np.inf
    assert L.wh_set_boundary_data(h, 0, bad3.ctypes.data) == -1
    assert L.wh_set_boundary_data(h, 1, bad3.ctypes.data) == -1
    L.wh_destroy(h)
