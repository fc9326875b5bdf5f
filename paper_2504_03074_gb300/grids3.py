"""Seeded synthetic three-dimensional overset grids: the stand-in for the
paper's grid generator (Ogen, Sec. 3.1) in 3D.

It builds component grids from analytic mappings x = G_g(r) -- an axis-aligned Cartesian
box, a spherical shell (periodic in azimuth, a polar band), and orthographic pole patches
-- cuts the hole of the background, classifies points as discretization / interpolation /
unused, finds 3 x 3 x 3 donor stencils (5 x 5 x 5 for the fourth-order Cartesian
problems the CPU oracle takes; explicit interpolation: donors are discretization or
Dirichlet points only) and their tensor-product Lagrange weights (Sec. 3.1), and
evaluates Gaussian sources (Eq. gaussianSource).  Like ``grids`` it holds none of the
WaveHoltz arithmetic: its outputs are the input data that both the CUDA library and the
CPU oracle consume.

Array conventions:

* a grid has ``n = (n0, n1, n2)`` points along parameter axes 0, 1, 2 (boundary points
  included, ghosts excluded; a periodic axis lists each point once);
* compact per-grid arrays have shape ``(n2, n1, n0)`` in C order (axis 0 fastest);
* the ghost width is p/2 on non-periodic axes (order p) and 0 on periodic ones; extended arrays
  (metrics) have shape ``(n2 + 2 g2, n1 + 2 g1, n0 + 2 g0)``;
* sides are ``[axis0-lo, axis0-hi, axis1-lo, axis1-hi, axis2-lo, axis2-hi]``;
* ``ortho`` is a bit mask of orthogonal axis pairs: bit 0 = (0, 1), bit 1 = (0, 2),
  bit 2 = (1, 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .grids import (BC_DIRICHLET, BC_NEUMANN, BC_NONE, BC_PERIODIC, CARTESIAN, CURVILINEAR,
                    DIRICHLET, DISC, INTERP, UNUSED, lagrange_weights)

ORDER = 2  # default order; 4 is taken on Cartesian grids (library and oracle)
_EPS = 1e-9  # index-space tolerance of "inside a grid" (points on a shared boundary)


@dataclass
class Grid3:
    """One component grid of a three-dimensional overset grid (Sec. 3.1)."""

    name: str
    kind: int
    n: tuple                      # (n0, n1, n2)
    bc: list                      # 6 side codes
    h: tuple                      # Cartesian: physical spacing; curvilinear: parameter spacing
    mask: np.ndarray              # int8 (n2, n1, n0)
    ortho: int = 7                # orthogonal axis pairs (bit mask)
    rx: np.ndarray | None = None  # float64 (9, e2, e1, e0): rx[3k + m] = dr_k / dx_m
    origin: tuple = (0.0, 0.0, 0.0)
    mapping: dict = field(default_factory=dict)

    def ghosts(self, order=ORDER):
        return tuple(0 if self.bc[2 * a] == BC_PERIODIC else order // 2 for a in range(3))

    @property
    def npts(self):
        return self.n[0] * self.n[1] * self.n[2]

    def coords(self, k=None):
        """Physical coordinates (3, n2, n1, n0), or of the plane k only (3, n1, n0)."""
        ks = np.arange(self.n[2]) if k is None else np.array([k])
        t = [np.arange(self.n[0]) * self.h[0], np.arange(self.n[1]) * self.h[1],
             ks * self.h[2]]
        T0, T1, T2 = np.meshgrid(t[0], t[1], t[2], indexing="ij")
        T0, T1, T2 = (np.ascontiguousarray(np.transpose(a, (2, 1, 0))) for a in (T0, T1, T2))
        out = self.mapping["map"](T0, T1, T2)
        return out if k is None else out[:, 0]

    def param(self, x, y, z):
        """Fractional point indices (fi, fj, fk) of physical points, and a mask of the
        points the mapping covers."""
        return self.mapping["inverse"](x, y, z)


@dataclass
class Interp3:
    """Receiver k of grid recv_grid at (recv_i, recv_j, recv_k) takes
    sum_{a,b,c} wx[k,a] wy[k,b] wz[k,c] u_donor(i0 + a, j0 + b, k0 + c)."""

    recv_grid: np.ndarray
    recv_i: np.ndarray
    recv_j: np.ndarray
    recv_k: np.ndarray
    donor_grid: np.ndarray
    donor_i0: np.ndarray
    donor_j0: np.ndarray
    donor_k0: np.ndarray
    wx: np.ndarray
    wy: np.ndarray
    wz: np.ndarray

    @property
    def n(self):
        return int(self.recv_grid.shape[0])

    @staticmethod
    def empty():
        z = np.zeros(0, np.int32)
        w = np.zeros((0, 3))
        return Interp3(z, z, z, z, z, z, z, z, w, w, w)


@dataclass
class Problem3:
    """c^2 Lap u + omega^2 u = f on a three-dimensional overset grid (Eq. HelmholtzBVP)."""

    grids: list
    interp: Interp3
    omega: float
    f: list                       # per-grid compact forcing (n2, n1, n0)
    c2: list | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)
    order: int = ORDER
    dim: int = 3
    g: list | None = None         # per-grid compact Dirichlet data (read at Dirichlet points)
    gn: list | None = None        # per-grid compact Neumann data du/dn (outward normal), read
                                  # at the discretization points of Neumann faces

    @property
    def n_active(self):
        return int(sum(int(np.count_nonzero(g.mask != UNUSED)) for g in self.grids))

    @property
    def n_total(self):
        return int(sum(g.npts for g in self.grids))

    def split(self, vec):
        out, o = [], 0
        for g in self.grids:
            out.append(vec[o:o + g.npts].reshape(g.n[2], g.n[1], g.n[0]))
            o += g.npts
        return out


# ----------------------------------------------------------------------------------
# Component grids
# ----------------------------------------------------------------------------------

def cartesian_grid3(name, n, lo, hi, bc):
    """Axis-aligned box [lo, hi] with n[a] points per axis; Dirichlet sides marked."""
    h = tuple((hi[a] - lo[a]) / (n[a] - 1) for a in range(3))
    mask = np.full((n[2], n[1], n[0]), DISC, np.int8)
    sl = [np.s_[:, :, 0], np.s_[:, :, -1], np.s_[:, 0, :], np.s_[:, -1, :],
          np.s_[0, :, :], np.s_[-1, :, :]]
    for s, code in enumerate(bc):
        if code == BC_DIRICHLET:
            mask[sl[s]] = DIRICHLET
    lo = tuple(float(v) for v in lo)

    def fmap(t0, t1, t2):
        return np.stack([lo[0] + t0, lo[1] + t1, lo[2] + t2])

    def inv(x, y, z):
        fi, fj, fk = (x - lo[0]) / h[0], (y - lo[1]) / h[1], (z - lo[2]) / h[2]
        ok = ((fi >= -_EPS) & (fi <= n[0] - 1 + _EPS) & (fj >= -_EPS) &
              (fj <= n[1] - 1 + _EPS) & (fk >= -_EPS) & (fk <= n[2] - 1 + _EPS))
        return fi, fj, fk, ok

    # Cartesian parameters are physical offsets: coords() maps t -> lo + t
    g = Grid3(name, CARTESIAN, tuple(n), list(bc), h, mask, 7, None, lo)
    g.mapping = dict(map=fmap, inverse=inv)
    return g


def shell_grid(name, nphi, nth, nr, r_in, width, th_lo_deg, th_hi_deg, order=ORDER):
    """Spherical shell x = r (sin th cos phi, sin th sin phi, cos th).

    Axis 0: phi = 2 pi t0 (periodic, nphi points), axis 1: th = th_lo + (th_hi - th_lo) t1
    (nth points), axis 2: r = r_in + width t2 (nr points).  Side axis2-lo is the sphere
    (Neumann); the polar edges and the outer shell are interpolation points.  All three
    pairs of grid lines are orthogonal.  Metrics are analytic and also evaluated on the
    ghost lines (order/2 of them); the interpolation layers are order/2 points thick.
    """
    gw = order // 2
    th0, th1 = math.radians(th_lo_deg), math.radians(th_hi_deg)
    d0, d1, d2 = 1.0 / nphi, 1.0 / (nth - 1), 1.0 / (nr - 1)
    dth = th1 - th0

    def fmap(t0, t1, t2):
        ph, th, r = 2 * np.pi * t0, th0 + dth * t1, r_in + width * t2
        return np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph),
                         r * np.cos(th)])

    def inv(x, y, z):
        r = np.sqrt(x * x + y * y + z * z)
        ph = np.mod(np.arctan2(y, x), 2 * np.pi)
        th = np.arccos(np.clip(z / np.maximum(r, 1e-300), -1.0, 1.0))
        fi = ph / (2 * np.pi) * nphi
        fj = (th - th0) / dth * (nth - 1)
        fk = (r - r_in) / width * (nr - 1)
        ok = (fj >= -_EPS) & (fj <= nth - 1 + _EPS) & (fk >= -_EPS) & (fk <= nr - 1 + _EPS)
        return fi, fj, fk, ok

    # inverse metrics on the extended extent (no ghosts on the periodic axis 0)
    t0 = np.arange(nphi) * d0
    t1 = np.arange(-gw, nth + gw) * d1
    t2 = np.arange(-gw, nr + gw) * d2
    T2, T1, T0 = np.meshgrid(t2, t1, t0, indexing="ij")
    ph, th, r = 2 * np.pi * T0, th0 + dth * T1, r_in + width * T2
    sp, cp, st, ct = np.sin(ph), np.cos(ph), np.sin(th), np.cos(th)
    rx = np.empty((9,) + T0.shape)
    # grad phi = (-sin phi, cos phi, 0) / (r sin th);  t0 = phi / (2 pi)
    rx[0], rx[1], rx[2] = -sp / (r * st) / (2 * np.pi), cp / (r * st) / (2 * np.pi), 0.0
    # grad th = (cos th cos phi, cos th sin phi, -sin th) / r;  t1 = (th - th0) / dth
    rx[3], rx[4], rx[5] = ct * cp / r / dth, ct * sp / r / dth, -st / r / dth
    # grad r = (sin th cos phi, sin th sin phi, cos th);  t2 = (r - r_in) / width
    rx[6], rx[7], rx[8] = st * cp / width, st * sp / width, ct / width
    mask = np.full((nr, nth, nphi), DISC, np.int8)
    mask[:, :gw, :] = INTERP
    mask[:, -gw:, :] = INTERP
    mask[-gw:, :, :] = INTERP
    bc = [BC_PERIODIC, BC_PERIODIC, BC_NONE, BC_NONE, BC_NEUMANN, BC_NONE]
    g = Grid3(name, CURVILINEAR, (nphi, nth, nr), bc, (d0, d1, d2), mask, 7, rx)
    g.mapping = dict(map=fmap, inverse=inv, r_in=r_in, width=width, th=(th0, th1))
    return g


def pole_patch_grid(name, na, nr, A, r_in, width, sign, order=ORDER):
    """Orthographic pole patch x = r (a, b, sign sqrt(1 - a^2 - b^2)), a, b in [-A, A].

    Axes 0, 1: a, b (na points each), axis 2: r = r_in + width t2 (nr points).  Side
    axis2-lo is the sphere (Neumann); the four (a, b) edges and the outer layer are
    interpolation points.  The radial lines are orthogonal to the (a, b) surfaces (pairs
    (0, 2) and (1, 2)); a and b lines are not (the mixed a-b term is present).  Ghost
    lines and interpolation layers are order/2 deep, as for the shell.
    """
    gw = order // 2
    d0 = d1 = 1.0 / (na - 1)
    d2 = 1.0 / (nr - 1)

    def fmap(t0, t1, t2):
        a, b, r = -A + 2 * A * t0, -A + 2 * A * t1, r_in + width * t2
        return np.stack([r * a, r * b, sign * r * np.sqrt(1.0 - a * a - b * b)])

    def inv(x, y, z):
        r = np.sqrt(x * x + y * y + z * z)
        rs = np.maximum(r, 1e-300)
        a, b = x / rs, y / rs
        fi = (a + A) / (2 * A) * (na - 1)
        fj = (b + A) / (2 * A) * (na - 1)
        fk = (r - r_in) / width * (nr - 1)
        ok = ((sign * z > 0) & (fi >= -_EPS) & (fi <= na - 1 + _EPS) & (fj >= -_EPS) &
              (fj <= na - 1 + _EPS) & (fk >= -_EPS) & (fk <= nr - 1 + _EPS))
        return fi, fj, fk, ok

    t = np.arange(-gw, na + gw) * d0
    t2 = np.arange(-gw, nr + gw) * d2
    T2, T1, T0 = np.meshgrid(t2, t, t, indexing="ij")
    a, b, r = -A + 2 * A * T0, -A + 2 * A * T1, r_in + width * T2
    c = sign * np.sqrt(1.0 - a * a - b * b)  # unit vector s = (a, b, c)
    rx = np.empty((9,) + T0.shape)
    # grad a = (e_x - a s) / r, grad b = (e_y - b s) / r, grad r = s
    rx[0], rx[1], rx[2] = (1 - a * a) / r, -a * b / r, -a * c / r
    rx[3], rx[4], rx[5] = -a * b / r, (1 - b * b) / r, -b * c / r
    rx[0:3] /= 2 * A
    rx[3:6] /= 2 * A
    rx[6], rx[7], rx[8] = a / width, b / width, c / width
    mask = np.full((nr, na, na), DISC, np.int8)
    mask[:, :, :gw] = INTERP
    mask[:, :, -gw:] = INTERP
    mask[:, :gw, :] = INTERP
    mask[:, -gw:, :] = INTERP
    mask[-gw:, :, :] = INTERP
    bc = [BC_NONE, BC_NONE, BC_NONE, BC_NONE, BC_NEUMANN, BC_NONE]
    g = Grid3(name, CURVILINEAR, (na, na, nr), bc, (d0, d1, d2), mask, 6, rx)
    g.mapping = dict(map=fmap, inverse=inv, A=A, sign=sign, r_in=r_in, width=width)
    return g


def cylinder_shell_grid(name, nth, nr, nz, r_in, r_out, lz, bc_in, bc_out, order=ORDER,
                        beta=0.0):
    """Annular cylinder x = r (cos th, sin th), z: axis 0 th = 2 pi t0 (periodic, nth
    points), axis 1 r = r_in + (r_out - r_in) q(t1) (nr points, stretched toward r_out by
    beta > 0), axis 2 z = lz t2 (periodic, nz points).  Sides axis1-lo / -hi (r_in, r_out)
    carry bc_in / bc_out (Dirichlet, Neumann or an interpolation face); all pairs of grid
    lines are orthogonal.  Metrics are analytic, on order/2 ghost lines too; a face with
    BC_NONE has order/2 interpolation layers."""
    gw = order // 2
    d0, d1, d2 = 1.0 / nth, 1.0 / (nr - 1), 1.0 / nz
    w = r_out - r_in
    eb = math.expm1(beta) if beta else 0.0

    def q(t):
        return t if not beta else 1.0 - np.expm1(beta * (1.0 - t)) / eb

    def dq(t):
        return np.ones_like(t) if not beta else beta * np.exp(beta * (1.0 - t)) / eb

    def fmap(t0, t1, t2):
        th, r = 2 * np.pi * t0, r_in + w * q(t1)
        return np.stack([r * np.cos(th), r * np.sin(th), lz * np.asarray(t2) + 0.0 * th])

    def inv(x, y, z):
        r = np.hypot(x, y)
        th = np.mod(np.arctan2(y, x), 2 * np.pi)
        u = (r - r_in) / w
        with np.errstate(invalid="ignore", divide="ignore"):
            t1 = u if not beta else 1.0 - np.log1p(eb * (1.0 - u)) / beta
        fk = np.mod(z / lz, 1.0) * nz
        ok = (t1 >= -_EPS) & (t1 <= 1.0 + _EPS)
        return th / (2 * np.pi) * nth, t1 * (nr - 1), fk, ok

    t0 = np.arange(nth) * d0
    t1 = np.arange(-gw, nr + gw) * d1
    t2 = np.arange(nz) * d2
    T2, T1, T0 = np.meshgrid(t2, t1, t0, indexing="ij")
    th, r = 2 * np.pi * T0, r_in + w * q(T1)
    rx = np.zeros((9,) + T0.shape)
    # grad th = (-sin th, cos th, 0) / r, t0 = th / (2 pi); grad r = (cos th, sin th, 0),
    # t1 = q^{-1}((r - r_in) / w); t2 = z / lz
    rx[0], rx[1] = -np.sin(th) / r / (2 * np.pi), np.cos(th) / r / (2 * np.pi)
    rx[3], rx[4] = np.cos(th) / (w * dq(T1)), np.sin(th) / (w * dq(T1))
    rx[8] = 1.0 / lz
    mask = np.full((nz, nr, nth), DISC, np.int8)
    for code, sl in ((bc_in, np.s_[:, :gw, :]), (bc_out, np.s_[:, -gw:, :])):
        if code == BC_NONE:
            mask[sl] = INTERP
    if bc_in == BC_DIRICHLET:
        mask[:, 0, :] = DIRICHLET
    if bc_out == BC_DIRICHLET:
        mask[:, -1, :] = DIRICHLET
    bc = [BC_PERIODIC, BC_PERIODIC, bc_in, bc_out, BC_PERIODIC, BC_PERIODIC]
    g = Grid3(name, CURVILINEAR, (nth, nr, nz), bc, (d0, d1, d2), mask, 7, rx)
    g.mapping = dict(map=fmap, inverse=inv, r_in=r_in, r_out=r_out, lz=lz)
    return g


def pipe(j=2, order=ORDER, radius=0.5, lz=1.0, wfac=None, wmax=0.3, cut=0.5, shift=1):
    """The paper's solid pipe (Sec. 6): the inside of a cylinder of the given radius,
    periodic in z over [0, lz), Dirichlet on the curved wall; target spacing h = 1/(10 j).
    A Cartesian background over [-radius, radius]^2 x [0, lz) (periodic in z) with the
    points beyond r_cut = r_in + cut W cut out (those within order/2 index layers of an
    active point become interpolation points), and a cylindrical shell of width
    W = min(wfac h, wmax) along the wall (r_in = radius - W; inner order/2 layers
    interpolated from the background; the wall Dirichlet).  Donor stencils of width
    order + 1 hold discretization or Dirichlet points only: centred stencils need a shell
    about 12 h wide at order 4 (wfac defaults to 8 at order 2, 12 at order 4, so j >= 3
    there under the cap); with ``shift`` > 0 (default 1) off-centred stencils, moved by
    up to that many points per axis, are taken where centred ones are not valid, which
    makes order 4 on the coarsest grid (j = 2, shell 6 h wide) possible.
    Returns (grids, interp)."""
    h = 1.0 / (10 * j)
    if wfac is None:
        wfac = 8.0 if order == 2 else 12.0
    W = min(wfac * h, wmax)
    r_in = radius - W
    w = order + 1
    nxy = int(round(2 * radius / h)) + 1
    nz = int(round(lz / h))
    B = cartesian_grid3("background", (nxy, nxy, nz), (-radius, -radius, 0.0),
                        (radius, radius, lz * (nz - 1) / nz),
                        [BC_NONE, BC_NONE, BC_NONE, BC_NONE, BC_PERIODIC, BC_PERIODIC])
    nth = int(round(2 * np.pi * radius / h))
    nr = int(round(W / h)) + 1
    S = cylinder_shell_grid("shell", nth, nr, nz, r_in, radius, lz, BC_NONE, BC_DIRICHLET,
                            order)
    x = -radius + B.h[0] * np.arange(nxy)
    rr = np.hypot(x[None, :], x[:, None])
    outside = np.broadcast_to(rr > r_in + cut * W, (nz, nxy, nxy)).copy()
    near = _near(~outside, order // 2)
    B.mask[outside & near] = INTERP
    B.mask[outside & ~near] = UNUSED
    grids = [B, S]
    parts = []
    for rgid, donors in ((0, (1,)), (1, (0,))):
        g = grids[rgid]
        ijk = _interp_points(g)
        pts = _points_of(g, ijk)
        dg, c, f = find_donors(grids, rgid, pts, donors, w, shift)
        parts.append((rgid, ijk, dg, c, f))
    interp = _assemble(grids, parts, w)
    check_explicit_interp3(grids, interp)
    return grids, interp


def pipe_problem(j=2, order=ORDER, omega=8.5, source=(0.1, 0.1, 0.5), amp=150.0, b=10.0,
                 **kw):
    """The pipe with the paper's Gaussian source (amplitude 150, exponent 10, centred at
    (0.1, 0.1, 0.5))."""
    grids, interp = pipe(j, order, **kw)
    x0 = np.array(source, np.float64)
    f = [gaussian3(g, x0, amp, b) for g in grids]
    return Problem3(grids, interp, omega, f, name=f"pipe-j{j}-o{order}",
                    meta=dict(source=list(source)), order=order)


def with_neumann_data3(problem, grad):
    """The same problem with Neumann data on every Neumann face: gn = grad u . n at its
    discretization points, n the outward unit normal (-+ grad r_a / |grad r_a| from the
    inverse metrics on a low / high face of axis a; the axis direction on Cartesian grids),
    grad(x, y, z) -> (u_x, u_y, u_z) the gradient of the intended solution."""
    import copy
    p = copy.copy(problem)
    p.gn = []
    for g in problem.grids:
        gn = np.zeros(g.mask.shape)
        gh = g.ghosts(problem.order)
        X = g.coords()
        for s in range(6):
            if g.bc[s] != BC_NEUMANN:
                continue
            a, hi = s // 2, s % 2
            sl = [slice(None)] * 3
            sl[2 - a] = -1 if hi else 0
            sl = tuple(sl)
            pts = g.mask[sl] == DISC
            if g.kind == CARTESIAN:
                nv = [np.full(pts.shape, 1.0 if m == a else 0.0) for m in range(3)]
            else:
                rx = g.rx[:, gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]
                nv = [rx[3 * a + m][sl] for m in range(3)]
                nrm = np.sqrt(nv[0] ** 2 + nv[1] ** 2 + nv[2] ** 2)
                nv = [v / nrm for v in nv]
            du = grad(X[0][sl], X[1][sl], X[2][sl])
            sign = 1.0 if hi else -1.0
            if np.any(pts & (gn[sl] != 0.0)):
                raise ValueError("Neumann data where two Neumann faces meet (one value per "
                                 "point cannot hold both normals)")
            gn[sl] = np.where(pts, sign * (du[0] * nv[0] + du[1] * nv[1] + du[2] * nv[2]), 0.0)
        p.gn.append(gn)
    p.name = problem.name + "-gn"
    return p


def annular_cylinder_problem(nth=32, nr=9, nz=10, r_in=0.3, r_out=0.6, lz=1.0,
                             bc_in=BC_DIRICHLET, bc_out=BC_DIRICHLET, order=ORDER,
                             omega=5.0, seed=0, b=40.0):
    """One closed curvilinear grid (periodic in th and z): a Gaussian source seeded in the
    annulus."""
    rng = np.random.default_rng(seed)
    g = cylinder_shell_grid("annulus", nth, nr, nz, r_in, r_out, lz, bc_in, bc_out, order)
    rr, th, z = rng.uniform(r_in + 0.3 * (r_out - r_in), r_out - 0.3 * (r_out - r_in)), \
        rng.uniform(0, 2 * np.pi), rng.uniform(0.3, 0.7) * lz
    x0 = np.array([rr * np.cos(th), rr * np.sin(th), z])
    return Problem3([g], Interp3.empty(), omega, [gaussian3(g, x0, 1.0, b)],
                    name=f"annular-cylinder-{nth}x{nr}x{nz}-o{order}",
                    meta=dict(source=x0.tolist(), seed=seed), order=order)


# ----------------------------------------------------------------------------------
# Donor search (explicit interpolation)
# ----------------------------------------------------------------------------------

def _stencil(g, fi, fj, fk, w=3):
    """Lower corners of the w-point stencils nearest (fi, fj, fk), shifted inside."""
    f = [fi, fj, fk]
    c = []
    for a in range(3):
        i0 = np.rint(f[a]).astype(np.int64) - w // 2
        if g.bc[2 * a] == BC_PERIODIC:
            i0 = np.mod(i0, g.n[a])
        else:
            i0 = np.clip(i0, 0, g.n[a] - w)
        c.append(i0)
    return c


def _valid(g, c, w=3):
    """True where all w^3 stencil points are discretization or Dirichlet points."""
    ok = np.ones(c[0].shape, bool)
    for dc in range(w):
        for db in range(w):
            for da in range(w):
                ii = [c[0] + da, c[1] + db, c[2] + dc]
                for a in range(3):
                    if g.bc[2 * a] == BC_PERIODIC:
                        ii[a] = np.mod(ii[a], g.n[a])
                m = g.mask[ii[2], ii[1], ii[0]]
                ok &= (m == DISC) | (m == DIRICHLET)
    return ok


def _shifts(s):
    """Stencil offsets d in {-s..s}^3 other than 0, nearest first (by |d|_1, then |d|_inf)."""
    r = range(-s, s + 1)
    ds = [(a, b, c) for c in r for b in r for a in r if (a, b, c) != (0, 0, 0)]
    return sorted(ds, key=lambda d: (sum(map(abs, d)), max(map(abs, d))))


def find_donors(grids, recv_gid, pts, order_of_donors, w=3, shift=0):
    """Donor stencils of width w for receivers of grid ``recv_gid`` at physical points
    pts (3, N), trying donor grids in the given order; raises if a receiver has no valid
    stencil.  With shift > 0 a receiver whose centred stencil touches a point that is not
    a discretization or Dirichlet point takes the nearest valid stencil moved by up to
    ``shift`` points per axis (off-centred Lagrange interpolation, same width)."""
    N = pts.shape[1]
    out_g = np.full(N, -1, np.int32)
    out_c = np.zeros((3, N), np.int64)
    out_f = np.zeros((3, N))
    for dgid in order_of_donors:
        todo = np.nonzero(out_g < 0)[0]
        if todo.size == 0:
            break
        g = grids[dgid]
        fi, fj, fk, ok = g.param(pts[0, todo], pts[1, todo], pts[2, todo])
        sel = np.nonzero(ok)[0]
        if sel.size == 0:
            continue
        c = _stencil(g, fi[sel], fj[sel], fk[sel], w)
        v = _valid(g, c, w)
        for d in (_shifts(shift) if shift > 0 else ()):
            if np.all(v):
                break
            bad = np.nonzero(~v)[0]
            cs = []
            for a in range(3):
                ca = c[a][bad] + d[a]
                if g.bc[2 * a] == BC_PERIODIC:
                    ca = np.mod(ca, g.n[a])
                else:
                    ca = np.clip(ca, 0, g.n[a] - w)
                cs.append(ca)
            vb = _valid(g, cs, w)
            for a in range(3):
                c[a][bad[vb]] = cs[a][vb]
            v[bad[vb]] = True
        take = todo[sel[v]]
        out_g[take] = dgid
        for a, fa in enumerate((fi, fj, fk)):
            out_c[a, take] = c[a][v]
            frac = fa[sel[v]] - c[a][v]
            if g.bc[2 * a] == BC_PERIODIC:  # distance along the periodic axis from i0
                frac = np.mod(frac + w // 2, g.n[a]) - w // 2
            out_f[a, take] = frac
    if np.any(out_g < 0):
        k = int(np.nonzero(out_g < 0)[0][0])
        raise ValueError(f"receiver {k} of grid {recv_gid} at {pts[:, k]} has no donor")
    return out_g, out_c, out_f


def check_explicit_interp3(grids, it):
    """Every donor is a discretization or Dirichlet point; receivers are INTERP points."""
    w = it.wx.shape[1]
    rg = it.recv_grid
    for gid, g in enumerate(grids):
        sel = rg == gid
        m = g.mask[it.recv_k[sel], it.recv_j[sel], it.recv_i[sel]]
        if not np.all(m == INTERP):
            raise ValueError(f"grid {gid}: a receiver is not an interpolation point")
        if int(np.count_nonzero(g.mask == INTERP)) != int(np.count_nonzero(sel)):
            raise ValueError(f"grid {gid}: interpolation points and receivers differ")
    for gid, g in enumerate(grids):
        sel = it.donor_grid == gid
        if not np.any(sel):
            continue
        c = [it.donor_i0[sel].astype(np.int64), it.donor_j0[sel].astype(np.int64),
             it.donor_k0[sel].astype(np.int64)]
        for a in range(3):
            if g.bc[2 * a] != BC_PERIODIC and (c[a].min() < 0 or c[a].max() > g.n[a] - w):
                raise ValueError(f"donor stencil outside grid {gid}")
        if not np.all(_valid(g, c, w)):
            raise ValueError(f"grid {gid}: a donor stencil touches a non-discretization point")


def _assemble(grids, parts, w=3):
    """Concatenate (recv_gid, ijk (3, N), donor g (N), corner (3, N), frac (3, N)) with
    width-w Lagrange weights."""
    cols = [[] for _ in range(11)]
    for rgid, ijk, dg, c, f in parts:
        n = ijk.shape[1]
        cols[0].append(np.full(n, rgid, np.int32))
        for a in range(3):
            cols[1 + a].append(ijk[a].astype(np.int32))
        cols[4].append(dg.astype(np.int32))
        for a in range(3):
            cols[5 + a].append(c[a].astype(np.int32))
        for a in range(3):
            cols[8 + a].append(lagrange_weights(f[a], w))
    arrs = [np.concatenate(c) for c in cols]
    return Interp3(*arrs)


def _interp_points(g):
    k, j, i = np.nonzero(g.mask == INTERP)
    return np.stack([i, j, k])


def _points_of(g, ijk):
    """Physical coordinates of the listed points of g."""
    t = [ijk[a] * g.h[a] for a in range(3)]
    return g.mapping["map"](t[0].astype(np.float64), t[1].astype(np.float64),
                            t[2].astype(np.float64))


# ----------------------------------------------------------------------------------
# Overset grids
# ----------------------------------------------------------------------------------

def sphere_in_box(nb=320, nphi=256, nth=128, nr=24, npatch=96, box=2.0, r_in=0.5,
                  width=0.3, band=(15.0, 165.0), patch_deg=24.0, r_hole=0.65, order=ORDER):
    """Cartesian background [-box, box]^3 (nb^3 points, Dirichlet) + spherical shell
    (nphi x nth x nr, polar band) + two orthographic pole patches (npatch^2 x nr).

    Background points with |x| < r_hole are cut out; the cut points within order/2 grid
    lines (along an axis) of a background discretization point become interpolation
    points.  Donors (stencils of width order + 1): background receivers from the shell,
    else a patch; shell receivers from a patch, else the background; patch receivers from
    the shell, else the background.  Returns (grids, interp).
    """
    w = order + 1
    B = cartesian_grid3("background", (nb, nb, nb), (-box,) * 3, (box,) * 3,
                        [BC_DIRICHLET] * 6)
    S = shell_grid("shell", nphi, nth, nr, r_in, width, band[0], band[1], order)
    A = math.sin(math.radians(patch_deg))
    PN = pole_patch_grid("north", npatch, nr, A, r_in, width, 1.0, order)
    PS = pole_patch_grid("south", npatch, nr, A, r_in, width, -1.0, order)
    # hole cutting, plane by plane
    x = -box + B.h[0] * np.arange(nb)
    inside = np.zeros((nb, nb, nb), bool)
    X2 = x[None, :] ** 2 + x[:, None] ** 2
    for k in range(nb):
        inside[k] = X2 + x[k] ** 2 < r_hole * r_hole
    near = _near(~inside, order // 2)
    B.mask[inside & near] = INTERP
    B.mask[inside & ~near] = UNUSED
    del inside, near
    grids = [B, S, PN, PS]
    parts = []
    for rgid, donors in ((0, (1, 2, 3)), (1, (2, 3, 0)), (2, (1, 0)), (3, (1, 0))):
        g = grids[rgid]
        ijk = _interp_points(g)
        pts = _points_of(g, ijk)
        dg, c, f = find_donors(grids, rgid, pts, donors, w)
        parts.append((rgid, ijk, dg, c, f))
    interp = _assemble(grids, parts, w)
    check_explicit_interp3(grids, interp)
    return grids, interp


def _near(active, reach):
    """Points within ``reach`` grid lines of an active point along one axis."""
    near = np.zeros_like(active)
    for d in range(1, reach + 1):
        near[d:] |= active[:-d]
        near[:-d] |= active[d:]
        near[:, d:] |= active[:, :-d]
        near[:, :-d] |= active[:, d:]
        near[:, :, d:] |= active[:, :, :-d]
        near[:, :, :-d] |= active[:, :, d:]
    return near


def box_in_box(nb=12, ni=10, box=1.0, inner=0.45, hole=0.25, order=ORDER):
    """Two Cartesian grids: background [-box, box]^3 (Dirichlet, nb^3) with a cubic hole
    |x|_inf < hole, and an inner box [-inner, inner]^3 (ni^3) whose faces are
    interpolation points.  A small overset grid for brute-force checks.  At order p the
    interpolation layers are p/2 points thick and the donor stencils p + 1 wide."""
    r, w = order // 2, order + 1
    B = cartesian_grid3("background", (nb,) * 3, (-box,) * 3, (box,) * 3, [BC_DIRICHLET] * 6)
    I = cartesian_grid3("inner", (ni,) * 3, (-inner,) * 3, (inner,) * 3, [BC_NONE] * 6)
    x = -box + B.h[0] * np.arange(nb)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    inside = np.maximum(np.maximum(abs(X), abs(Y)), abs(Z)) < hole
    near = _near(~inside, r)
    B.mask[inside & near] = INTERP
    B.mask[inside & ~near] = UNUSED
    I.mask[:, :, :r] = I.mask[:, :, -r:] = INTERP
    I.mask[:, :r, :] = I.mask[:, -r:, :] = INTERP
    I.mask[:r, :, :] = I.mask[-r:, :, :] = INTERP
    grids = [B, I]
    parts = []
    for rgid, donors in ((0, (1,)), (1, (0,))):
        g = grids[rgid]
        ijk = _interp_points(g)
        pts = _points_of(g, ijk)
        dg, c, f = find_donors(grids, rgid, pts, donors, w)
        parts.append((rgid, ijk, dg, c, f))
    interp = _assemble(grids, parts, w)
    check_explicit_interp3(grids, interp)
    return grids, interp


# ----------------------------------------------------------------------------------
# Sources and problems
# ----------------------------------------------------------------------------------

def gaussian3(g, x0, amp=1.0, b=200.0):
    """f(x) = amp exp(-b |x - x0|^2) on the points of g (compact (n2, n1, n0))."""
    out = np.empty((g.n[2], g.n[1], g.n[0]))
    for k in range(g.n[2]):
        X = g.coords(k)
        out[k] = amp * np.exp(-b * ((X[0] - x0[0]) ** 2 + (X[1] - x0[1]) ** 2 +
                                    (X[2] - x0[2]) ** 2))
    return out


def _seeded_point(rng, lo, hi, rmin):
    while True:
        p = rng.uniform(lo, hi, size=3)
        if np.linalg.norm(p) >= rmin:
            return p


def sphere_problem(nb=320, nphi=256, nth=128, nr=24, npatch=96, omega=30.0, seed=0,
                   width=0.3, r_hole=0.65, patch_deg=24.0, b=200.0, order=ORDER,
                   band=(15.0, 165.0), box=2.0):
    """Sphere-in-box: Gaussian point source seeded in the background away from the
    sphere.  Coarse test grids need a wider shell and a larger hole radius so that every
    receiver still has a full donor stencil."""
    rng = np.random.default_rng(seed)
    grids, interp = sphere_in_box(nb, nphi, nth, nr, npatch, width=width, r_hole=r_hole,
                                  patch_deg=patch_deg, order=order, band=band, box=box)
    x0 = _seeded_point(rng, -0.75 * box, 0.75 * box, 1.0)
    f = [gaussian3(g, x0, 1.0, b) for g in grids]
    return Problem3(grids, interp, omega, f,
                    name=f"sphere-in-box-{nb}^3+{nphi}x{nth}x{nr}+2x{npatch}^2x{nr}-o{order}",
                    meta=dict(source=x0.tolist(), seed=seed), order=order)


def unit_cube_problem(n=24, omega=10.0, seed=0, bc=BC_DIRICHLET, b=200.0, order=ORDER):
    """One Cartesian grid on [0, 1]^3 with n^3 points, Gaussian at x0 ~ U[0.3, 0.7]^3.
    ``bc`` is one code for all six faces or a list of six."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.3, 0.7, size=3)
    bcs = list(bc) if isinstance(bc, (list, tuple)) else [bc] * 6
    g = cartesian_grid3("cube", (n, n, n), (0.0,) * 3, (1.0,) * 3, bcs)
    return Problem3([g], Interp3.empty(), omega, [gaussian3(g, x0, 1.0, b)],
                    name=f"unit-cube-{n}^3", meta=dict(source=x0.tolist(), seed=seed),
                    order=order)


def box_in_box_problem(nb=12, ni=10, omega=6.0, seed=0, b=20.0, order=ORDER, hole=0.25):
    rng = np.random.default_rng(seed)
    grids, interp = box_in_box(nb, ni, hole=hole, order=order)
    x0 = _seeded_point(rng, -0.7, 0.7, 0.5)
    f = [gaussian3(g, x0, 1.0, b) for g in grids]
    return Problem3(grids, interp, omega, f, name=f"box-in-box-{nb}^3+{ni}^3",
                    meta=dict(source=x0.tolist(), seed=seed), order=order)


def with_boundary_data3(problem, fn):
    """The same problem with Dirichlet data g = fn(x, y, z) on every Dirichlet point (zero
    elsewhere): the Helmholtz solution takes the value g there."""
    import copy
    p = copy.copy(problem)
    p.g = []
    for g in problem.grids:
        X = g.coords()
        p.g.append(np.where(g.mask == DIRICHLET, fn(X[0], X[1], X[2]), 0.0))
    p.name = problem.name + "-g"
    return p


def random_state3(problem, seed):
    """A seeded random vector on the active points (zero on unused points)."""
    rng = np.random.default_rng(seed)
    out = []
    for g in problem.grids:
        v = rng.standard_normal(g.mask.shape)
        v[g.mask == UNUSED] = 0.0
        out.append(v.ravel())
    return np.concatenate(out)
