"""Seeded synthetic inputs: overset grid descriptions, Gaussian sources and sound speeds.

This module is the stand-in for the paper's grid generator (Ogen, Sec. 3.1): it builds
component grids from analytic mappings x = G_g(r), classifies their points as
discretization / interpolation / unused (Sec. 3.1), cuts holes, finds donor stencils
and the tensor-product Lagrange weights of width p+1 (Sec. 3.1), and evaluates the
Gaussian source of Eq. (gaussianSource, Sec. 6).  It holds none of the WaveHoltz
arithmetic (no difference operator, no time stepping, no filter): its outputs are
the *input data* that both the CUDA library and the CPU oracle consume.

Array conventions shared by every consumer:

* a grid has ``n = (n0, n1)`` points along parameter axes 0 and 1 (boundary points
  included, ghost points excluded; a periodic axis lists each point once);
* compact per-grid arrays have shape ``(n1, n0)`` in C order, i.e. flat index
  ``j * n0 + i`` with ``i`` (axis 0) fastest;
* ghost width is ``order // 2`` on non-periodic axes and 0 on periodic ones; the
  "extended" arrays (metrics) have shape ``(n1 + 2 g1, n0 + 2 g0)`` and start at
  index ``(-g1, -g0)``;
* sides are numbered ``[axis0-lo, axis0-hi, axis1-lo, axis1-hi]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# point classification (Sec. 3.1): discretization, interpolation, unused; Dirichlet
# boundary points are discretization points whose value the boundary condition sets.
UNUSED, DISC, INTERP, DIRICHLET = 0, 1, 2, 3
# boundary condition per side
BC_NONE, BC_DIRICHLET, BC_NEUMANN, BC_PERIODIC = 0, 1, 2, 3
# grid kinds
CARTESIAN, CURVILINEAR = 0, 1


@dataclass
class Grid:
    """One component grid G_g of an overset grid (Sec. 3.1)."""

    name: str
    kind: int
    n: tuple                      # (n0, n1) points per axis
    bc: list                      # 4 side codes
    h: tuple                      # Cartesian: physical spacing; curvilinear: parameter spacing
    mask: np.ndarray              # int8 (n1, n0)
    xy: np.ndarray                # float64 (2, n1, n0) physical coordinates
    orthogonal: bool = True       # grid lines meet at right angles (a12 == 0 identically)
    rx: np.ndarray | None = None  # float64 (4, n1+2g1, n0+2g0): dr1/dx, dr1/dy, dr2/dx, dr2/dy
    origin: tuple = (0.0, 0.0)    # Cartesian: coordinates of point (0, 0)
    instance: int = 0             # independent problem of a batch

    def ghosts(self, order):
        return tuple(0 if self.bc[2 * a] == BC_PERIODIC else order // 2 for a in (0, 1))

    @property
    def npts(self):
        return self.n[0] * self.n[1]


@dataclass
class Interp:
    """Interpolation data (Sec. 3.1): each receiver gets a (p+1)^2 donor stencil.

    The donor stencil's lower corner is ``(donor_i0, donor_j0)`` in the donor grid's
    index space (wrapping on periodic axes); the tensor-product weights are
    ``wx[k, a] * wy[k, b]`` for donor point ``(i0 + a, j0 + b)``.
    """

    recv_grid: np.ndarray
    recv_i: np.ndarray
    recv_j: np.ndarray
    donor_grid: np.ndarray
    donor_i0: np.ndarray
    donor_j0: np.ndarray
    wx: np.ndarray
    wy: np.ndarray

    @property
    def n(self):
        return int(self.recv_grid.shape[0])

    @staticmethod
    def empty(order):
        z = np.zeros(0, np.int32)
        w = np.zeros((0, order + 1))
        return Interp(z, z, z, z, z, z, w, w)


@dataclass
class Problem:
    """A Helmholtz problem c^2 Lap u + omega^2 u = f on an overset grid (Eq. HelmholtzBVP)."""

    grids: list
    interp: Interp
    order: int
    omega: float
    f: list                       # per-grid compact forcing, float64 (n1, n0)
    c2: list | None = None        # per-grid compact c(x)^2, or None for c = 1
    name: str = ""
    meta: dict = field(default_factory=dict)
    g: list | None = None         # per-grid compact Dirichlet data (read at Dirichlet points)
    gn: list | None = None        # per-grid compact Neumann data dU/dn (outward normal), read
                                  # at the discretization points of Neumann sides

    @property
    def n_active(self):
        return int(sum(int(np.count_nonzero(g.mask != UNUSED)) for g in self.grids))

    @property
    def n_total(self):
        return int(sum(g.npts for g in self.grids))

    def split(self, vec):
        """Split a concatenated compact vector into per-grid (n1, n0) views."""
        out, o = [], 0
        for g in self.grids:
            out.append(vec[o:o + g.npts].reshape(g.n[1], g.n[0]))
            o += g.npts
        return out


# ----------------------------------------------------------------------------------
# Lagrange weights (Sec. 3.1: tensor-product Lagrange interpolation of width p+1)
# ----------------------------------------------------------------------------------

def lagrange_weights(xi, width):
    """Weights of the Lagrange polynomial through nodes 0..width-1 evaluated at xi."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.ones(xi.shape + (width,))
    for a in range(width):
        for b in range(width):
            if b != a:
                w[..., a] *= (xi - b) / (a - b)
    return w


# ----------------------------------------------------------------------------------
# Component grids
# ----------------------------------------------------------------------------------

def cartesian_grid(name, n0, n1, x0, x1, y0, y1, bc, order):
    """Axis-aligned Cartesian grid on [x0,x1]x[y0,y1] with n0 x n1 points."""
    hx, hy = (x1 - x0) / (n0 - 1), (y1 - y0) / (n1 - 1)
    i = np.arange(n0)
    j = np.arange(n1)
    X = x0 + hx * i[None, :] + 0.0 * j[:, None]
    Y = y0 + hy * j[:, None] + 0.0 * i[None, :]
    mask = np.full((n1, n0), DISC, np.int8)
    for s, code in enumerate(bc):
        if code == BC_DIRICHLET:
            if s == 0:
                mask[:, 0] = DIRICHLET
            elif s == 1:
                mask[:, -1] = DIRICHLET
            elif s == 2:
                mask[0, :] = DIRICHLET
            else:
                mask[-1, :] = DIRICHLET
    return Grid(name, CARTESIAN, (n0, n1), list(bc), (hx, hy), mask, np.stack([X, Y]),
                True, None, (x0, y0))


def annulus_grid(name, nth, nr, r_in, width, beta, order, inner_bc=BC_NEUMANN):
    """Body-fitted annulus r(s) = r_in + width (e^{beta s}-1)/(e^beta-1), theta = 2 pi t.

    Axis 0 is the angle t in [0, 1) (periodic, nth points, no duplicate), axis 1 the
    radial parameter s in [0, 1] (nr points).  Side axis1-lo (s = 0) is the body; the
    outer p/2 lines are interpolation points.  The inverse metrics are analytic and
    are evaluated on ghost lines too (the mapping extends smoothly past s = 0, 1).
    """
    g1 = order // 2
    dt_, ds = 1.0 / nth, 1.0 / (nr - 1)
    t = np.arange(nth) * dt_
    s_ext = np.arange(-g1, nr + g1) * ds
    eb = math.exp(beta) - 1.0

    def radius(s):
        return r_in + width * (np.exp(beta * s) - 1.0) / eb

    def dradius(s):
        return width * beta * np.exp(beta * s) / eb

    th = 2.0 * np.pi * t
    R = radius(s_ext)[:, None]
    Rs = dradius(s_ext)[:, None]
    c, s_ = np.cos(th)[None, :], np.sin(th)[None, :]
    rx = np.empty((4, nr + 2 * g1, nth))
    rx[0] = -s_ / (2.0 * np.pi * R)   # dt/dx
    rx[1] = c / (2.0 * np.pi * R)     # dt/dy
    rx[2] = c / Rs                    # ds/dx
    rx[3] = s_ / Rs                   # ds/dy
    Rin = R[g1:g1 + nr]
    X = Rin * c
    Y = Rin * s_
    mask = np.full((nr, nth), DISC, np.int8)
    mask[nr - order // 2:, :] = INTERP
    if inner_bc == BC_DIRICHLET:
        mask[0, :] = DIRICHLET
    bc = [BC_PERIODIC, BC_PERIODIC, inner_bc, BC_NONE]
    g = Grid(name, CURVILINEAR, (nth, nr), bc, (dt_, ds), mask, np.stack([X, Y]), True, rx)
    g.mapping = dict(r_in=r_in, width=width, beta=beta)
    return g


def sheared_torus_grid(name, n0, n1, amp_x, amp_y, order):
    """Doubly periodic non-orthogonal grid x = r1 + ax sin(2 pi r2), y = r2 + ay sin(2 pi r1).

    A flat torus: no physical boundary, all points discretization points, and the mixed
    derivative term of the mapped Laplacian is present everywhere (tests).
    """
    d0, d1 = 1.0 / n0, 1.0 / n1
    r1 = np.arange(n0) * d0
    r2 = np.arange(n1) * d1
    R1, R2 = np.meshgrid(r1, r2)
    x_r1 = np.ones_like(R1)
    x_r2 = 2.0 * np.pi * amp_x * np.cos(2.0 * np.pi * R2)
    y_r1 = 2.0 * np.pi * amp_y * np.cos(2.0 * np.pi * R1)
    y_r2 = np.ones_like(R1)
    det = x_r1 * y_r2 - x_r2 * y_r1
    rx = np.stack([y_r2 / det, -x_r2 / det, -y_r1 / det, x_r1 / det])
    X = R1 + amp_x * np.sin(2.0 * np.pi * R2)
    Y = R2 + amp_y * np.sin(2.0 * np.pi * R1)
    mask = np.full((n1, n0), DISC, np.int8)
    g = Grid(name, CURVILINEAR, (n0, n1), [BC_PERIODIC] * 4, (d0, d1), mask,
             np.stack([X, Y]), False, rx)
    g.mapping = dict(amp_x=amp_x, amp_y=amp_y)
    return g


# ----------------------------------------------------------------------------------
# Overset assembly: hole cutting, classification, donor search (Ogen stand-in)
# ----------------------------------------------------------------------------------

def _annulus_param(gA, x, y):
    """Fractional (i, j) index of physical points in the annulus parameter space."""
    m = gA.mapping
    th = np.mod(np.arctan2(y, x), 2.0 * np.pi)
    ti = th / (2.0 * np.pi) * gA.n[0]
    r = np.hypot(x, y)
    eb = math.exp(m["beta"]) - 1.0
    s = np.log1p((r - m["r_in"]) * eb / m["width"]) / m["beta"]
    return ti, s * (gA.n[1] - 1)


def _cart_param(gB, x, y):
    return (x - gB.origin[0]) / gB.h[0], (y - gB.origin[1]) / gB.h[1]


def _donors(fi, fj, donor, order, clamp_j_hi, periodic_i):
    """Lower-corner indices of the width-(p+1) stencil nearest the point, shifted inward."""
    w = order + 1
    i0 = np.rint(fi).astype(np.int64) - order // 2
    j0 = np.rint(fj).astype(np.int64) - order // 2
    if not periodic_i:
        i0 = np.clip(i0, 0, donor.n[0] - w)
    j0 = np.clip(j0, 0, clamp_j_hi - w + 1)
    return i0, j0, lagrange_weights(fi - i0, w), lagrange_weights(fj - j0, w)


def disk_in_square(nb, nth, nr, order, box=2.0, r_in=0.5, width=0.3, beta=1.5,
                   r_cut=0.65):
    """Cartesian background [-box, box]^2 (nb^2 points, Dirichlet) + stretched annulus.

    Background points with |x| < r_cut are cut out; those within p/2 index layers
    (box neighbourhood) of a background discretization point become interpolation
    points, the rest unused.  The annulus's outer p/2 lines are interpolation points
    (donors on the background).  Donor stencils contain only discretization points
    (explicit interpolation).  Returns (grids, interp).
    """
    B = cartesian_grid("background", nb, nb, -box, box, -box, box, [BC_DIRICHLET] * 4, order)
    A = annulus_grid("annulus", nth, nr, r_in, width, beta, order)
    X, Y = B.xy
    inside = np.hypot(X, Y) < r_cut
    active = ~inside
    half = order // 2
    near = np.zeros_like(active)
    pad = np.pad(active, half)
    for dj in range(-half, half + 1):
        for di in range(-half, half + 1):
            near |= pad[half + dj:half + dj + nb, half + di:half + di + nb]
    B.mask[inside & near] = INTERP
    B.mask[inside & ~near] = UNUSED

    recv = []
    # background receivers <- annulus donors
    jb, ib = np.nonzero(B.mask == INTERP)
    fi, fj = _annulus_param(A, X[jb, ib], Y[jb, ib])
    last_disc = nr - 1 - half
    i0, j0, wx, wy = _donors(fi, fj, A, order, last_disc, True)
    recv.append((0, ib, jb, 1, i0, j0, wx, wy))
    # annulus receivers <- background donors
    ja, ia = np.nonzero(A.mask == INTERP)
    XA, YA = A.xy
    fi, fj = _cart_param(B, XA[ja, ia], YA[ja, ia])
    i0, j0, wx, wy = _donors(fi, fj, B, order, nb - 1, False)
    recv.append((1, ia, ja, 0, i0, j0, wx, wy))

    cols = list(zip(*recv))
    interp = Interp(
        np.concatenate([np.full(len(r[1]), r[0], np.int32) for r in recv]),
        np.concatenate(cols[1]).astype(np.int32), np.concatenate(cols[2]).astype(np.int32),
        np.concatenate([np.full(len(r[1]), r[3], np.int32) for r in recv]),
        np.concatenate(cols[4]).astype(np.int32), np.concatenate(cols[5]).astype(np.int32),
        np.concatenate(cols[6]), np.concatenate(cols[7]))
    grids = [B, A]
    check_explicit_interp(grids, interp, order)
    return grids, interp


def check_explicit_interp(grids, interp, order):
    """Every donor must be a discretization (or Dirichlet) point: explicit interpolation."""
    w = order + 1
    for k in range(interp.n):
        d = grids[interp.donor_grid[k]]
        ii = interp.donor_i0[k] + np.arange(w)
        jj = interp.donor_j0[k] + np.arange(w)
        if d.bc[0] == BC_PERIODIC:
            ii = np.mod(ii, d.n[0])
        if d.bc[2] == BC_PERIODIC:
            jj = np.mod(jj, d.n[1])
        if ii.min() < 0 or ii.max() >= d.n[0] or jj.min() < 0 or jj.max() >= d.n[1]:
            raise ValueError(f"receiver {k}: donor stencil out of range")
        m = d.mask[np.ix_(jj, ii)]
        if not np.all((m == DISC) | (m == DIRICHLET)):
            raise ValueError(f"receiver {k}: donor stencil touches a non-discretization point")


# ----------------------------------------------------------------------------------
# Several bodies in a square: disks and ellipses, each wrapped in a body-fitted grid
# ----------------------------------------------------------------------------------

@dataclass
class Body:
    """A body in the background square: a disk (a == b) or an axis-aligned ellipse (a > b)
    with semi-axes (a, b) centred at ``center``, wrapped in a body-fitted grid of nth x nr
    points whose outer edge lies ``width`` further out along the x semi-axis (stretched
    toward the body by ``beta``).  The background hole is the region whose radial grid
    parameter is below ``cut`` (0: the body itself, 1: the grid's outer edge)."""

    center: tuple
    a: float
    b: float
    width: float
    nth: int
    nr: int
    beta: float = 1.5
    cut: float = 0.5
    inner_bc: int = BC_NEUMANN


class _BodyMap:
    """The body grid's mapping x = G(t, s), t in [0, 1) around the body, s in [0, 1] out.

    A disk uses polar coordinates, r(s) = a + width q(s); an ellipse uses elliptic
    coordinates, x - c = f cosh(mu) cos(nu), y - c_y = f sinh(mu) sin(nu), f^2 = a^2 - b^2,
    mu(s) = mu0 + (mu1 - mu0) q(s), nu = 2 pi t, with q(s) = (e^{beta s} - 1) / (e^beta - 1).
    Both are orthogonal (the ellipse's conformal), as the Neumann ghost rule assumes."""

    def __init__(self, body):
        self.b = body
        self.cx, self.cy = body.center
        self.eb = math.exp(body.beta) - 1.0
        if body.a < body.b:
            raise ValueError("ellipses are taken with a >= b (x semi-axis the longer)")
        self.polar = body.a == body.b
        if self.polar:
            self.r0, self.r1 = body.a, body.a + body.width
        else:
            self.f = math.sqrt(body.a ** 2 - body.b ** 2)
            self.mu0 = math.atanh(body.b / body.a)
            self.mu1 = math.acosh((body.a + body.width) / self.f)

    def q(self, s):
        return (np.exp(self.b.beta * s) - 1.0) / self.eb

    def dq(self, s):
        return self.b.beta * np.exp(self.b.beta * s) / self.eb

    def lo_hi(self):
        return (self.r0, self.r1) if self.polar else (self.mu0, self.mu1)

    def xy(self, t, s):
        lo, hi = self.lo_hi()
        rho = lo + (hi - lo) * self.q(s)
        th = 2.0 * np.pi * t
        if self.polar:
            return self.cx + rho * np.cos(th), self.cy + rho * np.sin(th)
        return (self.cx + self.f * np.cosh(rho) * np.cos(th),
                self.cy + self.f * np.sinh(rho) * np.sin(th))

    def rx(self, t, s):
        """dt/dx, dt/dy, ds/dx, ds/dy at parameter points (analytic)."""
        lo, hi = self.lo_hi()
        rho = lo + (hi - lo) * self.q(s)
        drho_ds = (hi - lo) * self.dq(s)
        th = 2.0 * np.pi * t
        if self.polar:
            c, sn = np.cos(th), np.sin(th)
            return (-sn / (2.0 * np.pi * rho), c / (2.0 * np.pi * rho), c / drho_ds,
                    sn / drho_ds)
        # w = mu + i nu is analytic in z = x + i y with dw/dz = 1 / (f sinh w):
        # mu_x = nu_y = Re w', nu_x = -mu_y = Im w'
        w = rho + 1j * th
        wp = 1.0 / (self.f * np.sinh(w))
        mux, nux = wp.real, wp.imag
        return nux / (2.0 * np.pi), mux / (2.0 * np.pi), mux / drho_ds, -nux / drho_ds

    def param(self, x, y):
        """Fractional (t n_th, s (n_r - 1)) indices of physical points, and the radial
        parameter s itself (negative inside the body)."""
        lo, hi = self.lo_hi()
        if self.polar:
            th = np.mod(np.arctan2(y - self.cy, x - self.cx), 2.0 * np.pi)
            rho = np.hypot(x - self.cx, y - self.cy)
        else:
            # the principal branch has Re w >= 0 and Im w in (-pi, pi]
            w = np.arccosh(((x - self.cx) + 1j * (y - self.cy)) / self.f)
            rho, th = w.real, np.mod(w.imag, 2.0 * np.pi)
        u = (rho - lo) / (hi - lo) * self.eb
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(u > -1.0, np.log1p(u) / self.b.beta, -np.inf)
        return th / (2.0 * np.pi) * self.b.nth, s * (self.b.nr - 1), s


def body_grid(name, body, order):
    """The body-fitted grid of one Body: axis 0 periodic around the body (nth points),
    axis 1 outward (nr points); the body is side axis1-lo, the outer order/2 lines are
    interpolation points.  Inverse metrics analytic, on ghost lines too."""
    m = _BodyMap(body)
    g1 = order // 2
    nth, nr = body.nth, body.nr
    dt_, ds = 1.0 / nth, 1.0 / (nr - 1)
    t = (np.arange(nth) * dt_)[None, :]
    s_ext = (np.arange(-g1, nr + g1) * ds)[:, None]
    rx = np.stack([np.broadcast_to(v, (nr + 2 * g1, nth)) for v in m.rx(t, s_ext)])
    X, Y = m.xy(t, (np.arange(nr) * ds)[:, None])
    X, Y = np.broadcast_to(X, (nr, nth)).copy(), np.broadcast_to(Y, (nr, nth)).copy()
    mask = np.full((nr, nth), DISC, np.int8)
    mask[nr - g1:, :] = INTERP
    if body.inner_bc == BC_DIRICHLET:
        mask[0, :] = DIRICHLET
    bc = [BC_PERIODIC, BC_PERIODIC, body.inner_bc, BC_NONE]
    g = Grid(name, CURVILINEAR, (nth, nr), bc, (dt_, ds), mask, np.stack([X, Y]), True,
             np.ascontiguousarray(rx))
    g.mapping = dict(body=body)
    return g


def bodies_in_square(nb, bodies, order, box=2.0):
    """Cartesian background [-box, box]^2 (nb^2 points, Dirichlet) with holes cut for
    several bodies, each wrapped in its body-fitted grid (Sec. 3.1's overset grid with
    more than one curvilinear component).  Background points inside a body's cut become
    interpolation points within order/2 index layers of a background discretization point
    (donors on that body's grid), the rest unused; each body grid's outer order/2 lines
    take donors on the background.  Donor stencils hold discretization points only
    (explicit interpolation, checked).  Returns (grids, interp)."""
    B = cartesian_grid("background", nb, nb, -box, box, -box, box, [BC_DIRICHLET] * 4, order)
    maps = [_BodyMap(b) for b in bodies]
    grids = [B] + [body_grid("body%d" % k, b, order) for k, b in enumerate(bodies)]
    X, Y = B.xy
    half = order // 2
    # the body whose cut holds each background point (-1: none)
    owner = np.full(X.shape, -1, np.int64)
    for k, (m, b) in enumerate(zip(maps, bodies)):
        _, _, s = m.param(X, Y)
        inside = s < b.cut
        if np.any(inside & (owner >= 0)):
            raise ValueError("the cuts of two bodies overlap")
        owner[inside] = k
    active = owner < 0
    near = np.zeros_like(active)
    pad = np.pad(active, half)
    for dj in range(-half, half + 1):
        for di in range(-half, half + 1):
            near |= pad[half + dj:half + dj + nb, half + di:half + di + nb]
    B.mask[~active & near] = INTERP
    B.mask[~active & ~near] = UNUSED
    recv = []
    for k, (m, b) in enumerate(zip(maps, bodies)):
        A = grids[k + 1]
        # background receivers in this body's cut <- body donors
        jb, ib = np.nonzero((B.mask == INTERP) & (owner == k))
        fi, fj, sr = m.param(X[jb, ib], Y[jb, ib])
        if sr.size and not np.all(sr >= 0.0):
            raise ValueError("body %d: background interpolation points lie inside the body "
                             "(raise its cut or refine the background)" % k)
        i0, j0, wx, wy = _donors(fi, fj, A, order, b.nr - 1 - half, True)
        recv.append((0, ib, jb, k + 1, i0, j0, wx, wy))
        # body receivers <- background donors
        ja, ia = np.nonzero(A.mask == INTERP)
        fi, fj = _cart_param(B, A.xy[0][ja, ia], A.xy[1][ja, ia])
        i0, j0, wx, wy = _donors(fi, fj, B, order, nb - 1, False)
        recv.append((k + 1, ia, ja, 0, i0, j0, wx, wy))
    cols = list(zip(*recv))
    interp = Interp(
        np.concatenate([np.full(len(r[1]), r[0], np.int32) for r in recv]),
        np.concatenate(cols[1]).astype(np.int32), np.concatenate(cols[2]).astype(np.int32),
        np.concatenate([np.full(len(r[1]), r[3], np.int32) for r in recv]),
        np.concatenate(cols[4]).astype(np.int32), np.concatenate(cols[5]).astype(np.int32),
        np.concatenate(cols[6]), np.concatenate(cols[7]))
    check_explicit_interp(grids, interp, order)
    return grids, interp


# ----------------------------------------------------------------------------------
# The knife edge: a thin plate with a rounded tip standing on the bottom wall
# ----------------------------------------------------------------------------------

def _gauss01(n, lo=0.0, hi=1.0):
    """Gauss-Legendre nodes and weights on [lo, hi]."""
    g, w = np.polynomial.legendre.leggauss(n)
    return lo + 0.5 * (hi - lo) * (g + 1.0), 0.5 * (hi - lo) * w


class KnifeOutline:
    """Outline of the knife, traversed by arclength sigma from its base on the right
    (x = width/2, y = 0) up the right side, around the tip and down the left side: straight
    sides of height y_s joined by a tip of arclength ell whose curvature
    kappa = (2 pi / ell) sin^2(pi u), u = (sigma - y_s) / ell, turns the tangent by pi with
    kappa and kappa' continuous at the joins (the paper's rounded tip, smooth enough for
    fourth-order metrics).  ell and y_s are set by the width and the height of the apex.
    Beyond [0, S] the sides continue straight below the wall (ghost lines)."""

    def __init__(self, width=0.02, height=0.5):
        self.width, self.height = width, height
        self.w2 = 0.5 * width
        u, w = _gauss01(64)
        self.ell = width / -float(np.sum(w * np.cos(self.phi_tip(u))))
        u, w = _gauss01(64, 0.0, 0.5)
        self.ys = height - self.ell * float(np.sum(w * np.sin(self.phi_tip(u))))
        self.S = 2.0 * self.ys + self.ell
        self.kmax = 2.0 * math.pi / self.ell

    @staticmethod
    def phi_tip(u):
        """Tangent angle over the tip: pi/2 + pi u - sin(2 pi u) / 2, u in [0, 1]."""
        return 0.5 * np.pi + np.pi * u - 0.5 * np.sin(2.0 * np.pi * u)

    def frame(self, sigma):
        """Point (x, y), tangent angle phi and curvature kappa at arclength sigma."""
        sigma = np.asarray(sigma, np.float64)
        u = np.clip((sigma - self.ys) / self.ell, 0.0, 1.0)
        g, w = _gauss01(40)
        ph = self.phi_tip(u[..., None] * g)  # tip: quadrature of the unit tangent over [0, u]
        tx = self.w2 + self.ell * u * np.sum(w * np.cos(ph), axis=-1)
        ty = self.ys + self.ell * u * np.sum(w * np.sin(ph), axis=-1)
        right, left = sigma < self.ys, sigma > self.ys + self.ell
        x = np.where(right, self.w2, np.where(left, -self.w2, tx))
        y = np.where(right, sigma, np.where(left, self.ys - (sigma - self.ys - self.ell), ty))
        phi = np.where(right, 0.5 * np.pi, np.where(left, 1.5 * np.pi, self.phi_tip(u)))
        kap = np.where(right | left, 0.0, self.kmax * np.sin(np.pi * u) ** 2)
        return x, y, phi, kap


class _KnifeMap:
    """The knife grid's mapping x = gamma(sigma) + d n(sigma): sigma = S t0 along the
    outline, d = W q(t1) along the outward normal n = (sin phi, -cos phi), with
    q(s) = (e^{beta s} - 1) / (e^beta - 1).  Orthogonal; the outline is convex, so
    outward offsets never fold (dx/dsigma = (1 + d kappa) times the tangent)."""

    def __init__(self, outline, W, beta):
        self.o, self.W, self.beta = outline, W, beta
        self.eb = math.exp(beta) - 1.0
        sig = np.linspace(-0.05, outline.S + 0.05, 20001)
        x, y, _, _ = outline.frame(sig)
        from scipy.spatial import cKDTree
        self._sig, self._tree = sig, cKDTree(np.stack([x, y], axis=1))

    def q(self, s):
        return (np.exp(self.beta * s) - 1.0) / self.eb

    def dq(self, s):
        return self.beta * np.exp(self.beta * s) / self.eb

    def xy(self, t0, t1):
        x, y, phi, _ = self.o.frame(self.o.S * t0)
        d = self.W * self.q(t1)
        return x + d * np.sin(phi), y - d * np.cos(phi)

    def rx(self, t0, t1):
        """dt0/dx, dt0/dy, dt1/dx, dt1/dy (analytic in the outline's frame)."""
        _, _, phi, kap = self.o.frame(self.o.S * t0)
        d = self.W * self.q(t1)
        j0 = self.o.S * (1.0 + d * kap)
        j1 = self.W * self.dq(t1)
        return np.cos(phi) / j0, np.sin(phi) / j0, np.sin(phi) / j1, -np.cos(phi) / j1

    def param(self, x, y):
        """(sigma, d) of physical points: the nearest outline sample, then Newton on
        (p - gamma(sigma)) . t(sigma) = 0 (derivative -(1 + kappa d))."""
        x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
        _, k = self._tree.query(np.stack([x.ravel(), y.ravel()], axis=1))
        sig = self._sig[k].reshape(x.shape)
        for _ in range(8):
            gx, gy, phi, kap = self.o.frame(sig)
            tx, ty = np.cos(phi), np.sin(phi)
            f = (x - gx) * tx + (y - gy) * ty
            d = (x - gx) * ty - (y - gy) * tx
            sig = sig + f / np.maximum(1.0 + kap * d, 0.25)
        gx, gy, phi, _ = self.o.frame(sig)
        d = (x - gx) * np.sin(phi) - (y - gy) * np.cos(phi)
        return sig, d

    def index(self, x, y, n0, n1):
        """Fractional (i, j) indices of physical points in the knife grid."""
        sig, d = self.param(x, y)
        with np.errstate(invalid="ignore"):
            s = np.log1p(d / self.W * self.eb) / self.beta
        return sig / self.o.S * (n0 - 1), s * (n1 - 1), d


def knife_edge(j=32, order=4, width=0.02, height=0.5, wfac=12.0, n1=16, cut=0.4, beta=1.5):
    """The knife-edge overset grid (Sec. 6): a Cartesian background on
    [-0.5, 0.5] x [0, 0.55] with spacing 1/(10 j), Dirichlet on every side, and one
    body-fitted grid hugging the whole knife (a thin plate of the given width whose rounded
    tip reaches the given height, standing on the bottom wall): axis 0 along the outline
    (spacing half the background's), axis 1 outward over W = wfac background spacings
    (n1 lines stretched toward the knife).  Its sides: the two ends lie on the bottom wall
    and the knife surface, all Dirichlet; the outer order/2 lines are interpolation points
    (donors on the background), as are the wall points of those lines.  Background points
    within cut W of the knife (or inside it) are cut out; those within order/2 index layers
    of an active background point become interpolation points (donors on the knife grid),
    the rest unused.  The paper covers the same knife with a tip grid and two side grids;
    one grid along the whole outline keeps every component orthogonal.  Returns
    (grids, interp, outline)."""
    h = 1.0 / (10 * j)
    nx, ny = 10 * j + 1, int(round(0.55 / h)) + 1
    B = cartesian_grid("background", nx, ny, -0.5, 0.5, 0.0, (ny - 1) * h, [BC_DIRICHLET] * 4,
                       order)
    ko = KnifeOutline(width, height)
    W = wfac * h
    m = _KnifeMap(ko, W, beta)
    g1 = order // 2
    n0 = int(math.ceil(2.0 * ko.S / h)) + 1
    if 1.0 + ko.kmax * W * m.q(-g1 / (n1 - 1)) <= 0.25:
        raise ValueError("the knife grid's ghost lines fold at the tip: refine or widen")
    if height + W + (order // 2 + 1) * h > (ny - 1) * h:
        raise ValueError("the knife grid reaches the top wall: refine or lower the knife")
    d0, d1 = 1.0 / (n0 - 1), 1.0 / (n1 - 1)
    t0e = (np.arange(-g1, n0 + g1) * d0)[None, :]
    t1e = (np.arange(-g1, n1 + g1) * d1)[:, None]
    shape = (n1 + 2 * g1, n0 + 2 * g1)
    rx = np.stack([np.broadcast_to(v, shape) for v in m.rx(t0e, t1e)])
    X, Y = m.xy((np.arange(n0) * d0)[None, :], (np.arange(n1) * d1)[:, None])
    X, Y = np.broadcast_to(X, (n1, n0)).copy(), np.broadcast_to(Y, (n1, n0)).copy()
    mask = np.full((n1, n0), DISC, np.int8)
    mask[0, :] = DIRICHLET
    mask[:, 0] = DIRICHLET
    mask[:, -1] = DIRICHLET
    mask[n1 - g1:, :] = INTERP
    K = Grid("knife", CURVILINEAR, (n0, n1), [BC_DIRICHLET, BC_DIRICHLET, BC_DIRICHLET, BC_NONE],
             (d0, d1), mask, np.stack([X, Y]), True, np.ascontiguousarray(rx))
    K.mapping = dict(knife=m)
    # hole cutting
    XB, YB = B.xy
    _, _, dB = m.index(XB, YB, n0, n1)
    inside = dB < cut * W
    active = ~inside
    near = np.zeros_like(active)
    pad = np.pad(active, g1)
    for dj in range(-g1, g1 + 1):
        for di in range(-g1, g1 + 1):
            near |= pad[g1 + dj:g1 + dj + ny, g1 + di:g1 + di + nx]
    B.mask[inside & near] = INTERP
    B.mask[inside & ~near] = UNUSED
    recv = []
    jb, ib = np.nonzero(B.mask == INTERP)
    fi, fj, d = m.index(XB[jb, ib], YB[jb, ib], n0, n1)
    if d.size and not np.all(d > 0.0):
        raise ValueError("background interpolation points lie inside the knife")
    i0, j0, wx, wy = _donors(fi, fj, K, order, n1 - 1 - g1, False)
    recv.append((0, ib, jb, 1, i0, j0, wx, wy))
    jk, ik = np.nonzero(K.mask == INTERP)
    fi, fj = _cart_param(B, X[jk, ik], Y[jk, ik])
    i0, j0, wx, wy = _donors(fi, fj, B, order, ny - 1, False)
    recv.append((1, ik, jk, 0, i0, j0, wx, wy))
    cols = list(zip(*recv))
    interp = Interp(
        np.concatenate([np.full(len(r[1]), r[0], np.int32) for r in recv]),
        np.concatenate(cols[1]).astype(np.int32), np.concatenate(cols[2]).astype(np.int32),
        np.concatenate([np.full(len(r[1]), r[3], np.int32) for r in recv]),
        np.concatenate(cols[4]).astype(np.int32), np.concatenate(cols[5]).astype(np.int32),
        np.concatenate(cols[6]), np.concatenate(cols[7]))
    grids = [B, K]
    check_explicit_interp(grids, interp, order)
    return grids, interp, ko


# ----------------------------------------------------------------------------------
# The double ellipse (Penrose's unilluminable room)
# ----------------------------------------------------------------------------------

class _Segment:
    """A straight piece of an outline from p0 to p1, by arclength (straight beyond both
    ends).  frame(s) -> (x, y, tx, ty, kappa)."""

    def __init__(self, p0, p1):
        self.p0 = np.asarray(p0, np.float64)
        d = np.asarray(p1, np.float64) - self.p0
        self.L = float(np.hypot(d[0], d[1]))
        self.t = d / self.L

    def frame(self, s):
        s = np.asarray(s, np.float64)
        z = np.zeros_like(s)
        return (self.p0[0] + s * self.t[0], self.p0[1] + s * self.t[1], z + self.t[0],
                z + self.t[1], z)


class _EllipseArc:
    """The arc theta from th0 to th1 of the ellipse c + (a cos theta, b sin theta), by
    arclength s from th0 (the ellipse continues beyond both ends).  theta(s) by Newton on
    s(theta), the integral of the speed sqrt(a^2 sin^2 + b^2 cos^2) from a table of
    12-point Gauss-Legendre panels plus one partial panel.  kappa = dphi/ds, positive where
    the tangent turns counterclockwise."""

    def __init__(self, center, a, b, th0, th1, ext=0.5, panels=2048):
        self.c = np.asarray(center, np.float64)
        self.a, self.b = float(a), float(b)
        self.th0, self.sg = float(th0), 1.0 if th1 > th0 else -1.0
        psi_end = abs(th1 - th0)
        self.lo, self.dpsi = -ext, (psi_end + 2.0 * ext) / panels
        self.gx, self.gw = _gauss01(12)
        nodes = self.lo + self.dpsi * np.arange(panels)
        seg = self.dpsi * np.sum(self.gw * self._speed(nodes[:, None] + self.dpsi * self.gx),
                                 axis=1)
        self.cum = np.concatenate([[0.0], np.cumsum(seg)])
        self.s0 = 0.0
        self.s0 = float(self._s(np.array([0.0]))[0])
        self.L = float(self._s(np.array([psi_end]))[0])

    def _speed(self, psi):
        th = self.th0 + self.sg * psi
        return np.hypot(self.a * np.sin(th), self.b * np.cos(th))

    def _s(self, psi):
        k = np.clip(np.floor((psi - self.lo) / self.dpsi).astype(np.int64), 0,
                    len(self.cum) - 2)
        base = self.lo + k * self.dpsi
        d = psi - base
        part = d * np.sum(self.gw * self._speed(base[..., None] + d[..., None] * self.gx),
                          axis=-1)
        return self.cum[k] + part - self.s0

    def frame(self, s):
        s = np.asarray(s, np.float64)
        psi = s / max(self.a, self.b)
        for _ in range(60):
            step = (self._s(psi) - s) / self._speed(psi)
            psi = psi - step
            if np.all(np.abs(step) < 1e-14):
                break
        th = self.th0 + self.sg * psi
        sp = np.hypot(self.a * np.sin(th), self.b * np.cos(th))
        tx = -self.sg * self.a * np.sin(th) / sp
        ty = self.sg * self.b * np.cos(th) / sp
        kap = self.sg * self.a * self.b / sp ** 3
        return self.c[0] + self.a * np.cos(th), self.c[1] + self.b * np.sin(th), tx, ty, kap


class _Outline:
    """Pieces joined end to end with a continuous tangent, by arclength sigma in [0, S]
    (the first and last pieces continue beyond the ends)."""

    def __init__(self, pieces):
        self.pieces = pieces
        self.starts = np.concatenate([[0.0], np.cumsum([p.L for p in pieces])])
        self.S = float(self.starts[-1])

    def frame(self, sigma):
        sigma = np.asarray(sigma, np.float64)
        k = np.searchsorted(self.starts[1:-1], sigma, side="right")
        out = [np.zeros_like(sigma) for _ in range(5)]
        for i, p in enumerate(self.pieces):
            sel = k == i
            if np.any(sel):
                for o, v in zip(out, p.frame(sigma[sel] - self.starts[i])):
                    o[sel] = v
        return tuple(out)


class _OffsetMap:
    """x = gamma(sigma) + d n(sigma) with sigma = S t0 along an outline, d = W t1 along the
    right-hand normal n = (t_y, -t_x) (into the fluid), uniform in both.  Orthogonal:
    dx/dsigma = (1 + kappa d) t, dx/dd = n."""

    def __init__(self, outline, W, ext):
        self.o, self.W = outline, W
        sig = np.linspace(-ext, outline.S + ext, int((outline.S + 2 * ext) / (W / 400.0)) + 2)
        x, y, _, _, _ = outline.frame(sig)
        from scipy.spatial import cKDTree
        self._sig, self._tree = sig, cKDTree(np.stack([x, y], axis=1))

    def xy(self, t0, t1):
        x, y, tx, ty, _ = self.o.frame(self.o.S * t0)
        d = self.W * t1
        return x + d * ty, y - d * tx

    def rx(self, t0, t1):
        """dt0/dx, dt0/dy, dt1/dx, dt1/dy (analytic in the outline's frame)."""
        _, _, tx, ty, kap = self.o.frame(self.o.S * t0)
        j0 = self.o.S * (1.0 + self.W * t1 * kap)
        return tx / j0, ty / j0, ty / self.W, -tx / self.W

    def param(self, x, y):
        """(sigma, d) of physical points: the nearest outline sample, then Newton on
        (p - gamma(sigma)) . t(sigma) = 0 (derivative -(1 + kappa d)); the last residual."""
        x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
        _, k = self._tree.query(np.stack([x.ravel(), y.ravel()], axis=1))
        sig = self._sig[k].reshape(x.shape)
        for _ in range(12):
            gx, gy, tx, ty, kap = self.o.frame(sig)
            f = (x - gx) * tx + (y - gy) * ty
            d = (x - gx) * ty - (y - gy) * tx
            sig = sig + f / np.maximum(1.0 + kap * d, 0.25)
        gx, gy, tx, ty, _ = self.o.frame(sig)
        f = (x - gx) * tx + (y - gy) * ty
        return sig, (x - gx) * ty - (y - gy) * tx, f


def _offset_grid(name, outline, W, h, order, ends_physical):
    """The grid of an _OffsetMap: axis 0 along the outline (spacing about h), axis 1 into
    the fluid (W / h intervals).  The wall row is Dirichlet; the outer order/2 rows are
    interpolation points; the end columns are Dirichlet sides (ends_physical) or order/2
    interpolation columns (their wall points stay Dirichlet)."""
    g1 = order // 2
    m = _OffsetMap(outline, W, (g1 + 2) * h)
    n0 = int(math.ceil(outline.S / h)) + 1
    n1 = int(round(W / h)) + 1
    d0, d1 = 1.0 / (n0 - 1), 1.0 / (n1 - 1)
    t0e = (np.arange(-g1, n0 + g1) * d0)[None, :]
    t1e = (np.arange(-g1, n1 + g1) * d1)[:, None]
    shape = (n1 + 2 * g1, n0 + 2 * g1)
    rx = np.stack([np.broadcast_to(v, shape) for v in m.rx(t0e, t1e)])
    X, Y = m.xy((np.arange(n0) * d0)[None, :], (np.arange(n1) * d1)[:, None])
    X, Y = np.broadcast_to(X, (n1, n0)).copy(), np.broadcast_to(Y, (n1, n0)).copy()
    mask = np.full((n1, n0), DISC, np.int8)
    if ends_physical:
        mask[:, 0] = mask[:, -1] = DIRICHLET
    else:
        mask[:, :g1] = mask[:, n0 - g1:] = INTERP
    mask[n1 - g1:, :] = INTERP
    mask[0, :] = DIRICHLET
    side = BC_DIRICHLET if ends_physical else BC_NONE
    g = Grid(name, CURVILINEAR, (n0, n1), [side, side, BC_DIRICHLET, BC_NONE], (d0, d1), mask,
             np.stack([X, Y]), True, np.ascontiguousarray(rx))
    g.mapping = dict(offset=m)
    return g


class DoubleEllipseRoom:
    """Penrose's unilluminable room as the paper builds it (Sec. 6): the left and right
    walls are half-ellipses with semi-axes (a2, b2) = (3, 6) centred at (-+a1, 0); the top
    and bottom walls are half-ellipses with semi-axes (a1, b1) = (2, 1) centred at
    (0, +-f), f = sqrt(b2^2 - a2^2), whose ends sit at the large ellipses' foci
    (-+a1, +-f); vertical segments x = -+a1 from the foci to the large ellipses' ends
    (-+a1, +-b2) close the four alcoves.  The room spans [-5, 5] x [-6, 6]."""

    a1, b1, a2, b2 = 2.0, 1.0, 3.0, 6.0

    def __init__(self):
        self.f = math.sqrt(self.b2 ** 2 - self.a2 ** 2)

    def inside(self, x, y):
        a1, f = self.a1, self.f
        left = ((x + a1) / self.a2) ** 2 + (y / self.b2) ** 2 < 1.0
        right = ((x - a1) / self.a2) ** 2 + (y / self.b2) ** 2 < 1.0
        with np.errstate(invalid="ignore"):
            cap = f - self.b1 * np.sqrt(np.clip(1.0 - (x / a1) ** 2, 0.0, None))
        mid = (np.abs(x) < a1) & (np.abs(y) < cap)
        return np.where(x <= -a1, left, np.where(x >= a1, right, mid))

    def outlines(self, y0):
        """The four walls as outlines traversed with the fluid on the right: the left and
        right half-ellipses (end to end), and the top and bottom walls from y = +-y0 on
        one alcove segment, around the small half-ellipse, to y = +-y0 on the other."""
        a1, b1, a2, b2, f = self.a1, self.b1, self.a2, self.b2, self.f
        pi = math.pi
        left = _Outline([_EllipseArc((-a1, 0.0), a2, b2, 1.5 * pi, 0.5 * pi)])
        right = _Outline([_EllipseArc((a1, 0.0), a2, b2, 0.5 * pi, -0.5 * pi)])
        top = _Outline([_Segment((-a1, y0), (-a1, f)), _EllipseArc((0.0, f), a1, b1, pi, 2 * pi),
                        _Segment((a1, f), (a1, y0))])
        bottom = _Outline([_Segment((a1, -y0), (a1, -f)), _EllipseArc((0.0, -f), a1, b1, 0.0, pi),
                           _Segment((-a1, -f), (-a1, -y0))])
        return left, right, top, bottom


def _find_donors2(grids, index_fns, xq, yq, candidates, order, shift=1):
    """Width-(order+1) donor stencils for points (xq, yq): for each stencil offset (centred
    first, then moved by up to ``shift`` points per axis, nearest first; shifted inward
    at a grid's edge), each candidate grid in turn; a stencil is valid when it holds
    discretization or Dirichlet points only.  Returns (donor grid, i0, j0, wx, wy); raises if a point has
    none."""
    w = order + 1
    N = xq.size
    dg = np.full(N, -1, np.int64)
    i0 = np.zeros(N, np.int64)
    j0 = np.zeros(N, np.int64)
    fi_all, fj_all = np.zeros(N), np.zeros(N)
    frac = {}
    for c in candidates:
        fi, fj, ok = index_fns[c](xq, yq)
        frac[c] = (fi, fj, ok)
    r = range(-shift, shift + 1)
    offs = sorted(((a, b) for b in r for a in r), key=lambda o: (abs(o[0]) + abs(o[1]),
                                                                 max(abs(o[0]), abs(o[1]))))
    for oa, ob in offs:
        for c in candidates:
            todo = np.nonzero(dg < 0)[0]
            if todo.size == 0:
                break
            g = grids[c]
            fi, fj, ok = (v[todo] for v in frac[c])
            ci = np.rint(np.where(ok, fi, 0.0)).astype(np.int64) - order // 2 + oa
            cj = np.rint(np.where(ok, fj, 0.0)).astype(np.int64) - order // 2 + ob
            # near a grid's edge the stencil is shifted inward (one-sided interpolation)
            ci, cj = np.clip(ci, 0, g.n[0] - w), np.clip(cj, 0, g.n[1] - w)
            val = ok.copy()
            for b in range(w):
                for a in range(w):
                    m = g.mask[cj + b, ci + a]
                    val &= (m == DISC) | (m == DIRICHLET)
            take = todo[val]
            dg[take], i0[take], j0[take] = c, ci[val], cj[val]
            fi_all[take], fj_all[take] = fi[val], fj[val]
    if np.any(dg < 0):
        k = int(np.nonzero(dg < 0)[0][0])
        raise ValueError(f"point {k} at ({xq[k]:.4f}, {yq[k]:.4f}) has no donor stencil")
    return dg, i0, j0, lagrange_weights(fi_all - i0, w), lagrange_weights(fj_all - j0, w)


def double_ellipse(j=2, order=4, wfac=12.0, cut=0.4, shift=1):
    """The double-ellipse overset grid (Sec. 6) with target spacing h = 1/(10 j), j >= 2:
    a Cartesian background over the room's bounding box (three spacings of margin), and a
    grid of width W = wfac h along each of the four walls.  The two large half-ellipse
    grids end on the alcove segments, where their end columns are Dirichlet sides; the top
    and bottom grids follow segment, small half-ellipse and segment from y = +-(b2 - W / 2)
    and end in order/2 interpolation columns inside the large grids.  Background points
    outside the room or within cut W of a wall are cut out; those within order/2 index
    layers of an active point become interpolation points.  The paper covers the same room
    with nine grids (four curved, four small Cartesian grids on the alcove segments and the
    background); following each segment with the wall grid of the small ellipse keeps the
    component count at five.  Donor stencils are centred where valid, else moved by up to
    ``shift`` points per axis.  Returns (grids, interp, room)."""
    room = DoubleEllipseRoom()
    h = 1.0 / (10 * j)
    W = wfac * h
    if W >= room.b2 - room.f - 2.0 * h:
        raise ValueError("the wall grids are wider than the alcove segments: refine (j >= 2)")
    g1 = order // 2
    left, right, top, bottom = room.outlines(room.b2 - 0.5 * W)
    walls = [_offset_grid("left", left, W, h, order, True),
             _offset_grid("right", right, W, h, order, True),
             _offset_grid("top", top, W, h, order, False),
             _offset_grid("bottom", bottom, W, h, order, False)]
    mx, my = room.a1 + room.a2 + 3 * h, room.b2 + 3 * h
    nx, ny = int(round(2 * mx / h)) + 1, int(round(2 * my / h)) + 1
    B = cartesian_grid("background", nx, ny, -mx, mx, -my, my, [BC_NONE] * 4, order)
    grids = [B] + walls
    XB, YB = B.xy
    dist = np.full(XB.shape, np.inf)
    pts = np.stack([XB.ravel(), YB.ravel()], axis=1)
    for g in walls:
        o = g.mapping["offset"].o
        sig = np.linspace(0.0, o.S, int(o.S / (h / 50.0)) + 2)
        x, y, _, _, _ = o.frame(sig)
        from scipy.spatial import cKDTree
        d, _ = cKDTree(np.stack([x, y], axis=1)).query(pts)
        dist = np.minimum(dist, d.reshape(XB.shape))
    cutm = ~room.inside(XB, YB) | (dist < cut * W)
    active = ~cutm
    near = np.zeros_like(active)
    pad = np.pad(active, g1)
    for dj in range(-g1, g1 + 1):
        for di in range(-g1, g1 + 1):
            near |= pad[g1 + dj:g1 + dj + ny, g1 + di:g1 + di + nx]
    B.mask[cutm & near] = INTERP
    B.mask[cutm & ~near] = UNUSED

    def cart_index(x, y):
        fi, fj = _cart_param(B, x, y)
        return fi, fj, np.ones(fi.shape, bool)

    def wall_index(g):
        m = g.mapping["offset"]

        def fn(x, y):
            sig, d, res = m.param(x, y)
            ok = (np.abs(res) < 1e-9) & (d > -1e-12) & (d < m.W * (1 + 1e-12)) & \
                 (sig > -1e-12) & (sig < m.o.S * (1 + 1e-12))
            return sig / m.o.S * (g.n[0] - 1), d / m.W * (g.n[1] - 1), ok
        return fn

    index_fns = [cart_index] + [wall_index(g) for g in walls]
    recv = []
    for rg, cands in ((0, (1, 2, 3, 4)), (1, (0, 3, 4)), (2, (0, 3, 4)), (3, (0, 1, 2)),
                      (4, (0, 1, 2))):
        g = grids[rg]
        jr, ir = np.nonzero(g.mask == INTERP)
        X, Y = g.xy
        dgr, i0, j0, wx, wy = _find_donors2(grids, index_fns, X[jr, ir], Y[jr, ir], cands,
                                            order, shift)
        recv.append((rg, ir, jr, dgr, i0, j0, wx, wy))
    cols = list(zip(*recv))
    interp = Interp(
        np.concatenate([np.full(len(r[1]), r[0], np.int32) for r in recv]),
        np.concatenate(cols[1]).astype(np.int32), np.concatenate(cols[2]).astype(np.int32),
        np.concatenate(cols[3]).astype(np.int32),
        np.concatenate(cols[4]).astype(np.int32), np.concatenate(cols[5]).astype(np.int32),
        np.concatenate(cols[6]), np.concatenate(cols[7]))
    check_explicit_interp(grids, interp, order)
    return grids, interp, room


# ----------------------------------------------------------------------------------
# Sources and coefficients
# ----------------------------------------------------------------------------------

def gaussian(xy, x0, amp=1.0, b=200.0):
    """f(x) = amp * exp(-b |x - x0|^2) (Eq. gaussianSource without the cos(omega t))."""
    d2 = (xy[0] - x0[0]) ** 2 + (xy[1] - x0[1]) ** 2
    return amp * np.exp(-b * d2)


def bumps_c2(xy, centers, amp=0.2, width=0.2):
    """c(x)^2 with c = 1 + amp * sum_i exp(-|x - x_i|^2 / width^2)."""
    c = np.ones_like(xy[0])
    for x0 in centers:
        c += amp * np.exp(-((xy[0] - x0[0]) ** 2 + (xy[1] - x0[1]) ** 2) / width ** 2)
    return c * c


def _seeded_point_in_background(rng, lo, hi, rmin):
    while True:
        p = rng.uniform(lo, hi, size=2)
        if math.hypot(p[0], p[1]) >= rmin:
            return p


# ----------------------------------------------------------------------------------
# The workloads: unit square (64^2), disk-in-square (1024^2 + 2048x64), and scaled
# versions of the same recipes for tests.
# ----------------------------------------------------------------------------------

def unit_square_problem(n=64, order=2, omega=10.0, seed=0, bc=BC_DIRICHLET):
    """Single Cartesian grid on [0,1]^2 with n^2 points, Gaussian at x0 ~ U[0.3,0.7]^2."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.3, 0.7, size=2)
    g = cartesian_grid("square", n, n, 0.0, 1.0, 0.0, 1.0, [bc] * 4, order)
    f = gaussian(g.xy, x0, 1.0, 200.0)
    return Problem([g], Interp.empty(order), order, omega, [f], None,
                   name=f"unit-square-{n}x{n}-o{order}", meta=dict(x0=x0.tolist(), seed=seed))


def channel_problem(n=32, order=4, omega=7.0, seed=0, bc=BC_NEUMANN):
    """Cartesian channel: periodic in x on [0, 1), walls y = 0, 1 with condition ``bc``."""
    rng = np.random.default_rng(seed)
    g = cartesian_grid("channel", n, n, 0.0, (n - 1) / n, 0.0, 1.0,
                       [BC_PERIODIC, BC_PERIODIC, bc, bc], order)
    x0 = rng.uniform(0.3, 0.7, size=2)
    f = gaussian(g.xy, x0, 1.0, 30.0)
    return Problem([g], Interp.empty(order), order, omega, [f], None,
                   name=f"channel-{n}x{n}-o{order}-bc{bc}", meta=dict(x0=x0.tolist()))


def disk_problem(nb=1024, nth=2048, nr=64, order=4, omega=40.0, seed=0, n_src=1,
                 c_bumps=0, box=2.0, width=0.3, r_cut=0.65):
    """Disk-in-square overset problem: Gaussian source(s) seeded in the background.

    Coarse test grids need a wider annulus (``width``) and cut radius ``r_cut`` so that
    the overlap still holds a full donor stencil.
    """
    rng = np.random.default_rng(seed)
    grids, interp = disk_in_square(nb, nth, nr, order, box=box, width=width, r_cut=r_cut)
    srcs = [_seeded_point_in_background(rng, -1.5, 1.5, 1.0) for _ in range(n_src)]
    f = []
    for g in grids:
        fg = np.zeros(g.mask.shape)
        for x0 in srcs:
            fg += gaussian(g.xy, x0, 1.0, 200.0)
        f.append(fg)
    c2 = None
    centers = []
    if c_bumps:
        centers = [_seeded_point_in_background(rng, -1.8, 1.8, 0.8) for _ in range(c_bumps)]
        c2 = [bumps_c2(g.xy, centers) for g in grids]
    return Problem(grids, interp, order, omega, f, c2,
                   name=f"disk-in-square-{nb}^2+{nth}x{nr}-o{order}",
                   meta=dict(sources=[s.tolist() for s in srcs], seed=seed,
                             bumps=[c.tolist() for c in centers]))


def bodies_problem(nb, bodies, order=4, omega=10.0, seed=0, n_src=1, box=2.0, c_bumps=0,
                   name="bodies-in-square"):
    """Several bodies (disks, ellipses) in the square [-box, box]^2 with Gaussian source(s)
    seeded in the background at least 0.3 from every body grid's outer edge."""
    rng = np.random.default_rng(seed)
    grids, interp = bodies_in_square(nb, bodies, order, box=box)
    maps = [_BodyMap(b) for b in bodies]

    def clear(p):
        for m, b in zip(maps, bodies):
            for dx, dy in ((0.3, 0), (-0.3, 0), (0, 0.3), (0, -0.3), (0, 0)):
                if m.param(np.array([p[0] + dx]), np.array([p[1] + dy]))[2][0] <= 1.0:
                    return False
        return True

    srcs = []
    while len(srcs) < n_src:
        p = rng.uniform(-0.8 * box, 0.8 * box, size=2)
        if clear(p):
            srcs.append(p)
    f = []
    for g in grids:
        fg = np.zeros(g.mask.shape)
        for x0 in srcs:
            fg += gaussian(g.xy, x0, 1.0, 200.0)
        f.append(fg)
    c2 = None
    if c_bumps:
        centers = [rng.uniform(-0.9 * box, 0.9 * box, size=2) for _ in range(c_bumps)]
        c2 = [bumps_c2(g.xy, centers) for g in grids]
    return Problem(grids, interp, order, omega, f, c2,
                   name=f"{name}-{nb}^2+{len(bodies)}-o{order}",
                   meta=dict(sources=[q.tolist() for q in srcs], seed=seed))


def ellipses_problem(nb=512, order=4, omega=20.0, seed=0, scale=1):
    """Multi-object workload: two ellipses and a disk in [-2, 2]^2 with body-fitted grids
    (``scale`` multiplies the body grids' resolution: at scale 1 they match a 512^2
    background's spacing, at scale 2 a 1024^2 one's)."""
    s = scale
    bodies = [Body((-0.9, 0.55), 0.5, 0.25, 0.3, 320 * s, 24 * s),
              Body((0.85, -0.6), 0.6, 0.35, 0.3, 384 * s, 24 * s),
              Body((0.6, 1.05), 0.3, 0.3, 0.3, 256 * s, 24 * s)]
    return bodies_problem(nb, bodies, order=order, omega=omega, seed=seed,
                          name="ellipses-in-square")


def knife_edge_problem(j=32, order=4, omega=100.0, width=0.02, height=0.5, source=(-0.2, 0.2),
                       b=1000.0, **kw):
    """The knife edge (Sec. 6) with a Gaussian source at ``source`` (the paper's
    (-0.2, 0.2)); sizes and shape as in ``knife_edge``."""
    grids, interp, ko = knife_edge(j, order, width, height, **kw)
    f = [gaussian(g.xy, source, 1.0, b) for g in grids]
    return Problem(grids, interp, order, omega, f,
                   name=f"knife-edge-j{j}-w{width:g}-h{height:g}-o{order}",
                   meta=dict(source=list(source), outline=dict(ell=ko.ell, ys=ko.ys, S=ko.S)))


def double_ellipse_problem(j=2, order=4, omega=5.56, source=(0.0, 1.0), amp=400.0, b=10.0,
                           **kw):
    """The double ellipse (Sec. 6) with the paper's Gaussian source (amplitude 400,
    exponent 10, centred at (0, 1)) and omega = 5.56, Dirichlet walls."""
    grids, interp, room = double_ellipse(j, order, **kw)
    f = [gaussian(g.xy, source, amp, b) for g in grids]
    return Problem(grids, interp, order, omega, f, name=f"double-ellipse-j{j}-o{order}",
                   meta=dict(source=list(source)))


def with_boundary_data(problem, fn):
    """The same problem with Dirichlet data g = fn(x, y) on every Dirichlet point (zero
    elsewhere): the Helmholtz solution takes the value g there."""
    import copy
    p = copy.copy(problem)
    p.g = [np.where(g.mask == DIRICHLET, fn(g.xy[0], g.xy[1]), 0.0) for g in problem.grids]
    p.name = problem.name + "-g"
    return p


def sheared_channel_grid(name, n0, n1, shear, L, bc=BC_NEUMANN, order=2):
    """A channel periodic in x (period 1) with walls at y = 0 and y = L, on the
    non-orthogonal grid x = xi + shear * eta, y = L eta (xi periodic in [0, 1), eta in
    [0, 1]): the xi lines cross the walls at an angle (a_01 = -shear / L^2 != 0).
    Constant inverse metrics dxi/dx = 1, dxi/dy = -shear / L, deta/dx = 0, deta/dy = 1/L;
    the walls carry ``bc`` (Dirichlet or Neumann)."""
    g1 = order // 2
    d0, d1 = 1.0 / n0, 1.0 / (n1 - 1)
    xi = (np.arange(n0) * d0)[None, :]
    eta = (np.arange(n1) * d1)[:, None]
    X = np.broadcast_to(xi + shear * eta, (n1, n0)).copy()
    Y = np.broadcast_to(L * eta, (n1, n0)).copy()
    rx = np.empty((4, n1 + 2 * g1, n0))
    rx[0], rx[1], rx[2], rx[3] = 1.0, -shear / L, 0.0, 1.0 / L
    mask = np.full((n1, n0), DISC, np.int8)
    if bc == BC_DIRICHLET:
        mask[0, :] = mask[-1, :] = DIRICHLET
    g = Grid(name, CURVILINEAR, (n0, n1), [BC_PERIODIC, BC_PERIODIC, bc, bc], (d0, d1), mask,
             np.stack([X, Y]), shear == 0.0, rx)
    g.mapping = dict(shear=shear, L=L)
    return g


def sheared_channel_problem(n0=32, n1=17, shear=0.4, L=0.6, bc=BC_NEUMANN, order=2,
                            omega=7.0, seed=0, b=60.0):
    """One sheared channel grid with a Gaussian source seeded inside."""
    rng = np.random.default_rng(seed)
    g = sheared_channel_grid("channel", n0, n1, shear, L, bc, order)
    x0 = (rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7) * L)
    return Problem([g], Interp.empty(order), order, omega, [gaussian(g.xy, x0, 1.0, b)],
                   name=f"sheared-channel-{n0}x{n1}-s{shear:g}", meta=dict(source=x0))


def with_neumann_data(problem, grad):
    """The same problem with Neumann data on every Neumann side: gn = grad u . n at its
    discretization points, n the outward unit normal (-+ grad r_a / |grad r_a| from the
    grid's inverse metrics on a low / high side of axis a; the axis direction on Cartesian
    grids) and grad(x, y) -> (u_x, u_y) the gradient of the intended solution."""
    import copy
    p = copy.copy(problem)
    p.gn = []
    for g in problem.grids:
        gn = np.zeros(g.mask.shape)
        gh = g.ghosts(problem.order)
        for s in range(4):
            if g.bc[s] != BC_NEUMANN:
                continue
            a, hi = s // 2, s % 2
            sl = (slice(None), -1 if hi else 0) if a == 0 else (-1 if hi else 0, slice(None))
            pts = g.mask[sl] == DISC
            x, y = g.xy[0][sl], g.xy[1][sl]
            if g.kind == CARTESIAN:
                nx, ny = (1.0, 0.0) if a == 0 else (0.0, 1.0)
                nx, ny = np.full(x.shape, nx), np.full(x.shape, ny)
            else:
                rx = g.rx[:, gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]
                nx, ny = rx[2 * a][sl], rx[2 * a + 1][sl]
                nrm = np.hypot(nx, ny)
                nx, ny = nx / nrm, ny / nrm
            sign = 1.0 if hi else -1.0
            ux, uy = grad(x, y)
            gn[sl] = np.where(pts, sign * (ux * nx + uy * ny), 0.0)
        p.gn.append(gn)
    p.name = problem.name + "-gn"
    return p


def sheared_torus_problem(n0=32, n1=28, order=4, omega=9.0, seed=0):
    """One non-orthogonal, doubly periodic curvilinear grid (mixed terms everywhere)."""
    rng = np.random.default_rng(seed)
    g = sheared_torus_grid("torus", n0, n1, 0.1, 0.08, order)
    x0 = rng.uniform(0.3, 0.7, size=2)
    f = gaussian(g.xy, x0, 1.0, 30.0)
    return Problem([g], Interp.empty(order), order, omega, [f], None,
                   name=f"sheared-torus-{n0}x{n1}-o{order}", meta=dict(x0=x0.tolist()))


def batch_problems(problems):
    """Concatenate independent problems (same order p) into one batch: grid k of problem i
    keeps its data and gets instance i; the batch's omega is the list of omegas."""
    import copy
    order = problems[0].order
    grids, f, c2, recv, gb = [], [], [], [], []
    any_c2 = any(p.c2 is not None for p in problems)
    any_g = any(getattr(p, "g", None) is not None for p in problems)
    goff = 0
    for k, p in enumerate(problems):
        assert p.order == order
        for gi, g in enumerate(p.grids):
            g2 = copy.copy(g)
            g2.instance = k
            grids.append(g2)
            f.append(p.f[gi])
            c2.append(p.c2[gi] if p.c2 is not None else np.ones(g.mask.shape))
            pg = getattr(p, "g", None)
            gb.append(pg[gi] if pg is not None else None)
        it = p.interp
        recv.append((it.recv_grid + goff, it.recv_i, it.recv_j, it.donor_grid + goff,
                     it.donor_i0, it.donor_j0, it.wx, it.wy))
        goff += len(p.grids)
    cols = list(zip(*recv))
    interp = Interp(*[np.concatenate(c).astype(np.int32) for c in cols[:6]],
                    np.concatenate(cols[6]), np.concatenate(cols[7]))
    return Problem(grids, interp, order, [p.omega for p in problems], f,
                   c2 if any_c2 else None, name=f"batch-{len(problems)}",
                   meta=dict(members=[p.name for p in problems],
                             sizes=[p.n_total for p in problems]),
                   g=gb if any_g else None)


def batch_disk_problem(n_inst=256, seed=0, nb_range=(256, 1024), omega_range=(10.0, 50.0),
                       order=4, src_range=(1, 4), width=0.3, r_cut=0.65):
    """Uneven batch of disk-in-square problems: background N ~ U{nb_range} (N^2 points),
    annulus 2N x N/16, omega ~ U[omega_range], 1-4 seeded Gaussian sources each."""
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n_inst):
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        om = float(rng.uniform(*omega_range))
        ns = int(rng.integers(src_range[0], src_range[1] + 1))
        probs.append(disk_problem(nb=nb, nth=2 * nb, nr=max(nb // 16, 8 + order), order=order,
                                  omega=om, seed=int(rng.integers(1 << 30)), n_src=ns,
                                  width=width, r_cut=r_cut))
    return batch_problems(probs), probs


def receiver_matrix(problem, n=64, radius=1.5):
    """Receivers of a misfit: bilinear sampling of the background grid (grid 0, Cartesian) at
    n points (k + 1/2) 2 pi / n on a circle, as a scipy CSR matrix acting on compact vectors
    (n x n_total)."""
    import scipy.sparse as sp
    g = problem.grids[0]
    th = 2 * np.pi * (np.arange(n) + 0.5) / n
    rows, cols, vals = [], [], []
    for k, t in enumerate(th):
        fi = (radius * np.cos(t) - g.origin[0]) / g.h[0]
        fj = (radius * np.sin(t) - g.origin[1]) / g.h[1]
        i0, j0 = int(np.floor(fi)), int(np.floor(fj))
        a, b = fi - i0, fj - j0
        for di, dj, w in ((0, 0, (1 - a) * (1 - b)), (1, 0, a * (1 - b)), (0, 1, (1 - a) * b),
                          (1, 1, a * b)):
            rows.append(k)
            cols.append((j0 + dj) * g.n[0] + (i0 + di))
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, problem.n_total))


def misfit_problem(nb=512, omega=20.0, order=4, seed=0, width=0.3, r_cut=0.65):
    """The sound-speed inversion workload: disk-in-square at nb^2 (annulus 2nb x nb/16),
    c = 1 + 0.2 sum of 8 seeded Gaussian bumps of width 0.2, one seeded source."""
    return disk_problem(nb=nb, nth=2 * nb, nr=max(nb // 16, 8 + order), order=order,
                        omega=omega, seed=seed, c_bumps=8, width=width, r_cut=r_cut)


def perturbed_c2(problem, amp=0.05, center=(0.9, -0.4), width2=0.3):
    """c^2 of the "true" medium that makes a misfit's data: the problem's c^2 scaled by
    1 + amp exp(-|x - center|^2 / width2), per grid."""
    return [c * (1 + amp * np.exp(-((g.xy[0] - center[0]) ** 2 + (g.xy[1] - center[1]) ** 2)
                                  / width2))
            for c, g in zip(problem.c2, problem.grids)]


def random_state(problem, seed):
    """A seeded random vector on the active points (zero on unused points)."""
    rng = np.random.default_rng(seed)
    out = []
    for g in problem.grids:
        v = rng.standard_normal(g.mask.shape)
        v[g.mask == UNUSED] = 0.0
        out.append(v.ravel())
    return np.concatenate(out)
