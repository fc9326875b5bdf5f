"""Brute-force assembly of the three-dimensional discrete Helmholtz system (DHS) on
Cartesian overset grids, for pinning the 3D oracle.

The converged WaveHoltz iterate equals the direct solution of (Sec. 6, App. B.1)

    c^2 (D+D-_x + D+D-_y + D+D-_z) U + omega^2 U = f   at discretization points,
    U = 0                                              at Dirichlet boundary points,
    U - sum w U_donor = 0                              at interpolation points,
    U_ghost - U_inward = 0                             at Neumann ghost points,
    U = 0                                              everywhere else.

The rows come from the textbook 7-point stencil (on curvilinear grids the mapped Laplacian
with metric coefficients and mixed terms), independently of the oracle's C code, and are
solved with a sparse LU.  At fourth order (``problem.order == 4``) the second
differences take the 5-point weights (-1, 16, -30, 16, -1)/12, two ghost layers per face
carry the rows c^2 D_nn U_b = f_b (Dirichlet; the zero boundary values make the
tangential terms vanish) or 8 (U_1 - G_1) - (U_2 - G_2) = 0 (Neumann), each with the
extrapolation D+^5 G_2 = 0, and the interpolation stencils are 5 wide.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2504_03074_gb300 import grids as G


# off-centre second-difference weights (offset, weight) and the centre weight
D2W = {2: [(-1, 1.0), (1, 1.0)],
       4: [(-2, -1.0 / 12), (-1, 16.0 / 12), (1, 16.0 / 12), (2, -1.0 / 12)]}
D2C = {2: -2.0, 4: -30.0 / 12}
EXTRAP5 = [1.0, -5.0, 10.0, -10.0, 5.0, -1.0]  # on G2, G1, U0, U1, U2, U3


def _neumann_data(problem, gi, g, b, a):
    """gn / |grad r_a| at boundary point b (i, j, k) of a Neumann face of axis a: the
    parameter derivative du/dr_a along the inward direction is -(that), read from the
    problem's Neumann data (zero when it has none)."""
    gnl = getattr(problem, "gn", None)
    if gnl is None or gnl[gi] is None:
        return 0.0
    val = gnl[gi][b[2], b[1], b[0]]
    if g.kind == G.CARTESIAN or val == 0.0:
        return val
    gh = g.ghosts(problem.order)
    r = g.rx[:, b[2] + gh[2], b[1] + gh[1], b[0] + gh[0]]
    return val / np.sqrt(r[3 * a] ** 2 + r[3 * a + 1] ** 2 + r[3 * a + 2] ** 2)


def fourth_order_ghost_rows(problem, gi, g, L, c2, put, rhs, done, coef=None):
    """The two ghost rows of every boundary point of a Dirichlet or Neumann face; on a
    curvilinear grid (coef = (A, B) of curvilinear_coefficients) the Dirichlet row is
    c^2 (a_nn D_nn + b_n D_n) U_b = f_b with D_n along +r_a."""
    for s in range(6):
        code = g.bc[s]
        if code not in (G.BC_DIRICHLET, G.BC_NEUMANN):
            continue
        a, hi = s // 2, s % 2
        t1, t2 = (a + 1) % 3, (a + 2) % 3
        for v in range(g.n[t2]):
            for u in range(g.n[t1]):
                def pt(o):  # point at offset o along the inward normal (o < 0: ghosts)
                    ix = [0, 0, 0]
                    ix[t1], ix[t2] = u, v
                    ix[a] = g.n[a] - 1 - o if hi else o
                    return ix
                b = pt(0)
                m = g.mask[b[2], b[1], b[0]]
                if (code == G.BC_NEUMANN and m != G.DISC) or \
                        (code == G.BC_DIRICHLET and m != G.DIRICHLET):
                    continue
                G1, G2 = L.idx(gi, *pt(-1)), L.idx(gi, *pt(-2))
                U = [L.idx(gi, *pt(o)) for o in range(4)]
                for c_, col in zip(EXTRAP5, [G2, G1] + U):
                    put(G2, col, c_)
                if code == G.BC_NEUMANN:
                    # the undivided inward D_n equals -12 h du/dn-data / |grad r_a|
                    for c_, col in zip([1.0, -8.0, 8.0, -1.0], [G2, G1, U[1], U[2]]):
                        put(G1, col, c_)
                    rhs[G1] = -12.0 * g.h[a] * _neumann_data(problem, gi, g, b, a)
                else:
                    ann, bn = c2[b[2], b[1], b[0]], 0.0
                    if coef is not None:
                        ann = coef[0][a, a, b[2], b[1], b[0]]
                        bn = coef[1][a, b[2], b[1], b[0]]
                    w = ann / (12.0 * g.h[a] ** 2)
                    # +r_a is inward on a low side: D_n = (G2 - 8 G1 + 8 U1 - U2) / (12 h)
                    wb = (-1.0 if hi else 1.0) * bn / (12.0 * g.h[a])
                    for c_, d_, col in zip([-1.0, 16.0, -30.0, 16.0, -1.0],
                                           [1.0, -8.0, 0.0, 8.0, -1.0], [G2, G1] + U[:3]):
                        put(G1, col, w * c_ + wb * d_)
                    rhs[G1] = problem.f[gi][b[2], b[1], b[0]]
                done[G1] = done[G2] = True


# full difference tables (offsets -p/2 .. p/2) for curvilinear rows
D2F = {2: np.array([1.0, -2.0, 1.0]), 4: np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0}
D1F = {2: np.array([-0.5, 0.0, 0.5]), 4: np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / 12.0}


def curvilinear_coefficients(problem, gi, order):
    """c^2 a_kl (3 x 3) and c^2 b_k (3) at the grid's points, shape (n2, n1, n0): the
    mapping method of Sec. 3.1, a_kl = sum_m dr_k/dx_m dr_l/dx_m and
    b_k = sum_m sum_l dr_l/dx_m D_l(dr_k/dx_m) with D_l the order-p centred first
    difference of the (analytic, ghost-extended) metrics; a_kl of pairs declared orthogonal
    dropped."""
    g = problem.grids[gi]
    gh = g.ghosts(order)
    r = order // 2
    rx = g.rx  # (9, e2, e1, e0): rx[3k + m] = dr_k/dx_m
    n0, n1, n2 = g.n
    sl = (slice(gh[2], gh[2] + n2), slice(gh[1], gh[1] + n1), slice(gh[0], gh[0] + n0))

    def shifted(arr, a, k):
        ax = 2 - a  # array axis of parameter axis a
        if g.bc[2 * a] == G.BC_PERIODIC:
            return np.roll(arr, -k, axis=ax)[sl]
        s2 = list(sl)
        s2[ax] = slice(sl[ax].start + k, sl[ax].stop + k)
        return arr[tuple(s2)]

    def d1(arr, a):
        return sum(D1F[order][k + r] * shifted(arr, a, k) for k in range(-r, r + 1)) / g.h[a]

    inner = rx[(slice(None),) + sl]
    c2 = np.ones((n2, n1, n0)) if problem.c2 is None else problem.c2[gi]
    A = np.empty((3, 3, n2, n1, n0))
    for k in range(3):
        for l in range(3):
            A[k, l] = c2 * sum(inner[3 * k + m] * inner[3 * l + m] for m in range(3))
    for p_, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        if g.ortho >> p_ & 1:
            A[a, b] = A[b, a] = 0.0
    B = np.empty((3, n2, n1, n0))
    for k in range(3):
        B[k] = c2 * sum(inner[3 * l + m] * d1(rx[3 * k + m], l) for m in range(3)
                        for l in range(3))
    return A, B


def curvilinear_row(put, L, gi, g, i, j, k, A, B, order, r_row):
    """The mapped Laplacian's row at (i, j, k): sum_a A_aa D2_a + B_a D1_a + 2 sum_{a<b}
    A_ab D1_a D1_b (the centre weight is added by the caller's put accumulation)."""
    rr = order // 2
    for a in range(3):
        for s_ in range(-rr, rr + 1):
            d = [0, 0, 0]
            d[a] = s_
            w = (A[a, a, k, j, i] * D2F[order][s_ + rr] / g.h[a] ** 2 +
                 B[a, k, j, i] * D1F[order][s_ + rr] / g.h[a])
            if w != 0.0:
                put(r_row, L.idx(gi, i + d[0], j + d[1], k + d[2]), w)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        ab = A[a, b, k, j, i]
        if ab == 0.0:
            continue
        for sa in range(-rr, rr + 1):
            for sb in range(-rr, rr + 1):
                w = D1F[order][sa + rr] * D1F[order][sb + rr]
                if w == 0.0:
                    continue
                d = [0, 0, 0]
                d[a], d[b] = sa, sb
                put(r_row, L.idx(gi, i + d[0], j + d[1], k + d[2]),
                    2.0 * ab * w / (g.h[a] * g.h[b]))


class Layout3:
    def __init__(self, problem):
        self.p = problem
        self.off, self.ext, self.gh = [], [], []
        o = 0
        for g in problem.grids:
            gh = g.ghosts(getattr(problem, "order", 2))
            e = tuple(g.n[a] + 2 * gh[a] for a in range(3))
            self.off.append(o)
            self.ext.append(e)
            self.gh.append(gh)
            o += e[0] * e[1] * e[2]
        self.N = o

    def idx(self, gi, i, j, k):
        g = self.p.grids[gi]
        gh, e = self.gh[gi], self.ext[gi]
        ix = [i, j, k]
        for a in range(3):
            if g.bc[2 * a] == G.BC_PERIODIC:
                ix[a] %= g.n[a]
            assert -gh[a] <= ix[a] < g.n[a] + gh[a]
        return self.off[gi] + ((ix[2] + gh[2]) * e[1] + (ix[1] + gh[1])) * e[0] + ix[0] + gh[0]


def assemble(problem):
    """Sparse DHS matrix and right-hand side over every extended point."""
    L = Layout3(problem)
    om2 = problem.omega ** 2
    order = getattr(problem, "order", 2)
    rows, cols, vals = [], [], []
    rhs = np.zeros(L.N)
    done = np.zeros(L.N, bool)

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for gi, g in enumerate(problem.grids):
        curv = g.kind == G.CURVILINEAR
        if curv:
            A, B = curvilinear_coefficients(problem, gi, order)
        c2 = np.ones(g.mask.shape) if problem.c2 is None else problem.c2[gi]
        for k in range(g.n[2]):
            for j in range(g.n[1]):
                for i in range(g.n[0]):
                    m = g.mask[k, j, i]
                    r = L.idx(gi, i, j, k)
                    done[r] = True
                    if m == G.DISC and curv:
                        put(r, r, om2)
                        curvilinear_row(put, L, gi, g, i, j, k, A, B, order, r)
                        rhs[r] = problem.f[gi][k, j, i]
                    elif m == G.DISC:
                        diag = om2
                        for a in range(3):
                            w = c2[k, j, i] / g.h[a] ** 2
                            for s, cw in D2W[order]:
                                d = [0, 0, 0]
                                d[a] = s
                                put(r, L.idx(gi, i + d[0], j + d[1], k + d[2]), w * cw)
                            diag += w * D2C[order]
                        put(r, r, diag)
                        rhs[r] = problem.f[gi][k, j, i]
                    elif m != G.INTERP:
                        put(r, r, 1.0)
                        gb = getattr(problem, "g", None)
                        if m == G.DIRICHLET and gb is not None and gb[gi] is not None:
                            rhs[r] = gb[gi][k, j, i]  # U = g at Dirichlet points
        if order == 4:
            fourth_order_ghost_rows(problem, gi, g, L, c2, put, rhs, done,
                                    (A, B) if curv else None)
            continue
        # Neumann ghosts next to discretization points
        for s in range(6):
            if g.bc[s] != G.BC_NEUMANN:
                continue
            a, hi = s // 2, s % 2
            t1, t2 = (a + 1) % 3, (a + 2) % 3
            for v in range(g.n[t2]):
                for u in range(g.n[t1]):
                    ib, ig, inw = [0] * 3, [0] * 3, [0] * 3
                    for arr in (ib, ig, inw):
                        arr[t1], arr[t2] = u, v
                    ib[a] = g.n[a] - 1 if hi else 0
                    ig[a] = g.n[a] if hi else -1
                    inw[a] = g.n[a] - 2 if hi else 1
                    if g.mask[ib[2], ib[1], ib[0]] != G.DISC:
                        continue
                    r = L.idx(gi, *ig)
                    done[r] = True
                    put(r, r, 1.0)
                    put(r, L.idx(gi, *inw), -1.0)
                    rhs[r] = 2.0 * g.h[a] * _neumann_data(problem, gi, g, ib, a)
    it = problem.interp
    for q in range(it.n):
        r = L.idx(int(it.recv_grid[q]), int(it.recv_i[q]), int(it.recv_j[q]), int(it.recv_k[q]))
        put(r, r, 1.0)
        dg = int(it.donor_grid[q])
        wd = order + 1
        for c in range(wd):
            for b in range(wd):
                for a in range(wd):
                    w = it.wx[q, a] * it.wy[q, b] * it.wz[q, c]
                    put(r, L.idx(dg, int(it.donor_i0[q]) + a, int(it.donor_j0[q]) + b,
                                 int(it.donor_k0[q]) + c), -w)
    for r in np.nonzero(~done)[0]:
        put(int(r), int(r), 1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(L.N, L.N))
    return A, rhs, L


def solve(problem):
    """Direct DHS solution as a compact vector (grids concatenated, axis 0 fastest)."""
    A, rhs, L = assemble(problem)
    lu = spla.splu(A.tocsc())
    U = lu.solve(rhs)
    U = U + lu.solve(rhs - A @ U)  # one step of iterative refinement
    out = []
    for gi, g in enumerate(problem.grids):
        gh, e = L.gh[gi], L.ext[gi]
        Ue = U[L.off[gi]:L.off[gi] + e[0] * e[1] * e[2]].reshape(e[2], e[1], e[0])
        out.append(Ue[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]].ravel())
    return np.concatenate(out)
