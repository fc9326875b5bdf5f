"""Brute-force assembly of the discrete Helmholtz system (DHS), for pinning the oracle.

The converged WaveHoltz iterate equals the direct solution of the discretized
Helmholtz equations (Sec. 6, Eq. HelmholtzDiscrete of App. B.1):

    c^2 L_h U + omega^2 U = f   at discretization points,
    U = 0                       at Dirichlet boundary points,
    U - sum w U_donor = 0       at interpolation points,
    ghost-point rules           at ghost points (see below),
    U = 0                       everywhere else.

This module writes those rows as a scipy sparse matrix from textbook stencil tables,
independently of the oracle's C code (it shares no routine with it), and solves them
with a sparse LU.  Ghost rules (g = 0, orthogonal boundary lines):
order 2 Neumann: U_{-1} - U_{+1} = 0 (on a non-orthogonal grid the normal derivative
a_nn D0_n U + a_nt D0_t U = 0 along the side); with Neumann data gn (``problem.gn``) the
normal derivative along the outward unit normal equals gn instead of 0;
order 4 Neumann: 8(U_1 - G_1) - (U_2 - G_2) = 0 and D+^5 G_2 = 0;
order 4 Dirichlet: c^2 (a_nn D_nn U + b_n D_n U)_b = f_b and D+^5 G_2 = 0.
With Dirichlet data g (``problem.g``): U = g at Dirichlet points, and the order-4
compatibility row's right side is f_b - omega^2 g_b - c^2 (D_tt g)_b (Cartesian grids),
D_tt the fourth-order second difference along the side: centred, wrapped on a periodic
side, one-sided six-point at the ends.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2504_03074_gb300 import grids as G

# textbook central-difference weights, offsets -p/2..p/2
D2W = {2: np.array([1.0, -2.0, 1.0]), 4: np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0}
D1W = {2: np.array([-1.0, 0.0, 1.0]) / 2.0, 4: np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / 12.0}
EXTRAP5 = np.array([1.0, -5.0, 10.0, -10.0, 5.0, -1.0])   # D+^5 on G2, G1, U0, U1, U2, U3
# fourth-order second differences (times 12 h^2) one-sided at the first and second point
ONE_SIDED_D2 = {0: np.array([45.0, -154.0, 214.0, -156.0, 61.0, -10.0]),
                1: np.array([10.0, -15.0, -4.0, 14.0, -6.0, 1.0])}


def side_d2(line, t, periodic, h):
    """Fourth-order second difference of the values `line` along a side at index t."""
    n = len(line)
    if periodic or 2 <= t <= n - 3:
        return sum(D2W[4][k + 2] * line[(t + k) % n] for k in range(-2, 3)) / h ** 2
    if t < 2:
        return float(ONE_SIDED_D2[t] @ line[:6]) / (12.0 * h ** 2)
    return float(ONE_SIDED_D2[n - 1 - t] @ line[::-1][:6]) / (12.0 * h ** 2)


class Layout:
    def __init__(self, problem):
        self.p = problem
        self.order = problem.order
        self.off, self.ext, self.gh = [], [], []
        o = 0
        for g in problem.grids:
            gh = g.ghosts(problem.order)
            e = (g.n[0] + 2 * gh[0], g.n[1] + 2 * gh[1])
            self.off.append(o)
            self.ext.append(e)
            self.gh.append(gh)
            o += e[0] * e[1]
        self.N = o

    def idx(self, gi, i, j):
        g = self.p.grids[gi]
        gh, e = self.gh[gi], self.ext[gi]
        if g.bc[0] == G.BC_PERIODIC:
            i = i % g.n[0]
        if g.bc[2] == G.BC_PERIODIC:
            j = j % g.n[1]
        assert -gh[0] <= i < g.n[0] + gh[0] and -gh[1] <= j < g.n[1] + gh[1]
        return self.off[gi] + (j + gh[1]) * e[0] + (i + gh[0])


def coefficients(problem, gi):
    """c^2 a11, c^2 a12, c^2 a22, c^2 b1, c^2 b2 on the compact (n1, n0) points."""
    g = problem.grids[gi]
    order = problem.order
    gh = g.ghosts(order)
    rx = g.rx  # (4, e1, e0)
    n0, n1 = g.n
    r = order // 2
    w1 = D1W[order]

    def shifted(a, da, k):
        # value of extended array a at compact points shifted by k along axis da
        if da == 0:
            if g.bc[0] == G.BC_PERIODIC:
                return np.roll(a, -k, axis=1)[gh[1]:gh[1] + n1, :]
            return a[gh[1]:gh[1] + n1, gh[0] + k:gh[0] + k + n0]
        if g.bc[2] == G.BC_PERIODIC:
            return np.roll(a, -k, axis=0)[:, gh[0]:gh[0] + n0]
        return a[gh[1] + k:gh[1] + k + n1, gh[0]:gh[0] + n0]

    def deriv(a, da):
        return sum(w1[k + r] * shifted(a, da, k) for k in range(-r, r + 1)) / g.h[da]

    inner = rx[:, gh[1]:gh[1] + n1, gh[0]:gh[0] + n0]
    # rx index 2k+m = dr_k/dx_m
    a11 = inner[0] ** 2 + inner[1] ** 2
    a12 = inner[0] * inner[2] + inner[1] * inner[3]
    a22 = inner[2] ** 2 + inner[3] ** 2
    b = []
    for k in range(2):
        bk = np.zeros((n1, n0))
        for m in range(2):
            for l in range(2):
                bk += inner[2 * l + m] * deriv(rx[2 * k + m], l)
        b.append(bk)
    c2 = np.ones((n1, n0)) if problem.c2 is None else problem.c2[gi]
    return [c2 * a11, c2 * a12, c2 * a22, c2 * b[0], c2 * b[1]]


def assemble(problem, omega):
    lay = Layout(problem)
    order = problem.order
    r = order // 2
    rows, cols, vals = [], [], []
    rhs = np.zeros(lay.N)
    filled = np.zeros(lay.N, bool)

    def put(row, col, v):
        rows.append(row)
        cols.append(col)
        vals.append(v)

    for gi, g in enumerate(problem.grids):
        n0, n1 = g.n
        c2 = np.ones((n1, n0)) if problem.c2 is None else problem.c2[gi]
        coef = coefficients(problem, gi) if g.kind == G.CURVILINEAR else None
        for j in range(n1):
            for i in range(n0):
                row = lay.idx(gi, i, j)
                m = g.mask[j, i]
                filled[row] = True
                if m == G.DISC:
                    put(row, row, omega ** 2)
                    rhs[row] = problem.f[gi][j, i]
                    if g.kind == G.CARTESIAN:
                        for da in range(2):
                            for k in range(-r, r + 1):
                                ii, jj = (i + k, j) if da == 0 else (i, j + k)
                                put(row, lay.idx(gi, ii, jj),
                                    c2[j, i] * D2W[order][k + r] / g.h[da] ** 2)
                    else:
                        A11, A12, A22, B1, B2 = (c[j, i] for c in coef)
                        for da, (A, B) in enumerate(((A11, B1), (A22, B2))):
                            for k in range(-r, r + 1):
                                ii, jj = (i + k, j) if da == 0 else (i, j + k)
                                put(row, lay.idx(gi, ii, jj),
                                    A * D2W[order][k + r] / g.h[da] ** 2
                                    + B * D1W[order][k + r] / g.h[da])
                        if not g.orthogonal:
                            for k in range(-r, r + 1):
                                for l in range(-r, r + 1):
                                    wgt = D1W[order][k + r] * D1W[order][l + r]
                                    if wgt != 0.0:
                                        put(row, lay.idx(gi, i + k, j + l),
                                            2.0 * A12 * wgt / (g.h[0] * g.h[1]))
                elif m == G.INTERP:
                    put(row, row, 1.0)
                else:  # Dirichlet or unused
                    put(row, row, 1.0)
                    gb = getattr(problem, "g", None)
                    if m == G.DIRICHLET and gb is not None and gb[gi] is not None:
                        rhs[row] = gb[gi][j, i]
        # ghost rules
        for s in range(4):
            code = g.bc[s]
            if code not in (G.BC_DIRICHLET, G.BC_NEUMANN):
                continue
            a, hi = s // 2, s % 2
            nt = g.n[1 - a]
            for t in range(nt):
                def pt(k):
                    nrm = g.n[a] - 1 - k if hi else k
                    return lay.idx(gi, nrm, t) if a == 0 else lay.idx(gi, t, nrm)
                bi, bj = ((g.n[0] - 1 if hi else 0), t) if a == 0 else (t, (g.n[1] - 1 if hi else 0))
                m = g.mask[bj, bi]
                if code == G.BC_NEUMANN and m != G.DISC:
                    continue
                if code == G.BC_DIRICHLET and (m != G.DIRICHLET or order == 2):
                    continue
                gq = [pt(-k) for k in range(1, r + 1)]
                U = [pt(k) for k in range(4)]
                # Neumann data dU/dn = gn (outward unit normal -+ grad r_a / |grad r_a|):
                # |grad r_a| = sqrt(a_aa) without c^2 (1 on Cartesian grids)
                gnv = 0.0
                gns = getattr(problem, "gn", None)
                if code == G.BC_NEUMANN and gns is not None and gns[gi] is not None:
                    gnv = gns[gi][bj, bi]
                a_geo = 1.0 if g.kind == G.CARTESIAN else \
                    coef[0 if a == 0 else 2][bj, bi] / c2[bj, bi]
                if code == G.BC_NEUMANN and order == 2:
                    # grad r_a . grad U = a_aa U_{r_a} + a_at U_{r_t} = -+ gn |grad r_a| with
                    # centred differences (rows scaled by c^2 on curvilinear grids); a_at = 0
                    # on orthogonal grids (U_{-1} - U_{+1} = 0 without data)
                    ann, ant, scale = 1.0, 0.0, 1.0
                    if g.kind == G.CURVILINEAR:
                        ann, scale = coef[0 if a == 0 else 2][bj, bi], c2[bj, bi]
                        if not g.orthogonal:
                            ant = coef[1][bj, bi]
                    sg = -1.0 if hi else 1.0  # +r_a points inward on a low side
                    put(gq[0], gq[0], sg * -ann / (2 * g.h[a]))
                    put(gq[0], U[1], sg * ann / (2 * g.h[a]))
                    rhs[gq[0]] = -sg * scale * gnv * np.sqrt(a_geo)
                    if ant != 0.0:
                        ta = 1 - a
                        for dt_, wgt in ((1, 1.0), (-1, -1.0)):
                            tt = t + dt_
                            col = lay.idx(gi, bi, tt) if a == 0 else lay.idx(gi, tt, bj)
                            put(gq[0], col, wgt * ant / (2 * g.h[ta]))
                    filled[gq[0]] = True
                    continue
                # second row: fifth-order extrapolation of G2
                for c_, col in zip(EXTRAP5, [gq[1], gq[0]] + U):
                    put(gq[1], col, c_)
                filled[gq[1]] = True
                filled[gq[0]] = True
                if code == G.BC_NEUMANN:
                    # fourth-order centred derivative along the inward normal line
                    # (undivided) = -12 h gn / |grad r_a|
                    for c_, col in zip([1.0, -8.0, 8.0, -1.0], [gq[1], gq[0], U[1], U[2]]):
                        put(gq[0], col, c_)
                    rhs[gq[0]] = -12.0 * g.h[a] * gnv / np.sqrt(a_geo)
                else:
                    if g.kind == G.CARTESIAN:
                        ann, bn = c2[bj, bi], 0.0
                    else:
                        ann, bn = coef[0 if a == 0 else 2][bj, bi], coef[3 + a][bj, bi]
                    h = g.h[a]
                    # points ordered by +r_n coordinate: offsets -2..2 from the boundary
                    seq = [gq[1], gq[0], U[0], U[1], U[2]] if not hi else [U[2], U[1], U[0], gq[0], gq[1]]
                    for k, col in enumerate(seq):
                        put(gq[0], col, ann * D2W[4][k] / h ** 2 + bn * D1W[4][k] / h)
                    rhs[gq[0]] = problem.f[gi][bj, bi]
                    gb = getattr(problem, "g", None)
                    if gb is not None and gb[gi] is not None:
                        assert g.kind == G.CARTESIAN
                        line = gb[gi][:, bi] if a == 0 else gb[gi][bj, :]
                        per = g.bc[2 * (1 - a)] == G.BC_PERIODIC
                        rhs[gq[0]] -= omega ** 2 * gb[gi][bj, bi] + \
                            c2[bj, bi] * side_d2(line, t, per, g.h[1 - a])
    # interpolation rows
    it = problem.interp
    w = order + 1
    for k in range(it.n):
        row = lay.idx(int(it.recv_grid[k]), int(it.recv_i[k]), int(it.recv_j[k]))
        dg = int(it.donor_grid[k])
        for bb in range(w):
            for aa in range(w):
                put(row, lay.idx(dg, int(it.donor_i0[k]) + aa, int(it.donor_j0[k]) + bb),
                    -it.wx[k, aa] * it.wy[k, bb])
    # everything not yet given a row: U = 0
    for q in np.nonzero(~filled)[0]:
        put(q, q, 1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(lay.N, lay.N))
    return A, rhs, lay


def solve(problem, omega=None):
    """Direct sparse solve; returns the concatenated compact solution vector."""
    omega = problem.omega if omega is None else omega
    A, rhs, lay = assemble(problem, omega)
    lu = spla.splu(A.tocsc())
    U = lu.solve(rhs)
    # one step of iterative refinement: on grids with very small cells (the knife edge's
    # tip) the factorization alone leaves errors near 1e-10
    U = U + lu.solve(rhs - A @ U)
    out = []
    for gi, g in enumerate(problem.grids):
        e, gh = lay.ext[gi], lay.gh[gi]
        blk = U[lay.off[gi]:lay.off[gi] + e[0] * e[1]].reshape(e[1], e[0])
        out.append(blk[gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]].ravel())
    return np.concatenate(out)


def adjoint_gradients(problem, P, d, omega=None):
    """Gradients of J = 0.5 |P U - d|^2 for the direct discrete solution U with respect to
    c^2 and f at every grid point, by the transpose solve of the assembled system
    (independent of the WaveHoltz code):  A^T mu = E^T P^T (P U - d), and
      dJ/d c2_p = -sum_rows mu_r (dA/dc2_p U)_r,  dJ/d f_p = sum_rows mu_r d rhs_r / d f_p.
    Rows that scale with c2_p: the discretization row of p (its c^2 L_h part) and the
    compatibility ghost rows of a Dirichlet boundary point p (order 4).  Returns
    (U, J, grad_c2, grad_f) as compact vectors."""
    omega = problem.omega if omega is None else omega
    A, rhs, lay = assemble(problem, omega)
    lu = spla.splu(A.tocsc())
    Uext = lu.solve(rhs)
    # compact <-> extended maps
    idx = []
    for gi, g in enumerate(problem.grids):
        for j in range(g.n[1]):
            for i in range(g.n[0]):
                idx.append(lay.idx(gi, i, j))
    idx = np.array(idx)
    U = Uext[idx]
    r = P @ U - d
    J = 0.5 * float(r @ r)
    src = np.zeros(lay.N)
    src[idx] = P.T @ r
    mu = lu.solve(src, trans="T")
    AU = A @ Uext
    # which rows scale with which point's c^2, and which rows carry f
    n = len(idx)
    gc2 = np.zeros(n)
    gf = np.zeros(n)
    comp = {}  # extended index of a compact point -> compact position
    for k, q in enumerate(idx):
        comp[q] = k
    c2 = None if problem.c2 is None else np.concatenate([c.ravel() for c in problem.c2])
    off = 0
    for gi, g in enumerate(problem.grids):
        for j in range(g.n[1]):
            for i in range(g.n[0]):
                k = off + j * g.n[0] + i
                q = idx[k]
                c2p = 1.0 if c2 is None else c2[k]
                if g.mask[j, i] == G.DISC:
                    gc2[k] -= mu[q] * (AU[q] - omega ** 2 * Uext[q]) / c2p
                    gf[k] += mu[q]
        # Dirichlet order-4 compatibility rows: ghost G1 row of boundary point b
        if problem.order == 4:
            for s_ in range(4):
                if g.bc[s_] != G.BC_DIRICHLET:
                    continue
                a, hi = s_ // 2, s_ % 2
                for t in range(g.n[1 - a]):
                    bi, bj = ((g.n[0] - 1 if hi else 0), t) if a == 0 else (t, (g.n[1] - 1 if hi else 0))
                    if g.mask[bj, bi] != G.DIRICHLET:
                        continue
                    gpos = lay.idx(gi, bi - 1 if (a == 0 and not hi) else (bi + 1 if a == 0 else bi),
                                   bj - 1 if (a == 1 and not hi) else (bj + 1 if a == 1 else bj))
                    k = off + bj * g.n[0] + bi
                    c2p = 1.0 if c2 is None else c2[k]
                    gc2[k] -= mu[gpos] * AU[gpos] / c2p
                    gf[k] += mu[gpos]
        off += g.npts
    return U, J, gc2, gf
