"""Brute-force assembly of the three-dimensional discrete Helmholtz system (DHS) on
Cartesian overset grids, for pinning the 3D oracle.

The converged WaveHoltz iterate equals the direct solution of (Sec. 6, App. B.1)

    c^2 (D+D-_x + D+D-_y + D+D-_z) U + omega^2 U = f   at discretization points,
    U = 0                                              at Dirichlet boundary points,
    U - sum w U_donor = 0                              at interpolation points,
    U_ghost - U_inward = 0                             at Neumann ghost points,
    U = 0                                              everywhere else.

The rows come from the textbook 7-point stencil, independently of the oracle's C code, and
are solved with a sparse LU.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2504_03074_gb300 import grids as G


class Layout3:
    def __init__(self, problem):
        self.p = problem
        self.off, self.ext, self.gh = [], [], []
        o = 0
        for g in problem.grids:
            gh = g.ghosts()
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
    rows, cols, vals = [], [], []
    rhs = np.zeros(L.N)
    done = np.zeros(L.N, bool)

    def put(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for gi, g in enumerate(problem.grids):
        assert g.kind == G.CARTESIAN
        c2 = np.ones(g.mask.shape) if problem.c2 is None else problem.c2[gi]
        for k in range(g.n[2]):
            for j in range(g.n[1]):
                for i in range(g.n[0]):
                    m = g.mask[k, j, i]
                    r = L.idx(gi, i, j, k)
                    done[r] = True
                    if m == G.DISC:
                        diag = om2
                        for a in range(3):
                            w = c2[k, j, i] / g.h[a] ** 2
                            for s in (-1, 1):
                                d = [0, 0, 0]
                                d[a] = s
                                put(r, L.idx(gi, i + d[0], j + d[1], k + d[2]), w)
                            diag -= 2 * w
                        put(r, r, diag)
                        rhs[r] = problem.f[gi][k, j, i]
                    elif m != G.INTERP:
                        put(r, r, 1.0)
                        gb = getattr(problem, "g", None)
                        if m == G.DIRICHLET and gb is not None and gb[gi] is not None:
                            rhs[r] = gb[gi][k, j, i]  # U = g at Dirichlet points
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
    it = problem.interp
    for q in range(it.n):
        r = L.idx(int(it.recv_grid[q]), int(it.recv_i[q]), int(it.recv_j[q]), int(it.recv_k[q]))
        put(r, r, 1.0)
        dg = int(it.donor_grid[q])
        for c in range(3):
            for b in range(3):
                for a in range(3):
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
    U = spla.spsolve(A.tocsc(), rhs)
    out = []
    for gi, g in enumerate(problem.grids):
        gh, e = L.gh[gi], L.ext[gi]
        Ue = U[L.off[gi]:L.off[gi] + e[0] * e[1] * e[2]].reshape(e[2], e[1], e[0])
        out.append(Ue[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]].ravel())
    return np.concatenate(out)
