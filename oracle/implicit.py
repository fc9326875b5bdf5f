"""WaveHoltz iteration with implicit time-stepping -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this module.  It follows the paper's implicit variant (the scheme of Eq. implicitScheme,
the corrected form Eq. WaveSchemeImplicit / waveImplicitOrder2, Recipe
OmegaTildeImplicit) on the two-dimensional overset grids of ``oracle.oracle`` and the
three-dimensional ones of ``oracle.oracle3``, whose C pieces (the mapped Laplacian
``apply_lap``, the ghost rules ``apply_bc``, the overset ``interpolate``) serve as its
steps.  Nothing here comes from the CUDA library.

What it computes (one iteration v -> W_h(v, f)):

* time setup (Recipe OmegaTildeImplicit): N_t >= 5 steps per period,
  dt = (1/omega) sqrt(2 / cos(2 pi / N_t) - 2), omega_i = 2 pi / (N_t dt), so that
  cos(omega_i dt) = 1 / (1 + (omega dt)^2 / 2) (Eq. cosOmegaTilde); M = N_p N_t steps; the
  filter parameter alpha_d = tan(omega_i dt / 2) / tan(omega_i dt) (Eq. alphad with the
  filter frequency omega_i);
* the scheme D+tD-t W^n = (1/2) L_h (W^{n+1} + W^{n-1}) - f cos(omega_i t^n) cos(omega_i dt)
  at discretization points, i.e. with A = I - (dt^2 / 2) L_h
      A W^{n+1} = 2 W^n - A W^{n-1} - dt^2 cos(omega_i dt) cos(omega_i t^n) f ;
  the first step is implicit too (the paper asks for it with a large dt): D0t W^0 = 0 gives
  W^{-1} = W^1 and so A W^1 = W^0 - (dt^2 / 2) cos(omega_i dt) f;
* each implicit system holds, besides those rows, the level's boundary conditions and the
  interpolation equations (Sec. 3.2: "a sparse linear system ... representing the interior
  equations on all component grids, as well as equations for the boundary conditions and
  the interpolation between grids"): ghost points satisfy the ghost rules of the explicit
  oracle at time t^{n+1} (their forcing term scaled by cos(omega_i t^{n+1})), receivers their
  interpolation formula, Dirichlet points W = 0 and every other point W = 0.  The rows come
  from probing the oracle's pieces with unit vectors (each piece is affine; its linear part
  is read column by column); the system is solved with a sparse LU (the paper's direct
  sparse solver option);
* level 0: W^0 = v at discretization and interpolation points, then the ghost rules and
  the interpolation at t = 0, as in the explicit oracle;
* the trapezoid time filter of the explicit oracle with omega_i and T-bar = M dt.

Readings (where the paper defers to its reference): the ghost conditions of level n + 1 use
the forcing factor cos(omega_i t^{n+1}), so that W^n = U cos(omega_i t^n) with U the
discrete Helmholtz solution is a solution of the scheme; Dirichlet boundary data g != 0 are
not taken.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .oracle import Oracle

DISC, INTERP, DIRICHLET, UNUSED = 1, 2, 3, 0


def implicit_time_setup(omega, n_its, periods=1):
    """Recipe OmegaTildeImplicit with N_t = n_its steps per period; alpha_d of Eq. alphad."""
    if n_its < 5:
        raise ValueError("implicit time-stepping needs at least 5 steps per period")
    dt = math.sqrt(2.0 / math.cos(2.0 * math.pi / n_its) - 2.0) / omega
    omega_i = 2.0 * math.pi / (n_its * dt)
    return {"dt": dt, "omega_i": omega_i, "Nt": n_its, "M": periods * n_its,
            "alpha": math.tan(omega_i * dt / 2.0) / math.tan(omega_i * dt),
            "c1": math.cos(omega_i * dt), "periods": periods}


def lambda_implicit(lam_h, dt):
    """Eq. lambdaTildeImplicit: (1/dt) arccos(1 / (1 + (lambda dt)^2 / 2))."""
    return np.arccos(1.0 / (1.0 + (np.asarray(lam_h) * dt) ** 2 / 2.0)) / dt


class ImplicitOracle:
    """The implicit WaveHoltz map on one overset problem (``grids.Problem`` in two
    dimensions, ``grids3.Problem3`` in three)."""

    def __init__(self, problem, n_its=10, periods=1):
        gb = getattr(problem, "g", None)
        if gb is not None and any(x is not None and np.any(x != 0) for x in gb):
            raise ValueError("Dirichlet boundary data are not taken with implicit time-stepping")
        self.problem = problem
        # the operator pieces (their own time setup is not used): the 2D oracle, or the 3D
        # one for a three-dimensional problem (interpolation with a third index)
        self.dim = 3 if hasattr(problem.interp, "recv_k") else 2
        if self.dim == 3:
            from .oracle3 import Oracle3
            self.orc = Oracle3(problem)
        else:
            self.orc = Oracle(problem)
        self.time = implicit_time_setup(problem.omega, n_its, periods)
        self._layout()
        self._assemble()

    def _interior(self, gi):
        """The slice of grid gi's points in its extended (ghosted) array."""
        g, gh = self.problem.grids[gi], self.gh[gi]
        return tuple(slice(gh[a], gh[a] + g.n[a]) for a in reversed(range(self.dim)))

    # ---------------------------------------------------------------- layout
    def _layout(self):
        self.shapes, self.offs, self.gh, self.mask_ext = [], [], [], []
        o = 0
        for gi, g in enumerate(self.problem.grids):
            sh = self.orc.ext_shape(gi)
            gh = g.ghosts(self.problem.order)
            self.shapes.append(sh)
            self.offs.append(o)
            self.gh.append(gh)
            m = np.full(sh, UNUSED, np.int8)
            m[self._interior(gi)] = g.mask
            self.mask_ext.append(m)
            o += int(np.prod(sh))
        self.N = o
        self.mask = np.concatenate([m.ravel() for m in self.mask_ext])

    def _split(self, w):
        return [w[o:o + int(np.prod(s))].reshape(s).copy() for o, s in zip(self.offs, self.shapes)]

    def _join(self, ws):
        return np.concatenate([w.ravel() for w in ws])

    # ------------------------------------------------------------- assembly
    def _assemble(self):
        """Linear parts of L_h (discretization rows) and of the constraint map (ghost rules,
        then interpolation), column by column; the affine part of the ghost rules per unit
        forcing factor; the level matrix A."""
        rng = np.random.default_rng(0)
        ng = len(self.problem.grids)
        # ghost points the rules write: the entries apply_bc changes in a random array
        ghost = np.zeros(self.N, bool)
        aff = np.zeros(self.N)
        for gi in range(ng):
            r = rng.standard_normal(self.shapes[gi])
            changed = self.orc.apply_bc(gi, r, 0.0) != r
            o = self.offs[gi]
            ghost[o:o + r.size] = changed.ravel()
            aff[o:o + r.size] = self.orc.apply_bc(gi, np.zeros(self.shapes[gi]), 1.0).ravel()
        it = self.problem.interp
        recv = np.zeros(self.N, bool)
        idx = [it.recv_i, it.recv_j] + ([it.recv_k] if self.dim == 3 else [])
        for q in range(it.n):
            gi = int(it.recv_grid[q])
            gh = self.gh[gi]
            ijk = [int(idx[a][q]) + gh[a] for a in range(self.dim)]
            recv[self.offs[gi] + int(np.ravel_multi_index(tuple(reversed(ijk)),
                                                          self.shapes[gi]))] = True
        if np.any(ghost & recv):
            raise ValueError("a point is both a ghost and a receiver")
        self.ghost, self.recv = ghost, recv
        self.aff = np.where(ghost, aff, 0.0)
        disc = self.mask == DISC
        self.disc = disc
        Lr, Lc, Lv, Cr, Cc, Cv = [], [], [], [], [], []
        for gi in range(ng):
            o, sh = self.offs[gi], self.shapes[gi]
            size = int(np.prod(sh))
            d_loc = disc[o:o + size]
            g_loc = ghost[o:o + size]
            for j in range(size):
                e = np.zeros(size)
                e[j] = 1.0
                lap = self.orc.apply_lap(gi, e.reshape(sh)).ravel()
                nz = np.nonzero(d_loc & (lap != 0.0))[0]
                Lr.append(o + nz)
                Lc.append(np.full(nz.size, o + j))
                Lv.append(lap[nz])
                bc = self.orc.apply_bc(gi, e.reshape(sh), 0.0).ravel()
                nz = np.nonzero(g_loc & (bc != 0.0))[0]
                Cr.append(o + nz)
                Cc.append(np.full(nz.size, o + j))
                Cv.append(bc[nz])
                if it.n:
                    us = [np.zeros(s) for s in self.shapes]
                    us[gi] = e.reshape(sh)
                    out = self._join(self.orc.interpolate(us))
                    nz = np.nonzero(recv & (out != 0.0))[0]
                    Cr.append(nz)
                    Cc.append(np.full(nz.size, o + j))
                    Cv.append(out[nz])
        cat = np.concatenate
        self.L = sp.csr_matrix((cat(Lv), (cat(Lr), cat(Lc))), shape=(self.N, self.N))
        C = sp.csr_matrix((cat(Cv), (cat(Cr), cat(Cc))), shape=(self.N, self.N))
        dt = self.time["dt"]
        I = sp.identity(self.N, format="csr")
        # discretization rows: I - dt^2/2 L; constraint rows: I - C; all other rows: I
        self.A = (I - 0.5 * dt * dt * self.L - C).tocsc()
        self.lu = spla.splu(self.A)
        self.f = self._join([np.pad(f, [(gh[a], gh[a]) for a in reversed(range(self.dim))])
                             for f, gh in zip(self.problem.f, self.gh)])

    # ------------------------------------------------------------- the map
    def _initial(self, v, fs):
        ws = []
        o = 0
        for gi, g in enumerate(self.problem.grids):
            w = np.zeros(self.shapes[gi])
            vg = v[o:o + g.mask.size].reshape(g.mask.shape)
            keep = (g.mask == DISC) | (g.mask == INTERP)
            w[self._interior(gi)] = np.where(keep, vg, 0.0)
            ws.append(self.orc.apply_bc(gi, w, fs))
            o += g.mask.size
        return self._join(self.orc.interpolate(ws))

    def _rhs_constraints(self, fcos):
        return self.aff * fcos

    def iterate(self, v, forcing=True):
        T = self.time
        dt, wi, M, c1, alpha = T["dt"], T["omega_i"], T["M"], T["c1"], T["alpha"]
        fs = 1.0 if forcing else 0.0
        active = self.mask != UNUSED

        def wf(n):  # (2 / T-bar) sigma_n dt (cos(omega_i t^n) - alpha/2)
            sig = 0.5 if n in (0, M) else 1.0
            return 2.0 / (M * dt) * sig * dt * (math.cos(wi * n * dt) - alpha / 2.0)

        W0 = self._initial(np.asarray(v, np.float64), fs)
        V = np.where(active, wf(0) * W0, 0.0)
        disc = self.disc
        rhs = self._rhs_constraints(fs * math.cos(wi * dt))
        rhs[disc] = W0[disc] - 0.5 * dt * dt * c1 * fs * self.f[disc]
        W1 = self.lu.solve(rhs)
        Wm, Wc = W0, W1
        for n in range(1, M):
            V += np.where(active, wf(n) * Wc, 0.0)
            AWm = Wm - 0.5 * dt * dt * (self.L @ Wm)
            rhs = self._rhs_constraints(fs * math.cos(wi * (n + 1) * dt))
            rhs[disc] = (2.0 * Wc[disc] - AWm[disc] -
                         dt * dt * c1 * fs * math.cos(wi * n * dt) * self.f[disc])
            Wm, Wc = Wc, self.lu.solve(rhs)
        V += np.where(active, wf(M) * Wc, 0.0)
        out = []
        for gi, g in enumerate(self.problem.grids):
            Vg = V[self.offs[gi]:self.offs[gi] + int(np.prod(self.shapes[gi]))]
            out.append(Vg.reshape(self.shapes[gi])[self._interior(gi)].ravel())
        return np.concatenate(out)

    # the spatial operator's pieces (the same as the explicit oracle's): for the
    # eigenvalues lambda^2 of a deflation set
    def ext_shape(self, gi):
        return self.orc.ext_shape(gi)

    def apply_bc(self, gi, u_ext, fcos):
        return self.orc.apply_bc(gi, u_ext, fcos)

    def apply_lap(self, gi, u_ext):
        return self.orc.apply_lap(gi, u_ext)

    def zeros(self):
        return np.zeros(self.problem.n_total)

    def active(self):
        return np.concatenate([(g.mask != 0).ravel() for g in self.problem.grids])
