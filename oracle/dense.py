"""Direct solve of the discrete steady BTE (TEST INFRASTRUCTURE ONLY).

The source iteration of the paper (Methods, solution procedure) converges to
the unique solution of one *linear* system in the unknowns e_{c,b,d}
(solid cells c, bands b, directions d), once the lattice temperature is
eliminated as the linear functional T = W e of Eq. (updatee0_t):

    (L - P W - R) e = s

* L  -- per (b, d) the finite-volume upwind transport operator plus the
        1/tau term: the matrix A of Eq. (A_matrix) with S_ij/V_i = 1/h on a
        uniform Cartesian grid;
* P W e -- the re-emission C_b T_c / (4 pi tau_cb) of Eq. (bte-2);
* R  -- diffuse reflection (Boundary conditions: diffusely reflecting
        boundary) with the quadrature-consistent normaliser
        sum_{s.n<0} w |s.n| in place of pi, and specular reflection at
        domain faces of that type: the inflow of direction d is the
        outgoing value of the mirror direction (normal component reversed)
        in the same cell;
* s  -- per-band source Q_b phi_c (Q_b = C_b Q/(4 pi sum C)) plus the
        isothermal inflow v |s.n| C_b T_w / (4 pi h).

This module assembles that system as a sparse matrix and solves it with
scipy's direct sparse LU: the plain definition, for small grids only.  It is
written independently of the C sweep code (rows are assembled here; no
sweep order is involved).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

FOUR_PI = 4.0 * np.pi


class System:
    def __init__(self, p):
        self.p = p
        nx, ny, nz = p.n
        N = nx * ny * nz
        self.active = np.flatnonzero(p.mask)
        self.rank = -np.ones(N, dtype=np.int64)
        self.rank[self.active] = np.arange(self.active.size)
        self.B, self.D = p.B, p.D
        self.n_unknowns = self.active.size * p.B * p.D
        h = [p.length[a] / p.n[a] for a in range(3)]
        self.h = h
        self.tau_cb = np.zeros((N, p.B))
        for c in self.active:
            self.tau_cb[c] = p.tau * p.tau_scale[p.mask[c] - 1]
        self.K = np.zeros(N)
        self.K[self.active] = (p.C[None, :] / self.tau_cb[self.active]).sum(axis=1)
        self._assemble()

    def u(self, c, b, d):
        return (self.rank[c] * self.B + b) * self.D + d

    def coords(self, c):
        nx, ny, _ = self.p.n
        return [c % nx, (c // nx) % ny, c // (nx * ny)]

    def neighbour(self, c, side):
        idx = self.coords(c)
        a = side // 2
        idx[a] += 1 if side % 2 else -1
        if idx[a] < 0 or idx[a] >= self.p.n[a]:
            return -1
        nx, ny, _ = self.p.n
        return idx[0] + nx * (idx[1] + ny * idx[2])

    def _assemble(self):
        p = self.p
        rows, cols, vals = [], [], []
        rhs = np.zeros(self.n_unknowns)
        Csum = p.C.sum()
        # W: T_c = sum_{b,d} w_d e_cbd / (tau_cb K_c)
        wr, wc, wv = [], [], []
        for c in self.active:
            for b in range(p.B):
                for d in range(p.D):
                    wr.append(self.rank[c])
                    wc.append(self.u(c, b, d))
                    wv.append(p.w[d] / (self.tau_cb[c, b] * self.K[c]))
        self.W = sp.csr_matrix((wv, (wr, wc)), shape=(self.active.size, self.n_unknowns))
        # mirror[a][d]: the direction with component a reversed
        mirror = np.full((3, p.D), -1, dtype=np.int64)
        for a in range(3):
            want = p.s.copy()
            want[:, a] *= -1.0
            for d in range(p.D):
                hit = np.flatnonzero(np.abs(p.s - want[d]).sum(axis=1) < 1e-12)
                if hit.size:
                    mirror[a, d] = hit[0]
        norm = {}
        for side in range(6):
            a, sg = side // 2, (1.0 if side % 2 else -1.0)
            sn = p.s[:, a] * sg
            norm[side] = np.sum(p.w[sn < 0] * np.abs(sn[sn < 0]))
        for c in self.active:
            for b in range(p.B):
                tcb = self.tau_cb[c, b]
                for d in range(p.D):
                    r = self.u(c, b, d)
                    diag = 1.0 / tcb
                    if p.phi is not None:
                        rhs[r] += p.C[b] * p.Q_amp * p.phi[c] / (FOUR_PI * Csum)
                    for a in range(p.dim):
                        sa = p.s[d, a]
                        if sa == 0.0:
                            continue
                        coef = p.v[b] * abs(sa) / self.h[a]
                        diag += coef
                        side = 2 * a if sa > 0 else 2 * a + 1   # face it enters by
                        m = self.neighbour(c, side)
                        if m >= 0 and p.mask[m]:
                            rows.append(r); cols.append(self.u(m, b, d)); vals.append(-coef)
                        elif m < 0 and p.bc_type[side] == 0:
                            rhs[r] += coef * p.C[b] * p.bc_T[side] / FOUR_PI
                        elif m < 0 and p.bc_type[side] == 2:
                            if mirror[a, d] < 0:
                                raise ValueError("specular face without the mirror direction")
                            rows.append(r); cols.append(self.u(c, b, mirror[a, d])); vals.append(-coef)
                        else:
                            sg = 1.0 if side % 2 else -1.0
                            for d2 in range(p.D):
                                sn = p.s[d2, a] * sg
                                if sn > 0:
                                    rows.append(r); cols.append(self.u(c, b, d2))
                                    vals.append(-coef * p.w[d2] * sn / norm[side])
                    rows.append(r); cols.append(r); vals.append(diag)
                    # - P W: re-emission C_b T_c / (4 pi tau_cb)
                    pre = p.C[b] / (FOUR_PI * tcb)
                    for b2 in range(p.B):
                        for d2 in range(p.D):
                            rows.append(r); cols.append(self.u(c, b2, d2))
                            vals.append(-pre * p.w[d2] / (self.tau_cb[c, b2] * self.K[c]))
        self.A = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_unknowns, self.n_unknowns))
        self.s = rhs

    def unpack(self, x):
        p = self.p
        out = np.zeros((p.n_cells, p.B, p.D))
        out[self.active] = x.reshape(self.active.size, p.B, p.D)
        return out

    def solve(self):
        x = spla.spsolve(self.A.tocsc(), self.s)
        T = np.zeros(self.p.n_cells)
        T[self.active] = self.W @ x
        return dict(e=self.unpack(x), T=T, x=x)

    def adjoint(self, g):
        """Solve (L - P W - R)^T mu = W^T g directly."""
        rhs = self.W.T @ g[self.active]
        mu = spla.spsolve(self.A.T.tocsc(), rhs)
        return self.unpack(mu)


def solve(p):
    return System(p).solve()


def loss_probe(T, probes, T_obs):
    d = T[probes] - T_obs
    return 0.5 * float(d @ d)


def fd_gradients(p, probes, T_obs, rel: float = 1e-6, dTw: float = 1e-3):
    """Central differences of J = 1/2 sum_p (T_p - T_obs)^2 through the direct
    solve, w.r.t. tau_b, the isothermal wall temperatures and Q_amp."""
    def J(q):
        return loss_probe(System(q).solve()["T"], probes, T_obs)

    g_tau = np.zeros(p.B)
    for b in range(p.B):
        hb = rel * p.tau[b]
        tp, tm = p.tau.copy(), p.tau.copy()
        tp[b] += hb
        tm[b] -= hb
        g_tau[b] = (J(p.copy(tau=tp)) - J(p.copy(tau=tm))) / (2 * hb)
    g_Tw = np.zeros(6)
    for f in range(6):
        if f // 2 >= p.dim or p.bc_type[f] != 0:
            continue
        Tp, Tm = p.bc_T.copy(), p.bc_T.copy()
        Tp[f] += dTw
        Tm[f] -= dTw
        g_Tw[f] = (J(p.copy(bc_T=Tp)) - J(p.copy(bc_T=Tm))) / (2 * dTw)
    g_Q = 0.0
    if p.phi is not None and p.Q_amp != 0.0:
        hq = rel * p.Q_amp
        g_Q = (J(p.copy(Q_amp=p.Q_amp + hq)) - J(p.copy(Q_amp=p.Q_amp - hq))) / (2 * hq)
    return dict(g_tau=g_tau, g_Tw=g_Tw, g_Q=g_Q)
