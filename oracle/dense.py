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

With ``problem.order == 2`` the face values are the second-order ones of
"Spatial discretization" (upwind cell value plus its Green-Gauss gradient
times the centre-to-face vector), with the boundary readings of the oracle's
C source: Green-Gauss face value = inflow value where the direction enters a
boundary face, linear extrapolation from the neighbour where it leaves, no
gradient along an axis without a neighbour; reconstructed outgoing values
also in the reflections.  Every face value is assembled here as an explicit
linear combination of the unknowns, so the system is that scheme's plain
definition, which the deferred-correction iteration must reach.

``transient_step`` solves one implicit-Euler step (L + I/dt - P W - R) e =
s + e_prev/dt directly.
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
        self.mirror, self.norm = mirror, norm
        if getattr(p, "order", 1) == 2:
            self._assemble_order2()
            return
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

    # --- second-order faces: face values as {unknown: coefficient} + constant

    def _lin_add(self, acc, lin, scale):
        terms, const = lin
        for k, v in terms.items():
            acc[0][k] = acc[0].get(k, 0.0) + scale * v
        acc[1] += scale * const

    def _side_kind(self, c, side):
        """0 interior, 1 isothermal wall, 2 diffuse (wall or void), 3 specular wall."""
        p = self.p
        m = self.neighbour(c, side)
        if m < 0:
            t = p.bc_type[side]
            return 1 if t == 0 else (3 if t == 2 else 2)
        return 0 if p.mask[m] else 2

    def _inflow(self, c, b, d, side):
        """Boundary inflow value of (c, b, d) through `side` (second-order)."""
        p = self.p
        a = side // 2
        kind = self._side_kind(c, side)
        if kind == 1:
            return ({}, p.C[b] * p.bc_T[side] / FOUR_PI)
        if kind == 3:
            m = self.mirror[a, d]
            acc = [{self.u(c, b, m): 1.0}, 0.0]
            self._lin_add(acc, self._delta(c, b, m, a), 1.0)
            return (acc[0], acc[1])
        sg = 1.0 if side % 2 else -1.0
        acc = [{}, 0.0]
        for d2 in range(p.D):
            sn = p.s[d2, a] * sg
            if sn > 0:
                wgt = p.w[d2] * sn / self.norm[side]
                self._lin_add(acc, ({self.u(c, b, d2): 1.0}, 0.0), wgt)
                self._lin_add(acc, self._delta(c, b, d2, a), wgt)
        return (acc[0], acc[1])

    def _delta(self, c, b, d, a):
        """Reconstruction increment sign(s_a) h_a/2 grad_a e of (c, b, d)."""
        key = (c, b, d, a)
        if key in self._dcache:
            return self._dcache[key]
        p = self.p
        sa = p.s[d, a]
        out = ({}, 0.0)
        if sa != 0.0:
            side_in = 2 * a if sa > 0 else 2 * a + 1
            kinds = [self._side_kind(c, 2 * a), self._side_kind(c, 2 * a + 1)]
            if kinds[0] == 0 or kinds[1] == 0:
                G = []
                for sd in range(2):
                    side = 2 * a + sd
                    if kinds[sd] == 0:
                        nb = self.neighbour(c, side)
                        G.append(({self.u(c, b, d): 0.5, self.u(nb, b, d): 0.5}, 0.0))
                    elif side == side_in:
                        G.append(self._inflow(c, b, d, side))
                    else:
                        nb = self.neighbour(c, side ^ 1)
                        G.append(({self.u(c, b, d): 1.5, self.u(nb, b, d): -0.5}, 0.0))
                acc = [{}, 0.0]
                f = (1.0 if sa > 0 else -1.0) * 0.5   # sign(s_a) h/2 * (G+ - G-)/h
                self._lin_add(acc, G[1], f)
                self._lin_add(acc, G[0], -f)
                out = (acc[0], acc[1])
        self._dcache[key] = out
        return out

    def _assemble_order2(self):
        p = self.p
        self._dcache = {}
        rows, cols, vals = [], [], []
        rhs = np.zeros(self.n_unknowns)
        Csum = p.C.sum()
        for c in self.active:
            for b in range(p.B):
                tcb = self.tau_cb[c, b]
                for d in range(p.D):
                    r = self.u(c, b, d)
                    eq = [{r: 1.0 / tcb}, 0.0]   # left-hand side terms, constant moved right
                    if p.phi is not None:
                        rhs[r] += p.C[b] * p.Q_amp * p.phi[c] / (FOUR_PI * Csum)
                    for a in range(p.dim):
                        sa = p.s[d, a]
                        if sa == 0.0:
                            continue
                        coef = p.v[b] * abs(sa) / self.h[a]
                        side_in = 2 * a if sa > 0 else 2 * a + 1
                        # + coef * F_out
                        self._lin_add(eq, ({r: 1.0}, 0.0), coef)
                        self._lin_add(eq, self._delta(c, b, d, a), coef)
                        # - coef * F_in
                        m = self.neighbour(c, side_in)
                        if m >= 0 and p.mask[m]:
                            self._lin_add(eq, ({self.u(m, b, d): 1.0}, 0.0), -coef)
                            self._lin_add(eq, self._delta(m, b, d, a), -coef)
                        else:
                            self._lin_add(eq, self._inflow(c, b, d, side_in), -coef)
                    pre = p.C[b] / (FOUR_PI * tcb)
                    for b2 in range(p.B):
                        for d2 in range(p.D):
                            k = self.u(c, b2, d2)
                            eq[0][k] = eq[0].get(k, 0.0) - pre * p.w[d2] / (self.tau_cb[c, b2] * self.K[c])
                    for k, v in eq[0].items():
                        rows.append(r); cols.append(k); vals.append(v)
                    rhs[r] -= eq[1]
        self.A = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_unknowns, self.n_unknowns))
        self.s = rhs

    def transient_step(self, e_prev, dt):
        """One implicit-Euler step from e_prev (N, B, D): returns e and T."""
        xp = e_prev[self.active].reshape(-1)
        A = (self.A + sp.identity(self.n_unknowns, format="csr") / dt).tocsc()
        x = spla.spsolve(A, self.s + xp / dt)
        T = np.zeros(self.p.n_cells)
        T[self.active] = self.W @ x
        return dict(e=self.unpack(x), T=T)

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
    # domain lengths (the cell size h_a = L_a / n_a; the source stays per cell)
    g_L = np.zeros(3)
    for a in range(p.dim):
        hl = rel * p.length[a]
        Lp, Lm = list(p.length), list(p.length)
        Lp[a] += hl
        Lm[a] -= hl
        g_L[a] = (J(p.copy(length=tuple(Lp))) - J(p.copy(length=tuple(Lm)))) / (2 * hl)
    return dict(g_tau=g_tau, g_Tw=g_Tw, g_Q=g_Q, g_L=g_L)
