"""Independent physics checks used to pin the oracle (test code only).

Nothing here is called by the oracle or by the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.special as ss

FOUR_PI = 4.0 * np.pi


def boundary_outflow(p, e):
    """Net heat leaving the domain through all boundary faces (W, per unit
    length of every unresolved axis), evaluated from a converged e with the
    step face values: outgoing directions carry the cell value, incoming ones
    the boundary value (isothermal wall equilibrium, or the diffuse
    reflection of the same cell's outgoing energy)."""
    nx, ny, nz = p.n
    h = [p.length[a] / p.n[a] for a in range(3)]
    total = 0.0
    per_face = np.zeros(6)
    for c in np.flatnonzero(p.mask):
        idx = [c % nx, (c // nx) % ny, c // (nx * ny)]
        for a in range(p.dim):
            area = 1.0
            for o in range(p.dim):
                if o != a:
                    area *= h[o]
            for side in (2 * a, 2 * a + 1):
                sg = 1.0 if side % 2 else -1.0
                j = list(idx)
                j[a] += 1 if side % 2 else -1
                outside = j[a] < 0 or j[a] >= p.n[a]
                if not outside:
                    m = j[0] + nx * (j[1] + ny * j[2])
                    if p.mask[m]:
                        continue
                sn = p.s[:, a] * sg
                out_dirs, in_dirs = sn > 0, sn < 0
                for b in range(p.B):
                    f_out = np.sum(p.w[out_dirs] * sn[out_dirs] * e[c, b, out_dirs])
                    if outside and p.bc_type[side] == 0:
                        e_in = p.C[b] * p.bc_T[side] / FOUR_PI
                    else:
                        e_in = f_out / np.sum(p.w[in_dirs] * -sn[in_dirs])
                    f_in = np.sum(p.w[in_dirs] * sn[in_dirs]) * e_in
                    flux = p.v[b] * (f_out + f_in) * area
                    total += flux
                    if outside:
                        per_face[side] += flux
    return total, per_face


def heat_input(p):
    """Integral of Q over the solid (W, per unit length of unresolved axes)."""
    if p.phi is None:
        return 0.0
    vol = 1.0
    for a in range(p.dim):
        vol *= p.length[a] / p.n[a]
    return float(p.Q_amp * np.sum(p.phi[p.mask > 0]) * vol)


def gray_slab_integral_equation(eta_L: float, M: int = 4000):
    """Continuum nondimensional temperature phi = (T - T_c)/(T_h - T_c) of a
    gray slab of optical thickness eta_L = L/(v tau) between black walls,
    from the exponential-integral form of the gray BTE (isotropic scattering
    with the RTA re-emission, walls at T_h and T_c):

        phi(eta) = 1/2 E2(eta) + 1/2 int_0^eta_L E1(|eta - eta'|) phi(eta') d eta'

    solved by product-integration Nystrom on M panels with piecewise-constant
    phi (the E1 singularity is integrated exactly through E2)."""
    d = eta_L / M
    eta = (np.arange(M) + 0.5) * d
    lo, hi = eta - d / 2, eta + d / 2
    E2 = lambda u: ss.expn(2, u)
    K = np.abs(E2(np.abs(eta[:, None] - lo[None, :])) - E2(np.abs(eta[:, None] - hi[None, :])))
    K[np.arange(M), np.arange(M)] = 2.0 * (1.0 - E2(d / 2))
    phi = np.linalg.solve(np.eye(M) - 0.5 * K, 0.5 * E2(eta))
    return eta, phi


def gray_slab_discrete_ordinates(mu, w, L_over_mfp: float, M: int):
    """Spatially continuous solution of the discrete-ordinates gray slab:
    for each ordinate mu_i the transport along x is integrated exactly
    (exponential attenuation over the mean free path times |mu_i|), which
    leaves one integral equation for phi = (T - T_c)/(T_h - T_c) with the
    walls at phi = 1 (x = 0) and 0 (x = L):

        phi(x) = sum_{mu_i > 0} w_i/(4 pi) [exp(-x/l_i)
                    + int_0^x phi(x') exp(-(x - x')/l_i) dx'/l_i]
               + sum_{mu_i < 0} w_i/(4 pi) int_x^L phi(x') exp(-(x' - x)/l_i) dx'/l_i,

    l_i = |mu_i| (in units of the mean free path, L = L_over_mfp).  Solved
    by collocation at the midpoints of M panels with phi constant on each
    panel and the exponentials integrated exactly over it.  Only the angular
    discretisation is shared with a finite-volume solution, so it isolates
    the spatial discretisation error.  Returns (panel midpoints, phi)."""
    L = float(L_over_mfp)
    h = L / M
    xm = (np.arange(M) + 0.5) * h
    lo, hi = xm - h / 2, xm + h / 2
    K = np.zeros((M, M))
    f = np.zeros(M)
    for mi, wi in zip(mu, w):
        li = abs(mi)
        c = wi / FOUR_PI
        if mi > 0:
            f += c * np.exp(-xm / li)
            d_hi = np.clip(xm[:, None] - hi[None, :], 0.0, None)
            d_lo = np.clip(xm[:, None] - lo[None, :], 0.0, None)
            K += c * (np.exp(-d_hi / li) - np.exp(-d_lo / li))
        else:
            d_lo = np.clip(lo[None, :] - xm[:, None], 0.0, None)
            d_hi = np.clip(hi[None, :] - xm[:, None], 0.0, None)
            K += c * (np.exp(-d_lo / li) - np.exp(-d_hi / li))
    phi = np.linalg.solve(np.eye(M) - K, f)
    return xm, phi
