"""Seeded synthetic workloads for the steady RTA phonon BTE.

This module only *describes* problems: grids, masks, band tables, direction
sets, boundary conditions, heat-source profiles and probe locations.  It holds
none of the solver's arithmetic, so both the FP64 CPU oracle and the CUDA
library can read the same inputs without sharing any solver code.

The paper's workloads use DFT silicon bands and GiftBTE meshes that are not
available here.  The synthetic stand-ins keep the paper's shapes and sizes:
15 bands, 64/128 discrete ordinates, FinFET-scale grids, heat sources of
1e18-1e19 W/m^3 (Results, FinFET sections; Introduction cost example).

Conventions
-----------
* Cells are indexed ``c = i + nx*(j + ny*k)`` (x fastest).
* ``mask[c] == 0`` marks a void cell; ``mask[c] = r >= 1`` a solid cell of
  region ``r`` whose relaxation times are ``tau_b * tau_scale[r-1]``.
* Domain faces are numbered 0:x-, 1:x+, 2:y-, 3:y+, 4:z-, 5:z+.  Faces of
  axes that the problem does not resolve (``axis >= dim``) are ignored.
* ``bc_type`` is ``ISOTHERMAL`` (0), ``DIFFUSE`` (1) or ``SPECULAR`` (2).
  Faces between a solid and a void cell are always diffusely reflecting.
* Directions ``s[d]`` follow the paper's angle convention
  s = (cos(theta), sin(theta)cos(phi), sin(theta)sin(phi)) with the polar
  axis along x (Methods, angle discretisation); weights sum to 4*pi.
* The volumetric heat source is ``Q(x) = Q_amp * phi[c]`` in W/m^3.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

ISOTHERMAL = 0
DIFFUSE = 1
SPECULAR = 2

MASTER_SEED = 20250330

# Synthetic silicon-like band table (15 bands).
N_BANDS = 15
C_TOTAL = 1.66e6          # J/(m^3 K), total volumetric heat capacity
V_MAX, V_MIN = 8000.0, 800.0
TAU_MIN, TAU_MAX = 5e-12, 2e-9


@dataclasses.dataclass
class Problem:
    """One steady BTE instance on a masked Cartesian grid."""
    name: str
    dim: int
    n: tuple            # (nx, ny, nz)
    length: tuple       # (Lx, Ly, Lz) in metres
    mask: np.ndarray    # uint8 [nx*ny*nz]
    C: np.ndarray       # [B] J/(m^3 K)
    v: np.ndarray       # [B] m/s
    tau: np.ndarray     # [B] s
    tau_scale: np.ndarray  # [R] per-region multiplier on tau
    s: np.ndarray       # [D,3] unit direction vectors
    w: np.ndarray       # [D] solid-angle weights (sum 4*pi)
    bc_type: np.ndarray  # int32 [6]
    bc_T: np.ndarray     # float64 [6] wall temperatures (isothermal faces)
    phi: Optional[np.ndarray] = None   # [N] W/m^3 per unit amplitude
    Q_amp: float = 0.0
    T_init: float = 300.0
    probes: Optional[np.ndarray] = None   # int64 cell indices
    T_obs: Optional[np.ndarray] = None    # observed probe temperatures
    tol: float = 1e-6
    precision: str = "fp32"
    order: int = 1      # face values: 1 step (first-order) upwind, 2 Green-Gauss reconstructed

    @property
    def n_cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def B(self) -> int:
        return int(self.C.shape[0])

    @property
    def D(self) -> int:
        return int(self.w.shape[0])

    @property
    def h(self) -> tuple:
        return tuple(self.length[a] / self.n[a] for a in range(3))

    @property
    def n_active(self) -> int:
        return int(np.count_nonzero(self.mask))

    def copy(self, **changes) -> "Problem":
        fields = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        for k, val in fields.items():
            if isinstance(val, np.ndarray):
                fields[k] = val.copy()
        fields.update(changes)
        return Problem(**fields)


# ---------------------------------------------------------------------------
# direction sets
# ---------------------------------------------------------------------------

def _octant_sort(s: np.ndarray, w: np.ndarray, dim: int):
    """Order directions so that those sharing an octant (signs of the
    resolved components) are contiguous; the order inside an octant is kept."""
    key = np.zeros(s.shape[0], dtype=np.int64)
    for a in range(dim):
        key = key * 2 + (s[:, a] < 0)
    order = np.argsort(key, kind="stable")
    return s[order].copy(), w[order].copy()


def quadrature_1d(n_polar: int):
    """Gauss-Legendre nodes in mu = cos(theta) on [-1, 1], azimuth integrated
    analytically (weight 2*pi*w_i).  s = (mu, sqrt(1-mu^2), 0)."""
    mu, wg = np.polynomial.legendre.leggauss(n_polar)
    s = np.zeros((n_polar, 3))
    s[:, 0] = mu
    s[:, 1] = np.sqrt(1.0 - mu * mu)
    w = 2.0 * np.pi * wg
    return _octant_sort(s, w, 1)


def quadrature_polar_azimuth(n_polar: int, n_az: int, dim: int):
    """Gauss-Legendre in mu = cos(theta) (polar axis x) times uniform
    mid-point azimuths phi_k = (k+1/2)*2*pi/n_az with weight 2*pi/n_az."""
    mu, wg = np.polynomial.legendre.leggauss(n_polar)
    phis = (np.arange(n_az) + 0.5) * 2.0 * np.pi / n_az
    s = np.zeros((n_polar * n_az, 3))
    w = np.zeros(n_polar * n_az)
    d = 0
    for p in range(n_polar):
        st = np.sqrt(1.0 - mu[p] * mu[p])
        for k in range(n_az):
            s[d] = (mu[p], st * np.cos(phis[k]), st * np.sin(phis[k]))
            w[d] = wg[p] * 2.0 * np.pi / n_az
            d += 1
    return _octant_sort(s, w, dim)


# ---------------------------------------------------------------------------
# band tables
# ---------------------------------------------------------------------------

def synthetic_bands(rng: np.random.Generator, n_bands: int = N_BANDS):
    """v_b linear 8000..800 m/s; tau_b log-uniform in [5 ps, 2 ns] drawn
    independently of v_b; C_b = Dirichlet(2)*1.66e6 J/(m^3 K)."""
    v = np.linspace(V_MAX, V_MIN, n_bands)
    tau = np.exp(rng.uniform(np.log(TAU_MIN), np.log(TAU_MAX), n_bands))
    C = rng.dirichlet(2.0 * np.ones(n_bands)) * C_TOTAL
    return C, v, tau


def _children(n: int):
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(MASTER_SEED).spawn(n)]


def _bc(types, temps):
    return np.asarray(types, dtype=np.int32), np.asarray(temps, dtype=np.float64)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def gray_slab(nx: int = 200, L: float = 1e-6, n_polar: int = 16,
              v: float = 6400.0, tau: float = 40e-12, C: float = C_TOTAL,
              T_h: float = 301.0, T_c: float = 299.0) -> Problem:
    """1D gray cross-plane slab between isothermal walls (Kn = v*tau/L)."""
    s, w = quadrature_1d(n_polar)
    bct, bcT = _bc([ISOTHERMAL] * 6, [T_h, T_c, 300, 300, 300, 300])
    return Problem(
        name=f"slab1d_{nx}", dim=1, n=(nx, 1, 1), length=(L, 1.0, 1.0),
        mask=np.ones(nx, dtype=np.uint8),
        C=np.array([C]), v=np.array([v]), tau=np.array([tau]),
        tau_scale=np.array([1.0]), s=s, w=w, bc_type=bct, bc_T=bcT,
        T_init=0.5 * (T_h + T_c), tol=1e-10, precision="fp64")


def square_2d(n: int = 128, L: float = 2e-6, n_polar: int = 8, n_az: int = 8,
              T_left: float = 310.0, T_right: float = 300.0,
              seed_child: int = 1) -> Problem:
    """2D nongray square: left wall hot, right wall 300 K, top/bottom
    diffusely reflecting; 15 synthetic bands; 8x8 directions."""
    rng = _children(6)[seed_child]
    C, v, tau = synthetic_bands(rng)
    s, w = quadrature_polar_azimuth(n_polar, n_az, 2)
    bct, bcT = _bc([ISOTHERMAL, ISOTHERMAL, DIFFUSE, DIFFUSE, DIFFUSE, DIFFUSE],
                   [T_left, T_right, 300, 300, 300, 300])
    return Problem(
        name=f"square2d_{n}", dim=2, n=(n, n, 1), length=(L, L, 1.0),
        mask=np.ones(n * n, dtype=np.uint8), C=C, v=v, tau=tau,
        tau_scale=np.array([1.0]), s=s, w=w, bc_type=bct, bc_T=bcT,
        T_init=300.0, tol=1e-6)


def hotspot_3d(n: int = 64, L: float = 1e-6, n_polar: int = 8, n_az: int = 16,
               sigma: float = 50e-9, peak: float = 1e18) -> Problem:
    """3D cube, all faces isothermal at 300 K, Gaussian volumetric source
    (sigma 50 nm, peak 1e18 W/m^3) at the centre."""
    rng = _children(6)[2]
    C, v, tau = synthetic_bands(rng)
    s, w = quadrature_polar_azimuth(n_polar, n_az, 3)
    h = L / n
    xc = (np.arange(n) + 0.5) * h - 0.5 * L
    r2 = xc[None, None, :] ** 2 + xc[None, :, None] ** 2 + xc[:, None, None] ** 2
    phi = np.exp(-0.5 * r2 / sigma ** 2).reshape(-1)
    bct, bcT = _bc([ISOTHERMAL] * 6, [300.0] * 6)
    return Problem(
        name=f"hotspot3d_{n}", dim=3, n=(n, n, n), length=(L, L, L),
        mask=np.ones(n ** 3, dtype=np.uint8), C=C, v=v, tau=tau,
        tau_scale=np.array([1.0]), s=s, w=w, bc_type=bct, bc_T=bcT,
        phi=phi, Q_amp=peak, T_init=300.0, tol=1e-6)


def finfet_3d(scale: int = 1, n_polar: int = 8, n_az: int = 16,
              tau_b_scale: float = 1.0, T_sub: float = 300.0, Q_amp: float = 1e19,
              n_probes: int = 64) -> Problem:
    """FinFET-like masked 3D problem.  Domain 400x200x160 nm at 2.5 nm cells
    (160x80x64); substrate z < 100 nm; oxide (tau x 0.1) for 100 <= z < 120 nm
    outside the fin; fin 20 nm wide (centred in y) and 40 nm tall
    (100 <= z < 140 nm) over 100 <= x < 300 nm; Joule source in the fin's top
    10 nm.  Bottom face isothermal, every other face diffuse.  ``scale``
    divides the cell count per axis (coarser cells) for reduced cases."""
    rng = _children(6)[4]
    C, v, tau = synthetic_bands(rng)
    tau = tau * tau_b_scale
    s, w = quadrature_polar_azimuth(n_polar, n_az, 3)
    h = 2.5e-9 * scale
    nx, ny, nz = 160 // scale, 80 // scale, 64 // scale
    xs = (np.arange(nx) + 0.5) * h
    ys = (np.arange(ny) + 0.5) * h
    zs = (np.arange(nz) + 0.5) * h
    X = xs[None, None, :] + 0 * ys[None, :, None] + 0 * zs[:, None, None]
    Y = 0 * xs[None, None, :] + ys[None, :, None] + 0 * zs[:, None, None]
    Z = 0 * xs[None, None, :] + 0 * ys[None, :, None] + zs[:, None, None]
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    mask[Z < 100e-9] = 1
    oxide = (Z >= 100e-9) & (Z < 120e-9)
    mask[oxide] = 2
    fin = ((X >= 100e-9) & (X < 300e-9) & (np.abs(Y - 100e-9) < 10e-9)
           & (Z >= 100e-9) & (Z < 140e-9))
    mask[fin] = 1
    phi = (fin & (Z >= 130e-9)).astype(np.float64).reshape(-1)
    mask = mask.reshape(-1)
    bct, bcT = _bc([DIFFUSE, DIFFUSE, DIFFUSE, DIFFUSE, ISOTHERMAL, DIFFUSE],
                   [300.0, 300.0, 300.0, 300.0, T_sub, 300.0])
    active = np.flatnonzero(mask)
    prng = _children(6)[5]
    probes = np.sort(prng.choice(active, size=min(n_probes, active.size), replace=False))
    return Problem(
        name=f"finfet3d_s{scale}", dim=3, n=(nx, ny, nz), length=(nx * h, ny * h, nz * h),
        mask=mask, C=C, v=v, tau=tau, tau_scale=np.array([1.0, 0.1]), s=s, w=w,
        bc_type=bct, bc_T=bcT, phi=phi, Q_amp=Q_amp, T_init=300.0,
        probes=probes.astype(np.int64), tol=1e-6)


def finfet_specular_3d(**kw) -> Problem:
    """The FinFET of ``finfet_3d`` with the paper's mixed boundaries of its
    3D FinFET validation case: the base (substrate and oxide) reflects
    specularly at its four side faces (x and y domain faces), the fin
    surfaces (faces next to void cells) diffusely, the bottom is isothermal.
    Same grid, bands, directions, source and probes."""
    p = finfet_3d(**kw)
    bct = p.bc_type.copy()
    bct[0] = bct[1] = bct[2] = bct[3] = SPECULAR
    return p.copy(name=p.name.replace("finfet3d", "finfet3d_specbase"), bc_type=bct)


def ensemble_2d(n_instances: int = 256, n_min: int = 32, n_max: int = 160,
                L_min: float = 1e-7, L_max: float = 1e-5):
    """Batched ensemble of uneven 2D squares: side cells ~ U{n_min..n_max},
    domain size log-uniform in [L_min, L_max], left wall 300 K + dT with
    dT ~ U(1, 20) K, right wall 300 K, top/bottom diffuse.  All instances
    share the synthetic band table and the 8x8 direction set."""
    rng = _children(6)[3]
    base = square_2d(n=8)
    out = []
    for m in range(n_instances):
        n = int(rng.integers(n_min, n_max + 1))
        L = float(np.exp(rng.uniform(np.log(L_min), np.log(L_max))))
        dT = float(rng.uniform(1.0, 20.0))
        bct, bcT = _bc([ISOTHERMAL, ISOTHERMAL, DIFFUSE, DIFFUSE, DIFFUSE, DIFFUSE],
                       [300.0 + dT, 300.0, 300, 300, 300, 300])
        out.append(base.copy(name=f"ens{m}_{n}", n=(n, n, 1), length=(L, L, 1.0),
                             mask=np.ones(n * n, dtype=np.uint8),
                             bc_type=bct, bc_T=bcT))
    return out


# ---------------------------------------------------------------------------
# tiny problems for brute-force checks
# ---------------------------------------------------------------------------

def tiny(dim: int, n=(4, 4, 3), B: int = 2, n_polar: int = 2, n_az: int = 4,
         masked: bool = False, diffuse=(), source: bool = False, seed: int = 7,
         two_regions: bool = False, L: float = 40e-9, specular=()) -> Problem:
    """Small random problem for dense brute-force comparisons.  ``diffuse``
    and ``specular`` list the domain faces that reflect diffusely /
    specularly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx = n[0]
    ny = n[1] if dim >= 2 else 1
    nz = n[2] if dim >= 3 else 1
    C = rng.uniform(0.2, 1.0, B) * C_TOTAL / B
    v = rng.uniform(1000.0, 8000.0, B)
    tau = np.exp(rng.uniform(np.log(2e-12), np.log(5e-10), B))
    if dim == 1:
        s, w = quadrature_1d(2 * n_polar)
    else:
        s, w = quadrature_polar_azimuth(n_polar, n_az, dim)
    N = nx * ny * nz
    mask = np.ones(N, dtype=np.uint8)
    if two_regions:
        mask[rng.random(N) < 0.4] = 2
    types = [ISOTHERMAL] * 6
    for f in diffuse:
        types[f] = DIFFUSE
    for f in specular:
        types[f] = SPECULAR
    if masked:
        # knock out a few cells, then drop solid cells that no longer connect
        # to an isothermal domain face (they would form an adiabatic island
        # whose temperature is undetermined)
        kill = rng.random(N) < 0.25
        mask[kill] = 0
        mask = _keep_anchored(mask, (nx, ny, nz), dim, types)
    temps = rng.uniform(295.0, 310.0, 6)
    bct, bcT = _bc(types, temps)
    phi = rng.uniform(0.0, 1.0, N) if source else None
    h = L / nx
    # non-cubic cells (h_y = 1.25 h, h_z = 0.8 h) so that an axis mix-up in
    # the cell size cannot hide
    return Problem(
        name=f"tiny{dim}d", dim=dim, n=(nx, ny, nz),
        length=(nx * h, ny * h * 1.25 if dim >= 2 else 1.0, nz * h * 0.8 if dim >= 3 else 1.0),
        mask=mask, C=C, v=v, tau=tau,
        tau_scale=np.array([1.0, 0.3]) if two_regions else np.array([1.0]),
        s=s, w=w, bc_type=bct, bc_T=bcT, phi=phi, Q_amp=1e18 if source else 0.0,
        T_init=300.0, tol=1e-12, precision="fp64")


def _keep_anchored(mask, n, dim, types):
    """Zero the solid cells whose connected component touches no isothermal
    domain face.  Pure connectivity bookkeeping on the mask."""
    nx, ny, nz = n
    N = nx * ny * nz
    seen = np.zeros(N, dtype=bool)
    stack = []
    for c in range(N):
        if mask[c] == 0:
            continue
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        idx = (i, j, k)
        for a in range(dim):
            if (idx[a] == 0 and types[2 * a] == ISOTHERMAL) or \
               (idx[a] == n[a] - 1 and types[2 * a + 1] == ISOTHERMAL):
                seen[c] = True
                stack.append(c)
                break
    while stack:
        c = stack.pop()
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        for a in range(dim):
            for step in (-1, 1):
                idx = [i, j, k]
                idx[a] += step
                if 0 <= idx[a] < n[a]:
                    m = idx[0] + nx * (idx[1] + ny * idx[2])
                    if mask[m] and not seen[m]:
                        seen[m] = True
                        stack.append(m)
    out = mask.copy()
    out[~seen] = 0
    return out


CONFIGS = {
    "slab1d": gray_slab,
    "square2d": square_2d,
    "hotspot3d": hotspot_3d,
    "finfet3d": finfet_3d,
}
