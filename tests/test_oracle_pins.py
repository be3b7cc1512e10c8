"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped
1/tau, a missing 4*pi, a wrong upwind side, a transposed index in the
diffuse reflection, a wrong sign of the collision term) fails at least one:

* ballistic limit of the gray slab (closed form in the discrete setting),
  along x, and along y and z for the other two flux components,
* diffusive limit: Fourier conductivity k = sum_b C_b v_b^2 tau_b / 3,
* continuum solution of the gray slab (exponential-integral equation) with
  first-order convergence in the cell size,
* scattering conservation after every temperature update,
* global energy balance at convergence (boundary outflow = integral of Q),
* mirror symmetries of symmetric problems,
* agreement of the source iteration with the direct solve of the linear
  system it converges to (tiny 1D/2D/3D grids with masks, diffuse walls,
  two regions and sources).
"""
import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense
from tests import physics


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_ballistic_limit_gray_slab():
    """tau -> infinity: every interior cell sees the wall it looks at, so
    e = C T_h/(4 pi) for mu > 0 and C T_c/(4 pi) for mu < 0; hence
    T = (T_h + T_c)/2 (symmetric Gauss-Legendre puts exactly 2 pi of weight
    in each hemisphere) and q = C v (T_h - T_c)/(4 pi) * sum_{mu>0} w mu,
    the discrete value of C v dT / 4."""
    p = bi.gray_slab(nx=50, tau=1e3)
    r = oracle.solve(p, max_iter=50, tol=1e-14)
    T_h, T_c = p.bc_T[0], p.bc_T[1]
    np.testing.assert_allclose(r["T"], 0.5 * (T_h + T_c), rtol=1e-13)
    mu = p.s[:, 0]
    q_discrete = p.C[0] * p.v[0] * (T_h - T_c) / (4 * np.pi) * np.sum(p.w[mu > 0] * mu[mu > 0])
    np.testing.assert_allclose(r["q"][:, 0], q_discrete, rtol=1e-12)
    # and within the Gauss-Legendre half-range error of C v dT / 4
    np.testing.assert_allclose(q_discrete, p.C[0] * p.v[0] * (T_h - T_c) / 4, rtol=5e-3)


def ballistic_slab_along(axis, nc=24, n_polar=4, n_az=8):
    """Gray ballistic slab whose normal is the y (axis 1) or z (axis 2) axis:
    a single column of cells between isothermal walls T_h (minus side) and
    T_c (plus side), every other domain face specular, so that the problem
    is the 1D slab with mu = s_axis.  The cross-section is made wide so that
    the lagged specular coupling converges in a few iterations."""
    dim = axis + 1
    s, w = bi.quadrature_polar_azimuth(n_polar, n_az, dim)
    n = [1, 1, 1]
    n[axis] = nc
    length = [1e-3, 1e-3 if dim == 3 else 1.0, 1.0]
    length[axis] = 1e-6
    types = [bi.SPECULAR] * 6
    types[2 * axis], types[2 * axis + 1] = bi.ISOTHERMAL, bi.ISOTHERMAL
    temps = np.full(6, 300.0)
    temps[2 * axis], temps[2 * axis + 1] = 301.0, 299.0
    return bi.Problem(
        name=f"ballistic_axis{axis}", dim=dim, n=tuple(n), length=tuple(length),
        mask=np.ones(nc, dtype=np.uint8), C=np.array([bi.C_TOTAL]), v=np.array([6400.0]),
        tau=np.array([1e3]), tau_scale=np.array([1.0]), s=s, w=w,
        bc_type=np.asarray(types, dtype=np.int32), bc_T=temps, T_init=300.0,
        tol=1e-14, precision="fp64")


@pytest.mark.parametrize("axis", [1, 2])
def test_ballistic_limit_flux_along_y_and_z(axis):
    """The heat flux definition q = sum_b v_b sum_d w_d s_d e (Methods,
    Phonon BTE) in its y and z components: the ballistic slab along that
    axis gives q_axis = C v (T_h - T_c)/(4 pi) * sum_{s_axis > 0} w s_axis,
    and the two other components vanish (e depends only on the sign of
    s_axis, and the direction set is symmetric); T = (T_h + T_c)/2."""
    p = ballistic_slab_along(axis)
    r = oracle.solve(p, max_iter=200, tol=1e-15)
    np.testing.assert_allclose(r["T"], 300.0, rtol=1e-13)
    sa = p.s[:, axis]
    q_discrete = p.C[0] * p.v[0] * 2.0 / (4 * np.pi) * np.sum(p.w[sa > 0] * sa[sa > 0])
    np.testing.assert_allclose(r["q"][:, axis], q_discrete, rtol=1e-12)
    for other in {0, 1, 2} - {axis}:
        assert np.abs(r["q"][:, other]).max() < 1e-12 * q_discrete
    # and close to the continuum value C v dT / 4 (quadrature error only)
    np.testing.assert_allclose(q_discrete, p.C[0] * p.v[0] * 2.0 / 4, rtol=5e-2)


@pytest.mark.parametrize("nongray", [False, True])
def test_diffusive_limit_fourier(nongray):
    """Kn << 1: linear interior profile, q / (-dT/dx) = sum C v^2 tau / 3
    (Gauss-Legendre integrates mu^2 exactly, so sum w mu^2 = 4 pi / 3)."""
    if nongray:
        C = np.array([0.5e6, 0.7e6, 0.46e6])
        v = np.array([6000.0, 4000.0, 2000.0])
        tau = np.array([1e-12, 2e-12, 4e-12])
    else:
        C, v, tau = np.array([1.66e6]), np.array([6400.0]), np.array([40e-12])
    mfp = float((v * tau).max())
    nx = 200
    L = 100 * mfp
    p = bi.gray_slab(nx=nx, L=L).copy(C=C, v=v, tau=tau)
    sol = dense.solve(p)
    T = sol["T"]
    q = oracle.flux(p, sol["e"])[:, 0]
    x = (np.arange(nx) + 0.5) * L / nx
    mid = slice(nx // 4, 3 * nx // 4)
    fit = np.polyfit(x[mid], T[mid], 1)
    k = float((C * v * v * tau).sum() / 3)
    assert q[nx // 2] / (-fit[0]) == pytest.approx(k, rel=1e-6)
    assert np.abs(T[mid] - np.polyval(fit, x[mid])).max() < 1e-6 * abs(T[0] - T[-1])


def test_gray_slab_continuum_first_order():
    """Kn = 0.256 slab against the continuum integral-equation solution: the
    L2 error in (T - T_c)/(T_h - T_c) falls about linearly with the cell size
    (step upwind is first order) and is small at the configured 200 cells;
    the wall temperature slip is reproduced."""
    kn = 6400.0 * 40e-12 / 1e-6
    eta, phi = physics.gray_slab_integral_equation(1.0 / kn)
    errs = []
    for nx in (100, 200, 400):
        p = bi.gray_slab(nx=nx)
        r = oracle.solve(p, max_iter=10000, tol=1e-13)
        x = (np.arange(nx) + 0.5) / nx / kn
        ph = (r["T"] - p.bc_T[1]) / (p.bc_T[0] - p.bc_T[1])
        errs.append(np.sqrt(np.mean((ph - np.interp(x, eta, phi)) ** 2)))
        if nx == 200:
            assert ph[0] < 0.9 and ph[-1] > 0.1      # slip at both walls
    assert errs[1] < 1e-3
    assert 1.6 < errs[0] / errs[1] < 2.6
    assert 1.6 < errs[1] / errs[2] < 2.6


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_scattering_conservation_each_iterate():
    """sum_b sum_d w_d (e - C_b T/(4 pi)) / tau_cb = 0 in every solid cell
    after a temperature update (Eq. updatee0_t), to round-off."""
    p = bi.tiny(2, n=(5, 4, 1), B=3, masked=True, diffuse=(2, 3), source=True,
                two_regions=True)
    for k in (1, 3):
        r = oracle.solve(p, max_iter=k, tol=0.0)
        for c in np.flatnonzero(p.mask):
            tcb = p.tau * p.tau_scale[p.mask[c] - 1]
            terms = (p.w[None, :] * (r["e"][c] - p.C[:, None] * r["T"][c] / (4 * np.pi))
                     / tcb[:, None])
            scale = np.sum(np.abs(p.w[None, :] * r["e"][c] / tcb[:, None]))
            assert abs(terms.sum()) < 1e-13 * scale


@pytest.mark.parametrize("case", ["2d_mask_source", "3d_mask_diffuse", "1d_source"])
def test_global_energy_balance(case):
    """At convergence the boundary outflow equals the heat generated (the
    interior face fluxes cancel, the collision term sums to zero per cell and
    sum_b sum_d w_d Q_b = Q); diffuse faces carry no net heat."""
    if case == "2d_mask_source":
        p = bi.tiny(2, n=(6, 5, 1), B=2, masked=True, diffuse=(2, 3), source=True)
    elif case == "3d_mask_diffuse":
        p = bi.tiny(3, n=(4, 4, 3), B=2, masked=True, diffuse=(0, 3, 5), source=True,
                    two_regions=True)
    else:
        p = bi.tiny(1, n=(12, 1, 1), B=3, diffuse=(1,), source=True)
    for e in (dense.solve(p)["e"], oracle.solve(p, max_iter=100000, tol=1e-15)["e"]):
        out, per_face = physics.boundary_outflow(p, e)
        q_in = physics.heat_input(p)
        scale = np.abs(per_face).sum()
        assert abs(out - q_in) < 1e-10 * scale
        for f in range(2 * p.dim):
            if p.bc_type[f] == bi.DIFFUSE:
                assert abs(per_face[f]) < 1e-10 * scale


def test_mirror_symmetry_slab():
    """T(L - x) = T_h + T_c - T(x) for the gray slab."""
    r = oracle.solve(bi.gray_slab(nx=60), max_iter=10000, tol=1e-14)
    T = r["T"]
    np.testing.assert_allclose(T[::-1], 600.0 - T, atol=1e-11)


def test_mirror_symmetry_square():
    """Left/right isothermal, top/bottom diffuse: T symmetric about y = L/2."""
    p = bi.square_2d(n=8, L=0.5e-6).copy()
    p = p.copy(C=p.C[:3], v=p.v[:3], tau=p.tau[:3])
    r = oracle.solve(p, max_iter=100000, tol=1e-14)
    T = r["T"].reshape(8, 8)
    np.testing.assert_allclose(T, T[::-1, :], rtol=1e-13)


def test_mirror_symmetry_cube():
    """All walls at one temperature, centred source, polar axis x with
    mid-point azimuths: T symmetric under x, y, z reflections and y<->z."""
    p = bi.hotspot_3d(n=6, L=0.2e-6, n_polar=2, n_az=8, sigma=40e-9)
    p = p.copy(C=p.C[:2], v=p.v[:2], tau=p.tau[:2])
    r = oracle.solve(p, max_iter=100000, tol=1e-14)
    T = r["T"].reshape(6, 6, 6)  # [z, y, x]
    assert T.max() > 300.0 + 1e-6
    for sym in (T[:, :, ::-1], T[:, ::-1, :], T[::-1, :, :], np.swapaxes(T, 0, 1)):
        np.testing.assert_allclose(sym, T, rtol=1e-13)


# --------------------------------------------------------------------------
# source iteration against the direct solve of its fixed point
# --------------------------------------------------------------------------

TINY = [
    (1, dict(n=(8, 1, 1), B=3, diffuse=(1,), source=True)),
    (2, dict(n=(4, 4, 1), B=2)),
    (2, dict(n=(5, 4, 1), B=3, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    (3, dict(n=(3, 3, 3), B=2)),
    (3, dict(n=(4, 3, 3), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
]


@pytest.mark.parametrize("dim,kw", TINY)
def test_iteration_matches_direct_solve(dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    act = p.mask > 0
    np.testing.assert_allclose(r["T"][act], ref["T"][act], rtol=2e-13, atol=0)
    np.testing.assert_allclose(r["e"], ref["e"], rtol=0, atol=1e-12 * np.abs(ref["e"]).max())


def test_fixed_iteration_count_is_reproducible():
    p = bi.tiny(2, n=(5, 4, 1), B=2, diffuse=(2,), source=True)
    a = oracle.solve(p, max_iter=7, tol=0.0)
    b = oracle.solve(p, max_iter=7, tol=0.0)
    assert a["iters"] == 7
    np.testing.assert_array_equal(a["T"], b["T"])
    # eps_T follows the paper's definition from the two last iterates
    c = oracle.solve(p, max_iter=6, tol=0.0)
    act = p.mask > 0
    eps = np.sqrt(np.mean((a["T"][act] - c["T"][act]) ** 2)) / a["T"][act].max()
    assert a["eps"][-1] == pytest.approx(eps, rel=1e-12)
