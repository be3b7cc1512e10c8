"""Pins of the oracle's specular boundaries (Boundary conditions: specularly
reflecting walls; the first of the extensions after the diffuse/isothermal
hot path).  A specular domain face returns into direction d the energy the
cell sends out through it in the mirror direction of d (normal component
reversed), lagged one outer iteration like the diffuse inflow.

What pins it, independently of its own code:
  * the product direction set (Gauss-Legendre in mu times mid-point
    azimuths, an even number of them) is closed under the three axis
    reflections, so every mirror exists;
  * a slab between two isothermal walls whose other faces are specular is
    the one-dimensional slab: the solution is uniform across the specular
    axes and equals the 1D problem with the same mu nodes to round-off;
  * method of images: a specular face at y = 0 gives the same solution as
    the domain doubled across it with the mask, the source and the far
    boundary mirrored (an exact property of the discrete equations);
  * the direct sparse solve of the linear system (with the specular
    couplings written as matrix entries) and the source iteration agree;
  * at convergence every specular face carries zero net heat and the
    isothermal faces carry away exactly the injected heat;
  * the adjoint gradients agree with central finite differences.
"""
import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense
from tests import physics

S = bi.SPECULAR


def _mirror(s, a):
    m = np.full(s.shape[0], -1)
    for d in range(s.shape[0]):
        want = s[d].copy()
        want[a] = -want[a]
        hit = np.flatnonzero(np.abs(s - want).sum(axis=1) < 1e-12)
        if hit.size:
            m[d] = hit[0]
    return m


@pytest.mark.parametrize("n_polar,n_az", [(2, 4), (4, 8), (8, 16)])
def test_direction_set_is_reflection_closed(n_polar, n_az):
    s, w = bi.quadrature_polar_azimuth(n_polar, n_az, 3)
    for a in range(3):
        m = _mirror(s, a)
        assert (m >= 0).all()
        np.testing.assert_allclose(w[m], w, rtol=0, atol=0)
        assert (m[m] == np.arange(s.shape[0])).all()


@pytest.mark.parametrize("dim,n,spec", [(2, (14, 5, 1), (2, 3)), (3, (12, 4, 3), (2, 3, 4, 5))])
def test_specular_side_walls_reduce_to_the_1d_slab(dim, n, spec):
    """Isothermal x walls, specular walls on every other axis: T(x, y, z) is
    the 1D slab's T(x) with the same mu nodes (the per-mu azimuthal weights
    add up to the 1D weight 2 pi w_mu)."""
    n_polar = 4
    p = bi.tiny(dim, n=n, B=2, n_polar=n_polar, n_az=8, specular=spec)
    q = bi.tiny(1, n=(n[0], 1, 1), B=2, n_polar=n_polar // 2)  # 1D: quadrature_1d(2 * n_polar // 2)
    assert q.D == n_polar and np.allclose(q.C, p.C) and np.allclose(q.tau, p.tau)
    assert np.allclose(q.bc_T[:2], p.bc_T[:2]) and np.isclose(q.length[0], p.length[0])
    r2 = oracle.solve(p, max_iter=100000, tol=1e-15)
    r1 = oracle.solve(q, max_iter=100000, tol=1e-15)
    T2 = r2["T"].reshape(-1, n[0])
    span = np.ptp(r1["T"])
    assert np.abs(T2 - r1["T"][None, :]).max() < 1e-11 * span
    # and it is uniform across the specular axes
    assert np.abs(T2 - T2[0][None, :]).max() < 1e-11 * span


def test_method_of_images():
    """A specular y- face is a mirror: the doubled domain (mask, source and
    the y+ boundary mirrored onto y-) has the same solution in its upper
    half."""
    p = bi.tiny(2, n=(9, 6, 1), B=2, n_polar=2, n_az=8, specular=(2,), diffuse=(3,), source=True,
                masked=True, two_regions=True)
    nx, ny = p.n[0], p.n[1]
    m2 = p.mask.reshape(ny, nx)
    phi2 = p.phi.reshape(ny, nx)
    bc_type = p.bc_type.copy()
    bc_type[2] = p.bc_type[3]
    q = p.copy(n=(nx, 2 * ny, 1), length=(p.length[0], 2 * p.length[1], p.length[2]),
               mask=np.concatenate([m2[::-1], m2]).ravel().copy(),
               phi=np.concatenate([phi2[::-1], phi2]).ravel().copy(), bc_type=bc_type)
    rp = oracle.solve(p, max_iter=100000, tol=1e-15)
    rq = oracle.solve(q, max_iter=100000, tol=1e-15)
    Tq = rq["T"].reshape(2 * ny, nx)[ny:]
    act = p.mask.reshape(ny, nx) > 0
    Tp = rp["T"].reshape(ny, nx)
    assert np.abs(Tp - Tq)[act].max() < 1e-11 * np.abs(Tp[act]).max()


CASES = [
    ("2d_mixed", 2, dict(n=(6, 5, 1), B=2, specular=(2,), diffuse=(3,), source=True)),
    ("2d_mask", 2, dict(n=(7, 6, 1), B=3, specular=(1, 3), masked=True, source=True, two_regions=True)),
    ("3d_mask", 3, dict(n=(4, 4, 3), B=2, specular=(2, 5), diffuse=(4,), masked=True, source=True)),
]


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
def test_source_iteration_matches_direct_solve(name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    act = p.mask > 0
    assert np.abs(r["T"] - ref["T"])[act].max() < 1e-12 * np.abs(ref["T"][act]).max()
    assert np.abs(r["e"] - ref["e"]).max() < 1e-11 * np.abs(ref["e"]).max()


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
def test_specular_faces_carry_no_net_heat(name, dim, kw):
    p = bi.tiny(dim, **kw)
    e = dense.solve(p)["e"]
    nx, ny, nz = p.n
    h = [p.length[a] / p.n[a] for a in range(3)]
    spec_flux = np.zeros(6)
    iso_flux = 0.0
    for c in np.flatnonzero(p.mask):
        idx = [c % nx, (c // nx) % ny, c // (nx * ny)]
        for a in range(p.dim):
            area = np.prod([h[o] for o in range(p.dim) if o != a])
            mir = _mirror(p.s, a)
            for side in (2 * a, 2 * a + 1):
                if not ((side % 2 == 0 and idx[a] == 0) or (side % 2 == 1 and idx[a] == p.n[a] - 1)):
                    continue
                sg = 1.0 if side % 2 else -1.0
                sn = p.s[:, a] * sg
                for b in range(p.B):
                    out = np.sum(p.w[sn > 0] * sn[sn > 0] * e[c, b, sn > 0])
                    if p.bc_type[side] == S:
                        e_in = e[c, b, mir]
                    elif p.bc_type[side] == 0:
                        e_in = np.full(p.D, p.C[b] * p.bc_T[side] / (4.0 * np.pi))
                    else:
                        e_in = np.full(p.D, out / np.sum(p.w[sn < 0] * -sn[sn < 0]))
                    f = p.v[b] * area * (out + np.sum(p.w[sn < 0] * sn[sn < 0] * e_in[sn < 0]))
                    if p.bc_type[side] == S:
                        spec_flux[side] += f
                    elif p.bc_type[side] == 0:
                        iso_flux += f
    scale = max(abs(iso_flux), physics.heat_input(p), 1e-300)
    assert np.abs(spec_flux).max() < 1e-10 * scale
    # void-interface faces are adiabatic as well, so the isothermal faces
    # carry away what the source injects
    assert abs(iso_flux - physics.heat_input(p)) < 1e-9 * scale


@pytest.mark.parametrize("name,dim,kw", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_adjoint_gradients_match_fd(name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    rng = np.random.default_rng(5)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(5, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, ref["T"][probes] - T_obs)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(a["g_tau"], fd["g_tau"], rtol=1e-4)
    np.testing.assert_allclose(a["g_Tw"], fd["g_Tw"], rtol=1e-4, atol=1e-6 * np.abs(fd["g_Tw"]).max())
    assert a["g_Q"] == pytest.approx(fd["g_Q"], rel=1e-4)


def test_missing_mirror_is_refused():
    """A direction set without a mirror direction cannot carry a specular
    face: the oracle refuses it."""
    p = bi.tiny(2, n=(4, 3, 1), B=1, n_polar=2, n_az=4, specular=(2,))
    s = p.s.copy()
    s[0] = s[0] * np.array([1.0, 0.9, 1.0])
    s[0] /= np.linalg.norm(s[0])
    with pytest.raises(ValueError):
        oracle.solve(p.copy(s=s), max_iter=3, tol=0.0)
