"""Pins of the oracle's discrete adjoint (Forward and inverse modelling
workflow: the implicit solve is differentiated by a discrete adjoint).

* the adjoint state mu equals the direct solve of (L - P W - R)^T mu = W^T g,
* dJ/dtau_b, dJ/dT_wall, dJ/dQ_amp equal central finite differences of the
  direct forward solve (exact linear solves, so FD is accurate to ~1e-7),
* and central finite differences of the oracle's own source iteration.
"""
import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense

CASES = [
    (1, dict(n=(8, 1, 1), B=2, diffuse=(1,), source=True)),
    (2, dict(n=(4, 4, 1), B=2, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    (3, dict(n=(4, 4, 3), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
]


def _setup(dim, kw, seed=1):
    p = bi.tiny(dim, **kw)
    sysm = dense.System(p)
    sol = sysm.solve()
    rng = np.random.default_rng(seed)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(5, act.size), replace=False))
    T_obs = sol["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, sol["T"][probes] - T_obs)
    return p, sysm, sol, probes, T_obs, g


@pytest.mark.parametrize("dim,kw", CASES)
def test_adjoint_state_matches_direct(dim, kw):
    p, sysm, sol, probes, T_obs, g = _setup(dim, kw)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15, want_mu=True)
    mu_ref = sysm.adjoint(g)
    np.testing.assert_allclose(a["mu"], mu_ref, rtol=0, atol=1e-11 * np.abs(mu_ref).max())


@pytest.mark.parametrize("dim,kw", CASES)
def test_adjoint_gradients_match_direct_fd(dim, kw):
    p, sysm, sol, probes, T_obs, g = _setup(dim, kw)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(a["g_tau"], fd["g_tau"], rtol=2e-5)
    scale = np.abs(fd["g_Tw"]).max()
    np.testing.assert_allclose(a["g_Tw"], fd["g_Tw"], rtol=0, atol=1e-6 * scale)
    assert a["g_Q"] == pytest.approx(fd["g_Q"], rel=1e-6)


def test_adjoint_gradients_match_iterative_fd():
    """Central differences of the oracle's own source iteration (relative
    step 1e-4 on tau and Q_amp, 1e-3 K on the wall temperature)."""
    p, sysm, sol, probes, T_obs, g = _setup(2, CASES[1][1])

    def J(q):
        T = oracle.solve(q, max_iter=100000, tol=1e-15)["T"]
        d = T[probes] - T_obs
        return 0.5 * float(d @ d)

    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    for b in range(p.B):
        h = 1e-4 * p.tau[b]
        tp, tm = p.tau.copy(), p.tau.copy()
        tp[b] += h
        tm[b] -= h
        fd = (J(p.copy(tau=tp)) - J(p.copy(tau=tm))) / (2 * h)
        assert a["g_tau"][b] == pytest.approx(fd, rel=1e-3)
    Tp, Tm = p.bc_T.copy(), p.bc_T.copy()
    Tp[0] += 1e-3
    Tm[0] -= 1e-3
    fd = (J(p.copy(bc_T=Tp)) - J(p.copy(bc_T=Tm))) / 2e-3
    assert a["g_Tw"][0] == pytest.approx(fd, rel=1e-6)
    hq = 1e-4 * p.Q_amp
    fd = (J(p.copy(Q_amp=p.Q_amp + hq)) - J(p.copy(Q_amp=p.Q_amp - hq))) / (2 * hq)
    assert a["g_Q"] == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("dim,kw", CASES + [(2, dict(n=(6, 5, 1), B=2, specular=(2,), diffuse=(3,), source=True))])
def test_length_gradient_matches_direct_fd(dim, kw):
    """Geometric gradient (the paper's 1D inverse problem recovers a film
    thickness): dJ/dL_a of the adjoint against central differences of the
    direct solve with the domain length perturbed (cell size L_a / n_a)."""
    p, sysm, sol, probes, T_obs, g = _setup(dim, kw)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    fd = dense.fd_gradients(p, probes, T_obs)
    scale = np.abs(fd["g_L"]).max()
    assert scale > 0
    np.testing.assert_allclose(a["g_L"], fd["g_L"], rtol=1e-5, atol=1e-7 * scale)
    assert np.all(a["g_L"][p.dim:] == 0.0)


def test_film_thickness_gradient_1d():
    """The paper's 1D inverse case: gray film between isothermal walls,
    20 equally spaced observations of a thicker film; the gradient w.r.t.
    the thickness matches central differences of the oracle's own iteration
    and has the sign that moves L towards the truth."""
    p = bi.gray_slab(nx=50, L=0.5e-6, T_h=400.0, T_c=300.0)
    truth = bi.gray_slab(nx=50, L=1.0e-6, T_h=400.0, T_c=300.0)
    probes = np.linspace(1, 48, 20).astype(int)
    T_obs = oracle.solve(truth, max_iter=100000, tol=1e-14)["T"][probes]

    def J(q):
        T = oracle.solve(q, max_iter=100000, tol=1e-14)["T"]
        d = T[probes] - T_obs
        return 0.5 * float(d @ d)

    r = oracle.solve(p, max_iter=100000, tol=1e-14)
    g = np.zeros(p.n_cells)
    g[probes] = r["T"][probes] - T_obs
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-14)
    hL = 1e-4 * p.length[0]
    fd = (J(p.copy(length=(p.length[0] + hL, 1.0, 1.0))) - J(p.copy(length=(p.length[0] - hL, 1.0, 1.0)))) / (2 * hL)
    assert a["g_L"][0] == pytest.approx(fd, rel=1e-5)
    assert a["g_L"][0] < 0.0   # a thicker film lowers the misfit
