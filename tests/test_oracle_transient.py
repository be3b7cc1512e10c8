"""Pins of the oracle's transient steps (the transient BTE the paper's
Conclusion announces, de/dt + v s.grad e = -(e - e0)/tau + Q, in implicit
Euler steps, each converged by source iteration).

* One step equals the direct solve of (L + I/dt - P W - R) e = s + e_prev/dt
  (dense assembly) from the same e_prev.
* A step of infinite length is the steady solve.
* Many long steps reach the steady state.
* Exact discrete energy balance of every step: the change of the stored
  energy over dt equals the injected heat minus the net boundary outflow.
* Gray closed form: a heated box with specular walls only (adiabatic, no
  gradients) warms by Q dt / C per step, exactly.
* Planted mistakes in a copy of the C source are caught.
"""
import os

import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense
from tests import physics

CASES = [
    (1, dict(n=(9, 1, 1), B=2, diffuse=(1,), source=True)),
    (2, dict(n=(5, 4, 1), B=2, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    (2, dict(n=(6, 5, 1), B=2, specular=(2,), diffuse=(3,), source=True)),
    (3, dict(n=(4, 3, 3), B=2, masked=True, diffuse=(0, 3, 5), source=True)),
]
DT = 2e-11


def stored_energy(p, e):
    """sum over solid cells of V sum_b sum_d w_d e (per unit length of the
    unresolved axes)."""
    vol = np.prod([p.length[a] / p.n[a] for a in range(p.dim)])
    act = p.mask > 0
    return float(vol * np.einsum("cbd,d->", e[act], p.w))


def _steps_match_dense(p, n_steps=3, lib=None, rtol=1e-12):
    r = oracle.transient(p, DT, n_steps, tol=1e-15, lib=lib)
    sysm = dense.System(p)
    e = np.zeros((p.n_cells, p.B, p.D))
    act = p.mask > 0
    e[act] = (p.C[None, :, None] * p.T_init / (4 * np.pi)) * np.ones((1, 1, p.D))
    for m in range(n_steps):
        st = sysm.transient_step(e, DT)
        e = st["e"]
        if not np.abs(r["T_hist"][m] - st["T"])[act].max() < rtol * np.abs(st["T"][act]).max():
            return False
    return np.abs(r["e"] - e).max() < 10 * rtol * np.abs(e).max()


@pytest.mark.parametrize("dim,kw", CASES)
def test_steps_match_direct_implicit_euler(dim, kw):
    assert _steps_match_dense(bi.tiny(dim, **kw))


@pytest.mark.parametrize("dim,kw", CASES[:2])
def test_infinite_step_is_steady(dim, kw):
    p = bi.tiny(dim, **kw)
    r = oracle.transient(p, 1e300, 1, tol=1e-15)
    ref = dense.solve(p)
    act = p.mask > 0
    assert np.abs(r["T"] - ref["T"])[act].max() < 1e-12 * np.abs(ref["T"][act]).max()


def test_long_run_reaches_steady_state():
    p = bi.tiny(2, **CASES[1][1])
    r = oracle.transient(p, 1e-9, 40, tol=1e-15)
    ref = dense.solve(p)
    act = p.mask > 0
    assert np.abs(r["T"] - ref["T"])[act].max() < 1e-8 * np.ptp(ref["T"][act])
    # and the approach is monotone in the stored energy's distance to it
    d = [np.abs(T - ref["T"])[act].max() for T in r["T_hist"]]
    assert all(d[i + 1] <= d[i] * (1 + 1e-9) for i in range(len(d) - 1))


@pytest.mark.parametrize("dim,kw", CASES[:2] + CASES[3:])
def test_energy_balance_every_step(dim, kw):
    """(U^{m+1} - U^m)/dt = integral of Q - net outflow(e^{m+1}) with step
    faces (diffuse and void faces carry no net heat)."""
    p = bi.tiny(dim, **kw)
    e_prev = None
    T_prev = None
    for m in range(3):
        r = oracle.transient(p, DT, m + 1, tol=1e-15)
        if m > 0:
            out, _ = physics.boundary_outflow(p, r["e"])
            dU = (stored_energy(p, r["e"]) - stored_energy(p, e_prev)) / DT
            scale = abs(physics.heat_input(p)) + abs(out) + abs(dU)
            assert abs(dU - (physics.heat_input(p) - out)) < 1e-9 * scale
        e_prev = r["e"]


def test_adiabatic_gray_box_closed_form():
    """Gray band, specular walls everywhere, uniform source: e stays
    isotropic and uniform, so every step adds Q dt / C to T exactly."""
    n = 6
    s, w = bi.quadrature_1d(8)
    Q = 1e18
    C = 1.66e6
    p = bi.Problem(name="box", dim=1, n=(n, 1, 1), length=(60e-9, 1.0, 1.0),
                   mask=np.ones(n, dtype=np.uint8), C=np.array([C]), v=np.array([6400.0]),
                   tau=np.array([40e-12]), tau_scale=np.array([1.0]), s=s, w=w,
                   bc_type=np.array([2, 2, 2, 2, 2, 2], dtype=np.int32), bc_T=np.full(6, 300.0),
                   phi=np.ones(n), Q_amp=Q, T_init=300.0)
    r = oracle.transient(p, DT, 5, tol=1e-15)
    for m in range(5):
        np.testing.assert_allclose(r["T_hist"][m], 300.0 + (m + 1) * DT * Q / C, rtol=1e-14)


SRC = os.path.join(os.path.dirname(oracle.__file__), "bte_oracle.c")
MUTATIONS = {
    "no_time_diagonal": ("            diag += inv_dt;\n", "            diag += 0.0 * inv_dt;\n"),
    "previous_step_not_scaled": ("rhs += inv_dt * E(e_prev, c, b, d);", "rhs += E(e_prev, c, b, d);"),
    "previous_step_is_iterate": ("sweep_one(p, mirror, b, d, T_io, e_old, e_io, NULL, e_prev, inv_dt);",
                                 "sweep_one(p, mirror, b, d, T_io, e_old, e_io, NULL, e_old, inv_dt);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_transient_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_c(str(path), str(tmp_path / "mutant.so")))
    ok = all(_steps_match_dense(bi.tiny(dim, **kw), n_steps=2, lib=lib, rtol=1e-9) for dim, kw in CASES[:2])
    assert not ok, f"planted mistake {name} was not detected"
