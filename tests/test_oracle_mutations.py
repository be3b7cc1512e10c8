"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of ``oracle/bte_oracle.c``
(on the CPU), builds it, and checks that the battery of pins used by
``test_oracle_pins.py`` / ``test_oracle_adjoint.py`` rejects it.
"""
import os

import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense
from tests import physics
from tests.test_oracle_pins import ballistic_slab_along

SRC = os.path.join(os.path.dirname(oracle.__file__), "bte_oracle.c")

MUTATIONS = {
    "source_without_4pi": ("p->phi[c] / (FOUR_PI * Csum);", "p->phi[c] / Csum;"),
    "collision_sign": ("double rhs = p->C[b] * T[c] / (FOUR_PI * tc)",
                       "double rhs = -p->C[b] * T[c] / (FOUR_PI * tc)"),
    "temperature_without_tau": ("num += acc / tc;", "num += acc;"),
    "upwind_side_swapped": ("> 0.0) ? 2 * a : 2 * a + 1;", "> 0.0) ? 2 * a + 1 : 2 * a;"),
    "diffuse_from_incoming": ("if (sn > 0.0) acc += p->w[d] * sn * (E(e_old",
                              "if (sn < 0.0) acc += p->w[d] * sn * (E(e_old"),
    "diffuse_norm_pi": ("return acc / diffuse_norm(p, side);\n}\n\n/* Value entering",
                        "return acc / M_PI;\n}\n\n/* Value entering"),
    "coef_without_velocity": ("double coef = p->v[b] * fabs(sa) / p->h[a];   /* v|s.n| S / V */",
                              "double coef = fabs(sa) / p->h[a];"),
    "coef_wrong_axis": ("double coef = p->v[b] * fabs(sa) / p->h[a];   /* v|s.n| S / V */",
                        "double coef = p->v[b] * fabs(sa) / p->h[0];"),
    "adjoint_source_without_weight": ("double rhs = p->w[d] * Th[c] / tc;",
                                      "double rhs = Th[c] / tc;"),
    "adjoint_without_diffuse": ("rhs += p->w[d] * fabs(sa) * adj_diffuse_sum",
                                "rhs += 0.0 * adj_diffuse_sum"),
    "tau_gradient_sign": ("g_tau[b] += acc / (tc * p->tau[b]);",
                          "g_tau[b] -= acc / (tc * p->tau[b]);"),
    "theta_without_capacity": ("acc += p->C[b] / (FOUR_PI * tau_cb(p, c, b)) * sm;",
                               "acc += 1.0 / (FOUR_PI * tau_cb(p, c, b)) * sm;"),
    "length_gradient_wrong_axis": ("g_L[a] += E(mu, c, b, d) * coef * (E(e, c, b, d) - ein) / (p->h[a] * p->n[a]);",
                                   "g_L[a] += E(mu, c, b, d) * coef * (E(e, c, b, d) - ein) / (p->h[0] * p->n[0]);"),
    "length_gradient_no_inflow": ("g_L[a] += E(mu, c, b, d) * coef * (E(e, c, b, d) - ein) / (p->h[a] * p->n[a]);",
                                  "g_L[a] += E(mu, c, b, d) * coef * (E(e, c, b, d) - 0.0 * ein) / (p->h[a] * p->n[a]);"),
    "flux_axis_slip": ("q[3 * c + a] += p->v[b] * p->w[d] * p->s[3 * d + a] * E(e, c, b, d);",
                       "q[3 * c + a] += p->v[b] * p->w[d] * p->s[3 * d] * E(e, c, b, d);"),
    "flux_axes_swapped": ("q[3 * c + a] += p->v[b] * p->w[d] * p->s[3 * d + a] * E(e, c, b, d);",
                          "q[3 * c + a] += p->v[b] * p->w[d] * p->s[3 * d + (3 - a) % 3] * E(e, c, b, d);"),
}


def _battery(lib):
    """Run the pins against a build; return the names of those that fail."""
    failed = []
    # ballistic closed form
    p = bi.gray_slab(nx=20, tau=1e3)
    r = oracle.solve(p, max_iter=50, tol=1e-14, lib=lib)
    mu = p.s[:, 0]
    qd = p.C[0] * p.v[0] * 2.0 / (4 * np.pi) * np.sum(p.w[mu > 0] * mu[mu > 0])
    if not (np.allclose(r["T"], 300.0, rtol=1e-12) and np.allclose(r["q"][:, 0], qd, rtol=1e-10)):
        failed.append("ballistic")
    # the y and z flux components: ballistic slabs along y and along z
    for axis in (1, 2):
        p = ballistic_slab_along(axis)
        r = oracle.solve(p, max_iter=200, tol=1e-15, lib=lib)
        sa = p.s[:, axis]
        qd = p.C[0] * p.v[0] * 2.0 / (4 * np.pi) * np.sum(p.w[sa > 0] * sa[sa > 0])
        others = [o for o in range(3) if o != axis]
        if not (np.allclose(r["q"][:, axis], qd, rtol=1e-10)
                and np.abs(r["q"][:, others]).max() < 1e-10 * qd):
            failed.append(f"ballistic_axis{axis}")
    # iteration vs direct solve, energy balance, adjoint on masked cases
    for dim, kw in [(2, dict(n=(5, 4, 1), B=3, masked=True, diffuse=(2, 3), source=True,
                             two_regions=True)),
                    (3, dict(n=(4, 3, 3), B=2, masked=True, diffuse=(0, 3, 5), source=True,
                             two_regions=True))]:
        p = bi.tiny(dim, **kw)
        sysm = dense.System(p)
        ref = sysm.solve()
        r = oracle.solve(p, max_iter=20000, tol=1e-15, lib=lib)
        act = p.mask > 0
        if not np.allclose(r["T"][act], ref["T"][act], rtol=1e-11, atol=0):
            failed.append(f"direct{dim}")
        out, per_face = physics.boundary_outflow(p, r["e"])
        if not abs(out - physics.heat_input(p)) < 1e-9 * np.abs(per_face).sum():
            failed.append(f"energy{dim}")
        rng = np.random.default_rng(3)
        probes = np.sort(rng.choice(np.flatnonzero(act), 4, replace=False))
        T_obs = ref["T"][probes] - 1.0
        g = np.zeros(p.n_cells)
        np.add.at(g, probes, ref["T"][probes] - T_obs)
        a = oracle.adjoint(p, ref["e"], ref["T"], g, max_iter=20000, tol=1e-15, lib=lib)
        fd = dense.fd_gradients(p, probes, T_obs)
        ok = (np.allclose(a["g_tau"], fd["g_tau"], rtol=1e-4)
              and np.allclose(a["g_Tw"], fd["g_Tw"], rtol=1e-4, atol=1e-8)
              and abs(a["g_Q"] - fd["g_Q"]) <= 1e-4 * abs(fd["g_Q"])
              and np.allclose(a["g_L"], fd["g_L"], rtol=1e-4, atol=1e-6 * np.abs(fd["g_L"]).max()))
        if not ok:
            failed.append(f"adjoint{dim}")
    return failed


SPECULAR_MUTATIONS = {
    "specular_same_direction": ("int m = mirror[3 * d + a];\n        return E(e_old, c, b, m)",
                                "int m = d;\n        return E(e_old, c, b, m)"),
    "specular_wrong_axis": ("int m = mirror[3 * d + a];\n        return E(e_old, c, b, m)",
                            "int m = mirror[3 * d + (a + 1) % 3];\n        return E(e_old, c, b, m)"),
    "specular_as_diffuse": ("return (p->bc_type[side] == ORC_SPECULAR) ? 3 : 2;", "return 2;"),
    "adjoint_without_specular": ("rhs += coef * E(mu_old, c, b, mirror[3 * d + a]);",
                                 "rhs += 0.0 * E(mu_old, c, b, mirror[3 * d + a]);"),
}


def _specular_battery(lib):
    """Pins of the specular faces (see test_oracle_specular.py)."""
    failed = []
    p = bi.tiny(2, n=(10, 4, 1), B=2, n_polar=4, n_az=8, specular=(2, 3))
    q = bi.tiny(1, n=(10, 1, 1), B=2, n_polar=2)
    T2 = oracle.solve(p, max_iter=100000, tol=1e-15, lib=lib)["T"].reshape(-1, 10)
    T1 = oracle.solve(q, max_iter=100000, tol=1e-15, lib=lib)["T"]
    if not np.abs(T2 - T1[None, :]).max() < 1e-10 * np.ptp(T1):
        failed.append("slab1d")
    p = bi.tiny(2, n=(7, 6, 1), B=3, specular=(1, 3), masked=True, source=True, two_regions=True)
    ref = dense.solve(p)
    r = oracle.solve(p, max_iter=100000, tol=1e-15, lib=lib)
    act = p.mask > 0
    if not np.allclose(r["T"][act], ref["T"][act], rtol=1e-11, atol=0):
        failed.append("direct")
    rng = np.random.default_rng(5)
    probes = np.sort(rng.choice(np.flatnonzero(act), 4, replace=False))
    T_obs = ref["T"][probes] - 1.0
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, ref["T"][probes] - T_obs)
    a = oracle.adjoint(p, ref["e"], ref["T"], g, max_iter=20000, tol=1e-15, lib=lib)
    fd = dense.fd_gradients(p, probes, T_obs)
    if not (np.allclose(a["g_tau"], fd["g_tau"], rtol=1e-4) and abs(a["g_Q"] - fd["g_Q"]) <= 1e-4 * abs(fd["g_Q"])):
        failed.append("adjoint")
    return failed


def test_unmutated_oracle_passes_specular_battery():
    assert _specular_battery(oracle.load_library(oracle.build())) == []


@pytest.mark.parametrize("name", sorted(SPECULAR_MUTATIONS))
def test_planted_specular_mistake_is_caught(name, tmp_path):
    old, new = SPECULAR_MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_c(str(path), str(tmp_path / "mutant.so")))
    assert _specular_battery(lib), f"planted mistake {name} was not detected"


def test_unmutated_oracle_passes_battery():
    assert _battery(oracle.load_library(oracle.build())) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_c(str(path), str(tmp_path / "mutant.so")))
    assert _battery(lib), f"planted mistake {name} was not detected"
