"""Checkpoint and resume of the outer iteration (bte_get_state, ein_init).

The paper's solution procedure (Methods, steps 1-4) carries from one outer
iteration to the next only T and the inflow that diffuse boundary faces take
from the previous sweep.  A solve resumed from those two (bte_get_state, then
bte_solve with T_init and ein_init) continues the iteration: it must reach
what one uninterrupted solve reaches, up to the rounding of the deviation
from T_ref (a resumed solve takes T_ref from the checkpointed T)."""
import numpy as np
import pytest

import bte_inputs as bi
import oracle

pytestmark = pytest.mark.gpu

CASES = {
    "2d_masked_diffuse_source": (dict(dim=2, n=(9, 7, 1), B=3, masked=True, diffuse=(2, 3), source=True), 0),
    "2d_two_regions": (dict(dim=2, n=(8, 6, 1), B=2, diffuse=(0, 2, 3), two_regions=True), 0),
    "3d_masked_pipeline": (dict(dim=3, n=(6, 5, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True), 3),
}


def _problem(kw):
    kw = dict(kw)
    return bi.tiny(kw.pop("dim"), **kw)


@pytest.fixture(scope="module")
def bte():
    import paper_2503_23657_gb300 as m
    return m


@pytest.mark.parametrize("prec,rtol", [(1, 1e-12), (0, 2e-6)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_resume_continues_the_iteration(bte, case, prec, rtol):
    kw, tile = CASES[case]
    p = _problem(kw)
    k1, k2 = 7, 6
    act = p.mask > 0
    direct = bte.Plan(p)
    Ta = np.zeros(p.n_cells)
    direct.solve(Ta, precision=prec, tol=0.0, max_iter=k1 + k2, tile_kind=tile)

    plan = bte.Plan(p)
    T1 = np.zeros(p.n_cells)
    plan.solve(T1, precision=prec, tol=0.0, max_iter=k1, tile_kind=tile)
    Ts, ein = plan.get_state()
    assert ein.shape == (p.B, plan.n_faces()) and plan.n_faces() > 0
    np.testing.assert_array_equal(Ts, T1)
    Tb = np.zeros(p.n_cells)
    rc, st = plan.solve(Tb, precision=prec, tol=0.0, max_iter=k2, tile_kind=tile, T_init=Ts, ein_init=ein)
    assert st["iterations"] == k2
    scale = np.abs(Ta[act]).max()
    assert np.abs(Tb - Ta)[act].max() < rtol * scale
    # the oracle's k1 + k2 iterations (FP64) agree too
    ref = oracle.solve(p, max_iter=k1 + k2, tol=0.0)["T"]
    assert np.abs(Tb - ref)[act].max() < max(rtol, 1e-12) * 10 * scale

    # T alone is not the state: restarting the inflow from the equilibrium
    # of T^k1 gives another iterate
    Tc = np.zeros(p.n_cells)
    plan.solve(Tc, precision=1, tol=0.0, max_iter=k2, tile_kind=tile, T_init=Ts)
    Td = np.zeros(p.n_cells)
    plan.solve(Td, precision=1, tol=0.0, max_iter=k2, tile_kind=tile, T_init=Ts, ein_init=ein)
    assert np.abs(Tc - Td)[act].max() > 1e-9 * scale


def test_resume_converges_like_one_solve(bte):
    """Checkpoint after 10 iterations, resume to eps_T < 1e-10: the resumed
    solve ends where the uninterrupted one does, within one iteration."""
    p = _problem(CASES["2d_masked_diffuse_source"][0])
    act = p.mask > 0
    plan = bte.Plan(p)
    Ta = np.zeros(p.n_cells)
    rc, sa = plan.solve(Ta, precision=1, tol=1e-10, max_iter=100000)
    Tb = np.zeros(p.n_cells)
    plan.solve(Tb, precision=1, tol=0.0, max_iter=10)
    Ts, ein = plan.get_state()
    rc, sb = plan.solve(Tb, precision=1, tol=1e-10, max_iter=100000, T_init=Ts, ein_init=ein)
    assert abs(10 + sb["iterations"] - sa["iterations"]) <= 1
    assert np.abs(Tb - Ta)[act].max() < 1e-9 * np.abs(Ta[act]).max()


def test_state_arguments_are_checked(bte):
    from paper_2503_23657_gb300.binding import BTEError
    p = _problem(CASES["2d_two_regions"][0])
    plan = bte.Plan(p)
    with pytest.raises(BTEError) as ei:
        plan.get_state()
    assert ei.value.code == bte.BTE_ESTATE
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=1, tol=0.0, max_iter=3)
    Ts, ein = plan.get_state()
    with pytest.raises(BTEError) as ei:   # ein_init without T_init
        plan.solve(T, precision=1, tol=0.0, max_iter=3, ein_init=ein)
    assert ei.value.code == bte.BTE_EINVAL
    bad = ein.copy()
    bad[0, 0] = np.nan
    with pytest.raises(BTEError) as ei:
        plan.solve(T, precision=1, tol=0.0, max_iter=3, T_init=Ts, ein_init=bad)
    assert ei.value.code == bte.BTE_EINVAL
