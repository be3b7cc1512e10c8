"""Band-sharded solve through libbte (bte_shard_begin / _sweep / _apply).

One GPU here, so the ranks are emulated in one process: two plans of the
same problem each sweep their own bands, their W are added on the host (the
allreduce), and both form T from the sum.  The sharded iteration must be the
unsharded one (bte_solve) up to the order of the band additions, and must
converge where the oracle does."""
import numpy as np
import pytest
import torch

import bte_inputs as bi
import oracle
from paper_2503_23657_gb300.sharded import ShardedSolve, band_range

pytestmark = pytest.mark.gpu

CASES = {
    "2d_masked_source": (dict(dim=2, n=(9, 7, 1), B=3, masked=True, diffuse=(2, 3), source=True), 0),
    "2d_rowpipe": (dict(dim=2, n=(20, 40, 1), B=4, diffuse=(2, 3)), 3),
    "3d_pipeline_two_regions": (dict(dim=3, n=(6, 5, 4), B=3, masked=True, diffuse=(0, 3, 5), two_regions=True), 3),
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
def test_two_emulated_ranks_follow_the_unsharded_iteration(bte, case, prec, rtol):
    kw, tile = CASES[case]
    p = _problem(kw)
    act = p.mask > 0
    k = 9
    full = bte.Plan(p)
    Ta = np.zeros(p.n_cells)
    full.solve(Ta, precision=prec, tol=0.0, max_iter=k, tile_kind=tile)

    plans = [bte.Plan(p) for _ in range(2)]
    for pl in plans:
        pl.shard_begin(precision=prec, tile_kind=tile)
    Ts = [torch.zeros(p.n_cells, dtype=torch.float64, device="cuda") for _ in range(2)]
    for it in range(k):
        W = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        for r, pl in enumerate(plans):
            b0, b1 = band_range(p.B, r, 2)
            Wr = torch.zeros_like(W)
            pl.shard_sweep(b0, b1, Wr)
            W += Wr                                            # the allreduce
        eps = [pl.shard_apply(W, Ts[r]) for r, pl in enumerate(plans)]
        assert eps[0] == eps[1]
    torch.testing.assert_close(Ts[0], Ts[1], rtol=0, atol=0)   # every rank forms the same T
    Tb = Ts[0].cpu().numpy()
    assert np.abs(Tb - Ta)[act].max() < rtol * np.abs(Ta[act]).max()


def test_one_rank_sharded_solve_converges_like_bte_solve(bte):
    """ShardedSolve without a process group (one rank, every band)."""
    p = _problem(CASES["3d_pipeline_two_regions"][0])
    act = p.mask > 0
    plan = bte.Plan(p)
    Ta = np.zeros(p.n_cells)
    rc, st = plan.solve(Ta, precision=1, tol=1e-10, max_iter=100000)
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    it, eps, conv = ShardedSolve(plan).solve(T, tol=1e-10, max_iter=100000, precision=1)
    assert conv and abs(it - st["iterations"]) <= 1
    Tb = T.cpu().numpy()
    assert np.abs(Tb - Ta)[act].max() < 1e-9 * np.abs(Ta[act]).max()
    ref = oracle.solve(p, max_iter=100000, tol=1e-10)
    assert np.abs(Tb - ref["T"])[act].max() < 1e-9 * np.abs(ref["T"][act]).max()


def test_shard_calls_are_checked(bte):
    from paper_2503_23657_gb300.binding import BTEError
    p = _problem(CASES["2d_masked_source"][0])
    plan = bte.Plan(p)
    W = np.zeros(p.n_cells)
    with pytest.raises(BTEError) as ei:
        plan.shard_sweep(0, 1, W)
    assert ei.value.code == bte.BTE_ESTATE
    plan.shard_begin(precision=1)
    for b0, b1 in ((0, 0), (1, 0), (-1, 2), (0, p.B + 1)):
        with pytest.raises(BTEError) as ei:
            plan.shard_sweep(b0, b1, W)
        assert ei.value.code == bte.BTE_EINVAL
    q = bi.tiny(2, n=(8, 6, 1), B=2, specular=(2, 3))
    with pytest.raises(BTEError) as ei:
        bte.Plan(q).shard_begin(precision=1)
    assert ei.value.code == bte.BTE_EINVAL
