"""Batched solves (many uneven 2D instances in one graph of batched launches)
against the FP64 oracle and against one-plan solves.

A small ensemble of the batched-ensemble recipe (uneven squares, log-uniform
sizes, per-instance wall temperature) spans three 32-row size classes; the
oracle runs a fixed number of source iterations per instance.
"""
import numpy as np
import pytest

import bte_inputs as bi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bte():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_23657_gb300 as m
    m.load()
    return m


def small_ensemble(n_instances=9, n_min=12, n_max=80, B=4):
    probs = bi.ensemble_2d(n_instances=n_instances, n_min=n_min, n_max=n_max)
    return [p.copy(C=p.C[:B], v=p.v[:B], tau=p.tau[:B]) for p in probs]


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def ensemble(bte):
    probs = small_ensemble()
    plans = [bte.Plan(p) for p in probs]
    batch = bte.Batch(plans)
    return probs, plans, batch


def test_classes_span_row_blocks(ensemble):
    probs, plans, batch = ensemble
    nrb = {(p.n[1] + 31) // 32 for p in probs}
    assert len(nrb) >= 3


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)], ids=["fp64", "fp32"])
def test_batch_fixed_iterations_vs_oracle(bte, ensemble, prec, tol):
    probs, plans, batch = ensemble
    k = 6
    T = np.zeros(sum(p.n_cells for p in probs))
    rc, st, bs = batch.solve(T, precision=prec, tol=0.0, max_iter=k)
    assert bs["instances"] == len(probs) and bs["max_iterations"] == k
    for i, p in enumerate(probs):
        ref = oracle.solve(p, max_iter=k, tol=0.0)
        Ti = T[batch.offsets[i]:batch.offsets[i + 1]]
        assert st[i]["iterations"] == k
        assert rel(Ti, ref["T"]) < tol, (i, p.name)


def test_batch_equals_single_plan_solves(bte, ensemble):
    """Same kernels, same tile: the batched FP32 result is bitwise the one-plan
    result, per instance."""
    probs, plans, batch = ensemble
    k = 9
    T = np.zeros(sum(p.n_cells for p in probs))
    rc, st, bs = batch.solve(T, precision=0, tol=0.0, max_iter=k)
    for i, (p, pl) in enumerate(zip(probs, plans)):
        Ts = np.zeros(p.n_cells)
        pl.solve(Ts, precision=0, tol=0.0, max_iter=k, tile_kind=3, dirs_per_lane=st[i]["dirs_per_lane"],
                 dirs_per_cta=st[i]["dirs_per_cta"])
        np.testing.assert_array_equal(T[batch.offsets[i]:batch.offsets[i + 1]], Ts)


def test_batch_per_instance_convergence(bte):
    """Each instance stops on its own eps_T test: iteration counts and T equal
    the one-plan FP64 solves (bitwise), differ across the batch, and the
    smallest instances match the oracle's converged runs."""
    probs = [p.copy(C=p.C[:4], v=p.v[:4], tau=p.tau[:4])
             for p in bi.ensemble_2d(n_instances=8, n_min=12, n_max=72, L_min=1e-7, L_max=1e-6)]
    plans = [bte.Plan(p) for p in probs]
    batch = bte.Batch(plans)
    T = torch.zeros(sum(p.n_cells for p in probs), dtype=torch.float64, device="cuda")
    rc, st, bs = batch.solve(T, precision=1, tol=1e-7, max_iter=100000)
    assert bs["converged"] == len(probs)
    its = [s["iterations"] for s in st]
    assert len(set(its)) > 1 and bs["max_iterations"] == max(its)
    Th = T.cpu().numpy()
    for i, (p, pl) in enumerate(zip(probs, plans)):
        Ts = np.zeros(p.n_cells)
        rc, s1 = pl.solve(Ts, precision=1, tol=1e-7, max_iter=100000, tile_kind=3,
                          dirs_per_lane=st[i]["dirs_per_lane"], dirs_per_cta=st[i]["dirs_per_cta"])
        assert s1["iterations"] == its[i], (i, p.name)
        np.testing.assert_array_equal(Th[batch.offsets[i]:batch.offsets[i + 1]], Ts)
    for i in sorted(range(len(probs)), key=lambda i: probs[i].n_cells)[:2]:
        ref = oracle.solve(probs[i], max_iter=100000, tol=1e-7)
        assert its[i] == ref["iters"]
        assert rel(Th[batch.offsets[i]:batch.offsets[i + 1]], ref["T"]) < 1e-12


def test_batch_rejects_bad_inputs(bte):
    from paper_2503_23657_gb300.binding import BTEError
    p1 = bi.tiny(2, n=(6, 5, 1), B=2, diffuse=(2,))
    p2 = bi.tiny(2, n=(7, 6, 1), B=3, diffuse=(2,))
    ps = bi.tiny(2, n=(7, 6, 1), B=2, specular=(2,))
    p3 = bi.tiny(3, n=(4, 3, 3), B=2)
    a, b, c, d = bte.Plan(p1), bte.Plan(p2), bte.Plan(ps), bte.Plan(p3)
    for plans in ([a, b], [a, c], [a, d], [a, a]):
        with pytest.raises(BTEError) as ei:
            bte.Batch(plans)
        assert ei.value.code == -1


def rowpipe(p):
    """Unmasked single-region instances of at most 512 rows run the row
    pipeline in a batch; the others the general kernel."""
    return bool((p.mask == 1).all()) and len(p.tau_scale) == 1 and p.n[1] <= 512


def mixed_ensemble():
    """2D instances of one band table and direction set: unmasked
    single-region ones (row-pipeline classes) next to masked and two-region
    ones (general-kernel classes), over several 32-row block counts."""
    shapes = [(9, 7), (12, 10), (20, 40), (16, 70), (33, 33), (7, 5), (40, 100), (25, 20)]
    out = []
    for k, (nx, ny) in enumerate(shapes):
        out.append(bi.tiny(2, n=(nx, ny, 1), B=2, masked=(k % 2 == 0), diffuse=(2, 3), source=(k % 3 == 0),
                           two_regions=(k % 3 == 1), seed=7))
    return out


@pytest.fixture(scope="module")
def mixed(bte):
    probs = mixed_ensemble()
    kinds = ["rowpipe" if rowpipe(p) else "general" for p in probs]
    assert "general" in kinds and "rowpipe" in kinds
    plans = [bte.Plan(p) for p in probs]
    return probs, plans, bte.Batch(plans)


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)], ids=["fp64", "fp32"])
def test_mixed_batch_fixed_iterations_vs_oracle(bte, mixed, prec, tol):
    """Masked and several-region instances batched with unmasked ones (the
    general kernel's batched form next to the row pipeline's)."""
    probs, plans, batch = mixed
    k = 6
    T = np.zeros(sum(p.n_cells for p in probs))
    rc, st, bs = batch.solve(T, precision=prec, tol=0.0, max_iter=k)
    for i, p in enumerate(probs):
        ref = oracle.solve(p, max_iter=k, tol=0.0)
        act = p.mask > 0
        Ti = T[batch.offsets[i]:batch.offsets[i + 1]]
        assert st[i]["iterations"] == k
        assert np.abs(Ti - ref["T"])[act].max() < tol * np.abs(ref["T"][act]).max(), (i, p.name)
        assert st[i]["tile_kind"] == (3 if rowpipe(p) else 1)


def test_mixed_batch_converged_per_instance(bte, mixed):
    """Each instance converges on its own test to the oracle's iteration
    count and state, and equals its one-plan solve with the same tile
    bitwise."""
    probs, plans, batch = mixed
    T = np.zeros(sum(p.n_cells for p in probs))
    rc, st, bs = batch.solve(T, precision=1, tol=1e-10, max_iter=100000)
    assert bs["converged"] == len(probs)
    for i, (p, pl) in enumerate(zip(probs, plans)):
        Ti = T[batch.offsets[i]:batch.offsets[i + 1]]
        ref = oracle.solve(p, max_iter=100000, tol=1e-10)
        act = p.mask > 0
        assert st[i]["iterations"] == ref["iters"], (i, p.name)
        assert np.abs(Ti - ref["T"])[act].max() < 1e-12 * np.abs(ref["T"][act]).max()
        Ts = np.zeros(p.n_cells)
        pl.solve(Ts, precision=1, tol=1e-10, max_iter=100000, tile_kind=st[i]["tile_kind"],
                 dirs_per_lane=st[i]["dirs_per_lane"], dirs_per_cta=st[i]["dirs_per_cta"])
        np.testing.assert_array_equal(Ti, Ts)


def test_batch_per_instance_source_amplitudes(bte, mixed):
    """Q_amp per instance (bte_solve_opts.Q_amp_each): each instance's source
    is its own q_profile times its own amplitude; one number applies to all."""
    probs, plans, batch = mixed
    k = 5
    n = sum(p.n_cells for p in probs)
    amps = [p.Q_amp * (1.0 + 0.5 * i) for i, p in enumerate(probs)]
    for Q, qs in ((amps, amps), (3e17, [3e17] * len(probs))):
        T = np.zeros(n)
        batch.solve(T, precision=1, tol=0.0, max_iter=k, Q_amp=Q)
        for i, p in enumerate(probs):
            ref = oracle.solve(p.copy(Q_amp=qs[i]), max_iter=k, tol=0.0)
            act = p.mask > 0
            Ti = T[batch.offsets[i]:batch.offsets[i + 1]]
            assert np.abs(Ti - ref["T"])[act].max() < 1e-12 * np.abs(ref["T"][act]).max(), (i, p.name)
    with pytest.raises(ValueError):
        batch.solve(np.zeros(n), Q_amp=[1.0, 2.0])


def test_full_ensemble_sampled_instances_vs_oracle(bte):
    """The whole 256-instance ensemble (uneven squares n 32..160, 15 bands x
    64 directions) batched for 10 iterations in FP32; the smallest, the
    median and the largest instance against the oracle's 10 iterations."""
    probs = bi.ensemble_2d()
    plans = [bte.Plan(p) for p in probs]
    batch = bte.Batch(plans)
    k = 10
    T = np.zeros(sum(p.n_cells for p in probs))
    rc, st, bs = batch.solve(T, precision=0, tol=0.0, max_iter=k)
    order = np.argsort([p.n_cells for p in probs], kind="stable")
    for i in (order[0], order[len(order) // 2], order[-1]):
        p = probs[i]
        ref = oracle.solve(p, max_iter=k, tol=0.0)
        Ti = T[batch.offsets[i]:batch.offsets[i + 1]]
        assert st[i]["iterations"] == k
        assert np.abs(Ti - ref["T"]).max() < 1e-5 * np.abs(ref["T"]).max(), (i, p.name)
    batch.close()
    for pl in plans:
        pl.close()
