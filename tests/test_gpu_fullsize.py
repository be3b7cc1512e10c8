"""Parity at the full sizes of the 3D workloads (the 64^3 hotspot with 15 bands
x 128 directions, the 160x80x64 FinFET) after a few source iterations from
the same initial state, in the launch configuration the solver picks for them
(autotuned tile), plus edge cases: the row-pipeline kernel at its largest
CTA (16 row-block warps) and a single-cell grid.

The oracle needs 15-50 s per source iteration at these sizes, so the fixed
iteration counts are small."""
import numpy as np
import pytest

import bte_inputs as bi
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bte():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_23657_gb300 as m
    m.load()
    return m


def rel(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_dev(a, b, T_ref, mask=None):
    """Error relative to the largest deviation from T_ref (the quantity the
    sweeps carry)."""
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.abs(a - b).max() / np.abs(b - T_ref).max())


def test_hotspot_full_size(bte):
    p = bi.hotspot_3d()
    k = 2
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k)
    T32 = T.cpu().numpy()
    assert rel(T32, ref["T"]) < 1e-5
    assert rel_dev(T32, ref["T"], 300.0) < 1e-4
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k)
    assert rel(T.cpu().numpy(), ref["T"]) < 1e-12


def test_finfet_full_size(bte):
    p = bi.finfet_3d()
    k = 1
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    plan = bte.Plan(p)
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k)
    T32 = T.cpu().numpy()
    assert rel(T32, ref["T"], act) < 1e-5
    assert rel_dev(T32, ref["T"], 300.0, act) < 1e-4
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k)
    T64 = T.cpu().numpy()
    assert rel(T64, ref["T"], act) < 1e-12
    assert np.all(T64[~act] == 0.0)


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-5)], ids=["fp64", "fp32"])
def test_rowpipe_largest_cta(bte, prec, tol):
    """9 x 500 grid: 16 row blocks of 32 lanes (the last one ragged), one
    direction group per CTA = the 512-thread maximum of the row-pipeline
    kernel."""
    p = bi.tiny(2, n=(9, 500, 1), B=2, diffuse=(1, 2), source=True, n_polar=2, n_az=4)
    k = 4
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=prec, tol=0.0, max_iter=k, tile_kind=3, dirs_per_lane=2, dirs_per_cta=2)
    assert st["tile_kind"] == 3
    assert rel(T, ref["T"]) < tol


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_single_cell(bte, dim):
    p = bi.tiny(dim, n=(1, 1, 1), B=2, diffuse=(2,) if dim > 1 else (), source=True)
    ref = oracle.solve(p, max_iter=100000, tol=1e-13)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-13, max_iter=100000)
    assert st["iterations"] == ref["iters"]
    assert rel(T, ref["T"]) < 1e-12


def test_finfet_reduced_adjoint_vs_oracle(bte):
    """The inverse problem's gradients (config 5 geometry at 1/8 scale: two
    regions, mask, source, 16 directions): GPU adjoint against the oracle's
    own FP64 adjoint of the same converged state, FP64 and FP32 sweeps."""
    p = bi.finfet_3d(scale=8, n_polar=2, n_az=8)
    ref = oracle.solve(p, max_iter=100000, tol=1e-12)
    rng = np.random.default_rng(5)
    probes = np.asarray(p.probes)
    T_obs = ref["T"][probes] + rng.uniform(-0.5, 0.5, probes.size)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, ref["T"][probes] - T_obs)
    adj = oracle.adjoint(p, ref["e"], ref["T"], g, max_iter=100000, tol=1e-12)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-12, max_iter=100000)
    rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=1e-12, max_iter=100000)
    np.testing.assert_allclose(g_tau, adj["g_tau"], rtol=1e-8, atol=1e-8 * np.abs(adj["g_tau"]).max())
    np.testing.assert_allclose(g_Tw, adj["g_Tw"], rtol=1e-8, atol=1e-8 * np.abs(adj["g_Tw"]).max())
    assert g_Q == pytest.approx(adj["g_Q"], rel=1e-8)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-9, max_iter=100000, check=False)
    rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=1e-9, max_iter=100000, check=False)
    np.testing.assert_allclose(g_tau, adj["g_tau"], rtol=1e-3, atol=1e-3 * np.abs(adj["g_tau"]).max())
    np.testing.assert_allclose(g_Tw, adj["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(adj["g_Tw"]).max())
    assert g_Q == pytest.approx(adj["g_Q"], rel=1e-3)
