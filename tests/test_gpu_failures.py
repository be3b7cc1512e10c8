"""Failure paths and reporting of the C ABI on the GPU, made to happen
without any fault: a bounded device wait that runs out (a test hook shrinks
the row-pipeline kernel's poll limit, so the wait for the warp below gives up
at the first poll), a device allocation that cannot succeed, and the flux
residual eps_q of the convergence criteria."""
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


def test_expired_wait_reports_timeout_and_plan_recovers(bte):
    """The row-pipeline kernel's warps wait (bounded) for the warp below; with
    a limit of one poll the first wait gives up, the kernel records it and
    ends normally, and bte_solve returns BTE_ETIMEOUT.  With the default
    limit the same plan then solves correctly."""
    p = bi.square_2d(n=70, L=1e-6)
    p = p.copy(C=p.C[:3], v=p.v[:3], tau=p.tau[:3])
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.set_wait_limit(1)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-6, max_iter=64, tile_kind=3, check=False)
    assert rc == bte.BTE_ETIMEOUT
    assert "wait" in plan.error()
    plan.set_wait_limit(0)
    k = 8
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k, tile_kind=3)
    assert rc == bte.BTE_OK and st["tile_kind"] == 3
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    assert np.abs(T - ref["T"]).max() < 1e-5 * np.abs(ref["T"]).max()


def test_batched_expired_wait_reports_timeout(bte):
    """A batched solve with one instance whose waits run out stops polling
    that instance and reports BTE_ETIMEOUT (not a numeric failure)."""
    ps = [bi.square_2d(n=n, L=1e-6) for n in (40, 70)]
    ps = [q.copy(C=q.C[:3], v=q.v[:3], tau=q.tau[:3]) for q in ps]
    plans = [bte.Plan(q) for q in ps]
    plans[1].set_wait_limit(1)
    batch = bte.Batch(plans)
    T = np.zeros(sum(q.n_cells for q in ps))
    rc, st, bs = batch.solve(T, tol=1e-6, max_iter=4096, check=False)
    assert rc == bte.BTE_ETIMEOUT
    assert st[1]["iterations"] < 4096


def test_device_allocation_failure_is_enomem(bte):
    """A problem whose angular energy e (N B D values) cannot fit in device
    memory: bte_solve returns BTE_ENOMEM (no kernel runs before the failed
    allocation), the plan is destroyed cleanly and the context stays usable."""
    p = bi.square_2d(n=1024, L=10e-6, n_polar=8, n_az=640)
    assert p.n_cells * p.B * p.D * 4 > 300e9
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=1, tile_kind=1, dirs_per_lane=4,
                        check=False)
    assert rc == bte.BTE_ENOMEM, plan.error()
    plan.close()
    q = bi.tiny(2, n=(5, 4, 1), B=2)
    small = bte.Plan(q)
    T2 = np.zeros(q.n_cells)
    rc, st = small.solve(T2, precision=bte.BTE_FP64, tol=0.0, max_iter=3)
    ref = oracle.solve(q, max_iter=3, tol=0.0)
    assert np.abs(T2 - ref["T"]).max() < 1e-12 * np.abs(ref["T"]).max()


@pytest.mark.parametrize("dim,kw,kind", [
    (2, dict(n=(7, 6, 1), B=3, masked=True, diffuse=(2, 3), source=True, two_regions=True), 1),
    (2, dict(n=(20, 40, 1), B=2, diffuse=(2, 3)), 3),
    (3, dict(n=(6, 5, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True), 3),
])
def test_eps_q_matches_oracle(bte, dim, kw, kind):
    """eps_q = sqrt(mean (|q|^n - |q|^{n+1})^2) / max |q|^{n+1} (Methods,
    convergence criteria), for the returned iterate n and the next one."""
    p = bi.tiny(dim, **kw)
    k = 5
    a = oracle.solve(p, max_iter=k, tol=0.0)
    b = oracle.solve(p, max_iter=k + 1, tol=0.0)
    act = p.mask > 0
    m0 = np.linalg.norm(a["q"], axis=1)[act]
    m1 = np.linalg.norm(b["q"], axis=1)[act]
    ref = np.sqrt(np.mean((m0 - m1) ** 2)) / m1.max()
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    q = np.zeros((p.n_cells, 3))
    rc, st = plan.solve(T, q_out=q, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=kind)
    assert st["eps_q"] == pytest.approx(ref, rel=1e-8)
    # the returned state is still iterate k
    assert np.abs(q - a["q"]).max() < 1e-10 * np.abs(a["q"]).max()
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=kind)
    assert np.isnan(st["eps_q"])
