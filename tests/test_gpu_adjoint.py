"""GPU adjoint (bte_adjoint through the C ABI and the autograd wrapper)
against the oracle's FP64 adjoint and central finite differences."""
import numpy as np
import pytest

import bte_inputs as bi
import oracle
import oracle.dense as dense

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bte():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_23657_gb300 as m
    m.load()
    return m


CASES = [
    ("1d", 1, dict(n=(8, 1, 1), B=2, diffuse=(1,), source=True)),
    ("2d_mask", 2, dict(n=(6, 5, 1), B=2, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    ("3d_mask", 3, dict(n=(5, 4, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
]


def _setup(dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    rng = np.random.default_rng(11)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(6, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    return p, ref, probes, T_obs


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
def test_fp64_adjoint_matches_oracle_and_fd(bte, name, dim, kw):
    p, ref, probes, T_obs = _setup(dim, kw)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=1e-15, max_iter=100000)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, T[probes] - T_obs)
    rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-15)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    np.testing.assert_allclose(g_tau, a["g_tau"], rtol=1e-8)
    np.testing.assert_allclose(g_Tw, a["g_Tw"], rtol=1e-8, atol=1e-12 * np.abs(a["g_Tw"]).max())
    assert g_Q == pytest.approx(a["g_Q"], rel=1e-8)
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(g_tau, fd["g_tau"], rtol=1e-3)
    np.testing.assert_allclose(g_Tw, fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
    assert g_Q == pytest.approx(fd["g_Q"], rel=1e-3)


def test_adjoint_rowblock_matches_general(bte):
    """2D unmasked square: the row-block kernel's adjoint equals the general
    kernel's (FP64)."""
    p = bi.square_2d(n=20, L=0.3e-6)
    p = p.copy(C=p.C[:4], v=p.v[:4], tau=p.tau[:4])
    plan = bte.Plan(p)
    g = np.zeros(p.n_cells)
    g[[5, 77, 230, 399]] = [1.0, -0.5, 0.25, 2.0]
    out = []
    for kind in (1, 2):
        T = np.zeros(p.n_cells)
        plan.solve(T, precision=bte.BTE_FP64, tol=1e-13, tile_kind=kind)
        rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-13)
        out.append((g_tau, g_Tw))
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-9)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-9, atol=1e-15)


def test_adjoint_rowpipe_matches_general(bte):
    """2D unmasked 70 x 70 square (three 32-row blocks, the last ragged): the
    row-pipeline and row-block kernels' adjoints equal the general kernel's
    (FP64)."""
    p = bi.square_2d(n=70, L=0.6e-6)
    p = p.copy(C=p.C[:3], v=p.v[:3], tau=p.tau[:3])
    plan = bte.Plan(p)
    g = np.zeros(p.n_cells)
    g[[5, 777, 2300, 4899]] = [1.0, -0.5, 0.25, 2.0]
    out = []
    for kind in (1, 2, 3):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-13, tile_kind=kind)
        assert st["tile_kind"] == kind
        rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-13)
        out.append((g_tau, g_Tw, g_Q))
    for o in out[1:]:
        np.testing.assert_allclose(o[0], out[0][0], rtol=1e-9)
        np.testing.assert_allclose(o[1], out[0][1], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
def test_fp32_adjoint_within_fd_tolerance(bte, name, dim, kw):
    p, ref, probes, T_obs = _setup(dim, kw)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP32, tol=1e-9, max_iter=100000, check=False)
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, ref["T"][probes] - T_obs)
    rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-9, check=False)
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(g_tau, fd["g_tau"], rtol=1e-3)
    np.testing.assert_allclose(g_Tw, fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
    assert g_Q == pytest.approx(fd["g_Q"], rel=1e-3)


def test_autograd_function(bte):
    from paper_2503_23657_gb300.autograd import bte_temperature, probe_loss
    p, ref, probes, T_obs = _setup(*CASES[1][1:])
    plan = bte.Plan(p)
    tau = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
    Tw = torch.tensor(p.bc_T, dtype=torch.float64, requires_grad=True)
    Q = torch.tensor(p.Q_amp, dtype=torch.float64, requires_grad=True)
    T = bte_temperature(plan, tau, Tw, Q, precision=bte.BTE_FP64, tol=1e-14, adj_tol=1e-14)
    J = probe_loss(T, torch.as_tensor(probes, device="cuda"), torch.as_tensor(T_obs, device="cuda"))
    J.backward()
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(tau.grad.numpy(), fd["g_tau"], rtol=1e-3)
    np.testing.assert_allclose(Tw.grad.numpy(), fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
    assert float(Q.grad) == pytest.approx(fd["g_Q"], rel=1e-3)
