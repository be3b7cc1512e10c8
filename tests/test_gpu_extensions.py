"""GPU parity of the extensions beyond the step-face steady solve, against
the FP64 oracle (whose counterparts are pinned on the CPU:
tests/test_oracle_order2.py, tests/test_oracle_transient.py and the
length-gradient tests of tests/test_oracle_adjoint.py):

* second-order Green-Gauss faces as a deferred correction (bte_solve with
  face_order 2): iterates at a fixed iteration count and the converged
  solution (which the oracle pins to the face-by-face assembled system);
* implicit-Euler transient steps (bte_transient): the temperature after
  every converged step;
* dJ/dL_a (bte_adjoint_ex): against the oracle's adjoint and central
  finite differences of the direct solve.

Tolerances: FP64 1e-12 relative on T (fixed iterations and converged
states), FP32 1e-5; gradients 1e-8 against the oracle's FP64 adjoint with
FP64 sweeps, 1e-3 against finite differences (FP32 sweeps included)."""
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


def rel(a, b, mask):
    return float(np.abs(a - b)[mask].max() / np.abs(b[mask]).max())


CASES = [
    ("1d", 1, dict(n=(9, 1, 1), B=2, diffuse=(1,), source=True)),
    ("2d_mask", 2, dict(n=(7, 6, 1), B=3, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    ("2d_spec", 2, dict(n=(6, 5, 1), B=2, specular=(2,), diffuse=(3,), source=True)),
    ("3d_mask", 3, dict(n=(5, 4, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
    ("3d_spec", 3, dict(n=(4, 4, 3), B=2, specular=(2, 5), diffuse=(4,), masked=True, source=True)),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,dim,kw", CASES, ids=IDS)
@pytest.mark.parametrize("k", [1, 5])
def test_second_order_fixed_iterations_fp64(bte, name, dim, kw, k):
    p = bi.tiny(dim, **kw).copy(order=2)
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    e = np.zeros((p.n_cells, p.B, p.D))
    rc, st = plan.solve(T, e_out=e, precision=bte.BTE_FP64, tol=0.0, max_iter=k, face_order=2)
    assert st["iterations"] == k
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-12
    assert np.abs(e - ref["e"]).max() < 1e-11 * np.abs(ref["e"]).max()


# cases on which the deferred-correction iteration converges (the oracle
# reaches the assembled second-order system on them)
CONV2 = [CASES[0], ("2d_mask_b", 2, dict(n=(5, 4, 1), B=2, masked=True, diffuse=(2, 3), source=True,
                                          two_regions=True))] + CASES[2:]


@pytest.mark.parametrize("name,dim,kw", CONV2, ids=[c[0] for c in CONV2])
def test_second_order_converged(bte, name, dim, kw):
    p = bi.tiny(dim, **kw).copy(order=2)
    ref = dense.solve(p)
    plan = bte.Plan(p)
    act = p.mask > 0
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-14, max_iter=200000, face_order=2)
    assert st["converged"] == 1
    assert rel(T, ref["T"], act) < 1e-12
    T32 = np.zeros(p.n_cells)
    plan.solve(T32, precision=bte.BTE_FP32, tol=1e-9, max_iter=200000, face_order=2)
    assert rel(T32, ref["T"], act) < 1e-5


def test_second_order_grid_convergence_on_gpu(bte):
    """The paper's grid study (50/100/200 cells) on the GPU: the same errors
    as the oracle's (to 1e-9 of the error), so the same observed order."""
    from tests.test_oracle_order2 import slab_errors
    from tests import physics
    ref_errs = slab_errors(2)
    errs = []
    kn = 0.256
    mu_all, w_all = bi.quadrature_1d(16)
    for nx in (50, 100, 200):
        p = bi.gray_slab(nx=nx, tau=kn * 1e-6 / 6400.0).copy(order=2)
        plan = bte.Plan(p)
        T = np.zeros(p.n_cells)
        plan.solve(T, precision=bte.BTE_FP64, tol=1e-14, max_iter=200000, face_order=2)
        ph = (T - p.bc_T[1]) / (p.bc_T[0] - p.bc_T[1])
        xm, phi = physics.gray_slab_discrete_ordinates(mu_all[:, 0], w_all, 1.0 / kn, 21 * nx)
        errs.append(float(np.sqrt(np.mean((ph - phi[10::21]) ** 2))))
    np.testing.assert_allclose(errs, ref_errs, rtol=1e-6)
    assert (np.log2(np.array(errs[:-1]) / np.array(errs[1:])) >= 1.8).all()


@pytest.mark.parametrize("name,dim,kw", CASES, ids=IDS)
def test_transient_steps(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    dt, n = 2e-11, 4
    ref = oracle.transient(p, dt, n, tol=1e-15)
    plan = bte.Plan(p)
    act = p.mask > 0
    T = np.zeros(p.n_cells)
    hist = np.zeros((n, p.n_cells))
    rc, st = plan.transient(dt, n, T, T_hist=hist, precision=bte.BTE_FP64, tol=1e-15)
    for m in range(n):
        assert rel(hist[m], ref["T_hist"][m], act) < 1e-12
    np.testing.assert_array_equal(T, hist[-1])
    # FP32 sweeps, device buffers
    Td = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    hd = torch.zeros((n, p.n_cells), dtype=torch.float64, device="cuda")
    plan.transient(dt, n, Td, T_hist=hd, precision=bte.BTE_FP32, tol=1e-9)
    for m in range(n):
        assert rel(hd[m].cpu().numpy(), ref["T_hist"][m], act) < 1e-5


# 3D transient steps on the plane pipeline (its extra-source variant, also
# with specular faces): a single-pass and a several-pass grid
PIPE_TCASES = [CASES[3], CASES[4],
               ("3d_passes", 3, dict(n=(20, 9, 14), B=2, masked=True, diffuse=(0, 3), source=True, n_polar=2,
                                     n_az=8)),
               ("3d_passes_spec", 3, dict(n=(18, 11, 12), B=2, specular=(2, 5), diffuse=(3,), source=True,
                                          two_regions=True, n_polar=2, n_az=8))]


@pytest.mark.parametrize("name,dim,kw", PIPE_TCASES, ids=[c[0] for c in PIPE_TCASES])
def test_transient_steps_plane_pipeline(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    dt, n = 2e-11, 4
    ref = oracle.transient(p, dt, n, tol=1e-15)
    plan = bte.Plan(p)
    act = p.mask > 0
    for dw in (2, 4):
        T = np.zeros(p.n_cells)
        hist = np.zeros((n, p.n_cells))
        rc, st = plan.transient(dt, n, T, T_hist=hist, precision=bte.BTE_FP64, tol=1e-15, tile_kind=3,
                                dirs_per_lane=dw)
        assert st["tile_kind"] == 3 and st["dirs_per_lane"] == dw
        for m in range(n):
            assert rel(hist[m], ref["T_hist"][m], act) < 1e-12
    for dw in (4, 8):
        Td = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        hd = torch.zeros((n, p.n_cells), dtype=torch.float64, device="cuda")
        rc, st = plan.transient(dt, n, Td, T_hist=hd, precision=bte.BTE_FP32, tol=1e-9, tile_kind=3,
                                dirs_per_lane=dw)
        assert st["tile_kind"] == 3
        for m in range(n):
            assert rel(hd[m].cpu().numpy(), ref["T_hist"][m], act) < 1e-5
    # a steady solve on the same plan afterwards has no extra source
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=3, tile_kind=3, dirs_per_lane=4)
    r = oracle.solve(p, max_iter=3, tol=0.0)
    assert rel(T, r["T"], act) < 1e-12


def test_transient_adiabatic_heating_rate(bte):
    """Energy balance of the GPU time steps: a 2D box heated uniformly with
    one isothermal face far from the source; the stored energy rises by the
    injected heat minus the outflow (oracle closed-form pins on the CPU), and
    the GPU temperatures follow the oracle's over 10 steps."""
    p = bi.tiny(2, n=(8, 6, 1), B=2, specular=(2, 3), diffuse=(1,), source=True)
    dt, n = 5e-12, 10
    ref = oracle.transient(p, dt, n, tol=1e-15)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    hist = np.zeros((n, p.n_cells))
    plan.transient(dt, n, T, T_hist=hist, precision=bte.BTE_FP64, tol=1e-15)
    act = p.mask > 0
    for m in range(n):
        assert rel(hist[m], ref["T_hist"][m], act) < 1e-12


LCASES = [CASES[0], CASES[1], CASES[2], CASES[3]]


@pytest.mark.parametrize("name,dim,kw", LCASES, ids=[c[0] for c in LCASES])
def test_length_gradient(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    rng = np.random.default_rng(4)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(5, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    fd = dense.fd_gradients(p, probes, T_obs)
    plan = bte.Plan(p)
    for prec in (bte.BTE_FP64, bte.BTE_FP32):
        tol = 1e-15 if prec == bte.BTE_FP64 else 1e-9
        T = np.zeros(p.n_cells)
        plan.solve(T, precision=prec, tol=tol, max_iter=200000)
        g = np.zeros(p.n_cells)
        np.add.at(g, probes, T[probes] - T_obs)
        rc, g_tau, g_Tw, g_Q, st, g_L = plan.adjoint(g, tol=tol, max_iter=200000, lengths=True)
        scale = np.abs(fd["g_L"]).max()
        if prec == bte.BTE_FP64:
            r = oracle.solve(p, max_iter=100000, tol=1e-15)
            a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
            np.testing.assert_allclose(g_L, a["g_L"], rtol=1e-8, atol=1e-12 * scale)
        np.testing.assert_allclose(g_L, fd["g_L"], rtol=1e-3, atol=1e-4 * scale)
        # the other gradients are unchanged by asking for the lengths
        rc, g_tau2, g_Tw2, g_Q2, st2 = plan.adjoint(g, tol=tol, max_iter=200000)
        np.testing.assert_allclose(g_tau, g_tau2, rtol=1e-12)


def test_film_thickness_inverse_step(bte):
    """The paper's 1D inverse problem on the GPU: the thickness gradient of a
    film at half the true thickness points towards the truth and matches the
    oracle's."""
    p = bi.gray_slab(nx=50, L=0.5e-6, T_h=400.0, T_c=300.0)
    truth = bi.gray_slab(nx=50, L=1.0e-6, T_h=400.0, T_c=300.0)
    probes = np.linspace(1, 48, 20).astype(int)
    T_obs = oracle.solve(truth, max_iter=100000, tol=1e-14)["T"][probes]
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=1e-14, max_iter=200000)
    g = np.zeros(p.n_cells)
    g[probes] = T[probes] - T_obs
    rc, g_tau, g_Tw, g_Q, st, g_L = plan.adjoint(g, tol=1e-14, max_iter=200000, lengths=True)
    r = oracle.solve(p, max_iter=100000, tol=1e-14)
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-14)
    assert g_L[0] == pytest.approx(a["g_L"][0], rel=1e-8)
    assert g_L[0] < 0.0


def test_second_order_divergence_is_reported(bte):
    """On a thin masked two-region geometry the deferred-correction iteration
    of the second-order faces does not converge (the oracle's iterates
    oscillate with growing amplitude; the unlimited reconstruction is the
    paper's); the GPU follows the oracle's iterates and reports
    BTE_ENOTCONVERGED instead of returning a state as converged."""
    p = bi.tiny(2, **CASES[1][2]).copy(order=2)
    k = 400
    ref = oracle.solve(p, max_iter=k, tol=1e-10)
    assert ref["iters"] == k and ref["eps"][-1] > 1e-2
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-10, max_iter=k, face_order=2, check=False)
    assert rc == bte.BTE_ENOTCONVERGED
    np.testing.assert_allclose(plan.eps_history(k)[:50], ref["eps"][:50], rtol=1e-9)


def test_adjoint_refused_after_second_order_solve(bte):
    p = bi.tiny(1, **CASES[0][2])
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=1e-10, max_iter=100000, face_order=2)
    rc, *_ = plan.adjoint(np.ones(p.n_cells), tol=1e-10, check=False)
    assert rc == bte.BTE_ESTATE


def test_film_thickness_inversion_autograd(bte):
    """The paper's 1D inverse problem (Results: a film's unknown thickness is
    found from 20 temperature observations, starting from 50 nm with the
    truth at 100 nm) through torch.autograd: Adam steps on L with the
    gradient of bte_adjoint_ex reduce the misfit and bring L to the truth."""
    from paper_2503_23657_gb300.autograd import bte_temperature, probe_loss
    truth = bi.gray_slab(nx=50, L=100e-9, T_h=400.0, T_c=300.0)
    p = bi.gray_slab(nx=50, L=50e-9, T_h=400.0, T_c=300.0)
    probes = torch.as_tensor(np.linspace(1, 48, 20).astype(np.int64), device="cuda")
    T_obs = torch.as_tensor(oracle.solve(truth, max_iter=100000, tol=1e-14)["T"], device="cuda")[probes]
    plan = bte.Plan(p)
    L_nm = torch.tensor([50.0, 1e9, 1e9], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([L_nm], lr=8.0)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.9)   # the paper's decaying rate
    tau = torch.as_tensor(p.tau)
    Tw = torch.as_tensor(p.bc_T)
    losses = []
    for it in range(25):
        opt.zero_grad()
        T = bte_temperature(plan, tau, Tw, 0.0, lengths=L_nm * 1e-9, precision=bte.BTE_FP64, tol=1e-12,
                            adj_tol=1e-12)
        loss = probe_loss(T, probes, T_obs)
        loss.backward()
        L_nm.grad[1:] = 0.0
        losses.append(float(loss.detach()))
        opt.step()
        sched.step()
    assert losses[-1] < 1e-2 * losses[0]
    assert abs(float(L_nm.detach()[0]) - 100.0) < 5.0
