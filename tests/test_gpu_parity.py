"""GPU parity: libbte (through the C ABI) against the FP64 oracle.

Tolerances (north-star targets; "relative" = max_c |T_gpu - T_oracle| / max_c |T_oracle|):
  * FP64 sweeps: 1e-12 relative on T, same iteration count;
  * FP32 sweeps: 1e-5 relative on T;
  * gradients: 1e-3 relative to central finite differences.
Comparisons at a fixed iteration count run both sides from the same T_init for
exactly k iterations; comparisons at convergence use the same eps_T rule.
"""
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


def rowblock_eligible(p):
    """The row-block kernel handles unmasked 1D/2D grids with one region."""
    return p.dim <= 2 and bool(np.all(p.mask == 1)) and p.n[1] <= 256


def rel(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.abs(a - b).max() / np.abs(b).max())


TINY = [
    ("1d", 1, dict(n=(9, 1, 1), B=3, diffuse=(1,), source=True)),
    ("2d", 2, dict(n=(5, 4, 1), B=2)),
    ("2d_mask", 2, dict(n=(7, 6, 1), B=3, masked=True, diffuse=(2, 3), source=True, two_regions=True)),
    ("2d_tall", 2, dict(n=(3, 70, 1), B=2, diffuse=(0,), source=True)),
    ("3d", 3, dict(n=(4, 3, 3), B=2)),
    ("3d_mask", 3, dict(n=(6, 5, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
    ("3d_deep", 3, dict(n=(5, 40, 37), B=1, diffuse=(2, 5), source=True, n_polar=2, n_az=4)),
]


@pytest.mark.parametrize("name,dim,kw", TINY, ids=[t[0] for t in TINY])
@pytest.mark.parametrize("k", [1, 7])
@pytest.mark.parametrize("kind", [1, 2, 3])
def test_fp64_fixed_iterations(bte, name, dim, kw, k, kind):
    p = bi.tiny(dim, **kw)
    if kind >= 2 and not rowblock_eligible(p):
        pytest.skip("row-block kernel needs an unmasked 1D/2D grid")
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    q = np.zeros((p.n_cells, 3))
    e = np.zeros((p.n_cells, p.B, p.D))
    rc, st = plan.solve(T, q_out=q, e_out=e, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=kind)
    assert st["tile_kind"] == kind
    act = p.mask > 0
    assert st["iterations"] == k
    assert rel(T, ref["T"], act) < 1e-12
    assert np.abs(e - ref["e"]).max() < 1e-12 * np.abs(ref["e"]).max()
    assert np.abs(q - ref["q"]).max() < 1e-10 * np.abs(ref["q"]).max() + 1e-300
    np.testing.assert_allclose(plan.eps_history(k), ref["eps"], rtol=1e-9, atol=1e-300)


TILES = [(0, 0), (1, 4), (1, 8), (2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 4)]


@pytest.mark.parametrize("name,dim,kw", TINY, ids=[t[0] for t in TINY])
@pytest.mark.parametrize("kind,dw", TILES, ids=[f"k{a}dw{b}" for a, b in TILES])
def test_fp32_fixed_iterations(bte, name, dim, kw, kind, dw):
    p = bi.tiny(dim, **kw)
    if kind >= 2 and not rowblock_eligible(p):
        pytest.skip("row-block kernel needs an unmasked 1D/2D grid")
    k = 12
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=dw, tile_kind=kind)
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-5
    # and relative to the temperature variation itself
    assert np.abs(T - ref["T"])[act].max() < 1e-4 * np.ptp(ref["T"][act]) + 1e-9


@pytest.mark.parametrize("name,dim,kw", TINY, ids=[t[0] for t in TINY])
def test_fp64_converged_matches_direct_solve(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-14, max_iter=100000)
    assert st["converged"] == 1
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-12


def test_slab_fp64_to_convergence(bte):
    """1D gray slab, FP64, eps_T < 1e-10: same iteration count as the oracle
    and T within 1e-12."""
    p = bi.gray_slab()
    ref = oracle.solve(p, max_iter=100000, tol=1e-10)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-10, max_iter=100000)
    assert st["iterations"] == ref["iters"]
    assert rel(T, ref["T"]) < 1e-12


def test_square2d_full_size_fixed_iterations(bte):
    """The 128x128, 15-band, 64-direction square at full size, 20 iterations
    from T = 300 K: FP32 within 1e-5 and FP64 within 1e-12 of the oracle."""
    p = bi.square_2d()
    k = 20
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    for kind in (1, 2, 3):
        plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=kind)
        assert rel(T, ref["T"]) < 1e-12
    for kind, dw in [(1, 4), (1, 8), (1, 16), (2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 4), (0, 0)]:
        T32 = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        rc, st = plan.solve(T32, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=dw, tile_kind=kind)
        assert rel(T32.cpu().numpy(), ref["T"]) < 1e-5
        if kind:
            assert st["tile_kind"] == kind


def test_square2d_reduced_converged(bte):
    """32x32 square converged to eps_T < 1e-6 in FP32 and FP64: iteration
    count and T agree with the oracle."""
    p = bi.square_2d(n=32)
    ref = oracle.solve(p, max_iter=100000, tol=1e-6)
    plan = bte.Plan(p)
    for prec, tolT in ((bte.BTE_FP64, 1e-12), (bte.BTE_FP32, 1e-5)):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=prec, tol=1e-6, max_iter=100000)
        assert abs(st["iterations"] - ref["iters"]) <= (0 if prec == bte.BTE_FP64 else 2)
        assert rel(T, ref["T"]) < tolT


def test_hotspot3d_reduced_fixed_iterations(bte):
    p = bi.hotspot_3d(n=16, L=0.25e-6, sigma=12.5e-9)
    k = 3
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k)
    assert rel(T, ref["T"]) < 1e-12
    plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k)
    assert rel(T, ref["T"]) < 1e-5


def test_finfet_reduced_fixed_iterations(bte):
    p = bi.finfet_3d(scale=4, n_polar=4, n_az=8)
    k = 3
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    act = p.mask > 0
    plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k)
    assert rel(T, ref["T"], act) < 1e-12
    plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k)
    assert rel(T, ref["T"], act) < 1e-5


@pytest.mark.parametrize("cw", [1, 2, 4, 8, 16])
def test_rowpipe_direction_chunks(bte, cw):
    """Row-pipeline kernel with every chunk width on a 37 x 70 grid (three
    row blocks, the last one ragged) with a source and diffuse walls: FP64
    within 1e-12 of the oracle after 5 iterations."""
    p = bi.tiny(2, n=(37, 70, 1), B=2, diffuse=(1, 2), source=True, n_polar=4, n_az=16)
    k = 5
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    dw = min(cw, 4)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=3, dirs_per_lane=dw,
                        dirs_per_cta=cw)
    assert st["tile_kind"] == 3 and st["dirs_per_cta"] == cw
    assert rel(T, ref["T"]) < 1e-12


def test_device_and_host_outputs_agree(bte):
    p = bi.tiny(2, n=(6, 5, 1), B=2, diffuse=(2,), source=True)
    plan = bte.Plan(p)
    Th = np.zeros(p.n_cells)
    eh = np.zeros((p.n_cells, p.B, p.D), dtype=np.float32)
    plan.solve(Th, e_out=eh, precision=bte.BTE_FP32, tol=0.0, max_iter=5)
    Td = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    ed = torch.zeros((p.n_cells, p.B, p.D), dtype=torch.float32, device="cuda")
    plan.solve(Td, e_out=ed, precision=bte.BTE_FP32, tol=0.0, max_iter=5)
    np.testing.assert_array_equal(Td.cpu().numpy(), Th)
    np.testing.assert_array_equal(ed.cpu().numpy(), eh)


@pytest.mark.parametrize("kind", [2, 3])
def test_row_kernels_rejected_for_masked_grid(bte, kind):
    p = bi.tiny(2, n=(7, 6, 1), B=2, masked=True, diffuse=(2,))
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, tol=0.0, max_iter=2, tile_kind=kind, check=False)
    assert rc == -1


def test_store_every_iteration_same_result(bte):
    p = bi.tiny(3, n=(5, 4, 4), B=2, diffuse=(3,), source=True)
    plan = bte.Plan(p)
    a = np.zeros(p.n_cells)
    b = np.zeros(p.n_cells)
    plan.solve(a, precision=bte.BTE_FP32, tol=0.0, max_iter=6, store_e_every_iter=False)
    plan.solve(b, precision=bte.BTE_FP32, tol=0.0, max_iter=6, store_e_every_iter=True)
    np.testing.assert_array_equal(a, b)


def test_solve_is_deterministic(bte):
    p = bi.square_2d(n=48)
    plan = bte.Plan(p)
    a = np.zeros(p.n_cells)
    b = np.zeros(p.n_cells)
    plan.solve(a, tol=0.0, max_iter=40)
    plan.solve(b, tol=0.0, max_iter=40)
    np.testing.assert_array_equal(a, b)


def test_not_converged_status(bte):
    p = bi.square_2d(n=16)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, tol=1e-12, max_iter=3, check=False)
    assert rc == -4 and st["iterations"] == 3 and T.max() > 300.0


@pytest.mark.parametrize("dim", [2, 3])
def test_overflow_is_a_numeric_error(bte, dim):
    """A finite source amplitude too large for FP32 (the per-band source
    overflows to Inf in the sweep) is caught by the update's finiteness check
    and reported as BTE_ENUMERIC, not as convergence or a silent NaN field."""
    p = bi.tiny(dim, n=(6, 5, 4), B=2, source=True)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-6, max_iter=50, Q_amp=1e300, check=False)
    assert rc == -6
    # the plan stays usable
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=3)
    assert rc == 0 and np.isfinite(T).all()


def test_adjoint_before_solve_is_state_error(bte):
    p = bi.tiny(2)
    plan = bte.Plan(p)
    rc, *_ = plan.adjoint(np.zeros(p.n_cells), check=False)
    assert rc == -7


def test_sweep_timing_events(bte):
    """bte_set_sweep_timing: one event-timed sweep per iteration (forward and
    adjoint), durations inside the loop time, results unchanged."""
    p = bi.square_2d(n=40)
    plan = bte.Plan(p)
    a = np.zeros(p.n_cells)
    rc, s0 = plan.solve(a, tol=0.0, max_iter=37)
    assert s0["sweep_launches"] == 0 and s0["sweep_seconds"] == 0.0
    plan.set_sweep_timing(1)
    b = np.zeros(p.n_cells)
    rc, s1 = plan.solve(b, tol=0.0, max_iter=37)     # one 32-iteration graph + 5 direct
    np.testing.assert_array_equal(a, b)
    assert s1["sweep_launches"] == 37
    assert 0.0 < s1["sweep_seconds"] < s1["seconds"]
    rc, s3 = plan.solve(b, tol=0.0, max_iter=64)     # graph replays only
    assert s3["sweep_launches"] == 64
    assert 0.3 * s3["seconds"] < s3["sweep_seconds"] < s3["seconds"]
    g = np.zeros(p.n_cells)
    g[::7] = 1.0
    rc, *_, sa = plan.adjoint(g, tol=0.0, max_iter=21)
    assert sa["sweep_launches"] == 21 and 0.0 < sa["sweep_seconds"] < sa["seconds"]
    plan.set_sweep_timing(8)                          # iterations 0, 8, 16, 24 of each graph
    rc, s4 = plan.solve(b, tol=0.0, max_iter=64)
    assert s4["sweep_launches"] == 8
    assert 0.0 < s4["sweep_seconds"] < s4["seconds"] / 4
    plan.set_sweep_timing(0)
    c = np.zeros(p.n_cells)
    rc, s2 = plan.solve(c, tol=0.0, max_iter=37)
    np.testing.assert_array_equal(a, c)
    assert s2["sweep_launches"] == 0
