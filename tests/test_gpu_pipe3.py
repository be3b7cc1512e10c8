"""GPU parity of the plane-pipeline 3D sweep (tile_kind 3 on 3D grids) against
the FP64 oracle and the general wavefront kernel.

The cases cover: a single pass (all planes in flight at once), several passes
(the first warp of a pass reading the last plane of the previous one), a
ragged last pass, rows beyond the grid in the last 32-row warp, masks with
void cells inside and on the walls, two regions, diffuse and isothermal walls,
a source profile, and every instantiated number of directions per lane.
Tolerances as in test_gpu_parity: FP32 sweeps within 1e-5 of the oracle's T
(relative to max |T|) at a fixed iteration count from the same T_init.
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


def heights(n, lane_axis=1):
    """Warps along the plane axis the kernel accepts for an nx x ny x nz grid
    whose lanes hold rows along y (lane_axis 1, planes along z) or z
    (lane_axis 2, planes along y): at most 16 warps per CTA (ceil(rows / 32)
    along the rows), and a grid of several passes needs two warps along the
    planes and nx >= 4 H + 2."""
    nx, ny, nz = n
    rows, planes = (ny, nz) if lane_axis == 1 else (nz, ny)
    wy = -(-rows // 32)
    out = []
    for H in range(1, 17):
        if wy * H > 16 or H > planes:
            continue
        if -(-planes // H) > 1 and (H < 2 or nx < 4 * H + 2):
            continue
        out.append(H)
    return out


def rel(a, b, mask):
    return float(np.abs(a[mask] - b[mask]).max() / np.abs(b[mask]).max())


CASES = [
    ("one_pass", dict(n=(4, 3, 3), B=2)),
    ("one_pass_mask", dict(n=(6, 5, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)),
    ("passes", dict(n=(22, 40, 19), B=2, diffuse=(1, 2, 4), source=True, n_polar=4, n_az=16)),
    ("passes_mask", dict(n=(26, 35, 23), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True,
                         n_polar=2, n_az=16)),
    ("flat", dict(n=(40, 9, 2), B=3, diffuse=(2, 3), source=True, n_polar=2, n_az=16)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dw", [2, 4, 8])
@pytest.mark.parametrize("axis", [1, 2], ids=["rows_y", "rows_z"])
def test_fp32_fixed_iterations(bte, name, kw, dw, axis):
    p = bi.tiny(3, **kw)
    k = 12
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    plan = bte.Plan(p)
    hs = heights(p.n, axis)
    assert hs, "every case has a plane-pipeline tile"
    T_gen = np.zeros(p.n_cells)
    plan.solve(T_gen, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=dw if dw != 2 else 4, tile_kind=1)
    for H in sorted({hs[0], hs[len(hs) // 2], hs[-1]}):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=dw, tile_kind=3,
                            warps_z=H, lane_axis=axis)
        assert st["tile_kind"] == 3 and st["warps_z"] == H and st["dirs_per_lane"] == dw
        assert st["lane_axis"] == axis
        assert st["iterations"] == k
        assert rel(T, ref["T"], act) < 1e-5
        assert np.abs(T - ref["T"])[act].max() < 1e-4 * np.ptp(ref["T"][act]) + 1e-9
        # same arithmetic as the general kernel up to the direction grouping
        assert rel(T, T_gen, act) < 2e-6


@pytest.mark.parametrize("name,kw", CASES[2:4], ids=[c[0] for c in CASES[2:4]])
def test_matches_general_kernel_bitwise_at_same_grouping(bte, name, kw):
    """With four directions per lane both kernels form the same per-subset
    sums in the same order: the temperatures agree to the last bit."""
    p = bi.tiny(3, **kw)
    plan = bte.Plan(p)
    k = 9
    T_gen = np.zeros(p.n_cells)
    plan.solve(T_gen, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=4, tile_kind=1)
    for H in heights(p.n)[-2:]:
        T = np.zeros(p.n_cells)
        plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k, dirs_per_lane=4, tile_kind=3, warps_z=H,
                   lane_axis=1)
        np.testing.assert_array_equal(T, T_gen)


def test_e_output_and_flux(bte):
    """The regenerated final e (the e-store variant of the kernel) and the
    flux from it, against the oracle after a fixed iteration count."""
    p = bi.tiny(3, **CASES[3][1])
    k = 6
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    q = np.zeros((p.n_cells, 3))
    e = np.zeros((p.n_cells, p.B, p.D), dtype=np.float32)
    rc, st = plan.solve(T, q_out=q, e_out=e, precision=bte.BTE_FP32, tol=0.0, max_iter=k, tile_kind=3,
                        dirs_per_lane=4)
    assert st["tile_kind"] == 3 and st["warps_z"] > 0
    act = p.mask > 0
    escale = np.abs(ref["e"][act]).max()
    assert np.abs(e[act] - ref["e"][act]).max() < 2e-5 * escale
    qs = np.abs(ref["q"][act]).max()
    assert np.abs(q[act] - ref["q"][act]).max() < 1e-3 * qs


def test_converged_reduced_grid(bte):
    """A 3D case with passes converged to eps_T < 1e-6 in FP32: same
    iteration count as the oracle (within one) and T within 1e-5."""
    p = bi.tiny(3, **CASES[2][1])
    ref = oracle.solve(p, max_iter=100000, tol=1e-6)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-6, tile_kind=3)
    assert st["converged"] == 1 and st["tile_kind"] == 3
    assert abs(st["iterations"] - ref["iters"]) <= 1
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-5


def test_adjoint_matches_oracle_and_fd(bte):
    """FP32 adjoint through the plane-pipeline kernel (nu = mu / w carried in
    the sweep) on a masked two-region grid: gradients within 1e-3 of central
    finite differences and of the oracle's FP64 adjoint."""
    p = bi.tiny(3, n=(5, 4, 4), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True)
    ref = dense.solve(p)
    rng = np.random.default_rng(11)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(6, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-9, max_iter=100000, tile_kind=3, check=False)
    assert st["tile_kind"] == 3 and st["warps_z"] > 0
    g = np.zeros(p.n_cells)
    np.add.at(g, probes, ref["T"][probes] - T_obs)
    rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-9, check=False)
    fd = dense.fd_gradients(p, probes, T_obs)
    np.testing.assert_allclose(g_tau, fd["g_tau"], rtol=1e-3)
    np.testing.assert_allclose(g_Tw, fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
    assert g_Q == pytest.approx(fd["g_Q"], rel=1e-3)


def test_adjoint_passes_matches_general(bte):
    """Several passes and a mask: the FP32 adjoint gradients of the plane
    pipeline (rows along y and along z) agree with the general kernel's to
    1e-4."""
    p = bi.tiny(3, **CASES[3][1])
    plan = bte.Plan(p)
    act = np.flatnonzero(p.mask)
    g = np.zeros(p.n_cells)
    g[act[[3, 200, 1500, act.size - 7]]] = [1.0, -0.5, 0.25, 2.0]
    out = []
    for kind, axis in ((1, 0), (3, 1), (3, 2)):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=1e-7, tile_kind=kind, dirs_per_lane=4, lane_axis=axis,
                            check=False)
        assert st["lane_axis"] == axis
        rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-7, check=False)
        out.append((g_tau, g_Tw, g_Q))
    for o in out[1:]:
        np.testing.assert_allclose(o[0], out[0][0], rtol=1e-4)
        np.testing.assert_allclose(o[1], out[0][1], rtol=1e-4, atol=1e-4 * np.abs(out[0][1]).max())
        assert o[2] == pytest.approx(out[0][2], rel=1e-4)


def test_fp64_adjoint_gradients_match_oracle(bte):
    """FP64 adjoint through the plane pipeline (rows along y and along z, two
    warps along the planes: five or six passes), whose final pass runs the
    transposed sweep and then its gradient form, on a masked two-region grid
    with a source: dJ/dtau, dJ/dT_wall and dJ/dQ_amp within 1e-9 of the
    oracle's FP64 adjoint (1e-8 for the tiny dJ/dQ_amp), like the general
    kernel's."""
    p = bi.tiny(3, n=(14, 10, 12), B=2, masked=True, diffuse=(0, 3, 5), source=True, two_regions=True,
                n_polar=2, n_az=16)
    act = np.flatnonzero(p.mask)
    g = np.zeros(p.n_cells)
    g[act[[3, 50, 300, act.size - 7]]] = [1.0, -0.5, 0.25, 2.0]
    r = oracle.solve(p, max_iter=100000, tol=1e-13)
    a = oracle.adjoint(p, r["e"], r["T"], g, max_iter=100000, tol=1e-13)
    plan = bte.Plan(p)
    for kind, axis in ((1, 0), (3, 1), (3, 2)):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-13, max_iter=100000, tile_kind=kind,
                            dirs_per_lane=4, lane_axis=axis, warps_z=2 if kind == 3 else 0)
        assert st["lane_axis"] == axis and st["tile_kind"] == (3 if kind == 3 else 1)
        rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=1e-13, max_iter=100000)
        np.testing.assert_allclose(g_tau, a["g_tau"], rtol=1e-9)
        np.testing.assert_allclose(g_Tw, a["g_Tw"], rtol=1e-9, atol=1e-9 * np.abs(a["g_Tw"]).max())
        assert g_Q == pytest.approx(a["g_Q"], rel=1e-8)


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dw", [2, 4])
@pytest.mark.parametrize("axis", [1, 2], ids=["rows_y", "rows_z"])
def test_fp64_fixed_iterations(bte, name, kw, dw, axis):
    """FP64 sweeps through the plane pipeline: within 1e-12 of the oracle."""
    p = bi.tiny(3, **kw)
    k = 7
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    plan = bte.Plan(p)
    hs = heights(p.n, axis)
    for H in sorted({hs[0], hs[-1]}):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=k, dirs_per_lane=dw, tile_kind=3,
                            warps_z=H, lane_axis=axis)
        assert st["tile_kind"] == 3 and st["warps_z"] == H and st["lane_axis"] == axis
        assert rel(T, ref["T"], act) < 1e-12


def test_rejections(bte):
    """warps_z that the grid cannot take is refused (EINVAL), and FP64 has no
    eight-direction plane-pipeline tile."""
    from paper_2503_23657_gb300 import binding
    p = bi.tiny(3, **CASES[2][1])
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    bad = [H for H in range(1, 17) if H not in heights(p.n)]
    rc, st = plan.solve(T, tol=0.0, max_iter=2, tile_kind=3, warps_z=bad[0], check=False)
    assert rc == binding.BTE_EINVAL
    rc, st = plan.solve(T, tol=0.0, max_iter=2, tile_kind=3, warps_z=17, check=False)
    assert rc == binding.BTE_EINVAL
    rc, st = plan.solve(T, tol=0.0, max_iter=2, tile_kind=3, lane_axis=3, check=False)
    assert rc == binding.BTE_EINVAL
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=0.0, max_iter=2, tile_kind=3, dirs_per_lane=8, check=False)
    assert rc == binding.BTE_EINVAL
