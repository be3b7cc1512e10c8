"""GPU parity of specularly reflecting faces (Methods, Boundary conditions:
a specular wall returns into direction d what the cell sends out through it
in the mirror direction of d, taken from the previous iterate) against the
FP64 oracle, whose specular faces are pinned on the CPU (reduction to the 1D
slab, method of images, direct solve, zero net heat, finite differences).

Tolerances as in test_gpu_parity.py: FP64 1e-12 relative on T and e, FP32
1e-5 relative on T, adjoint gradients 1e-8 against the oracle's FP64 adjoint
(FP64 sweeps) and 1e-3 against central finite differences."""
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
    ("2d_mixed", 2, dict(n=(6, 5, 1), B=2, specular=(2,), diffuse=(3,), source=True)),
    ("2d_mask", 2, dict(n=(7, 6, 1), B=3, specular=(1, 3), masked=True, source=True, two_regions=True)),
    ("2d_slab", 2, dict(n=(14, 5, 1), B=2, n_polar=4, n_az=8, specular=(2, 3))),
    ("3d_mask", 3, dict(n=(4, 4, 3), B=2, specular=(2, 5), diffuse=(4,), masked=True, source=True)),
    ("3d_deep", 3, dict(n=(6, 40, 9), B=2, specular=(0, 3, 4), diffuse=(5,), masked=True, source=True)),
]


def rel(a, b, mask):
    return float(np.abs(a - b)[mask].max() / np.abs(b[mask]).max())


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("k", [1, 6])
def test_specular_fp64_fixed_iterations(bte, name, dim, kw, k):
    p = bi.tiny(dim, **kw)
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    q = np.zeros((p.n_cells, 3))
    e = np.zeros((p.n_cells, p.B, p.D))
    rc, st = plan.solve(T, q_out=q, e_out=e, precision=bte.BTE_FP64, tol=0.0, max_iter=k)
    # 1D/2D: the general kernel; 3D: whichever of it and the plane pipeline
    # the autotuner found faster
    assert st["tile_kind"] in ((1,) if dim < 3 else (1, 3)) and st["iterations"] == k
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-12
    assert np.abs(e - ref["e"]).max() < 1e-12 * np.abs(ref["e"]).max()
    assert np.abs(q - ref["q"]).max() < 1e-10 * np.abs(ref["q"]).max() + 1e-300
    np.testing.assert_allclose(plan.eps_history(k), ref["eps"], rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("name,dim,kw", CASES, ids=[c[0] for c in CASES])
def test_specular_fp32_fixed_iterations(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    k = 10
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k)
    act = p.mask > 0
    assert rel(T, ref["T"], act) < 1e-5


@pytest.mark.parametrize("name,dim,kw", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_specular_converged_matches_direct_solve(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-14, max_iter=200000)
    assert st["converged"] == 1
    assert rel(T, ref["T"], p.mask > 0) < 1e-12


@pytest.mark.parametrize("name,dim,kw", [CASES[1], CASES[3]], ids=[CASES[1][0], CASES[3][0]])
def test_specular_adjoint_matches_oracle_and_fd(bte, name, dim, kw):
    p = bi.tiny(dim, **kw)
    ref = dense.solve(p)
    rng = np.random.default_rng(5)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(5, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    fd = dense.fd_gradients(p, probes, T_obs)
    plan = bte.Plan(p)
    for prec, tol_or in ((bte.BTE_FP64, 1e-8), (bte.BTE_FP32, None)):
        T = np.zeros(p.n_cells)
        plan.solve(T, precision=prec, tol=1e-15 if prec == bte.BTE_FP64 else 1e-9, max_iter=200000)
        g = np.zeros(p.n_cells)
        np.add.at(g, probes, T[probes] - T_obs)
        rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=1e-15 if prec == bte.BTE_FP64 else 1e-9,
                                                max_iter=200000)
        if tol_or is not None:
            r = oracle.solve(p, max_iter=100000, tol=1e-15)
            a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
            np.testing.assert_allclose(g_tau, a["g_tau"], rtol=tol_or)
            np.testing.assert_allclose(g_Tw, a["g_Tw"], rtol=tol_or, atol=1e-12 * np.abs(a["g_Tw"]).max())
            assert g_Q == pytest.approx(a["g_Q"], rel=tol_or)
        np.testing.assert_allclose(g_tau, fd["g_tau"], rtol=1e-3)
        np.testing.assert_allclose(g_Tw, fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
        assert g_Q == pytest.approx(fd["g_Q"], rel=1e-3)


def test_specular_side_walls_give_the_1d_slab(bte):
    """Isothermal x walls, specular y walls: every row equals the 1D slab
    with the same mu nodes (the oracle's pin, here on the GPU in FP64)."""
    p = bi.tiny(2, n=(14, 5, 1), B=2, n_polar=4, n_az=8, specular=(2, 3))
    q = bi.tiny(1, n=(14, 1, 1), B=2, n_polar=2)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    plan.solve(T, precision=bte.BTE_FP64, tol=1e-15, max_iter=200000)
    r1 = oracle.solve(q, max_iter=100000, tol=1e-15)
    T2 = T.reshape(-1, 14)
    assert np.abs(T2 - r1["T"][None, :]).max() < 1e-11 * np.ptp(r1["T"])


def test_specular_other_kernels_refused(bte):
    """In 1D and 2D only the general kernel carries specular faces: asking
    for a row kernel is refused; a direction set without mirrors is
    refused."""
    p = bi.tiny(2, n=(5, 4, 1), B=2, specular=(2,))
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, tol=0.0, max_iter=2, tile_kind=3, check=False)
    assert rc == -1
    s = p.s.copy()
    s[0] = s[0] * np.array([1.0, 0.9, 1.0])
    s[0] /= np.linalg.norm(s[0])
    with pytest.raises(bte.BTEError) as err:
        bte.Plan(p.copy(s=s))
    assert err.value.code == -1


# ---------------------------------------------------------------------------
# the 3D plane pipeline (tile_kind 3) with specular faces: on the plane axis,
# the row axis and x, forward and adjoint, against the oracle
# ---------------------------------------------------------------------------

def pipe_heights(n, lane_axis):
    """Warps along the plane axis the plane pipeline accepts (at most 16
    warps, ceil(rows / 32) of them along the rows; several passes need two
    warps along the planes and nx >= 4 H + 2)."""
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


PCASES = [
    # specular y faces (the rows along y: the lanes' axis; along z: the
    # plane axis), a diffuse top, masked, two regions, several passes
    ("pipe_y", dict(n=(22, 37, 13), B=2, specular=(2, 3), diffuse=(5,), masked=True, source=True,
                    two_regions=True, n_polar=4, n_az=8)),
    # specular x- and both z faces, a diffuse y+ face
    ("pipe_xz", dict(n=(20, 9, 30), B=2, specular=(0, 4, 5), diffuse=(3,), source=True, n_polar=2, n_az=8)),
]


@pytest.mark.parametrize("name,kw", PCASES, ids=[c[0] for c in PCASES])
@pytest.mark.parametrize("axis", [1, 2], ids=["rows_y", "rows_z"])
@pytest.mark.parametrize("k", [1, 7])
def test_specular_plane_pipeline_fp64(bte, name, kw, axis, k):
    p = bi.tiny(3, **kw)
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    plan = bte.Plan(p)
    hs = pipe_heights(p.n, axis)
    assert hs
    for dw in (2, 4):
        for H in sorted({hs[0], hs[-1]}):
            T = np.zeros(p.n_cells)
            q = np.zeros((p.n_cells, 3))
            e = np.zeros((p.n_cells, p.B, p.D))
            rc, st = plan.solve(T, q_out=q, e_out=e, precision=bte.BTE_FP64, tol=0.0, max_iter=k, tile_kind=3,
                                dirs_per_lane=dw, warps_z=H, lane_axis=axis)
            assert st["tile_kind"] == 3 and st["warps_z"] == H and st["lane_axis"] == axis
            assert st["iterations"] == k
            assert rel(T, ref["T"], act) < 1e-12
            assert np.abs(e - ref["e"]).max() < 1e-12 * np.abs(ref["e"]).max()
            assert np.abs(q - ref["q"]).max() < 1e-10 * np.abs(ref["q"]).max()
            np.testing.assert_allclose(plan.eps_history(k), ref["eps"], rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("name,kw", PCASES, ids=[c[0] for c in PCASES])
@pytest.mark.parametrize("dw", [2, 4, 8])
def test_specular_plane_pipeline_fp32(bte, name, kw, dw):
    p = bi.tiny(3, **kw)
    k = 12
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    plan = bte.Plan(p)
    for axis in (1, 2):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=bte.BTE_FP32, tol=0.0, max_iter=k, tile_kind=3, dirs_per_lane=dw,
                            lane_axis=axis)
        assert st["tile_kind"] == 3 and st["dirs_per_lane"] == dw
        assert rel(T, ref["T"], act) < 1e-5


def test_specular_plane_pipeline_converged(bte):
    """Converged in FP64 on the plane pipeline: the oracle's fixed point,
    and the same iteration count."""
    p = bi.tiny(3, **PCASES[0][1])
    ref = oracle.solve(p, max_iter=100000, tol=1e-13)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-13, max_iter=100000, tile_kind=3, dirs_per_lane=4)
    assert st["converged"] == 1 and abs(st["iterations"] - ref["iters"]) <= 1
    assert rel(T, ref["T"], p.mask > 0) < 1e-12


def test_specular_plane_pipeline_adjoint_fd(bte):
    """A small single-pass case (one direction per octant, so every subset
    is partly empty): FP64 and FP32 adjoint gradients through the plane
    pipeline against central finite differences and the oracle's adjoint."""
    p = bi.tiny(3, n=(6, 5, 4), B=2, specular=(2, 5), diffuse=(3,), masked=True, source=True)
    ref = dense.solve(p)
    rng = np.random.default_rng(8)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=min(5, act.size), replace=False))
    T_obs = ref["T"][probes] + rng.normal(0.0, 0.5, probes.size)
    fd = dense.fd_gradients(p, probes, T_obs)
    plan = bte.Plan(p)
    for prec, tol in ((bte.BTE_FP64, 1e-15), (bte.BTE_FP32, 1e-9)):
        T = np.zeros(p.n_cells)
        rc, st = plan.solve(T, precision=prec, tol=tol, max_iter=200000, tile_kind=3, dirs_per_lane=2)
        assert st["tile_kind"] == 3
        g = np.zeros(p.n_cells)
        np.add.at(g, probes, T[probes] - T_obs)
        rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=tol, max_iter=200000)
        if prec == bte.BTE_FP64:
            r = oracle.solve(p, max_iter=100000, tol=1e-15)
            a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
            np.testing.assert_allclose(g_tau, a["g_tau"], rtol=1e-8)
            np.testing.assert_allclose(g_Tw, a["g_Tw"], rtol=1e-8, atol=1e-12 * np.abs(a["g_Tw"]).max())
            assert g_Q == pytest.approx(a["g_Q"], rel=1e-8)
        np.testing.assert_allclose(g_tau, fd["g_tau"], rtol=1e-3)
        np.testing.assert_allclose(g_Tw, fd["g_Tw"], rtol=1e-3, atol=1e-3 * np.abs(fd["g_Tw"]).max())
        assert g_Q == pytest.approx(fd["g_Q"], rel=1e-3)


@pytest.mark.parametrize("name,kw", PCASES, ids=[c[0] for c in PCASES])
def test_specular_plane_pipeline_adjoint_oracle(bte, name, kw):
    """Several passes: FP64 adjoint gradients of the plane pipeline (its
    final gradient form) against the oracle's adjoint, then the length
    gradient, whose final pass runs on the general kernel from the specular
    arrays the plane pipeline's adjoint iterations left (mu = w nu there)."""
    p = bi.tiny(3, **kw)
    r = oracle.solve(p, max_iter=100000, tol=1e-15)
    rng = np.random.default_rng(9)
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=8, replace=False))
    g = np.zeros(p.n_cells)
    g[probes] = r["T"][probes] - r["T"][probes].mean()
    a = oracle.adjoint(p, r["e"], r["T"], g, tol=1e-15)
    plan = bte.Plan(p)
    T = np.zeros(p.n_cells)
    rc, st = plan.solve(T, precision=bte.BTE_FP64, tol=1e-15, max_iter=200000, tile_kind=3, dirs_per_lane=4)
    assert st["tile_kind"] == 3
    rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=1e-15, max_iter=200000)
    np.testing.assert_allclose(g_tau, a["g_tau"], rtol=1e-8)
    np.testing.assert_allclose(g_Tw, a["g_Tw"], rtol=1e-8, atol=1e-12 * np.abs(a["g_Tw"]).max())
    assert g_Q == pytest.approx(a["g_Q"], rel=1e-8)
    rc, g_tau2, g_Tw2, g_Q2, sa2, g_L = plan.adjoint(g, tol=1e-15, max_iter=200000, lengths=True)
    np.testing.assert_allclose(g_L, a["g_L"], rtol=1e-8, atol=1e-12 * np.abs(a["g_L"]).max())
    np.testing.assert_allclose(g_tau2, a["g_tau"], rtol=1e-8)
