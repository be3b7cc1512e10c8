"""GPU parity with the caller's directions in an arbitrary order.

The library sorts the directions by octant internally and must return e in
the caller's order; every other input set of the test-suite lists the
directions octant by octant already, so here the direction set (s and w
together) is shuffled with a fixed seed before it reaches either side.  The
oracle takes any order (each direction is an independent sweep); T, q and e
of libbte must match it on the same shuffled input, with e read back both
into host memory (the host-side permutation) and into device memory (the
permutation kernel).
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


def shuffled(p, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(p.D)
    # the natural order of the product set mixes the octants
    return p.copy(s=p.s[perm].copy(), w=p.w[perm].copy())


CASES = [
    ("2d_square", lambda: bi.square_2d(n=20, L=0.3e-6, n_polar=4, n_az=8), (1, 3)),
    ("2d_mask", lambda: bi.tiny(2, n=(9, 7, 1), B=3, n_polar=4, n_az=8, masked=True, diffuse=(2, 3),
                                source=True, two_regions=True), (1,)),
    ("3d_mask", lambda: bi.tiny(3, n=(12, 9, 8), B=2, n_polar=4, n_az=8, masked=True, diffuse=(0, 3, 5),
                                source=True, two_regions=True), (1, 3)),
]


@pytest.mark.parametrize("name,make,kinds", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shuffled_direction_order(bte, name, make, kinds, prec):
    p = shuffled(make(), seed=17)
    signs = (p.s[:, :p.dim] < 0).astype(int) @ (1 << np.arange(p.dim))
    assert np.any(np.diff(signs) < 0), "the shuffled set must not be octant-sorted"
    k = 6
    ref = oracle.solve(p, max_iter=k, tol=0.0)
    act = p.mask > 0
    fp64 = prec == "fp64"
    tol_T, tol_e, tol_q = (1e-12, 1e-12, 1e-10) if fp64 else (1e-5, 2e-5, 1e-3)
    dt_np = np.float64 if fp64 else np.float32
    dt_t = torch.float64 if fp64 else torch.float32
    for kind in kinds:
        plan = bte.Plan(p)
        # e into host memory
        T = np.zeros(p.n_cells)
        q = np.zeros((p.n_cells, 3))
        e = np.zeros((p.n_cells, p.B, p.D), dtype=dt_np)
        rc, st = plan.solve(T, q_out=q, e_out=e, precision=bte.BTE_FP64 if fp64 else bte.BTE_FP32,
                            tol=0.0, max_iter=k, tile_kind=kind)
        assert st["tile_kind"] == kind and st["iterations"] == k
        escale = np.abs(ref["e"]).max()
        assert np.abs(T - ref["T"])[act].max() < tol_T * np.abs(ref["T"][act]).max()
        assert np.abs(e - ref["e"]).max() < tol_e * escale
        qs = np.abs(ref["q"]).max()
        assert np.abs(q - ref["q"]).max() < tol_q * qs
        # e into device memory
        Td = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
        ed = torch.zeros((p.n_cells, p.B, p.D), dtype=dt_t, device="cuda")
        rc, st = plan.solve(Td, e_out=ed, precision=bte.BTE_FP64 if fp64 else bte.BTE_FP32,
                            tol=0.0, max_iter=k, tile_kind=kind)
        assert np.abs(ed.cpu().numpy() - ref["e"]).max() < tol_e * escale
        np.testing.assert_array_equal(Td.cpu().numpy(), T)
