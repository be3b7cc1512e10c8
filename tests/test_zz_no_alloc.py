"""The allocation-free entry point bte_eps_T_noalloc, for callers that cannot
call cudaMalloc where they need the convergence measure (e.g. a host whose
device memory belongs to its own pool, or code running while another thread
captures a CUDA graph).  Its eps_T must equal the one bte_solve reports for
the same pair of iterates, on two calls in a row (the scratch array is shared
and reused).  Collected last on purpose."""
import numpy as np
import pytest

import bte_inputs as bi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_eps_matches_solver_history():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_23657_gb300 as m
    from paper_2503_23657_gb300 import binding

    p = bi.tiny(2, n=(9, 7, 1), B=2, masked=True, diffuse=(2, 3), source=True)
    plan = m.Plan(p)
    N = p.n_cells
    mask = torch.as_tensor(p.mask, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    iterates = {}
    for k in (4, 5, 6):
        T = torch.zeros(N, dtype=torch.float64, device="cuda")
        plan.solve(T, precision=m.BTE_FP64, tol=0.0, max_iter=k, stream=stream)
        iterates[k] = (T, plan.eps_history(k))
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for k in (5, 6):  # two calls in a row on the same scratch array
        binding.eps_T_noalloc(iterates[k - 1][0], iterates[k][0], out, mask=mask, stream=stream)
        torch.cuda.synchronize()
        eps, tmax, count = out.cpu().numpy()
        ref = iterates[k][1][k - 1]
        assert eps == pytest.approx(ref, rel=1e-12)
        assert tmax == pytest.approx(float(iterates[k][0][mask > 0].max()), rel=1e-15)
        assert count == float(np.count_nonzero(p.mask))


def test_noalloc_rejects_out_of_range_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_23657_gb300 import binding
    lib = binding.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = lib.bte_eps_T_noalloc(x.data_ptr(), x.data_ptr(), None, (1 << 24) + 1, out.data_ptr(), None)
    assert rc == binding.BTE_EINVAL
    assert b"BTE_NOALLOC_MAX_CELLS" in lib.bte_last_error(None)


def _torch_eps(T_old, T_new, mask):
    sel = torch.ones_like(T_new, dtype=torch.bool) if mask is None else mask > 0
    d = (T_old - T_new)[sel]
    return float(torch.sqrt(torch.mean(d * d)) / T_new[sel].max()), float(T_new[sel].max()), int(sel.sum())


@pytest.mark.parametrize("with_mask", [False, True])
def test_noalloc_large_grid_stride_and_block_combine(with_mask):
    """3e6 cells: more than the 1024 blocks x 256 threads of one pass, so the
    grid-stride loop and the combine of all 1024 block partials run; with and
    without a mask (NULL mask = every cell solid).  Checked against a plain
    torch reduction, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_23657_gb300 import binding

    g = torch.Generator(device="cuda").manual_seed(11)
    N = 3_000_000
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        T_old = 300.0 + torch.rand(N, dtype=torch.float64, device="cuda", generator=g)
        T_new = T_old + 1e-3 * torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
        mask = ((torch.rand(N, device="cuda", generator=g) < 0.7).to(torch.uint8) * (1 + call)
                if with_mask else None)
        binding.eps_T_noalloc(T_old, T_new, out, mask=mask)
        torch.cuda.synchronize()
        eps, tmax, count = out.cpu().numpy()
        ref_eps, ref_max, ref_count = _torch_eps(T_old, T_new, mask)
        assert eps == pytest.approx(ref_eps, rel=1e-12)
        assert tmax == ref_max
        assert count == ref_count


def test_noalloc_nan_temperature_gives_nan():
    """A NaN temperature makes eps_T NaN (the solver reads that as a numeric
    failure), also when the NaN cell would not be the maximum."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_23657_gb300 import binding

    N = 5000
    T_old = torch.full((N,), 300.0, dtype=torch.float64, device="cuda")
    T_new = T_old.clone()
    T_new[1234] = float("nan")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    binding.eps_T_noalloc(T_old, T_new, out)
    torch.cuda.synchronize()
    assert np.isnan(out[0].item())
    # and the next call on the shared scratch array is clean again
    T_new[1234] = 301.0
    binding.eps_T_noalloc(T_old, T_new, out)
    torch.cuda.synchronize()
    ref_eps, _, _ = _torch_eps(T_old, T_new, None)
    assert out[0].item() == pytest.approx(ref_eps, rel=1e-12)


def test_noalloc_binding_rejects_mismatched_buffers():
    """The binding refuses buffers of the wrong length, type or device before
    anything reaches the library."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_23657_gb300 import binding

    T = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        binding.eps_T_noalloc(T[:63], T, out)
    with pytest.raises(ValueError):
        binding.eps_T_noalloc(T, T, out, mask=torch.ones(63, dtype=torch.uint8, device="cuda"))
    with pytest.raises(TypeError):
        binding.eps_T_noalloc(T.float(), T, out)
    with pytest.raises(TypeError):
        binding.eps_T_noalloc(T.cpu(), T, out)
