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
