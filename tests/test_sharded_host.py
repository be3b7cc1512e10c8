"""Host logic of the band-sharded solve (paper_2503_23657_gb300/sharded.py),
on CPU ranks.

The band partition is checked directly.  The iteration loop and its one FP64
allreduce per iteration run on world_size 2 gloo ranks (spawned processes)
against a toy plan with the structure of the method's outer iteration: each
band's contribution to the per-cell sums depends on T and on that band's own
lagged boundary state, the temperature is T_ref + (sum over bands) / K.  Two
ranks must reproduce the one-rank iteration: the same iteration count on
every rank and the same T up to the order of the additions."""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2503_23657_gb300.sharded import ShardedSolve, band_range


@pytest.mark.parametrize("B", [1, 2, 3, 7, 15, 16])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 20])
def test_band_range_partitions_the_bands(B, world):
    ranges = [band_range(B, r, world) for r in range(world)]
    covered = [b for b0, b1 in ranges for b in range(b0, b1)]
    assert covered == list(range(B))                     # disjoint, ordered, complete
    sizes = [b1 - b0 for b0, b1 in ranges]
    assert max(sizes) - min(sizes) <= 1                  # balanced


class ToyProblem:
    def __init__(self, N=40, B=7):
        self.n_cells, self.B = N, B


class ToyPlan:
    """A contraction with the outer iteration's structure (CPU, FP64)."""

    def __init__(self, seed=3, N=40, B=7):
        rng = np.random.default_rng(seed)
        self.problem = ToyProblem(N, B)
        self.A = rng.uniform(0.0, 1.0, (B, N, N))
        self.A *= 0.9 / (B * self.A.sum(axis=2, keepdims=True))   # row sums 0.9 / B
        self.c = rng.uniform(0.0, 2.0, (B, N))
        self.d = rng.uniform(0.0, 0.005, B)   # keeps the iteration a contraction
        self.K = 1.0

    def shard_begin(self, T_init_uniform=300.0):
        N, B = self.problem.n_cells, self.problem.B
        self.T = np.full(N, T_init_uniform)
        self.y = np.full(B, T_init_uniform)      # each band's lagged boundary state

    def shard_sweep(self, b0, b1, W):
        w = np.zeros(self.problem.n_cells)
        y_next = self.y.copy()
        for b in range(b0, b1):
            w += self.A[b] @ self.T + self.c[b] + self.d[b] * self.y[b]
            y_next[b] = float(np.mean(self.A[b] @ self.T)) * self.problem.B
        self.y = y_next                            # only this rank's bands change
        W.copy_(torch.from_numpy(w))

    def shard_apply(self, W, T_out=None):
        T_new = W.numpy() / self.K
        eps = float(np.sqrt(np.mean((T_new - self.T) ** 2)) / np.max(T_new))
        self.T = T_new
        if T_out is not None:
            T_out[:] = T_new
        return eps


def _rank_main(rank, world, init_file, out_dir, tol):
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank, world_size=world)
    try:
        plan = ToyPlan()
        T = np.zeros(plan.problem.n_cells)
        it, eps, conv = ShardedSolve(plan, device="cpu").solve(T, tol=tol, max_iter=10000, T_init_uniform=300.0)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), T=T, it=it, eps=eps, conv=conv)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_rank():
    tol = 1e-12
    plan = ToyPlan()
    T1 = np.zeros(plan.problem.n_cells)
    it1, eps1, conv1 = ShardedSolve(plan, device="cpu").solve(T1, tol=tol, max_iter=10000, T_init_uniform=300.0)
    assert conv1 and it1 > 5
    with tempfile.TemporaryDirectory() as d:
        init_file = os.path.join(d, "init")
        mp.start_processes(_rank_main, args=(2, init_file, d, tol), nprocs=2, join=True, start_method="spawn")
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(2)]
    for r in res:
        assert bool(r["conv"]) and int(r["it"]) == it1
        assert np.abs(r["T"] - T1).max() < 1e-12 * np.abs(T1).max()
    np.testing.assert_array_equal(res[0]["T"], res[1]["T"])   # every rank forms the same T


def test_a_rank_without_bands_still_takes_part():
    """More ranks than bands: the extra ranks contribute zeros."""
    plan = ToyPlan(B=1)
    T1 = np.zeros(plan.problem.n_cells)
    it1, _, _ = ShardedSolve(plan, device="cpu").solve(T1, tol=1e-12, max_iter=10000)
    assert band_range(1, 1, 2) == (1, 1)
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main_b1, args=(2, os.path.join(d, "init"), d), nprocs=2, join=True,
                           start_method="spawn")
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(2)]
    for r in res:
        assert int(r["it"]) == it1 and np.abs(r["T"] - T1).max() < 1e-12 * np.abs(T1).max()


def _rank_main_b1(rank, world, init_file, out_dir):
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank, world_size=world)
    try:
        plan = ToyPlan(B=1)
        T = np.zeros(plan.problem.n_cells)
        it, eps, conv = ShardedSolve(plan, device="cpu").solve(T, tol=1e-12, max_iter=10000)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), T=T, it=it, eps=eps, conv=conv)
    finally:
        dist.destroy_process_group()
