"""Band-sharded solve of one instance over the ranks of a process group.

The outer iteration of the paper's solution procedure (Methods, steps 1-4)
sweeps every (band, direction) from the current T, then updates T from the
band-weighted direction sums of all bands (Eq. updatee0_t).  Sweeps of
different bands are independent given T, and a band's diffuse inflow depends
only on its own face sums, so the bands are split over the ranks: rank r
sweeps bands [b0_r, b1_r) (``bte_shard_sweep``), the ranks add their
per-cell weighted sums W_r with one FP64 allreduce of N values per iteration,
and every rank forms the same T from the sum (``bte_shard_apply``), the same
eps_T, and so stops at the same iteration.  Every step of the iteration runs
in libbte's kernels; this module only partitions the bands, calls the
collective and runs the loop.

A plan is any object with ``shard_begin``, ``shard_sweep``, ``shard_apply``
and ``problem`` (``binding.Plan`` on a GPU).
"""
from __future__ import annotations

import torch


def band_range(B: int, rank: int, world: int):
    """Contiguous bands [b0, b1) of rank ``rank``: the B bands split as evenly
    as possible (the first B mod world ranks take one more); empty for ranks
    beyond B."""
    if not (0 <= rank < world) or B < 0:
        raise ValueError("need 0 <= rank < world and B >= 0")
    q, r = divmod(B, world)
    b0 = rank * q + min(rank, r)
    return b0, b0 + q + (1 if rank < r else 0)


class ShardedSolve:
    """Iterate a plan's instance with its bands split over a process group
    (``torch.distributed``; without an initialised group, one rank holds
    every band).  ``device`` is where W lives for the collective: ``cuda``
    with NCCL, ``cpu`` with gloo."""

    def __init__(self, plan, group=None, device=None):
        import torch.distributed as dist
        self.plan = plan
        self.group = group
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.rank = self.dist.get_rank(group) if self.dist else 0
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.device = device or ("cuda" if torch.cuda.is_available() else "cpu")
        self.bands = band_range(plan.problem.B, self.rank, self.world)

    def solve(self, T_out=None, tol=1e-6, max_iter=100000, **begin):
        """Run to eps_T < tol (tol <= 0: exactly max_iter iterations).  T_out
        [N] receives the last T (on every rank).  Returns (iterations,
        eps_T, converged)."""
        p = self.plan.problem
        self.plan.shard_begin(**begin)
        b0, b1 = self.bands
        W = torch.zeros(p.n_cells, dtype=torch.float64, device=self.device)
        eps = float("nan")
        for it in range(1, max_iter + 1):
            if b1 > b0:
                self.plan.shard_sweep(b0, b1, W)
            else:
                W.zero_()
            if self.world > 1:
                self.dist.all_reduce(W, op=self.dist.ReduceOp.SUM, group=self.group)
            eps = self.plan.shard_apply(W, T_out)
            if tol > 0.0 and eps < tol:
                return it, eps, True
        return max_iter, eps, False


__all__ = ["band_range", "ShardedSolve"]
