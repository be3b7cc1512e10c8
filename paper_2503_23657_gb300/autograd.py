"""Differentiable steady solve: ``T = bte_temperature(plan, tau, T_wall, Q_amp[, lengths])``.

Forward runs ``bte_solve``; backward runs ``bte_adjoint`` -- the transposed,
downwind-ordered sweep iterated to the fixed point of the adjoint source
iteration -- and returns dJ/dtau_b, dJ/dT_wall (isothermal faces),
dJ/dQ_amp and, when the domain lengths are an input, dJ/dL_a (the paper's
inverse workflow differentiates its implicit solve with a discrete adjoint;
Forward and inverse modelling workflow; its 1D inverse case recovers a film
thickness).  A plan's geometry is fixed when it is created, so a forward
with other lengths than the plan's creates a plan for them.

The plan keeps the state of its last solve only.  If another solve ran on
the same plan between this forward and its backward, backward first repeats
the forward solve from the saved parameters (recomputation instead of
storing e: T and the diffuse inflow determine e).
"""
from __future__ import annotations

import torch

from .binding import BTE_FP32


class _BTESolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, T_wall, Q_amp, lengths, plan, opts):
        if lengths is not None:
            L = tuple(float(x) for x in lengths.detach().double().cpu().numpy())
            if L != tuple(float(x) for x in plan.problem.length):
                from .binding import Plan
                plan = Plan(plan.problem.copy(length=L))
        p = plan.problem
        T = torch.empty(p.n_cells, dtype=torch.float64, device="cuda")
        args = dict(opts)
        adj_tol = args.pop("adj_tol", 1e-10)
        args.update(tau=tau.detach().double().cpu().numpy(),
                    T_wall=T_wall.detach().double().cpu().numpy(),
                    Q_amp=float(Q_amp.detach().cpu()),
                    stream=torch.cuda.current_stream().cuda_stream)
        plan.solve(T, **args)
        plan._solve_id = getattr(plan, "_solve_id", 0) + 1
        ctx.plan = plan
        ctx.solve_id = plan._solve_id
        ctx.args = args
        ctx.adj_tol = adj_tol
        ctx.lengths = lengths is not None
        return T

    @staticmethod
    def backward(ctx, gT):
        plan = ctx.plan
        if getattr(plan, "_solve_id", None) != ctx.solve_id:
            tmp = torch.empty(plan.problem.n_cells, dtype=torch.float64, device="cuda")
            plan.solve(tmp, **ctx.args)
            plan._solve_id += 1
        torch.cuda.current_stream().synchronize()
        g = gT.detach().double().contiguous()
        g_L = None
        if ctx.lengths:
            rc, g_tau, g_Tw, g_Q, st, gl = plan.adjoint(g, tol=ctx.adj_tol, lengths=True)
            g_L = torch.from_numpy(gl)
        else:
            rc, g_tau, g_Tw, g_Q, st = plan.adjoint(g, tol=ctx.adj_tol)
        return (torch.from_numpy(g_tau), torch.from_numpy(g_Tw),
                torch.tensor(g_Q, dtype=torch.float64), g_L, None, None)


def bte_temperature(plan, tau, T_wall, Q_amp, lengths=None, precision=BTE_FP32, tol=1e-6, max_iter=100000,
                    adj_tol=1e-10, **kw):
    """Lattice temperature [N] (CUDA, float64) as a differentiable function of
    the band relaxation times ``tau`` [B], wall temperatures ``T_wall`` [6],
    source amplitude ``Q_amp`` and, if given, the domain lengths ``lengths``
    [3] in metres (CPU float64 tensors)."""
    opts = dict(precision=precision, tol=tol, max_iter=max_iter, adj_tol=adj_tol, **kw)
    return _BTESolve.apply(tau, T_wall, torch.as_tensor(Q_amp, dtype=torch.float64), lengths, plan, opts)


def probe_loss(T, probes, T_obs):
    """J = 1/2 sum_p (T_p - T_obs,p)^2 over probe cells."""
    d = T[probes] - T_obs
    return 0.5 * (d * d).sum()


__all__ = ["bte_temperature", "probe_loss"]
