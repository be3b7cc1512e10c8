// Convergence bookkeeping of a source iteration (solution procedure of the
// paper: eps_T = sqrt(mean (T_new - T_old)^2) / max T_new, stop when
// eps_T < tol), shared by the update kernel, the row-pipeline sweep (which
// finalizes the previous iteration in its prologue) and the finalize kernels.
#pragma once

#include <math.h>

#include "bte_internal.cuh"

namespace bte {

// Sum and max over one warp (fixed shuffle tree: deterministic).
__device__ __forceinline__ void fin_warp_reduce(double &a, double &m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
}

// One full warp: reduce the block partials in a fixed order (every lane a
// strided slice, loads issued sixteen at a time, then the shuffle tree);
// every lane returns the same eps_T, max and sum of squares.
__device__ __forceinline__ void fin_reduce(const FinalizeParams &F, double &eps, double &tmx, double &tss) {
    const int lane = threadIdx.x & 31;
    double s = 0.0, m = -INFINITY;
    for (int i0 = lane; i0 < F.nblocks; i0 += 32 * 16) {
        double2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = i0 + 32 * q;
            v[q] = i < F.nblocks ? __ldcg(reinterpret_cast<const double2 *>(F.blockpart) + i)
                                 : make_double2(0.0, -INFINITY);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            s += v[q].x;
            m = fmax(m, v[q].y);
        }
    }
    fin_warp_reduce(s, m);
    tss = __shfl_sync(0xffffffffu, s, 0);
    tmx = __shfl_sync(0xffffffffu, m, 0);
    eps = (tmx > 0.0) ? sqrt(tss / (double)F.n_active) / tmx : 0.0;
}

__device__ __forceinline__ bool fin_stop(const FinalizeParams &F, double eps) {
    return !isfinite(eps) || (F.tol > 0.0 && eps < F.tol);
}

// One thread: record the finalized iteration and its stop decision.
__device__ __forceinline__ void fin_record(const FinalizeParams &F, double eps, double tmx, double tss) {
    const int it = *F.iter;
    if (F.eps_hist && it < F.max_hist) F.eps_hist[it] = eps;
    F.last[0] = eps;
    F.last[1] = tmx;
    F.last[2] = tss;
    *F.iter = it + 1;
    // a NaN residual marks status 1 unless a sweep already recorded an
    // expired wait (2), which stays the reported cause
    if (!isfinite(eps)) atomicCAS(F.status, 0, 1);
    // an instance whose status is set (a non-finite residual, or a sweep's
    // bounded wait that expired) stops too, so a batched solve does not keep
    // iterating it until max_iter
    if (fin_stop(F, eps) || *((volatile const int *)F.status) != 0) {
        *F.done = 1;
        if (F.batch_done) atomicAdd(F.batch_done, 1);
    }
    *F.pending = 0;
}

}  // namespace bte
