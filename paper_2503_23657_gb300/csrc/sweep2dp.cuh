// Row-pipeline wavefront sweep for unmasked 1D/2D grids with one region.
//
// Same discrete equations as sweep.cuh (Eq. fvm-1 with step upwind faces,
// the lower-triangular matrix A of Eq. A_matrix), organised so that many
// warps share the work of one (band, direction) wavefront:
//
//   * one CTA per (direction chunk, band).  A chunk is G groups of DW
//     directions of one quadrant (one traversal order); group g owns DW
//     directions and NRB = ceil(ny / 32) warps (G * NRB <= 16), warp R of the group holding
//     rows 32 R .. 32 R + 31 (one row per lane);
//   * lane l of a warp updates column i = tau - l of its row at local step
//     tau: the x-upwind value is the lane's own register from the previous
//     step, the y-upwind value comes from lane l - 1 by one warp shuffle;
//     lane 0 takes it from the warp below (row 32 R - 1), which wrote it to
//     shared memory when it finished that column; for the first warp that
//     row is the upwind y wall, laid out the same way, and the last warp
//     writes the top row for the downwind y-wall sums.  The step has no
//     branches (predicated loads and stores), so the K unrolled steps of a
//     chunk schedule as one block;
//   * the warps of a group form a pipeline: after every chunk of K steps
//     warp R publishes how many columns of its top row are final (a release
//     store to a shared-memory counter); warp R + 1 waits (acquire loads,
//     bounded) until the columns of its next chunk are there.  Warp R never
//     waits on warp R + 1, so the pipeline cannot deadlock; warp R + 1 lags
//     by about K + 31 steps;
//   * forward and adjoint run the same recurrence.  The adjoint unknown
//     mu_d of the transposed system (Eq. adjoint) scaled by 1 / w_d obeys the
//     forward recurrence with the adjoint source and boundary values, so the
//     kernel carries nu_d = mu_d / w_d and forms sum_d mu_d = sum_d w_d nu_d
//     like the forward weighted sum; only the wall face-sum weights differ
//     (forward w_d |s_d.n|, adjoint a_d w_d);
//   * the per-cell source (T - T_ref or Theta, and the source profile) is
//     brought into shared memory once per CTA by a TMA bulk copy
//     (cp.async.bulk on an mbarrier, bounded wait); every group writes its
//     own partial set of per-cell weighted sums, so results do not depend
//     on scheduling; wall face sums are combined over groups in a fixed
//     order;
//   * the lanes of a step sit on a diagonal, so storing their sums directly
//     would touch 32 sectors per warp store.  Each warp parks them for 32
//     steps in a shared-memory tile [row][33] (conflict-free) and then
//     writes row by row: 32 steps of one row are 32 consecutive cells.
#pragma once

#include <stdint.h>

#include "bte_internal.cuh"
#include "finalize.cuh"
#include "tma.cuh"

namespace bte {

// Wait until *prog >= need, at most `limit` polls (with a short sleep; the
// plan's limit, kPipeSpinLimit by default).  False if the CTA has aborted or
// the wait ran out (the caller then records the failure and carries on
// without waiting: the values it reads are then wrong, every access stays in
// bounds, and the solve reports BTE_ETIMEOUT).
__device__ __forceinline__ bool pipe_wait(const int *prog, int need, volatile int *abort_flag, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (ld_acquire_cta(prog) >= need) return true;
        if (*abort_flag) return false;
        __nanosleep(32);
    }
    return false;
}

constexpr int kPipeMaxThreads = 512;

// One CTA's work: direction chunk s of band b of the problem P.
template <typename real, int DW, int K, bool PHI, bool STORE_E, bool STAGE>
__device__ __forceinline__ void sweep2dp_body(const Sweep2DParams<real> &P, const int s, const int b) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_abort;
    __shared__ int s_stop;
    const int nx = P.nx, ny = P.ny;
    const int N = nx * ny;
    const int Npad = (N + 15) & ~15;
    const int G = P.groups;
    const int NRB = (ny + 31) / 32;
    const bool adj = P.adj != 0;
    // STAGE: the per-cell source is copied to shared memory; otherwise every
    // lane reads its own row from global memory one chunk ahead
    real *s_t = reinterpret_cast<real *>(smem_raw);               // [Npad] T - T_ref or Theta (STAGE)
    real *s_phi = s_t + (STAGE ? Npad : 0);                       // [Npad] source profile (STAGE, forward)
    real *s_hand = s_phi + ((STAGE && PHI) ? Npad : 0);           // [G][NRB+1][nx][DW] row values
    real *s_tiles = s_hand + (size_t)G * (NRB + 1) * nx * DW;     // [G*NRB][32][33] transpose tiles
    real *s_fs = s_tiles + (size_t)G * NRB * 32 * 33;             // [G][nx + ny] wall sums
    real *s_wx = s_fs + G * (nx + ny);                            // [ny] upwind x-wall values
    int *s_prog = reinterpret_cast<int *>(s_wx + ny);             // [G][NRB+1] published columns

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nthr = blockDim.x;
    const Subset ch = P.sub[s];
    const bool negx = ch.neg & 1, negy = (ch.neg >> 1) & 1;
    const int up_x = negx ? 1 : 0, up_y = negy ? 3 : 2;
    const int cstep = negx ? -1 : 1;
    const int X0 = negx ? nx - 1 : 0;

    // ---- prologue: TMA bulk copy of the per-cell inputs, wall values ----
    // the next kernel may be launched now (it waits for this grid to finish);
    // everything below reads what the previous kernel wrote
    pdl_launch_dependents();
    pdl_wait();
    // the stop flag may be set while this kernel runs (deferred finalization
    // in CTA (0, 0)): one thread reads it, so every warp of the CTA takes
    // the same decision (a warp that left early would stall the pipeline)
    if (threadIdx.x == 0) {
        s_abort = 0;
        s_stop = (P.done != nullptr && *((volatile const int *)P.done) != 0) ? 1 : 0;
        if (!s_stop) {
            mbar_init(&s_bar, 1);
            mbar_fence_init();
        }
    }
    __syncthreads();
    if (s_stop) return;
    if (STAGE && threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(Npad * sizeof(real));
        mbar_arrive_expect_tx(&s_bar, PHI ? 2 * bytes : bytes);
        bulk_copy_g2s(s_t, P.tsrc, bytes, &s_bar);
        if (PHI) bulk_copy_g2s(s_phi, P.phi, bytes, &s_bar);
    }
    {
        const real *einb = P.ein + (long long)b * P.F;
        for (int y = threadIdx.x; y < ny; y += nthr) {
            const int f = P.wall_face[up_x * P.wall_stride + y];
            s_wx[y] = f >= 0 ? einb[f] : real(0);
        }
        // row -1 of every group: the upwind y-wall value of column i, in
        // traversal order, for each of the group's directions
        for (int q = threadIdx.x; q < G * nx; q += nthr) {
            const int gg = q / nx, i = q - gg * nx;
            const int f = P.wall_face[up_y * P.wall_stride + X0 + cstep * i];
            const real v = f >= 0 ? einb[f] : real(0);
            real *h = s_hand + ((size_t)gg * (NRB + 1) * nx + i) * DW;
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) h[dd] = v;
        }
        for (int q = threadIdx.x; q < G * (ny + nx); q += nthr) s_fs[q] = real(0);
        for (int q = threadIdx.x; q < G * (NRB + 1); q += nthr) s_prog[q] = (q % (NRB + 1) == 0) ? nx : 0;
    }
    const bool ok = STAGE ? mbar_wait_bounded(&s_bar, 0, kWaitPolls) : true;
    __syncthreads();
    if (!ok) {
        // the bulk copy did not complete: report, wait once more for it, stop
        if (threadIdx.x == 0) {
            atomicExch(P.status, 2);
            mbar_wait_bounded(&s_bar, 0, kWaitPolls);
        }
        return;
    }

    // ---- this warp: group g (DW directions), row block R ----
    const int g = warp / NRB;
    const int R = warp - g * NRB;
    const int set = s * G + g;
    const int d0 = ch.d0 + g * DW;
    const int ndir = max(0, min(DW, ch.cnt - g * DW));
    real ax[DW], ay[DW], w[DW], invd[DW];
#pragma unroll
    for (int dd = 0; dd < DW; ++dd) {
        if (dd < ndir) {
            const real *cf = P.coef + ((long long)b * P.D + d0 + dd) * 8;
            ax[dd] = cf[0];
            ay[dd] = cf[1];
            w[dd] = cf[3];
            invd[dd] = P.invdiag[(long long)b * P.D + d0 + dd];
        } else {
            ax[dd] = ay[dd] = w[dd] = invd[dd] = real(0);
        }
    }
    // face-sum weights (used after the sweep): forward w |s_a| (energy
    // leaving), adjoint a_a w (nu = mu / w)
    auto face_weight = [&](int dd, int axis) -> real {
        if (dd >= ndir) return real(0);
        const real *cf = P.coef + ((long long)b * P.D + d0 + dd) * 8;
        return adj ? cf[axis] * cf[3] : cf[4 + axis];
    };
    const real srck = P.srck[b];
    const real qb = PHI ? P.qb[b] : real(0);
    const int j = 32 * R + lane;  // row in traversal order
    const bool in = j < ny;
    const int Y = in ? (negy ? ny - 1 - j : j) : 0;
    const int t_lo = in ? lane : (1 << 29);  // rows beyond the grid are never valid
    const int c_base = X0 + nx * Y - cstep * lane;  // cell at local step t: c_base + cstep * t
    // the lane whose row the next warp (or the downwind y wall) needs
    const int feed_lane = (R + 1 < NRB) ? 31 : ((ny - 1) & 31);
    const bool feeds = lane == feed_lane;
    real *part_b = P.part + ((long long)b * P.Spad + set) * N;
    real *tile = s_tiles + warp * 32 * 33;
    // flush geometry: row r of this warp is grid row Yr = Y0 + r * ystep
    const int Y0 = negy ? ny - 1 - 32 * R : 32 * R;
    const int ystep = negy ? -1 : 1;
    const int rows_here = min(32, ny - 32 * R);
    const real *hand_in = s_hand + ((size_t)(g * (NRB + 1) + R) * nx) * DW;  // row 32 R - 1
    real *hand_out = s_hand + ((size_t)(g * (NRB + 1) + R + 1) * nx) * DW;   // this warp's feed row
    const int *prog_in = s_prog + g * (NRB + 1) + R;
    int *prog_out = s_prog + g * (NRB + 1) + R + 1;
    const long long eoff = (long long)b * P.D + d0;
    const int BD = P.B * P.D;

    // deferred finalization of the previous iteration: CTA (0, 0) records
    // eps_T and the stop decision; its last pipeline warp does it, since that
    // warp waits longest for its first columns anyway.  Nothing in this
    // kernel waits for it: a stop found here ends the solve at the update
    // that follows (which sees the flag), one sweep later.
    if (s == 0 && b == 0 && warp == G * NRB - 1 && P.fin.pending != nullptr &&
        *((volatile const int *)P.fin.pending) != 0) {
        double eps, tmx, tss;
        fin_reduce(P.fin, eps, tmx, tss);
        if (lane == 0) fin_record(P.fin, eps, tmx, tss);
    }
    // before its row enters the grid a lane holds the x-upwind wall value
    real old[DW];
    {
        const real ex = in ? s_wx[Y] : real(0);
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) old[dd] = ex;
    }

    const int n_steps = (nx + 31 + 31) & ~31;  // whole tiles of 32 steps
    // unstaged: the sources of the next chunk, loaded while this one runs
    real pre_t[STAGE ? 1 : K], pre_p[(STAGE || !PHI) ? 1 : K];
    if constexpr (!STAGE) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool v = (unsigned)(k - t_lo) < (unsigned)nx;
            const int c = c_base + cstep * k;
            pre_t[k] = v ? __ldg(P.tsrc + c) : real(0);
            if constexpr (PHI) pre_p[k] = v ? __ldg(P.phi + c) : real(0);
        }
    }
    bool waited_ok = true;
    for (int t0 = 0; t0 < n_steps; t0 += K) {
        real cur_t[STAGE ? 1 : K], cur_p[(STAGE || !PHI) ? 1 : K];
        if constexpr (!STAGE) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                cur_t[k] = pre_t[k];
                if constexpr (PHI) cur_p[k] = pre_p[k];
                const int t = t0 + K + k;
                const bool v = (unsigned)(t - t_lo) < (unsigned)nx;
                const int c = c_base + cstep * t;
                pre_t[k] = v ? __ldg(P.tsrc + c) : real(0);
                if constexpr (PHI) pre_p[k] = v ? __ldg(P.phi + c) : real(0);
            }
        }
        if (waited_ok) {
            // columns [t0, t0 + K) of row 32 R - 1 (row -1: the wall) must be final
            waited_ok = pipe_wait(prog_in, min(t0 + K, nx), &s_abort, P.spin_limit);
            if (!waited_ok) {
                s_abort = 1;
                if (lane == 0) atomicExch(P.status, 2);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = t0 + k;
            const int i = t - t_lo;
            const bool valid = (unsigned)i < (unsigned)nx;
            const int c = c_base + cstep * t;
            real base, srcp = real(0);
            if constexpr (STAGE) {
                base = valid ? s_t[c] : real(0);
                if constexpr (PHI) srcp = valid ? s_phi[c] : real(0);
            } else {
                base = cur_t[k];
                if constexpr (PHI) srcp = cur_p[k];
            }
            base *= srck;
            if (PHI) base = fma(srcp, qb, base);
            const bool take = (lane == 0) && valid;
            real vy[DW];
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                const real up = __shfl_up_sync(0xffffffffu, old[dd], 1);
                const real yin = take ? hand_in[t * DW + dd] : real(0);
                vy[dd] = lane == 0 ? yin : up;
            }
            real acc = real(0);
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                real r0 = fma(ax[dd], old[dd], base);
                r0 = fma(ay[dd], vy[dd], r0);
                const real en = r0 * invd[dd];
                old[dd] = valid ? en : old[dd];
                acc = fma(w[dd], en, acc);
            }
            tile[lane * 33 + (t & 31)] = acc;
            if (feeds && valid) {
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) hand_out[i * DW + dd] = old[dd];
            }
            if (STORE_E && valid) {
                real *ep = P.e + (long long)c * BD + eoff;
#pragma unroll
                for (int dd = 0; dd < DW; ++dd)
                    if (dd < ndir) ep[dd] = adj ? old[dd] * w[dd] : old[dd];
            }
        }
        // publish the columns of the feed row finished so far
        __syncwarp();
        if (feeds) st_release_cta(prog_out, min(max(t0 + K - feed_lane, 0), nx));
        if (((t0 + K) & 31) == 0) {
            // the last 32 steps of row r are 32 consecutive cells of that row:
            // write them row by row (lane q: step tb + q, column tb + q - r)
            const int tb = t0 + K - 32;
            for (int r = 0; r < rows_here; ++r) {
                const int x = tb + lane - r;
                const int Yr = Y0 + r * ystep;
                if ((unsigned)x < (unsigned)nx) part_b[nx * Yr + X0 + cstep * x] = tile[r * 33 + lane];
            }
            __syncwarp();
        }
    }
    real *fsy = s_fs + g * (nx + ny);
    real *fsx = fsy + nx;
    // downwind x-wall sums: after its last column every row keeps that value
    if (in) {
        real fs = real(0);
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) fs = fma(face_weight(dd, 0), old[dd], fs);
        fsx[Y] = fs;
    }
    // downwind y-wall sums from the top row, which the last warp fed
    if (R + 1 == NRB) {
        __syncwarp();
        real wsy[DW];
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) wsy[dd] = face_weight(dd, 1);
        for (int i = lane; i < nx; i += 32) {
            real fs = real(0);
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) fs = fma(wsy[dd], hand_out[i * DW + dd], fs);
            fsy[X0 + cstep * i] = fs;
        }
    }
    __syncthreads();
    // wall face sums of the chunk, groups in a fixed order
    real *fs_sb = P.fsum + ((long long)s * P.B + b) * P.F;
    for (int q = threadIdx.x; q < ny + nx; q += nthr) {
        real sum = real(0);
        for (int gg = 0; gg < G; ++gg) sum += s_fs[gg * (ny + nx) + q];
        int f;
        if (q < nx)
            f = P.wall_face[(up_y ^ 1) * P.wall_stride + q];
        else
            f = P.wall_face[(up_x ^ 1) * P.wall_stride + (q - nx)];
        if (f >= 0) fs_sb[f] = sum;
    }
}

template <typename real, int DW, int K, bool PHI, bool STORE_E, bool STAGE>
__global__ void __launch_bounds__(kPipeMaxThreads, 1)
sweep2dp_kernel(const __grid_constant__ Sweep2DParams<real> P) {
    sweep2dp_body<real, DW, K, PHI, STORE_E, STAGE>(P, blockIdx.x, blockIdx.y + P.b0);
}

// Batched form: blockIdx.z picks the instance (through `inst`, which lists
// the instances of one size class, largest first); every instance has its
// own parameters, buffers and convergence flag.
template <typename real, int DW, int K, bool PHI, bool STAGE>
__global__ void __launch_bounds__(kPipeMaxThreads, 1)
sweep2dp_batch_kernel(const Sweep2DParams<real> *__restrict__ params, const int *__restrict__ inst) {
    sweep2dp_body<real, DW, K, PHI, false, STAGE>(params[inst[blockIdx.z]], blockIdx.x, blockIdx.y);
}

// Dynamic shared memory of the row-pipeline kernel (bytes).
template <typename real>
size_t sweep2dp_smem_bytes(int nx, int ny, int with_phi, int groups, int dw, int stage) {
    const size_t N = (size_t)nx * ny;
    const size_t Npad = (N + 15) & ~(size_t)15;
    const size_t nrb = (size_t)(ny + 31) / 32;
    size_t n = (stage ? Npad * (with_phi ? 2 : 1) : 0) + (size_t)groups * (nrb + 1) * nx * dw + (size_t)groups * nrb * 32 * 33 +
               (size_t)groups * (nx + ny) + ny;
    return n * sizeof(real) + sizeof(int) * (size_t)groups * (nrb + 1);
}

template <typename real, int DW, int K, bool PHI, bool STORE_E, bool STAGE>
cudaError_t launch_sweep2dp_v(const Sweep2DParams<real> &p, cudaStream_t st) {
    const int nrb = (p.ny + 31) / 32;
    const int threads = p.groups * nrb * 32;
    if (p.groups < 1 || threads > kPipeMaxThreads) return cudaErrorInvalidConfiguration;
    const size_t smem = sweep2dp_smem_bytes<real>(p.nx, p.ny, PHI ? 1 : 0, p.groups, DW, STAGE ? 1 : 0);
    auto kern = sweep2dp_kernel<real, DW, K, PHI, STORE_E, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(kern, dim3(p.S, p.nb ? p.nb : p.B), dim3(threads), smem, st, p);
}

template <typename real, int DW, int K, bool PHI, bool STAGE>
cudaError_t launch_sweep2dp_batch_v(const Sweep2DBatch<real> &bt, cudaStream_t st) {
    const int threads = bt.groups * bt.nrb * 32;
    if (bt.groups < 1 || threads > kPipeMaxThreads || bt.n_inst < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = sweep2dp_smem_bytes<real>(bt.nx_max, bt.ny_max, PHI ? 1 : 0, bt.groups, DW, STAGE ? 1 : 0);
    auto kern = sweep2dp_batch_kernel<real, DW, K, PHI, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<dim3(bt.chunks, bt.B, bt.n_inst), threads, smem, st>>>(bt.params, bt.inst);
    return cudaGetLastError();
}

template <typename real, int DW, int K>
cudaError_t launch_sweep2dp_batch_t(const Sweep2DBatch<real> &bt, cudaStream_t st) {
    if (bt.stage)
        return bt.phi ? launch_sweep2dp_batch_v<real, DW, K, true, true>(bt, st)
                      : launch_sweep2dp_batch_v<real, DW, K, false, true>(bt, st);
    return bt.phi ? launch_sweep2dp_batch_v<real, DW, K, true, false>(bt, st)
                  : launch_sweep2dp_batch_v<real, DW, K, false, false>(bt, st);
}

// the source-profile term only in forward sweeps with a source; e only when asked
template <typename real, int DW, int K, bool STAGE>
cudaError_t launch_sweep2dp_s(const Sweep2DParams<real> &p, cudaStream_t st) {
    const bool phi = !p.adj && p.phi != nullptr;
    if (p.store_e)
        return phi ? launch_sweep2dp_v<real, DW, K, true, true, STAGE>(p, st)
                   : launch_sweep2dp_v<real, DW, K, false, true, STAGE>(p, st);
    return phi ? launch_sweep2dp_v<real, DW, K, true, false, STAGE>(p, st)
               : launch_sweep2dp_v<real, DW, K, false, false, STAGE>(p, st);
}

template <typename real, int DW, int K>
cudaError_t launch_sweep2dp_t(const Sweep2DParams<real> &p, cudaStream_t st) {
    return p.stage ? launch_sweep2dp_s<real, DW, K, true>(p, st) : launch_sweep2dp_s<real, DW, K, false>(p, st);
}

}  // namespace bte
