// Row-block wavefront sweep for unmasked 1D/2D grids with one region.
//
// Same discrete equations as sweep.cuh (Eq. fvm-1 with step upwind faces,
// the triangular matrix A of Eq. A_matrix), organised for small 2D grids:
//
//   * one CTA per (direction chunk, band): a chunk is up to W*DW directions
//     of one quadrant (one traversal order); warp w owns DW of them over ALL
//     ny rows.  Lane l of row block r holds row j = 32 r + l in registers
//     (RB blocks), so the y-upwind value of a row comes from lane-1 of the
//     same block (lane 0: lane 31 of block r-1) by one warp shuffle and the
//     x-upwind value is the lane's own register from the previous step;
//   * at step t row j updates x = t - j.  The set of row blocks inside the
//     wavefront changes only a few times per sweep, so each such phase runs
//     straight-line code over exactly its active blocks (a template per
//     (first, last) active block): the RB*DW independent recurrences of a
//     step interleave freely, with no per-block branch;
//   * the per-cell temperature deviation (and source profile) is brought
//     into shared memory once per CTA by a TMA bulk copy (cp.async.bulk on
//     an mbarrier, bounded wait), the band's upwind wall values are staged;
//   * per-cell weighted direction sums: every warp stores its own partial
//     set directly (one 4-byte store per lane and step; the lanes of a step
//     sit on a diagonal, so a warp store touches 32 sectors -- the store path,
//     not the arithmetic, is what larger DW amortises).  Results do not depend
//     on scheduling.  Wall face sums are combined over the CTA's warps in a
//     fixed order.
#pragma once

#include <stdint.h>

#include "bte_internal.cuh"
#include "tma.cuh"

namespace bte {


template <int DW, int RB>
struct Sweep2DTile {
    static constexpr int kMaxThreads = 512;
};

// Per-warp sweep state; everything lives in registers after inlining.
template <typename real, int DW, int RB, bool ADJ>
struct RowSweep {
    real old[RB][DW];  // value of this lane's row at its last x (the x-upwind value)
    int yrow[RB];      // Y (grid row) of this lane's row in block r
    int t_lo[RB];      // step at which the row enters the grid (x = 0)
    int c_base[RB];    // cell index at step t is c_base + cstep * t
    real ax[DW], ay[DW], w[DW], invd[DW], wsy[DW];
    int cstep, lane, nx, last_row, set;
    real srck, qb;
    bool with_phi, store_e, direct;
    const real *src_t, *src_phi, *wy;
    real *part_b;      // band b's partials, this warp's set
    real *fsy;         // this warp's downwind y-wall sums, by X
    real *e;
    long long eoff;    // b * D + d0
    int BD, ndir;

    // One wavefront step over the active blocks LO..HI, written as four
    // phases in program order: (A) indices and shared-memory loads of every
    // block, (B) all warp shuffles, (C) all arithmetic, (D) all stores.
    // The shuffles read the previous step's registers, so they all precede
    // the updates; keeping loads, shuffles and stores in separate phases
    // lets the independent recurrences of all blocks and directions overlap.
    template <int LO, int HI>
    __device__ __forceinline__ void step(int t, int slot) {
        constexpr int NB = HI - LO + 1;
        int dxs[NB], cs[NB];
        bool vals[NB];
        real base[NB];
        real Ey = real(0);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int R = LO + i;
            dxs[i] = t - t_lo[R];
            vals[i] = (unsigned)dxs[i] < (unsigned)nx;
            cs[i] = c_base[R] + cstep * t;
            real bv = vals[i] ? src_t[cs[i]] : real(0);
            bv *= srck;
            if (with_phi) bv = fma(vals[i] ? src_phi[cs[i]] : real(0), qb, bv);
            base[i] = bv;
            if (R == 0) Ey = (lane == 0 && vals[i]) ? wy[cs[i] - nx * yrow[0]] : real(0);
        }
        real vy[NB][DW];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int R = LO + i;
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                // lane 31 hands row 32R-1 (block R-1) to lane 0 of block R
                real prov = old[R][dd];
                if (R > 0) prov = (lane == 31) ? old[R > 0 ? R - 1 : 0][dd] : prov;
                vy[i][dd] = __shfl_sync(0xffffffffu, prov, (lane + 31) & 31);
            }
        }
        real acc[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int R = LO + i;
            acc[i] = real(0);
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                real yv = vy[i][dd];
                if (R == 0) yv = (lane == 0) ? (ADJ ? Ey * w[dd] : Ey) : yv;  // row 0: upwind y-wall
                real r0 = ADJ ? base[i] * w[dd] : base[i];
                r0 = fma(ax[dd], old[R][dd], r0);  // x-upwind (the wall value before x = 0)
                r0 = fma(ay[dd], yv, r0);
                const real en = r0 * invd[dd];
                old[R][dd] = vals[i] ? en : old[R][dd];
                acc[i] = ADJ ? acc[i] + en : fma(w[dd], en, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int R = LO + i;
            const bool valid = vals[i];
            const int c = cs[i];
            if (valid) part_b[c] = acc[i];
            if (store_e && valid) {
                real *ep = e + (long long)c * BD + eoff;
#pragma unroll
                for (int dd = 0; dd < DW; ++dd)
                    if (dd < ndir) ep[dd] = old[R][dd];
            }
            if (32 * R + lane == last_row && valid) {
                real fs = real(0);
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) fs = fma(wsy[dd], old[R][dd], fs);
                fsy[c - nx * yrow[R]] = fs;
            }
        }
    }

    template <int LO, int HI>
    __device__ __forceinline__ void steps(int t_begin, int t_end, int t0) {
        for (int t = t_begin; t < t_end; ++t) step<LO, HI>(t, t - t0);
    }

    static_assert(RB >= 1 && RB <= 5, "row blocks");
};

template <typename real, int DW, int RB, bool ADJ>
__global__ void __launch_bounds__(Sweep2DTile<DW, RB>::kMaxThreads)
sweep2d_kernel(const __grid_constant__ Sweep2DParams<real> P) {
    {
        // one thread reads the stop flag: every warp of the CTA decides alike
        __shared__ int s_done;
        if (threadIdx.x == 0) s_done = (P.done != nullptr && *((volatile const int *)P.done) != 0) ? 1 : 0;
        __syncthreads();
        if (s_done) return;
    }
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const int N = P.nx * P.ny;
    const int Npad = (N + 15) & ~15;
    const int W = P.warps_per_cta;
    const bool direct = (P.ring == 0);
    const bool with_phi = (!ADJ && P.phi != nullptr);
    real *s_t = reinterpret_cast<real *>(smem_raw);                  // [Npad] T - T_ref or Theta
    real *s_phi = s_t + Npad;                                        // [Npad] source profile (fwd)
    real *s_fs = s_phi + (with_phi ? Npad : 0);                      // [W][nx + ny] wall sums
    real *s_wx = s_fs + W * (P.ny + P.nx);                           // [ny] upwind x-wall values
    real *s_wy = s_wx + P.ny;                                        // [nx] upwind y-wall values

    const int s = blockIdx.x;  // chunk = partial set
    const int b = blockIdx.y + P.b0;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nthr = blockDim.x;
    const int B = P.B, D = P.D;
    const Subset ch = P.sub[s];
    const bool negx = ch.neg & 1, negy = (ch.neg >> 1) & 1;
    const int up_x = negx ? 1 : 0, up_y = negy ? 3 : 2;

    // ---- prologue: TMA bulk copy of the per-cell inputs, wall values ----
    {
        if (threadIdx.x == 0) {
            mbar_init(&s_bar, 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t bytes = (uint32_t)(Npad * sizeof(real));
            mbar_arrive_expect_tx(&s_bar, with_phi ? 2 * bytes : bytes);
            bulk_copy_g2s(s_t, P.tsrc, bytes, &s_bar);
            if (with_phi) bulk_copy_g2s(s_phi, P.phi, bytes, &s_bar);
        }
    }
    {
        const real *einb = P.ein + (long long)b * P.F;
        for (int y = threadIdx.x; y < P.ny; y += nthr) {
            const int f = P.wall_face[up_x * P.wall_stride + y];
            s_wx[y] = f >= 0 ? einb[f] : real(0);
        }
        for (int x = threadIdx.x; x < P.nx; x += nthr) {
            const int f = P.wall_face[up_y * P.wall_stride + x];
            s_wy[x] = f >= 0 ? einb[f] : real(0);
        }
        for (int i = threadIdx.x; i < W * (P.ny + P.nx); i += nthr) s_fs[i] = real(0);
    }
    const bool ok = mbar_wait_bounded(&s_bar, 0, kWaitPolls);
    __syncthreads();
    if (!ok) {
        // the bulk copy did not complete: report, wait once more for it, stop
        if (threadIdx.x == 0) {
            atomicExch(P.status, 2);
            mbar_wait_bounded(&s_bar, 0, kWaitPolls);
        }
        return;
    }

    // ---- this warp's directions ----
    RowSweep<real, DW, RB, ADJ> S;
    S.lane = lane;
    S.nx = P.nx;
    S.last_row = P.ny - 1;
    S.cstep = negx ? -1 : 1;
    S.with_phi = with_phi;
    S.store_e = P.store_e != 0;
    S.direct = direct;
    S.set = direct ? s * W + warp : s;
    // staged inputs only: shared-memory pointers the compiler can see as such
    S.src_t = s_t;
    S.src_phi = s_phi;
    S.wy = s_wy;
    // partial sums [B][sets][N]
    S.part_b = P.part + ((long long)b * P.Spad + S.set) * N;
    S.fsy = s_fs + warp * (P.ny + P.nx);
    real *fsx = S.fsy + P.nx;
    S.e = P.e;
    S.BD = B * D;
    S.srck = P.srck[b];
    S.qb = with_phi ? P.qb[b] : real(0);
    const int d0 = ch.d0 + warp * DW;
    S.ndir = max(0, min(DW, ch.cnt - warp * DW));
    S.eoff = (long long)b * D + d0;
    real wsx[DW];
#pragma unroll
    for (int dd = 0; dd < DW; ++dd) {
        if (dd < S.ndir) {
            const real *cf = P.coef + ((long long)b * D + d0 + dd) * 8;
            S.ax[dd] = cf[0];
            S.ay[dd] = cf[1];
            S.w[dd] = cf[3];
            // face-sum weights: forward w|s_a| (energy leaving), adjoint a_a
            wsx[dd] = ADJ ? cf[0] : cf[4];
            S.wsy[dd] = ADJ ? cf[1] : cf[5];
            S.invd[dd] = P.invdiag[(long long)b * D + d0 + dd];
        } else {
            S.ax[dd] = S.ay[dd] = S.w[dd] = S.invd[dd] = wsx[dd] = S.wsy[dd] = real(0);
        }
    }
    const int X0 = negx ? P.nx - 1 : 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int j = 32 * r + lane;
        const bool in = j < P.ny;
        const int Y = negy ? P.ny - 1 - j : j;
        S.yrow[r] = in ? Y : 0;
        S.t_lo[r] = in ? j : (1 << 29);  // rows beyond the grid are never valid
        S.c_base[r] = X0 + P.nx * Y - S.cstep * j;
        // before the row enters the grid its x-upwind value is the wall value
        const real ex = in ? s_wx[Y] : real(0);
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) S.old[r][dd] = ADJ ? ex * S.w[dd] : ex;
    }

    // ---- wavefront: phases of constant active blocks ----
    const int n_steps = P.nx + P.ny - 1;
    const int nblk = (P.ny + 31) / 32;
    int tt = 0;
    while (tt < n_steps) {
        const int lo = (tt - 31 - P.nx < 0) ? 0 : (tt - 31 - P.nx) / 32 + 1;
        const int hi = min(nblk - 1, tt / 32);
        int tn = n_steps;
        if (hi + 1 < nblk) tn = min(tn, 32 * (hi + 1));
        tn = min(tn, 32 * lo + 31 + P.nx);
#define BTE_PHASE(L, H)                                                \
    case (L) * 8 + (H):                                                \
        if constexpr ((H) < RB) S.template steps<(L), (H)>(tt, tn, 0); \
        break;
        switch (lo * 8 + hi) {
            BTE_PHASE(0, 0) BTE_PHASE(0, 1) BTE_PHASE(0, 2) BTE_PHASE(0, 3) BTE_PHASE(0, 4)
            BTE_PHASE(1, 1) BTE_PHASE(1, 2) BTE_PHASE(1, 3) BTE_PHASE(1, 4)
            BTE_PHASE(2, 2) BTE_PHASE(2, 3) BTE_PHASE(2, 4)
            BTE_PHASE(3, 3) BTE_PHASE(3, 4)
            BTE_PHASE(4, 4)
            default: break;
        }
#undef BTE_PHASE
        tt = tn;
    }
    // downwind x-wall sums: after its last column every row keeps that value
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (32 * r + lane < P.ny) {
            real fs = real(0);
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) fs = fma(wsx[dd], S.old[r][dd], fs);
            fsx[S.yrow[r]] = fs;
        }
    }
    __syncthreads();
    // wall face sums of the chunk: downwind y wall (by X), downwind x wall (by Y)
    real *fs_sb = P.fsum + ((long long)s * B + b) * P.F;
    for (int i = threadIdx.x; i < P.ny + P.nx; i += nthr) {
        real sum = real(0);
        for (int q = 0; q < W; ++q) sum += s_fs[q * (P.ny + P.nx) + i];
        int f;
        if (i < P.nx)
            f = P.wall_face[(up_y ^ 1) * P.wall_stride + i];
        else
            f = P.wall_face[(up_x ^ 1) * P.wall_stride + (i - P.nx)];
        if (f >= 0) fs_sb[f] = sum;
    }
}

template <typename real>
size_t sweep2d_smem_bytes(int nx, int ny, int stage, int with_phi, int warps, int rb, int ring) {
    const size_t N = (size_t)nx * ny;
    const size_t Npad = (N + 15) & ~(size_t)15;
    (void)ring;
    (void)rb;
    size_t n = (size_t)warps * (nx + ny) + nx + ny;
    (void)stage;
    n += Npad * (with_phi ? 2 : 1);  // per-cell inputs are always staged
    return n * sizeof(real);
}

template <typename real, int DW, int RB, bool ADJ>
cudaError_t launch_sweep2d_t(const Sweep2DParams<real> &p, cudaStream_t st) {
    const int threads = p.warps_per_cta * 32;
    if (threads > Sweep2DTile<DW, RB>::kMaxThreads || p.ny > 32 * RB) return cudaErrorInvalidConfiguration;
    const size_t smem =
        sweep2d_smem_bytes<real>(p.nx, p.ny, p.stage, (!ADJ && p.phi != nullptr) ? 1 : 0, p.warps_per_cta, RB,
                                 p.ring);
    auto kern = sweep2d_kernel<real, DW, RB, ADJ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<dim3(p.S, p.nb ? p.nb : p.B), threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace bte
