// Row-block wavefront sweep for unmasked 1D/2D grids with one region.
//
// Same discrete equations as sweep.cuh (Eq. fvm-1 with step upwind faces,
// the triangular matrix A of Eq. A_matrix), organised for small 2D grids:
//
//   * one CTA per (direction chunk, band); a chunk is up to W*DW directions
//     of one quadrant, so they share the traversal order;
//   * each warp owns DW directions over ALL ny rows: lane l of row block r
//     holds row j = 32 r + l in registers (RB blocks), so the y-upwind value
//     of every row comes from lane-1 of the same block (lane 0: lane 31 of
//     block r-1) by one warp shuffle -- no shared-memory exchange and no
//     barrier inside the wavefront loop; warps never wait on each other;
//   * at step t row j updates x = t - j; whole row blocks outside the
//     wavefront are skipped (warp-uniform);
//   * the per-cell source C_b (T - T_ref)/(4 pi tau_b) + Q_b phi (forward) or
//     Theta/tau_b (adjoint) is staged once per CTA in shared memory, as are
//     the upwind wall values; the per-cell weighted direction sum of the
//     CTA's warps is accumulated in shared memory and written once per cell
//     at the end, so a band has only (#chunks) partials per cell.
//
// The shared-memory accumulation uses 64-bit fixed-point integer atomics so
// the result does not depend on the order in which warps arrive (bitwise
// reproducible runs).  The fixed-point scale comes from the discrete maximum
// principle of the upwind update: e_c is a weighted mean of tau*src_c and
// its upwind values, so |e| <= max(tau_b max|src|, max|wall value|) and a
// CTA's per-cell sum is bounded by that times the sum of its weights.
#pragma once

#include "bte_internal.cuh"

namespace bte {

__device__ __forceinline__ long long to_fixed(float v) { return __float2ll_rn(v); }
__device__ __forceinline__ long long to_fixed(double v) { return __double2ll_rn(v); }

template <int DW, int RB>
struct Sweep2DTile {
    static constexpr int kMaxThreads = 512;
};

template <typename real, int DW, int RB, bool ADJ>
__global__ void __launch_bounds__(Sweep2DTile<DW, RB>::kMaxThreads)
sweep2d_kernel(const __grid_constant__ Sweep2DParams<real> P) {
    if (P.done != nullptr && *((volatile const int *)P.done) != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = P.nx * P.ny;
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(smem_raw);  // [N] if acc_smem
    unsigned long long *s_fx = s_acc + (P.acc_smem ? N : 0);  // [ny] downwind x-wall sums
    unsigned long long *s_fy = s_fx + P.ny;                  // [nx] downwind y-wall sums
    real *s_base = reinterpret_cast<real *>(s_fy + P.nx);    // [N]
    real *s_wx = s_base + ((N + 3) & ~3);                    // [ny] upwind x-wall values
    real *s_wy = s_wx + ((P.ny + 3) & ~3);                   // [nx] upwind y-wall values
    __shared__ double s_red[32];
    __shared__ double s_scale[2];

    const int s = blockIdx.x;
    const int b = blockIdx.y;
    const Subset ch = P.sub[s];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nthr = blockDim.x;
    const int B = P.B, D = P.D;
    const bool negx = ch.neg & 1, negy = (ch.neg >> 1) & 1;
    const int up_x = negx ? 1 : 0, up_y = negy ? 3 : 2;
    const int dn_x = up_x ^ 1, dn_y = up_y ^ 1;
    const int *wf = P.wall_face;
    const real *einb = P.ein + (long long)b * P.F;

    // ---- prologue: per-cell source, wall values, accumulators ----
    const real srck = P.srck[b];
    const real qb = (!ADJ && P.phi != nullptr) ? P.qb[b] : real(0);
    double mb = 0.0, mw = 0.0;
    for (int c = threadIdx.x; c < N; c += nthr) {
        real v = P.tsrc[c] * srck;
        if (!ADJ && P.phi != nullptr) v += P.phi[c] * qb;
        s_base[c] = v;
        mb = fmax(mb, fabs((double)v));
        if (P.acc_smem) s_acc[c] = 0ull;
    }
    for (int y = threadIdx.x; y < P.ny; y += nthr) {
        const int f = wf[up_x * P.wall_stride + y];
        s_wx[y] = f >= 0 ? einb[f] : real(0);
        mw = fmax(mw, fabs((double)s_wx[y]));
        s_fx[y] = 0ull;
    }
    for (int x = threadIdx.x; x < P.nx; x += nthr) {
        const int f = wf[up_y * P.wall_stride + x];
        s_wy[x] = f >= 0 ? einb[f] : real(0);
        mw = fmax(mw, fabs((double)s_wy[x]));
        s_fy[x] = 0ull;
    }
    // bound of |e| over the CTA's problems, then the fixed-point scales
    mb = fmax(mb * (double)P.taub[b], mw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) s_red[warp] = mb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bound = 0.0;
        for (int i = 0; i < (nthr >> 5); ++i) bound = fmax(bound, s_red[i]);
        double wsum = 0.0, wmax = 0.0, fsum = 0.0;
        for (int dd = 0; dd < ch.cnt; ++dd) {
            const real *cf = P.coef + ((long long)b * D + ch.d0 + dd) * 8;
            wsum += (double)cf[3];
            wmax = fmax(wmax, (double)cf[3]);
            fsum += ADJ ? fmax((double)cf[0], (double)cf[1]) : fmax((double)cf[4], (double)cf[5]);
        }
        if (ADJ) bound *= wmax;                      // adjoint sources and walls carry w_d
        // floor keeps the scale finite in the sweep precision (values below it
        // are far below the solver's resolution)
        const double floor_b = sizeof(real) == 4 ? 1e-18 : 1e-280;
        const double acc_bound = fmax(bound * (ADJ ? (double)ch.cnt : wsum) * 1.0001, floor_b);
        const double face_bound = fmax(bound * fsum * 1.0001, floor_b);
        s_scale[0] = 4611686018427387904.0 / acc_bound;   // 2^62
        s_scale[1] = 4611686018427387904.0 / face_bound;
    }
    __syncthreads();
    const real sc_acc = (real)s_scale[0];
    const real sc_face = (real)s_scale[1];

    const int d0 = ch.d0 + warp * DW;
    const int ndir = min(DW, ch.cnt - warp * DW);
    if (ndir > 0) {
        real ax[DW], ay[DW], w[DW], invd[DW], wsx[DW], wsy[DW];
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) {
            if (dd < ndir) {
                const real *cf = P.coef + ((long long)b * D + d0 + dd) * 8;
                ax[dd] = cf[0];
                ay[dd] = cf[1];
                w[dd] = cf[3];
                // face-sum weights: forward w|s_a| (energy leaving), adjoint a_a
                wsx[dd] = ADJ ? cf[0] : cf[4];
                wsy[dd] = ADJ ? cf[1] : cf[5];
                invd[dd] = P.invdiag[(long long)b * D + d0 + dd];
            } else {
                ax[dd] = ay[dd] = w[dd] = invd[dd] = wsx[dd] = wsy[dd] = real(0);
            }
        }
        real old[RB][DW];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) old[r][dd] = real(0);
        real *part_sb = P.part + ((long long)s * B + b) * N;
        const int n_steps = P.nx + P.ny - 1;
        const int src_lane = (lane + 31) & 31;
        for (int t = 0; t < n_steps; ++t) {
#pragma unroll
            for (int r = RB - 1; r >= 0; --r) {
                const int j0 = 32 * r;
                if (j0 >= P.ny || t < j0 || t - j0 - 31 >= P.nx) continue;  // block outside the wavefront
                const int j = j0 + lane;
                const int x = t - j;
                const bool valid = (j < P.ny) && (x >= 0) && (x < P.nx);
                const int X = negx ? P.nx - 1 - x : x;
                const int Y = negy ? P.ny - 1 - j : j;
                const int c = X + P.nx * Y;
                const real base = valid ? s_base[c] : real(0);
                const bool bx = (x == 0);
                const bool by = (j == 0);
                const real Ex = (valid && bx) ? s_wx[Y] : real(0);
                const real Ey = (valid && by) ? s_wy[X] : real(0);
                real acc = real(0);
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) {
                    // lane 31 hands row 32r-1 (block r-1) to lane 0 of block r
                    const real prov = (r > 0 && lane == 31) ? old[r > 0 ? r - 1 : 0][dd] : old[r][dd];
                    real vy = __shfl_sync(0xffffffffu, prov, src_lane);
                    real vx = old[r][dd];
                    if (ADJ) {
                        vx = bx ? Ex * w[dd] : vx;
                        vy = by ? Ey * w[dd] : vy;
                    } else {
                        vx = bx ? Ex : vx;
                        vy = by ? Ey : vy;
                    }
                    real r0 = ADJ ? base * w[dd] : base;
                    r0 = fma(ax[dd], vx, r0);
                    r0 = fma(ay[dd], vy, r0);
                    const real en = r0 * invd[dd];
                    if (valid) {
                        old[r][dd] = en;
                        acc = ADJ ? acc + en : fma(w[dd], en, acc);
                    }
                }
                if (valid) {
                    if (P.acc_smem)
                        atomicAdd(&s_acc[c], (unsigned long long)to_fixed(acc * sc_acc));
                    else
                        part_sb[c] = acc;
                    if (P.store_e) {
                        real *ep = P.e + ((long long)c * B + b) * D + d0;
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd)
                            if (dd < ndir) ep[dd] = old[r][dd];
                    }
                    if (x == P.nx - 1) {
                        real fs = real(0);
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd) fs = fma(wsx[dd], old[r][dd], fs);
                        atomicAdd(&s_fx[Y], (unsigned long long)to_fixed(fs * sc_face));
                    }
                    if (j == P.ny - 1) {
                        real fs = real(0);
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd) fs = fma(wsy[dd], old[r][dd], fs);
                        atomicAdd(&s_fy[X], (unsigned long long)to_fixed(fs * sc_face));
                    }
                }
            }
        }
    }
    __syncthreads();
    // ---- epilogue: one partial per cell and per wall face for the CTA ----
    const double inv_acc = 1.0 / s_scale[0], inv_face = 1.0 / s_scale[1];
    if (P.acc_smem) {
        real *part_sb = P.part + ((long long)s * B + b) * N;
        for (int c = threadIdx.x; c < N; c += nthr) part_sb[c] = (real)((double)(long long)s_acc[c] * inv_acc);
    }
    real *fs_sb = P.fsum + ((long long)s * B + b) * P.F;
    for (int y = threadIdx.x; y < P.ny; y += nthr) {
        const int f = wf[dn_x * P.wall_stride + y];
        if (f >= 0) fs_sb[f] = (real)((double)(long long)s_fx[y] * inv_face);
    }
    for (int x = threadIdx.x; x < P.nx; x += nthr) {
        const int f = wf[dn_y * P.wall_stride + x];
        if (f >= 0) fs_sb[f] = (real)((double)(long long)s_fy[x] * inv_face);
    }
}

template <typename real>
size_t sweep2d_smem_bytes(int nx, int ny, int acc_smem) {
    const size_t N = (size_t)nx * ny;
    const size_t fixed = 8 * ((acc_smem ? N : 0) + (size_t)nx + (size_t)ny);
    const size_t n = ((N + 3) & ~(size_t)3) + (((size_t)ny + 3) & ~(size_t)3) + (((size_t)nx + 3) & ~(size_t)3);
    return fixed + n * sizeof(real);
}

template <typename real, int DW, int RB, bool ADJ>
cudaError_t launch_sweep2d_t(const Sweep2DParams<real> &p, cudaStream_t st) {
    const int threads = p.warps_per_cta * 32;
    if (threads > Sweep2DTile<DW, RB>::kMaxThreads || p.ny > 32 * RB) return cudaErrorInvalidConfiguration;
    const size_t smem = sweep2d_smem_bytes<real>(p.nx, p.ny, p.acc_smem);
    auto kern = sweep2d_kernel<real, DW, RB, ADJ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<dim3(p.S, p.B), threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace bte
