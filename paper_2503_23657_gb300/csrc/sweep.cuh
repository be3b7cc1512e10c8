// Exact upwind transport sweep for a set of (band, direction) pairs.
//
// Each (band b, direction d) problem of Eq. (fvm-1) with step upwind faces is
// the lower-triangular system A of Eq. (A_matrix) in the sweep order of d's
// octant: cell c depends only on its upwind neighbours along x, y and z.
//   e_c = (src_c + a_x e_up_x + a_y e_up_y + a_z e_up_z) / (1/tau_cb + a_x + a_y + a_z)
// with a_axis = v_b |s_d,axis| / h_axis (S_ij / V_i = 1/h), and the upwind
// value replaced by the boundary value where the upwind neighbour is outside
// the domain or void.
//
// Work decomposition (one CTA per (direction subset, band)):
//   * a direction subset holds up to DW directions that share one octant, so
//     they share the traversal order; each lane carries all DW of them;
//   * lane (j, k) owns the pencil of cells (., j, k) in canonical (octant-
//     mirrored) coordinates: j = 32*warp_y + lane, k = LZ*warp_z + l for the
//     LZ layers it keeps in registers;
//   * at step t the lane updates x = t - j - k (a diagonal wavefront), so
//     the x-upwind value is its own register from step t-1, the y-upwind
//     value comes from lane-1 by warp shuffle (lane 0: from the warp below
//     through shared memory) and the z-upwind value from its own next-lower
//     layer register (layer 0: from the warp group below through shared
//     memory).  One barrier per step; exchange buffers are double-buffered.
//
// Extended variant (EXT): specularly reflecting domain faces and a per-
// (cell, band, direction) source term.  Specular faces: the inflow through a
// specular face on the upwind side of cell c along axis a is, per
// direction d, the previous iterate's value of the mirror direction of d (the
// axis-a component reversed) in the same cell.  The sweep itself provides it:
// where a cell's downwind side along a is specular, the cell's value of
// direction d is stored under mirror_a(d) in the next iterate's specular
// array.  The adjoint uses the same two rules on mu (the transposed coupling
// of a specular face is a_d mu_old(mirror d) at the face d leaves by, which is
// the face the flipped traversal enters by).  The extra source (forward
// sweeps): xscale * xsrc[c][b][d] is added to the right-hand side of each
// direction -- e_prev/dt of an implicit-Euler time step, or the deferred
// correction of second-order faces.
//
// The same kernel runs the transposed (adjoint) sweep: the host passes the
// octant signs flipped, so cells are visited downwind-first and couple to
// their forward-downwind neighbours; the source is w_d Theta_c / tau_cb and
// the boundary term of a diffuse face is w_d |s_d,axis| M_f,b (passed as
// M' = M h/v so that it is a_axis * (M' w_d)).
#pragma once

#include "bte_internal.cuh"

namespace bte {

template <typename real>
__device__ __forceinline__ real ldg(const real *p) { return __ldg(p); }

template <int DW, int LZ, bool Z>
struct SweepTile {
    static constexpr int kMaxThreads = (DW * LZ >= 16) ? ((LZ > 1) ? 1024 : 256) : 1024;
};

// The sweep of direction subset s of band b of problem P, by one CTA.
template <typename real, int DW, int LZ, bool Z, bool ADJ, bool EXT>
__device__ __forceinline__ void sweep_body(const SweepParams<real> &P, const int s, const int b) {
    {
        // one thread reads the stop flag: every warp of the CTA decides alike
        __shared__ int s_done;
        if (threadIdx.x == 0) s_done = (P.done != nullptr && *((volatile const int *)P.done) != 0) ? 1 : 0;
        __syncthreads();
        if (s_done) return;
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *s_invd = reinterpret_cast<real *>(smem_raw);                 // [R][DW]
    real *s_srck = s_invd + P.R * DW;                                    // [R]
    const int nwarps = P.WY * P.WZ;
    real *s_y = s_srck + ((P.R + 1) & ~1);                               // [2][nwarps][LZ][DW]
    real *s_z = s_y + 2 * nwarps * LZ * DW;                              // [2][nwarps][DW][32] (lane fastest)
    real *s_ein = s_z + (Z ? 2 * nwarps * 32 * DW : 0);                  // [F] (ein_smem)

    const Subset sub = P.sub[s];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wy = warp % P.WY;
    const int wz = warp / P.WY;
    const int j = wy * 32 + lane;
    const int k0 = wz * LZ;
    const int B = P.B, D = P.D;
    const long long N = P.N;

    // traversal orientation and the sides a cell is entered / left by
    const bool nx_ = sub.neg & 1, ny_ = (sub.neg >> 1) & 1, nz_ = (sub.neg >> 2) & 1;
    const int up_x = nx_ ? 1 : 0, up_y = ny_ ? 3 : 2, up_z = nz_ ? 5 : 4;

    // per-direction coefficients in registers
    real ax[DW], ay[DW], az[DW], w[DW];
#pragma unroll
    for (int dd = 0; dd < DW; ++dd) {
        if (dd < sub.cnt) {
            const real *cf = P.coef + ((long long)b * D + sub.d0 + dd) * 8;
            ax[dd] = cf[0];
            ay[dd] = cf[1];
            az[dd] = Z ? cf[2] : real(0);
            w[dd] = cf[3];
        } else {
            ax[dd] = ay[dd] = az[dd] = w[dd] = real(0);
        }
    }
    for (int i = threadIdx.x; i < P.R * DW; i += blockDim.x) {
        const int r = i / DW, dd = i % DW;
        s_invd[i] = (dd < sub.cnt) ? P.invdiag[((long long)r * B + b) * D + sub.d0 + dd] : real(0);
    }
    for (int r = threadIdx.x; r < P.R; r += blockDim.x) s_srck[r] = P.srck[r * B + b];
    const real qb = (!ADJ && P.phi != nullptr) ? P.qb[b] : real(0);
    const real cb4pi = (ADJ && P.read_e) ? P.cb4pi[b] : real(0);
    const real *einb = P.ein + (long long)b * P.F;
    if (P.ein_smem) {
        for (int f = threadIdx.x; f < P.F; f += blockDim.x) s_ein[f] = einb[f];
        einb = s_ein;
    }
    __syncthreads();

    real old[LZ][DW];
#pragma unroll
    for (int l = 0; l < LZ; ++l)
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) old[l][dd] = real(0);

    const bool vec_ok = (sub.cnt == DW) && ((D & 3) == 0) && ((sub.d0 & 3) == 0) && (DW % 4 == 0);
    const int n_steps = P.nx + P.ny + P.nz - 2;
    // partial sums [B][Spad][N]: this CTA's set s of band b
    real *const part_sb = P.part + ((long long)b * P.Spad + s) * N;
    real *const gpart_sb = (ADJ && P.read_e) ? P.gpart + ((long long)b * P.Spad + s) * N : nullptr;

    for (int t = 0; t < n_steps; ++t) {
        const int rb = (t + 1) & 1;  // buffer written at step t-1
        const int wb = t & 1;
#pragma unroll
        for (int l = LZ - 1; l >= 0; --l) {
            const int k = k0 + l;
            const int x = t - j - k;
            const bool inr = ((unsigned)x < (unsigned)P.nx) && (j < P.ny) && (k < P.nz);
            long long c = 0;
            int2 ci = make_int2(0, 0);
            real tsv = real(0), phv = real(0);
            if (inr) {
                const int X = nx_ ? P.nx - 1 - x : x;
                const int Y = ny_ ? P.ny - 1 - j : j;
                const int Zc = nz_ ? P.nz - 1 - k : k;
                c = X + (long long)P.nx * (Y + (long long)P.ny * Zc);
                // independent loads issued together (the source does not wait
                // for the cell record)
                ci = P.cell[c];
                tsv = ldg(P.tsrc + c);
                if (!ADJ && P.phi != nullptr) phv = ldg(P.phi + c);
            }
            const int region = ci.y & kRegionMask;
            const bool act = inr && (region != 0);
            const unsigned bm = ((unsigned)ci.y >> kSideShift) & 63u;
            const bool bx = (bm >> up_x) & 1u;
            const bool by = (bm >> up_y) & 1u;
            const bool bz = Z && ((bm >> up_z) & 1u);
            real Ex = real(0), Ey = real(0), Ez = real(0);
            if (bx) Ex = einb[face_of(ci.x, ci.y, up_x)];
            if (by) Ey = einb[face_of(ci.x, ci.y, up_y)];
            if (Z && bz) Ez = einb[face_of(ci.x, ci.y, up_z)];
            // specular upwind faces: per-direction inflow rows (-1: none)
            long long sx_row = -1, sy_row = -1, sz_row = -1;
            if (EXT && P.sidx) {
                const long long rb0 = (long long)b * P.Fs;
                int si;
                if (bx && (si = P.sidx[face_of(ci.x, ci.y, up_x)]) >= 0) sx_row = (rb0 + si) * D + sub.d0;
                if (by && (si = P.sidx[face_of(ci.x, ci.y, up_y)]) >= 0) sy_row = (rb0 + si) * D + sub.d0;
                if (Z && bz && (si = P.sidx[face_of(ci.x, ci.y, up_z)]) >= 0) sz_row = (rb0 + si) * D + sub.d0;
            }
            real base = real(0);
            real thc = real(0);
            if (act) {
                thc = tsv;
                base = thc * s_srck[region - 1];
                if (!ADJ && P.phi != nullptr) base += phv * qb;
            }
            const real *invd = s_invd + (act ? region - 1 : 0) * DW;
            real acc = real(0);
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) {
                real vy = __shfl_up_sync(0xffffffffu, old[l][dd], 1);
                if (lane == 0 && wy > 0) vy = s_y[((rb * nwarps + warp - 1) * LZ + l) * DW + dd];
                real vx = old[l][dd];
                real vz = real(0);
                if (Z) {
                    if (l > 0) vz = old[l - 1][dd];
                    else if (wz > 0) vz = s_z[((rb * nwarps + warp - P.WY) * DW + dd) * 32 + lane];
                }
                if (ADJ) {
                    vx = bx ? Ex * w[dd] : vx;
                    vy = by ? Ey * w[dd] : vy;
                    if (Z) vz = bz ? Ez * w[dd] : vz;
                } else {
                    vx = bx ? Ex : vx;
                    vy = by ? Ey : vy;
                    if (Z) vz = bz ? Ez : vz;
                }
                if (EXT && P.sidx && dd < sub.cnt) {
                    // mirror-direction inflow (e, or mu in the adjoint: no w factor)
                    if (sx_row >= 0) vx = P.spec_in[sx_row + dd];
                    if (sy_row >= 0) vy = P.spec_in[sy_row + dd];
                    if (Z && sz_row >= 0) vz = P.spec_in[sz_row + dd];
                }
                real r0 = ADJ ? base * w[dd] : base;
                if (EXT && !ADJ && P.xsrc && act && dd < sub.cnt)
                    r0 = fma(P.xscale, P.xsrc[(c * B + b) * (long long)D + sub.d0 + dd], r0);
                r0 = fma(ax[dd], vx, r0);
                r0 = fma(ay[dd], vy, r0);
                if (Z) r0 = fma(az[dd], vz, r0);
                const real en = r0 * invd[dd];
                if (act) {
                    old[l][dd] = en;
                    acc = ADJ ? acc + en : fma(w[dd], en, acc);
                }
            }
            if (act) {
                part_sb[c] = acc;
                real *ep = P.e + (c * B + b) * (long long)D + sub.d0;
                if (!ADJ && P.store_e) {
                    if (vec_ok) {
#pragma unroll
                        for (int q = 0; q < DW; q += 4) {
                            if constexpr (sizeof(real) == 4) {
                                *reinterpret_cast<float4 *>(ep + q) =
                                    make_float4(old[l][q], old[l][q + 1], old[l][q + 2], old[l][q + 3]);
                            } else {
                                *reinterpret_cast<double2 *>(ep + q) = make_double2(old[l][q], old[l][q + 1]);
                                *reinterpret_cast<double2 *>(ep + q + 2) = make_double2(old[l][q + 2], old[l][q + 3]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd)
                            if (dd < sub.cnt) ep[dd] = old[l][dd];
                    }
                }
                if (ADJ && P.read_e) {
                    // (mu - w Theta)(e - e0) with e0 = C_b (T - T_ref)/(4 pi)
                    const real e0 = cb4pi * P.tfwd[c];
                    real ev[DW];
                    if (vec_ok) {
                        // DW consecutive values of e, aligned: vector loads
#pragma unroll
                        for (int q = 0; q < DW; q += 4) {
                            if constexpr (sizeof(real) == 4) {
                                const float4 x = *reinterpret_cast<const float4 *>(ep + q);
                                ev[q] = x.x;
                                ev[q + 1] = x.y;
                                ev[q + 2] = x.z;
                                ev[q + 3] = x.w;
                            } else {
                                const double2 x = *reinterpret_cast<const double2 *>(ep + q);
                                const double2 y = *reinterpret_cast<const double2 *>(ep + q + 2);
                                ev[q] = x.x;
                                ev[q + 1] = x.y;
                                ev[q + 2] = y.x;
                                ev[q + 3] = y.y;
                            }
                        }
                    } else {
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd) ev[dd] = dd < sub.cnt ? ep[dd] : real(0);
                    }
                    real g = real(0);
#pragma unroll
                    for (int dd = 0; dd < DW; ++dd)
                        if (dd < sub.cnt) g = fma(old[l][dd] - w[dd] * thc, ev[dd] - e0, g);
                    gpart_sb[c] = g;
                    if (EXT && P.glpart) {
                        // cell-size derivative: sum_d mu_d a^a_d (e_d - e_in,a,d), the
                        // forward inflow e_in of axis a coming through the side
                        // this (flipped) traversal leaves by
                        for (int a = 0; a < P.dim; ++a) {
                            const int fside = (a == 0 ? up_x : (a == 1 ? up_y : up_z)) ^ 1;
                            const bool fb_bnd = (bm >> fside) & 1u;
                            long long nrow = 0, srow = -1;
                            real einv = real(0);
                            if (fb_bnd) {
                                const int f = face_of(ci.x, ci.y, fside);
                                const int si = P.sidx ? P.sidx[f] : -1;
                                if (si >= 0)
                                    srow = ((long long)b * P.Fs + si) * D + sub.d0;
                                else
                                    einv = P.ein_fwd[(long long)b * P.F + f];
                            } else {
                                const long long stride =
                                    a == 0 ? 1LL : (a == 1 ? (long long)P.nx : (long long)P.nx * P.ny);
                                const long long cn = (fside & 1) ? c + stride : c - stride;
                                nrow = (cn * B + b) * (long long)D + sub.d0;
                            }
                            real gl = real(0);
#pragma unroll
                            for (int dd = 0; dd < DW; ++dd) {
                                if (dd >= sub.cnt) continue;
                                const real ein_d =
                                    fb_bnd ? (srow >= 0 ? P.spec_fwd[srow + dd] : einv) : P.e[nrow + dd];
                                const real cf = a == 0 ? ax[dd] : (a == 1 ? ay[dd] : az[dd]);
                                gl = fma(old[l][dd] * cf, ev[dd] - ein_d, gl);
                            }
                            P.glpart[(((long long)a * B + b) * P.Spad + s) * N + c] = gl;
                        }
                    }
                }
                // face sums at the boundary sides the traversal leaves by
                if (bm & ((1u << (up_x ^ 1)) | (1u << (up_y ^ 1)) | (Z ? (1u << (up_z ^ 1)) : 0u))) {
#pragma unroll
                    for (int a = 0; a < (Z ? 3 : 2); ++a) {
                        const int upa = a == 0 ? up_x : (a == 1 ? up_y : up_z);
                        const int dn = upa ^ 1;
                        if (!((bm >> dn) & 1u)) continue;
                        if (EXT && P.sidx) {
                            const int si = P.sidx[face_of(ci.x, ci.y, dn)];
                            if (si >= 0) {
                                // this cell's outgoing values, stored under the mirror directions
                                real *so = P.spec_out + ((long long)b * P.Fs + si) * D;
#pragma unroll
                                for (int dd = 0; dd < DW; ++dd)
                                    if (dd < sub.cnt) so[P.mirror[a * D + sub.d0 + dd]] = old[l][dd];
                                continue;
                            }
                        }
                        real fs = real(0);
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd) {
                            if (dd >= sub.cnt) continue;
                            const real *cf = P.coef + ((long long)b * D + sub.d0 + dd) * 8;
                            // forward: w |s_a| (outgoing energy); adjoint: a_a (incoming coupling)
                            const real wt = ADJ ? cf[a] : cf[4 + a];
                            fs = fma(wt, old[l][dd], fs);
                        }
                        P.fsum[((long long)s * B + b) * P.F + face_of(ci.x, ci.y, dn)] = fs;
                    }
                }
            }
        }
        // publish this step's values to the neighbouring warps
        if (lane == 31) {
#pragma unroll
            for (int l = 0; l < LZ; ++l)
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) s_y[((wb * nwarps + warp) * LZ + l) * DW + dd] = old[l][dd];
        }
        if (Z) {
#pragma unroll
            for (int dd = 0; dd < DW; ++dd) s_z[((wb * nwarps + warp) * DW + dd) * 32 + lane] = old[LZ - 1][dd];
        }
        __syncthreads();
    }
}

template <typename real, int DW, int LZ, bool Z, bool ADJ, bool EXT = false>
__global__ void __launch_bounds__(SweepTile<DW, LZ, Z>::kMaxThreads)
sweep_kernel(const __grid_constant__ SweepParams<real> P) {
    sweep_body<real, DW, LZ, Z, ADJ, EXT>(P, blockIdx.x, blockIdx.y + P.b0);
}

// Batched form for 2D instances (forward): blockIdx.z = the instance among
// those of one class (same warps per CTA), whose parameters are read from
// device memory; subsets beyond an instance's own count do nothing.
template <typename real, int DW>
__global__ void __launch_bounds__(SweepTile<DW, 1, false>::kMaxThreads)
sweep_batch_kernel(const SweepParams<real> *__restrict__ params, const int *__restrict__ inst) {
    const SweepParams<real> &P = params[inst[blockIdx.z]];
    if ((int)blockIdx.x >= P.S || (int)blockIdx.y >= P.B) return;
    sweep_body<real, DW, 1, false, false, false>(P, blockIdx.x, blockIdx.y);
}

template <typename real, int DW, int LZ, bool Z>
size_t sweep_smem_bytes(int R, int nwarps, int F, int ein_smem) {
    size_t n = (size_t)R * DW + ((R + 1) & ~1) + 2 * (size_t)nwarps * LZ * DW;
    if (Z) n += 2 * (size_t)nwarps * 32 * DW;
    if (ein_smem) n += (size_t)F;
    return n * sizeof(real);
}

template <typename real, int DW, int LZ, bool Z, bool ADJ, bool EXT = false>
cudaError_t launch_sweep_t(const SweepParams<real> &p, cudaStream_t st) {
    const int nwarps = p.WY * p.WZ;
    const int threads = nwarps * 32;
    if (threads > SweepTile<DW, LZ, Z>::kMaxThreads) return cudaErrorInvalidConfiguration;
    if (!EXT && (p.sidx != nullptr || p.xsrc != nullptr || p.glpart != nullptr)) return cudaErrorInvalidConfiguration;
    const size_t smem = sweep_smem_bytes<real, DW, LZ, Z>(p.R, nwarps, p.F, p.ein_smem);
    auto kern = sweep_kernel<real, DW, LZ, Z, ADJ, EXT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(p.S, p.nb ? p.nb : p.B);
    kern<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace bte
