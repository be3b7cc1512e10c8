// Plane-pipeline wavefront sweep for 3D grids (masked, any number of regions).
//
// Same discrete equations as sweep.cuh (Eq. fvm-1 with step upwind faces,
// the lower-triangular matrix A of Eq. A_matrix in the sweep order of the
// direction's octant), with the work of one (band, direction subset) spread
// over a CTA as a pipeline of warps:
//
//   * one CTA per (direction subset of DW directions sharing an octant,
//     band).  x is marched; the lanes hold rows along the row axis (y, or z
//     when the host picks it: lane_axis) and the planes lie along the other
//     axis.  WY = ceil(rows / 32) warps along the row axis times H warps
//     along the plane axis; warp (wy, h) owns rows 32 wy .. 32 wy + 31 of
//     the planes h, h + H, h + 2H, ... (one pass of H planes after the
//     other); every lane carries the DW directions in registers.  Below,
//     "y" and "z" name the row and plane axes;
//   * in canonical (octant-mirrored) coordinates lane l of a warp handles the
//     virtual column u = tau - l at its local step tau, u = m nx + i meaning
//     column i of the warp's plane in pass m, so a lane streams through its
//     rows of all passes without a gap.  The x-upwind value is the lane's
//     own register from the previous step, the y-upwind value comes from
//     lane l - 1 by a shuffle (lane 0: from lane 31 of the warp below
//     through a shared-memory ring), the z-upwind value from the same lane
//     of the warp below in z through a shared-memory ring (the first warp
//     of a pass: from the last plane of the previous pass, which the last
//     warp left in a global buffer);
//   * the warps run in lockstep chunks of K steps with one CTA barrier per
//     chunk; warp (wy, h) runs (32 + K) wy + K h steps behind warp (0, 0),
//     so every value a warp reads was written in an earlier chunk, and the
//     rings are deep enough that no slot is rewritten before it is read;
//   * boundary values come from the per-cell record (face base and the
//     sides that are boundary faces: domain walls and faces next to void
//     cells), read four steps ahead; the source, the boundary face values
//     and the previous pass's plane are read two steps ahead, so the step
//     itself only waits on on-chip data.  The per-cell record, source and
//     source profile are read from diagonal-skewed copies (SkewLayout), in
//     which the 32 cells of a warp's step are consecutive: one coalesced
//     segment per warp and array instead of 32 scattered rows;
//   * specularly reflecting domain faces (Methods, Boundary conditions): the
//     inflow of direction d through such a face is the previous iterate's
//     value of the mirror direction of d in the same cell, read per
//     direction in the warp steps that meet one (rare, like the x and z
//     boundaries); a cell whose downwind side is specular stores its values
//     under the mirror directions for the next iterate.  The adjoint keeps
//     mu = w nu in those arrays (the general kernel's convention; its
//     transposed coupling is the same rule, the mirror swap preserving
//     |s_a|);
//   * forward and adjoint run the same recurrence: the adjoint unknown mu_d
//     of the transposed system (Eq. adjoint) scaled by 1 / w_d obeys the
//     forward recurrence with the adjoint source and boundary values, and
//     sum_d mu_d = sum_d w_d nu_d; only the face-sum weights differ
//     (forward w_d |s_d,a|, adjoint a_d w_d);
//   * the per-cell weighted sums of a step sit on a diagonal; each warp
//     parks them in a shared-memory tile [row][33] of its last 32 steps and
//     writes 4 of the 32 rows per chunk, each row's last 32 steps being 32
//     consecutive cells of that row (coalesced stores, and the same work for
//     every warp in every chunk, which the lockstep barrier rewards).
#pragma once

#include <stdint.h>

#include "bte_internal.cuh"
#include "finalize.cuh"
#include "tma.cuh"

namespace bte {

constexpr int kP3MaxThreads = 512;
constexpr int kP3RZ = 2 * kPipe3Chunk;  // z-ring depth (virtual columns)
constexpr int kP3RY = 4 * kPipe3Chunk;  // y-ring depth

__host__ __device__ constexpr int p3_round4(int n) { return (n + 3) & ~3; }


// DW consecutive values (16-byte aligned groups of 4, 8-byte aligned pairs)
// to and from registers; CG = through L2 only (data written in this launch)
template <bool CG>
__device__ __forceinline__ void p3_ld4(const float *p, float *v) {
    const float4 x = CG ? __ldcg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
template <bool CG>
__device__ __forceinline__ void p3_ld4(const double *p, double *v) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 x = CG ? __ldcg(q) : q[0];
    const double2 y = CG ? __ldcg(q + 1) : q[1];
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
}
template <bool CG>
__device__ __forceinline__ void p3_ld2(const float *p, float *v) {
    const float2 x = CG ? __ldcg(reinterpret_cast<const float2 *>(p)) : *reinterpret_cast<const float2 *>(p);
    v[0] = x.x;
    v[1] = x.y;
}
template <bool CG>
__device__ __forceinline__ void p3_ld2(const double *p, double *v) {
    const double2 x = CG ? __ldcg(reinterpret_cast<const double2 *>(p)) : *reinterpret_cast<const double2 *>(p);
    v[0] = x.x;
    v[1] = x.y;
}
template <int DW, bool CG = false, typename real>
__device__ __forceinline__ void p3_load(const real *p, real (&v)[DW]) {
    if constexpr (DW % 4 == 0) {
#pragma unroll
        for (int q = 0; q < DW; q += 4) p3_ld4<CG>(p + q, v + q);
    } else if constexpr (DW == 2) {
        p3_ld2<CG>(p, v);
    } else {
        v[0] = CG ? __ldcg(p) : p[0];
    }
}
__device__ __forceinline__ void p3_st4(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void p3_st4(double *p, const double *v) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void p3_st2(float *p, const float *v) { *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]); }
__device__ __forceinline__ void p3_st2(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
template <int DW, typename real>
__device__ __forceinline__ void p3_store(real *p, const real (&v)[DW]) {
    if constexpr (DW % 4 == 0) {
#pragma unroll
        for (int q = 0; q < DW; q += 4) p3_st4(p + q, v + q);
    } else if constexpr (DW == 2) {
        p3_st2(p, v);
    } else {
        p[0] = v[0];
    }
}

// Asynchronous global -> shared copy of DW consecutive values (cp.async in
// 16-byte pieces, through L2 only: the source was written by this CTA in this
// launch); a copy shorter than 16 bytes goes through registers instead.
// The caller commits the group.
template <int DW, typename real>
__device__ __forceinline__ void p3_cp_async(real *dst, const real *src) {
    constexpr int kBytes = DW * (int)sizeof(real);
    if constexpr (kBytes % 16 == 0) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
        const char *g = reinterpret_cast<const char *>(src);
#pragma unroll
        for (int o = 0; o < kBytes; o += 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + o), "l"(g + o) : "memory");
    } else {
        real v[DW];
        p3_load<DW, true>(src, v);
        p3_store<DW>(dst, v);
    }
}
__device__ __forceinline__ void p3_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void p3_cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// compile-time selector of a variant of the per-step direction loop
template <int V>
struct P3Kind {
    static constexpr int value = V;
};

// Shared-memory carve-up, in elements of real (X: the variant, bit 0 =
// specular faces, bit 1 = an extra per-direction source).
struct P3Smem {
    int invd, srck, fw, zr, yr, tile, mir, iw, spec, xs, total;
};
__host__ __device__ inline P3Smem p3_smem(int R, int WY, int H, int DW, int X) {
    const bool spec = (X & 1) != 0, xsrc = (X & 2) != 0;
    const int NW = WY * H;
    P3Smem s;
    s.invd = 0;                                        // [R][DW] 1 / diagonal
    s.srck = s.invd + p3_round4(R * DW);               // [R] source factor
    s.fw = s.srck + p3_round4(R);                      // [3][DW] face-sum weights
    s.zr = s.fw + p3_round4(3 * DW);                   // [NW][RZ][32][DW] z rings
    s.yr = s.zr + NW * kP3RZ * 32 * DW;                // [NW + 2][RY][DW] y rings
    s.tile = s.yr + (NW + 2) * kP3RY * DW;             // [NW][32][33] partial-sum tiles
    s.mir = s.tile + NW * 32 * 33;                     // [3][DW] mirror directions (int)
    s.iw = s.mir + (spec ? p3_round4(3 * DW) : 0);     // [DW] 1 / w
    s.spec = s.iw + (spec ? p3_round4(DW) : 0);        // [NW][32][DW] specular inflow of the next step
    s.xs = s.spec + (spec ? NW * 32 * DW : 0);         // [NW][32][DW] extra source of the next step
    s.total = s.xs + (xsrc ? NW * 32 * DW : 0);
    return s;
}

// Asynchronous global -> shared copy of DW consecutive values in pieces of
// 16 bytes where `wide` says both addresses are aligned to them, else of one
// value each.  The caller commits the group.
template <int DW, typename real>
__device__ __forceinline__ void p3_cp_async_row(real *dst, const real *src, bool wide) {
    constexpr int kBytes = DW * (int)sizeof(real);
    constexpr int kOne = (int)sizeof(real);
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *g = reinterpret_cast<const char *>(src);
    if (kBytes % 16 == 0 && wide) {
#pragma unroll
        for (int o = 0; o < kBytes; o += 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + o), "l"(g + o) : "memory");
    } else {
#pragma unroll
        for (int o = 0; o < kBytes; o += kOne)
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d + o), "l"(g + o), "n"(kOne) : "memory");
    }
}

// EM: 0 = a source-iteration sweep; 1 = the same that also writes e; 2 =
// the gradient form of the final adjoint pass: the per-cell sums become
// sum_d w_d (nu_d - Theta)(e_d - e0) = sum_d (mu_d - w_d Theta)(e_d - e0),
// e the forward solution's values and e0 = C_b (T - T_ref)/(4 pi) (the
// partials of dJ/dtau), and no face sums are formed
template <typename real, int DW, bool PHI, int EM, bool ZROWS, int X>
__global__ void __launch_bounds__(kP3MaxThreads, 1)
sweep3dp_kernel(const __grid_constant__ Sweep3DParams<real> P) {
    // X bit 0: specular faces; bit 1: the extra source xscale * xsrc[c][b][d]
    // of forward sweeps (implicit-Euler time steps: e of the previous step
    // over dt)
    constexpr bool SPEC = (X & 1) != 0, XS = (X & 2) != 0;
    constexpr bool RC = EM != 0 || XS;   // the cell index of every step is tracked
    constexpr int K = kPipe3Chunk, RZ = kP3RZ, RY = kP3RY;
    static_assert(K == 4, "the prefetch slots assume four steps per chunk");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_stop;

    const int s = blockIdx.x;
    const int b = blockIdx.y + P.b0;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int WY = P.WY, H = P.H;
    const int nx = P.nx, R = P.R;
    // axis roles: x is marched; the lanes hold rows along a1 (1 = y, 2 = z),
    // the warps along z of the CTA hold planes along a2 (the other one)
    constexpr int a1 = ZROWS ? 2 : 1, a2 = 3 - a1;
    const int n1 = a1 == 1 ? P.ny : P.nz;          // rows
    const int n2 = a1 == 1 ? P.nz : P.ny;          // planes
    const int s1 = a1 == 1 ? nx : nx * P.ny;       // cell stride of the next row
    const int s2 = a1 == 1 ? nx * P.ny : nx;       // cell stride of the next plane
    const P3Smem L = p3_smem(R, WY, H, DW, X);
    real *sm = reinterpret_cast<real *>(smem_raw);
    real *s_invd = sm + L.invd;
    real *s_srck = sm + L.srck;
    real *s_fw = sm + L.fw;
    const real *s_iw = sm + L.iw;   // (specular faces) 1 / w of the subset's directions

    // the next kernel may be launched now (it waits for this grid); all
    // reads below see what the previous kernel wrote
    pdl_launch_dependents();
    pdl_wait();
    // one thread reads the stop flag, so every warp of the CTA decides alike
    if (threadIdx.x == 0) s_stop = (P.done != nullptr && *((volatile const int *)P.done) != 0) ? 1 : 0;
    __syncthreads();
    if (s_stop) return;

    const Subset sub = P.sub[s];
    const int d0 = sub.d0;
    const int ndir = min(DW, sub.cnt);
    // a full subset at an aligned offset is written with vector stores (the
    // element count of one vector store of p3_store must divide D and d0)
    constexpr int kVA = sizeof(real) == 4 ? (DW >= 4 ? 4 : DW) : (DW >= 2 ? 2 : 1);
    const bool vec_e = ndir == DW && (P.D % kVA) == 0 && (d0 % kVA) == 0;
    const bool adj = P.adj != 0;
    for (int q = threadIdx.x; q < R * DW; q += blockDim.x) {
        const int r = q / DW, dd = q - r * DW;
        s_invd[q] = dd < ndir ? P.invdiag[((long long)r * P.B + b) * P.D + d0 + dd] : real(0);
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x) s_srck[r] = P.srck[r * P.B + b];
    {
        // the bottom row warps' y ring (never written) and the first plane
        // warps' z rings (filled from the previous pass from the second pass
        // on) start as zeros
        const int NW = WY * H;
        real *yz = sm + L.yr + NW * RY * DW;
        for (int q = threadIdx.x; q < RY * DW; q += blockDim.x) yz[q] = real(0);
        real *zz = sm + L.zr;
        for (int q = threadIdx.x; q < WY * RZ * 32 * DW; q += blockDim.x) zz[q] = real(0);
    }
    if constexpr (SPEC) {
        // mirror directions of the subset, per physical axis
        int *mir = reinterpret_cast<int *>(sm + L.mir);
        for (int q = threadIdx.x; q < 3 * DW; q += blockDim.x) {
            const int a = q / DW, dd = q - a * DW;
            mir[q] = dd < ndir ? P.mirror[a * P.D + d0 + dd] : 0;
        }
        real *iw = sm + L.iw;
        for (int dd = threadIdx.x; dd < DW; dd += blockDim.x)
            iw[dd] = dd < ndir ? real(1) / P.coef[((long long)b * P.D + d0 + dd) * 8 + 3] : real(0);
    }
    for (int q = threadIdx.x; q < 3 * DW; q += blockDim.x) {
        const int a = q / DW, dd = q - a * DW;
        real v = real(0);
        if (dd < ndir) {
            const real *cf = P.coef + ((long long)b * P.D + d0 + dd) * 8;
            // forward: w |s_a| (energy leaving); adjoint: a_a w (nu = mu / w)
            v = adj ? cf[a] * cf[3] : cf[4 + a];
        }
        s_fw[q] = v;
    }
    // deferred finalization of the previous iteration (CTA (0, 0)); nothing
    // in this kernel depends on it: a stop found here ends the solve at the
    // update that follows
    if (s == 0 && b == 0 && warp == 0 && P.fin.pending != nullptr && *((volatile const int *)P.fin.pending) != 0) {
        double eps, tmx, tss;
        fin_reduce(P.fin, eps, tmx, tss);
        if (lane == 0) fin_record(P.fin, eps, tmx, tss);
    }
    __syncthreads();

    // ---- this warp: rows 32 wy .. 32 wy + 31 of planes h + H m ----
    const int wy = warp % WY;
    const int h = warp / WY;
    const bool negx = sub.neg & 1, neg1 = (sub.neg >> a1) & 1, neg2 = (sub.neg >> a2) & 1;
    const int up_x = negx ? 1 : 0, up_1 = 2 * a1 + (neg1 ? 1 : 0), up_2 = 2 * a2 + (neg2 ? 1 : 0);
    const unsigned dn_mask = (1u << (up_x ^ 1)) | (1u << (up_1 ^ 1)) | (1u << (up_2 ^ 1));
    const unsigned below_x = (1u << up_x) - 1u, below_1 = (1u << up_1) - 1u, below_2 = (1u << up_2) - 1u;
    real ax[DW], ay[DW], az[DW], w[DW];
#pragma unroll
    for (int dd = 0; dd < DW; ++dd) {
        if (dd < ndir) {
            const real *cf = P.coef + ((long long)b * P.D + d0 + dd) * 8;
            ax[dd] = cf[0];
            ay[dd] = cf[a1];   // coefficient of the row (lane) axis
            az[dd] = cf[a2];   // coefficient of the plane axis
            w[dd] = cf[3];
        } else {
            ax[dd] = ay[dd] = az[dd] = w[dd] = real(0);
        }
    }
    const real qb = PHI ? P.qb[b] : real(0);
    const real cb4pi = (EM == 2) ? P.cb4pi[b] : real(0);
    const unsigned iso_skip = P.iso_fsum ? 0u : 63u;
    // the sides of the specular faces a cell's inflow comes through (none
    // without specular faces)
    const unsigned spec_up = SPEC ? ((1u << up_x) | (1u << up_1) | (1u << up_2)) : 0u;
    // 16-byte copies of the rows of DW directions where they are aligned (D
    // and d0)
    constexpr int kRowVec = 16 / (int)sizeof(real);
    const bool row_wide = (P.D % kRowVec) == 0 && (d0 % kRowVec) == 0;
    const real *einb = P.ein + (long long)b * P.F;
    const int j = 32 * wy + lane;
    const bool rowv = j < n1;
    const int Y = neg1 ? n1 - 1 - j : j;
    const int M = (n2 + H - 1) / H;        // passes
    const int Mh = (n2 - h + H - 1) / H;   // passes in which this warp's plane lies in the grid
    const int U = M * nx;                  // virtual columns of a lane
    const int n_loc = (U + 31 + 31) & ~31; // local steps (whole 32-step tiles)
    constexpr int Ly = 32 + K, Lz = K;     // lag of the next warp along y / z
    const int delta = wy * Ly + h * Lz;
    const int T = (WY - 1) * Ly + (H - 1) * Lz + n_loc;
    const int ld_wrap = WY * 32;
    const int sx = negx ? -1 : 1;          // dX / di
    const int sz = neg2 ? -1 : 1;          // dZ / dk
    const float inv_nx = 1.0f / (float)nx;
    // skewed inputs: the family of this octant (X + Y or X - Y constant
    // along a step); index of column i of pass m of this lane:
    //   sk0 + sx nyp i + sz H nd nyp m  (within a pass; see SkewLayout)
    // and a zero pad entry (2 fam) for the cells outside the grid
    const int fam = (negx != neg1) ? 1 : 0;
    const int sk_nd = P.skew.nd, sk_nyp = P.skew.nyp;
    const int sk_pad = 2 * (int)P.skew.fam;
    const int X0 = negx ? nx - 1 : 0;
    const int Zh = neg2 ? n2 - 1 - h : h;
    const int key0 = fam ? X0 + (n1 - 1 - Y) : X0 + Y;
    const int sk0 = (fam ? (int)P.skew.fam : 0) + (Zh * sk_nd + key0) * sk_nyp + Y;
    const int dsk = sx * sk_nyp;                                   // next column
    const int dsk_pass = (sz * H * sk_nd - sx * (nx - 1)) * sk_nyp; // column 0 of the next pass
    const bool wrap_rd = (h == 0) && M > 1;       // reads the previous pass's last plane
    const bool wrap_wr = (h == H - 1) && M > 1;   // writes this pass's last plane
    const bool feed_y = wy + 1 < WY;
    real *const part_b = P.part + ((long long)b * P.Spad + s) * P.N;
    real *const fs_sb = P.fsum + ((long long)s * P.B + b) * P.F;
    real *const wrap_c = (M > 1) ? P.wrap + ((long long)s * P.B + b) * (long long)nx * ld_wrap * DW : nullptr;
    real *const tile = sm + L.tile + warp * 32 * 33;
    real *const tile_l = tile + lane * 33;
    // z rings: slot (local step mod RZ) of this lane; the writer (warp below
    // in z) and the reader handle a given column at the same local step.
    // Warp w reads ring w and writes ring w + WY: the first plane warps read
    // rings they fill themselves from the wrap buffer (two steps ahead); the
    // last plane warps have no ring to write (their one predicated store is
    // all that differs; rings nobody reads would take the shared memory that
    // lets two CTAs of 8 warps share an SM).  y rings: warp w writes ring w for the warp above it in y (the top
    // row warps write ring NW + 1, read by nobody), the bottom row warps read
    // ring NW (zeros).
    real *const zr_out = sm + L.zr + (warp + WY) * RZ * 32 * DW + lane * DW;
    real *const zr_in = sm + L.zr + warp * RZ * 32 * DW + lane * DW;
    real *const yr_out = sm + L.yr + (feed_y ? warp : WY * H + 1) * RY * DW;
    const real *const yr_in = sm + L.yr + (wy > 0 ? warp - 1 : WY * H) * RY * DW;

    // record slots (local step mod 4) and data slots (local step mod 2)
    constexpr bool STORE_E = EM == 1, GRAD = EM == 2;
    int rs[4], rc[RC ? 4 : 1], rx[4], ry[4], riw[4];
    real dt[2], dp[2], dex[2], dey[2], dez[2];
    real dtf[GRAD ? 2 : 1], dev[GRAD ? 2 : 1][DW];   // gradient form: forward T - T_ref and e
    // tracker of the record read next (local step tau + 4): its virtual
    // column uf (= ui + nx um, column ui of pass um), the steps cnt until it
    // leaves the current pass, and its skewed index (valid once uf >= 0)
    int uf = -lane, cnt = nx + lane, um = 0;
    int sk_t = sk0 - lane * dsk;
    const unsigned Uh = (unsigned)(Mh * nx);        // columns whose plane lies in the grid
    const unsigned Uw = (unsigned)((M - 1) * nx);   // columns of passes that have a next pass
    auto fetch_record = [&](int q) {
        const bool v = rowv && (unsigned)uf < Uh;
        const int sk = v ? sk_t : sk_pad;
        rs[q] = sk;
        const int ui = nx - cnt;
        if (RC) {
            const int Xc = negx ? nx - 1 - ui : ui;
            const int k = h + H * um;
            const int Z = neg2 ? n2 - 1 - k : k;
            rc[RC ? q : 0] = v ? Xc + s1 * Y + s2 * Z : -1;
        }
        // wrap buffer column: read by the first warp of a pass (the value is
        // used only past the first pass), written by the last one
        if (wrap_wr)
            riw[q] = (v && (unsigned)uf < Uw) ? ui : -1;
        else if (wrap_rd)
            riw[q] = max(ui, 0);
        const int2 ci = __ldg(P.cell + sk);
        rx[q] = ci.x;
        ry[q] = ci.y;
        ++uf;
        sk_t += dsk;
        if (--cnt == 0) {
            cnt = nx;
            ++um;
            sk_t += dsk_pass - dsk;
        }
    };
    // source, boundary values and wrapped plane of the cell in record slot q,
    // used at local step tt; every load is unconditional (a side without a
    // boundary reads face 0, the same address for every such lane; a cell
    // outside the grid reads the zero pad entry) and the step selects
    auto fetch_data = [&](int q, int slot, int tt) {
        const int sk = rs[q];
        const int fb = rx[q], fl = ry[q];
        const unsigned bm = ((unsigned)fl >> kSideShift) & 63u;
        dt[slot] = __ldg(P.tsrc + sk);
        if (PHI) dp[slot] = __ldg(P.phi + sk);
        const int fx = ((bm >> up_x) & 1u) ? fb + __popc(bm & below_x) : 0;
        const int fy = ((bm >> up_1) & 1u) ? fb + __popc(bm & below_1) : 0;
        const int fz = ((bm >> up_2) & 1u) ? fb + __popc(bm & below_2) : 0;
        dex[slot] = __ldg(einb + fx);
        dey[slot] = __ldg(einb + fy);
        dez[slot] = __ldg(einb + fz);
        if constexpr (GRAD) {
            // the forward state of this cell (a cell outside the grid reads
            // cell 0's, which no solid cell uses)
            dtf[slot] = __ldg(P.tfwd + sk);
            const real *ep = P.e + ((long long)max(rc[q], 0) * P.B + b) * P.D + d0;
            if (vec_e) {
                p3_load<DW>(ep, dev[slot]);
            } else {
#pragma unroll
                for (int dd = 0; dd < DW; ++dd) dev[slot][dd] = dd < ndir ? ep[dd] : real(0);
            }
        }
        if (wrap_rd) {
            // the previous pass's last plane (written by this CTA earlier in
            // this launch) into this warp's own z ring slot of step tt
            p3_cp_async<DW>(zr_in + (tt & (RZ - 1)) * 32 * DW, wrap_c + ((long long)riw[q] * ld_wrap + j) * DW);
            p3_cp_commit();
        }
    };
    // before its rows enter the grid a lane's registers hold zeros; the first
    // cell of every row has its x-upwind side marked as a boundary, and a cell
    // next to a void or outside cell reads the boundary value instead of it
    real old[DW];
#pragma unroll
    for (int dd = 0; dd < DW; ++dd) old[dd] = real(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) fetch_record(q);
    fetch_data(0, 0, 0);
    fetch_data(1, 1, 1);
    // specular faces: the inflow of the next step's cell through its one
    // specular upwind face is copied into this warp's shared-memory slot a
    // step ahead (spec_side: that face's side, -1 none, -2 several: a domain
    // edge, whose rows the step reads itself)
    // The extra source of the next step's cell comes the same way (a cell
    // outside the grid or void keeps the slot's previous finite values).
    int spec_side = -1;
    real *const spec_slot = sm + L.spec + (warp * 32 + lane) * DW;
    real *const xs_slot = sm + L.xs + (warp * 32 + lane) * DW;
    if constexpr (XS) {
#pragma unroll
        for (int dd = 0; dd < DW; ++dd) xs_slot[dd] = real(0);
    }
    auto fetch_next = [&](int q) {
        if constexpr (SPEC) {
            const int fb1 = rx[q], fl1 = ry[q];
            const unsigned sb = ((unsigned)fl1 >> kSpecShift) & spec_up;
            spec_side = -1;
            if (sb != 0u) {
                if ((sb & (sb - 1u)) == 0u) {
                    spec_side = __ffs((int)sb) - 1;
                    const int off = (b * P.Fs + P.sidx[face_of(fb1, fl1, spec_side)]) * P.D + d0;
                    p3_cp_async_row<DW>(spec_slot, P.spec_in + off, row_wide);
                } else {
                    spec_side = -2;
                }
            }
        }
        if constexpr (XS) {
            const int c1 = rc[q];
            if (c1 >= 0) p3_cp_async_row<DW>(xs_slot, P.xsrc + ((long long)c1 * P.B + b) * P.D + d0, row_wide);
        }
        p3_cp_commit();
    };
    if constexpr (SPEC || XS) fetch_next(0);

    for (int t0 = 0; t0 < T; t0 += K) {
        const int tau0 = t0 - delta;
        if (tau0 >= 0 && tau0 < n_loc) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int tau = tau0 + k;
                // this step's cell (record read four steps ago, data two)
                const int c = RC ? rc[RC ? k : 0] : -1;
                const int fb = rx[k], fl = ry[k], iw = riw[k];
                const real tsv = dt[k & 1];
                const real phv = PHI ? dp[k & 1] : real(0);
                const real Ex = dex[k & 1], Ey = dey[k & 1], Ez = dez[k & 1];
                // gradient form: e - e0 of the forward solution in this cell
                real gde[GRAD ? DW : 1];
                if constexpr (GRAD) {
                    const real e0 = cb4pi * dtf[k & 1];
#pragma unroll
                    for (int dd = 0; dd < DW; ++dd) gde[dd] = dev[k & 1][dd] - e0;
                }
                // this step's z and y inputs (the first plane warps' own z
                // ring slot was filled by the copy issued two steps ago)
                const int zslot = (tau & (RZ - 1)) * 32 * DW;
                real zin[DW], yin[DW];
                if constexpr (SPEC || XS)
                    p3_cp_wait<0>();   // this step's slots (and the ring slots) are in
                else if (wrap_rd)
                    p3_cp_wait<1>();
                p3_load<DW>(zr_in + zslot, zin);
                p3_load<DW>(yr_in + (tau & (RY - 1)) * DW, yin);  // lane 0: u == tau
                // reads for later steps
                fetch_record(k);
                fetch_data((k + 2) & 3, k & 1, tau + 2);

                const int region = fl & kRegionMask;
                const bool act = region != 0;   // solid cell of the grid
                const unsigned bm = ((unsigned)fl >> kSideShift) & 63u;
                const bool bx = (bm >> up_x) & 1u;
                const bool by = (bm >> up_1) & 1u;
                const bool bz = (bm >> up_2) & 1u;
                const int r = act ? region - 1 : 0;
                real base = tsv * s_srck[r];
                if (PHI) base += phv * qb;
                real invd[DW];
                p3_load<DW>(s_invd + r * DW, invd);
                // cells that are not solid cells of the grid update garbage
                // that no solid cell reads (their downwind neighbours take
                // boundary values) and that the update kernel ignores
                real acc = real(0);
                // the directions of this step; the variant: 0 = only row-axis
                // boundaries, 1 = also x and z boundaries, 2 = also specular
                // faces (the per-direction inflow: the previous iterate's
                // value of the mirror direction, forward e; adjoint mu = w nu,
                // taken as nu; spx, spy, spz: offsets of the inflow rows in
                // spec_in, -1 where the side is not specular)
                int spx = -1, spy = -1, spz = -1;
                const int ssd = SPEC ? spec_side : -1;   // the side of this step's slot
                auto dirs = [&](auto kind) {
                    constexpr int V = decltype(kind)::value;
#pragma unroll
                    for (int dd = 0; dd < DW; ++dd) {
                        real vy = __shfl_up_sync(0xffffffffu, old[dd], 1);
                        if (lane == 0) vy = yin[dd];
                        real vx = old[dd], vz = zin[dd];
                        if constexpr (V >= 1) {
                            vx = bx ? Ex : vx;
                            vz = bz ? Ez : vz;
                        }
                        vy = by ? Ey : vy;
                        if constexpr (V == 2) {
                            if (dd < ndir) {
                                const real sc = adj ? s_iw[dd] : real(1);
                                const real sv = spec_slot[dd] * sc;
                                vx = ssd == up_x ? sv : vx;
                                vy = ssd == up_1 ? sv : vy;
                                vz = ssd == up_2 ? sv : vz;
                                if (spx >= 0) vx = P.spec_in[spx + dd] * sc;
                                if (spy >= 0) vy = P.spec_in[spy + dd] * sc;
                                if (spz >= 0) vz = P.spec_in[spz + dd] * sc;
                            }
                        }
                        real r0;
                        if constexpr (XS) {
                            r0 = fma(P.xscale, xs_slot[dd], base);
                            r0 = fma(ax[dd], vx, r0);
                        } else {
                            r0 = fma(ax[dd], vx, base);
                        }
                        r0 = fma(ay[dd], vy, r0);
                        r0 = fma(az[dd], vz, r0);
                        const real en = r0 * invd[dd];
                        old[dd] = en;
                        if constexpr (GRAD)
                            acc = fma(w[dd] * (en - tsv), gde[dd], acc);
                        else
                            acc = fma(w[dd], en, acc);
                    }
                };
                // x and z boundaries are met in few warp steps (a row's first
                // column, a pass's first plane, void neighbours), specular
                // faces in fewer: their selects and loads only run when a lane
                // of the warp needs them
                const unsigned sup = SPEC ? ((unsigned)fl >> kSpecShift) & spec_up : 0u;
                if (__any_sync(0xffffffffu, bx || bz || sup != 0u)) {
                    if (SPEC && __any_sync(0xffffffffu, sup != 0u)) {
                        if (ssd == -2) {
                            // a domain edge: the rows of all its specular
                            // sides (B Fs D < 2^31: checked on the host)
                            const int rb = b * P.Fs;
                            if ((sup >> up_x) & 1u) spx = (rb + P.sidx[face_of(fb, fl, up_x)]) * P.D + d0;
                            if ((sup >> up_1) & 1u) spy = (rb + P.sidx[face_of(fb, fl, up_1)]) * P.D + d0;
                            if ((sup >> up_2) & 1u) spz = (rb + P.sidx[face_of(fb, fl, up_2)]) * P.D + d0;
                        }
                        dirs(P3Kind<2>{});
                    } else {
                        dirs(P3Kind<1>{});
                    }
                } else {
                    dirs(P3Kind<0>{});
                }
                if constexpr (SPEC || XS) fetch_next((k + 1) & 3);
                tile_l[tau & 31] = acc;
                if (h + 1 < H) p3_store<DW>(zr_out + zslot, old);
                if (lane == 31) p3_store<DW>(yr_out + ((tau - 31) & (RY - 1)) * DW, old);
                if (wrap_wr && iw >= 0) p3_store<DW>(wrap_c + ((long long)iw * ld_wrap + j) * DW, old);
                // face sums at the boundary sides the traversal leaves by
                // (at isothermal domain faces only when asked: the iterations
                // never read them there, the final adjoint pass does)
                const unsigned fsm = bm & dn_mask & ~(((unsigned)fl >> kIsoShift) & iso_skip);
                if (!GRAD && act && fsm) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int dn = (a == 0 ? up_x : (a == 1 ? up_1 : up_2)) ^ 1;
                        const int pa = a == 0 ? 0 : (a == 1 ? a1 : a2);   // physical axis
                        if (!((fsm >> dn) & 1u)) continue;
                        const int f = face_of(fb, fl, dn);
                        if (SPEC && ((((unsigned)fl >> kSpecShift) >> dn) & 1u)) {
                            // a specular face: the next iterate's inflow of
                            // the mirror directions (adjoint: mu = w nu)
                            if (P.spec_out != nullptr) {
                                real *so = P.spec_out + (b * P.Fs + P.sidx[f]) * P.D;
                                const int *mr = reinterpret_cast<const int *>(sm + L.mir) + pa * DW;
#pragma unroll
                                for (int dd = 0; dd < DW; ++dd)
                                    if (dd < ndir) so[mr[dd]] = adj ? old[dd] * w[dd] : old[dd];
                            }
                            continue;
                        }
                        real fw[DW];
                        p3_load<DW>(s_fw + pa * DW, fw);
                        real fs = real(0);
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd) fs = fma(fw[dd], old[dd], fs);
                        fs_sb[f] = fs;
                    }
                }
                if (STORE_E && act && c >= 0) {
                    real *ep = P.e + ((long long)c * P.B + b) * P.D + d0;
                    real ev[DW];
#pragma unroll
                    for (int dd = 0; dd < DW; ++dd) ev[dd] = adj ? old[dd] * w[dd] : old[dd];
                    if (vec_e) {
                        p3_store<DW>(ep, ev);   // DW consecutive values, aligned: vector stores
                    } else {
#pragma unroll
                        for (int dd = 0; dd < DW; ++dd)
                            if (dd < ndir) ep[dd] = ev[dd];
                    }
                }
            }
            {
                // write 4 of the 32 rows of the sum tile (rows 4 g .. 4 g + 3,
                // g = this chunk's index mod 8): every row is written once per
                // 32 steps, covering its last 32 steps = 32 consecutive virtual
                // columns, and every warp does the same work in every chunk.
                // Lane q writes the column of the step whose tile slot is q.
                __syncwarp();
                const int te = tau0 + K - 1;
                const int g = (te >> 2) & 7;
                const int tq = te - ((te - lane) & 31);
                const int u_top = tq - 4 * g;
                // u_top / nx without an integer division (exact for the
                // column counts of a grid that fits in memory)
                int m = __float2int_rd(((float)u_top + 0.5f) * inv_nx);
                m -= (m * nx > u_top) ? 1 : 0;
                m += ((m + 1) * nx <= u_top) ? 1 : 0;
                int i = u_top - m * nx;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int rr = 4 * g + q;
                    if (q > 0 && --i < 0) {
                        i += nx;
                        --m;
                    }
                    const int k = h + H * m;
                    if (m >= 0 && k < n2 && 32 * wy + rr < n1) {
                        const int X = negx ? nx - 1 - i : i;
                        const int jr = 32 * wy + rr;
                        const int Yr = neg1 ? n1 - 1 - jr : jr;
                        const int Z = neg2 ? n2 - 1 - k : k;
                        part_b[X + s1 * Yr + s2 * Z] = tile[rr * 33 + lane];
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    if (SPEC || XS || wrap_rd) p3_cp_wait<0>();   // no copy outlives the kernel
}

template <typename real>
size_t sweep3dp_smem_bytes(int R, int WY, int H, int dw, int x) {
    return (size_t)p3_smem(R, WY, H, dw, x).total * sizeof(real);
}

template <typename real, int DW, bool PHI, int EM, bool ZROWS, int X>
cudaError_t launch_sweep3dp_v(const Sweep3DParams<real> &p, cudaStream_t st) {
    const int threads = p.WY * p.H * 32;
    if (p.H < 1 || p.WY < 1 || threads > kP3MaxThreads) return cudaErrorInvalidConfiguration;
    const size_t smem = sweep3dp_smem_bytes<real>(p.R, p.WY, p.H, DW, X);
    auto kern = sweep3dp_kernel<real, DW, PHI, EM, ZROWS, X>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(kern, dim3(p.S, p.nb ? p.nb : p.B), dim3(threads), smem, st, p);
}

// the source-profile term only in forward sweeps with a source; e only when
// asked; the gradient form only in adjoint sweeps
template <typename real, int DW, bool ZROWS, int X>
cudaError_t launch_sweep3dp_z(const Sweep3DParams<real> &p, cudaStream_t st) {
    const bool phi = !p.adj && p.phi != nullptr;
    if (p.grad) {
        if (!p.adj || p.store_e || !p.tfwd || !p.cb4pi || !p.e) return cudaErrorInvalidValue;
        if constexpr ((X & 2) != 0) {
            return cudaErrorInvalidValue;   // the extra source belongs to forward sweeps
        } else {
            return launch_sweep3dp_v<real, DW, false, 2, ZROWS, X>(p, st);
        }
    }
    if (p.store_e)
        return phi ? launch_sweep3dp_v<real, DW, true, 1, ZROWS, X>(p, st)
                   : launch_sweep3dp_v<real, DW, false, 1, ZROWS, X>(p, st);
    return phi ? launch_sweep3dp_v<real, DW, true, 0, ZROWS, X>(p, st)
               : launch_sweep3dp_v<real, DW, false, 0, ZROWS, X>(p, st);
}

// rows along y or along z
// (X: the variant: bit 0 for a problem with specular faces, bit 1 for a
// sweep with an extra source)
template <typename real, int DW, int X>
cudaError_t launch_sweep3dp_t(const Sweep3DParams<real> &p, cudaStream_t st) {
    if (((X & 1) != 0) != (p.Fs > 0) || ((X & 1) && !p.spec_in)) return cudaErrorInvalidValue;
    if (((X & 2) != 0) != (p.xsrc != nullptr) || ((X & 2) && p.adj)) return cudaErrorInvalidValue;
    if (p.lane_axis == 1) return launch_sweep3dp_z<real, DW, false, X>(p, st);
    if (p.lane_axis == 2) return launch_sweep3dp_z<real, DW, true, X>(p, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace bte
