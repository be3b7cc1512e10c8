// FP64 reductions between sweeps.
//
// Forward (Eq. updatee0_t): T_c = T_ref + sum_b (1/tau_cb) sum_s part[s][b][c] / K_c,
// K_c = sum_b C_b/tau_cb, where part[s][b][c] = sum over the subset's
// directions of w_d (e_cbd - C_b T_ref/(4 pi)) from the sweep (FP32 inside a
// subset, FP64 from here on).  Diffuse faces get the next inflow
// e_in = sum_{s.n>0} w |s.n| e / sum_{s.n<0} w |s.n| (diffusely reflecting
// boundary, quadrature-consistent normaliser).  The convergence measure is
// eps_T = sqrt(mean (T_new - T_old)^2) / max T_new (Methods, step 4).
//
// Adjoint: Theta_c = (dJ/dT_c + sum_b C_b/(4 pi tau_cb) sum_d mu_cbd) / K_c and
// the diffuse-face adjoint value M' = (sum over entering directions of
// a_d mu_d) h / (v_b N_side); the stop measure is the relative RMS change of
// Theta.
//
// Reductions over blocks are deterministic: every block writes its partial,
// the last block to finish (ticket counter) combines them in block order.
#include <math.h>

#include "bte_internal.cuh"
#include "finalize.cuh"
#include "tma.cuh"

namespace bte {

constexpr int kUpdThreads = 256;

// Sum of the S partial sets of one (band, cell); sets are N apart
// ([B][Spad][N] layout), so a warp's loads of one set are coalesced; eight
// independent loads are in flight, summed in a fixed order in the sweep
// precision.
// value of cell c into both families of a skewed field
template <typename T>
__device__ __forceinline__ void skew_store(const SkewLayout &L, long long c, T v, T *dst) {
    const long long row = c / L.nx;
    const int X = (int)(c - row * L.nx);
    const int Y = (int)(row % L.ny);
    const int Z = (int)(row / L.ny);
    const int R = L.a1 == 1 ? Y : Z;   // row coordinate
    const int P = L.a1 == 1 ? Z : Y;   // plane coordinate
    dst[skew_index(L, 0, X, R, P)] = v;
    dst[skew_index(L, 1, X, R, P)] = v;
}

// The sum over the S partial sets of one (band, cell): sets are N apart
// ([B][Spad][N] layout), taken in batches of eight, each batch summed as a
// fixed tree and added to the running sum, in the sweep precision.  Both cell
// paths below form every cell's sum in exactly this order.
template <typename real>
__device__ __forceinline__ real tree8(const real (&a)[8]) {
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}
template <typename real>
__device__ __forceinline__ real sum_sets(const real *pp, int S, long long N) {
    real sum = real(0);
    for (int s = 0; s < S; s += 8) {
        real a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = (s + q < S) ? __ldcg(pp + (long long)(s + q) * N) : real(0);
        sum += tree8(a);
    }
    return sum;
}

// Per cell, the update combines its bands in a fixed order: band b belongs to
// slot b mod 8, a slot accumulates S_b times the band weight of the cell's
// region in increasing b (fma chain, sweep precision), the eight slot sums
// are added in slot order (sweep precision), and only that total is taken to
// FP64: T is held as the deviation from T_ref, so the rounding of the band
// sums is far below the resolution of T, while T itself, the residual and
// every reduction across cells are FP64 (a warp-wide FP64 operation is slow
// on this GPU).  Face blocks come first; then the cell blocks, in one of two
// forms with the same per-cell arithmetic:
//   * scalar: 32 cells x 8 band slots per block, thread (cell, slot);
//   * vector (cell counts that are multiples of 4, so every partial set
//     starts on a 16-byte boundary): 128 consecutive cells per block, warp w
//     holds slot w for all of them, lane l cells 4 l .. 4 l + 3 (one 16-byte
//     load per set and band), which keeps four times the bytes in flight per
//     load and per register.
constexpr int kCellsPerBlock = 32;
constexpr int kBandSlots = kUpdThreads / kCellsPerBlock;
constexpr int kVecCells = 128;

__host__ __device__ inline int update_cell_blocks(long long N, bool vec) {
    return vec ? (int)((N + kVecCells - 1) / kVecCells) : (int)((N + kCellsPerBlock - 1) / kCellsPerBlock);
}
__host__ __device__ inline int update_face_blocks(int F, int B) {
    return (int)(((long long)F * B + kUpdThreads - 1) / kUpdThreads);
}

// Face block `blk`: the next inflow of diffuse faces from the face sums.
template <typename real>
__device__ __forceinline__ void update_faces(const UpdateParams<real> &P, const int blk) {
    if (!P.ignore_done && *((volatile int *)P.done) != 0) return;
    const long long fb = (long long)blk * kUpdThreads + threadIdx.x;
    if (fb >= (long long)P.F * P.B) return;
    const int b = (int)(fb / P.F);
    const int f = (int)(fb % P.F);
    if (P.ub1 != 0 && (b < P.ub0 || b >= P.ub1)) return;   // sharded: another rank's band
    const int side = P.face_side[f];
    const int a = side >> 1;
    const bool plus = side & 1;
    if (P.face_kind[f] == 2) {
        // specular faces: the sweeps carry their per-direction inflow
        P.ein_out[fb] = (real)0;
        if (P.fsum_total) P.fsum_total[fb] = 0.0;
    } else if (P.face_kind[f] == 0 && !P.adjoint) {
        P.ein_out[fb] = P.ein_fixed[fb];
    } else {
        // sets leaving the cell through this face: those running upward on
        // axis a for a plus face, downward otherwise
        double sum = 0.0;
        for (int s = 0; s < P.Sf; ++s) {
            const bool neg = (P.sub[s].neg >> a) & 1;
            if (neg != plus) sum += (double)P.fsum[((long long)s * P.B + b) * P.F + f];
        }
        if (P.fsum_total) P.fsum_total[fb] = sum;
        P.ein_out[fb] = (P.face_kind[f] == 0) ? (real)0 : (real)(sum * P.side_scale[side * P.B + b]);
    }
}

// The new value of cell c (region r, slot total tot, old value x_old): writes
// it and returns its contribution to the residual (squared change, maximum).
template <typename real>
__device__ __forceinline__ void update_cell_value(const UpdateParams<real> &P, long long c, int r, double tot,
                                                  double x_old, double &ss, double &mx) {
    ss = 0.0;
    mx = -INFINITY;
    if (r != 0) {
        double xn;
        real xd;
        if (!P.adjoint) {
            const double dev = tot * P.Kinv[r - 1];
            xn = P.T_ref + dev;
            xd = (real)dev;
            mx = xn;
        } else {
            xn = (P.g[c] + tot) * P.Kinv[r - 1];
            xd = (real)xn;
            mx = fabs(xn);
        }
        P.xdev_out[c] = xd;
        if (P.xskew_out) skew_store(P.skew, c, xd, P.xskew_out);
        const double d = xn - x_old;
        ss = d * d;
        if (!isfinite(xn)) {
            // a NaN sum of squares and an infinite maximum: eps_T is NaN
            // whatever the other cells hold (fmax would skip a NaN maximum)
            ss = NAN;
            mx = INFINITY;
        }
        P.x_out[c] = xn;
    } else {
        P.x_out[c] = 0.0;
        P.xdev_out[c] = (real)0;
        if (P.xskew_out) skew_store(P.skew, c, (real)0, P.xskew_out);
    }
}

// Warp 0 of cell block cb, lane 0 holding the block's residual partials:
// record them, then either mark the iteration pending (deferred
// finalization) or take a ticket; the last block reduces every block's
// partials in a fixed order and records the iteration.
template <typename real>
__device__ __forceinline__ void update_block_tail(const UpdateParams<real> &P, int cb, int cell_blocks, double ss,
                                                  double mx, int it_prev, int *is_last) {
    const int lane = threadIdx.x & 31;
    if (P.defer) {
        // deferred finalization: the block partials and the pending mark;
        // the next pipeline sweep (or the finalize kernel) reduces them
        if (lane == 0) {
            P.blockpart[2 * cb] = ss;
            P.blockpart[2 * cb + 1] = mx;
            if (cb == 0) *P.fin.pending = 1;
        }
        return;
    }
    if (lane == 0) {
        P.blockpart[2 * cb] = ss;
        P.blockpart[2 * cb + 1] = mx;
        __threadfence();
        const unsigned ticket = atomicAdd(P.counter, 1u);
        *is_last = (ticket == (unsigned)cell_blocks - 1);
    }
    __syncwarp();
    if (!*is_last) return;
    __threadfence();
    // last cell block, warp 0: the deterministic reduction of the block
    // partials (fixed slices, fixed shuffle tree)
    double eps, tmx, tss;
    fin_reduce(P.fin, eps, tmx, tss);
    if (lane == 0) {
        *P.counter = 0u;
        const int it = it_prev;
        if (P.eps_hist && it < P.max_hist) P.eps_hist[it] = eps;
        P.last[0] = eps;
        P.last[1] = tmx;
        P.last[2] = tss;
        if (!P.ignore_done) {
            *P.iter = it + 1;
            const bool stop_now = !isfinite(eps) || (P.tol > 0.0 && eps < P.tol);
            if (!isfinite(eps)) atomicCAS(P.status, 0, 1);   // keeps an expired-wait status (2)
            if (stop_now) {
                *P.done = 1;
                if (P.batch_done) atomicAdd(P.batch_done, 1);
            }
        }
    }
}

// Scalar cell block cb: 32 cells x 8 band slots.
template <typename real>
__device__ __forceinline__ void update_cells(const UpdateParams<real> &P, const int cb, const int cell_blocks) {
    __shared__ real sband[kBandSlots][kCellsPerBlock];
    __shared__ int is_last;
    const int tx = threadIdx.x % kCellsPerBlock;
    const int ty = threadIdx.x / kCellsPerBlock;
    const long long c = (long long)cb * kCellsPerBlock + tx;
    const bool cin = c < P.N;
    const long long cc = cin ? c : 0;
    // everything this block reads is independent of everything else it reads:
    // issue the loads together (the stop flag, the cell's region, the old
    // value, both band slots' partial sets) before any of them is used
    const int stop = P.ignore_done ? 0 : *((volatile int *)P.done);
    const int it_prev = (threadIdx.x == 0) ? *P.iter : 0;  // only the last block's lane 0 uses it
    const int r = cin ? (P.cell[cc].y & kRegionMask) : 0;
    const double x_old = (ty == 0) ? P.x_in[cc] : 0.0;
    const int b0 = ty, b1 = ty + kBandSlots;
    const real *pp0 = P.part + (long long)b0 * P.Spad * P.N + cc;
    const real *pp1 = P.part + (long long)b1 * P.Spad * P.N + cc;
    real s0 = real(0), s1 = real(0);
    for (int s = 0; s < P.S; s += 8) {
        real a0[8], a1[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool in_s = s + q < P.S;
            a0[q] = (in_s && b0 < P.B) ? __ldcg(pp0 + (long long)(s + q) * P.N) : real(0);
            a1[q] = (in_s && b1 < P.B) ? __ldcg(pp1 + (long long)(s + q) * P.N) : real(0);
        }
        s0 += tree8(a0);
        s1 += tree8(a1);
    }
    if (stop) return;  // converged earlier: this replayed iteration does nothing
    if (P.w_out) {
        // sharded solves: this rank's bands only, the band-weighted sum as
        // the output (the same slot and fma order over the bands it has)
        real accp = real(0);
        if (r != 0) {
            const real *wr = P.wgtr + (r - 1) * P.B;
            for (int b = P.ub0 + ty; b < P.ub1; b += kBandSlots)
                accp = fma(sum_sets(P.part + (long long)b * P.Spad * P.N + cc, P.S, P.N), wr[b], accp);
        }
        sband[ty][tx] = accp;
        __syncthreads();
        if (ty == 0 && cin) {
            real tot = real(0);
#pragma unroll
            for (int y = 0; y < kBandSlots; ++y) tot += sband[y][tx];
            P.w_out[c] = (double)tot;
        }
        return;
    }
    real acc = real(0);
    if (r != 0) {
        const real *wr = P.wgtr + (r - 1) * P.B;
        if (b0 < P.B) acc = fma(s0, wr[b0], acc);
        if (b1 < P.B) acc = fma(s1, wr[b1], acc);
        for (int b = ty + 2 * kBandSlots; b < P.B; b += kBandSlots)
            acc = fma(sum_sets(P.part + (long long)b * P.Spad * P.N + c, P.S, P.N), wr[b], acc);
    }
    sband[ty][tx] = acc;
    __syncthreads();
    if (ty != 0) return;
    double ss = 0.0, mx = -INFINITY;
    if (cin) {
        real tot = real(0);
#pragma unroll
        for (int y = 0; y < kBandSlots; ++y) tot += sband[y][tx];
        update_cell_value(P, c, r, (double)tot, x_old, ss, mx);
    }
    fin_warp_reduce(ss, mx);
    update_block_tail(P, cb, cell_blocks, ss, mx, it_prev, &is_last);
}

// Four consecutive values of a partial set, through L2 only.
__device__ __forceinline__ void ld_cells4(const float *p, float (&v)[4]) {
    const float4 x = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
__device__ __forceinline__ void ld_cells4(const double *p, double (&v)[4]) {
    const double2 x = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 y = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
}

__device__ __forceinline__ void st_cells4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st_cells4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Vector cell block cb: 128 cells; warp w = band slot w.
template <typename real>
__device__ __forceinline__ void update_cells_vec(const UpdateParams<real> &P, const int cb, const int cell_blocks) {
    __shared__ __align__(16) real sslot[kBandSlots][kVecCells];
    __shared__ double sred[2][kVecCells / 32];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (!P.ignore_done && *((volatile int *)P.done) != 0) return;  // converged earlier: nothing to do
    const long long c0 = (long long)cb * kVecCells + 4 * lane;
    const bool lin = c0 < P.N;   // N is a multiple of 4: all four cells or none
    int reg[4];
    if (lin) {
        const int4 q0 = *reinterpret_cast<const int4 *>(P.cell + c0);
        const int4 q1 = *reinterpret_cast<const int4 *>(P.cell + c0 + 2);
        reg[0] = q0.y & kRegionMask;
        reg[1] = q0.w & kRegionMask;
        reg[2] = q1.y & kRegionMask;
        reg[3] = q1.w & kRegionMask;
    } else {
        reg[0] = reg[1] = reg[2] = reg[3] = 0;
    }
    real acc[4] = {real(0), real(0), real(0), real(0)};
    for (int b = warp; b < P.B; b += kBandSlots) {
        const real *pp = P.part + (long long)b * P.Spad * P.N + (lin ? c0 : 0);
        real sb[4] = {real(0), real(0), real(0), real(0)};
        for (int s = 0; s < P.S; s += 8) {
            // a batch of eight sets as two halves of four (the same tree:
            // ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7)))
            real hs[2][4];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                real a[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int sq = s + 4 * half + q;
                    if (lin && sq < P.S) {
                        ld_cells4(pp + (long long)sq * P.N, a[q]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v) a[q][v] = real(0);
                    }
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) hs[half][v] = (a[0][v] + a[1][v]) + (a[2][v] + a[3][v]);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) sb[v] += hs[0][v] + hs[1][v];
        }
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (reg[v] != 0) acc[v] = fma(sb[v], P.wgtr[(reg[v] - 1) * P.B + b], acc[v]);
    }
    st_cells4(&sslot[warp][4 * lane], acc);
    __syncthreads();
    // one thread per cell for the FP64 part (warps 0 .. 3)
    const int t = threadIdx.x;
    if (t >= kVecCells) return;
    const long long c = (long long)cb * kVecCells + t;
    double ss = 0.0, mx = -INFINITY;
    if (c < P.N) {
        real tot = real(0);
#pragma unroll
        for (int y = 0; y < kBandSlots; ++y) tot += sslot[y][t];
        update_cell_value(P, c, P.cell[c].y & kRegionMask, (double)tot, P.x_in[c], ss, mx);
    }
    fin_warp_reduce(ss, mx);
    if (lane == 0) {
        sred[0][warp] = ss;
        sred[1][warp] = mx;
    }
    // the four warps' partials, in warp order (named barrier of warps 0 .. 3)
    asm volatile("bar.sync 1, %0;" ::"n"(kVecCells) : "memory");
    if (warp != 0) return;
    const int it_prev = (lane == 0) ? *P.iter : 0;
    ss = ((sred[0][0] + sred[0][1]) + (sred[0][2] + sred[0][3]));
    mx = fmax(fmax(sred[1][0], sred[1][1]), fmax(sred[1][2], sred[1][3]));
    update_block_tail(P, cb, cell_blocks, ss, mx, it_prev, &is_last);
}

// Block `blk` of the update of problem P (face blocks, then cell blocks).
template <typename real, bool VEC>
__device__ __forceinline__ void update_body(const UpdateParams<real> &P, const int blk) {
    // the next kernel may be launched now; wait for the sweep's results
    pdl_launch_dependents();
    pdl_wait();
    const int face_blocks = update_face_blocks(P.F, P.B);
    if (blk < face_blocks) {
        update_faces(P, blk);
        return;
    }
    const int cell_blocks = update_cell_blocks(P.N, VEC);
    if constexpr (VEC)
        update_cells_vec(P, blk - face_blocks, cell_blocks);
    else
        update_cells(P, blk - face_blocks, cell_blocks);
}

// (the FP64 vector form holds twice the bytes per load: three blocks per SM)
template <typename real, bool VEC>
__global__ void __launch_bounds__(kUpdThreads, (VEC && sizeof(real) == 8) ? 3 : 4)
update_kernel(const __grid_constant__ UpdateParams<real> P) {
    update_body<real, VEC>(P, blockIdx.x);
}

// Batched form: table[blockIdx.x] = {instance, block of that instance};
// each instance's blocks take its own form (vector or scalar cell blocks).
template <typename real>
__global__ void __launch_bounds__(kUpdThreads, sizeof(real) == 8 ? 3 : 4)
update_batch_kernel(const UpdateParams<real> *__restrict__ params, const int2 *__restrict__ table) {
    const int2 e = table[blockIdx.x];
    const UpdateParams<real> &P = params[e.x];
    if (P.vec)
        update_body<real, true>(P, e.y);
    else
        update_body<real, false>(P, e.y);
}

// Close a graph replay / an eager chunk under deferred finalization: one
// warp per problem reduces the pending block partials and records them.
template <typename real>
__global__ void __launch_bounds__(32) finalize_kernel(const UpdateParams<real> *__restrict__ params) {
    const UpdateParams<real> &P = params[blockIdx.x];
    if (!P.defer || P.fin.pending == nullptr || *((volatile const int *)P.fin.pending) == 0) return;
    double eps, tmx, tss;
    fin_reduce(P.fin, eps, tmx, tss);
    if (threadIdx.x == 0) fin_record(P.fin, eps, tmx, tss);
}

template <typename real>
cudaError_t launch_finalize(const UpdateParams<real> *params, int n, cudaStream_t st) {
    if (n < 1) return cudaErrorInvalidConfiguration;
    finalize_kernel<real><<<n, 32, 0, st>>>(params);
    return cudaGetLastError();
}

// Sharded solves: one thread per cell, 32 cells per block (the scalar cell
// blocks' count, so the finalization reduces the same block partials): the
// same per-cell step as the update from W (every band's weighted sum), then
// the residual and the ticketed finalization.
template <typename real>
__global__ void __launch_bounds__(kCellsPerBlock) apply_kernel(const __grid_constant__ UpdateParams<real> P,
                                                               const double *__restrict__ W) {
    __shared__ int is_last;
    const int cb = blockIdx.x;
    const long long c = (long long)cb * kCellsPerBlock + threadIdx.x;
    const int it_prev = (threadIdx.x == 0) ? *P.iter : 0;
    double ss = 0.0, mx = -INFINITY;
    if (c < P.N) update_cell_value(P, c, P.cell[c].y & kRegionMask, W[c], P.x_in[c], ss, mx);
    fin_warp_reduce(ss, mx);
    update_block_tail(P, cb, (int)gridDim.x, ss, mx, it_prev, &is_last);
}

template <typename real>
cudaError_t launch_apply(const UpdateParams<real> &p, const double *W, cudaStream_t st) {
    if (p.vec || p.defer || p.w_out) return cudaErrorInvalidValue;
    apply_kernel<real><<<update_cell_blocks(p.N, false), kCellsPerBlock, 0, st>>>(p, W);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_update(const UpdateParams<real> &p, cudaStream_t st) {
    const int blocks = update_face_blocks(p.F, p.B) + update_cell_blocks(p.N, p.vec != 0);
    if (p.w_out && p.vec) return cudaErrorInvalidValue;   // partial updates use the scalar blocks
    if (p.vec) {
        if (p.N % 4 != 0) return cudaErrorInvalidValue;
        return launch_pdl(update_kernel<real, true>, dim3(blocks), dim3(kUpdThreads), 0, st, p);
    }
    return launch_pdl(update_kernel<real, false>, dim3(blocks), dim3(kUpdThreads), 0, st, p);
}

template <typename real>
cudaError_t launch_update_batch(const UpdateParams<real> *params, const int2 *table, int blocks, cudaStream_t st) {
    if (blocks < 1) return cudaErrorInvalidConfiguration;
    update_batch_kernel<real><<<blocks, kUpdThreads, 0, st>>>(params, table);
    return cudaGetLastError();
}

int update_blocks(long long N, int F, int B, bool vec) { return update_face_blocks(F, B) + update_cell_blocks(N, vec); }
int update_cell_block_count(long long N, bool vec) { return update_cell_blocks(N, vec); }

// ---------------------------------------------------------------------------
// heat flux q_c = sum_b v_b sum_d w_d s_d e_cbd (one warp per cell)
// ---------------------------------------------------------------------------
template <typename real>
__global__ void flux_kernel(long long N, int B, int D, const int2 *__restrict__ cell,
                            const real *__restrict__ e, const double *__restrict__ vws,
                            const double *__restrict__ qshift, double *__restrict__ q) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= N) return;
    const bool act = (cell[c].y & kRegionMask) != 0;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0;
    if (act) {
        const real *ec = e + c * (long long)B * D;
        for (int i = lane; i < B * D; i += 32) {
            const double ev = (double)ec[i];
            q0 += vws[3 * i] * ev;
            q1 += vws[3 * i + 1] * ev;
            q2 += vws[3 * i + 2] * ev;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        q0 += __shfl_down_sync(0xffffffffu, q0, o);
        q1 += __shfl_down_sync(0xffffffffu, q1, o);
        q2 += __shfl_down_sync(0xffffffffu, q2, o);
    }
    if (lane == 0) {
        // e is stored relative to C_b T_ref/(4 pi); add that part's flux back
        q[3 * c] = act ? q0 + qshift[0] : 0.0;
        q[3 * c + 1] = act ? q1 + qshift[1] : 0.0;
        q[3 * c + 2] = act ? q2 + qshift[2] : 0.0;
    }
}

template <typename real>
cudaError_t launch_flux(long long N, int B, int D, const int2 *cell, const real *e, const double *vws,
                        const double *qshift, double *q, cudaStream_t st) {
    const long long threads = N * 32;
    flux_kernel<real><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, B, D, cell, e, vws, qshift, q);
    return cudaGetLastError();
}

// e_user[c][b][perm[d]] = e_int[c][b][d] + shift_b (absolute energy); 0 in void cells
template <typename real>
__global__ void permute_e_kernel(long long total, int D, int B, const int2 *__restrict__ cell,
                                 const real *__restrict__ e_int, const int *__restrict__ perm,
                                 const double *__restrict__ shift, real *__restrict__ e_user) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int d = (int)(i % D);
    const long long cb = i / D;
    const int b = (int)(cb % B);
    const bool act = (cell[cb / B].y & kRegionMask) != 0;
    e_user[cb * D + perm[d]] = act ? (real)((double)e_int[i] + shift[b]) : (real)0;
}

template <typename real>
cudaError_t launch_permute_e(long long N, int B, int D, const int2 *cell, const real *e_int, const int *perm,
                             const double *shift, real *e_user, cudaStream_t st) {
    const long long total = N * B * D;
    permute_e_kernel<real><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, D, B, cell, e_int, perm, shift,
                                                                            e_user);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gradients: dJ/dtau_b = sum_c (1/(tau_cb tau_b)) sum_d (mu - w Theta)(e - e0)
//            dJ/dT_f   = sum over isothermal faces of side f of sum_b C_b/(4 pi) sum_d a_d mu_d
//            dJ/dQ_amp = sum_c phi_c sum_b C_b/(4 pi sum C) sum_d mu_cbd
// ---------------------------------------------------------------------------
constexpr int kGradThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;
}

template <typename real>
__global__ void __launch_bounds__(kGradThreads) grad_kernel(const __grid_constant__ GradParams<real> G,
                                                            int cell_blocks) {
    __shared__ double sh[kGradThreads / 32];
    __shared__ int is_last;
    const int NO = G.B + 10;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool is_cell = (int)blockIdx.x < cell_blocks;
    const long long fi = (long long)(blockIdx.x - cell_blocks) * blockDim.x + threadIdx.x;
    int r = 0;
    if (is_cell && i < G.N) r = G.cell[i].y & kRegionMask;
    double gq = 0.0;
    for (int b = 0; b < G.B; ++b) {
        double v = 0.0;
        if (is_cell && r != 0) {
            double gs = 0.0, ms = 0.0;
            for (int s = 0; s < G.S; ++s) {
                const long long o = ((long long)b * G.Spad + s) * G.N + i;
                gs += (double)G.gpart[o];
                ms += (double)G.apart[o];
            }
            v = gs * G.inv_tt[(r - 1) * G.B + b];
            if (G.phi) gq += G.phi[i] * G.qcoef[b] * ms;
        }
        v = block_sum(v, sh);
        if (threadIdx.x == 0) G.blockpart[(long long)blockIdx.x * NO + b] = v;
    }
    for (int f6 = 0; f6 < 6; ++f6) {
        double v = 0.0;
        if (!is_cell && fi < G.F && G.face_kind[fi] == 0 && G.face_side[fi] == f6) {
            for (int b = 0; b < G.B; ++b) v += G.cb4pi[b] * G.msum[(long long)b * G.F + fi];
        }
        v = block_sum(v, sh);
        if (threadIdx.x == 0) G.blockpart[(long long)blockIdx.x * NO + G.B + f6] = v;
    }
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        if (G.glpart && is_cell && r != 0) {
            for (int b = 0; b < G.B; ++b)
                for (int s = 0; s < G.S; ++s)
                    v += (double)G.glpart[(((long long)a * G.B + b) * G.Spad + s) * G.N + i];
        }
        v = block_sum(v, sh);
        if (threadIdx.x == 0) G.blockpart[(long long)blockIdx.x * NO + G.B + 7 + a] = v;
    }
    gq = block_sum(gq, sh);
    if (threadIdx.x == 0) {
        G.blockpart[(long long)blockIdx.x * NO + G.B + 6] = gq;
        __threadfence();
        const unsigned ticket = atomicAdd(G.counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int o = 0; o < NO; ++o) {
        double acc = 0.0;
        for (int blk = threadIdx.x; blk < (int)gridDim.x; blk += blockDim.x)
            acc += __ldcg(&G.blockpart[(long long)blk * NO + o]);
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) G.out[o] = acc;
    }
    if (threadIdx.x == 0) *G.counter = 0u;
}

template <typename real>
cudaError_t launch_grad(const GradParams<real> &g, cudaStream_t st) {
    const int cell_blocks = (int)((g.N + kGradThreads - 1) / kGradThreads);
    const int face_blocks = (g.F + kGradThreads - 1) / kGradThreads;
    grad_kernel<real><<<cell_blocks + face_blocks, kGradThreads, 0, st>>>(g, cell_blocks);
    return cudaGetLastError();
}

template cudaError_t launch_update<float>(const UpdateParams<float> &, cudaStream_t);
template cudaError_t launch_update<double>(const UpdateParams<double> &, cudaStream_t);
template cudaError_t launch_apply<float>(const UpdateParams<float> &, const double *, cudaStream_t);
template cudaError_t launch_apply<double>(const UpdateParams<double> &, const double *, cudaStream_t);
template cudaError_t launch_update_batch<float>(const UpdateParams<float> *, const int2 *, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const UpdateParams<float> *, int, cudaStream_t);
template cudaError_t launch_finalize<double>(const UpdateParams<double> *, int, cudaStream_t);
template cudaError_t launch_update_batch<double>(const UpdateParams<double> *, const int2 *, int, cudaStream_t);
template cudaError_t launch_flux<float>(long long, int, int, const int2 *, const float *, const double *,
                                        const double *, double *, cudaStream_t);
template cudaError_t launch_flux<double>(long long, int, int, const int2 *, const double *, const double *,
                                         const double *, double *, cudaStream_t);
template cudaError_t launch_permute_e<float>(long long, int, int, const int2 *, const float *, const int *,
                                             const double *, float *, cudaStream_t);
template cudaError_t launch_permute_e<double>(long long, int, int, const int2 *, const double *, const int *,
                                              const double *, double *, cudaStream_t);
template cudaError_t launch_grad<float>(const GradParams<float> &, cudaStream_t);
template cudaError_t launch_grad<double>(const GradParams<double> &, cudaStream_t);

template <typename T>
__global__ void skew_kernel(long long N, SkewLayout L, const T *__restrict__ src, T *__restrict__ dst) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) skew_store(L, c, src[c], dst);
}

template <typename T>
cudaError_t launch_skew(long long N, const SkewLayout &L, const T *src, T *dst, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    skew_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, L, src, dst);
    return cudaGetLastError();
}
template cudaError_t launch_skew<float>(long long, const SkewLayout &, const float *, float *, cudaStream_t);
template cudaError_t launch_skew<double>(long long, const SkewLayout &, const double *, double *, cudaStream_t);
template cudaError_t launch_skew<int2>(long long, const SkewLayout &, const int2 *, int2 *, cudaStream_t);

}  // namespace bte
