// Second-order faces (Spatial discretization: the face value is the upwind
// cell's value plus its Green-Gauss gradient times the vector from the cell
// centre to the face centre), as a deferred correction of the step-face
// sweep (the paper's incremental form: the implicit operator keeps step
// faces, the increments of the previous iterate enter the source).  Per
// outer iteration, from the previous iterate e (all bands and directions):
//
//   reconstruct_kernel  one warp per (cell, band): the increments
//       delta_a(c,b,d) = sign(s_a) h_a/2 grad_a e = (G_out - G_in)/2
//     with the Green-Gauss face values G of the faces the direction leaves
//     (out) and enters (in) by along a: interior face (e_c + e_nb)/2,
//     boundary face left by it e_c + (e_c - e_nb)/2 (extrapolated from the
//     neighbour), boundary face entered by it its inflow value, and no
//     gradient along an axis without a neighbour.  The inflow values of the
//     next sweep at this cell's boundary faces are rebuilt from the
//     reconstructed outgoing values (diffuse: reflection of
//     sum w |s_a| (e + delta) over the normaliser; specular: e + delta of the
//     mirror direction), so the reflections stay conservative;
//   correct_kernel  one thread per (cell, band, direction): the source of
//     the next sweep, sum_a a^a (delta_a(upwind cell) [interior in-face]
//     - delta_a(c)).
//
// Both kernels return at once after the solve converged (the stop flag), so
// replayed iterations leave the converged state untouched.
#include <math.h>

#include "bte_internal.cuh"

namespace bte {

constexpr int kRecThreads = 128;

template <typename real>
__global__ void __launch_bounds__(kRecThreads) reconstruct_kernel(const __grid_constant__ Order2Params<real> P) {
    if (P.done && *((volatile const int *)P.done) != 0) return;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= P.N * P.B) return;
    const long long c = wid / P.B;
    const int b = (int)(wid - c * P.B);
    const int D = P.D;
    const int2 ci = P.cell[c];
    const bool act = (ci.y & kRegionMask) != 0;
    const long long row = (c * P.B + b) * (long long)D;
    if (!act) {
        for (int a = 0; a < 3; ++a)
            for (int d = lane; d < D; d += 32) P.del[a * P.NBD + row + d] = real(0);
        return;
    }
    const unsigned bm = ((unsigned)ci.y >> kSideShift) & 63u;
    const long long stride[3] = {1, (long long)P.nx, (long long)P.nx * P.ny};
    for (int a = 0; a < 3; ++a) {
        real *dl = P.del + a * P.NBD + row;
        if (a >= P.dim) {
            for (int d = lane; d < D; d += 32) dl[d] = real(0);
            continue;
        }
        const bool bnd[2] = {((bm >> (2 * a)) & 1u) != 0, ((bm >> (2 * a + 1)) & 1u) != 0};
        const real *e_c = P.e + row;
        const real *e_nb[2] = {bnd[0] ? nullptr : P.e + ((c - stride[a]) * P.B + b) * (long long)D,
                               bnd[1] ? nullptr : P.e + ((c + stride[a]) * P.B + b) * (long long)D};
        // pass 0: directions leaving through a boundary face (in-face interior)
        for (int d = lane; d < D; d += 32) {
            const real ax = P.coef[((long long)b * D + d) * 8 + a];
            const int in = ((P.dneg[d] >> a) & 1) ? 1 : 0;   // side index it enters by (0: minus)
            const int out = in ^ 1;
            real del = real(0);
            if (ax != real(0) && bnd[out] && !bnd[in]) del = (e_c[d] - e_nb[in][d]) * real(0.5);
            if (ax != real(0) && !bnd[out] && !bnd[in]) del = (e_nb[out][d] - e_nb[in][d]) * real(0.25);
            dl[d] = del;
        }
        __syncwarp();
        // inflow values of this cell's boundary faces along a, from the
        // reconstructed outgoing values
        real Bdiff[2] = {real(0), real(0)};
        for (int sd = 0; sd < 2; ++sd) {
            if (!bnd[sd]) continue;
            const int side = 2 * a + sd;
            const int f = face_of(ci.x, ci.y, side);
            const int kind = P.face_kind[f];
            if (kind == 1) {
                // diffuse: directions leaving through this side
                double acc = 0.0;
                for (int d = lane; d < D; d += 32) {
                    const int in = ((P.dneg[d] >> a) & 1) ? 1 : 0;
                    if ((in ^ 1) != sd) continue;
                    acc += (double)P.coef[((long long)b * D + d) * 8 + 4 + a] * (double)(e_c[d] + dl[d]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                Bdiff[sd] = (real)(acc * P.side_scale[side * P.B + b]);
                if (lane == 0) P.ein_out[(long long)b * P.F + f] = Bdiff[sd];
            } else if (kind == 0) {
                Bdiff[sd] = P.ein_fixed[(long long)b * P.F + f];
            }
        }
        __syncwarp();
        // pass 1: directions entering through a boundary face: the next
        // sweep's specular inflow, and their increments (out-face interior)
        for (int d = lane; d < D; d += 32) {
            const real ax = P.coef[((long long)b * D + d) * 8 + a];
            const int in = ((P.dneg[d] >> a) & 1) ? 1 : 0;
            const int out = in ^ 1;
            if (ax == real(0) || !bnd[in]) continue;
            const int side = 2 * a + in;
            const int f = face_of(ci.x, ci.y, side);
            real bin = Bdiff[in];
            if (P.face_kind[f] == 2) {
                const int m = P.mirror[a * D + d];
                bin = e_c[m] + dl[m];
                P.spec_out[((long long)b * P.Fs + P.sidx[f]) * D + d] = bin;
            }
            if (!bnd[out]) dl[d] = ((e_c[d] + e_nb[out][d]) * real(0.5) - bin) * real(0.5);
        }
        __syncwarp();
    }
}

template <typename real>
__global__ void correct_kernel(const __grid_constant__ Order2Params<real> P) {
    if (P.done && *((volatile const int *)P.done) != 0) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.NBD) return;
    const int d = (int)(i % P.D);
    const long long cb = i / P.D;
    const int b = (int)(cb % P.B);
    const long long c = cb / P.B;
    const int2 ci = P.cell[c];
    real corr = real(0);
    if ((ci.y & kRegionMask) != 0) {
        const unsigned bm = ((unsigned)ci.y >> kSideShift) & 63u;
        const long long stride[3] = {1, (long long)P.nx, (long long)P.nx * P.ny};
        for (int a = 0; a < P.dim; ++a) {
            const real ax = P.coef[((long long)b * P.D + d) * 8 + a];
            if (ax == real(0)) continue;
            const int in = ((P.dneg[d] >> a) & 1) ? 1 : 0;
            real r = -P.del[a * P.NBD + i];
            if (!((bm >> (2 * a + in)) & 1u)) {
                const long long up = in ? c + stride[a] : c - stride[a];
                r += P.del[a * P.NBD + (up * P.B + b) * (long long)P.D + d];
            }
            corr = fma(ax, r, corr);
        }
    }
    P.corr[i] = corr;
}

// e[c][b][d] = C_b (T_c - T_ref)/(4 pi) in solid cells (the equilibrium, as
// a deviation), 0 in void cells
template <typename real>
__global__ void equilibrium_kernel(long long N, int B, int D, const int2 *__restrict__ cell,
                                   const real *__restrict__ tdev, const real *__restrict__ cb4pi, real *__restrict__ e) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * B * D) return;
    const long long cb = i / D;
    const int b = (int)(cb % B);
    const long long c = cb / B;
    e[i] = ((cell[c].y & kRegionMask) != 0) ? cb4pi[b] * tdev[c] : real(0);
}

template <typename real>
cudaError_t launch_order2(const Order2Params<real> &p, cudaStream_t st) {
    const long long warps = p.N * p.B;
    const long long blocks = (warps * 32 + kRecThreads - 1) / kRecThreads;
    reconstruct_kernel<real><<<(unsigned)blocks, kRecThreads, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    correct_kernel<real><<<(unsigned)((p.NBD + 255) / 256), 256, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_equilibrium(long long N, int B, int D, const int2 *cell, const real *tdev, const real *cb4pi, real *e,
                               cudaStream_t st) {
    const long long n = N * B * D;
    equilibrium_kernel<real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(N, B, D, cell, tdev, cb4pi, e);
    return cudaGetLastError();
}

template cudaError_t launch_order2<float>(const Order2Params<float> &, cudaStream_t);
template cudaError_t launch_order2<double>(const Order2Params<double> &, cudaStream_t);
template cudaError_t launch_equilibrium<float>(long long, int, int, const int2 *, const float *, const float *, float *,
                                               cudaStream_t);
template cudaError_t launch_equilibrium<double>(long long, int, int, const int2 *, const double *, const double *,
                                                double *, cudaStream_t);

}  // namespace bte
