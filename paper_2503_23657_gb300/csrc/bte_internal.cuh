// Internal declarations of libbte: device data layout, kernel parameter
// blocks and launchers.  Not part of the public C ABI (include/bte.h).
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>

namespace bte {

// Launch with programmatic stream serialization: the kernel may be launched
// while the previous kernel in the stream still runs (it must call
// griddepcontrol.wait before reading that kernel's results).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// cell flags (second word of the per-cell int2; first word = face base index)
//   bits 0..3  region id (0 = void, r >= 1 solid of region r)
//   bits 4..9  side s (0:x- 1:x+ 2:y- 3:y+ 4:z- 5:z+) is a boundary face
//              (outside the domain or next to a void cell)
//   bits 10..15 side s is an isothermal domain face
//   bits 16..21 side s is a specularly reflecting domain face
// ---------------------------------------------------------------------------
constexpr int kRegionMask = 0xF;
constexpr int kSideShift = 4;
constexpr int kIsoShift = 10;
constexpr int kSpecShift = 16;
constexpr int kMaxRegions = 15;

__host__ __device__ inline int face_of(int base, int flags, int side) {
    const unsigned bm = (unsigned)(flags >> kSideShift) & 63u;
    return base + __builtin_popcount(bm & ((1u << side) - 1u));
}

// Diagonal-skewed copy of a per-cell field (plane-pipeline 3D sweep).  A warp
// of that sweep updates, at one step, one cell of each of its 32 rows, on a
// diagonal of the plane spanned by x and the row axis (y, or z when the
// lanes run along z; coordinate R, extent n1, the remaining axis P being
// the plane index) whose direction depends on the octant: X + R constant
// when the sweep runs along x and the row axis in the same sense, X - R
// constant otherwise.  Family 0 keys a cell by X + R, family 1 by
// X + (n1 - 1 - R); rows are innermost, so those 32 cells are 32 consecutive
// entries of one family.  Entries that are no cell (X outside the grid)
// hold zero.
struct SkewLayout {
    int nx, ny;      // grid (x, y extents: decode a cell index)
    int a1;          // row axis: 1 = y, 2 = z
    int n1;          // rows (extent of the row axis)
    int nd;          // nx + n1 - 1 diagonals per plane
    int nyp;         // entries per diagonal (n1 rounded up to 32)
    long long fam;   // entries of one family (planes * nd * nyp)
};
__host__ __device__ inline long long skew_index(const SkewLayout &L, int f, int X, int R, int P) {
    const int key = f ? X + (L.n1 - 1 - R) : X + R;
    return f * L.fam + ((long long)P * L.nd + key) * L.nyp + R;
}

// A subset of directions that share one sweep orientation (the signs of the
// resolved components of s), processed by one CTA per band.
struct Subset {
    int d0;    // first internal direction index
    int cnt;   // number of directions (<= directions per lane)
    int neg;   // bit a set: traversal runs from high to low index on axis a
    int pad;
};

// Parameters of one sweep launch (forward or transposed).  One CTA handles
// one (subset, band) pair over the whole grid; see sweep.cuh.
template <typename real>
struct SweepParams {
    int nx, ny, nz;
    int dim;                          // resolved axes
    int B, D, F, S, R;
    int b0, nb;                       // bands b0 .. b0 + nb - 1 are swept (nb 0: all B; sharded solves)
    int Spad;                         // S rounded up to a multiple of 4
    int WY, WZ;                       // warps along y, warp groups along z
    long long N;                      // nx*ny*nz
    const int2 *__restrict__ cell;    // {face base, flags}
    const real *__restrict__ tsrc;    // fwd: T - T_ref; adj: Theta   [N]
    const real *__restrict__ phi;     // fwd source profile [N] or null
    const real *__restrict__ ein;     // [B][F] boundary values
    real *__restrict__ part;          // [B][Spad][N] per-subset reduction
    real *__restrict__ fsum;          // [S][B][F] per-subset face sums
    real *__restrict__ e;             // [N][B][D] store (fwd) / read (adj)
    real *__restrict__ gpart;         // [B][Spad][N] adj: sum_d (mu_d - w_d Theta)(e_d - e0)
    const Subset *__restrict__ sub;   // [S]
    const real *__restrict__ coef;    // [B][D][8]: a_x a_y a_z w ws_x ws_y ws_z pad
    const real *__restrict__ invdiag; // [R][B][D]
    const real *__restrict__ srck;    // [R][B]  fwd C_b/(4 pi tau_rb); adj 1/tau_rb
    const real *__restrict__ qb;      // [B]     fwd Q_b per unit profile
    const real *__restrict__ tfwd;    // adj + read_e: forward T - T_ref [N]
    const real *__restrict__ cb4pi;   // adj + read_e: C_b/(4 pi) [B]
    const int *__restrict__ done;     // early exit when *done != 0 (nullable)
    int store_e;                      // fwd: write e
    int read_e;                       // adj: accumulate (mu-w Theta)(e-e0) into gpart
    int ein_smem;                     // stage this band's boundary values in shared memory
    // specularly reflecting domain faces (null sidx: the problem has none)
    const int *__restrict__ sidx;     // [F] index of a face among the specular faces, -1 otherwise
    const int *__restrict__ mirror;   // [3][D] direction with the axis-a component reversed
    const real *__restrict__ spec_in; // [B][Fs][D] inflow at specular faces (previous iterate)
    real *__restrict__ spec_out;      // [B][Fs][D] outgoing values stored under the mirror direction
    int Fs;
    // extra source of forward sweeps: xscale * xsrc[c][b][d] (null: none)
    const real *__restrict__ xsrc;
    real xscale;
    // adjoint gradient pass: per-axis cell-size partials (null: none)
    //   glpart[a][b][Spad][N] += sum_d mu_d a^a_d (e_d - e_in,a,d)
    real *__restrict__ glpart;
    const real *__restrict__ ein_fwd;   // [B][F] forward inflow values of the converged state
    const real *__restrict__ spec_fwd;  // [B][Fs][D] forward specular inflow of the converged state
};

// Parameters of the row-block sweep for unmasked 1D/2D grids with one region
// (sweep2d.cuh).  One CTA per (direction chunk, band); a chunk holds up to
// warps_per_cta * DW directions of one quadrant, DW per warp.
//
// Convergence bookkeeping of one source iteration (eps_T from the update's
// block partials, iteration counter, history, flags).  With deferred
// finalization the update only writes the block partials and sets *pending;
// the next row-pipeline sweep (or the finalize kernel that closes a graph
// replay) reduces them, records eps_T and decides whether to stop.
struct FinalizeParams {
    const double *blockpart;          // [nblocks] x {sum of squares, max}
    int nblocks;
    long long n_active;
    double tol;
    int *done, *iter, *status, *pending;
    double *last;                     // {eps, xmax, ss}
    double *eps_hist;                 // [max_hist] or null
    int max_hist;
    int *batch_done;                  // batched solves: instances converged so far (or null)
};

template <typename real>
struct Sweep2DParams {
    int nx, ny;
    int B, D, F, S;                   // S = number of chunks (face-sum sets)
    int b0, nb;                       // bands b0 .. b0 + nb - 1 are swept (nb 0: all B; sharded solves)
    int Spad;                         // cell partial sets rounded up to a multiple of 4
    int warps_per_cta;
    int ring;                         // 1: warps of a chunk combine per-cell sums through shared-
                                      //    memory slices (one cell partial set per chunk); 0: every
                                      //    warp writes its own set (chunk * warps_per_cta + warp)
    const real *__restrict__ tsrc;    // fwd: T - T_ref; adj: Theta [N, padded to 16 elements]
    const real *__restrict__ phi;     // fwd source profile [N, padded] or null
    const real *__restrict__ ein;     // [B][F] boundary values
    real *__restrict__ part;          // [B][Spad][N]
    real *__restrict__ fsum;          // [S][B][F]
    real *__restrict__ e;             // [N][B][D] (store_e)
    const Subset *__restrict__ sub;   // [S] chunks
    const real *__restrict__ coef;    // [B][D][8]
    const real *__restrict__ invdiag; // [B][D] (region 1)
    const real *__restrict__ srck;    // [B] fwd C_b/(4 pi tau_b); adj 1/tau_b
    const real *__restrict__ qb;      // [B]
    const int *__restrict__ wall_face;  // [6][wall_stride] face index or -1
    int wall_stride;
    const int *__restrict__ done;
    int *__restrict__ status;         // set to 2 if a bounded wait expires
    int store_e;
    int stage;                        // stage per-cell inputs in shared memory (TMA bulk copy)
    int groups;                       // row-pipeline kernel: direction groups per CTA
    int adj;                          // row-pipeline kernel: 1 = adjoint sweep
    long long spin_limit;             // row-pipeline kernel: polls of a wait for the warp below
    FinalizeParams fin;               // row-pipeline kernel: finalize the previous iteration
                                      // (fin.pending null: nothing to finalize)
};

// Default poll limit of the row-pipeline kernel's waits for the warp below
// (each poll sleeps ~32 ns: about 35 ms at most).
constexpr long long kPipeSpinLimit = 1LL << 20;

template <typename real>
cudaError_t launch_sweep2d(const Sweep2DParams<real> &p, int dirs_per_warp, int row_blocks, bool adjoint,
                           cudaStream_t st);
size_t sweep2d_smem(int nx, int ny, int stage, int with_phi, int warps, int rb, int ring, int real_bytes);
// Row-pipeline 2D kernel (groups of DW directions, one warp per 32 rows).
template <typename real>
cudaError_t launch_sweep2dp(const Sweep2DParams<real> &p, int dirs_per_warp, cudaStream_t st);
// A batched row-pipeline launch over the instances of one size class (same
// row-block count, groups and direction chunks).
template <typename real>
struct Sweep2DBatch {
    const Sweep2DParams<real> *params;  // device [all instances]
    const int *inst;                    // device [n_inst] instance indices of this class
    int n_inst, chunks, B, groups, nrb, nx_max, ny_max;
    int phi;                            // any instance with a source profile (forward)
    int stage;                          // per-cell source staged in shared memory (else read ahead)
};
template <typename real>
cudaError_t launch_sweep2dp_batch(const Sweep2DBatch<real> &bt, int dirs_per_warp, cudaStream_t st);
size_t sweep2dp_smem(int nx, int ny, int with_phi, int groups, int dw, int stage, int real_bytes);

// Parameters of the plane-pipeline 3D sweep (sweep3dp.cuh): masked grids,
// any number of regions.  One CTA per (direction subset, band); WY warps
// along y (32 rows each) times H warps along z, every warp one plane of a
// pass of H planes.
template <typename real>
struct Sweep3DParams {
    int nx, ny, nz;
    int B, D, F, S, R;                // S = direction subsets (cell and face-sum sets)
    int b0, nb;                       // bands b0 .. b0 + nb - 1 are swept (nb 0: all B; sharded solves)
    int Spad;                         // S rounded up to a multiple of 4
    int WY, H;                        // warps along the row axis, warps along the plane axis
    int lane_axis;                    // row (lane) axis: 1 = y, 2 = z; planes along the other
    long long N;
    SkewLayout skew;                  // layout of the three skewed per-cell inputs
    const int2 *__restrict__ cell;    // skewed {face base, flags}
    const real *__restrict__ tsrc;    // skewed fwd: T - T_ref; adj: Theta
    const real *__restrict__ phi;     // skewed fwd source profile, or null
    const real *__restrict__ ein;     // [B][F] boundary values
    real *__restrict__ part;          // [B][Spad][N]
    real *__restrict__ fsum;          // [S][B][F]
    real *__restrict__ e;             // [N][B][D] (store_e)
    real *__restrict__ wrap;          // [S][B][nx][WY*32][DW] top plane of a pass, read by the next pass
    const Subset *__restrict__ sub;   // [S]
    const real *__restrict__ coef;    // [B][D][8]
    const real *__restrict__ invdiag; // [R][B][D]
    const real *__restrict__ srck;    // [R][B] fwd C_b/(4 pi tau_rb); adj 1/tau_rb
    const real *__restrict__ qb;      // [B]
    const int *__restrict__ done;
    int store_e;
    int adj;                          // 1: adjoint sweep (carries nu = mu / w)
    int grad;                         // 1 (adjoint): gradient form, part receives the dJ/dtau partials
    int iso_fsum;                     // 1: face sums at isothermal domain faces too
    const real *__restrict__ tfwd;    // (grad) skewed forward T - T_ref
    const real *__restrict__ cb4pi;   // (grad) [B] C_b / (4 pi)
    // specular faces (Fs > 0): per-direction inflow of the previous iterate
    // and the next one's, stored under the mirror direction; the adjoint
    // keeps mu = w nu there, the same values as the general kernel's adjoint
    int Fs;
    const int *__restrict__ sidx;     // [F] specular index of a face (-1: not specular)
    const int *__restrict__ mirror;   // [3][D] direction with the axis-a component reversed
    const real *__restrict__ spec_in; // [B][Fs][D]
    real *__restrict__ spec_out;      // [B][Fs][D], or null (nothing stored)
    FinalizeParams fin;               // finalize the previous iteration (fin.pending null: nothing)
    // extra source of forward sweeps (implicit-Euler steps): xscale * xsrc
    // [N][B][D] (padded by 16 values) is added to every direction's
    // right-hand side; null: none
    const real *__restrict__ xsrc;
    real xscale;
};

template <typename real>
cudaError_t launch_sweep3dp(const Sweep3DParams<real> &p, int dirs_per_lane, cudaStream_t st);
size_t sweep3dp_smem(int R, int WY, int H, int dw, int real_bytes, int variant);
constexpr int kPipe3Chunk = 4;        // steps between the CTA barriers of the 3D pipeline

// Temperature (forward) / adjoint-temperature (adjoint) update, FP64.
template <typename real>
struct UpdateParams {
    long long N;
    int B, S, F, R;                   // S = cell partial sets
    int Spad;
    int Sf;                           // face-sum sets (entries of sub)
    int adjoint;
    double T_ref;
    const int2 *__restrict__ cell;
    const Subset *__restrict__ sub;
    const real *__restrict__ part;    // [B][Spad][N]
    const real *__restrict__ fsum;    // [S][B][F]
    const double *__restrict__ x_in;  // fwd T_old / adj Theta_old [N]
    double *__restrict__ x_out;       // [N]
    real *__restrict__ xdev_out;      // fwd T - T_ref / adj Theta, as real [N]
    real *__restrict__ xskew_out;     // the same in the skewed layout (both families), or null
    SkewLayout skew;
    const double *__restrict__ g;     // adj: dJ/dT [N]
    const double *__restrict__ wgt;   // [R][B] fwd 1/tau_rb ; adj C_b/(4 pi tau_rb)
    const real *__restrict__ wgtr;    // the same in the sweep precision
    const double *__restrict__ Kinv;  // [R]   1 / sum_b C_b/tau_rb
    const int *__restrict__ face_cell;
    const int *__restrict__ face_side;
    const int *__restrict__ face_kind;   // 0 isothermal domain face, 1 diffuse, 2 specular domain face
    const real *__restrict__ ein_fixed;  // [B][F] isothermal inflow (fwd)
    real *__restrict__ ein_out;          // [B][F]
    double *__restrict__ fsum_total;     // [B][F] raw face sums (adj, for gradients) or null
    const double *__restrict__ side_scale; // [6][B] fwd 1/N_side ; adj h_a/(v_b N_side)
    // residual bookkeeping
    double *__restrict__ blockpart;   // [gridDim] x {sum sq, max}
    unsigned int *__restrict__ counter;
    int *__restrict__ done;
    int *__restrict__ iter;
    double *__restrict__ eps_hist;    // [max_iter] or null
    double *__restrict__ last;        // {eps, xmax, ss}
    int *__restrict__ status;
    double tol;
    long long n_active;
    int max_hist;
    int ignore_done;                  // final replay passes
    int *batch_done;                  // batched solves: instances converged so far (or null)
    int defer;                        // 1: write the block partials, set *fin.pending, no ticket
    int vec;                          // 1: 128-cell vector cell blocks (N a multiple of 4)
    int ub0, ub1;                     // sharded solves: bands ub0 .. ub1 - 1 only (ub1 0: every band)
    double *__restrict__ w_out;       // sharded solves: per-cell band-weighted sum over those bands
                                      //   (sweep precision, as FP64) instead of T; null: a full update
    FinalizeParams fin;               // (defer) where the partials go
};

// Finalize the pending iteration of one problem / every instance of a batch
// (one warp each); used to close a graph replay under deferred finalization.
template <typename real>
cudaError_t launch_finalize(const UpdateParams<real> *params, int n, cudaStream_t st);

// Launchers (sweep_*.cu / update.cu).  launch_sweep returns
// cudaErrorInvalidConfiguration for a (dirs_per_lane, layers_per_lane, 3D)
// combination that is not instantiated or exceeds the tile's thread limit.
template <typename real>
cudaError_t launch_sweep(const SweepParams<real> &p, int dirs_per_lane, int layers_per_lane, bool three_d,
                         bool adjoint, cudaStream_t st);

// Largest CTA (threads) the sweep tile supports, or 0 if not instantiated.
int sweep_max_threads(int dirs_per_lane, int layers_per_lane, bool three_d);

// A batched launch of the general kernel over the instances of one class of
// 2D problems (same warps along y): grid chunks x B x instances.
template <typename real>
struct SweepBatch {
    const SweepParams<real> *params;  // device [all instances]
    const int *inst;                  // device [n_inst] instance indices of this class
    int n_inst, chunks, B, WY, R_max;
};
template <typename real>
cudaError_t launch_sweep_batch(const SweepBatch<real> &bt, int dirs_per_lane, cudaStream_t st);
// Directions per lane of the general kernel's extended variant (specular
// faces, extra source, cell-size gradient partials).
constexpr int kSpecDW = 4;

template <typename real>
cudaError_t launch_update(const UpdateParams<real> &p, cudaStream_t st);
// Sharded solves: T from the band-weighted sums W of every band (summed over
// the ranks), the residual and the iteration's finalization (scalar blocks).
template <typename real>
cudaError_t launch_apply(const UpdateParams<real> &p, const double *W, cudaStream_t st);
// natural-order per-cell field -> skewed layout (both families)
template <typename T>
cudaError_t launch_skew(long long N, const SkewLayout &L, const T *src, T *dst, cudaStream_t st);
// batched update: table[i] = {instance, block of that instance}, `blocks` entries
template <typename real>
cudaError_t launch_update_batch(const UpdateParams<real> *params, const int2 *table, int blocks, cudaStream_t st);
int update_blocks(long long N, int F, int B, bool vec);  // blocks of one instance's update launch
int update_cell_block_count(long long N, bool vec);  // cell blocks of an update (vector or scalar form)

template <typename real>
cudaError_t launch_flux(long long N, int B, int D, const int2 *cell, const real *e,
                        const double *vws /*[B][D][3] v_b w_d s_d*/, const double *qshift /*[3]*/,
                        double *q, cudaStream_t st);

template <typename real>
cudaError_t launch_permute_e(long long N, int B, int D, const int2 *cell, const real *e_int, const int *perm,
                             const double *shift /*[B]*/, real *e_user, cudaStream_t st);

// Second-order faces as a deferred correction (order2.cu).
template <typename real>
struct Order2Params {
    long long N, NBD;                 // cells, N * B * D
    int nx, ny, dim, B, D, F, Fs;
    const int2 *__restrict__ cell;
    const real *__restrict__ e;       // [N][B][D] previous iterate
    const real *__restrict__ coef;    // [B][D][8]
    const int *__restrict__ dneg;     // [D] bit a: s_a < 0
    const int *__restrict__ face_kind;
    const int *__restrict__ sidx;     // [F] or null
    const int *__restrict__ mirror;   // [3][D] or null
    const real *__restrict__ ein_fixed;   // [B][F] isothermal inflow
    const double *__restrict__ side_scale; // [6][B] 1 / diffuse normaliser
    real *__restrict__ del;           // [3][N][B][D] reconstruction increments
    real *__restrict__ corr;          // [N][B][D] source of the next sweep
    real *__restrict__ ein_out;       // [B][F] next sweep's inflow (diffuse entries rewritten)
    real *__restrict__ spec_out;      // [B][Fs][D] next sweep's specular inflow, or null
    const int *__restrict__ done;     // stop flag (null: none)
};
template <typename real>
cudaError_t launch_order2(const Order2Params<real> &p, cudaStream_t st);
template <typename real>
cudaError_t launch_equilibrium(long long N, int B, int D, const int2 *cell, const real *tdev, const real *cb4pi, real *e,
                               cudaStream_t st);

// Gradient reduction after the final adjoint sweep (all FP64 accumulation).
template <typename real>
struct GradParams {
    long long N;
    int B, S, F;
    int Spad;
    const int2 *__restrict__ cell;
    const real *__restrict__ apart;     // [B][Spad][N] sum_d mu_d
    const real *__restrict__ gpart;     // [B][Spad][N] sum_d (mu_d - w_d Theta)(e_d - e0)
    const double *__restrict__ phi;     // [N] source profile or null
    const double *__restrict__ inv_tt;  // [R][B] 1/(tau_rb tau_b)
    const double *__restrict__ qcoef;   // [B] Q_amp derivative weight C_b/(4 pi sum C)
    const double *__restrict__ cb4pi;   // [B] C_b/(4 pi)
    const int *__restrict__ face_side;
    const int *__restrict__ face_kind;  // 0 isothermal domain face
    const double *__restrict__ msum;    // [B][F] raw adjoint face sums sum_d a_d mu_d
    const real *__restrict__ glpart;    // [3][B][Spad][N] cell-size partials, or null
    double *__restrict__ blockpart;     // [gridDim][B+10]
    unsigned int *__restrict__ counter;
    double *__restrict__ out;           // [B + 10]: dJ/dtau_b, dJ/dT_wall[6], dJ/dQ_amp,
                                        //   sum mu a^a (e - e_in) per axis (x3)
};

template <typename real>
cudaError_t launch_grad(const GradParams<real> &g, cudaStream_t st);

}  // namespace bte
