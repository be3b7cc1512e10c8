/*
 * libbte -- steady nongray phonon Boltzmann transport (relaxation-time
 * approximation) on a masked Cartesian grid, solved on one GB300 GPU.
 *
 * Method (arXiv 2503.23657, Methods section):
 *   - Eq. (bte-2): v_b s.grad e_bs = -(e_bs - e0_b)/tau_b + Q_b, the RTA sign
 *     of the discretised equation (the first statement of the BTE in the
 *     paper prints the collision term with the opposite sign);
 *   - Eq. (updatee0_t): e0_b = C_b T/(4 pi), T = sum_b sum_s w_s e_bs/tau_b
 *     divided by sum_b C_b/tau_b;
 *   - Eq. (fvm-1) with first-order (step) upwind face values, i.e. the
 *     matrix A of Eq. (A_matrix) (face area S_ij included off the diagonal);
 *   - boundary conditions of the "Boundary conditions" subsection:
 *     isothermal walls and diffusely reflecting walls; faces between solid
 *     and void cells reflect diffusely;
 *   - the per-band source Q_b = C_b Q / (4 pi sum_b C_b) per steradian;
 *   - the outer iteration of the solution procedure (Methods, steps 1-4)
 *     with the convergence criterion eps_T of the same list.
 * Each (band, direction) transport problem is solved exactly by an upwind
 * wavefront sweep (A is triangular in sweep order on a Cartesian grid), so
 * the paper's incremental pseudo-time update reduces to source iteration.
 * The diffuse inflow of one iteration uses the previous iterate's outgoing
 * energy; the converged fixed point is unchanged.
 *
 * Conventions shared by every entry point
 *   - cells c = i + nx*(j + ny*k), x fastest; N = nx*ny*nz;
 *   - domain faces 0:x- 1:x+ 2:y- 3:y+ 4:z- 5:z+ (faces of axes >= dim are
 *     ignored);
 *   - e is laid out [cell][band][direction] with the directions in the
 *     caller's order;
 *   - all floating-point inputs are FP64; the solver sweeps in FP32 or FP64
 *     (bte_solve_opts.precision) and always reduces T, residuals and
 *     gradients in FP64.
 *
 * Ownership: bte_create copies every input (host memory); the caller may
 * free them on return.  Output buffers are caller-owned and may be host or
 * device memory (detected per pointer).  The plan owns its device memory.
 *
 * Errors: every int-returning call returns BTE_OK (0) or a negative code
 * below; bte_last_error() describes the last failure of a plan.  Nothing
 * aborts, traps or exits the process.  Device-side waits are bounded and
 * report BTE_ETIMEOUT instead of hanging.
 *
 * Threading: a plan is not thread-safe; use one plan per host thread.
 */
#ifndef BTE_H
#define BTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BTE_OK 0
#define BTE_EINVAL (-1)        /* invalid argument (see bte_last_error) */
#define BTE_ENOMEM (-2)        /* host or device allocation failed */
#define BTE_ECUDA (-3)         /* CUDA runtime error */
#define BTE_ENOTCONVERGED (-4) /* max_iter reached; outputs hold the last iterate */
#define BTE_ETIMEOUT (-5)      /* a bounded device-side wait expired */
#define BTE_ENUMERIC (-6)      /* NaN/Inf in the temperature update */
#define BTE_ESTATE (-7)        /* call order violated (e.g. adjoint before solve) */
#define BTE_ECORRUPT (-8)      /* debug mode (BTE_DEBUG set): a device buffer's guard words were
                                  overwritten, or an index table points outside its extent */

#define BTE_BC_ISOTHERMAL 0
#define BTE_BC_DIFFUSE 1
#define BTE_BC_SPECULAR 2

#define BTE_FP32 0
#define BTE_FP64 1

typedef struct bte_plan bte_plan; /* opaque, library-owned */

/* Grid: dim in {1,2,3}; n[a] cells and length[a] metres per axis; axes
 * a >= dim must have n[a] == 1 (their length is a unit depth). */
typedef struct {
    int dim;
    int n[3];
    double length[3];
} bte_grid;

/* Band table (Methods, band discretisation): B bands with heat capacity
 * C[b] J/(m^3 K) > 0, group speed v[b] m/s > 0, relaxation time tau[b] s > 0;
 * R regions, region r (mask value r+1) uses tau[b]*tau_scale[r] (> 0). */
typedef struct {
    int B;
    const double *C;
    const double *v;
    const double *tau;
    int R;
    const double *tau_scale;
} bte_bands;

/* Discrete ordinates (Methods, angle discretisation): D unit vectors
 * s[3*d+a] and weights w[d] > 0 with sum w = 4 pi (checked to 1e-10). */
typedef struct {
    int D;
    const double *s;
    const double *w;
} bte_quad;

/* Per domain face: type BTE_BC_ISOTHERMAL (wall temperature T[f], K),
 * BTE_BC_DIFFUSE or BTE_BC_SPECULAR (Methods, Boundary conditions: a
 * specularly reflecting wall returns into direction d the energy the cell
 * sends out through it in the mirror direction of d, the component normal to
 * the face reversed; like the diffuse inflow it is taken from the previous
 * iterate, which leaves the converged fixed point unchanged).  A specular
 * face needs the mirror of every direction in the direction set (a product
 * set of Gauss-Legendre polar nodes and an even number of mid-point azimuths
 * has them); on 3D grids the plane pipeline (tile_kind 3) carries them, and
 * the autotuner weighs it against the general kernel's extended variant
 * (tile_kind 1); 1D and 2D problems with specular faces are swept by the
 * latter.  At least one isothermal face must touch the solid. */
typedef struct {
    int type[6];
    double T[6];
} bte_bcs;

/*
 * bte_create -- validate the problem, build the sweep plan, copy the inputs
 * to the device.
 *   mask      N bytes, 0 = void, r >= 1 = solid of region r (r <= R)
 *   q_profile N doubles, W/m^3 per unit source amplitude, or NULL (no source)
 *   out       receives the plan (NULL on failure)
 * Returns BTE_OK, BTE_EINVAL (bad sizes, sum w != 4 pi, tau <= 0, mask value
 * > R, no isothermal face touching the solid, a specular face without the
 * mirror of every direction), BTE_ENOMEM or BTE_ECUDA.
 * Uses the current CUDA device.  On failure nothing is leaked.
 */
int bte_create(const bte_grid *g, const uint8_t *mask, const bte_bands *bands,
               const bte_quad *quad, const bte_bcs *bcs, const double *q_profile,
               bte_plan **out);

typedef struct {
    int precision;          /* BTE_FP32 (FP32 sweeps, FP64 reductions) or BTE_FP64 */
    double tol;             /* stop when eps_T < tol; tol <= 0 runs exactly max_iter */
    int max_iter;           /* > 0 */
    const double *T_init;   /* N doubles (host or device) or NULL */
    double T_init_uniform;  /* used when T_init == NULL (K, > 0) */
    double Q_amp;           /* source amplitude multiplying q_profile */
    const double *tau;      /* B overrides of bands->tau (host), or NULL */
    const double *T_wall;   /* 6 overrides of bcs->T (host), or NULL */
    void *stream;           /* cudaStream_t to run on (NULL = legacy default) */
    int poll_every;         /* iterations per device->host convergence poll (0 = auto) */
    int dirs_per_lane;      /* sweep tile: directions per lane/warp (0 = autotuned) */
    int store_e_every_iter; /* 1: write e to HBM on every sweep; 0: only the final one */
    int tile_kind;          /* 0 = autotuned; 1 = general wavefront kernel (any grid);
                               2 = row-block kernel (unmasked 1D/2D, one region);
                               3 = row-pipeline kernel (unmasked 1D/2D, one region; on 3D
                                   grids the plane-pipeline kernel: masks, several regions
                                   and specular faces allowed; FP32 with 2, 4 or 8
                                   directions per lane, FP64 with 2 or 4) */
    int dirs_per_cta;       /* row kernels: directions per CTA (0 = autotuned) */
    int source_staging;     /* row-pipeline kernel: 0 = autotuned, 1 = per-cell source staged in
                               shared memory, 2 = read ahead from global memory */
    int warps_z;            /* 3D plane-pipeline kernel: warps along the plane axis per CTA
                               (planes in flight per pass); 0 = autotuned */
    int lane_axis;          /* 3D plane-pipeline kernel: axis of the rows its lanes hold,
                               1 = y (planes along z), 2 = z (planes along y); 0 = autotuned */
    int face_order;         /* face values (Methods, Spatial discretization): 0 or 1 = step
                               (first-order) upwind faces; 2 = the paper's second-order faces,
                               upwind cell value plus its Green-Gauss gradient times the centre-to-
                               face vector, solved as a deferred correction (the incremental form:
                               step faces implicit, the reconstruction increments of the previous
                               iterate in the source).  Green-Gauss face values at a boundary face:
                               the inflow value where a direction enters it, linear extrapolation
                               from the neighbour where it leaves, no gradient along an axis without
                               a neighbour; outgoing boundary values are reconstructed, also in the
                               reflections.  face_order 2 runs the general kernel, stores e every
                               iteration and needs 4 N B D extra values of device memory */
    const double *Q_amp_each; /* bte_batch_solve only: n source amplitudes (host), one per instance
                               in plan order, each multiplying its own plan's q_profile; NULL =
                               Q_amp for every instance.  Must be NULL for bte_solve and
                               bte_transient (BTE_EINVAL otherwise) */
    const double *ein_init; /* resume (with T_init): B x F doubles (host or device), the inflow
                               energy density of every boundary face and band that the first
                               iteration reads (as bte_get_state returns it), instead of the
                               diffuse reflection of the equilibrium at T_init; NULL = that
                               default.  Isothermal faces take their wall values either way.
                               Not for bte_batch_solve (BTE_EINVAL) */
} bte_solve_opts;

typedef struct {
    int iterations;         /* outer iterations run */
    int converged;          /* eps_T < tol reached */
    double eps_T;           /* last eps_T (Methods, convergence criterion) */
    double T_max;           /* max T of the last iterate (K) */
    double seconds;         /* device time of the iteration loop */
    double updates_per_s;   /* iterations * solid cells * B * D / seconds */
    int dirs_per_lane;      /* tile used: directions per lane/warp */
    long long kernel_launches; /* kernels launched by the call (incl. early-exit ones) */
    int tile_kind;          /* tile used: 1 general, 2 row-block, 3 row-pipeline (see bte_solve_opts) */
    int dirs_per_cta;       /* tile used: directions per CTA */
    double sweep_seconds;   /* with sweep timing on (bte_set_sweep_timing): summed device
                               time of the call's timed source-iteration sweep launches,
                               each bracketed by CUDA events on its stream, over the
                               iterations the solve ran (a graph replay's iterations after
                               convergence return at once and are not counted); else 0 */
    long long sweep_launches; /* number of sweep launches summed in sweep_seconds */
    int source_staged;      /* row-pipeline tile: 1 = per-cell source staged in shared memory,
                               0 = read ahead from global memory (other kernels: 1) */
    int warps_z;            /* 3D plane-pipeline tile: warps along the plane axis per CTA
                               (other kernels: 0) */
    int lane_axis;          /* 3D plane-pipeline tile: row axis, 1 = y, 2 = z (other kernels: 0) */
    double eps_q;           /* bte_solve with q_out: the flux residual of the convergence criteria
                               (Methods, solution procedure), sqrt(mean_c (|q|^n - |q|^{n+1})^2) /
                               max_c |q|^{n+1} over solid cells, for the returned iterate n and one
                               more iteration from it (reported, not used to stop); NaN when not
                               computed (no q_out, specular faces, face_order 2, adjoint) */
} bte_stats;

/* Fill opts with defaults: FP32, tol 1e-6, max_iter 100000, T_init 300 K,
 * Q_amp 1, autotuned tile, poll every 16 iterations. */
void bte_default_opts(bte_solve_opts *o);

/*
 * bte_solve -- outer source iteration to eps_T < tol (or max_iter).
 *   T_out  N doubles: final lattice temperature (void cells 0), required
 *   q_out  3N doubles: heat flux q = sum_b v_b sum_d w_d s_d e of the final
 *          iterate, or NULL
 *   e_out  N*B*D values of the final iterate, FP32 if precision is FP32 and
 *          FP64 otherwise, [cell][band][direction], or NULL
 *   st     statistics, or NULL
 * The final e is the iterate from which T_out was computed.  The converged
 * state is kept in the plan for bte_adjoint.  Returns BTE_OK,
 * BTE_ENOTCONVERGED (outputs still written), BTE_EINVAL, BTE_ENUMERIC,
 * BTE_ECUDA.
 */
int bte_solve(bte_plan *p, const bte_solve_opts *o, double *T_out, double *q_out, void *e_out,
              bte_stats *st);

/*
 * bte_adjoint -- discrete adjoint of the last bte_solve (Forward and inverse
 * modelling workflow: implicit solves differentiated by a discrete adjoint).
 * Given dJ/dT (N doubles, host or device) of a loss J(T), solves
 * (L - P W - R)^T mu = W^T dJ/dT by the transposed (downwind-ordered)
 * fixed-point iteration and returns
 *   g_tau[B]   dJ/dtau_b (B doubles, host), or NULL
 *   g_Twall[6] dJ/dT_f for isothermal domain faces (0 elsewhere), or NULL
 *   g_Qamp[1]  dJ/dQ_amp, or NULL
 * tol/max_iter apply to the relative RMS change of the adjoint temperature
 * Theta.  Runs on the stream of the preceding bte_solve.  Returns BTE_ESTATE
 * if no solve preceded it.
 */
int bte_adjoint(bte_plan *p, const double *dJ_dT, double tol, int max_iter, double *g_tau,
                double *g_Twall, double *g_Qamp, bte_stats *st);

/*
 * bte_adjoint_ex -- bte_adjoint that also returns, when g_L is not NULL,
 *   g_L[3]     dJ/dL_a, the derivative with respect to the domain length
 *              along each resolved axis (0 for the others), host memory.
 * The cell size is h_a = L_a / n_a and the coupling a^a = v |s_a| / h_a, so
 * dJ/dL_a = (1/L_a) sum_{c,b,d} mu_cbd a^a_bd (e_cbd - e_in,a,cbd) with e_in
 * the value entering along a (upwind cell, wall or reflection of the
 * converged state); the source profile stays per cell.  (The paper's 1D
 * inverse problem recovers a film thickness this way.)  Needs 3 N B S extra
 * values of device memory (S direction subsets of the general kernel).
 * Returns as bte_adjoint; BTE_ESTATE also after a second-order solve (the
 * adjoint is that of the step-face system).
 */
int bte_adjoint_ex(bte_plan *p, const double *dJ_dT, double tol, int max_iter, double *g_tau,
                   double *g_Twall, double *g_Qamp, double *g_L, bte_stats *st);

/*
 * bte_transient -- transient phonon transport (the extension the paper's
 * Conclusion announces): n_steps implicit-Euler steps of length dt (s) of
 *   de/dt + v s.grad e = -(e - e0)/tau + Q
 * from the equilibrium at o->T_init (or T_init_uniform).  Every step is the
 * steady problem with 1/dt added to the diagonal and e^m/dt to the source,
 * solved by the same source iteration to eps_T < o->tol (at most o->max_iter
 * iterations per step); the temperature follows from the same energy
 * balance of the scattering term (Eq. updatee0_t).  Step faces; the general
 * kernel (tile_kind 1) or, on 3D grids, the plane pipeline (tile_kind 3),
 * whichever the autotuner finds faster (tile_kind 0).
 *   T_out   N doubles: T after the last step (host or device), required
 *   T_hist  n_steps * N doubles: T after every step (host or device), or NULL
 *   st      totals over the steps (iterations, seconds), or NULL
 * Returns BTE_OK, BTE_ENOTCONVERGED (a step reached max_iter; outputs still
 * written), BTE_EINVAL, BTE_ENUMERIC, BTE_ECUDA.  The plan holds no
 * adjoint-ready state afterwards.
 */
int bte_transient(bte_plan *p, const bte_solve_opts *o, double dt, int n_steps, double *T_out,
                  double *T_hist, bte_stats *st);

/*
 * bte_profile_sweep -- time the dominant kernel: `reps` forward sweep
 * launches (all bands x directions x cells, the tile of the last solve) on
 * the last solve's state and stream, bracketed by CUDA events after two
 * untimed launches.  Writes the mean duration of one launch (ms) to
 * *ms_per_sweep.  The plan's state is not modified.  Returns BTE_ESTATE if
 * no solve preceded it.
 */
int bte_profile_sweep(bte_plan *p, int reps, double *ms_per_sweep);

/*
 * bte_get_state -- checkpoint of the outer iteration (solution procedure of
 * the paper, steps 1-4: an iterate is fully determined by T and the diffuse
 * inflow its boundary faces carry into the next sweep): after a bte_solve,
 * T_out (N doubles, host or device, or NULL) receives the last iterate T^n
 * and ein_out (B x F doubles, host or device, or NULL; b-major) the inflow
 * energy density e_in of every boundary face and band that iteration n + 1
 * would read (absolute, J/m^3 per steradian).  A bte_solve with T_init =
 * T_out and ein_init = ein_out continues the iteration from there, up to
 * the rounding of the deviation from T_ref (T_ref is the mean of T_init).
 * Specular faces' per-direction inflow and the second-order correction are
 * not part of the state (they restart from the isotropic e of T_init).
 * Returns BTE_OK, BTE_EINVAL (null plan), BTE_ESTATE (no solve yet) or
 * BTE_ECUDA.
 */
int bte_get_state(bte_plan *p, double *T_out, double *ein_out);

/* bte_face_count -- F, the number of boundary faces of the plan (domain faces
 * of solid cells and faces between solid and void cells, in cell order then
 * side order): the extent of ein_init / bte_get_state's ein_out per band.
 * BTE_EINVAL for a null plan. */
int bte_face_count(const bte_plan *p);

/*
 * Sharded solves of one instance (bands split over ranks, one process per
 * GPU).  In the paper's outer iteration (Methods, steps 1-4) the sweeps of
 * different bands are independent given T, and a band's diffuse inflow
 * depends only on that band's own face sums; the temperature update needs,
 * per cell, the sum over all bands of the band-weighted direction sums
 * (Eq. updatee0_t).  So every rank holds a plan of the whole problem, sweeps
 * its own bands [b0, b1) and forms their weighted sums W (N doubles); the
 * ranks add their W (one FP64 allreduce per iteration, done by the caller);
 * every rank then forms the same T.  Iterating bte_shard_sweep, the
 * allreduce and bte_shard_apply until eps_T < tol reproduces bte_solve up to
 * rounding (the band sums are combined in another order).
 *
 * bte_shard_begin -- o: as for bte_solve (precision, T_init / T_init_uniform,
 *   ein_init, tau, T_wall, Q_amp, tile options; tol, max_iter and poll_every
 *   are the caller's loop's).  Sets the initial state (T_ref, the inflow) and
 *   the tile (a previous solve's autotuned tile in this precision, else the
 *   first candidate).  Every rank must pass the same options.  Not for
 *   specular faces or face_order 2 (BTE_EINVAL).  The plan holds no
 *   adjoint-ready state afterwards.
 * bte_shard_sweep -- one sweep of bands [b0, b1) (0 <= b0 < b1 <= B) from the
 *   current state; W_out (N doubles, host or device) receives, per cell, the
 *   sum over those bands of the band-weighted direction sums (zero in void
 *   cells); those bands' next inflow is kept in the plan.
 * bte_shard_apply -- W (N doubles, host or device): the sum of every rank's
 *   W_out.  Forms T^{n+1} (to T_out, N doubles, host or device, or NULL) and
 *   eps_T (to *eps_T, or NULL) and makes it the current state.  BTE_ENUMERIC
 *   for a non-finite eps_T.
 * Each returns BTE_OK, BTE_EINVAL, BTE_ESTATE (sweep or apply before begin)
 * or BTE_ECUDA.
 */
int bte_shard_begin(bte_plan *p, const bte_solve_opts *o);
int bte_shard_sweep(bte_plan *p, int b0, int b1, double *W_out);
int bte_shard_apply(bte_plan *p, const double *W, double *T_out, double *eps_T);

/*
 * bte_set_sweep_timing -- every >= 1: every following bte_solve / bte_adjoint
 * brackets the sweep launch of every `every`-th source iteration (counted
 * within each convergence poll interval, whose first iteration is always
 * timed; also inside the captured CUDA graphs) with a pair of CUDA events
 * and reports the summed durations and their number in
 * bte_stats.sweep_seconds / sweep_launches.  Each timed sweep adds a few
 * microseconds of launch latency; every = 0 (the default) records nothing.
 * Returns BTE_OK, BTE_EINVAL (null plan, every < 0) or BTE_ECUDA (event
 * creation failed).
 */
int bte_set_sweep_timing(bte_plan *p, int every);

/*
 * Batched solves (the paper has none; many independent 2D problems on one
 * GPU).  A batch borrows N plans made by bte_create -- 1D/2D grids of at most
 * 1024 rows (y cells) without specular faces, all with the same band and
 * direction counts, any sizes, masks and region counts -- and solves all of
 * them together: every outer iteration is one sweep launch per size class
 * plus one update launch over every instance, and the iterations are
 * replayed from a captured CUDA graph.  A size class holds the instances
 * with the same kernel and number of 32-row blocks: unmasked single-region
 * instances of at most 512 rows run the row-pipeline kernel, the others
 * (masks, several regions, more rows) the general wavefront kernel; the
 * classes run concurrently.  Each instance keeps its own convergence test
 * (eps_T < tol) and stops iterating when it converges; the solve ends when
 * all have converged or after max_iter.  Results are those of bte_solve on
 * each plan with the same tile.
 *
 * bte_batch_create -- n >= 1 distinct plans (the batch keeps the pointers;
 *   destroy the batch before the plans).  BTE_EINVAL for null or mismatched
 *   plans, BTE_ECUDA if device state cannot be allocated; the message is
 *   read with bte_batch_last_error(NULL).
 * bte_batch_solve -- o: as for bte_solve, except that T_init must be NULL,
 *   Q_amp_each may give each instance its own source amplitude
 *   (T_init_uniform applies to all), T_wall must be NULL (each plan's walls
 *   apply), and tile_kind is 0 or 3 (the batch picks each class's kernel;
 *   the tile is autotuned per size class unless dirs_per_lane /
 *   dirs_per_cta pin it).
 *   T_out: sum of the instances' cell counts doubles (host or device), the
 *   instances' temperatures concatenated in plan order.  st: n entries or
 *   NULL.  bs: batch totals or NULL.  Returns BTE_OK, BTE_EINVAL,
 *   BTE_ENOTCONVERGED (T_out still written), BTE_ENUMERIC, BTE_ETIMEOUT,
 *   BTE_ECUDA.  The plans hold no adjoint-ready state afterwards.
 */
typedef struct bte_batch bte_batch; /* opaque, library-owned */

typedef struct {
    int instances;           /* n */
    int converged;           /* instances that reached eps_T < tol */
    int max_iterations;      /* largest per-instance iteration count */
    double seconds;          /* device time of the iteration loop */
    double updates;          /* sum over instances of iterations * cells * B * D */
    double updates_per_s;    /* updates / seconds */
    long long kernel_launches; /* kernels launched by the iteration loop */
    int classes;             /* size classes (concurrent sweep launches per iteration) */
    double sweep_seconds;    /* with sweep timing on: summed device time of the timed sweep phases */
    long long sweep_iterations; /* number of sweep phases timed */
} bte_batch_stats;

int bte_batch_create(int n, bte_plan *const *plans, bte_batch **out);
int bte_batch_solve(bte_batch *b, const bte_solve_opts *o, double *T_out, bte_stats *st, bte_batch_stats *bs);
void bte_batch_destroy(bte_batch *b);
const char *bte_batch_last_error(const bte_batch *b);
/* bte_batch_set_sweep_timing -- on != 0: the sweep phase (all size classes,
 * fork to join) of the first iteration of every poll interval is bracketed by
 * CUDA events; bte_batch_stats reports the summed time and count.  Returns
 * BTE_OK, BTE_EINVAL or BTE_ECUDA. */
int bte_batch_set_sweep_timing(bte_batch *b, int on);

/*
 * bte_debug_set_wait_limit -- test hook: the number of polls after which the
 * row-pipeline kernel's waits for the warp below give up (0 restores the
 * default, about 1e6 polls of ~32 ns).  A wait that gives up records the
 * failure and the solve returns BTE_ETIMEOUT (its results are then not
 * valid); the kernel still ends normally, with every access in bounds, and
 * the plan stays usable.  Waits for bulk copies in flight keep their own
 * limit.  Returns BTE_OK or BTE_EINVAL (null plan, polls < 0).
 */
int bte_debug_set_wait_limit(bte_plan *p, long long polls);

/*
 * Debug mode (the environment variable BTE_DEBUG set to anything but "0" when
 * the library first allocates): every device buffer the library allocates
 * carries 256 guard bytes of a fixed pattern after its end; bte_solve,
 * bte_adjoint(_ex), bte_transient and bte_batch_solve check the guards of
 * every live buffer after they ran and return BTE_ECORRUPT if one was
 * overwritten; bte_create checks every index table of the plan (face cells
 * and sides, cell face bases, wall faces, direction permutation, specular
 * tables) against its extent before uploading it and returns BTE_ECORRUPT
 * for the first violation.  Off by default (the checks synchronise the
 * device).
 *
 * bte_debug_overwrite_guard -- test hook (debug mode only): overwrites one
 * guard byte of the plan's status buffer from the host (a write inside the
 * allocation), so that the next solve reports BTE_ECORRUPT.  Returns BTE_OK,
 * BTE_EINVAL (null plan), BTE_ESTATE (debug mode off) or BTE_ECUDA.
 */
int bte_debug_overwrite_guard(bte_plan *p);

/* Copy the eps_T history of the last bte_solve (one value per iteration,
 * at most n, the first 65536 iterations) into out (host).  Returns the
 * number of values copied or a negative code. */
int bte_eps_history(const bte_plan *p, double *out, int n);

/*
 * bte_eps_T_noalloc -- the outer iteration's convergence measure,
 * eps_T = sqrt(mean_c (T_old - T_new)^2) / max_c T_new over solid cells,
 * computed on the GPU without allocating any memory.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc
 * where they need the measure -- a host framework whose device memory all
 * belongs to its own pool, a loop that must never trigger the implicit
 * device synchronisation of cudaMalloc, or code that runs while another
 * thread captures a CUDA graph in global mode, where such calls are refused.
 *   T_old, T_new  N doubles, device memory
 *   mask          N bytes, device memory (0 = void, skipped), or NULL (all solid)
 *   N             1 <= N <= BTE_NOALLOC_MAX_CELLS
 *   out           3 doubles, device memory: {eps_T, max T_new, solid count}
 *   stream        cudaStream_t (NULL = legacy default stream)
 * Scratch lives in a fixed file-scope device array (about 24 KB, held by
 * every GPU that loads the library until the process exits).  The first call
 * on a device -- and the first after a device reset, which gives the device
 * a new context -- looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that call before any
 * stream capture.  All calls on a device share the array and it keeps the
 * last call's contents (the call clears its counter itself): calls that
 * overlap on the GPU race.  Returns BTE_OK, BTE_EINVAL (null pointer, N out
 * of range; see bte_last_error(NULL)) or BTE_ECUDA.  Asynchronous: out is
 * written when the stream reaches the launch.
 */
#define BTE_NOALLOC_MAX_CELLS (1LL << 24)
int bte_eps_T_noalloc(const double *T_old, const double *T_new, const uint8_t *mask, long long N,
                      double *out, void *stream);

/* Release every resource of the plan (NULL is a no-op). */
void bte_destroy(bte_plan *p);

/* Text of the last error on this plan, or of the last failed bte_create
 * when p is NULL.  Valid until the next call on the same plan. */
const char *bte_last_error(const bte_plan *p);

/* Library version string. */
const char *bte_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTE_H */
