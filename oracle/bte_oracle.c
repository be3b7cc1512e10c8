/*
 * FP64 CPU oracle for the steady, nongray phonon BTE under the
 * relaxation-time approximation (RTA) on a masked Cartesian grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (paper, Methods):
 *   - the discretised BTE of Eq. (bte-2), with the RTA sign of that equation
 *     (the collision term is -(e - e0)/tau; the earlier statement of the BTE
 *     prints the opposite sign, which is a typo),
 *   - integrated over a finite volume as in Eq. (fvm-1) with first-order
 *     (step) upwind face values, i.e. the matrix A of Eq. (A_matrix) with the
 *     face area S_ij also in the off-diagonal term,
 *   - the equilibrium energy e0 = C T / (4 pi) and the lattice temperature
 *     T = sum_b sum_d w_d e/tau / sum_b C_b/tau (Eq. updatee0_t),
 *   - the heat flux q = sum_b sum_d w_d v_b s_d e,
 *   - isothermal, diffusely reflecting and specularly reflecting domain
 *     faces (Boundary conditions section); faces between solid and void
 *     cells are diffuse.  A specular face returns, into direction d, the
 *     energy the cell sends out through it in the mirror direction of d
 *     (the normal component reversed), which the direction set must
 *     contain,
 *   - the per-band source Q_b = C_b Q / (4 pi sum C) per steradian, so that
 *     the divergence of q equals Q,
 *   - the outer iteration of the "solution procedure" list (Methods): start
 *     from e = e0(T_init), solve every (band, direction) transport problem
 *     exactly by sweeping in upwind order, update e0 and T, repeat until
 *     eps_T < tol (convergence criterion, Methods).
 *   The diffuse and specular inflows use the previous iterate's outgoing
 *   energy; the fixed point is unchanged by that lag.
 *
 * The adjoint (Forward and inverse modelling workflow: discrete adjoint of
 * the implicit solve) solves (L - P W - R)^T mu = W^T g by the transposed
 * fixed-point iteration and returns dJ/dtau_b, dJ/dT_wall, dJ/dQ_amp and the
 * geometric gradient dJ/dL_a (the paper's 1D inverse problem recovers a film
 * thickness): a^a = v |s_a| / h_a with h_a = L_a / n_a, so with the inflow
 * value e_in of axis a (upwind cell, wall or reflection)
 *   dJ/dL_a = (1/L_a) sum_{c,b,d} mu_cbd a^a_bd (e_cbd - e_in,a,cbd).
 *
 * Second-order faces (p->order == 2; Spatial discretization: the face value
 * is the upwind cell's value plus its Green-Gauss gradient times the vector
 * from the cell centre to the face centre), solved as the paper's
 * incremental form prescribes: the implicit operator keeps the step
 * (first-order) faces and the reconstruction increments
 *   delta_a(c) = sign(s_a) h_a/2 * grad_a e(c)
 * of the previous iterate enter the right-hand side (deferred correction),
 *   rhs += sum_a a^a (delta_a(upwind cell) [interior in-face] - delta_a(c)).
 * Green-Gauss gradient: grad_a e(c) = (G+ - G-)/h_a with the face values
 *   interior face                       (e_c + e_neighbour)/2,
 *   boundary face the direction enters  its inflow value,
 *   boundary face the direction leaves  e_c + (e_c - e_neighbour)/2 (linear
 *                                        extrapolation from the neighbour),
 * and grad_a = 0 in a cell that has no neighbour along a.  Outgoing face
 * values at boundary faces are reconstructed too (e_c + delta), also in the
 * diffuse and specular reflections.  Readings of the paper, which gives the
 * reconstruction but not its boundary treatment.
 *
 * Transient steps (orc_transient; the paper's Conclusion names transient
 * transport as the next extension): implicit Euler in time of
 *   de/dt + v s.grad e = -(e - e0)/tau + Q,
 * every step solved like the steady problem (source iteration with exact
 * sweeps) with 1/dt added to the diagonal and e^m/dt to the source.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ISOTHERMAL 0
#define ORC_DIFFUSE 1
#define ORC_SPECULAR 2

typedef struct {
    int dim;
    int n[3];
    double h[3];
    const unsigned char *mask;   /* n0*n1*n2, x fastest; 0 void, r>=1 region */
    int B;
    const double *C, *v, *tau;   /* per band */
    int R;
    const double *tau_scale;     /* per region */
    int D;
    const double *s;             /* D*3 */
    const double *w;             /* D */
    const int *bc_type;          /* 6 domain faces */
    const double *bc_T;          /* 6 */
    const double *phi;           /* N or NULL */
    double Q_amp;
    int order;                   /* 1: step faces; 2: Green-Gauss reconstructed faces */
} orc_problem;

static const double FOUR_PI = 4.0 * M_PI;

static long n_cells(const orc_problem *p) { return (long)p->n[0] * p->n[1] * p->n[2]; }

static long cell_index(const orc_problem *p, const int idx[3]) {
    return idx[0] + (long)p->n[0] * (idx[1] + (long)p->n[1] * idx[2]);
}

static double tau_cb(const orc_problem *p, long c, int b) {
    return p->tau[b] * p->tau_scale[p->mask[c] - 1];
}

/* Neighbour across side `side` (0:x-,1:x+,2:y-,...) or -1 if outside. */
static long neighbour(const orc_problem *p, long c, int side) {
    int idx[3];
    idx[0] = (int)(c % p->n[0]);
    idx[1] = (int)((c / p->n[0]) % p->n[1]);
    idx[2] = (int)(c / ((long)p->n[0] * p->n[1]));
    int a = side / 2;
    idx[a] += (side & 1) ? 1 : -1;
    if (idx[a] < 0 || idx[a] >= p->n[a]) return -1;
    return cell_index(p, idx);
}

/* Side of cell c through which direction d enters along axis a. */
static int upwind_side(const orc_problem *p, int d, int a) {
    return (p->s[3 * d + a] > 0.0) ? 2 * a : 2 * a + 1;
}

/* Outward normal sign of a side: -1 for the minus side, +1 for the plus side. */
static double side_sign(int side) { return (side & 1) ? 1.0 : -1.0; }

/* Sum over incoming directions of w |s.n| for a side (diffuse normaliser). */
static double diffuse_norm(const orc_problem *p, int side) {
    int a = side / 2;
    double sg = side_sign(side), acc = 0.0;
    for (int d = 0; d < p->D; ++d) {
        double sn = p->s[3 * d + a] * sg;
        if (sn < 0.0) acc += p->w[d] * fabs(sn);
    }
    return acc;
}

/* Boundary kind of side `side` of active cell c: 0 interior, 1 isothermal
 * domain face, 2 diffuse (domain face or solid/void interface), 3 specular
 * domain face. */
static int side_kind(const orc_problem *p, long c, int side) {
    long m = neighbour(p, c, side);
    if (m < 0) {
        if (p->bc_type[side] == ORC_ISOTHERMAL) return 1;
        return (p->bc_type[side] == ORC_SPECULAR) ? 3 : 2;
    }
    return p->mask[m] ? 0 : 2;
}

/* mirror[3 * d + a]: the direction whose axis-a component is reversed and
 * whose other components equal those of d (-1 if the set has none). */
static int *mirror_table(const orc_problem *p) {
    int *m = (int *)malloc(sizeof(int) * 3 * (size_t)p->D);
    if (!m) return NULL;
    for (int d = 0; d < p->D; ++d)
        for (int a = 0; a < 3; ++a) {
            m[3 * d + a] = -1;
            for (int k = 0; k < p->D; ++k) {
                double err = 0.0;
                for (int q = 0; q < 3; ++q) {
                    double want = (q == a) ? -p->s[3 * d + q] : p->s[3 * d + q];
                    err += fabs(p->s[3 * k + q] - want);
                }
                if (err < 1e-12) { m[3 * d + a] = k; break; }
            }
        }
    return m;
}

/* every specular face of the problem needs the mirror of every direction */
static int mirrors_complete(const orc_problem *p, const int *m) {
    for (int side = 0; side < 2 * p->dim; ++side) {
        if (p->bc_type[side] != ORC_SPECULAR) continue;
        for (int d = 0; d < p->D; ++d)
            if (m[3 * d + side / 2] < 0) return 0;
    }
    return 1;
}

static double Q_band(const orc_problem *p, long c, int b) {
    if (!p->phi) return 0.0;
    double Csum = 0.0;
    for (int k = 0; k < p->B; ++k) Csum += p->C[k];
    return p->C[b] * p->Q_amp * p->phi[c] / (FOUR_PI * Csum);
}

#define E(arr, c, b, d) (arr)[((c) * (long)p->B + (b)) * p->D + (d)]

/* Reconstruction increments of second-order faces: DEL(del, c, b, d, a). */
#define DEL(arr, c, b, d, a) (arr)[(((c) * (long)p->B + (b)) * p->D + (d)) * 3 + (a)]

/* Energy carried into a diffuse side of cell c, band b, by the previous
 * iterate: sum over outgoing d' of w |s.n| times the outgoing face value
 * (the cell value, plus its reconstruction increment for second-order
 * faces: del non-NULL), over the normaliser. */
static double diffuse_inflow(const orc_problem *p, const double *e_old, const double *del, long c, int b,
                             int side) {
    int a = side / 2;
    double sg = side_sign(side), acc = 0.0;
    for (int d = 0; d < p->D; ++d) {
        double sn = p->s[3 * d + a] * sg;
        if (sn > 0.0) acc += p->w[d] * sn * (E(e_old, c, b, d) + (del ? DEL(del, c, b, d, a) : 0.0));
    }
    return acc / diffuse_norm(p, side);
}

/* Value entering cell c (band b, direction d) through its boundary side
 * `side` of kind 1 (isothermal), 2 (diffuse) or 3 (specular), from the
 * previous iterate. */
static double boundary_inflow(const orc_problem *p, const int *mirror, const double *e_old, const double *del,
                              long c, int b, int d, int side, int kind) {
    int a = side / 2;
    if (kind == 1) return p->C[b] * p->bc_T[side] / FOUR_PI;
    if (kind == 3) {
        int m = mirror[3 * d + a];
        return E(e_old, c, b, m) + (del ? DEL(del, c, b, m, a) : 0.0);
    }
    return diffuse_inflow(p, e_old, del, c, b, side);
}

/* Second-order faces: the reconstruction increments delta_a(c, b, d) =
 * sign(s_a) h_a/2 grad_a e of iterate e, for every solid cell, band,
 * direction and resolved axis (zero for s_a = 0).  Directions that leave a
 * cell through a boundary face are done first (their Green-Gauss value there
 * is an extrapolation), since the inflow values of the others at that face
 * are built from them. */
static void reconstruct(const orc_problem *p, const int *mirror, const double *e, double *del) {
    long N = n_cells(p);
    for (long c = 0; c < N; ++c)
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                for (int a = 0; a < 3; ++a) DEL(del, c, b, d, a) = 0.0;
    for (int pass = 0; pass < 2; ++pass)
    for (long c = 0; c < N; ++c) {
        if (!p->mask[c]) continue;
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                for (int a = 0; a < p->dim; ++a) {
                    double sa = p->s[3 * d + a];
                    if (sa == 0.0) continue;
                    int side_in = upwind_side(p, d, a), side_out = side_in ^ 1;
                    int k_in = side_kind(p, c, side_in), k_out = side_kind(p, c, side_out);
                    /* pass 0: directions leaving through a boundary face; pass 1: the rest */
                    if ((pass == 0) != (k_out != 0)) continue;
                    double ec = E(e, c, b, d), g = 0.0;
                    if (k_in == 0 || k_out == 0) {
                        double G[2];   /* face values on the minus and plus sides of axis a */
                        for (int sd = 0; sd < 2; ++sd) {
                            int side = 2 * a + sd;
                            int kind = side_kind(p, c, side);
                            if (kind == 0) {
                                G[sd] = 0.5 * (ec + E(e, neighbour(p, c, side), b, d));
                            } else if (side == side_in) {
                                G[sd] = boundary_inflow(p, mirror, e, del, c, b, d, side, kind);
                            } else {
                                double en = E(e, neighbour(p, c, side ^ 1), b, d);
                                G[sd] = ec + 0.5 * (ec - en);
                            }
                        }
                        g = (G[1] - G[0]) / p->h[a];
                    }
                    DEL(del, c, b, d, a) = (sa > 0.0 ? 1.0 : -1.0) * 0.5 * p->h[a] * g;
                }
    }
}

/* One exact transport solve for (b, d) at frozen T and frozen reflected
 * inflow: a triple loop over the cells in the upwind order of d's octant.
 * del: reconstruction increments of the previous iterate (second-order
 * faces) or NULL; e_prev, inv_dt: the previous time step's e and 1/dt of a
 * transient step, or NULL and 0. */
static void sweep_one(const orc_problem *p, const int *mirror, int b, int d, const double *T,
                      const double *e_old, double *e_new, const double *del, const double *e_prev,
                      double inv_dt) {
    int start[3], stop[3], step[3];
    for (int a = 0; a < 3; ++a) {
        int fwd = (a >= p->dim) || (p->s[3 * d + a] >= 0.0);
        start[a] = fwd ? 0 : p->n[a] - 1;
        stop[a] = fwd ? p->n[a] : -1;
        step[a] = fwd ? 1 : -1;
    }
    int idx[3];
    for (idx[2] = start[2]; idx[2] != stop[2]; idx[2] += step[2])
    for (idx[1] = start[1]; idx[1] != stop[1]; idx[1] += step[1])
    for (idx[0] = start[0]; idx[0] != stop[0]; idx[0] += step[0]) {
        long c = cell_index(p, idx);
        if (!p->mask[c]) continue;
        double tc = tau_cb(p, c, b);
        double diag = 1.0 / tc;
        double rhs = p->C[b] * T[c] / (FOUR_PI * tc) + Q_band(p, c, b);
        if (e_prev) {
            diag += inv_dt;
            rhs += inv_dt * E(e_prev, c, b, d);
        }
        for (int a = 0; a < p->dim; ++a) {
            double sa = p->s[3 * d + a];
            if (sa == 0.0) continue;
            double coef = p->v[b] * fabs(sa) / p->h[a];   /* v|s.n| S / V */
            diag += coef;
            int side = upwind_side(p, d, a);
            int kind = side_kind(p, c, side);
            double ein;
            if (kind == 0) ein = E(e_new, neighbour(p, c, side), b, d);
            else ein = boundary_inflow(p, mirror, e_old, del, c, b, d, side, kind);
            rhs += coef * ein;
            if (del) {
                /* deferred correction: reconstructed minus step face values */
                if (kind == 0) rhs += coef * DEL(del, neighbour(p, c, side), b, d, a);
                rhs -= coef * DEL(del, c, b, d, a);
            }
        }
        E(e_new, c, b, d) = rhs / diag;
    }
}

/* T_c = sum_b (1/tau_cb) sum_d w_d e / sum_b C_b/tau_cb */
static void temperature(const orc_problem *p, const double *e, double *T) {
    long N = n_cells(p);
    for (long c = 0; c < N; ++c) {
        if (!p->mask[c]) { T[c] = 0.0; continue; }
        double num = 0.0, den = 0.0;
        for (int b = 0; b < p->B; ++b) {
            double tc = tau_cb(p, c, b), acc = 0.0;
            for (int d = 0; d < p->D; ++d) acc += p->w[d] * E(e, c, b, d);
            num += acc / tc;
            den += p->C[b] / tc;
        }
        T[c] = num / den;
    }
}

/* q_c = sum_b v_b sum_d w_d s_d e */
void orc_flux(const orc_problem *p, const double *e, double *q) {
    long N = n_cells(p);
    for (long c = 0; c < N; ++c) {
        for (int a = 0; a < 3; ++a) q[3 * c + a] = 0.0;
        if (!p->mask[c]) continue;
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                for (int a = 0; a < 3; ++a)
                    q[3 * c + a] += p->v[b] * p->w[d] * p->s[3 * d + a] * E(e, c, b, d);
    }
}

/* eps_T = sqrt(mean_c (T_old - T_new)^2) / max_c T_new over solid cells. */
static double eps_T(const orc_problem *p, const double *T_old, const double *T_new) {
    long N = n_cells(p), cnt = 0;
    double ss = 0.0, tmax = -INFINITY;
    for (long c = 0; c < N; ++c) {
        if (!p->mask[c]) continue;
        double dT = T_old[c] - T_new[c];
        ss += dT * dT;
        if (T_new[c] > tmax) tmax = T_new[c];
        ++cnt;
    }
    return sqrt(ss / (double)cnt) / tmax;
}

/*
 * Source iteration.  T_io holds T_init on entry and the final T on exit.
 * e_io receives the final e (N*B*D).  If tol > 0 the loop stops at the first
 * iteration with eps_T < tol, else it runs exactly max_iter iterations.
 * Returns the number of iterations; eps_hist (max_iter entries, may be NULL)
 * receives eps_T per iteration.
 */
int orc_solve(const orc_problem *p, double *T_io, double *e_io, int max_iter,
              double tol, double *eps_hist) {
    long N = n_cells(p);
    long NE = N * (long)p->B * p->D;
    double *e_old = (double *)malloc(sizeof(double) * NE);
    double *T_new = (double *)malloc(sizeof(double) * N);
    int *mirror = mirror_table(p);
    if (!e_old || !T_new || !mirror) { free(e_old); free(T_new); free(mirror); return -1; }
    if (!mirrors_complete(p, mirror)) { free(e_old); free(T_new); free(mirror); return -2; }
    /* step 1: e = e0(T_init) */
    for (long c = 0; c < N; ++c)
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                E(e_io, c, b, d) = p->mask[c] ? p->C[b] * T_io[c] / FOUR_PI : 0.0;
    double *del = NULL;
    if (p->order == 2) {
        del = (double *)malloc(sizeof(double) * NE * 3);
        if (!del) { free(e_old); free(T_new); free(mirror); return -1; }
    }
    int it = 0;
    while (it < max_iter) {
        memcpy(e_old, e_io, sizeof(double) * NE);
        if (del) reconstruct(p, mirror, e_old, del);
        /* step 2: exact transport solve of every (band, direction) */
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                sweep_one(p, mirror, b, d, T_io, e_old, e_io, del, NULL, 0.0);
        /* step 3: update e0 and T */
        temperature(p, e_io, T_new);
        double eps = eps_T(p, T_io, T_new);
        memcpy(T_io, T_new, sizeof(double) * N);
        if (eps_hist) eps_hist[it] = eps;
        ++it;
        /* step 4: convergence test */
        if (tol > 0.0 && eps < tol) break;
    }
    free(e_old);
    free(T_new);
    free(mirror);
    free(del);
    return it;
}

/*
 * Transient: n_steps implicit Euler steps of length dt from the equilibrium
 * at T_io (e = e0(T_init)).  Every step is converged by source iteration
 * (eps_T < tol, at most max_iter iterations; the first iteration of a step
 * starts from the previous step's T and e).  T_io holds the final T on exit,
 * e_io the final e; T_hist (n_steps * N, may be NULL) the temperature after
 * every step, iters (n_steps, may be NULL) the iterations of every step.
 * First-order faces.  Returns the total number of iterations, or -1/-2 as
 * orc_solve.
 */
int orc_transient(const orc_problem *p, double *T_io, double *e_io, double dt, int n_steps, int max_iter,
                  double tol, double *T_hist, int *iters) {
    long N = n_cells(p);
    long NE = N * (long)p->B * p->D;
    double *e_old = (double *)malloc(sizeof(double) * NE);
    double *e_prev = (double *)malloc(sizeof(double) * NE);
    double *T_new = (double *)malloc(sizeof(double) * N);
    int *mirror = mirror_table(p);
    if (!e_old || !e_prev || !T_new || !mirror) {
        free(e_old); free(e_prev); free(T_new); free(mirror);
        return -1;
    }
    if (!mirrors_complete(p, mirror)) {
        free(e_old); free(e_prev); free(T_new); free(mirror);
        return -2;
    }
    double inv_dt = 1.0 / dt;
    for (long c = 0; c < N; ++c)
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                E(e_io, c, b, d) = p->mask[c] ? p->C[b] * T_io[c] / FOUR_PI : 0.0;
    int total = 0;
    for (int m = 0; m < n_steps; ++m) {
        memcpy(e_prev, e_io, sizeof(double) * NE);
        int it = 0;
        while (it < max_iter) {
            memcpy(e_old, e_io, sizeof(double) * NE);
            for (int b = 0; b < p->B; ++b)
                for (int d = 0; d < p->D; ++d)
                    sweep_one(p, mirror, b, d, T_io, e_old, e_io, NULL, e_prev, inv_dt);
            temperature(p, e_io, T_new);
            double eps = eps_T(p, T_io, T_new);
            memcpy(T_io, T_new, sizeof(double) * N);
            ++it;
            if (tol > 0.0 && eps < tol) break;
        }
        total += it;
        if (iters) iters[m] = it;
        if (T_hist) memcpy(T_hist + (long)m * N, T_io, sizeof(double) * N);
    }
    free(e_old); free(e_prev); free(T_new); free(mirror);
    return total;
}

/* ----------------------------------------------------------------------- */
/* adjoint                                                                  */
/* ----------------------------------------------------------------------- */

/* K_c = sum_b C_b / tau_cb */
static double K_cell(const orc_problem *p, long c) {
    double k = 0.0;
    for (int b = 0; b < p->B; ++b) k += p->C[b] / tau_cb(p, c, b);
    return k;
}

/* Theta_c = (g_c + sum_b C_b/(4 pi tau_cb) sum_d mu_cbd) / K_c */
static void adj_theta(const orc_problem *p, const double *mu, const double *g, double *Th) {
    long N = n_cells(p);
    for (long c = 0; c < N; ++c) {
        if (!p->mask[c]) { Th[c] = 0.0; continue; }
        double acc = g[c];
        for (int b = 0; b < p->B; ++b) {
            double sm = 0.0;
            for (int d = 0; d < p->D; ++d) sm += E(mu, c, b, d);
            acc += p->C[b] / (FOUR_PI * tau_cb(p, c, b)) * sm;
        }
        Th[c] = acc / K_cell(p, c);
    }
}

/* Adjoint of the diffuse reflection at a side: sum over the directions that
 * enter through it of a_bd mu_cbd, over the normaliser. */
static double adj_diffuse_sum(const orc_problem *p, const double *mu_old, long c, int b, int side) {
    int a = side / 2;
    double sg = side_sign(side), acc = 0.0;
    for (int d = 0; d < p->D; ++d) {
        double sn = p->s[3 * d + a] * sg;
        if (sn < 0.0) acc += p->v[b] * fabs(p->s[3 * d + a]) / p->h[a] * E(mu_old, c, b, d);
    }
    return acc / diffuse_norm(p, side);
}

/* Transposed transport solve for (b, d): cells in downwind-first order; each
 * cell couples to the downwind neighbours that its upwind faces feed, and at
 * a specular face it leaves by, to the mirror direction that the face feeds. */
static void adj_sweep_one(const orc_problem *p, const int *mirror, int b, int d, const double *Th,
                          const double *mu_old, double *mu_new) {
    int start[3], stop[3], step[3];
    for (int a = 0; a < 3; ++a) {
        int fwd = (a >= p->dim) || (p->s[3 * d + a] >= 0.0);
        /* reverse of the forward order */
        start[a] = fwd ? p->n[a] - 1 : 0;
        stop[a] = fwd ? -1 : p->n[a];
        step[a] = fwd ? -1 : 1;
    }
    int idx[3];
    for (idx[2] = start[2]; idx[2] != stop[2]; idx[2] += step[2])
    for (idx[1] = start[1]; idx[1] != stop[1]; idx[1] += step[1])
    for (idx[0] = start[0]; idx[0] != stop[0]; idx[0] += step[0]) {
        long c = cell_index(p, idx);
        if (!p->mask[c]) continue;
        double tc = tau_cb(p, c, b);
        double diag = 1.0 / tc;
        double rhs = p->w[d] * Th[c] / tc;
        for (int a = 0; a < p->dim; ++a) {
            double sa = p->s[3 * d + a];
            if (sa == 0.0) continue;
            double coef = p->v[b] * fabs(sa) / p->h[a];
            diag += coef;
            int down = upwind_side(p, d, a) ^ 1;      /* the face d leaves by */
            int kind = side_kind(p, c, down);
            if (kind == 0) rhs += coef * E(mu_new, neighbour(p, c, down), b, d);
            else if (kind == 2)
                rhs += p->w[d] * fabs(sa) * adj_diffuse_sum(p, mu_old, c, b, down);
            else if (kind == 3)
                rhs += coef * E(mu_old, c, b, mirror[3 * d + a]);
        }
        E(mu_new, c, b, d) = rhs / diag;
    }
}

/*
 * Adjoint of the converged forward state (e, T) for the loss gradient
 * g = dJ/dT.  Iterates mu <- L^{-T}(W^T(P^T mu + g) + R^T mu) from mu = 0
 * until the relative RMS change of Theta drops below tol (or max_iter).
 * Outputs: g_tau[B], g_Tw[6] (isothermal domain faces), g_Q (scalar),
 * g_L[3] (dJ/dL_a, zero for unresolved axes).  mu_out (N*B*D) may be NULL.
 * Returns the iteration count (-3 for a second-order problem).
 */
int orc_adjoint(const orc_problem *p, const double *e, const double *T, const double *g,
                int max_iter, double tol, double *g_tau, double *g_Tw, double *g_Q,
                double *g_L, double *mu_out) {
    if (p->order == 2) return -3;   /* the adjoint is that of the step-face system */
    long N = n_cells(p);
    long NE = N * (long)p->B * p->D;
    double *mu = (double *)calloc(NE, sizeof(double));
    double *mu_old = (double *)malloc(sizeof(double) * NE);
    double *Th = (double *)malloc(sizeof(double) * N);
    double *Th_new = (double *)malloc(sizeof(double) * N);
    int *mirror = mirror_table(p);
    if (!mu || !mu_old || !Th || !Th_new || !mirror) {
        free(mu); free(mu_old); free(Th); free(Th_new); free(mirror);
        return -1;
    }
    if (!mirrors_complete(p, mirror)) {
        free(mu); free(mu_old); free(Th); free(Th_new); free(mirror);
        return -2;
    }
    adj_theta(p, mu, g, Th);
    int it = 0;
    while (it < max_iter) {
        memcpy(mu_old, mu, sizeof(double) * NE);
        for (int b = 0; b < p->B; ++b)
            for (int d = 0; d < p->D; ++d)
                adj_sweep_one(p, mirror, b, d, Th, mu_old, mu);
        adj_theta(p, mu, g, Th_new);
        double ss = 0.0, mx = 0.0;
        long cnt = 0;
        for (long c = 0; c < N; ++c) {
            if (!p->mask[c]) continue;
            double dd = Th_new[c] - Th[c];
            ss += dd * dd;
            if (fabs(Th_new[c]) > mx) mx = fabs(Th_new[c]);
            ++cnt;
        }
        memcpy(Th, Th_new, sizeof(double) * N);
        ++it;
        double eps = (mx > 0.0) ? sqrt(ss / (double)cnt) / mx : 0.0;
        if (tol > 0.0 && eps < tol) break;
    }
    /* gradients at the adjoint solution */
    double Csum = 0.0;
    for (int b = 0; b < p->B; ++b) Csum += p->C[b];
    for (int b = 0; b < p->B; ++b) g_tau[b] = 0.0;
    for (int f = 0; f < 6; ++f) g_Tw[f] = 0.0;
    *g_Q = 0.0;
    for (int a = 0; a < 3; ++a) g_L[a] = 0.0;
    for (long c = 0; c < N; ++c) {
        if (!p->mask[c]) continue;
        for (int b = 0; b < p->B; ++b) {
            double tc = tau_cb(p, c, b);
            double e0 = p->C[b] * T[c] / FOUR_PI;
            double acc = 0.0, musum = 0.0;
            for (int d = 0; d < p->D; ++d) {
                acc += (E(mu, c, b, d) - p->w[d] * Th[c]) * (E(e, c, b, d) - e0);
                musum += E(mu, c, b, d);
            }
            /* d/dtau_b of 1/tau_cb is -1/(tau_cb tau_b) */
            g_tau[b] += acc / (tc * p->tau[b]);
            if (p->phi) *g_Q += p->phi[c] * p->C[b] / (FOUR_PI * Csum) * musum;
            /* cell size: a^a = v |s_a| / h_a, h_a = L_a / n_a; the inflow
             * value of axis a is the upwind cell's, the wall's or the
             * reflection of the converged e */
            for (int d = 0; d < p->D; ++d)
                for (int a = 0; a < p->dim; ++a) {
                    double sa = p->s[3 * d + a];
                    if (sa == 0.0) continue;
                    int side = upwind_side(p, d, a);
                    int kind = side_kind(p, c, side);
                    double ein = (kind == 0) ? E(e, neighbour(p, c, side), b, d)
                                             : boundary_inflow(p, mirror, e, NULL, c, b, d, side, kind);
                    double coef = p->v[b] * fabs(sa) / p->h[a];
                    g_L[a] += E(mu, c, b, d) * coef * (E(e, c, b, d) - ein) / (p->h[a] * p->n[a]);
                }
            /* isothermal inflow a_bd C_b T_w / (4 pi) enters the source */
            for (int a = 0; a < p->dim; ++a) {
                for (int sd = 0; sd < 2; ++sd) {
                    int side = 2 * a + sd;
                    if (neighbour(p, c, side) >= 0) continue;
                    if (p->bc_type[side] != ORC_ISOTHERMAL) continue;
                    for (int d = 0; d < p->D; ++d) {
                        double sa = p->s[3 * d + a];
                        if (sa == 0.0 || upwind_side(p, d, a) != side) continue;
                        g_Tw[side] += p->v[b] * fabs(sa) / p->h[a] * p->C[b] / FOUR_PI
                                      * E(mu, c, b, d);
                    }
                }
            }
        }
    }
    if (mu_out) memcpy(mu_out, mu, sizeof(double) * NE);
    free(mu); free(mu_old); free(Th); free(Th_new); free(mirror);
    return it;
}
