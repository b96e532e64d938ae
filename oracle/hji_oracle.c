/*
 * FP64 CPU oracle for the warm-start HJI reachability time-march
 * (Herbert, Ghosh, Bansal, Tomlin, "Reachability-Based Safety Guarantees
 * using Efficient Initializations", arXiv:1903.07715).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, step by step, in the paper's order:
 *   - the problem model of Sec. II-A, Eq. (1): x' = f(x,u,d), u in a box U,
 *     d in a box D, written in control-affine form
 *       f(x,u,d) = c + A x + sum_t w_t phi_t(x[axis_t]) + G u + E d,
 *     phi in {tan, sin, cos} (the quadrotor of Sec. VI, Eq. (22), needs
 *     g tan(theta));
 *   - the Hamiltonian of Sec. II-B, Eq. (6): H(x,p) = max_u min_d <p, f(x,u,d)>
 *     (control maximises, disturbance minimises: the avoid game of Sec. II);
 *   - the HJI variational inequality of Sec. II-B, Eq. (7), marched backwards
 *     in time from V(x,0) = l(x) (standard initialisation, Sec. II-B) or from
 *     V(x,0) = min(k(x), l(x)) (warm start, Sec. III, Eq. (14) and the 0^-
 *     argument in the proof of Thm. 1, case b);
 *   - the per-step projection V <- min(V, l) that Eq. (7) and the dynamic
 *     programming recursion Eq. (8) impose;
 *   - convergence: the largest change of V over the grid in one step is
 *     compared with a tolerance (Sec. IV, first paragraph).
 * The paper delegates the numerical scheme to a level-set toolbox (Sec. II-B,
 * after Eq. (8)).  The scheme written here is the textbook one for that
 * toolbox family: upwind one-sided derivatives (ENO1, ENO2 of Osher and Shu,
 * HJ-WENO5 of Jiang and Peng), the Lax-Friedrichs numerical Hamiltonian with a
 * global per-axis dissipation coefficient, and TVD Runge-Kutta stages (Euler,
 * Heun, Shu-Osher) under a CFL-limited step.  Readings where the paper is
 * silent:
 *   - time runs backwards: with tau = -t, Eq. (5) reads dV/dtau = H;
 *   - ghost nodes beyond a non-periodic edge extrapolate V linearly:
 *     V[-j] = V[0] + j (V[0] - V[1]), likewise at the high end;
 *   - the ENO2 tie |a| == |b| takes the lower-index second difference;
 *   - the WENO5 epsilon is 1e-6 max(v_k^2) + 1e-99;
 *   - alpha_a = max over the grid of max_{u,d} |f_a|; dt = cfl / max over the
 *     grid of sum_a max_{u,d}|f_a(x,u,d)| / dx_a, fixed for a solve;
 *   - min(., l) is applied after each full Runge-Kutta step, not per stage.
 *
 * Compile with -ffp-contract=off: every + - * / rounds on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 4 /* state dimensions per grid */
#define OR_MAXU 4 /* control / disturbance components */
#define OR_MAXT 8 /* nonlinear terms w * phi(x[axis]) */

enum { OR_FN_TAN = 0, OR_FN_SIN = 1, OR_FN_COS = 2 };
enum { OR_ENO1 = 1, OR_ENO2 = 2, OR_WENO5 = 5 };

/* Variants of the march (flags of oracle_step / oracle_solve):
 *   OR_BRS: march the HJI PDE of Eq. (5) alone, without the projection onto
 *     V <= l of Eq. (7): the value of the backward reachable set at time
 *     tau (the target reached at exactly tau, Sec. II-B) instead of the
 *     tube;
 *   OR_LOCAL_LF: Lax-Friedrichs dissipation with the node's own
 *     coefficients alpha_a(x) = max_{u,d} |f_a(x,u,d)| instead of their
 *     maxima over the grid (dt stays the grid-wide CFL step). */
enum { OR_BRS = 1, OR_LOCAL_LF = 2 };

typedef struct {
    int ndim;
    int64_t n[OR_MAXD];
    double lo[OR_MAXD], hi[OR_MAXD];
    int periodic[OR_MAXD];
    int m, q, nterms;
    double c[OR_MAXD];
    double A[OR_MAXD * OR_MAXD]; /* A[i*OR_MAXD + j] multiplies x_j in f_i   */
    double G[OR_MAXD * OR_MAXU]; /* G[i*OR_MAXU + j] multiplies u_j in f_i   */
    double E[OR_MAXD * OR_MAXU]; /* E[i*OR_MAXU + k] multiplies d_k in f_i   */
    int term_row[OR_MAXT], term_axis[OR_MAXT], term_fn[OR_MAXT];
    double term_w[OR_MAXT];
    double ulo[OR_MAXU], uhi[OR_MAXU], dlo[OR_MAXU], dhi[OR_MAXU];
} oracle_problem;

typedef struct {
    int64_t steps;       /* full Runge-Kutta steps taken                   */
    double tau;          /* backward time reached, steps * dt              */
    double dt;           /* the fixed CFL step                             */
    double last_delta;   /* max |V^{n+1} - V^n| of the last step           */
    int converged;       /* 1 if last_delta < tol ended the march          */
    double alpha[OR_MAXD];
} oracle_stats;

/* ---------------------------------------------------------------- grid */

/* Node spacing: (hi-lo)/(N-1) for a closed axis, (hi-lo)/N for a periodic one. */
double oracle_spacing(const oracle_problem* P, int a) {
    if (P->periodic[a]) return (P->hi[a] - P->lo[a]) / (double)P->n[a];
    return (P->hi[a] - P->lo[a]) / (double)(P->n[a] - 1);
}

/* Coordinate of node i along axis a: lo + i * dx. */
double oracle_node(const oracle_problem* P, int a, int64_t i) {
    return P->lo[a] + (double)i * oracle_spacing(P, a);
}

int64_t oracle_num_cells(const oracle_problem* P) {
    int64_t total = 1;
    for (int a = 0; a < P->ndim; ++a) total *= P->n[a];
    return total;
}

/* C order, axis 0 slowest. */
static void unravel(const oracle_problem* P, int64_t flat, int64_t* idx) {
    for (int a = P->ndim - 1; a >= 0; --a) {
        idx[a] = flat % P->n[a];
        flat /= P->n[a];
    }
}

static int64_t ravel(const oracle_problem* P, const int64_t* idx) {
    int64_t flat = 0;
    for (int a = 0; a < P->ndim; ++a) flat = flat * P->n[a] + idx[a];
    return flat;
}

/* Value of W at idx shifted by `off` along axis a, with ghost nodes outside
 * the grid: periodic wrap, or linear extrapolation from the two edge nodes. */
static double value_at(const oracle_problem* P, const double* W, const int64_t* idx, int a,
                       int off) {
    int64_t j[OR_MAXD];
    for (int b = 0; b < P->ndim; ++b) j[b] = idx[b];
    int64_t N = P->n[a];
    int64_t s = idx[a] + off;
    if (s >= 0 && s < N) {
        j[a] = s;
        return W[ravel(P, j)];
    }
    if (P->periodic[a]) {
        int64_t w = s % N;
        if (w < 0) w += N;
        j[a] = w;
        return W[ravel(P, j)];
    }
    double k;    /* how many nodes beyond the edge */
    double edge, inner;
    if (s < 0) {
        k = (double)(-s);
        j[a] = 0;
        edge = W[ravel(P, j)];
        j[a] = 1;
        inner = W[ravel(P, j)];
    } else {
        k = (double)(s - (N - 1));
        j[a] = N - 1;
        edge = W[ravel(P, j)];
        j[a] = N - 2;
        inner = W[ravel(P, j)];
    }
    return edge + k * (edge - inner);
}

/* ---------------------------------------------------------- dynamics */

static double apply_fn(int fn, double x) {
    if (fn == OR_FN_TAN) return tan(x);
    if (fn == OR_FN_SIN) return sin(x);
    return cos(x);
}

/* f(x,u,d) of Eq. (1) in control-affine form. */
void oracle_dynamics(const oracle_problem* P, const double* x, const double* u,
                     const double* d, double* f) {
    int n = P->ndim;
    for (int i = 0; i < n; ++i) {
        double fi = P->c[i];
        for (int j = 0; j < n; ++j) fi += P->A[i * OR_MAXD + j] * x[j];
        for (int t = 0; t < P->nterms; ++t)
            if (P->term_row[t] == i)
                fi += P->term_w[t] * apply_fn(P->term_fn[t], x[P->term_axis[t]]);
        for (int j = 0; j < P->m; ++j) fi += P->G[i * OR_MAXU + j] * u[j];
        for (int k = 0; k < P->q; ++k) fi += P->E[i * OR_MAXU + k] * d[k];
        f[i] = fi;
    }
}

/* Vertex number `bits` of a box with bounds lo/hi in `dim` components. */
static void box_vertex(int dim, const double* lo, const double* hi, int bits, double* v) {
    for (int j = 0; j < dim; ++j) v[j] = ((bits >> j) & 1) ? hi[j] : lo[j];
}

static double dot(int n, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Eq. (6): H(x,p) = max_{u in U} min_{d in D} <p, f(x,u,d)>.
 * <p,f> is affine in u for fixed d and affine in d for fixed u, so over boxes
 * the inner min is attained at a vertex of D and the outer max at a vertex of
 * U; the oracle simply enumerates the vertices. */
double oracle_hamiltonian(const oracle_problem* P, const double* x, const double* p) {
    double u[OR_MAXU], d[OR_MAXU], f[OR_MAXD];
    double best = -INFINITY;
    for (int ub = 0; ub < (1 << P->m); ++ub) {
        box_vertex(P->m, P->ulo, P->uhi, ub, u);
        double worst = INFINITY;
        for (int db = 0; db < (1 << P->q); ++db) {
            box_vertex(P->q, P->dlo, P->dhi, db, d);
            oracle_dynamics(P, x, u, d, f);
            double v = dot(P->ndim, p, f);
            if (v < worst) worst = v;
        }
        if (worst > best) best = worst;
    }
    return best;
}

/* alpha_a(x) = max_{u in U, d in D} |f_a(x,u,d)|: the bound on |dH/dp_a| that
 * the Lax-Friedrichs dissipation needs.  f_a is affine in (u,d), so the max of
 * its magnitude over the box U x D is attained at a vertex. */
void oracle_alpha_point(const oracle_problem* P, const double* x, double* alpha) {
    double u[OR_MAXU], d[OR_MAXU], f[OR_MAXD];
    for (int a = 0; a < P->ndim; ++a) alpha[a] = 0.0;
    for (int ub = 0; ub < (1 << P->m); ++ub) {
        box_vertex(P->m, P->ulo, P->uhi, ub, u);
        for (int db = 0; db < (1 << P->q); ++db) {
            box_vertex(P->q, P->dlo, P->dhi, db, d);
            oracle_dynamics(P, x, u, d, f);
            for (int a = 0; a < P->ndim; ++a)
                if (fabs(f[a]) > alpha[a]) alpha[a] = fabs(f[a]);
        }
    }
}

static void node_coords(const oracle_problem* P, const int64_t* idx, double* x) {
    for (int a = 0; a < P->ndim; ++a) x[a] = oracle_node(P, a, idx[a]);
}

/* Dissipation coefficients alpha[a] = max over grid nodes of alpha_a(x), and
 * the CFL step dt = cfl / max over grid nodes of sum_a alpha_a(x)/dx_a.
 * Returns 0, or -1 when the dynamics vanish on the whole grid (no finite dt). */
int oracle_alpha_dt(const oracle_problem* P, double cfl, double* alpha, double* dt) {
    int64_t total = oracle_num_cells(P);
    double dx[OR_MAXD];
    for (int a = 0; a < P->ndim; ++a) {
        dx[a] = oracle_spacing(P, a);
        alpha[a] = 0.0;
    }
    double rate = 0.0;
    for (int64_t c = 0; c < total; ++c) {
        int64_t idx[OR_MAXD];
        double x[OR_MAXD], al[OR_MAXD];
        unravel(P, c, idx);
        node_coords(P, idx, x);
        oracle_alpha_point(P, x, al);
        double r = 0.0;
        for (int a = 0; a < P->ndim; ++a) {
            if (al[a] > alpha[a]) alpha[a] = al[a];
            r += al[a] / dx[a];
        }
        if (r > rate) rate = r;
    }
    if (!(rate > 0.0)) return -1;
    *dt = cfl / rate;
    return 0;
}

/* ------------------------------------------------- one-sided derivatives */

static int ghost_width(int scheme) {
    if (scheme == OR_ENO1) return 1;
    if (scheme == OR_ENO2) return 2;
    return 3;
}

int oracle_ghost_width(int scheme) { return ghost_width(scheme); }

/* Of two second differences, the one of smaller magnitude (ENO2 choice);
 * a tie keeps the first (lower-index) one. */
static double smaller_magnitude(double a, double b) { return fabs(a) <= fabs(b) ? a : b; }

/* HJ-WENO5 of Jiang and Peng: the weighted combination of the three
 * third-order ENO candidates built from five one-sided differences v1..v5. */
static double weno5(double v1, double v2, double v3, double v4, double v5) {
    double phi1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
    double phi2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
    double phi3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
    double s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3) +
                0.25 * (v1 - 4.0 * v2 + 3.0 * v3) * (v1 - 4.0 * v2 + 3.0 * v3);
    double s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4) +
                0.25 * (v2 - v4) * (v2 - v4);
    double s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) * (v3 - 2.0 * v4 + v5) +
                0.25 * (3.0 * v3 - 4.0 * v4 + v5) * (3.0 * v3 - 4.0 * v4 + v5);
    double vmax = v1 * v1;
    if (v2 * v2 > vmax) vmax = v2 * v2;
    if (v3 * v3 > vmax) vmax = v3 * v3;
    if (v4 * v4 > vmax) vmax = v4 * v4;
    if (v5 * v5 > vmax) vmax = v5 * v5;
    double eps = 1e-6 * vmax + 1e-99;
    double a1 = 0.1 / ((s1 + eps) * (s1 + eps));
    double a2 = 0.6 / ((s2 + eps) * (s2 + eps));
    double a3 = 0.3 / ((s3 + eps) * (s3 + eps));
    double sum = a1 + a2 + a3;
    return (a1 / sum) * phi1 + (a2 / sum) * phi2 + (a3 / sum) * phi3;
}

/* One-sided derivatives at the centre of a stencil line v[0..2g] (centre
 * v[g]) with spacing dx.  pm is the left-biased (backward) and pp the
 * right-biased (forward) approximation of dV/dx.
 * Undivided differences: D[k] = v[k+1] - v[k]; second differences
 * S[k] = D[k] - D[k-1] (= v[k+1] - 2 v[k] + v[k-1] up to rounding). */
void oracle_one_sided(int scheme, const double* v, double dx, double* pm, double* pp) {
    int g = ghost_width(scheme);
    int c = g;
    if (scheme == OR_ENO1) {
        *pm = (v[c] - v[c - 1]) / dx;
        *pp = (v[c + 1] - v[c]) / dx;
        return;
    }
    double D[7];
    for (int k = 0; k < 2 * g; ++k) D[k] = v[k + 1] - v[k];
    /* D[k] sits between nodes k and k+1; the backward difference at the
     * centre is D[c-1] and the forward one D[c]. */
    if (scheme == OR_ENO2) {
        double Sm = D[c - 1] - D[c - 2]; /* second difference centred at c-1 */
        double S0 = D[c] - D[c - 1];     /* centred at c                     */
        double Sp = D[c + 1] - D[c];     /* centred at c+1                   */
        /* p- = D-V + m(Q_{c-1}, Q_c), p+ = D+V - m(Q_c, Q_{c+1}), where
         * Q_j = S_j / (2 dx); the common factor 1/(2dx) > 0 does not change
         * which of the two has the smaller magnitude. */
        *pm = D[c - 1] / dx + smaller_magnitude(Sm, S0) / (2.0 * dx);
        *pp = D[c] / dx - smaller_magnitude(S0, Sp) / (2.0 * dx);
        return;
    }
    /* WENO5: backward uses D-V at c-2..c+2, i.e. D[c-3..c+1]; forward uses
     * D+V at c+2..c-2, i.e. D[c+2] down to D[c-2]. */
    *pm = weno5(D[c - 3] / dx, D[c - 2] / dx, D[c - 1] / dx, D[c] / dx, D[c + 1] / dx);
    *pp = weno5(D[c + 2] / dx, D[c + 1] / dx, D[c] / dx, D[c - 1] / dx, D[c - 2] / dx);
}

/* ------------------------------------------------------ spatial operator */

/* L(W) at every node: the Lax-Friedrichs approximation of the right-hand side
 * of dV/dtau = H(x, grad V):
 *   L = H(x, (p+ + p-)/2) + sum_a alpha_a (p+_a - p-_a) / 2. */
static void spatial_operator(const oracle_problem* P, int scheme, const double* alpha,
                             const double* W, double* L, int flags) {
    int64_t total = oracle_num_cells(P);
    int g = ghost_width(scheme);
    double dx[OR_MAXD];
    for (int a = 0; a < P->ndim; ++a) dx[a] = oracle_spacing(P, a);
#pragma omp parallel for schedule(static)
    for (int64_t cidx = 0; cidx < total; ++cidx) {
        int64_t idx[OR_MAXD];
        double x[OR_MAXD], pbar[OR_MAXD], pm[OR_MAXD], pp[OR_MAXD], line[7];
        unravel(P, cidx, idx);
        node_coords(P, idx, x);
        for (int a = 0; a < P->ndim; ++a) {
            for (int o = -g; o <= g; ++o) line[o + g] = value_at(P, W, idx, a, o);
            oracle_one_sided(scheme, line, dx[a], &pm[a], &pp[a]);
            pbar[a] = 0.5 * (pp[a] + pm[a]);
        }
        double h = oracle_hamiltonian(P, x, pbar);
        double al[OR_MAXD];
        if (flags & OR_LOCAL_LF) oracle_alpha_point(P, x, al);
        else
            for (int a = 0; a < P->ndim; ++a) al[a] = alpha[a];
        double diss = 0.0;
        for (int a = 0; a < P->ndim; ++a) diss += al[a] * 0.5 * (pp[a] - pm[a]);
        L[cidx] = h + diss;
    }
}

/* -------------------------------------------- optimal control, Eq. (9) */

/* Eq. (9) at one state: u* = argmax_u min_d <p, f(x,u,d)> with p standing
 * for grad V(x), and the disturbance d* that attains the inner minimum for
 * u*.  As for H, the max and min of these affine functions over boxes are
 * attained at vertices, which are enumerated.  Ties: the U-vertices are
 * visited from the all-upper vertex (bits 2^m - 1) down and a later vertex
 * must be strictly better to replace the kept one; the D-vertices from the
 * all-lower vertex (bits 0) up, again keeping the first of equal values. */
void oracle_control_at(const oracle_problem* P, const double* x, const double* p, double* u_opt,
                       double* d_opt) {
    double u[OR_MAXU], d[OR_MAXU], f[OR_MAXD];
    double best = -INFINITY;
    int best_ub = (1 << P->m) - 1, best_db = 0;
    for (int ub = (1 << P->m) - 1; ub >= 0; --ub) {
        box_vertex(P->m, P->ulo, P->uhi, ub, u);
        double worst = INFINITY;
        int worst_db = 0;
        for (int db = 0; db < (1 << P->q); ++db) {
            box_vertex(P->q, P->dlo, P->dhi, db, d);
            oracle_dynamics(P, x, u, d, f);
            double v = dot(P->ndim, p, f);
            if (v < worst) {
                worst = v;
                worst_db = db;
            }
        }
        if (worst > best) {
            best = worst;
            best_ub = ub;
            best_db = worst_db;
        }
    }
    box_vertex(P->m, P->ulo, P->uhi, best_ub, u_opt);
    if (d_opt) box_vertex(P->q, P->dlo, P->dhi, best_db, d_opt);
}

/* Eq. (9) at every node of the grid for the value V: grad V is taken as the
 * average of the scheme's one-sided derivatives, (p- + p+)/2, the same
 * gradient at which the march evaluates the Hamiltonian (ghost nodes as in
 * the march).  u_out holds m grid-shaped arrays one after another
 * (u_out[j * N + node]), d_out (may be NULL) q of them. */
void oracle_optimal_control(const oracle_problem* P, int scheme, const double* V, double* u_out,
                            double* d_out) {
    int64_t total = oracle_num_cells(P);
    int g = ghost_width(scheme);
    double dx[OR_MAXD];
    for (int a = 0; a < P->ndim; ++a) dx[a] = oracle_spacing(P, a);
#pragma omp parallel for schedule(static)
    for (int64_t cidx = 0; cidx < total; ++cidx) {
        int64_t idx[OR_MAXD];
        double x[OR_MAXD], pbar[OR_MAXD], pm, pp, line[7], u[OR_MAXU], d[OR_MAXU];
        unravel(P, cidx, idx);
        node_coords(P, idx, x);
        for (int a = 0; a < P->ndim; ++a) {
            for (int o = -g; o <= g; ++o) line[o + g] = value_at(P, V, idx, a, o);
            oracle_one_sided(scheme, line, dx[a], &pm, &pp);
            pbar[a] = 0.5 * (pp + pm);
        }
        oracle_control_at(P, x, pbar, u, d);
        for (int j = 0; j < P->m; ++j) u_out[(int64_t)j * total + cidx] = u[j];
        if (d_out)
            for (int k = 0; k < P->q; ++k) d_out[(int64_t)k * total + cidx] = d[k];
    }
}

/* The averaged gradient (p- + p+)/2 of the scheme at every node (grad[a * N
 * + node]), the gradient oracle_optimal_control uses; exposed for tests that
 * need to know where a control choice is decided by a clear margin. */
void oracle_gradient(const oracle_problem* P, int scheme, const double* V, double* grad) {
    int64_t total = oracle_num_cells(P);
    int g = ghost_width(scheme);
    double dx[OR_MAXD];
    for (int a = 0; a < P->ndim; ++a) dx[a] = oracle_spacing(P, a);
#pragma omp parallel for schedule(static)
    for (int64_t cidx = 0; cidx < total; ++cidx) {
        int64_t idx[OR_MAXD];
        double pm, pp, line[7];
        unravel(P, cidx, idx);
        for (int a = 0; a < P->ndim; ++a) {
            for (int o = -g; o <= g; ++o) line[o + g] = value_at(P, V, idx, a, o);
            oracle_one_sided(scheme, line, dx[a], &pm, &pp);
            grad[(int64_t)a * total + cidx] = 0.5 * (pp + pm);
        }
    }
}

/* The operator L(W) on its own, exposed for tests. */
int oracle_operator(const oracle_problem* P, int scheme, const double* alpha, const double* W,
                    double* L) {
    spatial_operator(P, scheme, alpha, W, L, 0);
    return 0;
}

/* One full time step of the HJI VI, Eq. (7): a TVD Runge-Kutta step of
 * dV/dtau = L(V) built from Euler stages E(W) = W + dt L(W),
 *   rk 1: V' = E(V)
 *   rk 2: V1 = E(V);  V' = V/2 + E(V1)/2                       (Heun)
 *   rk 3: V1 = E(V);  V2 = 3V/4 + E(V1)/4;  V' = V/3 + 2E(V2)/3 (Shu-Osher)
 * followed by the projection V' <- min(V', l) of Eq. (7)/(8).
 * Discounted reachability (Sec. II-C): with 0 < gamma < 1 the projection
 * becomes V' <- min(l, gamma V'), the discounted dynamic-programming step
 * with gamma = exp(-lambda dt) the factor of one step (gamma 0 or 1: off).
 * Writes V' to Vout and returns max |V' - V| through *delta. */
int oracle_step(const oracle_problem* P, int scheme, int rk, double dt, const double* alpha,
                const double* l, const double* V, double* Vout, double* delta, int flags,
                double gamma) {
    int64_t total = oracle_num_cells(P);
    double* L = (double*)malloc(sizeof(double) * (size_t)total);
    double* W1 = (double*)malloc(sizeof(double) * (size_t)total);
    double* W2 = (double*)malloc(sizeof(double) * (size_t)total);
    if (!L || !W1 || !W2) {
        free(L);
        free(W1);
        free(W2);
        return -1;
    }
    spatial_operator(P, scheme, alpha, V, L, flags);
    if (rk == 1) {
        for (int64_t c = 0; c < total; ++c) Vout[c] = V[c] + dt * L[c];
    } else {
        for (int64_t c = 0; c < total; ++c) W1[c] = V[c] + dt * L[c];
        spatial_operator(P, scheme, alpha, W1, L, flags);
        if (rk == 2) {
            for (int64_t c = 0; c < total; ++c) Vout[c] = 0.5 * V[c] + 0.5 * (W1[c] + dt * L[c]);
        } else {
            for (int64_t c = 0; c < total; ++c)
                W2[c] = 0.75 * V[c] + 0.25 * (W1[c] + dt * L[c]);
            spatial_operator(P, scheme, alpha, W2, L, flags);
            for (int64_t c = 0; c < total; ++c)
                Vout[c] = V[c] / 3.0 + 2.0 * (W2[c] + dt * L[c]) / 3.0;
        }
    }
    const int discounted = gamma > 0.0 && gamma < 1.0;
    double dmax = 0.0;
    for (int64_t c = 0; c < total; ++c) {
        if (discounted) Vout[c] = gamma * Vout[c];
        if (!(flags & OR_BRS) && l[c] < Vout[c]) Vout[c] = l[c];
        double ch = fabs(Vout[c] - V[c]);
        if (ch > dmax) dmax = ch;
    }
    *delta = dmax;
    free(L);
    free(W1);
    free(W2);
    return 0;
}

/* Initial value: V(x,0) = l(x) (standard, Sec. II-B) or, for a warm start
 * k, V(x,0) = min(k(x), l(x)) (Sec. III, proof of Thm. 1, case b). */
void oracle_init(const oracle_problem* P, const double* l, const double* k, double* V) {
    int64_t total = oracle_num_cells(P);
    for (int64_t c = 0; c < total; ++c) V[c] = (k && k[c] < l[c]) ? k[c] : l[c];
}

/* The whole march: initialise, then step until max|dV| < tol + tol_rate dt
 * (converged), or tau >= horizon (horizon > 0), or max_steps steps
 * (max_steps > 0).  tol is a bound on the change per step; tol_rate bounds
 * the change per unit of time, which is how Sec. IV states its rule (a
 * change below 0.001 over a time step of 0.01: tol_rate = 0.1).
 * gamma (0 or 1: off) discounts every step as oracle_step says.
 * If `history` is not NULL it receives max|dV| of the first hist_len steps.
 * Returns 0 converged, 1 stopped without converging, -1 bad input. */
int oracle_solve(const oracle_problem* P, int scheme, int rk, double cfl, double tol,
                 double horizon, int64_t max_steps, const double* l, const double* k,
                 double* V, oracle_stats* st, double* history, int64_t hist_len,
                 double tol_rate, double interval, double interval_tol, int flags,
                 double gamma) {
    double alpha[OR_MAXD], dt;
    if (oracle_alpha_dt(P, cfl, alpha, &dt) != 0) return -1;
    int64_t total = oracle_num_cells(P);
    double* Vn = (double*)malloc(sizeof(double) * (size_t)total);
    if (!Vn) return -1;
    /* The interval test of Sec. V: the value counts as converged when its
     * largest change over one interval of `interval` time units (0.01 in
     * the paper's examples) is below interval_tol (0.001 there).  An
     * interval is K = max(1, round(interval / dt)) CFL steps; V is compared
     * with its copy from K steps earlier after every K-th step. */
    int64_t K = 0;
    double* snap = NULL;
    if (interval > 0.0) {
        K = (int64_t)llround(interval / dt);
        if (K < 1) K = 1;
        snap = (double*)malloc(sizeof(double) * (size_t)total);
        if (!snap) {
            free(Vn);
            return -1;
        }
    }
    /* With the projection off (Eq. (5) alone) a given start k is taken as
     * it is; otherwise V(x,0) = min(k, l) (Sec. III). */
    if ((flags & OR_BRS) && k) memcpy(V, k, sizeof(double) * (size_t)total);
    else oracle_init(P, l, k, V);
    if (snap) memcpy(snap, V, sizeof(double) * (size_t)total);
    double tau = 0.0, delta = INFINITY;
    int64_t steps = 0;
    int converged = 0;
    for (;;) {
        if (oracle_step(P, scheme, rk, dt, alpha, l, V, Vn, &delta, flags, gamma) != 0) {
            free(Vn);
            free(snap);
            return -1;
        }
        memcpy(V, Vn, sizeof(double) * (size_t)total);
        if (history && steps < hist_len) history[steps] = delta;
        steps += 1;
        tau += dt;
        if (delta < tol + tol_rate * dt) {
            converged = 1;
            break;
        }
        if (snap && steps % K == 0) {
            double change = 0.0;
            for (int64_t c = 0; c < total; ++c) {
                double ch = fabs(V[c] - snap[c]);
                if (ch > change) change = ch;
            }
            memcpy(snap, V, sizeof(double) * (size_t)total);
            if (change < interval_tol) {
                converged = 1;
                break;
            }
        }
        if (horizon > 0.0 && tau >= horizon) break;
        if (max_steps > 0 && steps >= max_steps) break;
    }
    free(snap);
    free(Vn);
    if (st) {
        st->steps = steps;
        st->tau = tau;
        st->dt = dt;
        st->last_delta = delta;
        st->converged = converged;
        for (int a = 0; a < OR_MAXD; ++a) st->alpha[a] = a < P->ndim ? alpha[a] : 0.0;
    }
    return converged ? 0 : 1;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}
