/*
 * amfrw_oracle.c -- plain, serial, double-precision CPU reference for the
 * AMFR-W2 time stepping of the SABR-LMM pricing PDE on the component grids of
 * the (standard or modified) sparse-grid combination technique.
 *
 * Paper: J.G. Lopez-Salas, S. Perez-Rodriguez, C. Vazquez, "AMFR-W numerical
 * methods for solving high dimensional SABR/LIBOR PDE models" (arXiv 2408.00559).
 *
 * TEST INFRASTRUCTURE.  This file is the oracle the CUDA path is checked
 * against.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline load it; the CUDA library never links or calls it, and the two
 * share no source, header, table or helper.
 *
 * How it is written.  Every routine follows one passage of the paper, cited
 * beside it, in the paper's own order and notation: the full grid including
 * the Dirichlet ("Outer") nodes, the index map theta_0 of Sec. 3, Sketch 1
 * evaluated node by node, the directional solves of Lemma "ls" / Algorithm 1
 * line by line with a plain Thomas elimination, and the AMFR-W stage recipe of
 * eq. (amfrw) with the AMFR-W2 coefficients of eq. (coef_W2).  There is no
 * blocking, fusion or algebraic rewriting.  Build with -O2 -ffp-contract=off
 * and without -ffast-math.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *  - the AMF parameter nu is an input (the paper's kappa_N table is external);
 *  - the sweep order prod_{i=N}^{1} applied to a vector is i = 1 first;
 *  - the drift sum in eq. (coef_adv) runs j = 2..i exactly as printed;
 *  - interpolation cell c_i = min(floor(x_i/h_i), M_i - 1);
 *  - rho_ii is taken from the supplied correlation matrix (unit diagonal).
 *
 * Axes are 0-based here: axis a = i-1 for the paper's F_i; axis N-1 is V.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 8

typedef struct {
    int32_t N;        /* spatial axes: N-1 forward rates and V (Sec. 2)        */
    int32_t payoff;   /* 0: caplet (F_1-K)^+ ; 1: swaption payoff of Sec. 2    */
    int32_t n_steps;  /* uniform time steps over [0,T]                         */
    int32_t bc;       /* 0: Neumann upper faces (Sketch 1); 1: the earlier
                         Dirichlet conditions of eq. (bound1_0): u = g also on
                         every face F_j = F_j^max of a rate                      */
    double alpha[ORC_MAXD];            /* alpha_i, rates 1..N-1                */
    double phi[ORC_MAXD];              /* phi_i rate/vol correlations          */
    double tau[ORC_MAXD];              /* accrual fractions tau_i              */
    double F0[ORC_MAXD];               /* spot point, rates 1..N-1             */
    double Fmax[ORC_MAXD];             /* domain bounds; entry N-1 is V^max    */
    double rho[ORC_MAXD * ORC_MAXD];   /* rho_ij, row-major, leading dim 8     */
    double sigma, beta, V0, K, T, theta, nu, discount;
} orc_params;

typedef struct {
    int N;
    int bc;               /* orc_params.bc                                      */
    int M[ORC_MAXD];      /* M_i: the grid has M_i+1 nodes on axis i          */
    long E[ORC_MAXD];     /* E_1 = 1, E_i = prod_{r<i} (M_r+1)   (Sec. 3)      */
    long size;            /* prod (M_i+1)                                      */
    double h[ORC_MAXD];   /* h_i = F_i^max / M_i                               */
} orc_grid;

static void grid_init(orc_grid *g, const orc_params *p, const int32_t *levels)
{
    g->N = p->N;
    g->bc = p->bc;
    g->size = 1;
    for (int i = 0; i < p->N; ++i) {
        g->M[i] = 1 << levels[i];
        g->E[i] = g->size;
        g->size *= (long)(g->M[i] + 1);
        g->h[i] = p->Fmax[i] / (double)g->M[i];
    }
}

/* Lemma "algor1": components of theta_0^{-1}(J) by repeated mod. */
static void decode(const orc_grid *g, long J, int *j)
{
    long c = J;
    for (int i = 0; i < g->N; ++i) {
        long q = c % (long)(g->M[i] + 1);
        j[i] = (int)q;
        c = (c - q) / (long)(g->M[i] + 1);
    }
}

/* Outer (Dirichlet) nodes: a lower face of any axis; under eq. (bound1_0) also
 * the upper face of every rate axis (V keeps dU/dV = 0 at V^max). */
static int is_outer(const orc_grid *g, const int *j)
{
    for (int i = 0; i < g->N; ++i) {
        if (j[i] == 0) return 1;
        if (g->bc && i < g->N - 1 && j[i] == g->M[i]) return 1;
    }
    return 0;
}

/* Payoffs of Sec. 2.  Caplet on F_1: (F_1 - K)^+ (the tau and discount factors
 * are applied to the price by the caller).  Swaption T_1 x (T_N - T_1):
 * g = max{ sum_i tau_i (F_i - K) / prod_{l<=i} (1 + tau_l F_l), 0 }. */
static double payoff(const orc_params *p, const double *F)
{
    if (p->payoff == 0) {
        double v = F[0] - p->K;
        return v > 0.0 ? v : 0.0;
    }
    double s = 0.0, P = 1.0;
    for (int i = 0; i < p->N - 1; ++i) {
        P *= (1.0 + p->tau[i] * F[i]);
        s += p->tau[i] * (F[i] - p->K) / P;
    }
    return s > 0.0 ? s : 0.0;
}

/* Phi_beta(x, tau) = tau x^beta / (1 + tau x), after eq. (coef_adv). */
static double Phi_beta(double beta, double x, double tau)
{
    return tau * pow(x, beta) / (1.0 + tau * x);
}

/* eq. (coef_diff): d_i at the node with coordinates F (F[N-1] = V). */
static double coef_d(const orc_params *p, int a, const double *F)
{
    int N = p->N;
    double V = F[N - 1];
    if (a < N - 1)
        return 0.5 * p->alpha[a] * p->alpha[a] * p->rho[a * ORC_MAXD + a]
               * pow(F[a], 2.0 * p->beta) * V * V;
    return 0.5 * p->sigma * p->sigma * V * V;
}

/* eq. (coef_mix): m_ik, a < k. */
static double coef_m(const orc_params *p, int a, int k, const double *F)
{
    int N = p->N;
    double V = F[N - 1];
    if (k < N - 1)
        return p->alpha[a] * p->alpha[k] * p->rho[a * ORC_MAXD + k]
               * pow(F[a], p->beta) * pow(F[k], p->beta) * V * V;
    return p->alpha[a] * p->sigma * p->phi[a] * pow(F[a], p->beta) * V * V;
}

/* eq. (coef_adv): a_i for rates i = 2..N-1 (0-based a = 1..N-2); the inner
 * sum runs over rates j = 2..i. */
static double coef_a(const orc_params *p, int a, const double *F)
{
    int N = p->N;
    double V = F[N - 1];
    double s = 0.0;
    for (int jr = 1; jr <= a; ++jr)
        s += p->alpha[a] * p->alpha[jr] * p->rho[a * ORC_MAXD + jr]
             * Phi_beta(p->beta, F[jr], p->tau[jr]);
    return s * pow(F[a], p->beta) * V * V;
}

static void coords(const orc_grid *g, const int *j, double *F)
{
    for (int i = 0; i < g->N; ++i) F[i] = (double)j[i] * g->h[i];
}

/* Sketch 1: Y'(t) = F(Y).  which < 0 gives the whole operator; which = i >= 0
 * gives only the directional part F_i of eq. (ffis), d_i Delta^(i). */
static void apply_F_part(const orc_params *p, const orc_grid *g, const double *Y,
                         double *out, int which)
{
    int N = g->N;
    int j[ORC_MAXD];
    double F[ORC_MAXD];
    for (long J = 0; J < g->size; ++J) {
        decode(g, J, j);
        if (is_outer(g, j)) { out[J] = 0.0; continue; }
        coords(g, j, F);
        double sum_d = 0.0, sum_m = 0.0, sum_a = 0.0;
        for (int i = 0; i < N; ++i) {
            if (which >= 0 && which != i) continue;
            long E = g->E[i];
            double h = g->h[i];
            double lap;
            if (j[i] != g->M[i])
                lap = (Y[J + E] - 2.0 * Y[J] + Y[J - E]) / (h * h);
            else
                lap = (2.0 * Y[J - E] - 2.0 * Y[J]) / (h * h);
            sum_d += coef_d(p, i, F) * lap;
        }
        if (which < 0) {
            for (int i = 0; i < N - 1; ++i)
                for (int k = i + 1; k < N; ++k) {
                    if (j[i] == g->M[i] || j[k] == g->M[k]) continue;
                    long Ei = g->E[i], Ek = g->E[k];
                    double mix = (Y[J + Ei + Ek] + Y[J - Ei - Ek]
                                  - Y[J + Ei - Ek] - Y[J - Ei + Ek])
                                 / (4.0 * g->h[i] * g->h[k]);
                    sum_m += coef_m(p, i, k, F) * mix;
                }
            for (int i = 1; i < N - 1; ++i) {
                if (j[i] == g->M[i]) continue;
                long E = g->E[i];
                double grad = (Y[J + E] - Y[J - E]) / (2.0 * g->h[i]);
                sum_a += coef_a(p, i, F) * grad;
            }
        }
        out[J] = sum_d + sum_m + sum_a;
    }
}

/* Lemma "ls" / Algorithm 1: solve (I - nu*dt*A_i) K = G for one axis.  Every
 * line of Inner nodes along the axis is a tridiagonal system (eq. decomp1):
 * row 1 has no sub-diagonal (its neighbour is Outer); the last row is the
 * Neumann face M_i with the doubled sub-diagonal of the ghost node, or, under
 * eq. (bound1_0) on a rate axis, row M_i - 1 whose upper neighbour is Outer
 * (no super-diagonal).  Outer rows are the identity.  Solved by Thomas
 * elimination (the matrix is strictly diagonally dominant).  K may alias G. */
static void line_solve(const orc_params *p, const orc_grid *g, int axis,
                       double nu_dt, const double *G, double *K)
{
    int N = g->N;
    int neumann = !(g->bc && axis < N - 1);
    int Mi = neumann ? g->M[axis] : g->M[axis] - 1;   /* Inner rows per line */
    long Ei = g->E[axis];
    if (K != G) memcpy(K, G, sizeof(double) * (size_t)g->size);
    if (Mi < 1) return;
    double *R = (double *)malloc(sizeof(double) * (size_t)Mi);
    double *lo = (double *)malloc(sizeof(double) * (size_t)Mi);
    double *di = (double *)malloc(sizeof(double) * (size_t)Mi);
    double *up = (double *)malloc(sizeof(double) * (size_t)Mi);
    double *cp = (double *)malloc(sizeof(double) * (size_t)Mi);
    int j[ORC_MAXD];
    double F[ORC_MAXD];
    double h2 = g->h[axis] * g->h[axis];
    /* every line start: the Inner node with j_axis = 1 */
    for (long J0 = 0; J0 < g->size; ++J0) {
        decode(g, J0, j);
        if (j[axis] != 1 || is_outer(g, j)) continue;
        for (int r = 1; r <= Mi; ++r) {
            long J = J0 + (long)(r - 1) * Ei;
            j[axis] = r;
            coords(g, j, F);
            double P = coef_d(p, axis, F) / h2;      /* (delta_i)_J */
            R[r - 1] = K[J];
            di[r - 1] = 1.0 + 2.0 * nu_dt * P;
            up[r - 1] = (r < Mi) ? -nu_dt * P : 0.0;
            if (r == 1)
                lo[r - 1] = 0.0;
            else if (r < Mi || !neumann)
                lo[r - 1] = -nu_dt * P;
            else
                lo[r - 1] = -2.0 * nu_dt * P;
        }
        /* Thomas: forward elimination, back substitution */
        cp[0] = up[0] / di[0];
        R[0] = R[0] / di[0];
        for (int r = 1; r < Mi; ++r) {
            double m = di[r] - lo[r] * cp[r - 1];
            cp[r] = up[r] / m;
            R[r] = (R[r] - lo[r] * R[r - 1]) / m;
        }
        for (int r = Mi - 2; r >= 0; --r) R[r] = R[r] - cp[r] * R[r + 1];
        for (int r = 1; r <= Mi; ++r) K[J0 + (long)(r - 1) * Ei] = R[r - 1];
    }
    free(R); free(lo); free(di); free(up); free(cp);
}

/* One AMFR-W step, eq. (row-s) with W from eq. (Wmat1) expanded as eq.
 * (amfrw), AMFR-W2 coefficients of eq. (coef_W2): s = 2, a21 = 2/3,
 * q21 = -4/3, b = (5/4, 3/4).  F'(Y_n) K is F(K) because the problem is
 * linear (end of Sec. 4.1). */
static void amfrw2_step(const orc_params *p, const orc_grid *g, double dt, double *Y)
{
    const int s = 2;
    const double A[2][2] = {{0.0, 0.0}, {2.0 / 3.0, 0.0}};
    const double Q[2][2] = {{0.0, 0.0}, {-4.0 / 3.0, 0.0}};
    const double b[2] = {5.0 / 4.0, 3.0 / 4.0};
    size_t n = (size_t)g->size;
    double *Kr[2];
    Kr[0] = (double *)malloc(sizeof(double) * n);
    Kr[1] = (double *)malloc(sizeof(double) * n);
    double *W = (double *)malloc(sizeof(double) * n);
    double *T = (double *)malloc(sizeof(double) * n);
    double *K0 = (double *)malloc(sizeof(double) * n);
    double *KN = (double *)malloc(sizeof(double) * n);
    double nu_dt = p->nu * dt;
    for (int r = 0; r < s; ++r) {
        /* K_r^(0) = dt F(Y_n + sum a_rj K_j) + sum q_rj K_j */
        for (size_t J = 0; J < n; ++J) {
            double w = Y[J];
            for (int jj = 0; jj < r; ++jj) w += A[r][jj] * Kr[jj][J];
            W[J] = w;
        }
        apply_F_part(p, g, W, T, -1);
        for (size_t J = 0; J < n; ++J) {
            double k = dt * T[J];
            for (int jj = 0; jj < r; ++jj) k += Q[r][jj] * Kr[jj][J];
            K0[J] = k;
        }
        /* (I - nu dt A_i) K^(i) = K^(i-1), i = 1..N */
        memcpy(KN, K0, sizeof(double) * n);
        for (int i = 0; i < g->N; ++i) line_solve(p, g, i, nu_dt, KN, KN);
        /* Khat^(0) = 2 K^(0) - (I - theta dt F'(Y_n)) K^(N) */
        apply_F_part(p, g, KN, T, -1);
        for (size_t J = 0; J < n; ++J)
            Kr[r][J] = 2.0 * K0[J] - (KN[J] - p->theta * dt * T[J]);
        /* (I - nu dt A_i) Khat^(i) = Khat^(i-1), i = 1..N; K_r = Khat^(N) */
        for (int i = 0; i < g->N; ++i) line_solve(p, g, i, nu_dt, Kr[r], Kr[r]);
    }
    for (size_t J = 0; J < n; ++J) {
        double y = Y[J];
        for (int r = 0; r < s; ++r) y += b[r] * Kr[r][J];
        Y[J] = y;
    }
    free(Kr[0]); free(Kr[1]); free(W); free(T); free(K0); free(KN);
}

/* The theta-method with a fixed number of Gauss-Seidel iterations, read as a
 * W-method (Sec. 4.2, eqs. thetamet and GS): eq. (row-s) with W = P, the lower
 * triangle (diagonal included) of A = F'(Y) in the node order of theta_0,
 * a_rj = theta, q_rj = -1, b_r = 1 and s = s_iter stages:
 *   (I - theta dt P) K_r = dt F(Y_n + theta sum_{j<r} K_j) - sum_{j<r} K_j,
 *   Y_{n+1} = Y_n + sum_r K_r.
 * A (n x n, row-major) is the dense matrix of the linear map F; each stage's
 * triangular system is solved by forward substitution in node order. */
static void theta_gs_step(const orc_params *p, const orc_grid *g, const double *A, double dt,
                          int s_iter, double *Y)
{
    size_t n = (size_t)g->size;
    double *sumK = (double *)calloc(n, sizeof(double));
    double *W = (double *)malloc(sizeof(double) * n);
    double *T = (double *)malloc(sizeof(double) * n);
    double *Kr = (double *)malloc(sizeof(double) * n);
    double th = p->theta;
    for (int r = 0; r < s_iter; ++r) {
        for (size_t J = 0; J < n; ++J) W[J] = Y[J] + th * sumK[J];
        apply_F_part(p, g, W, T, -1);
        for (size_t J = 0; J < n; ++J) {
            double v = dt * T[J] - sumK[J];
            for (size_t c = 0; c < J; ++c) v += th * dt * A[J * n + c] * Kr[c];
            Kr[J] = v / (1.0 - th * dt * A[J * n + J]);
        }
        for (size_t J = 0; J < n; ++J) sumK[J] += Kr[J];
    }
    for (size_t J = 0; J < n; ++J) Y[J] += sumK[J];
    free(sumK); free(W); free(T); free(Kr);
}

/* Multilinear interpolation of the grid function Y at x (Sec. 5.1, Sec. 6). */
static double interp(const orc_grid *g, const double *Y, const double *x)
{
    int N = g->N;
    int c[ORC_MAXD];
    double w[ORC_MAXD];
    for (int i = 0; i < N; ++i) {
        double sx = x[i] / g->h[i];
        int ci = (int)floor(sx);
        if (ci > g->M[i] - 1) ci = g->M[i] - 1;
        if (ci < 0) ci = 0;
        c[i] = ci;
        w[i] = sx - (double)ci;
    }
    double u = 0.0;
    for (int corner = 0; corner < (1 << N); ++corner) {
        double wt = 1.0;
        long J = 0;
        for (int i = 0; i < N; ++i) {
            int bit = (corner >> i) & 1;
            wt *= bit ? w[i] : (1.0 - w[i]);
            J += (long)(c[i] + bit) * g->E[i];
        }
        u += wt * Y[J];
    }
    return u;
}

static void spot(const orc_params *p, double *x)
{
    for (int i = 0; i < p->N - 1; ++i) x[i] = p->F0[i];
    x[p->N - 1] = p->V0;
}

/* ---------------------------------------------------------------- exports */

long orc_grid_size(int32_t N, const int32_t *levels)
{
    long s = 1;
    for (int i = 0; i < N; ++i) s *= (long)((1 << levels[i]) + 1);
    return s;
}

/* Y = g on every node; Y_J for J in Outer stays g for the whole run (eq. dis0). */
void orc_payoff_grid(const orc_params *p, const int32_t *levels, double *Y)
{
    orc_grid g;
    grid_init(&g, p, levels);
    int j[ORC_MAXD];
    double F[ORC_MAXD];
    for (long J = 0; J < g.size; ++J) {
        decode(&g, J, j);
        coords(&g, j, F);
        Y[J] = payoff(p, F);
    }
}

void orc_apply_F(const orc_params *p, const int32_t *levels, const double *Y, double *out)
{
    orc_grid g;
    grid_init(&g, p, levels);
    apply_F_part(p, &g, Y, out, -1);
}

void orc_apply_Fi(const orc_params *p, const int32_t *levels, int32_t axis,
                  const double *Y, double *out)
{
    orc_grid g;
    grid_init(&g, p, levels);
    apply_F_part(p, &g, Y, out, axis);
}

void orc_line_solve(const orc_params *p, const int32_t *levels, int32_t axis,
                    double nu_dt, const double *G, double *K)
{
    orc_grid g;
    grid_init(&g, p, levels);
    line_solve(p, &g, axis, nu_dt, G, K);
}

/* n_steps AMFR-W2 steps of size dt = T / p->n_steps, starting from Y (in/out). */
void orc_run(const orc_params *p, const int32_t *levels, double *Y, int32_t n_steps)
{
    orc_grid g;
    grid_init(&g, p, levels);
    double dt = p->T / (double)p->n_steps;
    for (int n = 0; n < n_steps; ++n) amfrw2_step(p, &g, dt, Y);
}

/* n_steps steps of the theta-method + Gauss-Seidel W-method with s_iter
 * iterations, dt = T / p->n_steps, theta = p->theta, starting from Y
 * (in/out).  The dense matrix of F is assembled column by column, F(e_c), so
 * the grid may have at most 4096 nodes; returns -1 (Y untouched) beyond. */
int32_t orc_run_theta_gs(const orc_params *p, const int32_t *levels, double *Y, int32_t n_steps,
                         int32_t s_iter)
{
    orc_grid g;
    grid_init(&g, p, levels);
    size_t n = (size_t)g.size;
    if (n > 4096 || s_iter < 1) return -1;
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *e = (double *)calloc(n, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * n);
    for (size_t c = 0; c < n; ++c) {
        e[c] = 1.0;
        apply_F_part(p, &g, e, col, -1);
        e[c] = 0.0;
        for (size_t J = 0; J < n; ++J) A[J * n + c] = col[J];
    }
    double dt = p->T / (double)p->n_steps;
    for (int k = 0; k < n_steps; ++k) theta_gs_step(p, &g, A, dt, s_iter, Y);
    free(A); free(e); free(col);
    return 0;
}

double orc_interp(const orc_params *p, const int32_t *levels, const double *Y,
                  const double *x)
{
    orc_grid g;
    grid_init(&g, p, levels);
    return interp(&g, Y, x);
}

/* One component grid: Y = g, p->n_steps AMFR-W2 steps, value at the spot.
 * If Y_out is non-NULL it receives the final grid function (full grid). */
double orc_solve_grid(const orc_params *p, const int32_t *levels, double *Y_out)
{
    orc_grid g;
    grid_init(&g, p, levels);
    double *Y = (double *)malloc(sizeof(double) * (size_t)g.size);
    orc_payoff_grid(p, levels, Y);
    double dt = p->T / (double)p->n_steps;
    for (int n = 0; n < p->n_steps; ++n) amfrw2_step(p, &g, dt, Y);
    double x[ORC_MAXD];
    spot(p, x);
    double u = interp(&g, Y, x);
    if (Y_out) memcpy(Y_out, Y, sizeof(double) * (size_t)g.size);
    free(Y);
    return u;
}

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* Component grids and coefficients of eq. (standardCombTechnique) (psi = 0)
 * and eq. (modifiedCombTechnique) (psi >= 1): for q = 0..d-1 every l in N_0^d
 * with |l|_1 = n - q, coefficient (-1)^q C(d-1, q), levels psi + l_i.
 * full != 0: the single full grid with level n on every axis.  Returns the
 * number of grids; levels/coefs may be NULL to only count. */
int32_t orc_enumerate(int32_t d, int32_t n, int32_t psi, int32_t full,
                      int32_t *levels, double *coefs)
{
    if (full) {
        if (levels)
            for (int i = 0; i < d; ++i) levels[i] = n;
        if (coefs) coefs[0] = 1.0;
        return 1;
    }
    int count = 0;
    int l[ORC_MAXD];
    for (int q = 0; q < d; ++q) {
        int m = n - q;
        if (m < 0) continue;
        double c = ((q & 1) ? -1.0 : 1.0) * binom(d - 1, q);
        /* odometer over l_0..l_{d-2} in [0, m], l_{d-1} = m - sum */
        for (int i = 0; i < d; ++i) l[i] = 0;
        for (;;) {
            int s = 0;
            for (int i = 0; i < d - 1; ++i) s += l[i];
            if (s <= m) {
                l[d - 1] = m - s;
                if (levels)
                    for (int i = 0; i < d; ++i) levels[count * d + i] = psi + l[i];
                if (coefs) coefs[count] = c;
                ++count;
            }
            int i = 0;
            while (i < d - 1) {
                if (++l[i] <= m) break;
                l[i] = 0;
                ++i;
            }
            if (i >= d - 1) break;
        }
    }
    return count;
}

/* Price by the combination technique: discount * sum_l c_l u_l(x*).
 * per_grid_u (optional) receives u_l(x*) in enumeration order. */
double orc_price(const orc_params *p, int32_t n, int32_t psi, int32_t full,
                 double *per_grid_u)
{
    int d = p->N;
    int ng = orc_enumerate(d, n, psi, full, NULL, NULL);
    int32_t *lv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ng * d));
    double *cf = (double *)malloc(sizeof(double) * (size_t)ng);
    orc_enumerate(d, n, psi, full, lv, cf);
    double sum = 0.0;
    for (int k = 0; k < ng; ++k) {
        double u = orc_solve_grid(p, lv + k * d, NULL);
        if (per_grid_u) per_grid_u[k] = u;
        sum += cf[k] * u;
    }
    free(lv);
    free(cf);
    return p->discount * sum;
}
