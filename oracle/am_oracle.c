/*
 * am_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, scalar CPU implementation of the batched alternating-
 * minimization (AM) trajectory optimizer of Rastgar's thesis, Paper II
 * (Algorithm 2), with the projection-mode cost of Paper III (PRIEST projection
 * optimizer, eqs. projection_cost, affine_trans, matrix_vec). It exists only to
 * check the CUDA path: only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code with the CUDA library.
 *
 * Precision: REAL is double by default (the FP64 oracle). Compiling with
 * -DORACLE_REAL_FLOAT gives a float instantiation of the very same steps, used
 * only to tell rounding amplification apart from kernel bugs.
 *
 * Everything is literal: the dense constraint matrix F is built by stacking
 * (P repeated n_o times, then Pdot, then Pddot) per axis; the KKT matrix is
 * inverted by Gauss-Jordan elimination with partial pivoting; the angle steps
 * call atan2/cos/sin; the multiplier update multiplies by F^T explicitly.
 *
 * Readings of passages where the paper is silent, garbled or inconsistent
 * (each also listed in the design notes):
 *  R1 xi-step right-hand side is -q + lambda + rho F^T g (eq. zeta_1_sepration_3
 *     prints the opposite sign, which contradicts the augmented Lagrangian of
 *     eq. reform_formulation); one rho for all constraint groups.
 *  R2 multiplier update lambda <- lambda - rho F^T (F xi - g) (eq.
 *     update_lambda2_1 is dimensionally garbled; eq. lag of PRIEST has this form).
 *  R3 Algorithm 2 order (xi, alpha, d, lambda) in both cost modes; d, alpha are
 *     initialised by projecting xi0 and lambda0 = 0.
 *  R4 obstacle angles use coordinates normalised by the semi-axes:
 *     alpha = atan2(y~/b, x~/a); 3D beta = atan2(hypot(x~/a, y~/b), z~/c).
 *  R5 velocity/acceleration targets carry v_max / a_max (eq. fv, fa); d_v, d_a
 *     are minimised over [0, 1].
 *  R6 atan2(0, 0) = 0 (IEEE), i.e. a point at an obstacle centre is pushed +x.
 *  R7 Bernstein degree 10 on tau_t = t/(n_p-1), t = 0..n_p-1; time derivatives
 *     scale by 1/T and 1/T^2.
 *  R8 boundary rows: start position, velocity, acceleration and goal position
 *     (PRIEST eq. eq1_multiagent_1_priest with b0 = (start, 0, 0), bf = goal).
 *  R9 residuals are L-infinity over the grid points: max_{j,t} ||p - g_j||,
 *     max_t ||pdot - g_v||, max_t ||pddot - g_a||.
 *  R11 workspace bounds (PRIEST eqs. bound_con, lagrange): G = [-P; P] per axis,
 *     tau = [-lo; hi], slack s = max(0, tau - G xi) from the current iterate, and
 *     the rows' target e = tau - s; their residual norms join the obstacle group's
 *     maximum (column 0).
 *  R12 receding horizon (Paper II's MPC: the multipliers carried from one control
 *     loop to the next): the boundary rows take a start velocity and
 *     acceleration (start_va, NULL = zero, as in R8), and the loop may start from
 *     imported multipliers lam0 (NULL = 0): the initial projection is unchanged
 *     and lam0 replaces lambda0 = 0.
 *  R10 penalty continuation (Paper I, Algorithm 1 line 9; Paper IV's ten cached
 *     KKT inverses): penalties rho growth^l, l = 0 .. levels-1, each with its own
 *     KKT inverse; after iteration k >= 1, if the trajectory has not stopped and k
 *     is a multiple of rho_every, the next iteration uses the next level (up to
 *     the last). The level's rho enters the xi-step and the multiplier update.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_REAL_FLOAT
typedef float REAL;
#define R_ATAN2 atan2f
#define R_COS cosf
#define R_SIN sinf
#define R_SQRT sqrtf
#define R_HYPOT hypotf
#define R_FABS fabsf
#else
typedef double REAL;
#define R_ATAN2 atan2
#define R_COS cos
#define R_SIN sin
#define R_SQRT sqrt
#define R_HYPOT hypot
#define R_FABS fabs
#endif

#define NC 11 /* coefficients per axis: Bernstein degree 10 */
#define NE 4  /* boundary rows per axis */
#define NK (NC + NE)

/* ------------------------------------------------------------------------- */
/* Basis (eq. parameter; Remark on the Bernstein choice).                     */
/* ------------------------------------------------------------------------- */
static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

/* B^n_i(tau) = C(n,i) tau^i (1-tau)^(n-i); zero outside 0..n. */
static double bern(int n, int i, double tau) {
  if (i < 0 || i > n) return 0.0;
  return binom(n, i) * pow(tau, (double)i) * pow(1.0 - tau, (double)(n - i));
}

/* P, Pdot, Pddot as row-major [n_p][11] (reading R7). The derivative of a
 * degree-n Bernstein polynomial is n times a difference of degree n-1 ones. */
void orc_bernstein(int n_p, double T, double *P, double *Pd, double *Pdd) {
  const int n = NC - 1;
  for (int t = 0; t < n_p; ++t) {
    double tau = (n_p > 1) ? (double)t / (double)(n_p - 1) : 0.0;
    for (int i = 0; i < NC; ++i) {
      P[t * NC + i] = bern(n, i, tau);
      Pd[t * NC + i] = n * (bern(n - 1, i - 1, tau) - bern(n - 1, i, tau)) / T;
      Pdd[t * NC + i] = n * (n - 1) *
                        (bern(n - 2, i - 2, tau) - 2.0 * bern(n - 2, i - 1, tau) +
                         bern(n - 2, i, tau)) / (T * T);
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Gauss-Jordan inverse with partial pivoting (for eq. qp_sol / over_3).      */
/* Returns 0 on success, -1 if a pivot vanishes.                              */
/* ------------------------------------------------------------------------- */
int orc_invert(int n, const double *A, double *Ainv) {
  double *W = (double *)malloc(sizeof(double) * n * 2 * n);
  if (!W) return -2;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      W[r * 2 * n + c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(W[r * 2 * n + col]) > fabs(W[piv * 2 * n + col])) piv = r;
    if (W[piv * 2 * n + col] == 0.0) { free(W); return -1; }
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double tmp = W[col * 2 * n + c];
        W[col * 2 * n + c] = W[piv * 2 * n + c];
        W[piv * 2 * n + c] = tmp;
      }
    double inv = 1.0 / W[col * 2 * n + col];
    for (int c = 0; c < 2 * n; ++c) W[col * 2 * n + c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = W[r * 2 * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) W[r * 2 * n + c] -= f * W[col * 2 * n + c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = W[r * 2 * n + n + c];
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Problem description shared by the solver entry points.                     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int dim;         /* 2 or 3 */
  int n_p;         /* timesteps */
  double T;        /* horizon, s */
  int n_o;         /* obstacles */
  const double *centers, *semi_axes, *velocities; /* [n_o][dim] */
  const double *start, *goal;                      /* [dim] */
  double vmax, amax, rho, w_smooth, w_track;
  int cost_mode;   /* 0: smoothness + tracking (eq. Q_matrix); 1: projection (eq. matrix_vec) */
  const double *box_lo, *box_hi; /* [dim] workspace bounds (reading R11) or NULL */
  int rho_levels;  /* penalty continuation (reading R10); 1 or 0: a fixed rho */
  double rho_growth;
  int rho_every;
  const double *start_va; /* [2][dim] start velocity, then acceleration (R12), or NULL */
} orc_problem;

/* Dense F for one axis: (n_o + 2) n_p rows x 11 (F of Paper II without the
 * heading rows; F~ of eq. f_e per axis). Row j*n_p + t is P[t] (obstacle j),
 * row n_o*n_p + t is Pdot[t], row (n_o+1)*n_p + t is Pddot[t]. */
static void build_F(int n_p, int n_o, int box, const double *P, const double *Pd,
                    const double *Pdd, double *F) {
  for (int j = 0; j < n_o; ++j)
    for (int t = 0; t < n_p; ++t)
      memcpy(&F[((size_t)j * n_p + t) * NC], &P[t * NC], sizeof(double) * NC);
  memcpy(&F[(size_t)n_o * n_p * NC], Pd, sizeof(double) * n_p * NC);
  memcpy(&F[(size_t)(n_o + 1) * n_p * NC], Pdd, sizeof(double) * n_p * NC);
  if (box) /* workspace rows: -P (lower bounds), then P (upper bounds) (reading R11) */
    for (int t = 0; t < n_p; ++t)
      for (int i = 0; i < NC; ++i) {
        F[((size_t)(n_o + 2) * n_p + t) * NC + i] = -P[t * NC + i];
        F[((size_t)(n_o + 3) * n_p + t) * NC + i] = P[t * NC + i];
      }
}

/* KKT matrix K = [[Q + rho F^T F, A^T], [A, 0]] (eq. over_2 with eq.
 * zeta_1_sepration_3's Q-bar; eq. matrix_vec in projection mode). Q is the
 * same for every axis (block-diagonal D-bar, eq. simple), so one 15x15 K
 * serves all axes. Writes K (15x15) and its inverse; returns orc_invert's code. */
int orc_kkt(const orc_problem *pr, double *K, double *Kinv) {
  const int n_p = pr->n_p, n_o = pr->n_o, box = pr->box_lo != NULL;
  const size_t rows = (size_t)(n_o + 2 + 2 * box) * n_p;
  double *P = malloc(sizeof(double) * n_p * NC), *Pd = malloc(sizeof(double) * n_p * NC),
         *Pdd = malloc(sizeof(double) * n_p * NC), *F = malloc(sizeof(double) * rows * NC);
  orc_bernstein(n_p, pr->T, P, Pd, Pdd);
  build_F(n_p, n_o, box, P, Pd, Pdd, F);
  memset(K, 0, sizeof(double) * NK * NK);
  for (int a = 0; a < NC; ++a)
    for (int b = 0; b < NC; ++b) {
      double Q = 0.0;
      if (pr->cost_mode == 0) {
        for (int t = 0; t < n_p; ++t)
          Q += pr->w_smooth * Pdd[t * NC + a] * Pdd[t * NC + b] +
               pr->w_track * P[t * NC + a] * P[t * NC + b];
      } else {
        Q = (a == b) ? 1.0 : 0.0;
      }
      double FtF = 0.0;
      for (size_t r = 0; r < rows; ++r) FtF += F[r * NC + a] * F[r * NC + b];
      K[a * NK + b] = Q + pr->rho * FtF;
    }
  /* A = [P_0; Pdot_0; Pddot_0; P_{-1}] (reading R8) */
  const double *Arow[NE] = {&P[0], &Pd[0], &Pdd[0], &P[(n_p - 1) * NC]};
  for (int e = 0; e < NE; ++e)
    for (int b = 0; b < NC; ++b) {
      K[(NC + e) * NK + b] = Arow[e][b];
      K[b * NK + NC + e] = Arow[e][b];
    }
  int rc = orc_invert(NK, K, Kinv);
  free(P); free(Pd); free(Pdd); free(F);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Closed-form alpha/beta/d steps for one point (eqs. zeta_2, compute_d_mij,  */
/* d_max; 3D eqs. collision_priest, comp_alpha-comp_d). Given the offset      */
/* x~ = p - o and semi-axes (a_0..a_{dim-1}), writes the target offset        */
/* g - o = d * (a cos(alpha) sin(beta), ...). Exposed for the pin tests.      */
/* ------------------------------------------------------------------------- */
void orc_project_obstacle(int dim, const REAL *xt, const REAL *ax, REAL *goff) {
  if (dim == 2) {
    REAL alpha = R_ATAN2(xt[1] / ax[1], xt[0] / ax[0]);            /* R4 */
    REAL ca = R_COS(alpha), sa = R_SIN(alpha);
    /* d-step: least-squares minimiser of ||x~ - d (a ca, b sa)|| with d >= 1 */
    REAL d = (ax[0] * xt[0] * ca + ax[1] * xt[1] * sa) /
             (ax[0] * ax[0] * ca * ca + ax[1] * ax[1] * sa * sa);
    if (d < 1) d = 1;
    goff[0] = ax[0] * d * ca;
    goff[1] = ax[1] * d * sa;
  } else {
    REAL ux = xt[0] / ax[0], uy = xt[1] / ax[1], uz = xt[2] / ax[2];
    REAL alpha = R_ATAN2(uy, ux);                                    /* R4 */
    REAL beta = R_ATAN2(R_HYPOT(ux, uy), uz);
    REAL ca = R_COS(alpha), sa = R_SIN(alpha), cb = R_COS(beta), sb = R_SIN(beta);
    REAL e0 = ax[0] * ca * sb, e1 = ax[1] * sa * sb, e2 = ax[2] * cb;
    REAL d = (xt[0] * e0 + xt[1] * e1 + xt[2] * e2) / (e0 * e0 + e1 * e1 + e2 * e2);
    if (d < 1) d = 1;
    goff[0] = d * e0; goff[1] = d * e1; goff[2] = d * e2;
  }
}

/* Velocity / acceleration steps (eqs. alpha_v, alpha_a, compute_dv, compute_da;
 * 3D eqs. fv_priest, fa_priest): angle(s) of the vector, then the least-squares
 * d over [0, 1] (reading R5), target = d * bound * direction. */
void orc_project_bound(int dim, const REAL *w, REAL bound, REAL *g) {
  if (dim == 2) {
    REAL alpha = R_ATAN2(w[1], w[0]);
    REAL ca = R_COS(alpha), sa = R_SIN(alpha);
    REAL d = (w[0] * ca + w[1] * sa) / bound;
    if (d < 0) d = 0;
    if (d > 1) d = 1;
    g[0] = d * bound * ca;
    g[1] = d * bound * sa;
  } else {
    REAL alpha = R_ATAN2(w[1], w[0]);
    REAL beta = R_ATAN2(R_HYPOT(w[0], w[1]), w[2]);
    REAL ca = R_COS(alpha), sa = R_SIN(alpha), cb = R_COS(beta), sb = R_SIN(beta);
    REAL e0 = ca * sb, e1 = sa * sb, e2 = cb;
    REAL d = (w[0] * e0 + w[1] * e1 + w[2] * e2) / bound;
    if (d < 0) d = 0;
    if (d > 1) d = 1;
    g[0] = d * bound * e0; g[1] = d * bound * e1; g[2] = d * bound * e2;
  }
}

/* ------------------------------------------------------------------------- */
/* The AM loop (Algorithm 2) for n_traj trajectories of one problem.          */
/*                                                                            */
/* xi0[n_traj][dim][11]; lam0 (same shape, nullable: zero) the multipliers the */
/* loop starts from; outputs xi_out (same shape), lam_out (same shape,        */
/* nullable), residual_out[n_traj][3], iters_out[n_traj].                     */
/* iters_fixed (nullable): run exactly iters_fixed[b] iterations, no test.    */
/* Otherwise stop after the first iteration k >= 1 whose three residuals are  */
/* all <= tol (tol < 0 never stops early), or at max_iters.                   */
/* hist (nullable): residuals after init and after every iteration,           */
/* [n_traj][max_iters + 1][3] (entries past the stop are left untouched).     */
/* Returns 0, or a negative code for a singular KKT matrix / bad arguments.   */
/* ------------------------------------------------------------------------- */
int orc_am_solve(const orc_problem *pr, int n_traj, const double *xi0, const double *lam0,
                 int max_iters, double tol, const int *iters_fixed, double *xi_out,
                 double *lam_out, double *residual_out, int *iters_out, double *hist,
                 int n_threads) {
  const int dim = pr->dim, n_p = pr->n_p, n_o = pr->n_o, box = pr->box_lo != NULL;
  if (dim < 2 || dim > 3 || n_p < 2 || n_o < 0 || max_iters < 0) return -3;
  const size_t rows = (size_t)(n_o + 2 + 2 * box) * n_p;
  double *P = malloc(sizeof(double) * n_p * NC), *Pd = malloc(sizeof(double) * n_p * NC),
         *Pdd = malloc(sizeof(double) * n_p * NC), *F = malloc(sizeof(double) * rows * NC);
  const int levels = pr->rho_levels > 1 ? pr->rho_levels : 1;
  if (levels > 16) { free(P); free(Pd); free(Pdd); free(F); return -3; }
  double K[NK * NK], Kinv[16][NK * NK], rho_l[16];
  orc_bernstein(n_p, pr->T, P, Pd, Pdd);
  build_F(n_p, n_o, box, P, Pd, Pdd, F);
  for (int l = 0; l < levels; ++l) { /* one KKT inverse per penalty level (reading R10) */
    orc_problem pl = *pr;
    pl.rho = pr->rho * pow(pr->rho_growth, (double)l);
    rho_l[l] = pl.rho;
    if (orc_kkt(&pl, K, Kinv[l])) { free(P); free(Pd); free(Pdd); free(F); return -1; }
  }

  /* q per axis (eq. Q_matrix: q = -w_t P^T x_des, x_des the constant-velocity
   * straight line); b per axis = (start, v0, a0, goal) with v0 = a0 = 0 (reading
   * R8) unless a start state is given (reading R12). */
  double qa[3][NC], ba[3][NE];
  for (int a = 0; a < dim; ++a) {
    for (int i = 0; i < NC; ++i) {
      double s = 0.0;
      for (int t = 0; t < n_p; ++t) {
        double tau = (double)t / (double)(n_p - 1);
        double xdes = pr->start[a] + (pr->goal[a] - pr->start[a]) * tau;
        s += P[t * NC + i] * xdes;
      }
      qa[a][i] = -pr->w_track * s;
    }
    ba[a][0] = pr->start[a];
    ba[a][1] = pr->start_va ? pr->start_va[a] : 0.0;
    ba[a][2] = pr->start_va ? pr->start_va[dim + a] : 0.0;
    ba[a][3] = pr->goal[a];
  }
  double *tgrid = malloc(sizeof(double) * n_p);
  for (int t = 0; t < n_p; ++t) tgrid[t] = pr->T * (double)t / (double)(n_p - 1);

#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < n_traj; ++b) {
    REAL *xi = malloc(sizeof(REAL) * dim * NC), *lam = malloc(sizeof(REAL) * dim * NC);
    REAL *Fx = malloc(sizeof(REAL) * dim * rows), *g = malloc(sizeof(REAL) * dim * rows);
    REAL *Kall = malloc(sizeof(REAL) * levels * NK * NK), *Fr = malloc(sizeof(REAL) * rows * NC);
    for (int l = 0; l < levels; ++l)
      for (int k = 0; k < NK * NK; ++k) Kall[l * NK * NK + k] = (REAL)Kinv[l][k];
    int level = 0;
    REAL *Kr = Kall;
    REAL rho = (REAL)rho_l[0];
    for (size_t k = 0; k < rows * NC; ++k) Fr[k] = (REAL)F[k];
    for (int k = 0; k < dim * NC; ++k) {
      xi[k] = (REAL)xi0[(size_t)b * dim * NC + k];
      lam[k] = lam0 ? (REAL)lam0[(size_t)b * dim * NC + k] : 0; /* R3, or R12's carry */
    }
    /* projection mode (eq. matrix_vec): Q = I, q = -xi_sample, the trajectory's own xi0 */
    REAL q[3][NC];
    for (int a = 0; a < dim; ++a)
      for (int i = 0; i < NC; ++i)
        q[a][i] = pr->cost_mode == 0 ? (REAL)qa[a][i] : -(REAL)xi0[((size_t)b * dim + a) * NC + i];

    REAL res[3] = {0, 0, 0};
    int fixed = iters_fixed ? iters_fixed[b] : -1;
    int limit = fixed >= 0 ? fixed : max_iters;
    int k_done = 0;
    for (int k = 0; k <= limit; ++k) {
      if (k > 0) {
        /* Line 2 -- xi-step (eq. zeta_1_sepration_1 solved via eq. over_3):
         * xi = Kinv[0:11, :] [-q + lambda + rho F^T g; b] (reading R1). */
        for (int a = 0; a < dim; ++a) {
          REAL rhs[NK];
          for (int i = 0; i < NC; ++i) {
            REAL Ftg = 0;
            for (size_t r = 0; r < rows; ++r) Ftg += Fr[r * NC + i] * g[a * rows + r];
            rhs[i] = -q[a][i] + lam[a * NC + i] + rho * Ftg;
          }
          for (int e = 0; e < NE; ++e) rhs[NC + e] = (REAL)ba[a][e];
          for (int i = 0; i < NC; ++i) {
            REAL s = 0;
            for (int c = 0; c < NK; ++c) s += Kr[i * NK + c] * rhs[c];
            xi[a * NC + i] = s;
          }
        }
      }
      /* F xi: positions (repeated per obstacle), velocities, accelerations */
      for (int a = 0; a < dim; ++a)
        for (size_t r = 0; r < rows; ++r) {
          REAL s = 0;
          for (int i = 0; i < NC; ++i) s += Fr[r * NC + i] * xi[a * NC + i];
          Fx[a * rows + r] = s;
        }
      /* Lines 4-5 -- alpha- and d-steps, giving g (eqs. zeta_2, alpha_v, alpha_a,
       * compute_d_mij, compute_dv, compute_da; 3D: comp_alpha, comp_beta, comp_d). */
      res[0] = res[1] = res[2] = 0;
      for (int j = 0; j < n_o; ++j) {
        REAL ax[3];
        for (int a = 0; a < dim; ++a) ax[a] = (REAL)pr->semi_axes[j * dim + a];
        for (int t = 0; t < n_p; ++t) {
          size_t r = (size_t)j * n_p + t;
          REAL o[3], xt[3], goff[3], nrm = 0;
          for (int a = 0; a < dim; ++a) {
            o[a] = (REAL)(pr->centers[j * dim + a] + pr->velocities[j * dim + a] * tgrid[t]);
            xt[a] = Fx[a * rows + r] - o[a];
          }
          orc_project_obstacle(dim, xt, ax, goff);
          for (int a = 0; a < dim; ++a) {
            g[a * rows + r] = o[a] + goff[a];
            REAL e = Fx[a * rows + r] - g[a * rows + r];
            nrm += e * e;
          }
          nrm = R_SQRT(nrm);
          if (nrm > res[0]) res[0] = nrm;
        }
      }
      for (int grp = 0; grp < 2; ++grp) {
        REAL bound = grp == 0 ? (REAL)pr->vmax : (REAL)pr->amax;
        for (int t = 0; t < n_p; ++t) {
          size_t r = (size_t)(n_o + grp) * n_p + t;
          REAL w[3], gv[3], nrm = 0;
          for (int a = 0; a < dim; ++a) w[a] = Fx[a * rows + r];
          orc_project_bound(dim, w, bound, gv);
          for (int a = 0; a < dim; ++a) {
            g[a * rows + r] = gv[a];
            REAL e = w[a] - gv[a];
            nrm += e * e;
          }
          nrm = R_SQRT(nrm);
          if (nrm > res[1 + grp]) res[1 + grp] = nrm;
        }
      }
      /* workspace rows (reading R11): slack s = max(0, tau - G xi), target tau - s */
      if (box)
        for (int t = 0; t < n_p; ++t) {
          REAL nrm = 0;
          for (int side = 0; side < 2; ++side)
            for (int a = 0; a < dim; ++a) {
              size_t r = (size_t)(n_o + 2 + side) * n_p + t;
              REAL tau = side == 0 ? -(REAL)pr->box_lo[a] : (REAL)pr->box_hi[a];
              REAL sl = tau - Fx[a * rows + r];
              if (sl < 0) sl = 0;
              g[a * rows + r] = tau - sl;
              REAL e = Fx[a * rows + r] - g[a * rows + r];
              nrm += e * e;
            }
          nrm = R_SQRT(nrm);
          if (nrm > res[0]) res[0] = nrm;
        }
      /* Line 6 -- multiplier update lambda <- lambda - rho F^T (F xi - g) (reading R2).
       * At k = 0 (initialisation) lambda keeps its initial value (0, or the carried
       * multipliers of R12) and only g0 is formed (reading R3). */
      if (k > 0)
        for (int a = 0; a < dim; ++a)
          for (int i = 0; i < NC; ++i) {
            REAL s = 0;
            for (size_t r = 0; r < rows; ++r)
              s += Fr[r * NC + i] * (Fx[a * rows + r] - g[a * rows + r]);
            lam[a * NC + i] -= rho * s;
          }
      if (hist)
        for (int c = 0; c < 3; ++c) hist[((size_t)b * (max_iters + 1) + k) * 3 + c] = res[c];
      k_done = k;
      if (fixed < 0 && k > 0 && tol >= 0 && res[0] <= tol && res[1] <= tol && res[2] <= tol)
        break;
      /* penalty continuation (reading R10): not stopped after iteration k */
      if (k > 0 && pr->rho_every > 0 && level + 1 < levels && k % pr->rho_every == 0) {
        ++level;
        Kr = Kall + (size_t)level * NK * NK;
        rho = (REAL)rho_l[level];
      }
    }
    for (int k = 0; k < dim * NC; ++k) {
      xi_out[(size_t)b * dim * NC + k] = xi[k];
      if (lam_out) lam_out[(size_t)b * dim * NC + k] = lam[k];
    }
    for (int c = 0; c < 3; ++c) residual_out[(size_t)b * 3 + c] = res[c];
    iters_out[b] = k_done;
    free(xi); free(lam); free(Fx); free(g); free(Kall); free(Fr);
  }
  free(P); free(Pd); free(Pdd); free(F); free(tgrid);
  return 0;
}

/* Flat-argument wrapper (plain pointers, callable through ctypes). */
int orc_am_solve_flat(int dim, int n_p, double T, int n_o, const double *centers,
                      const double *semi_axes, const double *velocities, const double *start,
                      const double *goal, double vmax, double amax, double rho,
                      double w_smooth, double w_track, int cost_mode, int n_traj,
                      const double *xi0, int max_iters, double tol, const int *iters_fixed,
                      double *xi_out, double *lam_out, double *residual_out, int *iters_out,
                      double *hist, int n_threads, int rho_levels, double rho_growth,
                      int rho_every, const double *box_lo, const double *box_hi,
                      const double *start_va, const double *lam0) {
  orc_problem pr = {dim, n_p, T, n_o, centers, semi_axes, velocities, start, goal,
                    vmax, amax, rho, w_smooth, w_track, cost_mode, box_lo, box_hi, rho_levels,
                    rho_growth, rho_every, start_va};
  return orc_am_solve(&pr, n_traj, xi0, lam0, max_iters, tol, iters_fixed, xi_out, lam_out,
                      residual_out, iters_out, hist, n_threads);
}

int orc_kkt_flat(int dim, int n_p, double T, int n_o, double rho, double w_smooth,
                 double w_track, int cost_mode, double *K, double *Kinv) {
  orc_problem pr = {dim, n_p, T, n_o, NULL, NULL, NULL, NULL, NULL,
                    0, 0, rho, w_smooth, w_track, cost_mode, NULL, NULL, 1, 1.0, 0, NULL};
  return orc_kkt(&pr, K, Kinv);
}

int orc_real_size(void) { return (int)sizeof(REAL); }
