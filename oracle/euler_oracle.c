/*
 * euler_oracle.c -- plain FP64 CPU oracle for the hyperbolic (Euler) operator
 * S_H of Guermond, Kronbichler, Maier, Popov & Tomas, "On the implementation of
 * a robust and efficient finite element-based parallel solver for the
 * compressible Navier-Stokes equations" (arXiv:2106.02159).
 *
 * TEST INFRASTRUCTURE. This file is the slow, obviously-correct reference that
 * the CUDA library is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order (Appendix B, Algorithm 1):
 *   Step 1  graph viscosity d_ij (Sec. 3.1) and the indicator alpha_i (Sec. 3.2)
 *   Step 2  transpose fill, d_ii, CFL time step (Sec. 3.1, eq. dtCfl)
 *   Step 3  bar states, low-order update, local bounds, high-order fluxes
 *           (Sec. 3.1 eqs. bar_state / loworder_bis, Sec. 3.2)
 *   Step 4+ limiter directions P_ij, line search, symmetrisation, limited
 *           update, second limiter pass (Sec. 3.3)
 * followed by the boundary post-processing of Sec. 4 (slip, supersonic inflow
 * = Dirichlet state, supersonic outflow = do nothing) and the SSPRK(3,3)
 * driver of Sec. 4.1 (eq. SPPRK33).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *  - lambda_max: the paper uses "the non-iterative guaranteed upper bound" of
 *    Guermond-Popov 2016 without printing it. Here: the two-rarefaction
 *    pressure p_tr as the upper bound on p*, then the shock-speed formulas of
 *    the 1- and 3-waves evaluated at p_tr (valid for 1 < gamma <= 5/3).
 *  - alpha_i: the paper cites other works. Here: the entropy-viscosity
 *    commutator with eta(U) = -rho s, s = ln(eps rho^-gamma)/(gamma-1),
 *    entropy flux q = v eta, normalised by the sum of the absolute values of
 *    its per-edge terms, so that 0 <= alpha_i <= 1 and alpha_i = O(h) wherever
 *    the solution is smooth (the paper asks for alpha small there).
 *  - local bounds: strict by default (the paper's text). An opt-in relaxation
 *    scales them by (1 -/+ r_i), r_i = (m_i/|D|)^{1.5/d}, |D| = sum_i m_i; it
 *    keeps positivity and lets smooth extrema converge at second order.
 *  - the line search for l_j^i: density by a closed-form ratio, the entropy
 *    bound psi(l) = eps(U + lP) - Phi_min rho(U + lP)^gamma (concave in l) by
 *    six fixed secant(left)/Newton(right) bracketing iterations.
 *  - d_ij takes the max of both directions only when i and j are both
 *    boundary nodes (c_ji = -c_ij exactly whenever one of them is interior).
 *  - every limiter pass is symmetrised, l_ij = min(l_j^i, l_i^j).
 *  - P_ij = 0 (a pass after l_ij = 1, uniform flow): every l gives the same
 *    state and the line search returns 1, the largest.
 *  - sums over I(i) are written in increment form (differences U_j - U_i,
 *    f(U_j) - f(U_i)), which equals the paper's form because sum_j c_ij = 0
 *    and sum_j d_ij = 0, and makes uniform states exact fixed points; the
 *    SSP combinations likewise as u + 1/4 (v - u) and u + 2/3 (v - u).
 *  - boundary post-processing is applied to each forward-Euler result before
 *    the SSP combination; a node touching an inflow face is a Dirichlet node,
 *    otherwise a node touching a slip face is a slip node.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -fopenmp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 3
#define MAXS 5
/* fixed number of bracketing iterations of the entropy line search */
#define LINE_SEARCH_ITERATIONS 6

enum { BC_SLIP = 1, BC_DIRICHLET = 2, BC_DO_NOTHING = 3, BC_CHARACTERISTIC = 4, BC_GODUNOV = 5 };

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_ARG = 1,
  ORACLE_ERR_MESH = 2,
  ORACLE_ERR_NOT_ADMISSIBLE = 3,
  ORACLE_ERR_OOM = 4
};

/* Mesh + parameters. All arrays are borrowed from the caller. State vectors
 * are stored component-major: U[s * n + i], s = 0 (rho), 1..dim (momentum),
 * dim+1 (total energy E). */
typedef struct {
  int dim;
  int n;
  int64_t nnz;
  const int64_t *row_ptr; /* [n+1] */
  const int32_t *col;     /* [nnz], sorted within each row, diagonal present */
  const double *cij;      /* [dim][nnz], c_ij = int phi_i grad phi_j */
  const double *mij;      /* [nnz], consistent mass m_ij */
  const double *mi;       /* [n], lumped mass m_i */
  int n_bnd;
  const int32_t *bnd_node;   /* [n_bnd] */
  const int32_t *bnd_kind;   /* [n_bnd] BC_* */
  const double *bnd_normal;  /* [dim][n_bnd], unit slip normal n^s_i */
  const double *bnd_state;   /* [dim+2][n_bnd], Dirichlet states (may be NULL) */
  double gamma;
  double cfl;
  int limiter_passes;
  int bound_relaxation; /* 0: strict local bounds, 1: relaxed by r_i */
} oracle_problem;

/* Optional outputs of one forward-Euler stage (any pointer may be NULL). */
typedef struct {
  double *dij;      /* [nnz]  d^L_ij, diagonal included */
  double *alpha;    /* [n] */
  double *UL;       /* [S][n] low-order update */
  double *FH;       /* [S][n] high-order fluxes F^H_i */
  double *bounds;   /* [3][n] rho_min, rho_max, Phi_min */
  double *P;        /* [S][nnz] first-pass limiter directions P_ij (0 on diagonal) */
  double *lij;      /* [passes][nnz] symmetrised limiters of every pass */
  double *Upass;    /* [passes][S][n] state after every limiter pass */
  double tau_bound; /* out: this stage's own CFL bound c_cfl min_i m_i/(2|d_ii|) */
} oracle_trace;

typedef struct {
  oracle_problem p;
  int S;
  int64_t *transpose; /* [nnz] position of (j,i) for the entry (i,j) */
  unsigned char *is_bnd; /* [n] */
  double *relax;         /* [n] r_i, or 0 */
  /* work arrays */
  double *dij, *alpha, *UL, *FH, *bounds, *P, *lij, *lraw, *Ucur, *Unext;
  /* nodes whose low-order update U^L left the admissible set, summed over
   * the stages since the last reset (the check of the adaptive CFL step) */
  int64_t low_not_admissible;
} oracle_ctx;

/* ------------------------------------------------------------------------- */
/* Sec. 2.1: state functions of the ideal gas law                            */
/* ------------------------------------------------------------------------- */

/* Internal energy eps(U) = E - |m|^2 / (2 rho) (Sec. 3.1, below eq. loworder_bis). */
static double internal_energy(const double *u, int dim) {
  double m2 = 0.0;
  for (int k = 0; k < dim; ++k) m2 += u[1 + k] * u[1 + k];
  return u[dim + 1] - m2 / (2.0 * u[0]);
}

/* p(U) = (gamma - 1) rho e(U) = (gamma - 1) eps(U) (Sec. 2.1). */
static double pressure(const double *u, int dim, double gamma) {
  return (gamma - 1.0) * internal_energy(u, dim);
}

/* Phi(U) = eps(U) rho^-gamma, the exponential of the specific entropy that
 * the limiter bounds from below (Sec. 3.1). */
static double entropy_phi(const double *u, int dim, double gamma) {
  return internal_energy(u, dim) * pow(u[0], -gamma);
}

/* Flux f(U) = (m, v (x) m + p I_d, v (E + p)) in R^{(d+2) x d} (Sec. 2.1). */
static void flux(const double *u, int dim, double gamma, double f[MAXS][MAXD]) {
  double rho = u[0];
  double p = pressure(u, dim, gamma);
  double v[MAXD];
  for (int k = 0; k < dim; ++k) v[k] = u[1 + k] / rho;
  for (int k = 0; k < dim; ++k) f[0][k] = u[1 + k];
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) f[1 + a][b] = v[b] * u[1 + a] + (a == b ? p : 0.0);
  for (int k = 0; k < dim; ++k) f[dim + 1][k] = v[k] * (u[dim + 1] + p);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.1: guaranteed upper bound lambda_max(U_L, U_R, n)                  */
/* ------------------------------------------------------------------------- */

/* Upper bound on the largest wave speed of the 1D Riemann problem with left
 * state ul, right state ur and flux f(w) n. The star pressure is bounded from
 * above by the two-rarefaction pressure
 *   p_tr = ((a_L + a_R - (gamma-1)/2 (u_R - u_L)) /
 *           (a_L p_L^-z + a_R p_R^-z))^(1/z),   z = (gamma-1)/(2 gamma),
 * (an upper bound for 1 < gamma <= 5/3); the outer wave speeds are then
 *   lambda_1^- = u_L - a_L sqrt(1 + (gamma+1)/(2 gamma) (p_tr - p_L)_+ / p_L),
 *   lambda_3^+ = u_R + a_R sqrt(1 + (gamma+1)/(2 gamma) (p_tr - p_R)_+ / p_R),
 * and lambda_max = max((lambda_1^-)_-, (lambda_3^+)_+). */
double oracle_lambda_max(const double *ul, const double *ur, const double *n, int dim, double gamma) {
  double rho_l = ul[0], rho_r = ur[0];
  double un_l = 0.0, un_r = 0.0;
  for (int k = 0; k < dim; ++k) {
    un_l += ul[1 + k] * n[k];
    un_r += ur[1 + k] * n[k];
  }
  un_l /= rho_l;
  un_r /= rho_r;
  double p_l = pressure(ul, dim, gamma), p_r = pressure(ur, dim, gamma);
  double a_l = sqrt(gamma * p_l / rho_l), a_r = sqrt(gamma * p_r / rho_r);
  double z = (gamma - 1.0) / (2.0 * gamma);
  double num = a_l + a_r - 0.5 * (gamma - 1.0) * (un_r - un_l);
  if (num < 0.0) num = 0.0;
  double den = a_l * pow(p_l, -z) + a_r * pow(p_r, -z);
  double p_tr = pow(num / den, 1.0 / z);
  double k = (gamma + 1.0) / (2.0 * gamma);
  double lam1 = un_l - a_l * sqrt(1.0 + k * fmax(p_tr - p_l, 0.0) / p_l);
  double lam3 = un_r + a_r * sqrt(1.0 + k * fmax(p_tr - p_r, 0.0) / p_r);
  return fmax(fmax(-lam1, 0.0), fmax(lam3, 0.0));
}

/* lambda_max for m independent pairs; ul, ur: [m][dim+2], n: [m][dim]. */
void oracle_lambda_max_batch(int64_t m, const double *ul, const double *ur, const double *n, int dim, double gamma,
                             double *out) {
  int S = dim + 2;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < m; ++q) out[q] = oracle_lambda_max(ul + q * S, ur + q * S, n + q * dim, dim, gamma);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2: entropy-production indicator alpha_i                            */
/* ------------------------------------------------------------------------- */

/* Mathematical entropy eta(U) = -rho s(U), s = ln(eps rho^-gamma)/(gamma-1). */
static double entropy_eta(const double *u, int dim, double gamma) {
  double s = log(internal_energy(u, dim) * pow(u[0], -gamma)) / (gamma - 1.0);
  return -u[0] * s;
}

/* Gradient of eta with respect to the conserved variables:
 *   d eta/d rho = -s - rho/(gamma-1) (|v|^2/(2 eps) - gamma/rho)
 *   d eta/d m   = rho v / ((gamma-1) eps)
 *   d eta/d E   = -rho / ((gamma-1) eps). */
void oracle_entropy_gradient(const double *u, int dim, double gamma, double *out) {
  double rho = u[0];
  double eps = internal_energy(u, dim);
  double s = log(eps * pow(rho, -gamma)) / (gamma - 1.0);
  double v2 = 0.0;
  for (int k = 0; k < dim; ++k) v2 += (u[1 + k] / rho) * (u[1 + k] / rho);
  out[0] = -s - rho / (gamma - 1.0) * (v2 / (2.0 * eps) - gamma / rho);
  for (int k = 0; k < dim; ++k) out[1 + k] = rho * (u[1 + k] / rho) / ((gamma - 1.0) * eps);
  out[dim + 1] = -rho / ((gamma - 1.0) * eps);
}

double oracle_entropy_eta(const double *u, int dim, double gamma) { return entropy_eta(u, dim, gamma); }

/* alpha_i = |N_i| / D_i with, for j in I*(i),
 *   a_ij = (q(U_j) - q(U_i)) . c_ij,
 *   b_ij = eta'(U_i) . ((f(U_j) - f(U_i)) c_ij),
 *   N_i = sum_j (a_ij - b_ij),  D_i = sum_j (|a_ij| + |b_ij|),
 *   alpha_i = 0 when D_i = 0. */
static double indicator(const oracle_ctx *c, const double *U, int i) {
  const oracle_problem *p = &c->p;
  int dim = p->dim, S = c->S, n = p->n;
  double ui[MAXS], uj[MAXS], deta[MAXS], fi[MAXS][MAXD], fj[MAXS][MAXD];
  for (int s = 0; s < S; ++s) ui[s] = U[s * n + i];
  oracle_entropy_gradient(ui, dim, p->gamma, deta);
  flux(ui, dim, p->gamma, fi);
  double eta_i = entropy_eta(ui, dim, p->gamma);
  double N = 0.0, D = 0.0;
  for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
    int j = p->col[k];
    if (j == i) continue;
    for (int s = 0; s < S; ++s) uj[s] = U[s * n + j];
    flux(uj, dim, p->gamma, fj);
    double eta_j = entropy_eta(uj, dim, p->gamma);
    double a = 0.0, b = 0.0;
    for (int d = 0; d < dim; ++d) {
      double cd = p->cij[(int64_t)d * p->nnz + k];
      double qj = uj[1 + d] / uj[0] * eta_j;
      double qi = ui[1 + d] / ui[0] * eta_i;
      a += (qj - qi) * cd;
      for (int s = 0; s < S; ++s) b += deta[s] * (fj[s][d] - fi[s][d]) * cd;
    }
    N += a - b;
    D += fabs(a) + fabs(b);
  }
  return D > 0.0 ? fabs(N) / D : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.3: line search for the largest l in [0,1] keeping the bounds       */
/* ------------------------------------------------------------------------- */

static double psi(const double *ub, const double *P, double l, int dim, double gamma, double phi_min) {
  double u[MAXS];
  for (int s = 0; s < dim + 2; ++s) u[s] = ub[s] + l * P[s];
  return internal_energy(u, dim) - phi_min * pow(u[0], gamma);
}

/* d psi / d l = d eps/d l - Phi_min gamma rho^(gamma-1) rho(P), with
 * d eps/d l = E(P) - v . m(P) + |v|^2/2 rho(P) at U + l P. */
static double dpsi(const double *ub, const double *P, double l, int dim, double gamma, double phi_min) {
  double u[MAXS];
  for (int s = 0; s < dim + 2; ++s) u[s] = ub[s] + l * P[s];
  double v2 = 0.0, vP = 0.0;
  for (int k = 0; k < dim; ++k) {
    double v = u[1 + k] / u[0];
    v2 += v * v;
    vP += v * P[1 + k];
  }
  double deps = P[dim + 1] - vP + 0.5 * v2 * P[0];
  return deps - phi_min * gamma * pow(u[0], gamma - 1.0) * P[0];
}

/* Largest l in [0,1] (or a lower estimate of it) such that
 *   rho_min <= rho(ub + l P) <= rho_max  and  Phi(ub + l P) >= Phi_min.
 * Density: closed form. Entropy: psi is concave along the segment, so a secant
 * through a feasible left point and an infeasible right point lands on the
 * feasible side (new left point) and a Newton step from the right point stays
 * on the infeasible side (new right point); LINE_SEARCH_ITERATIONS such
 * iterations, then the left point is returned. */
double oracle_line_search(const double *ub, const double *P, double rho_min, double rho_max, double phi_min,
                          int dim, double gamma) {
  /* P = 0: every l gives the same state; the largest one, 1, is returned */
  int zero = 1;
  for (int s = 0; s < dim + 2; ++s) zero &= P[s] == 0.0;
  if (zero) return 1.0;
  double l = 1.0;
  double rb = ub[0], rp = P[0];
  if (rp > 0.0) {
    l = fmin(l, (rho_max - rb) / rp);
  } else if (rp < 0.0) {
    l = fmin(l, (rho_min - rb) / rp);
  }
  l = fmax(0.0, fmin(1.0, l));

  double pr = psi(ub, P, l, dim, gamma, phi_min);
  if (pr >= 0.0) return l;
  double pl = psi(ub, P, 0.0, dim, gamma, phi_min);
  if (pl <= 0.0) return 0.0;
  double lL = 0.0, lR = l;
  for (int it = 0; it < LINE_SEARCH_ITERATIONS; ++it) {
    double ls = lL + pl * (lR - lL) / (pl - pr);
    double dr = dpsi(ub, P, lR, dim, gamma, phi_min);
    double ln = dr < 0.0 ? lR - pr / dr : lR;
    if (ln < ls) ln = ls;
    double ps = psi(ub, P, ls, dim, gamma, phi_min);
    double pn = psi(ub, P, ln, dim, gamma, phi_min);
    if (ps >= 0.0) {
      lL = ls;
      pl = ps;
    }
    if (pn < 0.0) {
      lR = ln;
      pr = pn;
    } else {
      lL = ln;
      pl = pn;
    }
  }
  return lL;
}

/* ------------------------------------------------------------------------- */
/* Setup: transpose index and boundary flags                                 */
/* ------------------------------------------------------------------------- */

static int64_t find_in_row(const oracle_problem *p, int row, int colv) {
  int64_t lo = p->row_ptr[row], hi = p->row_ptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int c = p->col[mid];
    if (c == colv) return mid;
    if (c < colv) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

void oracle_destroy(oracle_ctx *c) {
  if (!c) return;
  free(c->transpose); free(c->is_bnd); free(c->relax);
  free(c->dij); free(c->alpha); free(c->UL); free(c->FH); free(c->bounds);
  free(c->P); free(c->lij); free(c->lraw); free(c->Ucur); free(c->Unext);
  free(c);
}

/* Validates the mesh (sorted rows, diagonal present, symmetric pattern, valid
 * boundary list) and builds the transpose index. Returns NULL on error and
 * writes the status to *status. */
oracle_ctx *oracle_create(const oracle_problem *prob, int *status) {
  *status = ORACLE_ERR_ARG;
  if (!prob || prob->dim < 1 || prob->dim > MAXD || prob->n <= 0 || prob->nnz <= 0) return NULL;
  if (prob->limiter_passes < 1 || !(prob->gamma > 1.0) || !(prob->cfl > 0.0)) return NULL;
  oracle_ctx *c = (oracle_ctx *)calloc(1, sizeof(oracle_ctx));
  if (!c) { *status = ORACLE_ERR_OOM; return NULL; }
  c->p = *prob;
  c->S = prob->dim + 2;
  const oracle_problem *p = &c->p;
  int n = p->n, S = c->S;
  int64_t nnz = p->nnz;
  *status = ORACLE_ERR_MESH;
  if (p->row_ptr[0] != 0 || p->row_ptr[n] != nnz) { oracle_destroy(c); return NULL; }
  for (int i = 0; i < n; ++i) {
    int has_diag = 0;
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      if (p->col[k] < 0 || p->col[k] >= n) { oracle_destroy(c); return NULL; }
      if (k > p->row_ptr[i] && p->col[k] <= p->col[k - 1]) { oracle_destroy(c); return NULL; }
      if (p->col[k] == i) has_diag = 1;
    }
    if (!has_diag || p->row_ptr[i + 1] - p->row_ptr[i] < 2) { oracle_destroy(c); return NULL; }
  }
  c->transpose = (int64_t *)malloc(sizeof(int64_t) * nnz);
  c->is_bnd = (unsigned char *)calloc(n, 1);
  c->relax = (double *)calloc(n, sizeof(double));
  if (!c->transpose || !c->is_bnd || !c->relax) { oracle_destroy(c); *status = ORACLE_ERR_OOM; return NULL; }
  if (p->bound_relaxation) {
    double area = 0.0;
    for (int i = 0; i < n; ++i) area += p->mi[i];
    for (int i = 0; i < n; ++i) c->relax[i] = pow(p->mi[i] / area, 1.5 / p->dim);
  }
  for (int i = 0; i < n; ++i)
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      int64_t t = find_in_row(p, p->col[k], i);
      if (t < 0) { oracle_destroy(c); return NULL; }
      c->transpose[k] = t;
    }
  for (int b = 0; b < p->n_bnd; ++b) {
    int i = p->bnd_node[b];
    int kind = p->bnd_kind[b];
    if (i < 0 || i >= n || kind < BC_SLIP || kind > BC_GODUNOV) { oracle_destroy(c); return NULL; }
    if (kind != BC_SLIP && kind != BC_DO_NOTHING && !p->bnd_state) { oracle_destroy(c); return NULL; }
    c->is_bnd[i] = 1;
  }
  int passes = p->limiter_passes;
  c->dij = (double *)malloc(sizeof(double) * nnz);
  c->alpha = (double *)malloc(sizeof(double) * n);
  c->UL = (double *)malloc(sizeof(double) * S * n);
  c->FH = (double *)malloc(sizeof(double) * S * n);
  c->bounds = (double *)malloc(sizeof(double) * 3 * n);
  c->P = (double *)malloc(sizeof(double) * S * nnz);
  c->lij = (double *)malloc(sizeof(double) * nnz);
  c->lraw = (double *)malloc(sizeof(double) * nnz);
  c->Ucur = (double *)malloc(sizeof(double) * S * n);
  c->Unext = (double *)malloc(sizeof(double) * S * n);
  (void)passes;
  if (!c->dij || !c->alpha || !c->UL || !c->FH || !c->bounds || !c->P || !c->lij || !c->lraw || !c->Ucur ||
      !c->Unext) {
    oracle_destroy(c);
    *status = ORACLE_ERR_OOM;
    return NULL;
  }
  *status = ORACLE_OK;
  return c;
}

int oracle_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* Admissible set A = {rho > 0, e > 0} (Sec. 2.1). Returns the number of
 * non-admissible nodes. */
int64_t oracle_count_not_admissible(const oracle_ctx *c, const double *U) {
  int n = c->p.n, S = c->S, dim = c->p.dim;
  int64_t bad = 0;
  for (int i = 0; i < n; ++i) {
    double u[MAXS];
    for (int s = 0; s < S; ++s) u[s] = U[s * n + i];
    if (!(u[0] > 0.0) || !(internal_energy(u, dim) > 0.0)) ++bad;
  }
  return bad;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1, steps 1-2: d_ij, alpha_i, d_ii and the CFL bound             */
/* ------------------------------------------------------------------------- */

static void viscosity(oracle_ctx *c, const double *U, double *tau_bound_out) {
  const oracle_problem *p = &c->p;
  int n = p->n, S = c->S, dim = p->dim;
  double gamma = p->gamma;
  /* Step 1: alpha_i and d_ij for j > i. */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    c->alpha[i] = indicator(c, U, i);
    double ui[MAXS], uj[MAXS];
    for (int s = 0; s < S; ++s) ui[s] = U[s * n + i];
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      int j = p->col[k];
      if (j <= i) continue;
      for (int s = 0; s < S; ++s) uj[s] = U[s * n + j];
      double cv[MAXD], nv[MAXD], norm = 0.0;
      for (int d = 0; d < dim; ++d) {
        cv[d] = p->cij[(int64_t)d * p->nnz + k];
        norm += cv[d] * cv[d];
      }
      norm = sqrt(norm);
      for (int d = 0; d < dim; ++d) nv[d] = cv[d] / norm;
      double dij = oracle_lambda_max(ui, uj, nv, dim, gamma) * norm;
      if (c->is_bnd[i] && c->is_bnd[j]) {
        int64_t kt = c->transpose[k];
        double ct[MAXD], nt[MAXD], normt = 0.0;
        for (int d = 0; d < dim; ++d) {
          ct[d] = p->cij[(int64_t)d * p->nnz + kt];
          normt += ct[d] * ct[d];
        }
        normt = sqrt(normt);
        for (int d = 0; d < dim; ++d) nt[d] = ct[d] / normt;
        double dji = oracle_lambda_max(uj, ui, nt, dim, gamma) * normt;
        dij = fmax(dij, dji);
      }
      c->dij[k] = dij;
    }
  }
  /* Step 2: fill j < i from the transpose, d_ii = -sum_{j != i} d_ij and the
   * bound c_cfl * m_i / (2 |d_ii|) of eq. dtCfl. */
  double tau = INFINITY;
#pragma omp parallel for schedule(static) reduction(min : tau)
  for (int i = 0; i < n; ++i) {
    double sum = 0.0;
    int64_t kdiag = -1;
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      int j = p->col[k];
      if (j == i) { kdiag = k; continue; }
      if (j < i) c->dij[k] = c->dij[c->transpose[k]];
      sum += c->dij[k];
    }
    c->dij[kdiag] = -sum;
    double t = -p->cfl * p->mi[i] / (2.0 * c->dij[kdiag]);
    if (t < tau) tau = t;
  }
  *tau_bound_out = tau;
}

double oracle_cfl_dt(oracle_ctx *c, const double *U) {
  double tau;
  viscosity(c, U, &tau);
  return tau;
}

/* ------------------------------------------------------------------------- */
/* One forward-Euler stage (Algorithm 1) without boundary post-processing    */
/* ------------------------------------------------------------------------- */

/* tau > 0: use it; tau <= 0: use the CFL bound of this stage. */
int oracle_forward_euler(oracle_ctx *c, const double *U, double tau, double *Uout, double *tau_used,
                         oracle_trace *tr) {
  const oracle_problem *p = &c->p;
  int n = p->n, S = c->S, dim = p->dim;
  int64_t nnz = p->nnz;
  double gamma = p->gamma;
  if (oracle_count_not_admissible(c, U) > 0) return ORACLE_ERR_NOT_ADMISSIBLE;

  double tau_bound;
  viscosity(c, U, &tau_bound);
  if (!(tau > 0.0)) tau = tau_bound;
  if (tau_used) *tau_used = tau;
  if (tr) tr->tau_bound = tau_bound;

  /* Step 3: bar states, low-order update, local bounds, high-order flux. */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double ui[MAXS], uj[MAXS], fi[MAXS][MAXD], fj[MAXS][MAXD];
    for (int s = 0; s < S; ++s) ui[s] = U[s * n + i];
    flux(ui, dim, gamma, fi);
    double inc[MAXS] = {0}, fh[MAXS] = {0};
    double rho_min = ui[0], rho_max = ui[0];
    double phi_min = entropy_phi(ui, dim, gamma);
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      int j = p->col[k];
      if (j == i) continue;
      for (int s = 0; s < S; ++s) uj[s] = U[s * n + j];
      flux(uj, dim, gamma, fj);
      double dfc[MAXS];
      for (int s = 0; s < S; ++s) {
        dfc[s] = 0.0;
        for (int d = 0; d < dim; ++d) dfc[s] += (fj[s][d] - fi[s][d]) * p->cij[(int64_t)d * nnz + k];
      }
      double dL = c->dij[k];
      double dH = 0.5 * (c->alpha[i] + c->alpha[j]) * dL;
      double ubar[MAXS];
      for (int s = 0; s < S; ++s) {
        ubar[s] = dL > 0.0 ? 0.5 * (ui[s] + uj[s]) - dfc[s] / (2.0 * dL) : ui[s];
        inc[s] += dL * (ubar[s] - ui[s]);
        fh[s] += -dfc[s] + dH * (uj[s] - ui[s]);
      }
      rho_min = fmin(rho_min, ubar[0]);
      rho_max = fmax(rho_max, ubar[0]);
      phi_min = fmin(phi_min, entropy_phi(uj, dim, gamma));
    }
    for (int s = 0; s < S; ++s) {
      c->UL[s * n + i] = ui[s] + 2.0 * tau / p->mi[i] * inc[s];
      c->FH[s * n + i] = fh[s];
    }
    {
      double ul[MAXS];
      for (int s = 0; s < S; ++s) ul[s] = c->UL[s * n + i];
      if (!(ul[0] > 0.0 && internal_energy(ul, dim) > 0.0)) {
#pragma omp atomic
        c->low_not_admissible += 1;
      }
    }
    /* optional relaxation of the local bounds (off by default) */
    double r = c->relax[i];
    c->bounds[0 * n + i] = (1.0 - r) * rho_min;
    c->bounds[1 * n + i] = (1.0 + r) * rho_max;
    c->bounds[2 * n + i] = (1.0 - r) * phi_min;
  }

  /* Step 4: P_ij (Sec. 3.3) and the first line search.
   * P_ij = tau/(m_i lambda_i) (b_ij F^H_j - b_ji F^H_i + (d^H_ij - d^L_ij)(U_j - U_i)),
   * b_ij = -m_ij/m_j, b_ji = -m_ji/m_i for j != i, lambda_i = 1/(card I(i) - 1). */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    int64_t k0 = p->row_ptr[i], k1 = p->row_ptr[i + 1];
    double lambda_i = 1.0 / (double)(k1 - k0 - 1);
    double ul[MAXS];
    for (int s = 0; s < S; ++s) ul[s] = c->UL[s * n + i];
    for (int64_t k = k0; k < k1; ++k) {
      int j = p->col[k];
      if (j == i) {
        for (int s = 0; s < S; ++s) c->P[(int64_t)s * nnz + k] = 0.0;
        c->lraw[k] = 1.0;
        continue;
      }
      double bij = -p->mij[k] / p->mi[j];
      double bji = -p->mij[c->transpose[k]] / p->mi[i];
      double dL = c->dij[k];
      double dH = 0.5 * (c->alpha[i] + c->alpha[j]) * dL;
      double Pk[MAXS];
      for (int s = 0; s < S; ++s) {
        double val = bij * c->FH[s * n + j] - bji * c->FH[s * n + i] + (dH - dL) * (U[s * n + j] - U[s * n + i]);
        Pk[s] = tau / (p->mi[i] * lambda_i) * val;
        c->P[(int64_t)s * nnz + k] = Pk[s];
      }
      c->lraw[k] = oracle_line_search(ul, Pk, c->bounds[i], c->bounds[n + i], c->bounds[2 * n + i], dim, gamma);
    }
  }

  /* Limiter passes: symmetrise, update, shrink P, search again (Sec. 3.3). */
  double *Ucur = c->Ucur;
  memcpy(Ucur, c->UL, sizeof(double) * S * n);
  for (int pass = 0; pass < p->limiter_passes; ++pass) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nnz; ++k) c->lij[k] = fmin(c->lraw[k], c->lraw[c->transpose[k]]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      int64_t k0 = p->row_ptr[i], k1 = p->row_ptr[i + 1];
      double lambda_i = 1.0 / (double)(k1 - k0 - 1);
      double u[MAXS];
      for (int s = 0; s < S; ++s) u[s] = Ucur[s * n + i];
      for (int64_t k = k0; k < k1; ++k) {
        if (p->col[k] == i) continue;
        for (int s = 0; s < S; ++s) u[s] += lambda_i * c->lij[k] * c->P[(int64_t)s * nnz + k];
      }
      for (int s = 0; s < S; ++s) c->Unext[s * n + i] = u[s];
    }
    if (tr && tr->lij) memcpy(tr->lij + (int64_t)pass * nnz, c->lij, sizeof(double) * nnz);
    if (tr && tr->P && pass == 0) memcpy(tr->P, c->P, sizeof(double) * S * nnz);
    memcpy(Ucur, c->Unext, sizeof(double) * S * n);
    if (tr && tr->Upass) memcpy(tr->Upass + (int64_t)pass * S * n, Ucur, sizeof(double) * S * n);
    if (pass + 1 == p->limiter_passes) break;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double u[MAXS], Pk[MAXS];
      for (int s = 0; s < S; ++s) u[s] = Ucur[s * n + i];
      for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
        if (p->col[k] == i) { c->lraw[k] = 1.0; continue; }
        for (int s = 0; s < S; ++s) {
          Pk[s] = (1.0 - c->lij[k]) * c->P[(int64_t)s * nnz + k];
          c->P[(int64_t)s * nnz + k] = Pk[s];
        }
        c->lraw[k] = oracle_line_search(u, Pk, c->bounds[i], c->bounds[n + i], c->bounds[2 * n + i], dim, gamma);
      }
    }
  }
  memcpy(Uout, Ucur, sizeof(double) * S * n);

  if (tr) {
    if (tr->dij) memcpy(tr->dij, c->dij, sizeof(double) * nnz);
    if (tr->alpha) memcpy(tr->alpha, c->alpha, sizeof(double) * n);
    if (tr->UL) memcpy(tr->UL, c->UL, sizeof(double) * S * n);
    if (tr->FH) memcpy(tr->FH, c->FH, sizeof(double) * S * n);
    if (tr->bounds) memcpy(tr->bounds, c->bounds, sizeof(double) * 3 * n);
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 4: boundary post-processing                                          */
/* ------------------------------------------------------------------------- */

/* Primitive quantities of a state along the unit normal nrm: rho, the normal
 * velocity vn, the tangential velocity vt = v - vn n, p and a (Sec. 4.2.2). */
typedef struct {
  double rho, vn, vt[MAXD], p, a;
} nprim;

static nprim normal_primitives(const double *u, const double *nrm, int dim, double gamma) {
  nprim w;
  w.rho = u[0];
  w.vn = 0.0;
  for (int d = 0; d < dim; ++d) w.vn += u[1 + d] / u[0] * nrm[d];
  for (int d = 0; d < dim; ++d) w.vt[d] = u[1 + d] / u[0] - w.vn * nrm[d];
  w.p = pressure(u, dim, gamma);
  w.a = sqrt(gamma * w.p / w.rho);
  return w;
}

/* The conserved state with density rho, velocity vn n + vt and pressure p. */
static void conserved_from(double rho, double vn, const double *vt, double p, const double *nrm, int dim, double gamma,
                           double *out) {
  double v2 = 0.0;
  out[0] = rho;
  for (int d = 0; d < dim; ++d) {
    double v = vn * nrm[d] + vt[d];
    out[1 + d] = rho * v;
    v2 += v * v;
  }
  out[dim + 1] = p / (gamma - 1.0) + 0.5 * rho * v2;
}

/* Sec. 4.2.2, characteristic variables: C_1 = v_n - 2a/(gamma-1) and
 * C_3 = v_n + 2a/(gamma-1) with speeds v_n -/+ a, S = p rho^-gamma and v^perp
 * with speed v_n. Incoming characteristics (negative speed along the outward
 * normal) take the Dirichlet state's values, outgoing ones keep U's; the four
 * cases give eqs. Supersonic_inflow, Subsonic_inflow, Subsonic_outflow and
 * Supersonic_outflow. u is replaced by the post-processed state. */
void oracle_bc_characteristic(double *u, const double *nrm, const double *ud, int dim, double gamma) {
  nprim w = normal_primitives(u, nrm, dim, gamma);
  if (w.vn < 0.0 && w.a < -w.vn) { /* supersonic inflow */
    for (int s = 0; s < dim + 2; ++s) u[s] = ud[s];
    return;
  }
  if (w.vn >= 0.0 && w.a <= w.vn) return; /* supersonic outflow */
  nprim wd = normal_primitives(ud, nrm, dim, gamma);
  double c3 = w.vn + 2.0 * w.a / (gamma - 1.0);   /* outgoing in both subsonic cases */
  double c1d = wd.vn - 2.0 * wd.a / (gamma - 1.0); /* incoming in both subsonic cases */
  /* subsonic inflow: entropy and tangential velocity come in; outflow: they go out */
  const nprim *src = w.vn < 0.0 ? &wd : &w;
  double s_ent = src->p * pow(src->rho, -gamma);
  double a_p = 0.25 * (gamma - 1.0) * (c3 - c1d);
  double vn_p = 0.5 * (c1d + c3);
  double rho_p = pow(a_p * a_p / (gamma * s_ent), 1.0 / (gamma - 1.0));
  double p_p = s_ent * pow(rho_p, gamma);
  conserved_from(rho_p, vn_p, src->vt, p_p, nrm, dim, gamma, u);
}

/* Toro's pressure function of side K and its derivative (Riemann problem of
 * the Euler equations along a line): shock branch for p > p_K, rarefaction
 * branch otherwise. */
static void toro_f(double p, const nprim *k, double gamma, double *f, double *df) {
  if (p > k->p) {
    double A = 2.0 / ((gamma + 1.0) * k->rho), B = (gamma - 1.0) / (gamma + 1.0) * k->p;
    double q = sqrt(A / (p + B));
    *f = (p - k->p) * q;
    *df = q * (1.0 - 0.5 * (p - k->p) / (p + B));
  } else {
    double z = (gamma - 1.0) / (2.0 * gamma);
    *f = 2.0 * k->a / (gamma - 1.0) * (pow(p / k->p, z) - 1.0);
    *df = pow(p / k->p, -(gamma + 1.0) / (2.0 * gamma)) / (k->rho * k->a);
  }
}

/* State at x/t = 0 of the exact solution of the Riemann problem with left
 * state l and right state r (normal velocities vn, tangential velocities
 * carried by the contact): rho, vn, vt, p. */
static void riemann_at_zero(const nprim *l, const nprim *r, int dim, double gamma, nprim *out) {
  const double g1 = (gamma - 1.0) / (2.0 * gamma), g2 = (gamma + 1.0) / (2.0 * gamma);
  const double g4 = 2.0 / (gamma - 1.0), g5 = 2.0 / (gamma + 1.0), g6 = (gamma - 1.0) / (gamma + 1.0);
  const double g7 = 0.5 * (gamma - 1.0);
  const double du = r->vn - l->vn;
  if (g4 * (l->a + r->a) <= du) { /* the two rarefactions leave a vacuum between them */
    double sl = l->vn + g4 * l->a, sr = r->vn - g4 * r->a;
    if (l->vn - l->a >= 0.0) { *out = *l; return; }
    if (sl > 0.0) { /* inside the left fan */
      double c = g5 * (l->a + g7 * l->vn);
      out->rho = l->rho * pow(c / l->a, g4);
      out->vn = g5 * (l->a + g7 * l->vn);
      out->p = l->p * pow(c / l->a, 1.0 / g1);
      for (int d = 0; d < dim; ++d) out->vt[d] = l->vt[d];
      return;
    }
    if (sr >= 0.0) { /* vacuum */
      out->rho = 0.0;
      out->vn = 0.0;
      out->p = 0.0;
      for (int d = 0; d < dim; ++d) out->vt[d] = 0.0;
      return;
    }
    if (r->vn + r->a > 0.0) { /* inside the right fan */
      double c = g5 * (r->a - g7 * r->vn);
      out->rho = r->rho * pow(c / r->a, g4);
      out->vn = g5 * (-r->a + g7 * r->vn);
      out->p = r->p * pow(c / r->a, 1.0 / g1);
      for (int d = 0; d < dim; ++d) out->vt[d] = r->vt[d];
      return;
    }
    *out = *r;
    return;
  }
  /* p*: Newton's method on f_L(p) + f_R(p) + (v_R - v_L) = 0 from the
   * two-rarefaction pressure, kept positive, to a relative change of 1e-15 */
  double p = pow((l->a + r->a - g7 * du) / (l->a / pow(l->p, g1) + r->a / pow(r->p, g1)), 1.0 / g1);
  for (int it = 0; it < 100; ++it) {
    double fl, dfl, fr, dfr;
    toro_f(p, l, gamma, &fl, &dfl);
    toro_f(p, r, gamma, &fr, &dfr);
    double pn = p - (fl + fr + du) / (dfl + dfr);
    if (pn <= 0.0) pn = 0.5 * p;
    double change = fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change < 1e-15) break;
  }
  double fl, dfl, fr, dfr;
  toro_f(p, l, gamma, &fl, &dfl);
  toro_f(p, r, gamma, &fr, &dfr);
  const double vs = 0.5 * (l->vn + r->vn) + 0.5 * (fr - fl); /* contact speed */
  if (vs >= 0.0) { /* x = 0 lies left of the contact */
    for (int d = 0; d < dim; ++d) out->vt[d] = l->vt[d];
    if (p > l->p) { /* left shock */
      double s = l->vn - l->a * sqrt(g2 * p / l->p + g1);
      if (s >= 0.0) { *out = *l; return; }
      out->rho = l->rho * (p / l->p + g6) / (g6 * p / l->p + 1.0);
      out->vn = vs;
      out->p = p;
      return;
    }
    if (l->vn - l->a >= 0.0) { *out = *l; return; } /* left rarefaction ahead of x = 0 */
    double cs = l->a * pow(p / l->p, g1);
    if (vs - cs < 0.0) { /* x = 0 in the left star region */
      out->rho = l->rho * pow(p / l->p, 1.0 / gamma);
      out->vn = vs;
      out->p = p;
      return;
    }
    double c = g5 * (l->a + g7 * l->vn); /* inside the left fan */
    out->rho = l->rho * pow(c / l->a, g4);
    out->vn = c;
    out->p = l->p * pow(c / l->a, 1.0 / g1);
    return;
  }
  for (int d = 0; d < dim; ++d) out->vt[d] = r->vt[d];
  if (p > r->p) { /* right shock */
    double s = r->vn + r->a * sqrt(g2 * p / r->p + g1);
    if (s <= 0.0) { *out = *r; return; }
    out->rho = r->rho * (p / r->p + g6) / (g6 * p / r->p + 1.0);
    out->vn = vs;
    out->p = p;
    return;
  }
  if (r->vn + r->a <= 0.0) { *out = *r; return; } /* right rarefaction behind x = 0 */
  double cs = r->a * pow(p / r->p, g1);
  if (vs + cs > 0.0) { /* x = 0 in the right star region */
    out->rho = r->rho * pow(p / r->p, 1.0 / gamma);
    out->vn = vs;
    out->p = p;
    return;
  }
  double c = g5 * (r->a - g7 * r->vn); /* inside the right fan */
  out->rho = r->rho * pow(c / r->a, g4);
  out->vn = -c;
  out->p = r->p * pow(c / r->a, 1.0 / g1);
}

/* Sec. 4.2.1, eq. Godunov_bc: U^P = the value at x = 0 of the exact solution
 * of the Riemann problem along the outward normal with left state U and
 * right state U^D. u is replaced by it. */
void oracle_bc_godunov(double *u, const double *nrm, const double *ud, int dim, double gamma) {
  nprim l = normal_primitives(u, nrm, dim, gamma), r = normal_primitives(ud, nrm, dim, gamma), z;
  riemann_at_zero(&l, &r, dim, gamma, &z);
  conserved_from(z.rho, z.vn, z.vt, z.p, nrm, dim, gamma, u);
}

/* Slip (eq. slip_bc): M <- M - (M . n^s) n^s. Supersonic inflow (eq.
 * Supersonic_inflow): U <- U^D. Supersonic outflow (eq. Supersonic_outflow):
 * nothing. Non-reflecting nodes: the characteristic post-processing or the
 * Godunov one (Sec. 4.2), with the node's normal and Dirichlet state. */
void oracle_apply_bc(const oracle_ctx *c, double *U) {
  const oracle_problem *p = &c->p;
  int n = p->n, dim = p->dim, S = c->S;
  for (int b = 0; b < p->n_bnd; ++b) {
    int i = p->bnd_node[b];
    int kind = p->bnd_kind[b];
    if (kind == BC_SLIP) {
      double mn = 0.0;
      for (int d = 0; d < dim; ++d) mn += U[(1 + d) * n + i] * p->bnd_normal[(int64_t)d * p->n_bnd + b];
      for (int d = 0; d < dim; ++d) U[(1 + d) * n + i] -= mn * p->bnd_normal[(int64_t)d * p->n_bnd + b];
    } else if (kind == BC_DIRICHLET) {
      for (int s = 0; s < S; ++s) U[s * n + i] = p->bnd_state[(int64_t)s * p->n_bnd + b];
    } else if (kind == BC_CHARACTERISTIC || kind == BC_GODUNOV) {
      double u[MAXS], ud[MAXS], nrm[MAXD];
      for (int s = 0; s < S; ++s) {
        u[s] = U[s * n + i];
        ud[s] = p->bnd_state[(int64_t)s * p->n_bnd + b];
      }
      for (int d = 0; d < dim; ++d) nrm[d] = p->bnd_normal[(int64_t)d * p->n_bnd + b];
      if (kind == BC_CHARACTERISTIC)
        oracle_bc_characteristic(u, nrm, ud, dim, p->gamma);
      else
        oracle_bc_godunov(u, nrm, ud, dim, p->gamma);
      for (int s = 0; s < S; ++s) U[s * n + i] = u[s];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.1, eq. SPPRK33: one SSPRK(3,3) step                                */
/* ------------------------------------------------------------------------- */

/* U is advanced in place. dt > 0: use it; dt <= 0: the CFL step of the first
 * stage, reused by the other two stages (Sec. 3.1). stage_tau_bound (may be
 * NULL) receives the three stages' own CFL bounds. */
/* Remark "High aspect-ratio meshes" (Sec. 3.1): one SSPRK(3,3) step with a
 * CFL number above 1. The step is tried with c_cfl = cfl_max; if the
 * low-order update U^L of any stage, or the result, leaves the admissible set,
 * the step restarts from U with c_cfl halved, until it passes (c_cfl <= 1
 * always passes: U^L is then a convex combination of admissible bar states).
 * U is advanced in place; dt_used, cfl_used and restarts (may be NULL)
 * receive the accepted step, its CFL number and the number of restarts. */
int oracle_ssprk3_step(oracle_ctx *c, double *U, double dt, double *dt_used, double *stage_tau_bound);

int oracle_ssprk3_step_adaptive(oracle_ctx *c, double *U, double cfl_max, double *dt_used, double *cfl_used,
                                int *restarts) {
  if (!(cfl_max > 0.0)) return ORACLE_ERR_ARG;
  size_t bytes = sizeof(double) * c->S * c->p.n;
  double *u_in = (double *)malloc(bytes);
  if (!u_in) return ORACLE_ERR_OOM;
  memcpy(u_in, U, bytes);
  const double cfl_saved = c->p.cfl;
  double cfl = cfl_max, dt = 0.0;
  int r = 0, st;
  for (;;) {
    c->p.cfl = cfl;
    c->low_not_admissible = 0;
    memcpy(U, u_in, bytes);
    st = oracle_ssprk3_step(c, U, 0.0, &dt, NULL);
    int failed = st == ORACLE_ERR_NOT_ADMISSIBLE || (st == ORACLE_OK && (c->low_not_admissible > 0 ||
                                                                          oracle_count_not_admissible(c, U) > 0));
    if (st != ORACLE_OK && st != ORACLE_ERR_NOT_ADMISSIBLE) break;
    if (!failed) break;
    if (cfl <= 1.0) {
      st = ORACLE_ERR_NOT_ADMISSIBLE;
      break;
    }
    cfl *= 0.5;
    ++r;
  }
  c->p.cfl = cfl_saved;
  if (st != ORACLE_OK) memcpy(U, u_in, bytes);
  free(u_in);
  if (dt_used) *dt_used = dt;
  if (cfl_used) *cfl_used = cfl;
  if (restarts) *restarts = r;
  return st;
}

int oracle_ssprk3_step(oracle_ctx *c, double *U, double dt, double *dt_used, double *stage_tau_bound) {
  const oracle_problem *p = &c->p;
  int n = p->n, S = c->S;
  size_t bytes = sizeof(double) * S * n;
  double *u0 = (double *)malloc(bytes), *w = (double *)malloc(bytes), *v = (double *)malloc(bytes);
  if (!u0 || !w || !v) { free(u0); free(w); free(v); return ORACLE_ERR_OOM; }
  memcpy(u0, U, bytes);
  oracle_trace tr;
  memset(&tr, 0, sizeof(tr));
  double tau;
  int st = oracle_forward_euler(c, u0, dt, w, &tau, &tr);
  if (st) goto done;
  if (stage_tau_bound) stage_tau_bound[0] = tr.tau_bound;
  oracle_apply_bc(c, w);
  st = oracle_forward_euler(c, w, tau, v, NULL, &tr);
  if (st) goto done;
  if (stage_tau_bound) stage_tau_bound[1] = tr.tau_bound;
  oracle_apply_bc(c, v);
  for (int64_t q = 0; q < (int64_t)S * n; ++q) w[q] = u0[q] + 0.25 * (v[q] - u0[q]);
  st = oracle_forward_euler(c, w, tau, v, NULL, &tr);
  if (st) goto done;
  if (stage_tau_bound) stage_tau_bound[2] = tr.tau_bound;
  oracle_apply_bc(c, v);
  for (int64_t q = 0; q < (int64_t)S * n; ++q) U[q] = u0[q] + (2.0 / 3.0) * (v[q] - u0[q]);
  if (dt_used) *dt_used = tau;
done:
  free(u0); free(w); free(v);
  return st;
}

/* nsteps SSPRK(3,3) steps with the CFL step (dt <= 0) or a fixed dt. */
int oracle_run(oracle_ctx *c, double *U, int nsteps, double dt, double *t_out) {
  double t = 0.0;
  for (int s = 0; s < nsteps; ++s) {
    double used;
    int st = oracle_ssprk3_step(c, U, dt, &used, NULL);
    if (st) return st;
    t += used;
  }
  if (t_out) *t_out = t;
  return ORACLE_OK;
}

/* Advance to t_final exactly (the last step is shortened). */
int oracle_run_to(oracle_ctx *c, double *U, double t_final, int max_steps, double *t_out, int *steps_out) {
  double t = 0.0;
  int steps = 0;
  while (t < t_final && steps < max_steps) {
    double dt = oracle_cfl_dt(c, U);
    if (t + dt > t_final) dt = t_final - t;
    double used;
    int st = oracle_ssprk3_step(c, U, dt, &used, NULL);
    if (st) return st;
    t += used;
    ++steps;
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 5: the parabolic sub-step S_P and the Strang-split Navier-Stokes step */
/* ------------------------------------------------------------------------- */

/* Finite-element data of the viscous and Fourier terms (2D P1/Q1) and the
 * physical constants. L_ij = int grad phi_i . grad phi_j;
 * G_ij[k][m] = int d_k phi_i d_m phi_j; quadrature data of the cells for the
 * viscous energy source K_i. Velocity: no slip (v = 0) at the wall nodes,
 * homogeneous Neumann elsewhere; internal energy: homogeneous Neumann. */
typedef struct {
  const double *L;      /* [nnz] */
  const double *G;      /* [2][2][nnz] */
  int n_cells, nv, nq;
  const int32_t *cells; /* [n_cells][nv] */
  const double *qw;     /* [n_cells][nq] weights x |det J| */
  const double *qphi;   /* [n_cells][nq][nv] */
  const double *qgrad;  /* [n_cells][nq][2][nv] */
  int n_wall;
  const int32_t *wall;  /* no-slip nodes */
  double mu, lambda, kappa_cv; /* shear and bulk viscosity, kappa / c_v */
  double cg_tol;        /* relative residual of the CG solves */
  int cg_max_iter;
} oracle_parabolic;

typedef struct {
  int cg_iter_velocity, cg_iter_energy, cg_iter_low; /* iterations (low: 0 if not needed) */
  int limited;          /* 1 if the high-order internal energy had a non-positive value */
  double min_e;         /* min_i e_i^{n+1} */
} oracle_parabolic_info;

/* The operator y = D x + c A x of the velocity system: D = diag(rho_i m_i),
 * A_ij[k][m] = mu delta_km L_ij + mu G_ij[m][k] + (lambda - 2 mu/3) G_ij[k][m]
 * (eq. mt_parabolic_discrete: a(phi_j e_m, phi_i e_k) with
 * sigma(v) = 2 mu eps(v) + (lambda - 2 mu/3) div v I). Wall rows are the
 * identity and wall columns drop out (zero Dirichlet values). x, y: [n][2]. */
static void velocity_apply(const oracle_ctx *c, const oracle_parabolic *pp, const double *D, const unsigned char *wall,
                           double coef, const double *x, double *y) {
  const oracle_problem *p = &c->p;
  const int n = p->n;
  const int64_t nnz = p->nnz;
  const double lm = pp->lambda - 2.0 * pp->mu / 3.0;
  for (int i = 0; i < n; ++i) {
    if (wall[i]) {
      y[2 * i] = x[2 * i];
      y[2 * i + 1] = x[2 * i + 1];
      continue;
    }
    double acc[2] = {0.0, 0.0};
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
      const int j = p->col[k];
      if (wall[j]) continue;
      for (int a = 0; a < 2; ++a)
        for (int m = 0; m < 2; ++m) {
          double Aam = (a == m ? pp->mu * pp->L[k] : 0.0) + pp->mu * pp->G[(m * 2 + a) * nnz + k] +
                       lm * pp->G[(a * 2 + m) * nnz + k];
          acc[a] += Aam * x[2 * j + m];
        }
    }
    for (int a = 0; a < 2; ++a) y[2 * i + a] = D[i] * x[2 * i + a] + coef * acc[a];
  }
}

/* y = D x + coef L x (scalar, energy systems). */
static void energy_apply(const oracle_ctx *c, const oracle_parabolic *pp, const double *D, double coef, const double *x,
                         double *y) {
  const oracle_problem *p = &c->p;
  for (int i = 0; i < p->n; ++i) {
    double acc = 0.0;
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) acc += pp->L[k] * x[p->col[k]];
    y[i] = D[i] * x[i] + coef * acc;
  }
}

static double dotv(const double *a, const double *b, int64_t m) {
  double s = 0.0;
  for (int64_t q = 0; q < m; ++q) s += a[q] * b[q];
  return s;
}

/* Preconditioned conjugate gradients (diagonal preconditioner Pd) for the
 * symmetric positive definite system of size m applied by apply(x, y);
 * x holds the initial guess and receives the solution; stops when
 * ||r|| <= tol ||b||. Returns the iteration count, or -1 without convergence. */
static int pcg(const oracle_ctx *c, const oracle_parabolic *pp, const double *D, const unsigned char *wall, double coef,
               int scalar, const double *Pd, const double *b, double *x, int64_t m) {
  double *r = (double *)malloc(sizeof(double) * m), *z = (double *)malloc(sizeof(double) * m);
  double *d = (double *)malloc(sizeof(double) * m), *q = (double *)malloc(sizeof(double) * m);
  int it = -1;
  if (!r || !z || !d || !q) goto out;
  if (scalar) energy_apply(c, pp, D, coef, x, q); else velocity_apply(c, pp, D, wall, coef, x, q);
  for (int64_t s = 0; s < m; ++s) r[s] = b[s] - q[s];
  const double bn = sqrt(dotv(b, b, m));
  if (sqrt(dotv(r, r, m)) <= pp->cg_tol * bn) { it = 0; goto out; }
  for (int64_t s = 0; s < m; ++s) { z[s] = r[s] / Pd[s]; d[s] = z[s]; }
  double rz = dotv(r, z, m);
  for (int k = 1; k <= pp->cg_max_iter; ++k) {
    if (scalar) energy_apply(c, pp, D, coef, d, q); else velocity_apply(c, pp, D, wall, coef, d, q);
    const double alpha = rz / dotv(d, q, m);
    for (int64_t s = 0; s < m; ++s) { x[s] += alpha * d[s]; r[s] -= alpha * q[s]; }
    if (sqrt(dotv(r, r, m)) <= pp->cg_tol * bn) { it = k; goto out; }
    for (int64_t s = 0; s < m; ++s) z[s] = r[s] / Pd[s];
    const double rz_new = dotv(r, z, m);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t s = 0; s < m; ++s) d[s] = z[s] + beta * d[s];
  }
out:
  free(r); free(z); free(d); free(q);
  return it;
}

/* eq. def_Ki_nplusone: K_i = (1/m_i) int sigma(v):eps(v) phi_i, with the
 * cells' quadrature. v: [n][2]. */
static void viscous_source(const oracle_ctx *c, const oracle_parabolic *pp, const double *v, double *K) {
  const oracle_problem *p = &c->p;
  const double lm = pp->lambda - 2.0 * pp->mu / 3.0;
  for (int i = 0; i < p->n; ++i) K[i] = 0.0;
  for (int e = 0; e < pp->n_cells; ++e) {
    const int32_t *cn = pp->cells + (int64_t)e * pp->nv;
    for (int q = 0; q < pp->nq; ++q) {
      const double *gr = pp->qgrad + ((int64_t)e * pp->nq + q) * 2 * pp->nv;
      double Dv[2][2] = {{0.0, 0.0}, {0.0, 0.0}}; /* Dv[k][m] = d_m v_k */
      for (int a = 0; a < pp->nv; ++a)
        for (int k = 0; k < 2; ++k)
          for (int m = 0; m < 2; ++m) Dv[k][m] += v[2 * cn[a] + k] * gr[m * pp->nv + a];
      double ee = 0.0;
      for (int k = 0; k < 2; ++k)
        for (int m = 0; m < 2; ++m) {
          double eps = 0.5 * (Dv[k][m] + Dv[m][k]);
          ee += eps * eps;
        }
      const double div = Dv[0][0] + Dv[1][1];
      const double se = 2.0 * pp->mu * ee + lm * div * div; /* sigma(v):eps(v) */
      const double w = pp->qw[(int64_t)e * pp->nq + q];
      for (int a = 0; a < pp->nv; ++a) K[cn[a]] += w * pp->qphi[((int64_t)e * pp->nq + q) * pp->nv + a] * se;
    }
  }
  for (int i = 0; i < p->n; ++i) K[i] /= p->mi[i];
}

/* One parabolic sub-step over dt (2 tau in the Strang splitting), U in place:
 * rho unchanged; velocity by Crank-Nicolson (eqs. mt_parabolic_discrete,
 * vel_parabolic_discrete); internal energy by Crank-Nicolson with the viscous
 * source K (eqs. def_Ki_nplusone, high_int_energy_CN); if some e_i^{n+1} <= 0,
 * the low-order backward-Euler update (eq. low_order_update_internal_energy)
 * and FCT limiting of A_ij (eq. Aij_for_internal_energy); total energy by
 * eq. energy_parabolic_discrete. */
int oracle_parabolic_step(oracle_ctx *c, const oracle_parabolic *pp, double *U, double dt,
                          oracle_parabolic_info *info) {
  const oracle_problem *p = &c->p;
  if (p->dim != 2 || !pp || !(dt > 0.0)) return ORACLE_ERR_ARG;
  const int n = p->n;
  const int64_t nnz = p->nnz;
  int st = ORACLE_OK;
  double *D = malloc(sizeof(double) * n), *V = malloc(sizeof(double) * 2 * n), *Vh = malloc(sizeof(double) * 2 * n);
  double *bv = malloc(sizeof(double) * 2 * n), *Pd = malloc(sizeof(double) * 2 * n);
  double *en = malloc(sizeof(double) * n), *eh = malloc(sizeof(double) * n), *eH = malloc(sizeof(double) * n);
  double *eL = malloc(sizeof(double) * n), *K = malloc(sizeof(double) * n), *be = malloc(sizeof(double) * n);
  double *Pe = malloc(sizeof(double) * n);
  unsigned char *wall = calloc(n, 1);
  if (!D || !V || !Vh || !bv || !Pd || !en || !eh || !eH || !eL || !K || !be || !Pe || !wall) {
    st = ORACLE_ERR_OOM;
    goto done;
  }
  for (int w = 0; w < pp->n_wall; ++w) wall[pp->wall[w]] = 1;
  if (info) memset(info, 0, sizeof(*info));
  const double lm = pp->lambda - 2.0 * pp->mu / 3.0;
  for (int i = 0; i < n; ++i) {
    const double rho = U[i];
    D[i] = rho * p->mi[i];
    V[2 * i] = U[n + i] / rho;
    V[2 * i + 1] = U[2 * n + i] / rho;
    en[i] = U[3 * n + i] / rho - 0.5 * (V[2 * i] * V[2 * i] + V[2 * i + 1] * V[2 * i + 1]);
  }
  /* velocity: (D + dt/2 A) V^{n+1/2} = D V^n (m_i M_i = rho_i m_i V_i), wall rows 0 */
  for (int i = 0; i < n; ++i) {
    int64_t kd = -1;
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
      if (p->col[k] == i) kd = k;
    for (int a = 0; a < 2; ++a) {
      bv[2 * i + a] = wall[i] ? 0.0 : D[i] * V[2 * i + a];
      Vh[2 * i + a] = wall[i] ? 0.0 : V[2 * i + a];
      Pd[2 * i + a] = wall[i] ? 1.0
                              : D[i] + 0.5 * dt * (pp->mu * pp->L[kd] + pp->mu * pp->G[(a * 2 + a) * nnz + kd] +
                                                   lm * pp->G[(a * 2 + a) * nnz + kd]);
    }
  }
  int it = pcg(c, pp, D, wall, 0.5 * dt, 0, Pd, bv, Vh, 2 * (int64_t)n);
  if (it < 0) { st = ORACLE_ERR_ARG; goto done; }
  if (info) info->cg_iter_velocity = it;
  /* internal energy: (D + dt/2 b) e^{n+1/2} = D e^n + dt/2 m K */
  viscous_source(c, pp, Vh, K);
  for (int i = 0; i < n; ++i) {
    int64_t kd = -1;
    for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
      if (p->col[k] == i) kd = k;
    be[i] = D[i] * en[i] + 0.5 * dt * p->mi[i] * K[i];
    eh[i] = en[i];
    Pe[i] = D[i] + 0.5 * dt * pp->kappa_cv * pp->L[kd];
  }
  it = pcg(c, pp, D, wall, 0.5 * dt * pp->kappa_cv, 1, Pe, be, eh, n);
  if (it < 0) { st = ORACLE_ERR_ARG; goto done; }
  if (info) info->cg_iter_energy = it;
  int negative = 0;
  for (int i = 0; i < n; ++i) {
    eH[i] = 2.0 * eh[i] - en[i];
    if (!(eH[i] > 0.0)) negative = 1;
  }
  if (negative) {
    /* low order: (D + dt b) e^L = D e^n + dt m K (the source over the whole
     * step; with it m_i rho_i (e^H_i - e^L_i) = sum_j A_ij holds) */
    for (int i = 0; i < n; ++i) {
      int64_t kd = -1;
      for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
        if (p->col[k] == i) kd = k;
      be[i] = D[i] * en[i] + dt * p->mi[i] * K[i];
      eL[i] = en[i];
      Pe[i] = D[i] + dt * pp->kappa_cv * pp->L[kd];
    }
    it = pcg(c, pp, D, wall, dt * pp->kappa_cv, 1, Pe, be, eL, n);
    if (it < 0) { st = ORACLE_ERR_ARG; goto done; }
    if (info) { info->cg_iter_low = it; info->limited = 1; }
    /* FCT (Zalesak) with the local bounds of the low-order solution */
    double *Rp = malloc(sizeof(double) * n), *Rm = malloc(sizeof(double) * n);
    if (!Rp || !Rm) { free(Rp); free(Rm); st = ORACLE_ERR_OOM; goto done; }
    for (int i = 0; i < n; ++i) {
      double emin = eL[i], emax = eL[i], pp_ = 0.0, pm = 0.0;
      const double xi = eH[i] + en[i] - 2.0 * eL[i];
      for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
        const int j = p->col[k];
        if (j == i) continue;
        emin = fmin(emin, eL[j]);
        emax = fmax(emax, eL[j]);
        const double A = -0.5 * dt * pp->kappa_cv * pp->L[k] * ((eH[j] + en[j] - 2.0 * eL[j]) - xi);
        if (A > 0.0) pp_ += A; else pm += A;
      }
      const double qp = D[i] * (emax - eL[i]), qm = D[i] * (emin - eL[i]);
      Rp[i] = pp_ > 0.0 ? fmin(1.0, qp / pp_) : 1.0;
      Rm[i] = pm < 0.0 ? fmin(1.0, qm / pm) : 1.0;
    }
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      const double xi = eH[i] + en[i] - 2.0 * eL[i];
      for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
        const int j = p->col[k];
        if (j == i) continue;
        const double A = -0.5 * dt * pp->kappa_cv * pp->L[k] * ((eH[j] + en[j] - 2.0 * eL[j]) - xi);
        const double l = A > 0.0 ? fmin(Rp[i], Rm[j]) : fmin(Rm[i], Rp[j]);
        acc += l * A;
      }
      eh[i] = eL[i] + acc / D[i]; /* limited e^{n+1} (eh reused) */
    }
    free(Rp);
    free(Rm);
    for (int i = 0; i < n; ++i) eH[i] = eh[i];
  }
  double emin = INFINITY;
  for (int i = 0; i < n; ++i) {
    const double rho = U[i];
    const double v0 = 2.0 * Vh[2 * i] - V[2 * i], v1 = 2.0 * Vh[2 * i + 1] - V[2 * i + 1];
    U[n + i] = rho * v0;
    U[2 * n + i] = rho * v1;
    U[3 * n + i] = rho * eH[i] + 0.5 * rho * (v0 * v0 + v1 * v1);
    emin = fmin(emin, eH[i]);
  }
  if (info) info->min_e = emin;
done:
  free(D); free(V); free(Vh); free(bv); free(Pd); free(en); free(eh); free(eH); free(eL); free(K); free(be);
  free(Pe); free(wall);
  return st;
}

/* eq. continuous_Strang: U <- H(tau) P(2 tau) H(tau) U, tau the CFL step of
 * the first hyperbolic step (dt <= 0) or dt. */
int oracle_ns_step(oracle_ctx *c, const oracle_parabolic *pp, double *U, double dt, double *tau_used,
                   oracle_parabolic_info *info) {
  double tau = 0.0;
  int st = oracle_ssprk3_step(c, U, dt, &tau, NULL);
  if (st) return st;
  st = oracle_parabolic_step(c, pp, U, 2.0 * tau, info);
  if (st) return st;
  st = oracle_ssprk3_step(c, U, tau, NULL, NULL);
  if (st) return st;
  if (tau_used) *tau_used = tau;
  return ORACLE_OK;
}
