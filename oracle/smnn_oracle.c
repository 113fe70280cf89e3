/*
 * smnn_oracle.c -- plain FP64 CPU oracle for the S-MNN weighted least-squares
 * solve (Scalable Mechanistic Neural Networks, Sec. 3.1-3.2, App. A.1, A.3).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. Only the tests, the package smoke check
 * and the benchmark's CPU-baseline leg load it. The CUDA library never links,
 * loads or calls it, and it shares no code, header or table with that library.
 *
 * What it computes, for one system (one sequence/dimension pair) of V variables with
 * Q governing equations per step (Sec. 3.1; V = Q = 1 is the scalar case):
 *
 *   1. The rows of A, b and the diagonal weight matrix W, written out one
 *      constraint at a time exactly as Sec. 3.1 states them:
 *        Eq. 4  governing rows per step t, q < Q:
 *                   sum_{v,r} c_{t,q,v,r} y_{t,v,r} = d_{t,q}
 *        Eq. 5  initial-value rows, t <= T_init, v < V, r <= R_init:  y_{t,v,r} = u_{t,v,r}
 *        Eq. 6  forward smoothness, t < T, v < V, r <= R:
 *                   y_{t+1,v,r} = sum_{r'>=r} s_t^{r'-r}/(r'-r)! y_{t,v,r'}
 *        Eq. 7  backward smoothness, t < T, v < V, r <= R:
 *                   y_{t,v,r}   = sum_{r'>=r} (-s_t)^{r'-r}/(r'-r)! y_{t+1,v,r'}
 *      Row order and signs follow App. A.1 (A_gov, A_init, A_smooth_forward
 *      = [A+_t, -I], A_smooth_backward = [-I, A-_t]); b is d, u, then zeros;
 *      the weights are w_gov^2, w_init^2 and (w_smooth s_t^r)^2 (App. A.1).
 *      Unknown y_{t,v,r} sits at column t*V(R+1) + v(R+1) + r (Sec. 3.2, 0-based
 *      here); the step size s_t is shared by the V variables.
 *   2. y = (A^T W A)^{-1} A^T W b (Eq. 9), by forming M = A^T W A and
 *      beta = A^T W b from the rows and factoring M with a textbook scalar
 *      band Cholesky (half-bandwidth 2(R+1)-1), or densely (Cholesky, or
 *      Householder QR of W^{1/2} A) for tiny systems; or, for any T and for
 *      ill-conditioned problems, as argmin ||W^{1/2}(A y - b)|| by a band QR of
 *      W^{1/2} A with plane rotations (no normal equations).  No block
 *      structure, no App. A.2 closed forms, no reordering.
 *   3. Gradients for a loss l(y) given dl/dy (Sec. 3.2, Eq. 14): with
 *      g = M^{-1} dl/dy and per-row residual e_k = b_k - a_k.y,
 *        dl/dtheta = sum_k [ (da_k.g) w_k e_k + (a_k.g) dw_k e_k
 *                            + (a_k.g) w_k db_k - (a_k.g) w_k (da_k.y) ]
 *      where da_k, dw_k, db_k are the derivatives of row k's entries, weight
 *      and right-hand side with respect to theta, written out entry by entry
 *      from the constraint definitions (e.g. d(s^k/k!)/ds = s^{k-1}/(k-1)!).
 *      This is the chain rule of dy = M^{-1}(dbeta - dM y) with M = A^T W A.
 *
 * Pins (tests in tests/test_oracle_*.py check this file against them):
 *   - App. A.2's closed-form blocks M_t, N_t, beta_t equal A^T W A, A^T W b;
 *   - a hand-worked R=1, T=2 example of the rows (tests/golden/);
 *   - row count m of Eq. 8;
 *   - exact recovery of degree<=R polynomial trajectories (zero residual);
 *   - w_gov = 0, R_init = R reduces to Taylor propagation y_{t+1}=exp(s_t N)y_t;
 *   - dense Householder QR, dense Cholesky, band Cholesky and band QR agree,
 *     the band factor solves the same system as LAPACK's band Cholesky, and
 *     band QR matches numpy's least-squares solver where the normal
 *     equations lose digits;
 *   - symmetry, positive definiteness and A^T W (b - A y) = 0;
 *   - gradients against central finite differences of the solve;
 *   - the closed-form ODE solutions of App. B.1 land near Table 5's errors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_R 7
#define ORC_MAX_NZ 16   /* nonzeros of a row: V(R+1) for a governing row, <= R+2 otherwise */

typedef struct {
  int32_t R;       /* highest derivative order; R+1 unknowns per step   */
  int32_t R_init;  /* initial values given for orders 0..R_init          */
  int32_t T_init;  /* initial values given for steps 1..T_init           */
  int32_t V;       /* variables per step (Sec. 3.1), >= 1                */
  int32_t Q;       /* governing equations per step, >= 1                 */
  int32_t pad_;
  double w_gov, w_init, w_smooth; /* importance weights (unsquared)      */
} orc_params;

enum { ROW_GOV = 0, ROW_INIT = 1, ROW_FWD = 2, ROW_BWD = 3 };

/* One row of A with its right-hand side and weight, plus the derivatives of
 * its entries and weight with respect to the step size s_t it depends on. */
typedef struct {
  int32_t kind, t, r, nnz;
  int64_t col[ORC_MAX_NZ];
  double val[ORC_MAX_NZ];
  double dval_ds[ORC_MAX_NZ];
  double b, w, dw_ds;
  double dw_dimp;  /* d w / d (the row's importance weight w_gov, w_init or w_smooth) */
} orc_row;

static double orc_factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}

/* x^k for integer k >= 0, with x^0 = 1 (also for x = 0). */
static double orc_powi(double x, int k) {
  double p = 1.0;
  for (int i = 0; i < k; ++i) p *= x;
  return p;
}

/* Unknowns per step. */
static int orc_nb(const orc_params* p) { return p->V * (p->R + 1); }

static int orc_params_ok(const orc_params* p) {
  return p->R >= 0 && p->R <= ORC_MAX_R && p->R_init >= 0 && p->R_init <= p->R && p->T_init >= 1 &&
         p->V >= 1 && p->Q >= 1 && orc_nb(p) <= ORC_MAX_NZ;
}

/* m of Eq. 8. */
int64_t orc_num_rows(const orc_params* p, int64_t T) {
  return T * p->Q + (int64_t)p->T_init * p->V * (p->R_init + 1) + 2 * (T - 1) * (int64_t)orc_nb(p);
}

/* One row of each kind (App. A.1), written out from its constraint.  c: [T][Q][V(R+1)],
 * d: [T][Q], s: [T], u: [T_init][V][R_init+1] of one system.  The row is cleared first. */

/* Eq. 4: sum_{v,r} c_{t,q,v,r} y_{t,v,r} = d_{t,q}, weight w_gov^2. */
static void orc_gov_row(const orc_params* p, int64_t t, int q, const double* c, const double* d,
                        orc_row* w) {
  const int nb = orc_nb(p);
  memset(w, 0, sizeof(*w));
  w->kind = ROW_GOV; w->t = (int32_t)t; w->r = q; w->nnz = nb;
  for (int a = 0; a < nb; ++a) {
    w->col[a] = t * nb + a;
    w->val[a] = c[(t * p->Q + q) * nb + a];
  }
  w->b = d[t * p->Q + q];
  w->w = p->w_gov * p->w_gov;
  w->dw_dimp = 2.0 * p->w_gov;
}

/* Eq. 5: y_{t,v,r} = u_{t,v,r} for t < T_init, r <= R_init, weight w_init^2. */
static void orc_init_row(const orc_params* p, int64_t t, int v, int r, const double* u, orc_row* w) {
  const int nb = orc_nb(p), r1 = p->R + 1;
  memset(w, 0, sizeof(*w));
  w->kind = ROW_INIT; w->t = (int32_t)t; w->r = v * (p->R_init + 1) + r; w->nnz = 1;
  w->col[0] = t * nb + v * r1 + r;
  w->val[0] = 1.0;
  w->b = u[(t * p->V + v) * (p->R_init + 1) + r];
  w->w = p->w_init * p->w_init;
  w->dw_dimp = 2.0 * p->w_init;
}

/* Eq. 6 as the row  sum_{r'>=r} s^{r'-r}/(r'-r)! y_{t,r'} - y_{t+1,r} = 0
 * (App. A.1: block t is A+_t, block t+1 is -I); weight (w_smooth s_t^r)^2. */
static void orc_fwd_row(const orc_params* p, int64_t t, int v, int r, const double* s, orc_row* w) {
  const int nb = orc_nb(p), r1 = p->R + 1;
  const double st = s[t];
  memset(w, 0, sizeof(*w));
  w->kind = ROW_FWD; w->t = (int32_t)t; w->r = r; w->nnz = 0;
  for (int rp = r; rp < r1; ++rp) {
    const int q = rp - r;
    w->col[w->nnz] = t * nb + v * r1 + rp;
    w->val[w->nnz] = orc_powi(st, q) / orc_factorial(q);
    w->dval_ds[w->nnz] = q > 0 ? orc_powi(st, q - 1) / orc_factorial(q - 1) : 0.0;
    w->nnz++;
  }
  w->col[w->nnz] = (t + 1) * nb + v * r1 + r;
  w->val[w->nnz] = -1.0;
  w->dval_ds[w->nnz] = 0.0;
  w->nnz++;
  w->b = 0.0;
  w->w = orc_powi(p->w_smooth * orc_powi(st, r), 2);
  w->dw_ds = r > 0 ? 2.0 * r * p->w_smooth * p->w_smooth * orc_powi(st, 2 * r - 1) : 0.0;
  w->dw_dimp = 2.0 * p->w_smooth * orc_powi(st, 2 * r);
}

/* Eq. 7 as the row  -y_{t,r} + sum_{r'>=r} (-s)^{r'-r}/(r'-r)! y_{t+1,r'} = 0
 * (App. A.1: block t is -I, block t+1 is A-_t); same weight as Eq. 6. */
static void orc_bwd_row(const orc_params* p, int64_t t, int v, int r, const double* s, orc_row* w) {
  const int nb = orc_nb(p), r1 = p->R + 1;
  const double st = s[t];
  memset(w, 0, sizeof(*w));
  w->kind = ROW_BWD; w->t = (int32_t)t; w->r = r; w->nnz = 0;
  w->col[w->nnz] = t * nb + v * r1 + r;
  w->val[w->nnz] = -1.0;
  w->dval_ds[w->nnz] = 0.0;
  w->nnz++;
  for (int rp = r; rp < r1; ++rp) {
    const int q = rp - r;
    w->col[w->nnz] = (t + 1) * nb + v * r1 + rp;
    w->val[w->nnz] = orc_powi(-st, q) / orc_factorial(q);
    /* d/ds (-s)^q/q! = -(-s)^{q-1}/(q-1)! */
    w->dval_ds[w->nnz] = q > 0 ? -orc_powi(-st, q - 1) / orc_factorial(q - 1) : 0.0;
    w->nnz++;
  }
  w->b = 0.0;
  w->w = orc_powi(p->w_smooth * orc_powi(st, r), 2);
  w->dw_ds = r > 0 ? 2.0 * r * p->w_smooth * p->w_smooth * orc_powi(st, 2 * r - 1) : 0.0;
  w->dw_dimp = 2.0 * p->w_smooth * orc_powi(st, 2 * r);
}

/* Rows of A, b, W for one system of T steps, in App. A.1's order: governing rows, initial
 * rows, forward smoothness rows, backward smoothness rows. */
void orc_build_rows(const orc_params* p, int64_t T, const double* c, const double* d,
                    const double* s, const double* u, orc_row* rows) {
  const int r1 = p->R + 1;
  int64_t k = 0;
  for (int64_t t = 0; t < T; ++t)
    for (int q = 0; q < p->Q; ++q) orc_gov_row(p, t, q, c, d, &rows[k++]);
  for (int64_t t = 0; t < p->T_init; ++t)
    for (int v = 0; v < p->V; ++v)
      for (int r = 0; r <= p->R_init; ++r) orc_init_row(p, t, v, r, u, &rows[k++]);
  for (int64_t t = 0; t + 1 < T; ++t)
    for (int v = 0; v < p->V; ++v)
      for (int r = 0; r < r1; ++r) orc_fwd_row(p, t, v, r, s, &rows[k++]);
  for (int64_t t = 0; t + 1 < T; ++t)
    for (int v = 0; v < p->V; ++v)
      for (int r = 0; r < r1; ++r) orc_bwd_row(p, t, v, r, s, &rows[k++]);
}

/* ---------------------------------------------------------------------------
 * Dense forms, for tiny systems.
 * ------------------------------------------------------------------------- */

/* Explicit A [m][n], b [m], w [m] (the diagonal of W). */
void orc_dense_system(const orc_params* p, int64_t T, const double* c, const double* d,
                      const double* s, const double* u, double* A, double* b, double* w) {
  const int64_t m = orc_num_rows(p, T), n = T * orc_nb(p);
  orc_row* rows = (orc_row*)malloc(sizeof(orc_row) * (size_t)m);
  orc_build_rows(p, T, c, d, s, u, rows);
  memset(A, 0, sizeof(double) * (size_t)(m * n));
  for (int64_t k = 0; k < m; ++k) {
    for (int j = 0; j < rows[k].nnz; ++j) A[k * n + rows[k].col[j]] += rows[k].val[j];
    b[k] = rows[k].b;
    w[k] = rows[k].w;
  }
  free(rows);
}

/* In-place dense Cholesky of the n x n row-major SPD matrix a (lower part).
 * Returns 0, or j+1 for the first non-positive pivot j. */
static int orc_dense_cholesky(int64_t n, double* a) {
  for (int64_t j = 0; j < n; ++j) {
    double djj = a[j * n + j];
    for (int64_t k = 0; k < j; ++k) djj -= a[j * n + k] * a[j * n + k];
    if (!(djj > 0.0)) return (int)(j + 1);
    const double ljj = sqrt(djj);
    a[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double v = a[i * n + j];
      for (int64_t k = 0; k < j; ++k) v -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = v / ljj;
    }
  }
  return 0;
}

/* y = (A^T W A)^{-1} A^T W b with a dense Cholesky of M (Eq. 9). */
int orc_solve_dense_normal(const orc_params* p, int64_t T, const double* c, const double* d,
                           const double* s, const double* u, double* y) {
  const int64_t m = orc_num_rows(p, T), n = T * orc_nb(p);
  double* A = (double*)malloc(sizeof(double) * (size_t)(m * n));
  double* b = (double*)malloc(sizeof(double) * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * (size_t)m);
  double* M = (double*)calloc((size_t)(n * n), sizeof(double));
  orc_dense_system(p, T, c, d, s, u, A, b, w);
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t k = 0; k < m; ++k) acc += A[k * n + i] * w[k] * b[k];
    y[i] = acc;
    for (int64_t j = 0; j <= i; ++j) {
      double mij = 0.0;
      for (int64_t k = 0; k < m; ++k) mij += A[k * n + i] * w[k] * A[k * n + j];
      M[i * n + j] = mij;
    }
  }
  const int info = orc_dense_cholesky(n, M);
  if (info == 0) {
    for (int64_t i = 0; i < n; ++i) {           /* L z = beta */
      double v = y[i];
      for (int64_t k = 0; k < i; ++k) v -= M[i * n + k] * y[k];
      y[i] = v / M[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {      /* L^T y = z */
      double v = y[i];
      for (int64_t k = i + 1; k < n; ++k) v -= M[k * n + i] * y[k];
      y[i] = v / M[i * n + i];
    }
  }
  free(A); free(b); free(w); free(M);
  return info;
}

/* y = argmin || W^{1/2}(A y - b) || by Householder QR of W^{1/2} A, without
 * forming the normal equations (the brute-force least-squares definition). */
int orc_solve_dense_qr(const orc_params* p, int64_t T, const double* c, const double* d,
                       const double* s, const double* u, double* y) {
  const int64_t m = orc_num_rows(p, T), n = T * orc_nb(p);
  double* A = (double*)malloc(sizeof(double) * (size_t)(m * n));
  double* b = (double*)malloc(sizeof(double) * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * (size_t)m);
  double* v = (double*)malloc(sizeof(double) * (size_t)m);
  orc_dense_system(p, T, c, d, s, u, A, b, w);
  for (int64_t k = 0; k < m; ++k) {
    const double sw = sqrt(w[k]);
    for (int64_t j = 0; j < n; ++j) A[k * n + j] *= sw;
    b[k] *= sw;
  }
  int info = 0;
  for (int64_t j = 0; j < n; ++j) {
    double norm = 0.0;
    for (int64_t k = j; k < m; ++k) norm += A[k * n + j] * A[k * n + j];
    norm = sqrt(norm);
    if (norm == 0.0) { info = (int)(j + 1); break; }
    const double alpha = A[j * n + j] > 0 ? -norm : norm;
    for (int64_t k = j; k < m; ++k) v[k] = A[k * n + j];
    v[j] -= alpha;
    double vv = 0.0;
    for (int64_t k = j; k < m; ++k) vv += v[k] * v[k];
    for (int64_t jj = j; jj < n; ++jj) {        /* A <- (I - 2 v v^T / v^T v) A */
      double dot = 0.0;
      for (int64_t k = j; k < m; ++k) dot += v[k] * A[k * n + jj];
      const double f = 2.0 * dot / vv;
      for (int64_t k = j; k < m; ++k) A[k * n + jj] -= f * v[k];
    }
    double dot = 0.0;
    for (int64_t k = j; k < m; ++k) dot += v[k] * b[k];
    const double f = 2.0 * dot / vv;
    for (int64_t k = j; k < m; ++k) b[k] -= f * v[k];
  }
  if (info == 0) {
    for (int64_t i = n - 1; i >= 0; --i) {      /* R y = Q^T W^{1/2} b */
      double acc = b[i];
      for (int64_t k = i + 1; k < n; ++k) acc -= A[i * n + k] * y[k];
      y[i] = acc / A[i * n + i];
    }
  }
  free(A); free(b); free(w); free(v);
  return info;
}

/* ---------------------------------------------------------------------------
 * Band forms, for any T.  Lower band storage: band[i*(kd+1) + (i-j)] holds
 * M[i][j] for 0 <= i-j <= kd; kd = 2(R+1)-1 is the widest column distance
 * inside one row of A (a backward smoothness row spans y_{t,r}..y_{t+1,R}).
 * ------------------------------------------------------------------------- */

int orc_band_width(const orc_params* p) { return 2 * orc_nb(p) - 1; }

/* M = A^T W A and beta = A^T W b accumulated row by row. */
static void orc_normal_band_rows(const orc_row* rows, int64_t m, int64_t n, int kd,
                                 double* band, double* beta) {
  memset(band, 0, sizeof(double) * (size_t)(n * (kd + 1)));
  memset(beta, 0, sizeof(double) * (size_t)n);
  for (int64_t k = 0; k < m; ++k) {
    const orc_row* w = &rows[k];
    for (int a = 0; a < w->nnz; ++a) {
      beta[w->col[a]] += w->w * w->val[a] * w->b;
      for (int q = 0; q < w->nnz; ++q) {
        if (w->col[a] >= w->col[q])
          band[w->col[a] * (kd + 1) + (w->col[a] - w->col[q])] += w->w * w->val[a] * w->val[q];
      }
    }
  }
}

/* Textbook band Cholesky, in place.  Returns 0 or (first bad row)+1. */
int orc_band_cholesky(int64_t n, int kd, double* a) {
  const int ld = kd + 1;
  for (int64_t j = 0; j < n; ++j) {
    double djj = a[j * ld];
    const int64_t k0 = j - kd > 0 ? j - kd : 0;
    for (int64_t k = k0; k < j; ++k) djj -= a[j * ld + (j - k)] * a[j * ld + (j - k)];
    if (!(djj > 0.0)) return (int)(j + 1);
    const double ljj = sqrt(djj);
    a[j * ld] = ljj;
    const int64_t iend = j + kd < n - 1 ? j + kd : n - 1;
    for (int64_t i = j + 1; i <= iend; ++i) {
      double v = a[i * ld + (i - j)];
      const int64_t kk0 = i - kd > 0 ? i - kd : 0;
      for (int64_t k = kk0; k < j; ++k) v -= a[i * ld + (i - k)] * a[j * ld + (j - k)];
      a[i * ld + (i - j)] = v / ljj;
    }
  }
  return 0;
}

/* Solve L L^T x = rhs with the band factor, in place on x. */
void orc_band_solve(int64_t n, int kd, const double* l, double* x) {
  const int ld = kd + 1;
  for (int64_t i = 0; i < n; ++i) {
    double v = x[i];
    const int64_t k0 = i - kd > 0 ? i - kd : 0;
    for (int64_t k = k0; k < i; ++k) v -= l[i * ld + (i - k)] * x[k];
    x[i] = v / l[i * ld];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double v = x[i];
    const int64_t kend = i + kd < n - 1 ? i + kd : n - 1;
    for (int64_t k = i + 1; k <= kend; ++k) v -= l[k * ld + (k - i)] * x[k];
    x[i] = v / l[i * ld];
  }
}

/* Band M and beta of one system (for comparison with a library band solver). */
void orc_normal_band(const orc_params* p, int64_t T, const double* c, const double* d,
                     const double* s, const double* u, double* band, double* beta) {
  const int64_t m = orc_num_rows(p, T), n = T * orc_nb(p);
  orc_row* rows = (orc_row*)malloc(sizeof(orc_row) * (size_t)m);
  orc_build_rows(p, T, c, d, s, u, rows);
  orc_normal_band_rows(rows, m, n, orc_band_width(p), band, beta);
  free(rows);
}

/* Solve one system in band mode; returns 0 or the failing unknown's index+1. */
static int orc_solve_one_band(const orc_params* p, int64_t T, const double* c, const double* d,
                              const double* s, const double* u, double* y) {
  const int64_t m = orc_num_rows(p, T), n = T * orc_nb(p);
  const int kd = orc_band_width(p);
  orc_row* rows = (orc_row*)malloc(sizeof(orc_row) * (size_t)m);
  double* band = (double*)malloc(sizeof(double) * (size_t)(n * (kd + 1)));
  orc_build_rows(p, T, c, d, s, u, rows);
  orc_normal_band_rows(rows, m, n, kd, band, y);
  const int info = orc_band_cholesky(n, kd, band);
  if (info == 0) orc_band_solve(n, kd, band, y);
  free(rows); free(band);
  return info;
}

/* ---------------------------------------------------------------------------
 * Band Givens QR of W^{1/2} A, for any T: the least-squares definition of Eq. 9 solved
 * without forming the normal equations, whose condition number is the square of that of
 * W^{1/2} A (what an ill-conditioned problem needs; Golub & Van Loan's banded QR by plane
 * rotations).  A row's nonzeros lie in columns [f, f+kd], kd = 2V(R+1)-1; so do the rows of
 * R = Q^T W^{1/2} A shifted to their diagonal: R[i][j] for 0 <= j-i <= kd, stored at
 * rb[i*(kd+1) + (j-i)].  Each row of W^{1/2} A, W^{1/2} b is merged into R and q = Q^T W^{1/2} b
 * as it is generated (step by step, never all rows at once): for pivot j = f, f+1, ... its
 * leading entry is annihilated by a rotation with R's row j, after which its nonzeros lie in
 * [j+1, j+kd]; a row reaching an R row not yet filled becomes that row.  Then R y = q.
 * ------------------------------------------------------------------------- */

static void orc_qr_merge_row(const orc_row* w, int64_t n, int kd, double* rb, unsigned char* filled,
                             double* q) {
  const int ld = kd + 1;
  double a[2 * ORC_MAX_NZ];
  const double sw = sqrt(w->w);
  int64_t j = w->col[0];
  for (int k = 1; k < w->nnz; ++k) j = w->col[k] < j ? w->col[k] : j;
  for (int k = 0; k < ld; ++k) a[k] = 0.0;
  for (int k = 0; k < w->nnz; ++k) a[w->col[k] - j] += sw * w->val[k];
  double beta = sw * w->b;
  for (; j < n; ++j) {
    if (a[0] != 0.0) {
      double* rj = rb + j * ld;
      if (!filled[j]) {                      /* the row becomes R's row j */
        for (int k = 0; k < ld; ++k) rj[k] = a[k];
        q[j] = beta;
        filled[j] = 1;
        return;
      }
      const double r = hypot(rj[0], a[0]);
      const double cs = rj[0] / r, sn = a[0] / r;
      for (int k = 0; k < ld; ++k) {
        const double rv = rj[k], av = a[k];
        rj[k] = cs * rv + sn * av;
        a[k] = cs * av - sn * rv;
      }
      const double qv = q[j];
      q[j] = cs * qv + sn * beta;
      beta = cs * beta - sn * qv;
    }
    int nz = 0;                              /* next pivot: shift the window by one column */
    for (int k = 0; k + 1 < ld; ++k) {
      a[k] = a[k + 1];
      nz |= a[k] != 0.0;
    }
    a[ld - 1] = 0.0;
    if (!nz) return;                         /* only its residual share beta is left */
  }
}

/* y of one system by band QR; returns 0 or (first zero pivot of R)+1. */
static int orc_solve_one_qr_band(const orc_params* p, int64_t T, const double* c, const double* d,
                                 const double* s, const double* u, double* y) {
  const int nb = orc_nb(p), r1 = p->R + 1, kd = orc_band_width(p), ld = kd + 1;
  const int64_t n = T * nb;
  double* rb = (double*)calloc((size_t)(n * ld), sizeof(double));
  double* q = (double*)calloc((size_t)n, sizeof(double));
  unsigned char* filled = (unsigned char*)calloc((size_t)n, 1);
  orc_row w;
  for (int64_t t = 0; t < T; ++t) {          /* the rows of step t and of the pair (t, t+1) */
    for (int qq = 0; qq < p->Q; ++qq) { orc_gov_row(p, t, qq, c, d, &w); orc_qr_merge_row(&w, n, kd, rb, filled, q); }
    if (t < p->T_init)
      for (int v = 0; v < p->V; ++v)
        for (int r = 0; r <= p->R_init; ++r) { orc_init_row(p, t, v, r, u, &w); orc_qr_merge_row(&w, n, kd, rb, filled, q); }
    if (t + 1 < T)
      for (int v = 0; v < p->V; ++v)
        for (int r = 0; r < r1; ++r) {
          orc_fwd_row(p, t, v, r, s, &w); orc_qr_merge_row(&w, n, kd, rb, filled, q);
          orc_bwd_row(p, t, v, r, s, &w); orc_qr_merge_row(&w, n, kd, rb, filled, q);
        }
  }
  int info = 0;
  for (int64_t i = n - 1; i >= 0; --i) {     /* R y = q */
    const double* ri = rb + i * ld;
    if (!filled[i] || ri[0] == 0.0) { info = (int)(i + 1); break; }
    double acc = q[i];
    const int64_t kend = i + kd < n - 1 ? i + kd : n - 1;
    for (int64_t k = i + 1; k <= kend; ++k) acc -= ri[k - i] * y[k];
    y[i] = acc / ri[0];
  }
  free(rb); free(q); free(filled);
  return info;
}

/* Gradients of one system (see the file header for the formula).
 * gy: dl/dy [T][R+1]; outputs y, gc [T][R+1], gd [T], gs [T] (this system's
 * share; the last entry is 0), gu [T_init][R_init+1]. */
static int orc_grad_one(const orc_params* p, int64_t T, const double* c, const double* d,
                        const double* s, const double* u, const double* gy, double* y,
                        double* gc, double* gd, double* gs, double* gu, double* gw) {
  const int nb = orc_nb(p);
  const int64_t m = orc_num_rows(p, T), n = T * nb;
  const int kd = orc_band_width(p);
  orc_row* rows = (orc_row*)malloc(sizeof(orc_row) * (size_t)m);
  double* band = (double*)malloc(sizeof(double) * (size_t)(n * (kd + 1)));
  double* g = (double*)malloc(sizeof(double) * (size_t)n);
  orc_build_rows(p, T, c, d, s, u, rows);
  orc_normal_band_rows(rows, m, n, kd, band, y);
  const int info = orc_band_cholesky(n, kd, band);
  memset(gc, 0, sizeof(double) * (size_t)(n * p->Q));
  memset(gd, 0, sizeof(double) * (size_t)(T * p->Q));
  memset(gs, 0, sizeof(double) * (size_t)T);
  memset(gu, 0, sizeof(double) * (size_t)(p->T_init * p->V * (p->R_init + 1)));
  gw[0] = gw[1] = gw[2] = 0.0;
  if (info == 0) {
    orc_band_solve(n, kd, band, y);                   /* y = M^{-1} beta    */
    memcpy(g, gy, sizeof(double) * (size_t)n);
    orc_band_solve(n, kd, band, g);                   /* g = M^{-1} dl/dy   */
    for (int64_t k = 0; k < m; ++k) {
      const orc_row* w = &rows[k];
      double ay = 0.0, ag = 0.0, day = 0.0, dag = 0.0;
      for (int j = 0; j < w->nnz; ++j) {
        ay += w->val[j] * y[w->col[j]];
        ag += w->val[j] * g[w->col[j]];
        day += w->dval_ds[j] * y[w->col[j]];
        dag += w->dval_ds[j] * g[w->col[j]];
      }
      const double e = w->b - ay;
      /* theta = the row's importance weight: da = db = 0, dw = dw_dimp (App. A.1's W). */
      gw[w->kind == ROW_GOV ? 0 : (w->kind == ROW_INIT ? 1 : 2)] += ag * w->dw_dimp * e;
      if (w->kind == ROW_GOV) {
        /* theta = c_{t,q,a}: da = unit vector at column (t,a); dw = db = 0.
         * theta = d_{t,q}:   db = 1. */
        const int64_t gq = (int64_t)w->t * p->Q + w->r;
        for (int j = 0; j < w->nnz; ++j) {
          const int64_t col = w->col[j];
          gc[gq * nb + (col - (int64_t)w->t * nb)] += g[col] * w->w * e - ag * w->w * y[col];
        }
        gd[gq] += ag * w->w;
      } else if (w->kind == ROW_INIT) {
        /* theta = u_{t,v,r}: db = 1 (w->r = v (R_init+1) + r). */
        gu[(int64_t)w->t * p->V * (p->R_init + 1) + w->r] += ag * w->w;
      } else {
        /* theta = s_t: da = dval_ds, dw = dw_ds, db = 0. */
        gs[w->t] += dag * w->w * e + ag * w->dw_ds * e - ag * w->w * day;
      }
    }
  }
  free(rows); free(band); free(g);
  return info;
}

/* ---------------------------------------------------------------------------
 * Batched entry points (OpenMP over systems).  System i has T_sys[i] steps;
 * its per-step arrays start at step offset off[i] (c, y, gc, gy: off[i]*(R+1);
 * d, gd: off[i]); its step sizes start at s + soff[i]; its initial values at
 * u + i*T_init*(R_init+1).  Systems that share soff share one sequence's s,
 * and gs (indexed like s) receives the sum of their shares.
 * info[i]: 0, or the 1-based step of the first non-positive pivot.
 * ------------------------------------------------------------------------- */

int orc_solve_batch(const orc_params* p, int64_t S, const int64_t* T_sys, const int64_t* off,
                    const int64_t* soff, const double* c, const double* d, const double* s,
                    const double* u, double* y, int32_t* info, int nthreads) {
  const int nb = orc_nb(p), nq = p->Q;
  const int nu = p->T_init * p->V * (p->R_init + 1);
  if (!orc_params_ok(p)) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < S; ++i) {
    const int r = orc_solve_one_band(p, T_sys[i], c + off[i] * nq * nb, d + off[i] * nq, s + soff[i],
                                     u + i * nu, y + off[i] * nb);
    info[i] = r == 0 ? 0 : (int32_t)((r - 1) / nb + 1);
  }
  return 0;
}

int orc_grad_batch(const orc_params* p, int64_t S, const int64_t* T_sys, const int64_t* off,
                   const int64_t* soff, const double* c, const double* d, const double* s,
                   const double* u, const double* gy, double* y, double* gc, double* gd,
                   double* gs, double* gu, double* gs_sys, double* gw_sys, int32_t* info,
                   int nthreads) {
  const int nb = orc_nb(p), nq = p->Q;
  const int nu = p->T_init * p->V * (p->R_init + 1);
  if (!orc_params_ok(p)) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < S; ++i) {
    const int r = orc_grad_one(p, T_sys[i], c + off[i] * nq * nb, d + off[i] * nq, s + soff[i],
                               u + i * nu, gy + off[i] * nb, y + off[i] * nb, gc + off[i] * nq * nb,
                               gd + off[i] * nq, gs_sys + off[i], gu + i * nu, gw_sys + 3 * i);
    info[i] = r == 0 ? 0 : (int32_t)((r - 1) / nb + 1);
  }
  /* chain rule for the shared step sizes: sum the systems' shares in order */
  for (int64_t i = 0; i < S; ++i)
    for (int64_t t = 0; t < T_sys[i]; ++t) gs[soff[i] + t] = 0.0;
  for (int64_t i = 0; i < S; ++i)
    for (int64_t t = 0; t < T_sys[i]; ++t) gs[soff[i] + t] += gs_sys[off[i] + t];
  return 0;
}

/* Band-QR batch (any T, OpenMP over systems); layout and info as orc_solve_batch. */
int orc_solve_qr_batch(const orc_params* p, int64_t S, const int64_t* T_sys, const int64_t* off,
                       const int64_t* soff, const double* c, const double* d, const double* s,
                       const double* u, double* y, int32_t* info, int nthreads) {
  const int nb = orc_nb(p), nq = p->Q;
  const int nu = p->T_init * p->V * (p->R_init + 1);
  if (!orc_params_ok(p)) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < S; ++i) {
    const int r = orc_solve_one_qr_band(p, T_sys[i], c + off[i] * nq * nb, d + off[i] * nq, s + soff[i],
                                        u + i * nu, y + off[i] * nb);
    info[i] = r == 0 ? 0 : (int32_t)((r - 1) / nb + 1);
  }
  return 0;
}

/* Dense-mode batch (tiny systems): mode 0 = dense Cholesky, 1 = Householder QR. */
int orc_solve_dense_batch(const orc_params* p, int64_t S, const int64_t* T_sys, const int64_t* off,
                          const int64_t* soff, const double* c, const double* d, const double* s,
                          const double* u, double* y, int32_t* info, int mode) {
  const int nb = orc_nb(p), nq = p->Q;
  const int nu = p->T_init * p->V * (p->R_init + 1);
  if (!orc_params_ok(p)) return -1;
  for (int64_t i = 0; i < S; ++i) {
    const int r = mode == 0
        ? orc_solve_dense_normal(p, T_sys[i], c + off[i] * nq * nb, d + off[i] * nq, s + soff[i], u + i * nu, y + off[i] * nb)
        : orc_solve_dense_qr(p, T_sys[i], c + off[i] * nq * nb, d + off[i] * nq, s + soff[i], u + i * nu, y + off[i] * nb);
    info[i] = r == 0 ? 0 : (int32_t)((r - 1) / nb + 1);
  }
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
