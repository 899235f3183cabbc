/*
 * Plain FP64 CPU oracle for BiCGStab with k right-hand sides.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  It shares no code with the CUDA path and
 * is never linked into it: only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.
 *
 * Source: B. Krasnopolsky, "Revisiting Performance of BiCGStab Methods for
 * Solving Systems with Multiple Right-Hand Sides" (arXiv:1907.12874).
 *   - Algorithm 1  (classical BiCGStab)             -> classical_basic()
 *   - Algorithm 2  (merged BiCGStab)                -> classical_merged()
 *   - Algorithm 4  (merged Pipelined BiCGStab)      -> pipelined_*()
 *   - Algorithm 6  (merged Reordered BiCGStab, M^-1 = identity applied as a
 *                   vector copy, as in the paper's benchmarks, Sec. 2.3)
 *                                                   -> reordered_*()
 *   - Algorithm 5  (merged preconditioned BiCGStab)  -> precond_*()
 *   - Algorithm 7  (merged preconditioned Pipelined BiCGStab; the listing's
 *                   "w^_0 = M^-1 w^_0" is read as w^_0 = M^-1 w_0 and its
 *                   "w^_j = M^-1 w_j, t_j = A w^_j" after the w-update as
 *                   w^_{j+1}, t_{j+1})                -> ppipe_*()
 *   - Algorithm 3  (merged Improved BiCGStab, with f_0 = A^T r_0 and the two
 *                   corrections as printed in the listing) -> improved_*()
 *   The preconditioner is the identity applied as a copy (Sec. 2.3) or, with
 *   ORACLE_JACOBI, the Jacobi matrix M = diag(A) (a zero or missing diagonal
 *   entry counts as 1).
 *   - "basic" forms: one BLAS-like loop per vector operation, the
 *     4-vector update of Algorithm 4 split into two calls (Table 2 and its
 *     footnote); "merged" forms: one loop per merged line of the listings.
 *   - Multi-vector layout: the k vectors are stored row-wise in one array,
 *     element (i, c) at i*k + c (Sec. 3.1).
 *
 * How it is written (so a reader can check it against the listings by eye):
 *   - every column c is solved on its own, as a strided view of the
 *     interleaved arrays; nothing couples columns, so column c of a k-RHS
 *     solve is bitwise the single-RHS solve of that column;
 *   - every listing step is one loop over the rows, in listing order;
 *   - dot products are Neumaier-compensated sums in ascending row order;
 *   - build with -ffp-contract=off: no fused multiply-add, every + - * / and
 *     sqrt is one IEEE round-to-nearest operation, evaluated left to right as
 *     written.
 *
 * Readings where the paper is silent (the CUDA path follows the same rules):
 *   R1 stop test: the listings compare a squared residual norm with eps^2;
 *      eps = tol * ||b_c||_2 (relative tolerance), strict "<", per column.
 *   R2 before the loop: ||b_c|| == 0 -> x_c = 0, converged, 0 iterations;
 *      (r0,r0) < eps^2 -> converged with x0, 0 iterations.
 *   R3 a column stops on its own break; its iteration count is the number of
 *      iterates x_{j+1} it formed.  x_{j+1} is formed as soon as omega_j is
 *      known and finite.  After maxit passes the status is MAXIT.
 *   R4 shadow residual r^_0 = r_0.
 *   R5 psi (classical), phi (Pipelined, Reordered): a zero denominator of
 *      omega sets omega = 0.  Any other division by an exact zero in the
 *      scalar recurrences (delta, rho, omega in beta, the alpha denominator
 *      of Algorithm 4) is BREAKDOWN; a non-finite scalar is NONFINITE.
 *   R6 merged norm estimates (theta - omega*phi, pi - omega*theta,
 *      eta - omega*theta) are used as written for the stop test; the history
 *      records sqrt(max(0, estimate)).  The basic classical form computes
 *      (r,r) directly (Algorithm 1, conv-check line).
 *   R7 Algorithm 4: the vectors of step j-1 start at zero, beta_{-1} = 0,
 *      omega_{-1} = 0, alpha_0 = rho_0/(r_0,w_0).
 *   R8 flag ORACLE_NO_STOP_TEST: no convergence test at all (fixed iteration
 *      count benchmarking, Sec. 2.3 uses N_it = 1000); breakdown rules stay.
 *
 * Memory-traffic bookkeeping: every loop reports how many distinct full
 * vectors it reads and writes (SpMV and the identity-preconditioner copies
 * are counted apart), which reproduces the per-iteration counts of Table 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_CLASSICAL_BASIC 0
#define ORACLE_CLASSICAL_MERGED 1
#define ORACLE_REORDERED_BASIC 2
#define ORACLE_REORDERED_MERGED 3
#define ORACLE_PIPELINED_BASIC 4
#define ORACLE_PIPELINED_MERGED 5
#define ORACLE_PRECOND_BASIC 6
#define ORACLE_PRECOND_MERGED 7
#define ORACLE_PPIPE_BASIC 8
#define ORACLE_PPIPE_MERGED 9
#define ORACLE_IMPROVED_BASIC 10
#define ORACLE_IMPROVED_MERGED 11

#define ST_CONVERGED 0
#define ST_MAXIT 1
#define ST_BREAKDOWN 2
#define ST_NONFINITE 3

#define ORACLE_NO_STOP_TEST 1
#define ORACLE_JACOBI 2 /* M = diag(A) instead of the identity (Algorithms 5, 6, 7) */

typedef struct {
  int64_t n;
  const int32_t *rowptr, *colidx;
  const double *vals;
} csr_t;

/* A column of an interleaved N x k block: element i lives at p[i * s]. */
typedef struct {
  double *p;
  int64_t s;
} col_t;

/* Vector read / write counters of the current solve (SpMV and copies apart). */
typedef struct {
  int64_t reads, writes, copies, spmv;
} traffic_t;

static traffic_t g_tr;
static void rw(int r, int w) { g_tr.reads += r; g_tr.writes += w; }

#define AT(v, i) ((v).p[(i) * (v).s])

/* ---------------- primitives ---------------- */

/* y = A x (one SpMV over a strided column). */
static void spmv(const csr_t *A, col_t x, col_t y) {
  g_tr.spmv++;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A->n; ++i) {
    double acc = 0.0;
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) acc += A->vals[e] * AT(x, A->colidx[e]);
    AT(y, i) = acc;
  }
}

/* Neumaier-compensated sum of x_i * y_i, i ascending. */
static double dot(const csr_t *A, col_t x, col_t y) {
  double sum = 0.0, comp = 0.0;
  for (int64_t i = 0; i < A->n; ++i) {
    double p = AT(x, i) * AT(y, i);
    double t = sum + p;
    if (fabs(sum) >= fabs(p))
      comp += (sum - t) + p;
    else
      comp += (p - t) + sum;
    sum = t;
  }
  return sum + comp;
}

/* Compensated accumulator used inside merged loops (same arithmetic as dot()). */
typedef struct {
  double sum, comp;
} acc_t;
static void acc_add(acc_t *a, double p) {
  double t = a->sum + p;
  if (fabs(a->sum) >= fabs(p))
    a->comp += (a->sum - t) + p;
  else
    a->comp += (p - t) + a->sum;
  a->sum = t;
}
static double acc_val(const acc_t *a) { return a->sum + a->comp; }

/* Inverse Jacobi diagonal of the current solve (NULL: M = identity). */
static const double *g_invdiag = NULL;

/* y = M^{-1} x: the identity applied as a copy (Sec. 2.3), or x_i / a_ii (Jacobi). */
static void precond_copy(const csr_t *A, col_t x, col_t y) {
  g_tr.copies++;
  if (g_invdiag) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; ++i) AT(y, i) = AT(x, i) * g_invdiag[i];
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; ++i) AT(y, i) = AT(x, i);
  }
}

/* y = A^T x: y_j = sum_i a_ij x_i, accumulated over i ascending. */
static void spmv_t(const csr_t *A, col_t x, col_t y) {
  g_tr.spmv++;
  for (int64_t j = 0; j < A->n; ++j) AT(y, j) = 0.0;
  for (int64_t i = 0; i < A->n; ++i)
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) AT(y, A->colidx[e]) += A->vals[e] * AT(x, i);
}

static void set_zero(const csr_t *A, col_t y) {
  for (int64_t i = 0; i < A->n; ++i) AT(y, i) = 0.0;
}

static double hist_value(double est) {
  if (isnan(est)) return est;
  return est > 0.0 ? sqrt(est) : 0.0;
}

static int finite(double v) { return isfinite(v) ? 1 : 0; }

/* Per-column result record. */
typedef struct {
  int32_t iters, status;
} res_t;

/* Common set-up shared by every variant: r = b - A x, ||b||^2, rho0, eps^2.
 * Returns 1 if the column is already finished (R2), 0 if it must iterate. */
static int setup(const csr_t *A, col_t b, col_t x, col_t r, col_t tmp, double tol, int flags,
                 double *rho0, double *eps2, double *hist, int64_t hs, res_t *out) {
  spmv(A, x, tmp);
  for (int64_t i = 0; i < A->n; ++i) AT(r, i) = AT(b, i) - AT(tmp, i);
  double bn2 = dot(A, b, b);
  *rho0 = dot(A, r, r);
  *eps2 = tol * tol * bn2;
  hist[0] = hist_value(*rho0);
  (void)hs;
  out->iters = 0;
  if (bn2 == 0.0) { /* R2: b = 0 -> x = 0 */
    set_zero(A, x);
    hist[0] = 0.0;
    out->status = ST_CONVERGED;
    return 1;
  }
  if (!finite(bn2) || !finite(*rho0)) {
    out->status = ST_NONFINITE;
    return 1;
  }
  if (!(flags & ORACLE_NO_STOP_TEST) && *rho0 < *eps2) {
    out->status = ST_CONVERGED;
    return 1;
  }
  return 0;
}

/* ---------------- Algorithm 1: classical BiCGStab, basic form ---------------- */
static void classical_basic(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit,
                            int flags, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], p = w[1], v = w[2], s = w[3], t = w[4];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) AT(r0, i) = AT(r, i); /* r^_0 = r_0 (R4) */
  for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i);  /* p_0 = r_0 */
  for (int j = 0; j < maxit; ++j) {
    spmv(A, p, v);                         /* v_j = A p_j */
    double delta = dot(A, v, r0); rw(2, 0); /* delta_j = (v_j, r_0) */
    if (!finite(delta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (delta == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double alpha = rho / delta;
    if (!finite(alpha)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(r, i) - alpha * AT(v, i); /* s_j */
    rw(2, 1);
    spmv(A, s, t);                        /* t_j = A s_j */
    double phi = dot(A, t, s); rw(2, 0);  /* phi_j = (t_j, s_j) */
    double psi = dot(A, t, t); rw(1, 0);  /* psi_j = (t_j, t_j) */
    if (!finite(phi) || !finite(psi)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double omega = psi == 0.0 ? 0.0 : phi / psi; /* R5 */
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * AT(s, i);
    rw(3, 1);
    for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(s, i) - omega * AT(t, i);
    rw(2, 1);
    out->iters = j + 1;
    double rr = dot(A, r, r); rw(1, 0);   /* (r_{j+1}, r_{j+1}) */
    hist[(j + 1) * hs] = hist_value(rr);
    if (!finite(rr)) { out->status = ST_NONFINITE; return; }
    if (!(flags & ORACLE_NO_STOP_TEST) && rr < eps2) { out->status = ST_CONVERGED; return; }
    double rho1 = dot(A, r, r0); rw(2, 0); /* rho_{j+1} = (r_{j+1}, r_0) */
    if (!finite(rho1)) { out->status = ST_NONFINITE; return; }
    if (rho == 0.0 || omega == 0.0) { out->status = ST_BREAKDOWN; return; }
    double beta = (rho1 / rho) * (alpha / omega);
    if (!finite(beta)) { out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i) + beta * (AT(p, i) - omega * AT(v, i));
    rw(3, 1);
    rho = rho1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- Algorithm 2: merged BiCGStab ---------------- */
static void classical_merged(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit,
                             int flags, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], p = w[1], v = w[2], s = w[3], t = w[4];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) { AT(r0, i) = AT(r, i); AT(p, i) = AT(r, i); }
  for (int j = 0; j < maxit; ++j) {
    spmv(A, p, v);
    double delta = dot(A, v, r0); rw(2, 0);
    if (!finite(delta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (delta == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double alpha = rho / delta;
    if (!finite(alpha)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(r, i) - alpha * AT(v, i);
    rw(2, 1);
    spmv(A, s, t);
    /* group 1: phi = (t,s), psi = (t,t), theta = (s,s) in one pass over t and s */
    acc_t aphi = {0, 0}, apsi = {0, 0}, ath = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
      double ti = AT(t, i), si = AT(s, i);
      acc_add(&aphi, ti * si);
      acc_add(&apsi, ti * ti);
      acc_add(&ath, si * si);
    }
    rw(2, 0);
    double phi = acc_val(&aphi), psi = acc_val(&apsi), theta = acc_val(&ath);
    if (!finite(phi) || !finite(psi) || !finite(theta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double omega = psi == 0.0 ? 0.0 : phi / psi;
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double est = theta - omega * phi; /* (r_{j+1}, r_{j+1}) = (s,s) - omega (s,t) */
    hist[(j + 1) * hs] = hist_value(est);
    int stop = !finite(est) || (!(flags & ORACLE_NO_STOP_TEST) && est < eps2);
    if (stop) {
      /* group 2 (break branch): x and r update in one pass */
      for (int64_t i = 0; i < n; ++i) {
        double si = AT(s, i);
        AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * si;
        AT(r, i) = si - omega * AT(t, i);
      }
      rw(4, 2);
      out->iters = j + 1;
      out->status = finite(est) ? ST_CONVERGED : ST_NONFINITE;
      return;
    }
    /* group 3: x, r update and rho_{j+1} = (r_{j+1}, r_0) in one pass */
    acc_t arho = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
      double si = AT(s, i);
      AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * si;
      double ri = si - omega * AT(t, i);
      AT(r, i) = ri;
      acc_add(&arho, ri * AT(r0, i));
    }
    rw(5, 2);
    out->iters = j + 1;
    double rho1 = acc_val(&arho);
    if (!finite(rho1)) { out->status = ST_NONFINITE; return; }
    if (rho == 0.0 || omega == 0.0) { out->status = ST_BREAKDOWN; return; }
    double beta = (rho1 / rho) * (alpha / omega);
    if (!finite(beta)) { out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i) + beta * (AT(p, i) - omega * AT(v, i));
    rw(3, 1);
    rho = rho1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- Algorithm 6: Reordered BiCGStab, M^-1 = copy ---------------- */
static void reordered(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit, int flags,
                      int merged, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], z = w[1], vh = w[2], v = w[3], s = w[4], th = w[5], t = w[6], rt = w[7], q = w[8];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) AT(r0, i) = AT(r, i); /* r^_0 = r_0 */
  precond_copy(A, r, z);                                /* z_0 = M^-1 r_0 */
  for (int64_t i = 0; i < n; ++i) AT(vh, i) = AT(z, i); /* v^_0 = z_0 */
  for (int j = 0; j < maxit; ++j) {
    spmv(A, vh, v);                        /* v_j = A v^_j */
    double delta = dot(A, v, r0); rw(2, 0); /* delta_j = (v_j, r_0) */
    precond_copy(A, v, s);                 /* s_j = M^-1 v_j */
    if (!finite(delta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (delta == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double alpha = rho / delta;
    if (!finite(alpha)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(th, i) = AT(z, i) - alpha * AT(s, i); /* t^_j */
    rw(2, 1);
    spmv(A, th, t);                        /* t_j = A t^_j */
    double theta, phi, psi, eta;
    if (merged) {
      /* r~ = r - alpha v with theta = (t,r~), phi = (t,t), psi = (t,r_0), eta = (r~,r~) */
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0}, a4 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double ri = AT(r, i) - alpha * AT(v, i);
        AT(rt, i) = ri;
        double ti = AT(t, i);
        acc_add(&a1, ti * ri);
        acc_add(&a2, ti * ti);
        acc_add(&a3, ti * AT(r0, i));
        acc_add(&a4, ri * ri);
      }
      rw(4, 1);
      theta = acc_val(&a1); phi = acc_val(&a2); psi = acc_val(&a3); eta = acc_val(&a4);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(rt, i) = AT(r, i) - alpha * AT(v, i);
      rw(2, 1);
      theta = dot(A, t, rt); rw(2, 0);
      phi = dot(A, t, t); rw(1, 0);
      psi = dot(A, t, r0); rw(2, 0);
      eta = dot(A, rt, rt); rw(1, 0);
    }
    precond_copy(A, t, q);                 /* q_j = M^-1 t_j */
    if (!finite(theta) || !finite(phi) || !finite(psi) || !finite(eta)) {
      out->iters = j; out->status = ST_NONFINITE; return;
    }
    double omega = phi == 0.0 ? 0.0 : theta / phi;
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(rt, i) - omega * AT(t, i); /* r_{j+1} */
    rw(2, 1);
    double est = eta - omega * theta;
    hist[(j + 1) * hs] = hist_value(est);
    int status = -1;
    if (!finite(est)) status = ST_NONFINITE;
    else if (!(flags & ORACLE_NO_STOP_TEST) && est < eps2) status = ST_CONVERGED;
    double rho1 = 0.0, beta = 0.0;
    if (status < 0) {
      rho1 = -omega * psi; /* rho_{j+1} = -omega_j psi_j */
      if (rho == 0.0 || omega == 0.0) status = ST_BREAKDOWN;
      else {
        beta = (rho1 / rho) * (alpha / omega);
        if (!finite(beta) || !finite(rho1)) status = ST_NONFINITE;
      }
    }
    if (status >= 0) { /* break branch: only x_{j+1} */
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(vh, i) + omega * AT(th, i);
      rw(3, 1);
      out->iters = j + 1;
      out->status = status;
      return;
    }
    if (merged) {
      /* x, z and v^ in one pass */
      for (int64_t i = 0; i < n; ++i) {
        double vhi = AT(vh, i), thi = AT(th, i);
        AT(x, i) = AT(x, i) + alpha * vhi + omega * thi;
        double zi = thi - omega * AT(q, i);
        AT(z, i) = zi;
        AT(vh, i) = zi + beta * (vhi - omega * AT(s, i));
      }
      rw(5, 3);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(vh, i) + omega * AT(th, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(z, i) = AT(th, i) - omega * AT(q, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(vh, i) = AT(z, i) + beta * (AT(vh, i) - omega * AT(s, i));
      rw(3, 1);
    }
    out->iters = j + 1;
    rho = rho1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- Algorithm 4: Pipelined BiCGStab ---------------- */
static void pipelined(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit, int flags,
                      int merged, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], wv = w[1], t = w[2], p = w[3], s = w[4], z = w[5], v = w[6], q = w[7], y = w[8], tmp = w[9];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) AT(r0, i) = AT(r, i);
  spmv(A, r, wv); /* w_0 = A r_0 */
  spmv(A, wv, t); /* t_0 = A w_0 */
  double rw0 = dot(A, r0, wv);
  if (!finite(rw0)) { out->status = ST_NONFINITE; return; }
  if (rw0 == 0.0) { out->status = ST_BREAKDOWN; return; }
  double alpha = rho / rw0; /* alpha_0 = rho_0 / (r_0, w_0) */
  if (!finite(alpha)) { out->status = ST_NONFINITE; return; }
  double beta = 0.0, omega = 0.0; /* beta_{-1} = 0, omega_{-1} = 0 (R7) */
  set_zero(A, p); set_zero(A, s); set_zero(A, z); set_zero(A, v);
  for (int j = 0; j < maxit; ++j) {
    double theta, phi, pi;
    if (merged) {
      /* p, s, z, q, y in one pass with theta = (q,y), phi = (y,y), pi = (q,q) */
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double ri = AT(r, i), wi = AT(wv, i), si = AT(s, i), zi = AT(z, i);
        double pn = ri + beta * (AT(p, i) - omega * si);
        double sn = wi + beta * (si - omega * zi);
        double zn = AT(t, i) + beta * (zi - omega * AT(v, i));
        double qn = ri - alpha * sn;
        double yn = wi - alpha * zn;
        AT(p, i) = pn; AT(s, i) = sn; AT(z, i) = zn; AT(q, i) = qn; AT(y, i) = yn;
        acc_add(&a1, qn * yn);
        acc_add(&a2, yn * yn);
        acc_add(&a3, qn * qn);
      }
      rw(7, 5);
      theta = acc_val(&a1); phi = acc_val(&a2); pi = acc_val(&a3);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i) + beta * (AT(p, i) - omega * AT(s, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(wv, i) + beta * (AT(s, i) - omega * AT(z, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(z, i) = AT(t, i) + beta * (AT(z, i) - omega * AT(v, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(q, i) = AT(r, i) - alpha * AT(s, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(y, i) = AT(wv, i) - alpha * AT(z, i);
      rw(2, 1);
      theta = dot(A, q, y); rw(2, 0);
      phi = dot(A, y, y); rw(1, 0);
      pi = dot(A, q, q); rw(1, 0);
    }
    spmv(A, z, v); /* v_j = A z_j */
    if (!finite(theta) || !finite(phi) || !finite(pi)) { out->iters = j; out->status = ST_NONFINITE; return; }
    omega = phi == 0.0 ? 0.0 : theta / phi;
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (merged) {
      for (int64_t i = 0; i < n; ++i) {
        double qi = AT(q, i);
        AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * qi;
        AT(r, i) = qi - omega * AT(y, i);
      }
      rw(4, 2);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(p, i) + omega * AT(q, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(q, i) - omega * AT(y, i);
      rw(2, 1);
    }
    out->iters = j + 1;
    double est = pi - omega * theta;
    hist[(j + 1) * hs] = hist_value(est);
    if (!finite(est)) { out->status = ST_NONFINITE; return; }
    if (!(flags & ORACLE_NO_STOP_TEST) && est < eps2) { out->status = ST_CONVERGED; return; }
    double rho1, psi, sigma, delta;
    if (merged) {
      /* w_{j+1} = y - omega (t - alpha v) with rho, psi, sigma, delta in one pass */
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0}, a4 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double wn = AT(y, i) - omega * (AT(t, i) - alpha * AT(v, i));
        AT(wv, i) = wn;
        double r0i = AT(r0, i);
        acc_add(&a1, r0i * AT(r, i));
        acc_add(&a2, r0i * AT(z, i));
        acc_add(&a3, r0i * wn);
        acc_add(&a4, r0i * AT(s, i));
      }
      rw(7, 1);
      rho1 = acc_val(&a1); psi = acc_val(&a2); sigma = acc_val(&a3); delta = acc_val(&a4);
    } else {
      /* the 4-vector update takes two BLAS-like calls (Table 2 footnote) */
      for (int64_t i = 0; i < n; ++i) AT(tmp, i) = AT(t, i) - alpha * AT(v, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(wv, i) = AT(y, i) - omega * AT(tmp, i);
      rw(2, 1);
      rho1 = dot(A, r0, r); rw(2, 0);
      psi = dot(A, r0, z); rw(2, 0);
      sigma = dot(A, r0, wv); rw(2, 0);
      delta = dot(A, r0, s); rw(2, 0);
    }
    spmv(A, wv, t); /* t_{j+1} = A w_{j+1} */
    if (!finite(rho1) || !finite(psi) || !finite(sigma) || !finite(delta)) { out->status = ST_NONFINITE; return; }
    if (rho == 0.0 || omega == 0.0) { out->status = ST_BREAKDOWN; return; }
    beta = (alpha / omega) * (rho1 / rho);
    double den = sigma + beta * delta - beta * omega * psi;
    if (!finite(beta) || !finite(den)) { out->status = ST_NONFINITE; return; }
    if (den == 0.0) { out->status = ST_BREAKDOWN; return; }
    alpha = rho1 / den;
    if (!finite(alpha)) { out->status = ST_NONFINITE; return; }
    rho = rho1;
  }
  out->status = ST_MAXIT;
}


/* ---------------- Algorithm 5: preconditioned BiCGStab ---------------- */
static void precond(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit, int flags,
                    int merged, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], p = w[1], v = w[2], s = w[3], t = w[4], ph = w[5], sh = w[6];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) { AT(r0, i) = AT(r, i); AT(p, i) = AT(r, i); }
  for (int j = 0; j < maxit; ++j) {
    precond_copy(A, p, ph);                /* p^_j = M^-1 p_j */
    spmv(A, ph, v);                        /* v_j = A p^_j */
    double delta = dot(A, v, r0); rw(2, 0);
    if (!finite(delta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (delta == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double alpha = rho / delta;
    if (!finite(alpha)) { out->iters = j; out->status = ST_NONFINITE; return; }
    for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(r, i) - alpha * AT(v, i);
    rw(2, 1);
    precond_copy(A, s, sh);                /* s^_j = M^-1 s_j */
    spmv(A, sh, t);                        /* t_j = A s^_j */
    double phi, psi, theta = 0.0;
    if (merged) {
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double ti = AT(t, i), si = AT(s, i);
        acc_add(&a1, ti * si);
        acc_add(&a2, ti * ti);
        acc_add(&a3, si * si);
      }
      rw(2, 0);
      phi = acc_val(&a1); psi = acc_val(&a2); theta = acc_val(&a3);
    } else {
      phi = dot(A, t, s); rw(2, 0);
      psi = dot(A, t, t); rw(1, 0);
    }
    if (!finite(phi) || !finite(psi) || !finite(theta)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double omega = psi == 0.0 ? 0.0 : phi / psi;
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    int status = -1;
    double rho1 = 0.0;
    if (merged) {
      double est = theta - omega * phi;
      hist[(j + 1) * hs] = hist_value(est);
      if (!finite(est)) status = ST_NONFINITE;
      else if (!(flags & ORACLE_NO_STOP_TEST) && est < eps2) status = ST_CONVERGED;
      if (status >= 0) { /* break branch: x and r, two lines */
        for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(sh, i);
        rw(3, 1);
        for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(s, i) - omega * AT(t, i);
        rw(2, 1);
        out->iters = j + 1;
        out->status = status;
        return;
      }
      /* r_{j+1} = s - omega t with rho_{j+1} = (r_{j+1}, r_0) in one pass */
      acc_t ar = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double ri = AT(s, i) - omega * AT(t, i);
        AT(r, i) = ri;
        acc_add(&ar, ri * AT(r0, i));
      }
      rw(3, 1);
      rho1 = acc_val(&ar);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(sh, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(s, i) - omega * AT(t, i);
      rw(2, 1);
      out->iters = j + 1;
      double rr = dot(A, r, r); rw(1, 0);
      hist[(j + 1) * hs] = hist_value(rr);
      if (!finite(rr)) { out->status = ST_NONFINITE; return; }
      if (!(flags & ORACLE_NO_STOP_TEST) && rr < eps2) { out->status = ST_CONVERGED; return; }
      rho1 = dot(A, r, r0); rw(2, 0);
    }
    double beta = 0.0;
    if (!finite(rho1)) status = ST_NONFINITE;
    else if (rho == 0.0 || omega == 0.0) status = ST_BREAKDOWN;
    else {
      beta = (rho1 / rho) * (alpha / omega);
      if (!finite(beta)) status = ST_NONFINITE;
    }
    if (merged) { /* x_{j+1} = x_j + alpha p^ + omega s^ (its own line, after beta) */
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(sh, i);
      rw(3, 1);
      out->iters = j + 1;
    }
    if (status >= 0) { out->status = status; return; }
    for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i) + beta * (AT(p, i) - omega * AT(v, i));
    rw(3, 1);
    rho = rho1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- Algorithm 7: preconditioned Pipelined BiCGStab ---------------- */
static void ppipe(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit, int flags,
                  int merged, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], wv = w[1], t = w[2], ph = w[3], sh = w[4], zh = w[5], qh = w[6], rh = w[7], wh = w[8];
  col_t s = w[9], z = w[10], q = w[11], y = w[12], v = w[13], tmp = w[14];
  double rho, eps2;
  if (setup(A, b, x, r, v, tol, flags, &rho, &eps2, hist, hs, out)) return;
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) AT(r0, i) = AT(r, i);
  precond_copy(A, r, rh);  /* r^_0 = M^-1 r_0 */
  spmv(A, rh, wv);         /* w_0 = A r^_0 */
  precond_copy(A, wv, wh); /* w^_0 = M^-1 w_0 */
  spmv(A, wh, t);          /* t_0 = A w^_0 */
  double rw0 = dot(A, r0, wv);
  if (!finite(rw0)) { out->status = ST_NONFINITE; return; }
  if (rw0 == 0.0) { out->status = ST_BREAKDOWN; return; }
  double alpha = rho / rw0;
  if (!finite(alpha)) { out->status = ST_NONFINITE; return; }
  double beta = 0.0, omega = 0.0;
  set_zero(A, ph); set_zero(A, sh); set_zero(A, zh); set_zero(A, s); set_zero(A, z); set_zero(A, v);
  for (int j = 0; j < maxit; ++j) {
    double theta, phi, pi;
    if (merged) {
      /* p^, s^, q^ in one pass */
      for (int64_t i = 0; i < n; ++i) {
        double shi = AT(sh, i), rhi = AT(rh, i);
        AT(ph, i) = rhi + beta * (AT(ph, i) - omega * shi);
        double sn = AT(wh, i) + beta * (shi - omega * AT(zh, i));
        AT(sh, i) = sn;
        AT(qh, i) = rhi - alpha * sn;
      }
      rw(5, 3);
      /* s, z, q, y with theta = (q,y), phi = (y,y), pi = (q,q) in one pass */
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double wi = AT(wv, i), si = AT(s, i), zi = AT(z, i);
        double sn = wi + beta * (si - omega * zi);
        double zn = AT(t, i) + beta * (zi - omega * AT(v, i));
        double qn = AT(r, i) - alpha * sn;
        double yn = wi - alpha * zn;
        AT(s, i) = sn; AT(z, i) = zn; AT(q, i) = qn; AT(y, i) = yn;
        acc_add(&a1, qn * yn);
        acc_add(&a2, yn * yn);
        acc_add(&a3, qn * qn);
      }
      rw(6, 4);
      theta = acc_val(&a1); phi = acc_val(&a2); pi = acc_val(&a3);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(ph, i) = AT(rh, i) + beta * (AT(ph, i) - omega * AT(sh, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(sh, i) = AT(wh, i) + beta * (AT(sh, i) - omega * AT(zh, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(qh, i) = AT(rh, i) - alpha * AT(sh, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(wv, i) + beta * (AT(s, i) - omega * AT(z, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(z, i) = AT(t, i) + beta * (AT(z, i) - omega * AT(v, i));
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(q, i) = AT(r, i) - alpha * AT(s, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(y, i) = AT(wv, i) - alpha * AT(z, i);
      rw(2, 1);
      theta = dot(A, q, y); rw(2, 0);
      phi = dot(A, y, y); rw(1, 0);
      pi = dot(A, q, q); rw(1, 0);
    }
    precond_copy(A, z, zh); /* z^_j = M^-1 z_j */
    spmv(A, zh, v);         /* v_j = A z^_j */
    if (!finite(theta) || !finite(phi) || !finite(pi)) { out->iters = j; out->status = ST_NONFINITE; return; }
    omega = phi == 0.0 ? 0.0 : theta / phi;
    if (!finite(omega)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double est = pi - omega * theta;
    hist[(j + 1) * hs] = hist_value(est);
    int stop = !finite(est) || (!(flags & ORACLE_NO_STOP_TEST) && est < eps2);
    if (stop) { /* break branch: x and r */
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(qh, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(q, i) - omega * AT(y, i);
      rw(2, 1);
      out->iters = j + 1;
      out->status = finite(est) ? ST_CONVERGED : ST_NONFINITE;
      return;
    }
    double rho1, psi, sigma, delta;
    if (merged) {
      /* x and r^ in one pass */
      for (int64_t i = 0; i < n; ++i) {
        double qhi = AT(qh, i);
        AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * qhi;
        AT(rh, i) = qhi - omega * (AT(wh, i) - alpha * AT(zh, i));
      }
      rw(5, 2);
      /* r, w and rho, psi, sigma, delta in one pass */
      acc_t a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0}, a4 = {0, 0};
      for (int64_t i = 0; i < n; ++i) {
        double yi = AT(y, i);
        double rn = AT(q, i) - omega * yi;
        double wn = yi - omega * (AT(t, i) - alpha * AT(v, i));
        AT(r, i) = rn; AT(wv, i) = wn;
        double r0i = AT(r0, i);
        acc_add(&a1, r0i * rn);
        acc_add(&a2, r0i * AT(z, i));
        acc_add(&a3, r0i * wn);
        acc_add(&a4, r0i * AT(s, i));
      }
      rw(7, 2);
      rho1 = acc_val(&a1); psi = acc_val(&a2); sigma = acc_val(&a3); delta = acc_val(&a4);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + alpha * AT(ph, i) + omega * AT(qh, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(tmp, i) = AT(wh, i) - alpha * AT(zh, i);  /* 4-vector op: 2 calls */
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(rh, i) = AT(qh, i) - omega * AT(tmp, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(q, i) - omega * AT(y, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(tmp, i) = AT(t, i) - alpha * AT(v, i);    /* 4-vector op: 2 calls */
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(wv, i) = AT(y, i) - omega * AT(tmp, i);
      rw(2, 1);
      rho1 = dot(A, r0, r); rw(2, 0);
      psi = dot(A, r0, z); rw(2, 0);
      sigma = dot(A, r0, wv); rw(2, 0);
      delta = dot(A, r0, s); rw(2, 0);
    }
    out->iters = j + 1;
    precond_copy(A, wv, wh); /* w^_{j+1} = M^-1 w_{j+1} */
    spmv(A, wh, t);          /* t_{j+1} = A w^_{j+1} */
    if (!finite(rho1) || !finite(psi) || !finite(sigma) || !finite(delta)) { out->status = ST_NONFINITE; return; }
    if (rho == 0.0 || omega == 0.0) { out->status = ST_BREAKDOWN; return; }
    beta = (alpha / omega) * (rho1 / rho);
    double den = sigma + beta * delta - beta * omega * psi;
    if (!finite(beta) || !finite(den)) { out->status = ST_NONFINITE; return; }
    if (den == 0.0) { out->status = ST_BREAKDOWN; return; }
    alpha = rho1 / den;
    if (!finite(alpha)) { out->status = ST_NONFINITE; return; }
    rho = rho1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- Algorithm 3: Improved BiCGStab ---------------- */
static void improved(const csr_t *A, col_t b, col_t x, col_t r, col_t *w, double tol, int maxit, int flags,
                     int merged, double *hist, int64_t hs, res_t *out) {
  col_t r0 = w[0], u = w[1], f0 = w[2], q = w[3], v = w[4], z = w[5], s = w[6], t = w[7];
  double phi, eps2;
  if (setup(A, b, x, r, v, tol, flags, &phi, &eps2, hist, hs, out)) return;  /* phi_0 = (r_0, r_0) */
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) AT(r0, i) = AT(r, i);
  spmv(A, r, u);    /* u_0 = A r_0 */
  spmv_t(A, r, f0); /* f_0 = A^T r_0 */
  set_zero(A, q); set_zero(A, v); set_zero(A, z);
  double sigma_prev = 0.0, pi = 0.0, tau = 0.0;
  double sigma = dot(A, r0, u);
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  for (int j = 0; j < maxit; ++j) {
    /* scalar recurrences of the iteration (divisions guarded as in R5) */
    double rho1 = phi - omega * sigma_prev + omega * alpha * pi;
    if (!finite(rho1) || !finite(sigma)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (rho == 0.0 || omega == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double delta1 = (rho1 / rho) * alpha;
    double beta1 = delta1 / omega;
    double tau1 = sigma + beta1 * tau - delta1 * pi;
    if (!finite(delta1) || !finite(beta1) || !finite(tau1)) { out->iters = j; out->status = ST_NONFINITE; return; }
    if (tau1 == 0.0) { out->iters = j; out->status = ST_BREAKDOWN; return; }
    double alpha1 = rho1 / tau1;
    if (!finite(alpha1)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double cz = beta1 * (alpha1 / alpha), cv = alpha1 * delta1;
    if (merged) {
      /* z, v, s in one pass */
      for (int64_t i = 0; i < n; ++i) {
        double ri = AT(r, i), vi = AT(v, i);
        AT(z, i) = alpha1 * ri + cz * AT(z, i) - cv * vi;
        double vn = AT(u, i) + beta1 * vi - delta1 * AT(q, i);
        AT(v, i) = vn;
        AT(s, i) = ri - alpha1 * vn;
      }
      rw(5, 3);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(z, i) = alpha1 * AT(r, i) + cz * AT(z, i) - cv * AT(v, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(v, i) = AT(u, i) + beta1 * AT(v, i) - delta1 * AT(q, i);
      rw(3, 1);
      for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(r, i) - alpha1 * AT(v, i);
      rw(2, 1);
    }
    spmv(A, v, q); /* q_{j+1} = A v_{j+1} */
    double phi1, pi1, gam, eta, theta, kappa, nu;
    if (merged) {
      /* t with the seven dot products in one pass */
      acc_t a[7] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
      for (int64_t i = 0; i < n; ++i) {
        double qi = AT(q, i), si = AT(s, i), r0i = AT(r0, i), fi = AT(f0, i);
        double ti = AT(u, i) - alpha1 * qi;
        AT(t, i) = ti;
        acc_add(&a[0], r0i * si);
        acc_add(&a[1], r0i * qi);
        acc_add(&a[2], fi * si);
        acc_add(&a[3], fi * ti);
        acc_add(&a[4], si * ti);
        acc_add(&a[5], ti * ti);
        acc_add(&a[6], si * si);
      }
      rw(5, 1);
      phi1 = acc_val(&a[0]); pi1 = acc_val(&a[1]); gam = acc_val(&a[2]); eta = acc_val(&a[3]);
      theta = acc_val(&a[4]); kappa = acc_val(&a[5]); nu = acc_val(&a[6]);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(t, i) = AT(u, i) - alpha1 * AT(q, i);
      rw(2, 1);
      phi1 = dot(A, r0, s); rw(2, 0);
      pi1 = dot(A, r0, q); rw(2, 0);
      gam = dot(A, f0, s); rw(2, 0);
      eta = dot(A, f0, t); rw(2, 0);
      theta = dot(A, s, t); rw(2, 0);
      kappa = dot(A, t, t); rw(1, 0);
      nu = dot(A, s, s); rw(1, 0);
    }
    if (!finite(phi1) || !finite(pi1) || !finite(gam) || !finite(eta) || !finite(theta) || !finite(kappa) ||
        !finite(nu)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double omega1 = kappa == 0.0 ? 0.0 : theta / kappa;
    if (!finite(omega1)) { out->iters = j; out->status = ST_NONFINITE; return; }
    double sigma1 = gam - omega1 * eta;
    if (merged) {
      for (int64_t i = 0; i < n; ++i) {
        double si = AT(s, i);
        AT(r, i) = si - omega1 * AT(t, i);
        AT(x, i) = AT(x, i) + AT(z, i) + omega1 * si;
      }
      rw(4, 2);
    } else {
      for (int64_t i = 0; i < n; ++i) AT(r, i) = AT(s, i) - omega1 * AT(t, i);
      rw(2, 1);
      for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + AT(z, i) + omega1 * AT(s, i);
      rw(3, 1);
    }
    out->iters = j + 1;
    double est = nu - omega1 * theta;
    hist[(j + 1) * hs] = hist_value(est);
    if (!finite(est)) { out->status = ST_NONFINITE; return; }
    if (!(flags & ORACLE_NO_STOP_TEST) && est < eps2) { out->status = ST_CONVERGED; return; }
    spmv(A, r, u); /* u_{j+1} = A r_{j+1} */
    sigma_prev = sigma; sigma = sigma1; rho = rho1; alpha = alpha1; omega = omega1; phi = phi1; pi = pi1;
    tau = tau1;
  }
  out->status = ST_MAXIT;
}

/* ---------------- exported entry points ---------------- */

/* Number of N-vectors of scratch per column a variant needs. */
static int n_work(int variant) {
  switch (variant) {
    case ORACLE_CLASSICAL_BASIC:
    case ORACLE_CLASSICAL_MERGED: return 5;
    case ORACLE_REORDERED_BASIC:
    case ORACLE_REORDERED_MERGED: return 9;
    case ORACLE_PIPELINED_BASIC:
    case ORACLE_PIPELINED_MERGED: return 10;
    case ORACLE_PRECOND_BASIC:
    case ORACLE_PRECOND_MERGED: return 7;
    case ORACLE_PPIPE_BASIC:
    case ORACLE_PPIPE_MERGED: return 15;
    case ORACLE_IMPROVED_BASIC:
    case ORACLE_IMPROVED_MERGED: return 8;
    default: return -1;
  }
}

/* y = A x for an interleaved N x k block (SpMV per column, Eq. for Sigma_mul's operation). */
int oracle_spmm(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals, int32_t k,
                const double *X, double *Y) {
  if (n < 0 || k < 1) return -1;
  csr_t A = {n, rowptr, colidx, vals};
  for (int32_t c = 0; c < k; ++c) {
    col_t x = {(double *)X + c, k}, y = {Y + c, k};
    spmv(&A, x, y);
  }
  return 0;
}

/* Solve A X = B column by column.
 *   B, X0 (nullable = zero), X, R (nullable): N x k interleaved.
 *   hist (nullable): (maxit+1) x k, entry (j, c) = estimate of ||r_j|| of column c,
 *     NaN where column c formed no iterate j.
 *   true_relres (nullable): ||b_c - A x_c|| / ||b_c|| after the solve (0 when b_c = 0).
 *   traffic (nullable, 4 int64): vector reads, writes, identity copies, SpMVs summed over all
 *     columns and iterations (set-up included).
 * Returns 0, or -1 on a bad argument. */
int oracle_solve(int variant, int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals,
                 int32_t k, const double *B, const double *X0, double tol, int32_t maxit, int32_t flags,
                 double *X, double *R, int32_t *iters, int32_t *status, double *hist, double *true_relres,
                 int64_t *traffic) {
  int nw = n_work(variant);
  if (nw < 0 || n < 0 || k < 1 || maxit < 0 || !(tol >= 0.0)) return -1;
  csr_t A = {n, rowptr, colidx, vals};
  memset(&g_tr, 0, sizeof(g_tr));
  double *work = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(nw + 2));
  double *hbuf = (double *)malloc(sizeof(double) * (size_t)(maxit + 1));
  double *invd = (flags & ORACLE_JACOBI) ? (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)) : NULL;
  if (!work || !hbuf || ((flags & ORACLE_JACOBI) && !invd)) { free(work); free(hbuf); free(invd); return -2; }
  if (invd) { /* M = diag(A); a zero or missing diagonal entry counts as 1 */
    for (int64_t i = 0; i < n; ++i) {
      double d = 0.0;
      for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) d += vals[e];
      invd[i] = d == 0.0 ? 1.0 : 1.0 / d;
    }
  }
  g_invdiag = invd;
  for (int32_t c = 0; c < k; ++c) {
    col_t w[16];
    for (int q = 0; q < nw; ++q) w[q] = (col_t){work + (size_t)q * n, 1};
    col_t rloc = {work + (size_t)nw * n, 1};
    col_t b = {(double *)B + c, k};
    col_t x = {X + c, k};
    for (int64_t i = 0; i < n; ++i) AT(x, i) = X0 ? X0[i * k + c] : 0.0;
    for (int32_t j = 0; j <= maxit; ++j) hbuf[j] = NAN;
    res_t res = {0, ST_MAXIT};
    switch (variant) {
      case ORACLE_CLASSICAL_BASIC: classical_basic(&A, b, x, rloc, w, tol, maxit, flags, hbuf, 1, &res); break;
      case ORACLE_CLASSICAL_MERGED: classical_merged(&A, b, x, rloc, w, tol, maxit, flags, hbuf, 1, &res); break;
      case ORACLE_REORDERED_BASIC: reordered(&A, b, x, rloc, w, tol, maxit, flags, 0, hbuf, 1, &res); break;
      case ORACLE_REORDERED_MERGED: reordered(&A, b, x, rloc, w, tol, maxit, flags, 1, hbuf, 1, &res); break;
      case ORACLE_PIPELINED_BASIC: pipelined(&A, b, x, rloc, w, tol, maxit, flags, 0, hbuf, 1, &res); break;
      case ORACLE_PIPELINED_MERGED: pipelined(&A, b, x, rloc, w, tol, maxit, flags, 1, hbuf, 1, &res); break;
      case ORACLE_PRECOND_BASIC: precond(&A, b, x, rloc, w, tol, maxit, flags, 0, hbuf, 1, &res); break;
      case ORACLE_PRECOND_MERGED: precond(&A, b, x, rloc, w, tol, maxit, flags, 1, hbuf, 1, &res); break;
      case ORACLE_PPIPE_BASIC: ppipe(&A, b, x, rloc, w, tol, maxit, flags, 0, hbuf, 1, &res); break;
      case ORACLE_PPIPE_MERGED: ppipe(&A, b, x, rloc, w, tol, maxit, flags, 1, hbuf, 1, &res); break;
      case ORACLE_IMPROVED_BASIC: improved(&A, b, x, rloc, w, tol, maxit, flags, 0, hbuf, 1, &res); break;
      case ORACLE_IMPROVED_MERGED: improved(&A, b, x, rloc, w, tol, maxit, flags, 1, hbuf, 1, &res); break;
    }
    if (iters) iters[c] = res.iters;
    if (status) status[c] = res.status;
    if (hist)
      for (int32_t j = 0; j <= maxit; ++j) hist[(int64_t)j * k + c] = hbuf[j];
    if (R)
      for (int64_t i = 0; i < n; ++i) R[i * k + c] = AT(rloc, i);
    if (true_relres) {
      col_t ax = {work + (size_t)(nw + 1) * n, 1};
      spmv(&A, x, ax);
      for (int64_t i = 0; i < n; ++i) AT(ax, i) = AT(b, i) - AT(ax, i);
      double bn2 = dot(&A, b, b), rn2 = dot(&A, ax, ax);
      true_relres[c] = bn2 == 0.0 ? 0.0 : sqrt(rn2) / sqrt(bn2);
    }
  }
  if (traffic) {
    traffic[0] = g_tr.reads; traffic[1] = g_tr.writes; traffic[2] = g_tr.copies; traffic[3] = g_tr.spmv;
  }
  g_invdiag = NULL;
  free(work);
  free(hbuf);
  free(invd);
  return 0;
}

/* ---------------- mixed precision: FP64 refinement around FP32 inner solves ----------------
 *
 * Not in the paper (its solvers run in FP64).  The inner solver is Algorithm 2 with FP32
 * vectors and FP32 matrix values: every vector update is FP32 arithmetic with the scalars
 * rounded to FP32; the dot products are formed in FP64 (a product of two floats is exact in
 * double) with the compensated sum of dot(); the scalar recurrences and the stop rules
 * (R1-R6) are FP64, as in classical_merged().  The outer loop is iterative refinement in
 * FP64: r = b - A x, stop when (r,r) < eps^2 (R1) or after max_outer passes, else solve
 * A d = fl32(r) from d = 0 to the relative tolerance inner_tol and add d to x. */

typedef struct {
  float *p;
  int64_t s;
} fcol_t;

static void spmv32(const csr_t *A, const float *vals32, fcol_t x, fcol_t y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < A->n; ++i) {
    float acc = 0.0f;
    for (int32_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) acc += vals32[e] * AT(x, A->colidx[e]);
    AT(y, i) = acc;
  }
}

static double dot32(const csr_t *A, fcol_t x, fcol_t y) {
  double sum = 0.0, comp = 0.0;
  for (int64_t i = 0; i < A->n; ++i) {
    double p = (double)AT(x, i) * (double)AT(y, i); /* exact */
    double t = sum + p;
    if (fabs(sum) >= fabs(p))
      comp += (sum - t) + p;
    else
      comp += (p - t) + sum;
    sum = t;
  }
  return sum + comp;
}

/* Algorithm 2 in FP32 storage for A d = b32, d_0 = 0.  Returns the iterations formed. */
static int inner_merged32(const csr_t *A, const float *vals32, fcol_t b, fcol_t d, fcol_t *w, double tol,
                          int maxit) {
  fcol_t r = w[0], r0 = w[1], p = w[2], v = w[3], s = w[4], t = w[5];
  const int64_t n = A->n;
  for (int64_t i = 0; i < n; ++i) {
    AT(d, i) = 0.0f;
    AT(r, i) = AT(b, i);
    AT(r0, i) = AT(b, i);
    AT(p, i) = AT(b, i);
  }
  double bn2 = dot32(A, b, b), rho = dot32(A, r, r);
  double eps2 = tol * tol * bn2;
  if (bn2 == 0.0 || !finite(rho) || rho < eps2) return 0;
  int iters = 0;
  for (int j = 0; j < maxit; ++j) {
    spmv32(A, vals32, p, v);
    double delta = dot32(A, v, r0);
    if (!finite(delta) || delta == 0.0) return iters;
    double alpha = rho / delta;
    if (!finite(alpha)) return iters;
    float af = (float)alpha;
    for (int64_t i = 0; i < n; ++i) AT(s, i) = AT(r, i) - af * AT(v, i);
    spmv32(A, vals32, s, t);
    double phi = dot32(A, t, s), psi = dot32(A, t, t), theta = dot32(A, s, s);
    if (!finite(phi) || !finite(psi) || !finite(theta)) return iters;
    double omega = psi == 0.0 ? 0.0 : phi / psi;
    if (!finite(omega)) return iters;
    float of = (float)omega;
    for (int64_t i = 0; i < n; ++i) {
      float si = AT(s, i);
      AT(d, i) = AT(d, i) + af * AT(p, i) + of * si;
      AT(r, i) = si - of * AT(t, i);
    }
    iters = j + 1;
    double est = theta - omega * phi;
    if (!finite(est) || est < eps2) return iters;
    double rho1 = dot32(A, r, r0);
    if (!finite(rho1) || rho == 0.0 || omega == 0.0) return iters;
    double beta = (rho1 / rho) * (alpha / omega);
    if (!finite(beta)) return iters;
    float bf = (float)beta;
    for (int64_t i = 0; i < n; ++i) AT(p, i) = AT(r, i) + bf * (AT(p, i) - of * AT(v, i));
    rho = rho1;
  }
  return iters;
}

/* Mixed-precision solve, column by column.  hist (nullable): (max_outer+1) x k, entry (j, c) =
 * ||b - A x|| before pass j, NaN after the column stopped. */
int oracle_solve_mixed(int64_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals, int32_t k,
                       const double *B, const double *X0, double tol, int32_t max_outer, double inner_tol,
                       int32_t max_inner, double *X, int32_t *outer_iters, int32_t *inner_iters, int32_t *status,
                       double *hist, double *true_relres) {
  if (n < 1 || k < 1 || max_outer < 0 || max_inner < 1 || !(tol >= 0.0) || !(inner_tol > 0.0)) return -1;
  csr_t A = {n, rowptr, colidx, vals};
  int64_t nnz = rowptr[n];
  float *vals32 = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  double *ax = (double *)malloc(sizeof(double) * (size_t)n);
  float *fw = (float *)malloc(sizeof(float) * (size_t)n * 8);
  if (!vals32 || !r || !ax || !fw) { free(vals32); free(r); free(ax); free(fw); return -2; }
  for (int64_t e = 0; e < nnz; ++e) vals32[e] = (float)vals[e];
  for (int32_t c = 0; c < k; ++c) {
    col_t b = {(double *)B + c, k}, x = {X + c, k};
    col_t rc = {r, 1}, axc = {ax, 1};
    fcol_t b32 = {fw, 1}, d32 = {fw + n, 1};
    fcol_t w[6];
    for (int q = 0; q < 6; ++q) w[q] = (fcol_t){fw + (size_t)(q + 2) * n, 1};
    for (int64_t i = 0; i < n; ++i) AT(x, i) = X0 ? X0[i * k + c] : 0.0;
    if (hist)
      for (int32_t j = 0; j <= max_outer; ++j) hist[(int64_t)j * k + c] = NAN;
    double bn2 = dot(&A, b, b), eps2 = tol * tol * bn2;
    int st = ST_MAXIT, outer = 0, inner = 0;
    double rr = 0.0;
    if (bn2 == 0.0) {
      set_zero(&A, x);
      st = ST_CONVERGED;
    } else if (!finite(bn2)) {
      st = ST_NONFINITE;
    } else {
      for (int j = 0;; ++j) {
        spmv(&A, x, axc);
        for (int64_t i = 0; i < n; ++i) AT(rc, i) = AT(b, i) - AT(axc, i);
        rr = dot(&A, rc, rc);
        if (hist) hist[(int64_t)j * k + c] = hist_value(rr);
        if (!finite(rr)) { st = ST_NONFINITE; break; }
        if (rr < eps2) { st = ST_CONVERGED; break; }
        if (j >= max_outer) { st = ST_MAXIT; break; }
        outer = j + 1;
        for (int64_t i = 0; i < n; ++i) AT(b32, i) = (float)AT(rc, i);
        inner += inner_merged32(&A, vals32, b32, d32, w, inner_tol, max_inner);
        for (int64_t i = 0; i < n; ++i) AT(x, i) = AT(x, i) + (double)AT(d32, i);
      }
    }
    outer_iters[c] = outer;
    inner_iters[c] = inner;
    status[c] = st;
    if (true_relres) true_relres[c] = bn2 == 0.0 ? 0.0 : sqrt(rr) / sqrt(bn2);
  }
  free(vals32);
  free(r);
  free(ax);
  free(fw);
  return 0;
}

/* Threads the OpenMP runtime will use for the parallel loops (1 without OpenMP). */
/* Thread count for the following calls (timing the oracle on one core and on all of them). */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
void oracle_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
}
#else
int oracle_threads(void) { return 1; }
void oracle_set_threads(int n) { (void)n; }
#endif
