/*
 * CPU ORACLE -- test infrastructure only.  Plain, slow, obviously correct FP64
 * restatement of the block staircase iteration (Besozzi, Della Bartola,
 * Gemignani, arXiv 2302.07551).  Only tests, the package smoke check and the
 * benchmark's CPU-baseline leg may call it; the GPU library never does, and
 * this file shares no code with it.
 *
 * Problem (Eq. 1): Q^T pi = 0, pi >= 0, e^T pi = 1 for an irreducible generator
 * Q.  The blocks Q_{i,j} of the paper are the blocks of Q^T (Sect. 2); here
 * T = Q^T, built from generator blocks of Q given per level l = 0..L-1:
 *     dn[l] = Q_{l,l-1},  loc[l] = Q_{l,l},  up[l] = Q_{l,l+1}
 * so that  T_lo[l] = T_{l,l-1} = up[l-1]^T,  T_dd[l] = loc[l]^T,
 *          T_up[l] = T_{l,l+1} = dn[l+1]^T   (row-major m x m each).
 *
 * Splittings T = M - N (Sect. 2, regular splittings) and one step of the
 * scheme of Eq. (2): solve M z = N x, then z <- z / e^T z.
 *   STAIR1: M = stair matrix of type 1; Algorithm 2 steps 1-3.
 *   STAIR2: M = stair matrix of type 2 (parity of the block rows swapped).
 *   BGS   : M = block lower triangle of T (block Gauss-Seidel).
 *   BJ    : M = block diagonal of T (block Jacobi).
 * Paper indices are 1-based: block row i (1-based) is level l = i-1 here.
 *
 * Compile: gcc -O2 -ffp-contract=off [-fopenmp].  Every level inside one
 * parallel step of Algorithm 2 is computed independently with a fixed order,
 * so the OpenMP build gives bit-identical results to the serial one.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_STAIR1 = 1, OR_STAIR2 = 2, OR_BGS = 3, OR_BJ = 4 };

#define BLK(P, l, m) ((P) + (size_t)(l) * (size_t)(m) * (size_t)(m))

/* T = Q^T from generator blocks (Sect. 2 block partition of Q^T). */
void or_build_T(int64_t L, int m, const double* dn, const double* loc, const double* up,
                double* Tlo, double* Tdd, double* Tup) {
  for (int64_t l = 0; l < L; ++l)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        BLK(Tdd, l, m)[i * m + j] = BLK(loc, l, m)[j * m + i];
        BLK(Tlo, l, m)[i * m + j] = (l > 0) ? BLK(up, l - 1, m)[j * m + i] : 0.0;
        BLK(Tup, l, m)[i * m + j] = (l < L - 1) ? BLK(dn, l + 1, m)[j * m + i] : 0.0;
      }
}

/*
 * Textbook Gaussian elimination with partial pivoting, in place, row-major:
 * P A = L U with unit lower L below the diagonal and U on and above it.
 * piv[k] = row exchanged with row k at step k.  Returns the number of row
 * exchanges, or -1 if a pivot is zero or not finite.
 */
int or_lu(int m, double* A, int* piv) {
  int swaps = 0;
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(A[k * m + k]);
    for (int i = k + 1; i < m; ++i)
      if (fabs(A[i * m + k]) > best) { best = fabs(A[i * m + k]); p = i; }
    piv[k] = p;
    if (p != k) {
      ++swaps;
      for (int j = 0; j < m; ++j) { double t = A[k * m + j]; A[k * m + j] = A[p * m + j]; A[p * m + j] = t; }
    }
    double d = A[k * m + k];
    if (!(d != 0.0) || !isfinite(d)) return -1;
    for (int i = k + 1; i < m; ++i) {
      double lik = A[i * m + k] / d;
      A[i * m + k] = lik;
      for (int j = k + 1; j < m; ++j) A[i * m + j] -= lik * A[k * m + j];
    }
  }
  return swaps;
}

/* Solve A x = b in place from or_lu's factors: b <- U^{-1} L^{-1} P b. */
void or_lu_solve(int m, const double* LU, const int* piv, double* b) {
  for (int k = 0; k < m; ++k)
    if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[i * m + j] * b[j];
    b[i] = s;
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < m; ++j) s -= LU[i * m + j] * b[j];
    b[i] = s / LU[i * m + i];
  }
}

/* Factor every diagonal block T_dd[l]; returns total row exchanges or -1. */
int64_t or_factor(int64_t L, int m, const double* Tdd, double* LU, int* piv) {
  int64_t swaps = 0;
  int bad = 0;
  for (int64_t l = 0; l < L; ++l) {
    memcpy(BLK(LU, l, m), BLK(Tdd, l, m), sizeof(double) * (size_t)m * m);
    int s = or_lu(m, BLK(LU, l, m), piv + (size_t)l * m);
    if (s < 0) bad = 1; else swaps += s;
  }
  return bad ? -1 : swaps;
}

/* y <- y + B v  (m x m block, natural index order). */
static void gemv_acc(int m, const double* B, const double* v, double* y) {
  for (int i = 0; i < m; ++i) {
    double s = y[i];
    for (int j = 0; j < m; ++j) s += B[i * m + j] * v[j];
    y[i] = s;
  }
}

/*
 * Is block row l (0-based) a "diagonal-only" row of the stair matrix?
 * Type 1 (M_1): paper rows 1, 3, 5, ... (1-based odd) hold only Q_{i,i};
 * rows 2, 4, ... hold Q_{i,i-1}, Q_{i,i}, Q_{i,i+1}.  Type 2 swaps the roles.
 * Row l (0-based) is paper row l+1, so it is 1-based odd iff l is even.
 */
static int stair_diag_only(int type, int64_t l) {
  int one_based_odd = ((l + 1) % 2) == 1;
  return type == 1 ? one_based_odd : !one_based_odd;
}

/*
 * One unnormalised step z = M^{-1} N x of the chosen splitting.
 * STAIR types follow Algorithm 2 (with J_i the index set of the paper, and
 * step 1 summing over k outside J_i and k != i, since Q_{i,i} belongs to M):
 *   step 1 (all block rows i):  z_i <- - sum_{k not in J_i, k != i} Q_{i,k} x_k
 *   step 2 (diagonal-only rows): z_i <- Q_{i,i}^{-1} z_i
 *   step 3 (coupled rows):       z_i <- Q_{i,i}^{-1} (z_i - sum_{k in J_i} Q_{i,k} z_k)
 * With T block tridiagonal, step 1 leaves z_i = 0 on coupled rows.
 * Returns 0, or -1 on an unknown method.
 */
int or_sweep(int64_t L, int m, int method, const double* Tlo, const double* Tup,
             const double* LU, const int* piv, const double* x, double* z) {
  const size_t N = (size_t)L * m;
  if (method == OR_STAIR1 || method == OR_STAIR2) {
    const int type = method == OR_STAIR1 ? 1 : 2;
    /* step 1 */
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l) {
      double* zl = z + (size_t)l * m;
      for (int i = 0; i < m; ++i) zl[i] = 0.0;
      if (stair_diag_only(type, l)) {
        /* J = {l}: every off-diagonal block of the row is off the staircase */
        double* acc = (double*)calloc((size_t)m, sizeof(double));
        if (l > 0) gemv_acc(m, BLK(Tlo, l, m), x + (size_t)(l - 1) * m, acc);
        if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), x + (size_t)(l + 1) * m, acc);
        for (int i = 0; i < m; ++i) zl[i] = -acc[i];
        free(acc);
      }
    }
    /* step 2 */
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l)
      if (stair_diag_only(type, l))
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, z + (size_t)l * m);
    /* step 3 */
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l)
      if (!stair_diag_only(type, l)) {
        double* zl = z + (size_t)l * m;
        double* acc = (double*)calloc((size_t)m, sizeof(double));
        if (l > 0) gemv_acc(m, BLK(Tlo, l, m), z + (size_t)(l - 1) * m, acc);
        if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), z + (size_t)(l + 1) * m, acc);
        for (int i = 0; i < m; ++i) zl[i] = zl[i] - acc[i];
        free(acc);
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, zl);
      }
    return 0;
  }
  if (method == OR_BGS) {
    /* M = block lower triangle: level by level, newest values below. */
    for (int64_t l = 0; l < L; ++l) {
      double* zl = z + (size_t)l * m;
      double* acc = (double*)calloc((size_t)m, sizeof(double));
      if (l > 0) gemv_acc(m, BLK(Tlo, l, m), z + (size_t)(l - 1) * m, acc);
      if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), x + (size_t)(l + 1) * m, acc);
      for (int i = 0; i < m; ++i) zl[i] = -acc[i];
      free(acc);
      or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, zl);
    }
    return 0;
  }
  if (method == OR_BJ) {
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l) {
      double* zl = z + (size_t)l * m;
      double* acc = (double*)calloc((size_t)m, sizeof(double));
      if (l > 0) gemv_acc(m, BLK(Tlo, l, m), x + (size_t)(l - 1) * m, acc);
      if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), x + (size_t)(l + 1) * m, acc);
      for (int i = 0; i < m; ++i) zl[i] = -acc[i];
      free(acc);
      or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, zl);
    }
    return 0;
  }
  (void)N;
  return -1;
}

/*
 * One step of the same splitting with a right-hand side:  z = M^{-1} (N x + b).
 * This is the correction equation of iterative refinement: with r = T pi and
 * b = -r, the fixed point d of z = M^{-1}(N d - r) solves T d = -r (Eq. (2)
 * applied to T d = -r instead of T pi = 0).  Stair types follow the steps of
 * Algorithm 2 with b added to step 1; BGS and BJ as in or_sweep.  b = 0 gives
 * or_sweep.  Returns 0, or -1 on an unknown method.
 */
int or_sweep_rhs(int64_t L, int m, int method, const double* Tlo, const double* Tup,
                 const double* LU, const int* piv, const double* x, const double* b, double* z) {
  if (or_sweep(L, m, method, Tlo, Tup, LU, piv, x, z) != 0) return -1;
  /* z currently holds M^{-1} N x; add M^{-1} b by solving M w = b the same way */
  const size_t N = (size_t)L * m;
  double* w = (double*)malloc(sizeof(double) * N);
  if (method == OR_STAIR1 || method == OR_STAIR2) {
    const int type = method == OR_STAIR1 ? 1 : 2;
    for (int64_t l = 0; l < L; ++l)          /* diagonal-only rows: w_l = Q_ll^{-1} b_l */
      if (stair_diag_only(type, l)) {
        memcpy(w + (size_t)l * m, b + (size_t)l * m, sizeof(double) * (size_t)m);
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, w + (size_t)l * m);
      }
    for (int64_t l = 0; l < L; ++l)          /* coupled rows: w_l = Q_ll^{-1}(b_l - Q_{l,l-1} w_{l-1} - Q_{l,l+1} w_{l+1}) */
      if (!stair_diag_only(type, l)) {
        double* acc = (double*)calloc((size_t)m, sizeof(double));
        if (l > 0) gemv_acc(m, BLK(Tlo, l, m), w + (size_t)(l - 1) * m, acc);
        if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), w + (size_t)(l + 1) * m, acc);
        for (int i = 0; i < m; ++i) w[(size_t)l * m + i] = b[(size_t)l * m + i] - acc[i];
        free(acc);
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, w + (size_t)l * m);
      }
  } else if (method == OR_BGS) {
    for (int64_t l = 0; l < L; ++l) {
      double* acc = (double*)calloc((size_t)m, sizeof(double));
      if (l > 0) gemv_acc(m, BLK(Tlo, l, m), w + (size_t)(l - 1) * m, acc);
      for (int i = 0; i < m; ++i) w[(size_t)l * m + i] = b[(size_t)l * m + i] - acc[i];
      free(acc);
      or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, w + (size_t)l * m);
    }
  } else {
    for (int64_t l = 0; l < L; ++l) {
      memcpy(w + (size_t)l * m, b + (size_t)l * m, sizeof(double) * (size_t)m);
      or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, w + (size_t)l * m);
    }
  }
  for (size_t i = 0; i < N; ++i) z[i] += w[i];
  free(w);
  return 0;
}

/* The residual vector r = T x (Eq. (1)), from the blocks of T = Q^T. */
void or_residual_vec(int64_t L, int m, const double* Tlo, const double* Tdd, const double* Tup,
                     const double* x, double* r) {
  for (int64_t l = 0; l < L; ++l) {
    double* acc = r + (size_t)l * m;
    for (int i = 0; i < m; ++i) acc[i] = 0.0;
    if (l > 0) gemv_acc(m, BLK(Tlo, l, m), x + (size_t)(l - 1) * m, acc);
    gemv_acc(m, BLK(Tdd, l, m), x + (size_t)l * m, acc);
    if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), x + (size_t)(l + 1) * m, acc);
  }
}

/* ||T x||_1 computed directly from the blocks of T = Q^T. */
double or_residual(int64_t L, int m, const double* Tlo, const double* Tdd, const double* Tup,
                   const double* x) {
  double r = 0.0;
  double* acc = (double*)malloc(sizeof(double) * (size_t)m);
  for (int64_t l = 0; l < L; ++l) {
    for (int i = 0; i < m; ++i) acc[i] = 0.0;
    if (l > 0) gemv_acc(m, BLK(Tlo, l, m), x + (size_t)(l - 1) * m, acc);
    gemv_acc(m, BLK(Tdd, l, m), x + (size_t)l * m, acc);
    if (l < L - 1) gemv_acc(m, BLK(Tup, l, m), x + (size_t)(l + 1) * m, acc);
    for (int i = 0; i < m; ++i) r += fabs(acc[i]);
  }
  free(acc);
  return r;
}

/*
 * The normalised iteration of Eq. (2) as in Algorithm 2:
 *   z <- M^{-1} N x;  z <- z / e^T z;  err <- ||z - x||_1;  x <- z.
 * Starts from x (x0 supplied by the caller, e.g. uniform 1/N).  Stops after
 * the first sweep k with  resid_k <= tol  (if tol > 0; resid_k = ||T x_k||_1,
 * evaluated every `check_every` sweeps and at maxit),  or  err_k <= eps  (if
 * eps > 0),  or  k >= maxit.  err_hist[k-1] receives err_k (may be NULL).
 * Returns the number of sweeps done, or -1 on breakdown (e^T z <= 0 or not
 * finite), -2 on a bad method.  out[0] = last resid (NaN if never
 * evaluated), out[1] = last err.
 */
int64_t or_solve(int64_t L, int m, int method, const double* Tlo, const double* Tdd,
                 const double* Tup, const double* LU, const int* piv, double* x,
                 double tol, double eps, int64_t maxit, int64_t check_every,
                 double* err_hist, double* out) {
  const size_t N = (size_t)L * m;
  double* z = (double*)malloc(sizeof(double) * N);
  double err = INFINITY, resid = NAN;
  int64_t k = 0;
  if (check_every < 1) check_every = 1;
  while (k < maxit) {
    if (or_sweep(L, m, method, Tlo, Tup, LU, piv, x, z) != 0) { free(z); return -2; }
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) s += z[i];
    if (!(s > 0.0) || !isfinite(s)) { free(z); out[0] = resid; out[1] = err; return -1; }
    err = 0.0;
    for (size_t i = 0; i < N; ++i) {
      double zi = z[i] / s;
      err += fabs(zi - x[i]);
      x[i] = zi;
    }
    ++k;
    if (err_hist) err_hist[k - 1] = err;
    if (eps > 0.0 && err <= eps) break;
    if (tol > 0.0 && (k % check_every == 0 || k == maxit)) {
      resid = or_residual(L, m, Tlo, Tdd, Tup, x);
      if (resid <= tol) break;
    }
  }
  out[0] = resid;
  out[1] = err;
  free(z);
  return k;
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* Set the OpenMP thread count (n <= 0: leave as is); returns the count in use. */
int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/*
 * Block-banded T = Q^T (Sect. 2 block partition, Algorithm 2 in full): nd
 * block diagonals with offsets off[0..nd) (T_{l, l+off[j]}), blocks row-major
 * in TB[j][l] (zero where l+off[j] is outside [0, L)); the diagonal offset 0
 * must be present (index jd).  One unnormalised step z = M^{-1} N x:
 *   stair types: step 1 z_i = -sum_{k not in J_i, k != i} Q_{i,k} x_k,
 *     J_i = {i} on diagonal-only rows and {i-1, i+1} on coupled rows;
 *     step 2 diagonal-only rows z_i = Q_ii^{-1} z_i;
 *     step 3 coupled rows z_i = Q_ii^{-1}(z_i - Q_{i,i-1} z_{i-1} - Q_{i,i+1} z_{i+1});
 *   BGS: z_l = Q_ll^{-1}(- sum_{d<0} Q_{l,l+d} z_{l+d} - sum_{d>0} Q_{l,l+d} x_{l+d});
 *   BJ:  z_l = Q_ll^{-1}(- sum_{d!=0} Q_{l,l+d} x_{l+d}).
 * Returns 0, or -1 on a bad method / missing diagonal.
 */
int or_sweep_banded(int64_t L, int m, int nd, const int* off, const double* TB, const double* LU,
                    const int* piv, int method, const double* x, double* z) {
  int jd = -1;
  for (int j = 0; j < nd; ++j) if (off[j] == 0) jd = j;
  if (jd < 0) return -1;
  (void)jd;
  const size_t mm = (size_t)m * m;
#define TBLK(j, l) (TB + ((size_t)(j) * (size_t)L + (size_t)(l)) * mm)
  if (method == OR_STAIR1 || method == OR_STAIR2) {
    const int type = method == OR_STAIR1 ? 1 : 2;
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l) {          /* step 1 */
      double* acc = (double*)calloc((size_t)m, sizeof(double));
      const int diag_only = stair_diag_only(type, l);
      for (int j = 0; j < nd; ++j) {
        const int d = off[j];
        if (d == 0) continue;
        if (!diag_only && (d == -1 || d == 1)) continue;   /* in J_i */
        const int64_t k = l + d;
        if (k < 0 || k >= L) continue;
        gemv_acc(m, TBLK(j, l), x + (size_t)k * m, acc);
      }
      for (int i = 0; i < m; ++i) z[(size_t)l * m + i] = -acc[i];
      free(acc);
    }
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l)            /* step 2 */
      if (stair_diag_only(type, l))
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, z + (size_t)l * m);
#pragma omp parallel for
    for (int64_t l = 0; l < L; ++l)            /* step 3 */
      if (!stair_diag_only(type, l)) {
        double* acc = (double*)calloc((size_t)m, sizeof(double));
        for (int j = 0; j < nd; ++j) {
          const int d = off[j];
          if (d != -1 && d != 1) continue;
          const int64_t k = l + d;
          if (k < 0 || k >= L) continue;
          gemv_acc(m, TBLK(j, l), z + (size_t)k * m, acc);
        }
        for (int i = 0; i < m; ++i) z[(size_t)l * m + i] -= acc[i];
        free(acc);
        or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, z + (size_t)l * m);
      }
    return 0;
  }
  if (method == OR_BGS || method == OR_BJ) {
    for (int64_t l = 0; l < L; ++l) {
      double* acc = (double*)calloc((size_t)m, sizeof(double));
      for (int j = 0; j < nd; ++j) {
        const int d = off[j];
        if (d == 0) continue;
        const int64_t k = l + d;
        if (k < 0 || k >= L) continue;
        const double* v = (method == OR_BGS && d < 0) ? z : x;
        gemv_acc(m, TBLK(j, l), v + (size_t)k * m, acc);
      }
      for (int i = 0; i < m; ++i) z[(size_t)l * m + i] = -acc[i];
      free(acc);
      or_lu_solve(m, BLK(LU, l, m), piv + (size_t)l * m, z + (size_t)l * m);
    }
    return 0;
  }
#undef TBLK
  return -1;
}

/* ||T x||_1 for block-banded T (Eq. (1)). */
double or_residual_banded(int64_t L, int m, int nd, const int* off, const double* TB,
                          const double* x) {
  const size_t mm = (size_t)m * m;
  double r = 0.0;
  double* acc = (double*)malloc(sizeof(double) * (size_t)m);
  for (int64_t l = 0; l < L; ++l) {
    for (int i = 0; i < m; ++i) acc[i] = 0.0;
    for (int j = 0; j < nd; ++j) {
      const int64_t k = l + off[j];
      if (k < 0 || k >= L) continue;
      gemv_acc(m, TB + ((size_t)j * (size_t)L + (size_t)l) * mm, x + (size_t)k * m, acc);
    }
    for (int i = 0; i < m; ++i) r += fabs(acc[i]);
  }
  free(acc);
  return r;
}
