/* CPU oracle for the generalized Kohn-Sham eigenproblem H C = S C eps (paper Sec. 2,
 * generalized eigenvalue problem; Bloch form Eq. eigenval_problem; noncollinear form in
 * Sec. 2 and Sec. 3.2).  TEST INFRASTRUCTURE: plain, slow, unblocked FP64 textbook
 * algorithms written from the mathematics (Golub & Van Loan, "Matrix Computations",
 * Secs. 4.2, 5.1, 8.3), sharing no code with the CUDA path.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may call it.
 *
 * Steps: (1) unblocked Cholesky of S; (2) H' = L^-1 H L^-H by the two-sided column recurrence;
 * (3) Householder tridiagonalization (Hermitian reflectors) and a diagonal phase that
 * makes the off-diagonal real; (4) implicit QL with Wilkinson shift on the real
 * tridiagonal with rotation accumulation; (5) ascending sort; (6) X = Q D Z and
 * C = L^-H X by explicit back substitution.
 *
 * OpenMP runs the independent loops of these steps in parallel (rows of a rank-1/rank-2
 * update, rows of a matrix-vector product, columns of a substitution, rows receiving a
 * sweep's rotations); every matrix element still receives the same operations, with the
 * same operands, in the same order as in the sequential loops, so the results do not
 * depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------- real tridiagonal eigensolver: implicit QL with Wilkinson shift ---------- */

/* Eigen-decomposition of the real symmetric tridiagonal T (diag d[0..n-1], off-diagonal
 * e[0..n-2]).  On exit d holds eigenvalues (unsorted) and the columns of Z (row-major
 * n x n, initialised by the caller, typically to I) are multiplied by the rotations, so
 * that Z_out = Z_in * Q with T = Q diag(d) Q^T.  Each QL sweep works on an unreduced
 * block [p, q]; the shift is the eigenvalue of the leading 2 x 2 of the block that is
 * closer to d[p]; the bulge is chased from the bottom of the block to the top.
 * Returns 0, or 1 + p if the block starting at p needs more than 60 sweeps. */
static int tridiag_ql_(int n, double *d, double *e, double *Z, double *rc_, double *rs_);
static int tridiag_ql(int n, double *d, double *e, double *Z) {
  double *rc_ = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *rs_ = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  int r = tridiag_ql_(n, d, e, Z, rc_, rs_);
  free(rc_);
  free(rs_);
  return r;
}
static int tridiag_ql_(int n, double *d, double *e, double *Z, double *rc_, double *rs_) {
  const double eps = 2.220446049250313e-16;
  for (int p = 0; p < n; p++) {
    int sweeps = 0;
    for (;;) {
      int q = p;
      while (q < n - 1) {
        double scale = fabs(d[q]) + fabs(d[q + 1]);
        if (fabs(e[q]) <= eps * scale) { e[q] = 0.0; break; }
        q++;
      }
      if (q == p) break;                       /* d[p] has converged */
      if (++sweeps > 60) return 1 + p;
      /* Wilkinson shift from the top 2x2 [[d_p, e_p], [e_p, d_{p+1}]] */
      double delta = 0.5 * (d[p + 1] - d[p]);
      double r = hypot(delta, e[p]);
      double shift = d[p] - e[p] * e[p] / (delta + (delta >= 0.0 ? r : -r));
      /* implicit QL sweep: rotations in planes (k-1, k), k = q .. p+1; the rotations only
       * depend on d and e, so they are recorded and applied to the rows of Z afterwards */
      double x = d[q] - shift;
      double z = e[q - 1];
      for (int k = q; k > p; k--) {
        /* rotation R = [[c, s], [-s, c]] on (k-1, k) with R^T (z, x)^T = (0, r)^T */
        double rr = hypot(x, z);
        double c = (rr == 0.0) ? 1.0 : x / rr;
        double s = (rr == 0.0) ? 0.0 : z / rr;
        if (k < q) e[k] = rr;                   /* the element chased up into (k+1, k) */
        double a = d[k - 1], b = e[k - 1], cc = d[k];
        d[k - 1] = a * c * c - 2.0 * b * c * s + cc * s * s;
        d[k] = a * s * s + 2.0 * b * c * s + cc * c * c;
        e[k - 1] = c * s * (a - cc) + b * (c * c - s * s);
        rc_[k] = c;
        rs_[k] = s;
        if (k - 1 > p) {                        /* new bulge at (k-2, k) */
          x = e[k - 1];
          z = s * e[k - 2];
          e[k - 2] = c * e[k - 2];
        }
      }
      /* Z <- Z R_q R_{q-1} ... R_{p+1}: each row takes the sweep's rotations in order */
#pragma omp parallel for schedule(static) if ((size_t)n * (q - p) > 20000)
      for (int row = 0; row < n; row++) {
        double *zr_ = Z + (size_t)row * n;
        for (int k = q; k > p; k--) {
          double zl = zr_[k - 1], zk = zr_[k];
          zr_[k - 1] = rc_[k] * zl - rs_[k] * zk;
          zr_[k] = rs_[k] * zl + rc_[k] * zk;
        }
      }
    }
  }
  return 0;
}

/* Ascending sort of eigenvalues (ties keep the lower original index first) with the
 * matching permutation of the columns of Z. */
static void sort_ascending(int n, double *d, double *Z, int *perm) {
  for (int i = 0; i < n; i++) perm[i] = i;
  for (int i = 1; i < n; i++) {                 /* insertion sort: stable */
    int pi = perm[i];
    int j = i - 1;
    while (j >= 0 && d[perm[j]] > d[pi]) { perm[j + 1] = perm[j]; j--; }
    perm[j + 1] = pi;
  }
  double *dd = (double *)malloc(sizeof(double) * n);
  for (int i = 0; i < n; i++) dd[i] = d[perm[i]];
  memcpy(d, dd, sizeof(double) * n);
#pragma omp parallel
  {
    double *row = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp for schedule(static)
    for (int r = 0; r < n; r++) {
      for (int c = 0; c < n; c++) row[c] = Z[(size_t)r * n + perm[c]];
      memcpy(Z + (size_t)r * n, row, sizeof(double) * n);
    }
    free(row);
  }
  free(dd);
}

int oracle_tridiag_eig(int n, double *d, double *e, double *Z) {
  int *perm = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
  int rc = tridiag_ql(n, d, e, Z);
  if (!rc) sort_ascending(n, d, Z, perm);
  free(perm);
  return rc;
}

/* ---------- real instantiation ---------- */
#define SCALAR double
#define SFX(name) name##_d
#define CONJ(x) (x)
#define ABS2(x) ((x) * (x))
#define REALPART(x) (x)
#define SCALE_PHASE(x) ((x) < 0.0 ? -1.0 : 1.0)
#include "oracle_core.inc"
#undef SCALAR
#undef SFX
#undef CONJ
#undef ABS2
#undef REALPART
#undef SCALE_PHASE

/* ---------- complex instantiation ---------- */
static inline double complex unit_phase(double complex x) {
  double a = cabs(x);
  return a > 0.0 ? x / a : 1.0;
}
#define SCALAR double complex
#define SFX(name) name##_z
#define CONJ(x) conj(x)
#define ABS2(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define REALPART(x) creal(x)
#define SCALE_PHASE(x) unit_phase(x)
#include "oracle_core.inc"
