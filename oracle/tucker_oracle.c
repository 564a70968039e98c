/*
 * Plain FP64 CPU oracle for the Tucker (HOSVD) approximation of covariance
 * tensors, following arXiv:1711.06874.
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code with the CUDA library.  Parity status of each
 * routine and the pin that fixes it are listed with the routine.
 *
 * Built with -ffp-contract=off so that x86-64 and AArch64 hosts give the same
 * bits.  OpenMP only splits independent output entries across threads; no
 * sum is ever split, so results do not depend on the thread count.
 */
#include "tucker_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  double s, c;
} nacc;

static inline void nacc_add(nacc* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nacc_val(const nacc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Modified Bessel function of the second kind, K_nu(z).                    */
/*                                                                          */
/* Sec. 2.2 names K_nu but gives no method.  The oracle uses the integral   */
/*   K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt,   z > 0,             */
/* written as exp(-z) * int_0^inf exp(-z (cosh t - 1)) cosh(nu t) dt, and   */
/* evaluated by the trapezoid rule on [0, T], halving the step until two    */
/* successive sums agree to 1e-15.  The integrand is analytic and decays    */
/* doubly exponentially, so the trapezoid sums converge exponentially.      */
/* Pins: closed forms at nu = 1/2, 3/2, 5/2, the order recurrence, scipy.   */
/* ------------------------------------------------------------------------ */
static double kint_log(double nu, double z, double t) {
  double s = sinh(0.5 * t);
  return -2.0 * z * s * s + nu * t; /* -z (cosh t - 1) + nu t */
}

static double kint(double nu, double z, double t) {
  double s = sinh(0.5 * t);
  double e = -2.0 * z * s * s;
  return 0.5 * (exp(e + nu * t) + exp(e - nu * t));
}

double or_bessel_k_scaled(double nu, double z) {
  if (!(z > 0.0)) return INFINITY;
  nu = fabs(nu); /* K_{-nu} = K_nu */
  /* peak of the dominant exponent -z (cosh t - 1) + nu t */
  double tpk = asinh(nu / z);
  double gpk = kint_log(nu, z, tpk);
  /* truncation: beyond T the log-integrand is 46 below its peak and falling */
  double T = tpk + 0.5;
  for (int it = 0; it < 10000; ++it) {
    double slope = -z * sinh(T) + nu;
    if (kint_log(nu, z, T) < gpk - 46.0 && slope < -1.0) break;
    T += 0.25 * (T > 1.0 ? T : 1.0);
  }
  double zz = z + nu + 1.0;
  double h = 0.5 / sqrt(zz);
  if (h > 0.5) h = 0.5;
  long m = (long)ceil(T / h);
  h = T / (double)m;
  double s = 0.5 * kint(nu, z, 0.0);
  for (long k = 1; k <= m; ++k) s += kint(nu, z, k * h);
  double prev = s * h;
  for (int halving = 1; halving <= 30; ++halving) {
    double odd = 0.0;
    for (long k = 1; k <= 2 * m; k += 2) odd += kint(nu, z, k * 0.5 * h);
    s += odd;
    m *= 2;
    h *= 0.5;
    double cur = s * h;
    if (halving >= 3 && fabs(cur - prev) <= 1e-15 * fabs(cur)) return cur;
    prev = cur;
  }
  return prev;
}

double or_bessel_k(double nu, double z) { return exp(-z) * or_bessel_k_scaled(nu, z); }

/* Eq. (Matern): C = sigma2 2^(1-nu) / Gamma(nu) z^nu K_nu(z), z = sqrt(2 nu) r / ell.
 * C(0) = sigma2 is the limit z -> 0. */
double or_matern_z(double nu, double sigma2, double z) {
  if (z <= 0.0) return sigma2;
  double lp = (1.0 - nu) * log(2.0) - lgamma(nu) + nu * log(z) - z;
  return sigma2 * exp(lp) * or_bessel_k_scaled(nu, z);
}

/* Covariance at x relative to the origin.  The anisotropic distance of Sec. 2.2
 * uses A = diag(1/ell_a^2): r_A^2 = sum_a x_a^2 / ell_a^2.  With equal ell this is
 * r / ell of Eq. (Matern). */
double or_kernel_value(const or_kernel* k, const double x[3]) {
  double ra2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    double u = x[a] / k->ell[a];
    ra2 += u * u;
  }
  double ra = sqrt(ra2);
  switch (k->kind) {
    case OR_MATERN:
      return or_matern_z(k->nu, k->sigma2, sqrt(2.0 * k->nu) * ra);
    case OR_SLATER_P:
      return k->sigma2 * exp(-pow(ra, k->p));
    case OR_GAUSSIAN:
      return k->sigma2 * exp(-ra2);
    case OR_MATERN_SD:
      /* Eq. (SD_matern), d = 3 */
      return k->sigma2 / pow(k->p * k->p + ra2, k->nu + 1.5);
    default:
      return NAN;
  }
}

void or_grid_axis(int kind, int n, double b, double* x) {
  for (int i = 0; i < n; ++i) {
    if (kind == OR_VERTEX)
      x[i] = (n == 1) ? 0.0 : -b + (double)i * (2.0 * b / (double)(n - 1));
    else
      x[i] = -b + ((double)i + 0.5) * (2.0 * b / (double)n);
  }
}

/* Collocation tensor of Sec. 3.7: F[i1][i2][i3] = q(x_i1, x_i2, x_i3). */
void or_tensor(const or_kernel* k, const or_grid* g, double* F) {
  int n1 = g->n[0], n2 = g->n[1], n3 = g->n[2];
  double* x1 = (double*)malloc(sizeof(double) * n1);
  double* x2 = (double*)malloc(sizeof(double) * n2);
  double* x3 = (double*)malloc(sizeof(double) * n3);
  or_grid_axis(g->kind, n1, g->b[0], x1);
  or_grid_axis(g->kind, n2, g->b[1], x2);
  or_grid_axis(g->kind, n3, g->b[2], x3);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int l = 0; l < n3; ++l) {
        double x[3] = {x1[i], x2[j], x3[l]};
        F[((long long)i * n2 + j) * n3 + l] = or_kernel_value(k, x);
      }
  free(x1);
  free(x2);
  free(x3);
}

/* ------------------------------------------------------------------------ */
/* Unfolding and Gram (Sec. 3.2: the HOSVD takes the SVD of A_(l); the Gram  */
/* A_(l) A_(l)^T has the same left singular vectors, eigenvalues sigma^2).   */
/* ------------------------------------------------------------------------ */
void or_unfold(const double* F, const int n[3], int mode, double* A) {
  int n1 = n[0], n2 = n[1], n3 = n[2];
  long long N = (long long)n1 * n2 * n3;
  long long cols = N / n[mode];
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int l = 0; l < n3; ++l) {
        double v = F[((long long)i * n2 + j) * n3 + l];
        long long row, col;
        if (mode == 0) {
          row = i;
          col = (long long)j * n3 + l;
        } else if (mode == 1) {
          row = j;
          col = (long long)i * n3 + l;
        } else {
          row = l;
          col = (long long)i * n2 + j;
        }
        A[row * cols + col] = v;
      }
}

void or_gram(const double* F, const int n[3], int mode, double* G) {
  int m = n[mode];
  long long N = (long long)n[0] * n[1] * n[2];
  long long cols = N / m;
  double* A = (double*)malloc(sizeof(double) * (size_t)N);
  or_unfold(F, n, mode, A);
#pragma omp parallel for schedule(dynamic, 1)
  for (int a = 0; a < m; ++a) {
    const double* ra = A + (long long)a * cols;
    for (int c = a; c < m; ++c) {
      const double* rc = A + (long long)c * cols;
      nacc s = {0.0, 0.0};
      for (long long t = 0; t < cols; ++t) nacc_add(&s, ra[t] * rc[t]);
      double v = nacc_val(&s);
      G[(long long)a * m + c] = v;
      G[(long long)c * m + a] = v;
    }
  }
  free(A);
}

double or_norm2(const double* X, long long len) {
  nacc s = {0.0, 0.0};
  for (long long t = 0; t < len; ++t) nacc_add(&s, X[t] * X[t]);
  return nacc_val(&s);
}

/* ------------------------------------------------------------------------ */
/* Eigenpairs of a symmetric matrix by cyclic Jacobi rotations.             */
/* Each rotation in the (p, q) plane annihilates a_pq; sweeps repeat until  */
/* no off-diagonal entry exceeds 1e-18 |A|_F.  Pins: brute-force SVD of the */
/* unfoldings at small n, rank-one Gaussian, full-rank exactness.           */
/* ------------------------------------------------------------------------ */
static void canonical_sign(int n, double* V, int col) {
  /* the entry of largest magnitude among the first ceil(n/2) rows is made
   * positive; on an exact tie the lowest index wins */
  int half = (n + 1) / 2;
  int best = 0;
  double bv = -1.0;
  for (int i = 0; i < half; ++i) {
    double a = fabs(V[(long long)i * n + col]);
    if (a > bv) {
      bv = a;
      best = i;
    }
  }
  if (V[(long long)best * n + col] < 0.0)
    for (int i = 0; i < n; ++i) V[(long long)i * n + col] = -V[(long long)i * n + col];
}

static void sort_desc(int n, double* lam, double* V) {
  /* selection sort of eigenvalues, moving eigenvector columns along */
  for (int a = 0; a < n; ++a) {
    int best = a;
    for (int c = a + 1; c < n; ++c)
      if (lam[c] > lam[best]) best = c;
    if (best != a) {
      double t = lam[a];
      lam[a] = lam[best];
      lam[best] = t;
      for (int i = 0; i < n; ++i) {
        double u = V[(long long)i * n + a];
        V[(long long)i * n + a] = V[(long long)i * n + best];
        V[(long long)i * n + best] = u;
      }
    }
  }
}

int or_sym_eig(int n, const double* G, double* lam, double* V) {
  double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
  memcpy(A, G, sizeof(double) * (size_t)n * n);
  for (long long t = 0; t < (long long)n * n; ++t) V[t] = 0.0;
  for (int i = 0; i < n; ++i) V[(long long)i * n + i] = 1.0;
  double fro = sqrt(or_norm2(A, (long long)n * n));
  double tau = 1e-18 * fro;
  int sweep;
  for (sweep = 1; sweep <= 100; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(long long)p * n + q];
        if (!(fabs(apq) > tau)) continue;
        double app = A[(long long)p * n + p], aqq = A[(long long)q * n + q];
        /* tan of the rotation angle: the smaller root of t^2 + 2 theta t - 1 = 0 */
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double s = t * c;
        /* A <- J^T A J with J the identity except J_pp = J_qq = c, J_pq = s, J_qp = -s */
        for (int k = 0; k < n; ++k) {
          double akp = A[(long long)k * n + p], akq = A[(long long)k * n + q];
          A[(long long)k * n + p] = c * akp - s * akq;
          A[(long long)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[(long long)p * n + k], aqk = A[(long long)q * n + k];
          A[(long long)p * n + k] = c * apk - s * aqk;
          A[(long long)q * n + k] = s * apk + c * aqk;
        }
        A[(long long)p * n + q] = 0.0;
        A[(long long)q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          double vkp = V[(long long)k * n + p], vkq = V[(long long)k * n + q];
          V[(long long)k * n + p] = c * vkp - s * vkq;
          V[(long long)k * n + q] = s * vkp + c * vkq;
        }
        rotated = 1;
      }
    if (!rotated) break;
  }
  for (int i = 0; i < n; ++i) lam[i] = A[(long long)i * n + i];
  free(A);
  sort_desc(n, lam, V);
  for (int j = 0; j < n; ++j) canonical_sign(n, V, j);
  return sweep;
}

/* One-sided Jacobi on the columns of M = A_(m)^T (cols x n_m): rotations make
 * the columns mutually orthogonal; the column norms are the singular values of
 * A_(m) and the accumulated rotations its left singular vectors.  This is the
 * HOSVD exactly as Sec. 3.2 states it (SVD of the unfolding), without forming
 * the Gram.  Used at small sizes as the second route. */
int or_unfolding_svd(const double* F, const int n[3], int mode, double* sigma, double* U) {
  int m = n[mode];
  long long N = (long long)n[0] * n[1] * n[2];
  long long len = N / m;
  double* A = (double*)malloc(sizeof(double) * (size_t)N); /* row a = column a of M */
  or_unfold(F, n, mode, A);
  for (long long t = 0; t < (long long)m * m; ++t) U[t] = 0.0;
  for (int i = 0; i < m; ++i) U[(long long)i * m + i] = 1.0;
  int sweep;
  for (sweep = 1; sweep <= 100; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        double* x = A + (long long)p * len;
        double* y = A + (long long)q * len;
        nacc al = {0, 0}, be = {0, 0}, ga = {0, 0};
        for (long long t = 0; t < len; ++t) {
          nacc_add(&al, x[t] * x[t]);
          nacc_add(&be, y[t] * y[t]);
          nacc_add(&ga, x[t] * y[t]);
        }
        double alpha = nacc_val(&al), beta = nacc_val(&be), gamma = nacc_val(&ga);
        if (!(fabs(gamma) > 1e-17 * sqrt(alpha * beta)) || gamma == 0.0) continue;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (long long k = 0; k < len; ++k) {
          double u = x[k], v = y[k];
          x[k] = c * u - s * v;
          y[k] = s * u + c * v;
        }
        for (int k = 0; k < m; ++k) {
          double u = U[(long long)k * m + p], v = U[(long long)k * m + q];
          U[(long long)k * m + p] = c * u - s * v;
          U[(long long)k * m + q] = s * u + c * v;
        }
        rotated = 1;
      }
    if (!rotated) break;
  }
  for (int a = 0; a < m; ++a) sigma[a] = sqrt(or_norm2(A + (long long)a * len, len));
  free(A);
  sort_desc(m, sigma, U);
  for (int j = 0; j < m; ++j) canonical_sign(m, U, j);
  return sweep;
}

/* ------------------------------------------------------------------------ */
/* Truncation.  Task 1 (Sec. 2.1) asks for an approximation within eps; the  */
/* paper does not say how eps is shared between modes.  Reading: the HOSVD   */
/* bound |F - X|^2 <= sum_k sum_{i > r_k} lam_i^(k) is split evenly, so each */
/* mode keeps the smallest r with discarded sum <= eps^2 |F|^2 / 3.          */
/* ------------------------------------------------------------------------ */
int or_rank(const double* lam, int n, double normF2, double eps, int rmax, int* flags) {
  double thr = eps * eps * normF2 / 3.0;
  double* suffix = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  nacc s = {0.0, 0.0};
  suffix[n] = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    nacc_add(&s, lam[i] > 0.0 ? lam[i] : 0.0);
    suffix[i] = nacc_val(&s);
  }
  int r = n;
  for (int q = 1; q <= n; ++q)
    if (suffix[q] <= thr) {
      r = q;
      break;
    }
  free(suffix);
  int f = 0;
  if (r > rmax) {
    r = rmax;
    f |= OR_RANK_CAPPED;
  }
  if (thr < 10.0 * ldexp(1.0, -53) * (double)n * normF2) f |= OR_EPS_UNREACHABLE;
  if (flags) *flags = f;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Core and reconstruction by direct loops (Sec. 3.1 Tucker format,         */
/* Sec. 3.2 final step: B = A x_1 V1^T x_2 V2^T x_3 V3^T).                  */
/* ------------------------------------------------------------------------ */
void or_core(const double* F, const int n[3], const double* U1, int ld1, const double* U2, int ld2,
             const double* U3, int ld3, const int r[3], double* B) {
  int n1 = n[0], n2 = n[1], n3 = n[2];
  int r1 = r[0], r2 = r[1], r3 = r[2];
  double* T1 = (double*)malloc(sizeof(double) * (size_t)n1 * n2 * r3);
  double* T2 = (double*)malloc(sizeof(double) * (size_t)n1 * r2 * r3);
  /* T1[i][j][c] = sum_l F[i][j][l] U3[l][c] */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int c = 0; c < r3; ++c) {
        double s = 0.0;
        for (int l = 0; l < n3; ++l) s += F[((long long)i * n2 + j) * n3 + l] * U3[(long long)l * ld3 + c];
        T1[((long long)i * n2 + j) * r3 + c] = s;
      }
  /* T2[i][b][c] = sum_j U2[j][b] T1[i][j][c] */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n1; ++i)
    for (int b = 0; b < r2; ++b)
      for (int c = 0; c < r3; ++c) {
        double s = 0.0;
        for (int j = 0; j < n2; ++j) s += U2[(long long)j * ld2 + b] * T1[((long long)i * n2 + j) * r3 + c];
        T2[((long long)i * r2 + b) * r3 + c] = s;
      }
  /* B[a][b][c] = sum_i U1[i][a] T2[i][b][c] */
  for (int a = 0; a < r1; ++a)
    for (int b = 0; b < r2; ++b)
      for (int c = 0; c < r3; ++c) {
        double s = 0.0;
        for (int i = 0; i < n1; ++i) s += U1[(long long)i * ld1 + a] * T2[((long long)i * r2 + b) * r3 + c];
        B[((long long)a * r2 + b) * r3 + c] = s;
      }
  free(T1);
  free(T2);
}

void or_reconstruct(const double* B, const int r[3], const double* U1, int ld1, const double* U2,
                    int ld2, const double* U3, int ld3, const int n[3], double* X) {
  int n1 = n[0], n2 = n[1], n3 = n[2];
  int r1 = r[0], r2 = r[1], r3 = r[2];
  double* W1 = (double*)malloc(sizeof(double) * (size_t)n1 * r2 * r3);
  double* W2 = (double*)malloc(sizeof(double) * (size_t)n1 * n2 * r3);
  /* W1[i][b][c] = sum_a U1[i][a] B[a][b][c] */
  for (int i = 0; i < n1; ++i)
    for (int b = 0; b < r2; ++b)
      for (int c = 0; c < r3; ++c) {
        double s = 0.0;
        for (int a = 0; a < r1; ++a) s += U1[(long long)i * ld1 + a] * B[((long long)a * r2 + b) * r3 + c];
        W1[((long long)i * r2 + b) * r3 + c] = s;
      }
  /* W2[i][j][c] = sum_b U2[j][b] W1[i][b][c] */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int c = 0; c < r3; ++c) {
        double s = 0.0;
        for (int b = 0; b < r2; ++b) s += U2[(long long)j * ld2 + b] * W1[((long long)i * r2 + b) * r3 + c];
        W2[((long long)i * n2 + j) * r3 + c] = s;
      }
  /* X[i][j][l] = sum_c U3[l][c] W2[i][j][c] */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n2; ++j)
      for (int l = 0; l < n3; ++l) {
        double s = 0.0;
        for (int c = 0; c < r3; ++c) s += U3[(long long)l * ld3 + c] * W2[((long long)i * n2 + j) * r3 + c];
        X[((long long)i * n2 + j) * n3 + l] = s;
      }
  free(W1);
  free(W2);
}

double or_tucker_point(const double* B, const int r[3], const double* U1, int ld1, const double* U2,
                       int ld2, const double* U3, int ld3, const int idx[3]) {
  nacc s = {0.0, 0.0};
  for (int a = 0; a < r[0]; ++a)
    for (int b = 0; b < r[1]; ++b)
      for (int c = 0; c < r[2]; ++c)
        nacc_add(&s, B[((long long)a * r[1] + b) * r[2] + c] * U1[(long long)idx[0] * ld1 + a] *
                         U2[(long long)idx[1] * ld2 + b] * U3[(long long)idx[2] * ld3 + c]);
  return nacc_val(&s);
}

/* Eq. (FNorm) by direct subtraction with compensated sums (never through
 * |F|^2 - |B|^2, which cancels at small errors). */
double or_rel_error(const double* F, const double* X, long long len) {
  nacc d = {0.0, 0.0}, f = {0.0, 0.0};
  for (long long t = 0; t < len; ++t) {
    double e = F[t] - X[t];
    nacc_add(&d, e * e);
    nacc_add(&f, F[t] * F[t]);
  }
  return sqrt(nacc_val(&d) / nacc_val(&f));
}

/* ------------------------------------------------------------------------ */
/* Full HOSVD pipeline: sample, three Grams, eigenpairs, ranks, core, error. */
/* ------------------------------------------------------------------------ */
int or_hosvd(const or_kernel* k, const or_grid* g, double eps, const int rmax[3], const int rfix[3],
             int ranks[3], int flags[3], double* U1, double* U2, double* U3, double* lam1,
             double* lam2, double* lam3, double* B, double* out) {
  const int* n = g->n;
  long long N = (long long)n[0] * n[1] * n[2];
  double* F = (double*)malloc(sizeof(double) * (size_t)N);
  if (!F) return -1;
  or_tensor(k, g, F);
  double normF2 = or_norm2(F, N);
  double* U[3] = {U1, U2, U3};
  double* lam[3] = {lam1, lam2, lam3};
  for (int m = 0; m < 3; ++m) {
    double* G = (double*)malloc(sizeof(double) * (size_t)n[m] * n[m]);
    or_gram(F, n, m, G);
    or_sym_eig(n[m], G, lam[m], U[m]);
    free(G);
    int f = 0;
    int r = or_rank(lam[m], n[m], normF2, eps, rmax[m], &f);
    if (rfix && rfix[m] > 0) {
      r = rfix[m] < n[m] ? rfix[m] : n[m];
      f = 0;
    }
    ranks[m] = r;
    flags[m] = f;
  }
  or_core(F, n, U1, n[0], U2, n[1], U3, n[2], ranks, B);
  double* X = (double*)malloc(sizeof(double) * (size_t)N);
  or_reconstruct(B, ranks, U1, n[0], U2, n[1], U3, n[2], n, X);
  out[0] = normF2;
  out[1] = or_rel_error(F, X, N);
  out[2] = or_norm2(B, (long long)ranks[0] * ranks[1] * ranks[2]);
  free(X);
  free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tucker-ALS (Sec. 3.2, second part of the algorithm).                      */
/* Parity: pinned by the d = 2 reduction (from a random start the sweeps     */
/* reach the Eckart-Young optimum of the matrix SVD), exact recovery of a    */
/* tensor of exact multilinear rank after one sweep from a random start,     */
/* the monotone core norm, |F|^2 = |B|^2 + |F - X|^2, and the HOSVD factors  */
/* of a rank-one tensor as a fixed point.                                    */
/* ------------------------------------------------------------------------ */
void or_ttm(const double* X, const int d[3], int mode, const double* U, int ld, int r, double* Y) {
  int e[3] = {d[0], d[1], d[2]};
  e[mode] = r;
  long long outer = 1, inner = 1;
  for (int a = 0; a < mode; ++a) outer *= d[a];
  for (int a = mode + 1; a < 3; ++a) inner *= d[a];
  const int m = d[mode];
  (void)e;
  /* Y[o][c][t] = sum_i X[o][i][t] U[i][c] */
#pragma omp parallel for schedule(static)
  for (long long o = 0; o < outer; ++o)
    for (int c = 0; c < r; ++c)
      for (long long t = 0; t < inner; ++t) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += X[(o * m + i) * inner + t] * U[(long long)i * ld + c];
        Y[(o * r + c) * inner + t] = s;
      }
}

int or_hooi(const double* F, const int n[3], double* U1, double* U2, double* U3, const int r[3], int sweeps,
            double* B, double* core_norm2) {
  double* U[3] = {U1, U2, U3};
  int nmax = n[0];
  for (int a = 1; a < 3; ++a)
    if (n[a] > nmax) nmax = n[a];
  long long big = 0;
  for (int k = 0; k < 3; ++k) {
    /* the largest of the two intermediates of mode k's projections */
    int d[3] = {n[0], n[1], n[2]};
    int first = (k == 2) ? 0 : 2;
    d[first] = r[first];
    long long sz = (long long)d[0] * d[1] * d[2];
    if (sz > big) big = sz;
  }
  double* T = (double*)malloc(sizeof(double) * (size_t)big);
  double* Y = (double*)malloc(sizeof(double) * (size_t)big);
  double* sig = (double*)malloc(sizeof(double) * (size_t)nmax);
  double* W = (double*)malloc(sizeof(double) * (size_t)nmax * nmax);
  if (!T || !Y || !sig || !W) {
    free(T);
    free(Y);
    free(sig);
    free(W);
    return -1;
  }
  for (int sweep = 0; sweep < sweeps; ++sweep)
    for (int k = 0; k < 3; ++k) {
      /* single-hole tensor: every mode but k mapped into its subspace */
      const int m1 = (k == 2) ? 0 : 2, m2 = (k == 1) ? 0 : 1;
      int d[3] = {n[0], n[1], n[2]};
      or_ttm(F, d, m1, U[m1], r[m1], r[m1], T);
      d[m1] = r[m1];
      or_ttm(T, d, m2, U[m2], r[m2], r[m2], Y);
      d[m2] = r[m2];
      /* U_k: leading left singular vectors of the mode-k unfolding of Y */
      or_unfolding_svd(Y, d, k, sig, W);
      nacc c2 = {0.0, 0.0};
      for (int a = 0; a < r[k]; ++a) nacc_add(&c2, sig[a] * sig[a]);
      if (core_norm2) core_norm2[sweep * 3 + k] = nacc_val(&c2);
      for (int i = 0; i < n[k]; ++i)
        for (int a = 0; a < r[k]; ++a) U[k][(long long)i * r[k] + a] = W[(long long)i * n[k] + a];
    }
  or_core(F, n, U1, r[0], U2, r[1], U3, r[2], r, B);
  free(T);
  free(Y);
  free(sig);
  free(W);
  return 0;
}
