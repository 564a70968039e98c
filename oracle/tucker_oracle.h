/*
 * Plain FP64 CPU oracle for the Tucker (HOSVD) approximation of Matern,
 * p-Slater and Gaussian covariance tensors (Litvinenko, Keyes, Khoromskaia,
 * Khoromskij, Matthies, "Tucker tensor analysis of Matern functions in
 * spatial statistics", arXiv:1711.06874).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine follows a definition of the paper step by step, in FP64,
 * without blocking or reordering beyond what the definition states.
 */
#ifndef TUCKER_ORACLE_H
#define TUCKER_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Covariance kinds.  OR_MATERN_SD: the 3D spectral density of the Matern
 * covariance, Sec. 3.7, Eq. (SD_matern) with d = 3, C = sigma2, alpha = p:
 * sigma2 / (alpha^2 + r_A^2)^(nu + 3/2).  OR_MATERN: Sec. 2.2, Eq. (Matern).  OR_SLATER_P: the
 * p-Slater function of Sec. 3.7, Eq. (exp_p).  OR_GAUSSIAN: the nu -> infinity
 * limit named in Sec. 2.2, written exp(-|x|^2/ell^2) (rank one, Sec. 4.4). */
enum { OR_MATERN = 0, OR_SLATER_P = 1, OR_GAUSSIAN = 2, OR_MATERN_SD = 3 };
/* Grid kinds.  OR_CELL: x_i = -b + (i + 1/2) 2b/n.  OR_VERTEX: Eq. (grid_points),
 * x_i = -b + (i - 1) h, h = 2b/(n - 1), with 1-based i. */
enum { OR_CELL = 0, OR_VERTEX = 1 };
/* Result flags. */
enum { OR_RANK_CAPPED = 1, OR_EPS_UNREACHABLE = 2 };

typedef struct {
  int kind;
  double nu;      /* Matern smoothness, nu > 0 */
  double ell[3];  /* per-axis length scale: the diagonal A = diag(1/ell^2) of Sec. 2.2 */
  double sigma2;  /* variance factor */
  double p;       /* p-Slater exponent */
} or_kernel;

typedef struct {
  int n[3];
  double b[3];
  int kind;
} or_grid;

/* K_nu(z) * exp(z) for z > 0 (trapezoid rule on the integral representation). */
double or_bessel_k_scaled(double nu, double z);
/* K_nu(z) for z > 0. */
double or_bessel_k(double nu, double z);
/* Matern covariance as a function of z = sqrt(2 nu) r / ell (Eq. (Matern)). */
double or_matern_z(double nu, double sigma2, double z);
/* Covariance at the point x (3 coordinates) relative to the origin. */
double or_kernel_value(const or_kernel* k, const double x[3]);
/* Grid coordinates of one axis, n values. */
void or_grid_axis(int kind, int n, double b, double* x);
/* Collocation tensor (Sec. 3.7): F[i1][i2][i3], row-major, i3 fastest. */
void or_tensor(const or_kernel* k, const or_grid* g, double* F);
/* Mode-m unfolding A_(m) (Sec. 3.2, Fig. Unfolding): n_m x (N / n_m), row-major. */
void or_unfold(const double* F, const int n[3], int mode, double* A);
/* Gram matrix G = A_(m) A_(m)^T with compensated sums, n_m x n_m. */
void or_gram(const double* F, const int n[3], int mode, double* G);
/* Compensated squared Frobenius norm of an array. */
double or_norm2(const double* X, long long len);
/* Cyclic Jacobi eigensolver: lam descending, V (n x n, row-major) column j is the
 * eigenvector of lam[j] with the canonical sign.  Returns the number of sweeps. */
int or_sym_eig(int n, const double* G, double* lam, double* V);
/* One-sided (Hestenes) Jacobi on the columns of M^T where M = A_(m): returns the
 * singular values (descending) and left singular vectors U (n_m x n_m). */
int or_unfolding_svd(const double* F, const int n[3], int mode, double* sigma, double* U);
/* Truncation rule: smallest r >= 1 whose discarded eigenvalue sum (negatives
 * clamped to zero, summed smallest first) is <= eps^2 normF2 / 3, capped at rmax. */
int or_rank(const double* lam, int n, double normF2, double eps, int rmax, int* flags);
/* Core B = F x_3 U3^T x_2 U2^T x_1 U1^T (mode 3 first).  U_k are n_k x ld_k
 * row-major with the first r_k columns used. */
void or_core(const double* F, const int n[3], const double* U1, int ld1, const double* U2, int ld2,
             const double* U3, int ld3, const int r[3], double* B);
/* Reconstruction X = B x_1 U1 x_2 U2 x_3 U3. */
void or_reconstruct(const double* B, const int r[3], const double* U1, int ld1, const double* U2,
                    int ld2, const double* U3, int ld3, const int n[3], double* X);
/* Value of the Tucker tensor at one multi-index (i1, i2, i3). */
double or_tucker_point(const double* B, const int r[3], const double* U1, int ld1, const double* U2,
                       int ld2, const double* U3, int ld3, const int idx[3]);
/* Relative Frobenius error |F - X| / |F| (Eq. (FNorm)) by direct subtraction. */
double or_rel_error(const double* F, const double* X, long long len);

/* Full HOSVD: tensor, three Grams, eigenpairs, ranks, core, error.
 *   rmax[3]  rank caps; rfix[3] > 0 forces that rank instead of the eps rule.
 *   U_k      n_k x n_k, row-major (all eigenvectors; the first r_k are the factors)
 *   lam_k    n_k eigenvalues, descending
 *   B        r1 r2 r3 core (caller sizes it n1 n2 n3)
 *   out[0] = |F|^2, out[1] = relative error, out[2] = |B|^2. */
int or_hosvd(const or_kernel* k, const or_grid* g, double eps, const int rmax[3], const int rfix[3],
             int ranks[3], int flags[3], double* U1, double* U2, double* U3, double* lam1,
             double* lam2, double* lam3, double* B, double* out);

/* Mode-m product Y = X x_m U^T (Sec. 3.1): X has dims d[3], U is d[m] x ld
 * row-major with its first r columns used; Y has dims d with d[m] replaced by r. */
void or_ttm(const double* X, const int d[3], int mode, const double* U, int ld, int r, double* Y);

/* Tucker-ALS (Sec. 3.2): `sweeps` sweeps over the modes 1, 2, 3 in order.  For
 * mode k the single-hole tensor Y_k = F x_{m != k} U_m^T is formed and U_k is
 * replaced by the r_k leading left singular vectors of its mode-k unfolding
 * (one-sided Jacobi, canonical signs).  U_k: n_k x r_k row-major, in and out.
 * B (r1 r2 r3) = F x_1 U1^T x_2 U2^T x_3 U3^T with the final factors.
 * core_norm2 (3 * sweeps, may be NULL): the sum of the r_k leading squared
 * singular values after each update, which is |F x_1 U1^T x_2 U2^T x_3 U3^T|^2
 * with the factors of that moment.  Returns 0, or -1 if memory ran out. */
int or_hooi(const double* F, const int n[3], double* U1, double* U2, double* U3, const int r[3], int sweeps,
            double* B, double* core_norm2);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
