// Tucker-ALS (Sec. 3.2, the alternating part after the HOSVD), FP64.
//
// One sweep visits the modes 1, 2, 3 in order.  For mode k the other two
// modes of F are mapped into their current subspaces, giving the single-hole
// tensor Y_k = F x_{m != k} U_m^T, and U_k becomes the r_k leading left
// singular vectors of Y_k's mode-k unfolding.  They are taken as the leading
// eigenvectors of the unfolding's Gram (an FP64 GEMM: the unfolding is only
// r_m r_l wide; the single-hole products write it with mode k outermost) by
// the subspace eigensolver of the HOSVD, whose eigenvalues are the squared singular
// values: their leading sum is |F x_1 U1^T x_2 U2^T x_3 U3^T|^2 right after
// the update.  The core is formed from the last single-hole tensor.
//
// The products reuse each other within a sweep: T1 = F x_3 U3^T serves
// modes 1 and 2 (U3 does not change between them), and mode 3 projects F on
// the new U1 and U2.  Per sweep F is contracted twice (2 r n^3 FLOP each);
// everything else is O(n^2 r^2) plus the three eigensolves.
#include <algorithm>

#include "tk_internal.h"

namespace tk {

void als_sizes(const int n[3], const int r[3], size_t out[kAlsBuffers]) {
  const size_t n1 = n[0], n2 = n[1], n3 = n[2], r1 = r[0], r2 = r[1], r3 = r[2];
  out[0] = n1 * n2 * r3;                                                  // T1
  out[1] = std::max(n1 * r2 * r3, std::max(r1 * n2 * r3, r1 * r2 * n3));  // Y_k, unfolded
  out[2] = r1 * n2 * n3;                                                  // W = F x_1 U1^T
  out[3] = 0;                                                             // Gram of Y_k's unfolding
  out[4] = 0;                                                             // eigensolver
  out[5] = 8;                                                             // trace of the Gram
  for (int k = 0; k < 3; ++k) {
    out[3] = std::max(out[3], (size_t)n[k] * n[k]);
    out[4] = std::max(out[4], sym_eig_batch_scratch_doubles(n[k], r[k], 1));
  }
}

namespace {

// G = Y Y^T for the unfolding Y (rows x K, row-major): every entry's sum
// runs over k in the same order, so G is exactly symmetric
void gram_rows(const double* Y, int rows, int K, double* G, cudaStream_t s) {
  GemmDesc g{rows, rows, K, 1, Y, 0, K, 1, Y, 0, 1, K, G, 0, rows, 1};
  gemm_f64(g, s);
}

}  // namespace

void als_f64(const double* F, const int n[3], double* const U[3], const int r[3], int sweeps, double* B,
             double* lam_log, const AlsBuffers& w, cudaStream_t s) {
  const long long n1 = n[0], n2 = n[1], n3 = n[2], r1 = r[0], r2 = r[1], r3 = r[2];
  // T1[i][j][c] = sum_l F[i][j][l] U3[l][c]
  const GemmDesc t1{(int)(n1 * n2), (int)r3, (int)n3, 1, F, 0, n3, 1, U[2], 0, r3, 1, w.T1, 0, r3, 1};
  if (sweeps == 0) {  // the core of the given factors: F x_3 U3^T, x_2 U2^T, x_1 U1^T
    gemm_f64(t1, s);
    GemmDesc y1{(int)r2, (int)r3, (int)n2, (int)n1, U[1], 0, 1, r2, w.T1, n2 * r3, r3, 1, w.Y, r2 * r3, r3, 1};
    gemm_f64(y1, s);
    GemmDesc bc{(int)r1, (int)(r2 * r3), (int)n1, 1, U[0], 0, 1, r1, w.Y, 0, r2 * r3, 1, B, 0, r2 * r3, 1};
    gemm_f64(bc, s);
    return;
  }
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    double* lam = lam_log + (size_t)sweep * 3 * kAlsLamStride;
    // mode 1: Y1[i][b][c] = sum_j U2[j][b] T1[i][j][c], unfolded as n1 x (r2 r3)
    gemm_f64(t1, s);
    GemmDesc y1{(int)r2, (int)r3, (int)n2, (int)n1, U[1], 0, 1, r2, w.T1, n2 * r3, r3, 1, w.Y, r2 * r3, r3, 1};
    gemm_f64(y1, s);
    gram_rows(w.Y, (int)n1, (int)(r2 * r3), w.G, s);
    sym_eig_batch(w.G, n[0], r[0], 1, lam, U[0], w.trace, w.eig_scr, s);
    // mode 2: Y2[j][a][c] = sum_i U1[i][a] T1[i][j][c] (U3 unchanged since T1),
    // written with j outermost: the unfolding n2 x (r1 r3)
    GemmDesc y2{(int)r1, (int)r3, (int)n1, (int)n2, U[0], 0, 1, r1, w.T1, r3, n2 * r3, 1, w.Y, r1 * r3, r3, 1};
    gemm_f64(y2, s);
    gram_rows(w.Y, (int)n2, (int)(r1 * r3), w.G, s);
    sym_eig_batch(w.G, n[1], r[1], 1, lam + kAlsLamStride, U[1], w.trace, w.eig_scr, s);
    // mode 3: W[a][j][l] = sum_i U1[i][a] F[i][j][l]; Y3[l][a][b] = sum_j U2[j][b] W[a][j][l],
    // written with l outermost: the unfolding n3 x (r1 r2)
    GemmDesc wd{(int)r1, (int)(n2 * n3), (int)n1, 1, U[0], 0, 1, r1, F, 0, n2 * n3, 1, w.W, 0, n2 * n3, 1};
    gemm_f64(wd, s);
    GemmDesc y3{(int)r2, (int)n3, (int)n2, (int)r1, U[1], 0, 1, r2, w.W, n2 * n3, n3, 1, w.Y, r2, 1, r1 * r2};
    gemm_f64(y3, s);
    gram_rows(w.Y, (int)n3, (int)(r1 * r2), w.G, s);
    sym_eig_batch(w.G, n[2], r[2], 1, lam + 2 * kAlsLamStride, U[2], w.trace, w.eig_scr, s);
  }
  // B[a][b][c] = sum_l Y3[l][a][b] U3[l][c]
  GemmDesc bc{(int)(r1 * r2), (int)r3, (int)n3, 1, w.Y, 0, 1, r1 * r2, U[2], 0, r3, 1, B, 0, r3, 1};
  gemm_f64(bc, s);
}

}  // namespace tk
