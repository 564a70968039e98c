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

// Contraction of a long tensor with one thin factor, C(line, c) =
// sum_k X(line, k) U(k, c) for c < R, where every operand of F is read once:
// the two products over F (F x_3 U3^T with K = n3 along contiguous rows, and
// F x_1 U1^T with K = n1 along strided columns) are such "lines" of F.  The
// FP64 pipe bounds it (R FMAs per loaded value), so each lane owns a line and
// all R of its outputs (no tile padding beyond R), and U sits in shared
// memory (read as broadcasts).  The pipe is per SM, so the 32-line tasks are
// dealt to SMs evenly: one CTA per SM, task t to CTA t mod grid, as many warps
// per CTA as there are tasks per SM (up to 32).  Each output is one FMA chain
// in k order.
struct ThinDesc {
  const double* X;
  long long sXl, sXk;  // X(line, k) = X[line sXl + k sXk]
  const double* U;     // K x R row-major
  double* C;
  long long sCl, sCc;  // C(line, c) = C[line sCl + c sCc]
  long long lines;
  int K;
};

template <int R>
__global__ void __launch_bounds__(1024, 1) k_thin_contract(ThinDesc d) {
  TK_PDL_ENTRY();
  extern __shared__ double us[];  // K x R
  for (int e = threadIdx.x; e < d.K * R; e += blockDim.x) us[e] = d.U[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long tasks = (d.lines + 31) >> 5;
  for (long long t = blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5); t < tasks; t += warps) {
    const long long line = t * 32 + lane;
    const bool live = line < d.lines;
    const double* x = d.X + (live ? line : 0) * d.sXl;
    double acc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] = 0.0;
    for (int k = 0; k < d.K; ++k) {
      const double v = __ldg(x + (long long)k * d.sXk);
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] = fma(v, us[k * R + c], acc[c]);
    }
    if (live) {
      double* o = d.C + line * d.sCl;
#pragma unroll
      for (int c = 0; c < R; ++c) o[c * d.sCc] = acc[c];
    }
  }
}

constexpr int kThinMaxR = 16;
constexpr size_t kThinSmemMax = 64 * 1024;

template <int R>
void thin_launch(const ThinDesc& d, int sm_count, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)d.K * R;
  if (smem > 48 * 1024)
    TK_CUDA(cudaFuncSetAttribute(k_thin_contract<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kThinSmemMax));
  const long long tasks = (d.lines + 31) / 32;
  const long long blocks = std::min<long long>(tasks, std::max(sm_count, 1));
  const long long wpb = std::min<long long>((tasks + blocks - 1) / blocks, 32);
  launch_pdl("k_thin_contract", k_thin_contract<R>, dim3((unsigned)blocks), dim3((unsigned)(32 * wpb)), smem, s, d);
}

template <int R = 1>
void thin_dispatch(int r, const ThinDesc& d, int sm_count, cudaStream_t s) {
  if constexpr (R <= kThinMaxR) {
    if (r == R) return thin_launch<R>(d, sm_count, s);
    thin_dispatch<R + 1>(r, d, sm_count, s);
  }
}

bool thin_applies(int K, int r) { return r <= kThinMaxR && sizeof(double) * (size_t)K * r <= kThinSmemMax; }

// G = Y Y^T for the unfolding Y (rows x K, row-major): every entry's sum
// runs over k in the same order, so G is exactly symmetric
void gram_rows(const double* Y, int rows, int K, double* G, cudaStream_t s) {
  GemmDesc g{rows, rows, K, 1, Y, 0, K, 1, Y, 0, 1, K, G, 0, rows, 1};
  gemm_f64(g, s);
}

}  // namespace

void als_f64(const double* F, const int n[3], double* const U[3], const int r[3], int sweeps, double* B,
             double* lam_log, const AlsBuffers& w, int sm_count, cudaStream_t s) {
  const long long n1 = n[0], n2 = n[1], n3 = n[2], r1 = r[0], r2 = r[1], r3 = r[2];
  // T1[i][j][c] = sum_l F[i][j][l] U3[l][c]
  const GemmDesc t1{(int)(n1 * n2), (int)r3, (int)n3, 1, F, 0, n3, 1, U[2], 0, r3, 1, w.T1, 0, r3, 1};
  const bool thin3 = thin_applies((int)n3, (int)r3), thin1 = thin_applies((int)n1, (int)r1);
  auto product3 = [&] {
    if (thin3)
      thin_dispatch((int)r3, ThinDesc{F, n3, 1, U[2], w.T1, r3, 1, n1 * n2, (int)n3}, sm_count, s);
    else
      gemm_f64(t1, s);
  };
  if (sweeps == 0) {  // the core of the given factors: F x_3 U3^T, x_2 U2^T, x_1 U1^T
    product3();
    GemmDesc y1{(int)r2, (int)r3, (int)n2, (int)n1, U[1], 0, 1, r2, w.T1, n2 * r3, r3, 1, w.Y, r2 * r3, r3, 1};
    gemm_f64(y1, s);
    GemmDesc bc{(int)r1, (int)(r2 * r3), (int)n1, 1, U[0], 0, 1, r1, w.Y, 0, r2 * r3, 1, B, 0, r2 * r3, 1};
    gemm_f64(bc, s);
    return;
  }
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    double* lam = lam_log + (size_t)sweep * 3 * kAlsLamStride;
    // mode 1: Y1[i][b][c] = sum_j U2[j][b] T1[i][j][c], unfolded as n1 x (r2 r3)
    product3();
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
    if (thin1) {
      thin_dispatch((int)r1, ThinDesc{F, 1, n2 * n3, U[0], w.W, 1, n2 * n3, n2 * n3, (int)n1}, sm_count, s);
    } else {
      GemmDesc wd{(int)r1, (int)(n2 * n3), (int)n1, 1, U[0], 0, 1, r1, F, 0, n2 * n3, 1, w.W, 0, n2 * n3, 1};
      gemm_f64(wd, s);
    }
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
