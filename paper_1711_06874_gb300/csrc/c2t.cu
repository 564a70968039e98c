// Canonical-to-Tucker (C2T) of Sec. 3.4, FP64: the Tucker approximation of a
// tensor given in the canonical format of Eq. (Can_Contr),
//   A = sum_k c_k u_k^(1) o u_k^(2) o u_k^(3),  U_l = [u_1^(l) .. u_R^(l)] (n_l x R),
// without forming or unfolding A.
//
// Reduced HOSVD (the initial guess).  The factor of mode l is spanned by the
// leading left singular vectors of the side matrix U_l alone; they are taken
// as the leading eigenvectors of U_l U_l^T (n_l x n_l), whose eigenvalues are
// the squared singular values s_k^2 and whose trace is |U_l|_F^2 = sum s_k^2.
// Rank rule: r_l is the smallest r whose discarded tail (sum_{k>=r} s_k^2)^(1/2)
// is at most eps |A| / (3 |c|), so that the RHOSVD bound
// |A - A_r| <= |c| sum_l (sum_{k>=r_l} s_{l,k}^2)^(1/2) gives E <= eps; capped
// at rmax_l, replaced by rfix_l where that is set.  |A|^2 =
// sum_{k,k'} c_k c_k' prod_l (U_l^T U_l)_{k k'}.
//
// Tucker-ALS sweeps.  For mode l (the other two m < q), the single-hole
// tensor A x_m Z_m^T x_q Z_q^T has the mode-l unfolding
//   M = U_l diag(c) (W_m (.) W_q)^T,  W_j = Z_j^T U_j (r_j x R),
// with (W_m (.) W_q)[(a r_q + b), k] = W_m[a][k] W_q[b][k] (the Khatri-Rao
// product, row a r_q + b); Z_l becomes the r_l leading eigenvectors of M M^T
// (the leading left singular vectors of M), and the sum of the r_l leading
// eigenvalues is |B|^2 right after the update.  Modes 1, 2, 3 in order, each
// update using the factors already updated in the sweep.
//
// Core.  B = A x_1 Z_1^T x_2 Z_2^T x_3 Z_3^T = sum_k c_k W_1[:, k] o W_2[:, k] o
// W_3[:, k], formed in the canonical format.
//
// Signs follow the HOSVD's convention (the entry of largest magnitude among
// the first ceil(n/2) of each column is positive).  The eigenvectors come from
// FP64 Grams, so a direction is fixed to about u s_1^2 / (its gap in s^2).
#include <algorithm>
#include <cmath>
#include <vector>

#include "tk_internal.h"

namespace tk {

namespace {

// |A|^2 = sum_{k,k'} c_k c_k' G1 G2 G3 (one CTA; Neumaier sums per thread,
// then a fixed tree).
__global__ void k_cp_norm2(const double* __restrict__ c, const double* __restrict__ G1,
                           const double* __restrict__ G2, const double* __restrict__ G3, int R,
                           double* __restrict__ out) {
  __shared__ double rs[256], rc[256];
  double sm = 0.0, cm = 0.0;
  for (long long e = threadIdx.x; e < (long long)R * R; e += blockDim.x) {
    const int k = (int)(e / R), kk = (int)(e - (long long)k * R);
    const double x = c[k] * c[kk] * G1[e] * G2[e] * G3[e];
    const double t = sm + x;
    cm += (fabs(sm) >= fabs(x)) ? (sm - t) + x : (x - t) + sm;
    sm = t;
  }
  rs[threadIdx.x] = sm;
  rc[threadIdx.x] = cm;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double a = rs[threadIdx.x], ac = rc[threadIdx.x] + rc[threadIdx.x + w];
      const double x = rs[threadIdx.x + w], t = a + x;
      ac += (fabs(a) >= fabs(x)) ? (a - t) + x : (x - t) + a;
      rs[threadIdx.x] = t;
      rc[threadIdx.x] = ac;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = rs[0] + rc[0];
}

// Uc[i][k] = U[i][k] c[k]
__global__ void k_scale_cols(const double* __restrict__ U, const double* __restrict__ c, int n, int R,
                             double* __restrict__ Uc) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * R;
       e += (long long)gridDim.x * blockDim.x)
    Uc[e] = U[e] * c[e % R];
}

// KR[(a rq + b)][k] = Wm[a][k] Wq[b][k]
__global__ void k_khatri_rao(const double* __restrict__ Wm, const double* __restrict__ Wq, int rm, int rq, int R,
                             double* __restrict__ KR) {
  const long long total = (long long)rm * rq * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / R;
    const int k = (int)(e - row * R);
    const int a = (int)(row / rq), b = (int)(row - (long long)a * rq);
    KR[e] = Wm[(size_t)a * R + k] * Wq[(size_t)b * R + k];
  }
}

// B[a][b][d] = sum_k c_k W1[a][k] W2[b][k] W3[d][k], one FMA chain in k order.
__global__ void k_cp_core(const double* __restrict__ c, const double* __restrict__ W1,
                          const double* __restrict__ W2, const double* __restrict__ W3, int r1, int r2, int r3,
                          int R, double* __restrict__ B) {
  const long long total = (long long)r1 * r2 * r3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long long)r2 * r3));
    const int rem = (int)(e - (long long)a * r2 * r3);
    const int b = rem / r3, d = rem - b * r3;
    const double *w1 = W1 + (size_t)a * R, *w2 = W2 + (size_t)b * R, *w3 = W3 + (size_t)d * R;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(c[k] * w1[k], w2[k] * w3[k], s);
    B[e] = s;
  }
}

unsigned blocks_for(long long total) { return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4096)); }

// C = X X^T for X (rows x K, row-major): every entry one k-order chain
void gram_of_rows(const double* X, int rows, int K, double* C, cudaStream_t s) {
  GemmDesc g{rows, rows, K, 1, X, 0, K, 1, X, 0, 1, K, C, 0, rows, 1};
  gemm_f64(g, s);
}

// W = Z^T U (r x R) for Z (n x r) and U (n x R), row-major
void project(const double* Z, const double* U, int n, int r, int R, double* W, cudaStream_t s) {
  GemmDesc g{r, R, n, 1, Z, 0, 1, r, U, 0, R, 1, W, 0, R, 1};
  gemm_f64(g, s);
}

// compensated host sum of x[from .. to)
double host_sum(const double* x, int from, int to) {
  double sm = 0.0, cm = 0.0;
  for (int k = from; k < to; ++k) {
    const double v = std::max(0.0, x[k]);
    const double t = sm + v;
    cm += (std::fabs(sm) >= std::fabs(v)) ? (sm - t) + v : (v - t) + sm;
    sm = t;
  }
  return sm + cm;
}

}  // namespace

tk_result* c2t_solve(tk_ctx* ctx, int R, const double* c, const double* const U[3], const int n[3], double eps,
                     const int rmax_in[3], const int rfix_in[3], int sweeps, double* hist_out, cudaStream_t s) {
  // Eigenpairs: every pair of an n_l x n_l Gram by Jacobi when n_l <= 96 (the
  // spectra of general CP inputs need not decay), else the leading ones by
  // the subspace eigensolver (fast-decaying spectra, as the sinc CP's).
  int nmax = 0, rcap[3], mcap[3], meig[3];
  for (int l = 0; l < 3; ++l) {
    nmax = std::max(nmax, n[l]);
    const int full = std::min(n[l], R);
    rcap[l] = std::min(rmax_in ? rmax_in[l] : full, full);
    mcap[l] = std::min(std::max(rcap[l], (rfix_in && rfix_in[l] > 0) ? std::min(rfix_in[l], full) : 0), 96);
    if (mcap[l] < 1) fail(TK_EINVAL, "c2t: empty rank cap");
    meig[l] = n[l] <= 96 ? n[l] : mcap[l];
  }
  // ---- workspace: Grams U^T U, |A|^2, c (scaled copies), G (n x n), eigen scratch,
  // eigenvectors, eigenvalues, traces, W per mode, Khatri-Rao, unfolding, eigenvalue log
  size_t eig = 0;
  for (int l = 0; l < 3; ++l) eig = std::max(eig, sym_eig_batch_scratch_doubles(n[l], meig[l], 1));
  const size_t RR = (size_t)R * R;
  const size_t sizes[] = {3 * RR,
                          8,
                          (size_t)nmax * R,                       // U diag(c)
                          (size_t)nmax * nmax,                    // G
                          eig,
                          3 * (size_t)nmax * 96,                  // eigenvectors of the side Grams
                          3 * 96 + 8,                             // their eigenvalues, traces
                          3 * (size_t)96 * R};                    // W_l
  size_t need = 0;
  for (size_t z : sizes) need += carve_bytes<double>(std::max<size_t>(z, 1));
  ctx->ws.reserve(need, s);
  Workspace& ws = ctx->ws;
  double* Gam = ws.take<double>(3 * RR);
  double* small = ws.take<double>(8);  // [0] |A|^2
  double* Uc = ws.take<double>((size_t)nmax * R);
  double* G = ws.take<double>((size_t)nmax * nmax);
  double* escr = ws.take<double>(eig);
  double* V = ws.take<double>(3 * (size_t)nmax * 96);
  double* lam = ws.take<double>(3 * 96 + 8);
  double* trace = lam + 3 * 96;  // [3]
  double* Wall = ws.take<double>(3 * (size_t)96 * R);
  double* W[3] = {Wall, Wall + (size_t)96 * R, Wall + 2 * (size_t)96 * R};

  // |A|^2 from the side-matrix Grams
  for (int l = 0; l < 3; ++l) {
    GemmDesc g{R, R, n[l], 1, U[l], 0, 1, R, U[l], 0, R, 1, Gam + l * RR, 0, R, 1};
    gemm_f64(g, s);
  }
  k_cp_norm2<<<1, 256, 0, s>>>(c, Gam, Gam + RR, Gam + 2 * RR, R, small);
  TK_LAUNCH("k_cp_norm2");
  std::vector<double> ch(R);
  double normA2 = 0.0;
  TK_CUDA(cudaMemcpyAsync(ch.data(), c, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(&normA2, small, sizeof(double), cudaMemcpyDeviceToHost, s));

  // ---- reduced HOSVD: leading eigenpairs of U_l U_l^T, rank rule on the host.
  // Above 96 rows the subspace solver runs with 16 pairs, then 48, then the
  // cap, until the rule finds its rank among the pairs computed.
  TK_CUDA(cudaStreamSynchronize(s));
  double cn2 = 0.0;
  for (int k = 0; k < R; ++k) cn2 += ch[k] * ch[k];
  const double cn = std::sqrt(cn2);
  const double tol = cn > 0.0 ? eps * std::sqrt(std::max(normA2, 0.0)) / (3.0 * cn) : 0.0;
  std::vector<double> lh[3];
  int r[3];
  unsigned flags[3] = {0, 0, 0};
  for (int l = 0; l < 3; ++l) {
    const int full = std::min(n[l], R);
    const int need_fix = (rfix_in && rfix_in[l] > 0) ? std::min(rfix_in[l], full) : 0;
    gram_of_rows(U[l], n[l], R, G, s);
    int q = 0;
    const int rounds[3] = {16, 48, 96};
    for (int ri = 0; ri < 3; ++ri) {
      int mr = n[l] <= 96 ? meig[l] : std::min(mcap[l], std::max(rounds[ri], need_fix));
      if (ri > 0 && n[l] > 96 && mr <= meig[l]) continue;  // this round adds no pairs
      meig[l] = mr;
      sym_eig_batch(G, n[l], mr, 1, lam + l * 96, V + (size_t)l * nmax * 96, trace + l, escr, s);
      const int mh = std::min(mr, mcap[l]);
      lh[l].assign(mh, 0.0);
      double total = 0.0;
      TK_CUDA(cudaMemcpyAsync(lh[l].data(), lam + l * 96, sizeof(double) * mh, cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaMemcpyAsync(&total, trace + l, sizeof(double), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      // smallest q >= 1 with (sum_{k>=q} s_k^2)^(1/2) <= tol (q = full keeps
      // everything).  With every eigenvalue computed the tail is the sum of
      // the discarded ones (negative rounding clamped to zero, summed from the
      // smallest); otherwise trace - sum_{k<q} s_k^2.  The Gram's eigenvalues
      // carry rounding of about n u trace (u = 2^-53): a tail at or below
      // that floor cannot be told from zero, so it meets any tolerance, and a
      // tolerance below the floor is flagged as unreachable in FP64.
      const double floor2 = (double)n[l] * 0x1p-53 * total;
      const double thr2 = std::max(tol * tol, floor2);
      if (tol * tol < floor2) flags[l] |= TK_EPS_UNREACHABLE_AT_PRECISION;
      std::vector<double> suffix(mh + 1, 0.0);  // suffix[k] = sum_{j>=k} max(s_j^2, 0)
      for (int k = mh - 1; k >= 0; --k) suffix[k] = suffix[k + 1] + std::max(lh[l][k], 0.0);
      q = 0;
      for (int cand = 1; cand <= mh; ++cand) {
        const double tail =
            mh == n[l] ? suffix[cand] : std::max(0.0, total - host_sum(lh[l].data(), 0, cand));
        if (cand == full || tail <= thr2) {
          q = cand;
          break;
        }
      }
      if (q > 0 || mh >= mcap[l] || n[l] <= 96) break;
    }
    if (q == 0) q = full;  // the rule wants more pairs than the cap allows
    if (q > rcap[l]) {
      flags[l] |= TK_RANK_CAPPED;
      q = rcap[l];
    }
    if (need_fix > 0) q = need_fix;
    r[l] = std::min(q, std::min(meig[l], mcap[l]));
  }
  for (int l = 0; l < 3; ++l)
    if ((long long)r[l] > (long long)r[(l + 1) % 3] * r[(l + 2) % 3])
      fail(TK_EINVAL, "the RHOSVD ranks are not a multilinear rank (r_l > r_m r_q)");

  // the sweeps' buffers, sized by the ranks: Khatri-Rao product, unfolding M,
  // eigenvalue log
  int rmq_max = 1;
  for (int l = 0; l < 3; ++l) rmq_max = std::max(rmq_max, r[(l + 1) % 3] * r[(l + 2) % 3]);
  ctx->ws2.reserve(carve_bytes<double>((size_t)rmq_max * R) + carve_bytes<double>((size_t)nmax * rmq_max) +
                       carve_bytes<double>((size_t)std::max(1, sweeps) * 3 * 96),
                   s);
  double* KR = ctx->ws2.take<double>((size_t)rmq_max * R);
  double* M = ctx->ws2.take<double>((size_t)nmax * rmq_max);
  double* lamlog = ctx->ws2.take<double>((size_t)std::max(1, sweeps) * 3 * 96);

  tk_result* res = new tk_result();
  try {
    res->ctx = ctx;
    res->precision = TK_FP64;
    res->normF2 = normA2;
    for (int l = 0; l < 3; ++l) {
      res->n[l] = n[l];
      res->r[l] = r[l];
      res->m[l] = r[l];
      res->flags[l] = flags[l];
      TK_CUDA(cudaMalloc(&res->U[l], sizeof(double) * (size_t)n[l] * r[l]));
      // Z_l = the first r_l eigenvectors (n_l x mcap_l -> n_l x r_l)
      TK_CUDA(cudaMemcpy2DAsync(res->U[l], sizeof(double) * r[l], V + (size_t)l * nmax * 96,
                                sizeof(double) * meig[l], sizeof(double) * r[l], n[l], cudaMemcpyDeviceToDevice, s));
      res->lam[l].assign(lh[l].begin(), lh[l].begin() + r[l]);
    }
    TK_CUDA(cudaMalloc(&res->core, sizeof(double) * (size_t)r[0] * r[1] * r[2]));
    for (int l = 0; l < 3; ++l) project(res->U[l], U[l], n[l], r[l], R, W[l], s);

    // ---- Tucker-ALS sweeps in the canonical format
    for (int sw = 0; sw < sweeps; ++sw) {
      for (int l = 0; l < 3; ++l) {
        const int m = (l == 0) ? 1 : 0, q = (l == 2) ? 1 : 2;
        const int rmq = r[m] * r[q];
        k_scale_cols<<<blocks_for((long long)n[l] * R), 256, 0, s>>>(U[l], c, n[l], R, Uc);
        TK_LAUNCH("k_scale_cols");
        k_khatri_rao<<<blocks_for((long long)rmq * R), 256, 0, s>>>(W[m], W[q], r[m], r[q], R, KR);
        TK_LAUNCH("k_khatri_rao");
        // M = U_l diag(c) KR^T (n_l x r_m r_q)
        GemmDesc md{n[l], rmq, R, 1, Uc, 0, R, 1, KR, 0, 1, R, M, 0, rmq, 1};
        gemm_f64(md, s);
        gram_of_rows(M, n[l], rmq, G, s);
        double* lrec = lamlog + ((size_t)sw * 3 + l) * 96;
        const int me = n[l] <= 96 ? n[l] : r[l];
        if (me == r[l]) {
          sym_eig_batch(G, n[l], r[l], 1, lrec, res->U[l], trace, escr, s);
        } else {
          sym_eig_batch(G, n[l], me, 1, lrec, V, trace, escr, s);
          TK_CUDA(cudaMemcpy2DAsync(res->U[l], sizeof(double) * r[l], V, sizeof(double) * me,
                                    sizeof(double) * r[l], n[l], cudaMemcpyDeviceToDevice, s));
        }
        project(res->U[l], U[l], n[l], r[l], R, W[l], s);
      }
    }
    k_cp_core<<<blocks_for((long long)r[0] * r[1] * r[2]), 256, 0, s>>>(c, W[0], W[1], W[2], r[0], r[1], r[2], R,
                                                                         res->core);
    TK_LAUNCH("k_cp_core");
    if (sweeps > 0) {
      std::vector<double> lg((size_t)sweeps * 3 * 96);
      TK_CUDA(cudaMemcpyAsync(lg.data(), lamlog, sizeof(double) * lg.size(), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      for (int sw = 0; sw < sweeps; ++sw)
        for (int l = 0; l < 3; ++l) {
          const double* x = lg.data() + ((size_t)sw * 3 + l) * 96;
          if (hist_out) hist_out[sw * 3 + l] = host_sum(x, 0, r[l]);
          if (sw == sweeps - 1) res->lam[l].assign(x, x + r[l]);
        }
    }
    TK_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tk_result_free(res);
    throw;
  }
  return res;
}

}  // namespace tk
