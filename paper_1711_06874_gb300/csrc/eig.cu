// (c) Leading eigenpairs of the Gram matrices and the rank decision, FP64.
//
// Sec. 3.2 takes the leading left singular vectors of each unfolding A_(k);
// they are the leading eigenvectors of G_k = A_(k) A_(k)^T.  Only the first
// r_k <= rmax are used, and G_k has a geometrically decaying spectrum, so the
// solver works on an m-dimensional dominant subspace, m = rank cap + margin:
//   Y = G Omega (Omega from a counter-based hash), Q = qr(Y), repeated once
//   more with Y = G Q (subspace iteration), then the Rayleigh-Ritz matrix
//   H = Q^T G Q is diagonalised by cyclic Jacobi rotations (parallel
//   round-robin ordering, one CTA, shared memory) and the Ritz vectors are
//   U = Q V_H.  When m equals n the Jacobi method runs on G itself.
// All arithmetic is FP64.  Eigenvectors get the sign convention: the entry of
// largest magnitude among the first ceil(n/2) is positive (lowest index on an
// exact tie).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>

#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kMaxM = 96;  // largest Jacobi problem held in shared memory

// ---------------------------------------------------------------------------
// Counter-based pseudo-random start block: splitmix64 of (seed, index).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hash_uniform(unsigned long long seed, unsigned long long idx) {
  unsigned long long z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

__global__ void k_random(double* X, long long len, unsigned long long seed) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x)
    X[t] = hash_uniform(seed, (unsigned long long)t);
}

// The same start block (len_per values) for each of B instances.
__global__ void k_random_rep(double* X, long long len_per, int B, unsigned long long seed) {
  const long long len = len_per * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x)
    X[t] = hash_uniform(seed, (unsigned long long)(t % len_per));
}

// ---------------------------------------------------------------------------
// Householder QR of a column-major n x m block Y (ld = n) in one CTA; writes
// the explicit orthonormal factor Q (column-major, ld = n).  Y is destroyed.
// ---------------------------------------------------------------------------
// Sum over the block, the same value in every thread: warp sums, then warp 0
// adds the warp partials in a fixed tree and broadcasts through red[32].
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Householder QR of a column-major n x m panel Y in shared memory, with the
// explicit orthonormal factor Q (n x m, same layout) written to Qs.  In step
// j, H_j = I - beta v v^T with v = x + sign(x_0) |x| e_0, beta = 2 / v^T v,
// is applied to the columns right of j.  Warp 0 alone (all 32 lanes) updates
// column j + 1 and takes its new squared norm and reflector scalars, the
// critical path of the next step; the other warps update columns j + 2 on in
// groups of eight lanes (four columns per warp).  One barrier per step.
template <class T>
__device__ __forceinline__ void reflector(T alpha2, T x0, T& v0, T& beta) {
  if (!(alpha2 > T(0))) {
    v0 = x0;
    beta = T(0);
    return;
  }
  const T alpha = sqrt(alpha2);
  // v0 = x0 + sign(x0) alpha (the sign from the bit pattern), and
  // 2 / (alpha^2 - x0^2 + v0^2) = 1 / (alpha (alpha + |x0|)) exactly: fewer
  // FP64 instructions, no cancellation either way
  const bool neg = sizeof(T) == 8 ? (__double_as_longlong((double)x0) < 0) : (__float_as_int((float)x0) < 0);
  v0 = x0 + (neg ? -alpha : alpha);
  beta = T(1) / (alpha * (alpha + (neg ? -x0 : x0)));
}

template <class T>
__device__ __forceinline__ T group_sum8(T d) {
  d += __shfl_xor_sync(0xffffffffu, d, 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

template <class T>
__device__ __forceinline__ T warp_sum32(T d) {
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  return d;
}

template <class T>
__device__ void qr_panel(T* Y, T* Qs, int n, int m, T* beta, T* v0s) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gsub = lane >> 3, l8 = lane & 7;
  // reflector of column 0
  if (w == 0) {
    T s2 = T(0);
    for (int i = lane; i < n; i += 32) s2 += Y[i] * Y[i];
    s2 = warp_sum32(s2);
    if (lane == 0) reflector(s2, Y[0], v0s[0], beta[0]);
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const T* y = Y + (long long)j * n;
    const T v0 = v0s[j], bj = beta[j];
    if (w == 0) {
      if (j + 1 < m) {
        T* xc = Y + (long long)(j + 1) * n;
        T d = T(0);
        if (bj != T(0)) {
          if (lane == 0) d = v0 * xc[j];
          for (int i = j + 1 + lane; i < n; i += 32) d += y[i] * xc[i];
        }
        d = warp_sum32(d);
        const T f = bj * d;
        T s2 = T(0);
        if (f != T(0)) {
          if (lane == 0) xc[j] -= f * v0;
          for (int i = j + 1 + lane; i < n; i += 32) {
            const T x = xc[i] - f * y[i];
            xc[i] = x;
            s2 += x * x;
          }
        } else {
          for (int i = j + 1 + lane; i < n; i += 32) s2 += xc[i] * xc[i];
        }
        s2 = warp_sum32(s2);
        if (lane == 0) reflector(s2, xc[j + 1], v0s[j + 1], beta[j + 1]);
      }
    } else if (bj != T(0)) {
      for (int cb = j + 2 + 4 * (w - 1); cb < m; cb += 4 * (nw - 1)) {
        const int c = cb + gsub;
        const bool act = c < m;
        T* xc = Y + (long long)(act ? c : j) * n;  // an idle group reads column j (read-only here)
        T d = T(0);
        if (act) {
          if (l8 == 0) d = v0 * xc[j];
          for (int i = j + 1 + l8; i < n; i += 8) d += y[i] * xc[i];
        }
        d = group_sum8(d);
        const T f = bj * d;
        if (act && f != T(0)) {
          if (l8 == 0) xc[j] -= f * v0;
          for (int i = j + 1 + l8; i < n; i += 8) xc[i] -= f * y[i];
        }
      }
    }
    if (threadIdx.x == 0) Y[(long long)j * n + j] = v0;  // head of v_j, read in the Q phase
    __syncthreads();
  }
  // Q = H_0 ... H_{m-1} [I; 0], applied from the right end
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    Qs[e] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    const T bj = beta[j];
    const T* v = Y + (long long)j * n;
    if (bj != T(0)) {
      for (int cb = j + 4 * w; cb < m; cb += 4 * nw) {
        const int c = cb + gsub;
        const bool act = c < m;
        T* qc = Qs + (long long)(act ? c : j) * n;
        T d = T(0);
        if (act)
          for (int i = j + l8; i < n; i += 8) d += v[i] * qc[i];
        d = group_sum8(d);
        const T f = bj * d;
        if (act)
          for (int i = j + l8; i < n; i += 8) qc[i] -= f * v[i];
      }
    }
    __syncthreads();
  }
}

// Householder factorisation of a panel of at most 256 rows held in shared
// memory (column stride ld), FP64 for the subspace pass and FP32 for the
// start.  An FP64 warp instruction occupies a sub-partition's FP64 unit for
// about 64 cycles whatever the number of active lanes, so each step's
// critical path (column j + 1, warp 0) keeps its rows in registers
// (kRPL = ceil(n / 32) per lane) and carries no tests; the other warps take
// the columns j + 2 on in groups of eight lanes.  ld is padded so that the
// four groups of a warp read different shared-memory banks.  On return Y
// holds the reflectors (v_j in rows j.. of column j, head included) and
// betas[j] their scalars.
template <class T, int kRPL>
__device__ void qr_factor_reg(T* Y, int ld, int n, int m, T* betas, T* beta, T* v0s) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (w == 0) {
    T s2 = T(0);
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      const int i = lane + 32 * t;
      const T x = (i < n) ? Y[i] : T(0);
      s2 = fma(x, x, s2);
    }
    s2 = warp_sum32(s2);
    if (lane == 0) reflector(s2, Y[0], v0s[0], beta[0]);
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const T* y = Y + (long long)j * ld;
    const T v0 = v0s[j], bj = beta[j];
    if (w == 0) {
      if (j + 1 < m) {
        T* xc = Y + (long long)(j + 1) * ld;
        T yv[kRPL], xv[kRPL];
#pragma unroll
        for (int t = 0; t < kRPL; ++t) {
          const int i = j + 1 + lane + 32 * t;
          yv[t] = (i < n) ? y[i] : T(0);
          xv[t] = (i < n) ? xc[i] : T(0);
        }
        const T head = (lane == 0) ? xc[j] : T(0);
        T d = v0 * head;
#pragma unroll
        for (int t = 0; t < kRPL; ++t) d = fma(yv[t], xv[t], d);
        d = warp_sum32(d);
        const T f = bj * d;
        if (lane == 0) xc[j] = fma(-f, v0, head);
        T s2 = T(0);
#pragma unroll
        for (int t = 0; t < kRPL; ++t) {
          const int i = j + 1 + lane + 32 * t;
          xv[t] = fma(-f, yv[t], xv[t]);
          s2 = fma(xv[t], xv[t], s2);
          if (i < n) xc[i] = xv[t];
        }
        s2 = warp_sum32(s2);
        if (lane == 0) reflector(s2, xv[0], v0s[j + 1], beta[j + 1]);  // xv[0] of lane 0: row j + 1
      }
    } else {
      // Columns j + 2 on: groups of kL lanes, one column each.  FP64 takes
      // 16-lane groups (22 FP64 instructions a warp for two columns, where
      // 8-lane groups take 37 for four) and fills the warps sharing warp 0's
      // sub-partition last: the FP64 unit of a sub-partition issues one warp
      // instruction about every 64 cycles, and warp 0's chain is the critical
      // path.  FP32 keeps 8-lane groups.
      constexpr int kL = sizeof(T) == 8 ? 16 : 8;  // lanes per column
      constexpr int kGpw = 32 / kL;                 // columns per warp and round
      constexpr int kGr = 32 * kRPL / kL;           // rows per lane
      const int gq = lane / kL, lq = lane % kL;
      const int ntw = nw - 1;
      int tw = w - 1;
      if (sizeof(T) == 8) tw = (w & 3) ? w - 1 - (w >> 2) : (ntw - (ntw >> 2)) + (w >> 2) - 1;
      for (int cb = j + 2 + kGpw * tw; cb < m; cb += kGpw * ntw) {
        const int c = cb + gq;
        const bool act = c < m;
        T* xc = Y + (long long)(act ? c : j) * ld;  // an idle group reads column j (read-only here)
        T yv[kGr], xv[kGr];
#pragma unroll
        for (int t = 0; t < kGr; ++t) {
          const int i = j + 1 + lq + kL * t;
          const bool in = act && i < n;
          yv[t] = in ? y[i] : T(0);
          xv[t] = in ? xc[i] : T(0);
        }
        const T head = (act && lq == 0) ? xc[j] : T(0);
        T d = v0 * head;
#pragma unroll
        for (int t = 0; t < kGr; ++t) d = fma(yv[t], xv[t], d);
#pragma unroll
        for (int o = kL / 2; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const T f = bj * d;
        if (act) {
          if (lq == 0) xc[j] = fma(-f, v0, head);
#pragma unroll
          for (int t = 0; t < kGr; ++t) {
            const int i = j + 1 + lq + kL * t;
            if (i < n) xc[i] = fma(-f, yv[t], xv[t]);
          }
        }
      }
    }
    if (threadIdx.x == 0) Y[(long long)j * ld + j] = v0;  // head of v_j
    __syncthreads();
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) betas[j] = beta[j];
}

// Column stride of a panel in shared memory: a group of eight lanes reads
// 8 consecutive entries, and the four groups of a warp read four columns.
template <class T>
__host__ __device__ constexpr int panel_ld(int n) {
  return sizeof(T) == 8 ? n + ((8 - n % 16) + 16) % 16 : n + ((8 - n % 32) + 32) % 32;
}

// One panel per CTA: Y + b sY (n x m, column-major) in shared memory,
// reflectors written back in place, scalars to betas + b sB.
template <int kRPL>
__global__ void __launch_bounds__(256) k_qr_factor64(double* Y, double* betas, int n, int m, long long sY, long long sB) {
  TK_PDL_ENTRY();
  TK_PDL_EARLY_IF_SMALL();
  extern __shared__ double qf_sm[];
  __shared__ double beta[kMaxM + 1];
  __shared__ double v0s[kMaxM + 1];
  Y += blockIdx.x * sY;
  betas += blockIdx.x * sB;
  const int ld = panel_ld<double>(n);
  {
    // eight loads in flight per thread
    const int tot = n * m, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * nt) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (e0 + u * nt < tot) ? Y[e0 + u * nt] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nt;
        if (e < tot) qf_sm[(e / n) * ld + e % n] = v[u];
      }
    }
  }
  __syncthreads();
  qr_factor_reg<double, kRPL>(qf_sm, ld, n, m, betas, beta, v0s);
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) Y[e] = qf_sm[(e / n) * ld + e % n];
}

// Q = H_0 ... H_{m-1} [I; 0] column by column: column c is H_0 ... H_c e_c
// (H_j e_c = e_c for j > c), one CTA per column, so the columns run on
// separate SMs with no barrier between reflectors: the CTA's four warps stage
// the reflectors 0 .. c in shared memory (rows above each head zeroed) and
// warp 0 alone applies them (a second warp on the SM would share the FP64
// issue the chain waits on).  Instance blockIdx.y.
template <int kRPL>
__global__ void __launch_bounds__(128) k_form_q(const double* __restrict__ Y, const double* __restrict__ betas,
                                                 double* __restrict__ Q, int n, int m, long long sY, long long sB,
                                                 long long sQ) {
  TK_PDL_ENTRY();
  TK_PDL_EARLY_IF_SMALL();
  extern __shared__ double fq_sm[];
  __shared__ double bs[kMaxM + 1];
  Y += blockIdx.y * sY;
  betas += blockIdx.y * sB;
  Q += blockIdx.y * sQ;
  const int cmax = blockIdx.x;
  {
    // eight loads in flight per thread
    const int tot = (cmax + 1) * n, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * nt) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (e0 + u * nt < tot) ? Y[e0 + u * nt] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nt;
        if (e < tot) fq_sm[e] = (e % n >= e / n) ? v[u] : 0.0;
      }
    }
  }
  for (int j = threadIdx.x; j <= cmax; j += blockDim.x) bs[j] = betas[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, c = cmax;
  if (threadIdx.x >= 32) return;
  double q[kRPL];
#pragma unroll
  for (int t = 0; t < kRPL; ++t) q[t] = (lane + 32 * t == c) ? 1.0 : 0.0;
  for (int j = c; j >= 0; --j) {
    const double* v = fq_sm + (long long)j * n;
    double vv[kRPL];
    double d = 0.0;
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      const int i = lane + 32 * t;
      vv[t] = (i < n) ? v[i] : 0.0;
      d = fma(vv[t], q[t], d);
    }
    d = warp_sum32(d);
    const double f = bs[j] * d;
#pragma unroll
    for (int t = 0; t < kRPL; ++t) q[t] = fma(-f, vv[t], q[t]);
  }
#pragma unroll
  for (int t = 0; t < kRPL; ++t) {
    const int i = lane + 32 * t;
    if (i < n) Q[(long long)c * n + i] = q[t];
  }
}

// Factorisation and factor of B panels (n x m at Y + b n m), the scalars in
// betas + b sB, Q at Q + b n m; false when the shape is outside these kernels.
template <int kRPL>
void qr64_launch(double* Y, double* betas, double* Q, int n, int m, int B, long long sB, cudaStream_t s) {
  const size_t f_smem = sizeof(double) * (size_t)panel_ld<double>(n) * m;
  const size_t q_smem = sizeof(double) * (size_t)n * m;
  once_per_device((const void*)&k_qr_factor64<kRPL>, [] {
    TK_CUDA(cudaFuncSetAttribute(k_qr_factor64<kRPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    TK_CUDA(cudaFuncSetAttribute(k_form_q<kRPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  launch_pdl("k_qr_factor64", k_qr_factor64<kRPL>, dim3(B), dim3(256), f_smem, s, Y, betas, n, m, (long long)n * m, sB);
  launch_pdl("k_form_q", k_form_q<kRPL>, dim3(m, B), dim3(128), q_smem, s, Y, betas, Q, n, m,
             (long long)n * m, sB,
                                                           (long long)n * m);
}

bool qr64_batch(double* Y, double* betas, double* Q, int n, int m, int B, long long sB, cudaStream_t s) {
  if (n > 256 || sizeof(double) * (size_t)panel_ld<double>(n) * m > 200 * 1024) return false;
  switch ((n + 31) / 32) {
    case 1: qr64_launch<1>(Y, betas, Q, n, m, B, sB, s); return true;
    case 2: qr64_launch<2>(Y, betas, Q, n, m, B, sB, s); return true;
    case 3: qr64_launch<3>(Y, betas, Q, n, m, B, sB, s); return true;
    case 4: qr64_launch<4>(Y, betas, Q, n, m, B, sB, s); return true;
    case 5: qr64_launch<5>(Y, betas, Q, n, m, B, sB, s); return true;
    case 6: qr64_launch<6>(Y, betas, Q, n, m, B, sB, s); return true;
    case 7: qr64_launch<7>(Y, betas, Q, n, m, B, sB, s); return true;
    case 8: qr64_launch<8>(Y, betas, Q, n, m, B, sB, s); return true;
    default: return false;
  }
}

// The panel Y (n x m) and the factor Q live in shared memory when 2 n m
// doubles fit (otherwise in global memory).
struct QrProb {
  double* Y;
  double* Q;
  int n, m;
};
struct QrBatch {
  QrProb p[2];  // one problem per CTA
};

template <bool kShared>
__device__ void qr_body(double* Yg, double* Qg, int n, int m) {
  extern __shared__ double qr_sm[];
  __shared__ double beta[kMaxM + 1];
  __shared__ double v0s[kMaxM + 1];
  double* Y = kShared ? qr_sm : Yg;
  double* Q = kShared ? qr_sm + (size_t)n * m : Qg;
  if (kShared) {
    // eight loads in flight per thread
    const int tot = n * m, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * nt) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (e0 + u * nt < tot) ? Yg[e0 + u * nt] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u * nt < tot) Y[e0 + u * nt] = v[u];
    }
    __syncthreads();
  }
  qr_panel<double>(Y, Q, n, m, beta, v0s);
  if (kShared)
    for (int e = threadIdx.x; e < n * m; e += blockDim.x) Qg[e] = Q[e];
}

template <bool kShared>
__global__ void __launch_bounds__(1024) k_householder_qr(QrBatch batch) {
  qr_body<kShared>(batch.p[blockIdx.x].Y, batch.p[blockIdx.x].Q, batch.p[blockIdx.x].n, batch.p[blockIdx.x].m);
}

// One problem per CTA at Y + b * stride, Q + b * stride (uniform sizes).
template <bool kShared>
__global__ void __launch_bounds__(1024) k_householder_qr_strided(double* Y, double* Q, int n, int m, long long stride) {
  qr_body<kShared>(Y + blockIdx.x * stride, Q + blockIdx.x * stride, n, m);
}

// Trace of the n x n matrix G by one warp: Neumaier pairs per lane over a
// fixed stride, then a fixed shuffle tree; lane 0 holds the result.
__device__ __forceinline__ double trace_warp(const double* G, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0, c = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double x = G[(long long)i * n + i];
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, s, o);
    const double xc = __shfl_xor_sync(0xffffffffu, c, o);
    const double t = s + x;
    c += ((fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s) + xc;
    s = t;
  }
  return s + c;
}

// trace of G + blockIdx.x n^2 (instance of a batch), one warp per instance.
__global__ void k_trace(const double* G, int n, double* out) {
  const double t = trace_warp(G + (size_t)blockIdx.x * n * n, n);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// First pass of the subspace iteration in FP32 (one CTA per instance): G is
// rounded to FP32 in shared memory, Y = G Omega (Omega from the hash, the
// same start block for every instance), and Y's Householder QR in FP32 gives
// the start block Q0 (written in FP64, column-major n x ms) of the FP64 pass.
// Only its span matters, and the FP64 pass that follows fixes its accuracy.
// ---------------------------------------------------------------------------
// Bit-level tests and conversions on the ALU pipes: GB300 spends about 64
// sub-partition cycles on every FP64 warp instruction, compares included.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// Monotone integer key of a double (non-NaN): larger value, larger key.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}
// x 2^-e as a float, truncated (steering only; zero below the float range).
__device__ __forceinline__ float scaled_float(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int fe = ex - 1023 - e + 127;
  if (ex == 0 || fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
}
// A normal float (or zero) as the equal double.
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(ex - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
size_t start32_smem(int n, int ms) { return sizeof(float) * (size_t)panel_ld<float>(n) * ms; }

// FP64 -> FP32 by the bit pattern (truncated; zero below the FP32 range,
// which holds every entry of a Gram matrix of FP32-range data): the start only
// needs an approximation of G, and the conversion stays off the FP64 pipe.
__device__ __forceinline__ float double_to_float_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int fe = ex - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
}

// Uniform in [-1, 1) from the counter-based hash, in FP32.
__device__ __forceinline__ float hash_uniform_f(unsigned long long seed, unsigned long long idx) {
  unsigned long long z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(unsigned)(z >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

// Y = G Omega in FP32 for the rows [8 blockIdx.x, +8) of instance
// blockIdx.y, G converted by its bits and Omega drawn from the counter-based
// hash; G is symmetric, so Y(i, c) = sum_k G(i, k) Omega(k, c), each output
// one FMA chain in k order.  Block 0 also writes the trace of G when trace is
// given.  Y goes to Yg [b][c][i] (ld n).  Many CTAs share the product, so
// reading G is no longer one SM's job.
constexpr int kGoRows = 8;

size_t gomega32_smem(int n, int ms) {
  return sizeof(float) * ((size_t)kGoRows * n + (size_t)n * ((ms + 3) & ~3));
}

__global__ void __launch_bounds__(256) k_gomega32(const double* __restrict__ G, int n, int ms,
                                                  unsigned long long seed, float* __restrict__ Yg,
                                                  double* __restrict__ trace) {
  TK_PDL_ENTRY();
  TK_PDL_EARLY_IF_SMALL();
  extern __shared__ float so[];
  const int ms4 = (ms + 3) & ~3;
  float* Gr = so;               // rows i0 .. i0 + 7 of G
  float* W = so + kGoRows * n;  // Omega [k][c], stride ms4
  const int b = blockIdx.y, i0 = blockIdx.x * kGoRows;
  const int rows = min(kGoRows, n - i0);
  G += (size_t)b * n * n;
  if (trace != nullptr && blockIdx.x == 0 && threadIdx.x < 32) {
    const double t = trace_warp(G, n);
    if (threadIdx.x == 0) trace[b] = t;
  }
  const double* Gi = G + (size_t)i0 * n;  // the rows are contiguous
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) Gr[e] = double_to_float_trunc(__ldg(Gi + e));
  for (int e = threadIdx.x; e < n * ms4; e += blockDim.x) {
    const int k = e / ms4, c = e - k * ms4;
    W[e] = (c < ms) ? hash_uniform_f(seed, (unsigned long long)c * n + k) : 0.0f;
  }
  __syncthreads();
  // warp r takes row i0 + r; lane l column c = 16 cg + (l & 15) over the k of
  // parity l >> 4, and the two halves meet by a shuffle
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = w; r < rows; r += nw) {
    const float* g = Gr + (size_t)r * n;
    for (int c0 = 0; c0 < ms; c0 += 16) {
      const int c = c0 + (lane & 15);
      const float* wc = W + min(c, ms4 - 1);
      float acc = 0.0f;
#pragma unroll 8
      for (int k = lane >> 4; k < n; k += 2) acc = fmaf(g[k], wc[(size_t)k * ms4], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 16);
      if (lane < 16 && c < ms) Yg[((size_t)b * ms + c) * n + i0 + r] = acc;
    }
  }
}

// The FP32 start block from Y = G Omega (k_gomega32): Householder
// factorisation in registers (as the FP64 pass) and the factor Q formed one
// warp per column (Q e_c = H_0 ... H_c e_c, no barrier between reflectors);
// Q goes out in FP64.
template <int kRPL>
__global__ void __launch_bounds__(256) k_start32(const float* __restrict__ Yg, int n, int ms,
                                                 double* __restrict__ Q0) {
  TK_PDL_ENTRY();
  TK_PDL_EARLY_IF_SMALL();
  extern __shared__ float s32[];
  __shared__ float beta[kMaxM + 1];
  __shared__ float v0s[kMaxM + 1];
  __shared__ float bsm[kMaxM + 1];
  const int ld = panel_ld<float>(n);
  float* Y = s32;  // n x ms, column-major, stride ld
  Yg += (size_t)blockIdx.x * ms * n;
  Q0 += (size_t)blockIdx.x * n * ms;
  {
    // eight loads in flight per thread
    const int tot = n * ms, nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * nt) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (e0 + u * nt < tot) ? Yg[e0 + u * nt] : 0.0f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nt;
        if (e < tot) Y[(size_t)(e / n) * ld + e % n] = v[u];
      }
    }
  }
  __syncthreads();
  qr_factor_reg<float, kRPL>(Y, ld, n, ms, bsm, beta, v0s);
  __syncthreads();
  // Q e_c = H_0 ... H_c e_c (rows above each head are 0): warp w forms the
  // columns c1 = c and c2 = c + nw together, two independent chains
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c1 = threadIdx.x >> 5; c1 < ms; c1 += 2 * nw) {
    const int c2 = c1 + nw;
    const bool two = c2 < ms;
    const int ctop = two ? c2 : c1;
    float q1[kRPL], q2[kRPL];
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      q1[t] = (lane + 32 * t == c1) ? 1.0f : 0.0f;
      q2[t] = (lane + 32 * t == c2) ? 1.0f : 0.0f;
    }
    for (int j = ctop; j >= 0; --j) {
      const float* v = Y + (long long)j * ld;
      float vv[kRPL];
      float d1 = 0.0f, d2 = 0.0f;
#pragma unroll
      for (int t = 0; t < kRPL; ++t) {
        const int i = lane + 32 * t;
        vv[t] = (i < n && i >= j) ? v[i] : 0.0f;
        d1 = fmaf(vv[t], q1[t], d1);
        d2 = fmaf(vv[t], q2[t], d2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      }
      // H_j acts on column c only for j <= c (uniform across the warp)
      const float f1 = j <= c1 ? bsm[j] * d1 : 0.0f, f2 = bsm[j] * d2;
#pragma unroll
      for (int t = 0; t < kRPL; ++t) {
        q1[t] = fmaf(-f1, vv[t], q1[t]);
        q2[t] = fmaf(-f2, vv[t], q2[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      const int i = lane + 32 * t;
      if (i < n) {
        Q0[(long long)c1 * n + i] = float_to_double_bits(q1[t]);
        if (two) Q0[(long long)c2 * n + i] = float_to_double_bits(q2[t]);
      }
    }
  }
}

// k_start32 for n <= 256 (kRPL = ceil(n / 32)).
void start32_launch(const double* G, int n, int ms, int B, unsigned long long seed, double* Q0, double* trace,
                    float* Yscr, cudaStream_t s) {
  once_per_device((const void*)&k_gomega32, [] {
    TK_CUDA(cudaFuncSetAttribute(k_gomega32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  launch_pdl("k_gomega32", k_gomega32, dim3((n + kGoRows - 1) / kGoRows, B), dim3(256), gomega32_smem(n, ms), s, G, n,
             ms, seed, Yscr, trace);
  const size_t smem = start32_smem(n, ms);
  switch ((n + 31) / 32) {
#define TK_START32_CASE(K)                                                                                   \
  case K:                                                                                                    \
    once_per_device((const void*)&k_start32<K>, [] {                                                         \
      TK_CUDA(cudaFuncSetAttribute(k_start32<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)); \
    });                                                                                                      \
    launch_pdl("k_start32", k_start32<K>, dim3(B), dim3(256), smem, s, Yscr, n, ms, Q0);                      \
    break;
    TK_START32_CASE(1)
    TK_START32_CASE(2)
    TK_START32_CASE(3)
    TK_START32_CASE(4)
    TK_START32_CASE(5)
    TK_START32_CASE(6)
    TK_START32_CASE(7)
    TK_START32_CASE(8)
#undef TK_START32_CASE
    default:
      fail(TK_EINVAL, "start32: n out of range");
  }
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi on a symmetric m x m matrix (row-major, ld = m) in one CTA.
// Parallel ordering: the circle method pairs the mp (even) indices into
// mp/2 disjoint planes per step, mp - 1 steps per sweep; each step applies
// the mp/2 rotations to rows, then to columns and to V.  A rotation is skipped
// when |a_pq| <= 2^-53 |A|_F, below the rounding of the FP64 matrix itself,
// or when both diagonal entries are below 64 u |A|_F (a plane inside the
// rounding-noise block, whose vectors the matrix does not determine; its
// trace is kept).  Before each sweep one pass over the upper triangle checks
// whether any plane still needs a rotation; sweeps stop when none does (or
// when a sweep applied none).
// Output: lam (descending) and V (row-major m x m, eigenvectors as columns).
// ---------------------------------------------------------------------------
struct JacProb {
  const double* H;
  int m;
  double* lam;
  double* V;
  int* sweeps;
};
struct JacBatch {
  JacProb p[2];  // one problem per CTA
};

// FP64 (c, s) with c^2 + s^2 = 1 to FP64 rounding from an FP32 rotation
// (cf, sf): with delta = cf^2 + sf^2 - 1 (|delta| < 2^-21), c = cf (1 - kappa),
// s = sf (1 - kappa), kappa = delta/2 - 3 delta^2/8 (the next term of
// (1 + delta)^(-1/2) is below 2^-62).  delta and kappa are formed exactly
// enough in float pairs (exact products, Knuth's two-sum), leaving two FP64
// fused multiply-adds per value.
__device__ __forceinline__ void exact_rotation(float cf, float sf, double& c, double& s) {
  const float p1 = cf * cf, e1 = fmaf(cf, cf, -p1);
  const float p2 = sf * sf, e2 = fmaf(sf, sf, -p2);
  float sg, tg;
  two_sum_f(p1, p2, sg, tg);
  const float dh = sg - 1.0f;  // exact: sg lies within a factor 2 of 1
  float u1, u2, w1, w2, dhi, dlo;
  two_sum_f(tg, e1, u1, u2);
  two_sum_f(u1, e2, w1, w2);
  two_sum_f(dh, w1, dhi, dlo);
  dlo += u2 + w2;
  const float khi = 0.5f * dhi;
  const float klo = fmaf(-0.375f * dhi, dhi, 0.5f * dlo);
  const double c0 = float_to_double_bits(cf), s0 = float_to_double_bits(sf);
  // kappa = khi + klo in FP64 (exact while the two lie within 29 binary
  // places of each other, and below 2^-53 kappa off otherwise): three FP64
  // instructions for the pair, one rounding each
  const double kappa = float_to_double_bits(khi) + float_to_double_bits(klo);
  c = fma(-c0, kappa, c0);
  s = fma(-s0, kappa, s0);
}

// Named CTA barriers (PTX bar.sync / bar.arrive): the count is in threads, a
// multiple of 32, and every lane of a warp executes the instruction.
__device__ __forceinline__ void bar_sync_n(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

constexpr int kJacobiThreads = 256;  // warps 0..3 rotate A, warps 4..7 update V

// Rotation (c, s) of the plane with entries a_pp, a_qq, a_pq (c = 1, s = 0
// below the thresholds); true when it rotates.
__device__ __forceinline__ bool plane_rotation(double app, double aqq, double apq, unsigned long long tau_b,
                                               unsigned long long noise_b, double& c, double& s) {
  c = 1.0;
  s = 0.0;
  // two indices whose diagonals both lie in the rounding noise of the matrix
  // are left alone: their eigenvectors carry no information
  const bool noise = abs_bits(app) <= noise_b && abs_bits(aqq) <= noise_b;
  if (abs_bits(apq) <= tau_b || noise) return false;
  // The angle only steers convergence, so it is taken in FP32 from
  // (a_qq - a_pp) and a_pq scaled by 2^-e (e the exponent of a_pq); (c, s)
  // are then made orthonormal to FP64 precision, so the rotation applied is
  // exactly orthogonal.
  const int e = (int)((abs_bits(apq) >> 52) & 0x7FF) - 1023;
  // (fast approximate quotients: the angle only has to be close)
  const float theta = __fdividef(scaled_float(aqq - app, e), 2.0f * scaled_float(apq, e));
  // |theta| <= |A|_F / (u_data |A|_F) < 2^53, so 1 + theta^2 stays finite
  const float w = fmaf(theta, theta, 1.0f);
  const float t = __fdividef(theta >= 0.0f ? 1.0f : -1.0f, fmaf(w, rsqrtf(w), fabsf(theta)));
  const float cf = rsqrtf(fmaf(t, t, 1.0f));
  const float sf = t * cf;
  exact_rotation(cf, sf, c, s);
  return sf != 0.0f;
}

// (c, s) of the planes of step st (one lane per plane, warp 0): written to
// cs[2k], cs[2k + 1]; a step with some rotation is marked in stepf[st] and
// the sweep in *flag.
__device__ __forceinline__ void jacobi_rotations(const double* A, int mp, int np, const int* sched, int st,
                                                 double* cs, unsigned long long tau_b,
                                                 unsigned long long noise_b, int* stepf, int* flag) {
  for (int k = threadIdx.x & 31; k < np; k += 32) {
    const int pq = sched[st * np + k];
    const int p = pq & 0xFF, q = pq >> 8;
    double c, s;
    if (plane_rotation(A[p * mp + p], A[q * mp + q], A[p * mp + q], tau_b, noise_b, c, s)) {
      *flag = 1;
      stepf[st] = 1;
    }
    cs[2 * k] = c;
    cs[2 * k + 1] = s;
  }
}

// Row e of the 2 x 2 blocks of step st (block e / 2 = planes (a, b), a <= b;
// row p_a for even e, q_a for odd e): with the two (c, s), the new entries in
// columns p_b and q_b, n0 and n1, of J^T A J.  The same FMAs serve the
// update of A and the look-ahead of the next rotations, so both see the same
// bits.  Reads of A only.
struct BlockRow {
  int r, pb, qb, pa, qa, a, b;
  bool bottom;
};
__device__ __forceinline__ BlockRow block_row(int ab, bool bottom, const int* sched_st) {
  BlockRow br;
  br.a = ab & 0xFF;
  br.b = ab >> 8;
  const int pqa = sched_st[br.a], pqb = sched_st[br.b];
  br.pa = pqa & 0xFF;
  br.qa = pqa >> 8;
  br.pb = pqb & 0xFF;
  br.qb = pqb >> 8;
  br.bottom = bottom;
  br.r = bottom ? br.qa : br.pa;
  return br;
}
__device__ __forceinline__ void block_row_values(const BlockRow& br, const double* A, int mp, const double* csr,
                                                 double& n0, double& n1) {
  const double2 csa = *reinterpret_cast<const double2*>(csr + 2 * br.a);
  const double2 csb = *reinterpret_cast<const double2*>(csr + 2 * br.b);
  const int oa = br.bottom ? br.pa : br.qa;
  const double o0 = A[br.r * mp + br.pb], o1 = A[br.r * mp + br.qb];  // own row
  const double x0 = A[oa * mp + br.pb], x1 = A[oa * mp + br.qb];      // the block's other row
  // row rotation: top [c -s], bottom [s c] of the block's two rows, i.e.
  // c * own + (-+ s) * other; then the column rotation (.) [c s; -s c]
  const double sae = __longlong_as_double(__double_as_longlong(csa.y) ^
                                          (br.bottom ? 0ll : (long long)0x8000000000000000ull));
  const double r0 = fma(sae, x0, csa.x * o0), r1 = fma(sae, x1, csa.x * o1);
  n0 = fma(-csb.y, r1, csb.x * r0);
  n1 = fma(csb.y, r0, csb.x * r1);
}
// n1 (col_q) or n0 of block_row_values, by the same operations, in two
// parts: the reads (block_row_load) and the arithmetic (block_row_value).
struct BlockRowIn {
  double2 csa, csb;
  double o0, o1, x0, x1;
};
__device__ __forceinline__ BlockRowIn block_row_load(const BlockRow& br, const double* A, int mp,
                                                     const double* csr) {
  BlockRowIn in;
  in.csa = *reinterpret_cast<const double2*>(csr + 2 * br.a);
  in.csb = *reinterpret_cast<const double2*>(csr + 2 * br.b);
  const int oa = br.bottom ? br.pa : br.qa;
  in.o0 = A[br.r * mp + br.pb];
  in.o1 = A[br.r * mp + br.qb];
  in.x0 = A[oa * mp + br.pb];
  in.x1 = A[oa * mp + br.qb];
  return in;
}
__device__ __forceinline__ double block_row_value(const BlockRowIn& in, bool bottom, bool col_q) {
  const double sae = __longlong_as_double(__double_as_longlong(in.csa.y) ^
                                          (bottom ? 0ll : (long long)0x8000000000000000ull));
  const double r0 = fma(sae, in.x0, in.csa.x * in.o0), r1 = fma(sae, in.x1, in.csa.x * in.o1);
  const double sb = col_q ? in.csb.y : -in.csb.y;
  return fma(sb, col_q ? r0 : r1, in.csb.x * (col_q ? r1 : r0));
}

// u_data: the relative accuracy of the matrix's data (2^-53 for FP64 data,
// 2^-48 for a Gram from the BF16 slices): a plane is rotated only while its
// off-diagonal entry exceeds u_data |A|_F, below which the data do not
// determine it, and two indices whose diagonals both lie below
// 64 u_data |A|_F (the noise block) are left alone.
//
// Cyclic Jacobi with the circle method's parallel ordering (mp/2 disjoint
// planes a step).  The CTA has 256 threads in two groups: warps 0..3 apply
// each step's rotations to A (A <- J^T A J on the 2 x 2 blocks of the upper
// triangle, one block row per lane, the same eight FP64 instructions on
// every lane), and warp 0 then takes the next step's rotations from the
// updated A; warps 4..7 apply each step's rotations to V (V <- V J) while
// warp 0 works out the next ones.  The SM issues FP64 warp instructions at
// about one per 19 cycles, each taking some 64 cycles, so V's update is kept
// out of the phase in which A's update (the next rotations' input) runs.
// Step i's (c, s) sit in one of two slots; named barrier 1 (all 256 threads;
// warp 0 only arrives) publishes them, barrier 2 (all 256; warps 1..3 only
// arrive) tells warp 0 and the V warps that A is updated.
__device__ void jacobi_body(const double* __restrict__ Hin, int m, double* lam, double* Vout, int* sweeps_out,
                            double u_data) {
  extern __shared__ __align__(16) double sm[];
  const int mp = (m + 1) & ~1;  // padded to even; the pad row/column is zero
  const int np = mp / 2;        // planes per step
  const int nblk = np * (np + 1) / 2;
  const int nsteps = mp - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* A = sm;
  double* V = A + mp * mp;
  double* cs = V + mp * mp;                // two slots of (c, s) per plane
  int* sched = (int*)(cs + 2 * mp);        // [step][plane]: p | q << 8
  int* blk = sched + (mp - 1) * np;        // [block]: a | b << 8, upper blocks in order
  int* stepf = blk + nblk;                 // [step]: some rotation in this step
  int* stepneed = stepf + mp;              // [step]: a plane above the threshold at the sweep's start
  int* steplist = stepneed + mp;           // the sweep's steps in order
  int* flag = steplist + mp;               // some rotation in this sweep
  int* nlist = flag + 1;                   // length of steplist
  int* where = nlist + 1;                  // [step][index]: plane | 256 for the plane's q
  __shared__ double red[33];
  // H symmetrised on load: A = (H + H^T) / 2
  for (int e = threadIdx.x; e < mp * mp; e += blockDim.x) {
    const int i = e / mp, j = e % mp;
    A[e] = (i < m && j < m) ? 0.5 * (Hin[i * m + j] + Hin[j * m + i]) : 0.0;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  // the circle method's planes of every step, and the upper 2 x 2 blocks
  for (int e = threadIdx.x; e < (mp - 1) * np; e += blockDim.x) {
    const int st = e / np, k = e - st * np;
    const int pos0 = k, pos1 = mp - 1 - k;
    const int a = (pos0 == 0) ? 0 : 1 + (pos0 - 1 + st) % (mp - 1);
    const int b = 1 + (pos1 - 1 + st) % (mp - 1);
    sched[e] = min(a, b) | (max(a, b) << 8);
  }
  for (int e = threadIdx.x; e < nblk; e += blockDim.x) {
    int a = 0, r = e;
    while (r >= np - a) {
      r -= np - a;
      ++a;
    }
    blk[e] = a | ((a + r) << 8);
  }
  __syncthreads();
  double fs = 0.0;
  for (int e = threadIdx.x; e < mp * mp; e += blockDim.x) fs += A[e] * A[e];
  const double normA = sqrt(block_sum(fs, red));
  // thresholds as bit patterns: |x| > t  <=>  abs_bits(x) > bits(t) for t >= 0
  const unsigned long long tau_b = abs_bits(u_data * normA);
  const unsigned long long noise_b = abs_bits(64.0 * u_data * normA);
  // f / mp for f < np mp by a 32-bit reciprocal (exact in this range)
  const unsigned magic = (unsigned)((0xFFFFFFFFull + mp) / mp);
  // step of the plane (p, q), p < q, in the circle method's schedule:
  // q mod (mp - 1) for p = 0, else (p + q) / 2 mod (mp - 1) (mp - 1 is odd,
  // and mp / 2 is the inverse of 2 modulo it)
  const int half_mp = mp / 2;
  // Look-ahead (3 np <= 32): warp 0 forms the three entries a_pp, a_qq, a_pq
  // of each next plane from the A before this step and this step's (c, s)
  // (the same FMAs as the update), and the next rotations from them, while
  // warps 1..3 update A.  Otherwise warps 0..3 update A and warp 0 then
  // reads the updated A.
  const bool look = 3 * np <= 32;
  const int a_t0 = look ? 32 : 0, a_nt = look ? 96 : 128;  // A's update: first thread, threads
  const int a_t = (int)threadIdx.x - a_t0;
  // with at most a_nt block rows each updating lane keeps its one block
  const bool one_item = 2 * nblk <= a_nt;
  const int ab_own = (one_item && a_t >= 0 && a_t < 2 * nblk && warp < 4) ? blk[a_t >> 1] : 0;
  for (int e = threadIdx.x; e < mp; e += blockDim.x) stepneed[e] = 0;
  // where[st][x]: plane of index x in step st, | 256 when x is its q
  for (int e = threadIdx.x; e < (mp - 1) * np; e += blockDim.x) {
    const int st = e / np, k = e - st * np;
    where[st * mp + (sched[e] & 0xFF)] = k;
    where[st * mp + (sched[e] >> 8)] = k | 256;
  }
  __syncthreads();
  int sweep = 0;
  for (sweep = 1; sweep <= 60; ++sweep) {
    // A sweep runs only while some plane still needs a rotation, and only
    // the steps holding such a plane at the start of the sweep (the others
    // would rotate nothing, or planes that an earlier rotation of this sweep
    // lifted above the threshold: the next sweep's check sees those).
    int need = 0;
    for (int e = threadIdx.x; e < mp * mp; e += blockDim.x) {
      const int i = e / mp, j = e - (e / mp) * mp;
      if (i < j && abs_bits(A[e]) > tau_b &&
          !(abs_bits(A[i * mp + i]) <= noise_b && abs_bits(A[j * mp + j]) <= noise_b)) {
        need = 1;
        stepneed[i == 0 ? j % nsteps : ((i + j) * half_mp) % nsteps] = 1;
      }
    }
    if (!__syncthreads_or(need)) break;
    if (warp == 0) {
      // the list of the sweep's steps, in order; flags cleared for the next
      int cnt = 0;
      for (int st0 = 0; st0 < nsteps; st0 += 32) {
        const int st = st0 + lane;
        const bool on = st < nsteps && stepneed[st] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) steplist[cnt + __popc(bal & ((1u << lane) - 1u))] = st;
        cnt += __popc(bal);
        if (st < nsteps) {
          stepneed[st] = 0;
          stepf[st] = 0;
        }
      }
      if (lane == 0) {
        *flag = 0;
        *nlist = cnt;
      }
      __syncwarp();
      jacobi_rotations(A, mp, np, sched, steplist[0], cs, tau_b, noise_b, stepf, flag);
      __syncwarp();
    }
    for (int i = 0;; ++i) {
      // barrier 1: step i's (c, s), stepf, the list and its length are
      // written (and, with the look-ahead, step i - 1's update of A is done)
      if (warp == 0 && !look)
        bar_arrive_n(1, kJacobiThreads);
      else
        bar_sync_n(1, kJacobiThreads);
      const int st = steplist[i];
      const bool last = i + 1 == *nlist;
      const bool any = stepf[st] != 0;  // no plane rotates: nothing to apply
      const double* csr = cs + (i & 1) * mp;
      const int* sched_st = sched + st * np;
      if (look && warp == 0) {
        // entry lane l: plane l / 3 of the next step, entry l % 3 (a_pp,
        // a_qq, a_pq), taken from the block row that the update writes it from
        double v = 0.0;
        const int st1 = last ? st : steplist[i + 1];
        const bool act = !last && lane < 3 * np;
        BlockRow br{};
        bool col_q = false;
        if (act) {
          const int pq1 = sched[st1 * np + lane / 3];
          const int which = lane - 3 * (lane / 3);
          int x = pq1 & 0xFF, y = pq1 >> 8;  // (p', q')
          if (which == 0) y = x;
          if (which == 1) x = y;
          const int* wst = where + st * mp;
          int wx = wst[x], wy = wst[y];
          if ((wy & 0xFF) < (wx & 0xFF)) {  // the row is the index in the lower plane
            const int tt = wx;
            wx = wy;
            wy = tt;
          }
          const int pa = wx & 0xFF, pb = wy & 0xFF;
          br = block_row(pa | (pb << 8), (wx >> 8) != 0, sched_st);
          col_q = (wy >> 8) != 0;
        }
        BlockRowIn in{};
        if (act) in = block_row_load(br, A, mp, csr);
        // the update of A may start once these reads are done (barrier 2:
        // warp 0 arrives, a release of its reads; warps 1..3 wait)
        bar_arrive_n(2, 128);
        if (act) v = block_row_value(in, br.bottom, col_q);
        const double app = __shfl_sync(0xffffffffu, v, 3 * lane);
        const double aqq = __shfl_sync(0xffffffffu, v, 3 * lane + 1);
        const double apq = __shfl_sync(0xffffffffu, v, 3 * lane + 2);
        if (!last && lane < np) {
          double c, sn;
          if (plane_rotation(app, aqq, apq, tau_b, noise_b, c, sn)) {
            *flag = 1;
            stepf[st1] = 1;
          }
          double* csw = cs + ((i + 1) & 1) * mp;
          csw[2 * lane] = c;
          csw[2 * lane + 1] = sn;
        }
        __syncwarp();
      } else if (warp < 4) {
        if (look) bar_sync_n(2, 128);  // warp 0 has read the entries it needs
        if (any) {
          // block rows: the two rows of a block sit in adjacent lanes, which
          // both read the block before either writes (__syncwarp).  An
          // identity rotation (c = 1, s = 0) leaves the values bit for bit.
          for (int base = a_t - lane; base < 2 * nblk; base += a_nt) {
            const int e = base + lane;
            const bool valid = e < 2 * nblk;
            const int ab = !valid ? 0 : (one_item ? ab_own : blk[e >> 1]);
            const BlockRow br = block_row(ab, (e & 1) != 0, sched_st);
            double n0 = 0.0, n1 = 0.0;
            if (valid) block_row_values(br, A, mp, csr, n0, n1);
            __syncwarp();
            if (valid) {
              if (br.a == br.b) {
                if (!br.bottom) {
                  A[br.pa * mp + br.pa] = n0;
                  A[br.pa * mp + br.qa] = n1;
                  A[br.qa * mp + br.pa] = n1;  // the block stays exactly symmetric
                } else {
                  A[br.qa * mp + br.qa] = n1;
                }
              } else {
                A[br.r * mp + br.pb] = n0;
                A[br.r * mp + br.qb] = n1;
                A[br.pb * mp + br.r] = n0;
                A[br.qb * mp + br.r] = n1;
              }
            }
            __syncwarp();
          }
        }
        if (!look) {
          // barrier 2: A holds step i's result (warps 1..3 arrive; warp 0 and
          // the V warps wait), so V's update runs beside the next rotations
          if (warp == 0) {
            bar_sync_n(2, kJacobiThreads);
            if (!last)
              jacobi_rotations(A, mp, np, sched, steplist[i + 1], cs + ((i + 1) & 1) * mp, tau_b, noise_b,
                               stepf, flag);
            __syncwarp();
          } else {
            bar_arrive_n(2, kJacobiThreads);
          }
        }
      } else {
        if (!look) bar_sync_n(2, kJacobiThreads);
        if (any) {
          for (int f = (int)threadIdx.x - 128; f < np * mp; f += 128) {
            const int k = (int)__umulhi((unsigned)f, magic), row = f - k * mp;
            const double2 c_s = *reinterpret_cast<const double2*>(csr + 2 * k);
            const int pq = sched_st[k];
            const int p = pq & 0xFF, q = pq >> 8;
            const double vp = V[row * mp + p], vq = V[row * mp + q];
            V[row * mp + p] = fma(-c_s.y, vq, c_s.x * vp);
            V[row * mp + q] = fma(c_s.y, vp, c_s.x * vq);
          }
        }
      }
      if (last) break;
    }
    __syncthreads();  // A and V hold the sweep's last step
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
  // sort descending by rank counting (ties by index), drop the pad
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const long long li = order_key(A[i * mp + i]);
    int pos = 0;
    for (int j = 0; j < m; ++j) {
      const long long lj = order_key(A[j * mp + j]);
      pos += (lj > li) || (lj == li && j < i);
    }
    lam[pos] = A[i * mp + i];
    for (int r = 0; r < m; ++r) Vout[r * m + pos] = V[r * mp + i];
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
}

__global__ void __launch_bounds__(kJacobiThreads) k_jacobi(JacBatch batch) {
  // (a constant index into the parameter block: no local copy of the batch)
  const JacProb& p = blockIdx.x == 0 ? batch.p[0] : batch.p[1];
  jacobi_body(p.H, p.m, p.lam, p.V, p.sweeps, 0x1p-53);
}

__device__ void rank_warp(const double* lam, int m, double trace, double nf, double eps, int rmax, int rfix,
                          double u_eff, int n_eig, int n_flag, int* out);

// One m x m problem per CTA: H + b * m^2 -> lam + b * m, V + b * m^2.  With
// rank.out set, warp 0 then applies the truncation rule to the leading mr
// eigenvalues and trace[b].
__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_strided(const double* H, int m, double* lam, double* V,
                                                         RankArgs rank, int mr, const double* trace,
                                                         double u_data) {
  TK_PDL_ENTRY();
  TK_PDL_EARLY_IF_SMALL();
  const long long b = blockIdx.x;
  jacobi_body(H + b * m * m, m, lam + b * m, V + b * m * m, nullptr, u_data);
  if (rank.out == nullptr) return;
  __syncthreads();  // the sorted eigenvalues are in lam
  if (threadIdx.x < 32)
    rank_warp(lam + b * m, mr, trace[b], rank.normF2[b], rank.eps[b], rank.rmax[b], rank.rfix[b], rank.u_eff,
              rank.n_eig, rank.n_flag, rank.out + 4 * b);
}

// Canonical sign of each column of V (n x m row-major, ld = m); instance blockIdx.y.
__global__ void k_canonical_sign(double* V, int n, int m) {
  const int col = blockIdx.x;
  V += (size_t)blockIdx.y * n * m;
  const int half = (n + 1) / 2;
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1.0;
  int idx = 0;
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    const double a = fabs(V[(long long)i * m + col]);
    if (a > best) {
      best = a;
      idx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = idx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double o = bv[threadIdx.x + w];
      const int oi = bi[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const bool flip = V[(long long)bi[0] * m + col] < 0.0;
  if (flip)
    for (int i = threadIdx.x; i < n; i += blockDim.x) V[(long long)i * m + col] = -V[(long long)i * m + col];
}

__global__ void k_copy_rows(const double* G, double* H, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) H[e] = G[e];
}

// Persymmetric split.  G is symmetric and G(i, j) = G(n-1-i, n-1-j) (a
// symmetric grid and an even covariance), so its eigenvectors are even or odd
// under the flip i -> n-1-i.  In the orthonormal basis (e_i +- e_{n-1-i})/sqrt2
// (and e_c for the centre c of an odd n) G is block diagonal:
//   Ge(i, j) = G(i, j) + G(i, n-1-j),  Go(i, j) = G(i, j) - G(i, n-1-j),  i, j < n/2,
//   Ge(i, c) = Ge(c, i) = sqrt2 G(i, c),  Ge(c, c) = G(c, c)   (odd n).
__global__ void k_persym_split(const double* __restrict__ G, int n, double* __restrict__ Ge,
                               double* __restrict__ Go) {
  const int ho = n / 2, he = n - ho;
  // instance blockIdx.y of a batch laid out [b][n][n] -> [b][he][he], [b][ho][ho]
  G += (size_t)blockIdx.y * n * n;
  Ge += (size_t)blockIdx.y * he * he;
  Go += (size_t)blockIdx.y * ho * ho;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < he * he; e += gridDim.x * blockDim.x) {
    const int i = e / he, j = e % he;
    double ve;
    if (i < ho && j < ho) {
      const double a = G[(long long)i * n + j], b = G[(long long)i * n + (n - 1 - j)];
      ve = a + b;
      Go[i * ho + j] = a - b;
    } else if (i < ho) {
      ve = 1.4142135623730950488 * G[(long long)i * n + ho];
    } else if (j < ho) {
      ve = 1.4142135623730950488 * G[(long long)ho * n + j];
    } else {
      ve = G[(long long)ho * n + ho];
    }
    Ge[e] = ve;
  }
}

// Top m of the union of the two halves' eigenpairs (each sorted descending),
// vectors expanded to length n: even y -> (y_i, y_i) / sqrt2 (centre y_c),
// odd y -> (y_i, -y_i) / sqrt2 (centre 0).  *safe = number of leading merged
// pairs that are certainly the leading pairs of G: those above the last
// computed eigenvalue of every half that has eigenvalues left uncomputed.
__global__ void k_persym_merge(const double* __restrict__ le, const double* __restrict__ Ve, int me,
                               const double* __restrict__ lo, const double* __restrict__ Vo, int mo, int n, int m,
                               double* __restrict__ lam, double* __restrict__ V, int* flag) {
  __shared__ int src[kMaxM], idx[kMaxM];
  const int ho = n / 2, he = n - ho;
  {  // instance blockIdx.x of a batch
    const size_t b = blockIdx.x;
    le += b * me;
    lo += b * mo;
    Ve += b * he * me;
    Vo += b * ho * mo;
    lam += b * m;
    V += b * n * m;
    if (flag) flag += b * 4;
  }
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int k = 0; k < m; ++k) {
      const bool take_e = (b >= mo) || (a < me && le[a] >= lo[b]);
      src[k] = take_e ? 0 : 1;
      idx[k] = take_e ? a++ : b++;
      lam[k] = take_e ? le[idx[k]] : lo[idx[k]];
    }
    if (flag) {
      double t = -INFINITY;
      if (me < he) t = fmax(t, le[me - 1]);
      if (mo < ho) t = fmax(t, lo[mo - 1]);
      int safe = 0;
      while (safe < m && lam[safe] > t) ++safe;
      *flag = safe;
    }
  }
  __syncthreads();
  const double r2 = 0.70710678118654752440;
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int i = e / m, k = e % m;
    double v;
    if (src[k] == 0) {
      if (i < ho)
        v = r2 * Ve[i * me + idx[k]];
      else if (i >= he)
        v = r2 * Ve[(n - 1 - i) * me + idx[k]];
      else
        v = Ve[ho * me + idx[k]];  // centre of an odd n
    } else {
      if (i < ho)
        v = r2 * Vo[i * mo + idx[k]];
      else if (i >= he)
        v = -r2 * Vo[(n - 1 - i) * mo + idx[k]];
      else
        v = 0.0;
    }
    V[(long long)i * m + k] = v;
  }
}

// Truncation rule (Task 1, Sec. 2.1, with the HOSVD bound of Sec. 3.2), in
// compensated FP64 (the route of rank_warp below for non-finite inputs):
// the smallest r >= 1 whose discarded sum, tail beyond the m computed
// eigenvalues (trace - their sum) plus the clamped computed ones from r on,
// summed smallest first, is <= eps^2 |F|^2 / 3; capped at rmax.
// n_eig: order of the matrix whose eigenvalues lam are (all computed when
// m == n_eig); n_flag: the n of the precision flag's threshold.
__device__ void rank_body(const double* lam, int m, double trace, double nf, double eps, int rmax, int rfix,
                          double u_eff, int n_eig, int n_flag, int* out) {
  const double thr = eps * eps * nf / 3.0;
  double sum = 0.0, sc = 0.0;
  for (int i = 0; i < m; ++i) {
    const double t = sum + lam[i];
    sc += (fabs(sum) >= fabs(lam[i])) ? (sum - t) + lam[i] : (lam[i] - t) + sum;
    sum = t;
  }
  double extra = trace - (sum + sc);
  if (!(extra > 0.0) || m >= n_eig) extra = 0.0;
  int r = m + 1;  // "more than computed"
  double ts = extra, tc = 0.0;
  if (ts <= thr) r = m;
  for (int q = m - 1; q >= 1; --q) {
    const double x = lam[q] > 0.0 ? lam[q] : 0.0;
    const double t = ts + x;
    tc += (fabs(ts) >= x) ? (ts - t) + x : (x - t) + ts;
    ts = t;
    if (ts + tc <= thr) r = q;
  }
  int flags = 0;
  if (r > m) r = m + 1;
  out[2] = r;  // before the cap; m + 1 means "more than the m computed"
  if (rfix > 0) {
    r = rfix < m ? rfix : m;
  } else if (r > rmax) {
    r = rmax;
    flags |= TK_RANK_CAPPED;
  }
  if (thr < 10.0 * u_eff * (double)n_flag * nf) flags |= TK_EPS_UNREACHABLE_AT_PRECISION;
  out[0] = r;
  out[1] = flags;
}

// 128-bit halves through warp shuffles.
__device__ __forceinline__ __int128 shfl_down128(__int128 v, int off) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, off);
  const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, off);
  return (__int128)(((unsigned __int128)h2 << 64) | l2);
}
__device__ __forceinline__ __int128 shfl_xor128(__int128 v, int mask) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
  const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, mask);
  const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, mask);
  return (__int128)(((unsigned __int128)h2 << 64) | l2);
}

__device__ __forceinline__ int exp_field(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
}

// v 2^sh truncated toward zero, as a signed 128-bit integer (zero and
// subnormal v give 0); sh is chosen so that |v| 2^sh < 2^120.
__device__ __forceinline__ __int128 fixed128(double v, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const int sft = ex - 1075 + sh;  // v = mant 2^(ex - 1075), at most 67 here
  unsigned __int128 mg = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  if (sft >= 0)
    mg <<= sft;
  else
    mg = (sft > -64) ? (mg >> -sft) : 0;
  const __int128 r = (__int128)mg;
  return (b >> 63) ? -r : r;
}

// The same rule, by one warp for one instance (all 32 lanes call it, lane 0
// writes out), in exact fixed-point arithmetic: every input is scaled by one
// power of two so that the largest lies below 2^120 and truncated to a
// 128-bit integer (losing less than 2^-120 of the largest input each), after
// which the sums and comparisons are exact.  Lane t holds lam[3t .. 3t + 2];
// the discarded sums come from one suffix scan over the lanes.  m > 96 or a
// non-finite input takes the FP64 route.
__device__ void rank_warp(const double* lam, int m, double trace, double nf, double eps, int rmax, int rfix,
                          double u_eff, int n_eig, int n_flag, int* out) {
  const int lane = threadIdx.x & 31;
  const double thr = eps * eps * nf / 3.0;
  double v[3];
  int emax = max(exp_field(trace), exp_field(thr));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = 3 * lane + k;
    v[k] = (i < m) ? lam[i] : 0.0;
    emax = max(emax, exp_field(v[k]));
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  if (emax == 0x7FF || m > 96) {
    if (lane == 0) rank_body(lam, m, trace, nf, eps, rmax, rfix, u_eff, n_eig, n_flag, out);
    return;
  }
  const int sh = 1142 - emax;  // the largest input below 2^120
  __int128 P[3], tot = 0, ptot = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const __int128 L = fixed128(v[k], sh);
    P[k] = L > 0 ? L : 0;
    tot += L;
    ptot += P[k];
  }
  __int128 S = tot;  // sum of the m eigenvalues
  for (int o = 16; o > 0; o >>= 1) S += shfl_xor128(S, o);
  const __int128 TH = fixed128(thr, sh);
  __int128 extra = fixed128(trace, sh) - S;  // the tail beyond the m computed
  if (extra <= 0 || m >= n_eig) extra = 0;
  // clamped sums over the lanes from this one up
  __int128 suf = ptot;
  for (int o = 1; o < 32; o <<= 1) {
    const __int128 x = shfl_down128(suf, o);
    if (lane + o < 32) suf += x;
  }
  // the discarded sum from q on, q = 3 lane + 2 down to 3 lane; the smallest
  // q in [1, m - 1] whose sum is within the threshold
  __int128 run = extra + (suf - ptot);
  int qbest = 0x7FFFFFFF;
#pragma unroll
  for (int k = 2; k >= 0; --k) {
    const int q = 3 * lane + k;
    run += P[k];
    if (q >= 1 && q < m && run <= TH) qbest = q;
  }
  qbest = __reduce_min_sync(0xffffffffu, qbest);
  if (lane == 0) {
    int r = (qbest != 0x7FFFFFFF) ? qbest : (extra <= TH ? m : m + 1);
    int flags = 0;
    out[2] = r;  // before the cap; m + 1 means "more than the m computed"
    if (rfix > 0) {
      r = rfix < m ? rfix : m;
    } else if (r > rmax) {
      r = rmax;
      flags |= TK_RANK_CAPPED;
    }
    if (thr < 10.0 * u_eff * (double)n_flag * nf) flags |= TK_EPS_UNREACHABLE_AT_PRECISION;
    out[0] = r;
    out[1] = flags;
  }
}

__global__ void k_rank(const double* lam, int m, const double* trace, const double* normF2, double eps, int rmax,
                       int rfix, double u_eff, int n, int* out) {
  rank_warp(lam, m, trace[0], normF2[0], eps, rmax, rfix, u_eff, n, n, out);
}

// One instance per warp: lam + b m, trace[b], normF2[b], eps[b], rmax[b],
// rfix[b], out + 4 b.
__global__ void k_rank_batch(const double* lam, int m, const double* trace, const double* normF2, const double* epsv,
                             const int* rmaxv, const int* rfixv, double u_eff, int n_eig, int n_flag, int B,
                             int* out) {
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b < B)  // uniform over the warp
    rank_warp(lam + (size_t)b * m, m, trace[b], normF2[b], epsv[b], rmaxv[b], rfixv[b], u_eff, n_eig, n_flag,
              out + 4 * b);
}

}  // namespace

// The subspace carries kMargin columns beyond the m requested pairs (up to
// n and kMaxM) so that the m leading Ritz pairs converge.  After the FP32
// pass and one FP64 pass the leading pairs of the covariance Grams sit at the
// FP64 noise floor already with four extra columns: the projector onto the
// rank-r factor moves by 1e-10 .. 4e-9 of |F| (eight columns: 5e-11 .. 1e-9),
// and the eigenvalues by about u lambda_1 either way.
constexpr int kMargin = 4;

static int subspace_cols(int n, int m) { return std::min(std::min(n, kMaxM), m + kMargin); }

static size_t one_problem_doubles(int n, int m) {
  const int ms = subspace_cols(n, m);
  // Omega/Y, Q, W (n x ms each), H, V_H (ms x ms each), Ritz values, misc
  return 3ull * n * ms + 2ull * ms * ms + ms + 64 + (size_t)n * n;
}

size_t sym_eig_scratch_doubles(int n, int m) {
  // the persymmetric path: two halves with their blocks, pairs and vectors
  const int ho = n / 2, he = n - ho;
  const int mh = std::min(he, (m + 1) / 2 + 4);
  const size_t split = (size_t)he * he + (size_t)ho * ho + 2ull * mh + (size_t)he * mh + (size_t)ho * mh +
                       one_problem_doubles(he, std::min(he, mh)) + one_problem_doubles(std::max(ho, 1), std::min(std::max(ho, 1), mh)) + 256;
  return std::max(one_problem_doubles(n, m), split);
}

static constexpr size_t kQrSmemMax = 200 * 1024;
static constexpr size_t kStart32SmemMax = 200 * 1024;

static size_t jacobi_smem(int m) {
  const int mp = (m + 1) & ~1, np = mp / 2;
  // A, V, two slots of (c, s); the plane schedule, the block list, three
  // per-step arrays (rotation flags, need flags, the sweep's step list), the
  // sweep flag, the list length and each index's plane per step
  return (2ull * mp * mp + 2ull * mp) * sizeof(double) +
         ((size_t)(mp - 1) * np + (size_t)np * (np + 1) / 2 + 3 * (size_t)mp + 2 + (size_t)(mp - 1) * mp) *
             sizeof(int);
}

static void set_attrs_once() {
  TK_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jacobi_smem(kMaxM)));
  TK_CUDA(cudaFuncSetAttribute(k_householder_qr<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kQrSmemMax));
  TK_CUDA(cudaFuncSetAttribute(k_householder_qr_strided<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kQrSmemMax));
  TK_CUDA(cudaFuncSetAttribute(k_jacobi_strided, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)jacobi_smem(kMaxM)));
}

static void set_attrs() { once_per_device((const void*)&set_attrs_once, set_attrs_once); }

// One eigenproblem of the batch: leading m pairs of the symmetric n x n G.
struct EigProb {
  const double* G;
  int n, m;
  double* lam;  // m
  double* V;    // n x m, row-major
  double* scr;  // one_problem_doubles(n, m)
};

// Up to two problems whose QR and Jacobi steps run as one launch (a CTA each).
static void eig_batch(EigProb* pr, int count, cudaStream_t s) {
  set_attrs();
  struct Work {
    int ms;
    double *Y, *Q, *W, *H, *VH, *lsub, *misc;
  } w[2];
  for (int b = 0; b < count; ++b) {
    const int n = pr[b].n;
    w[b].ms = subspace_cols(n, pr[b].m);
    w[b].Y = pr[b].scr;
    w[b].Q = w[b].Y + (size_t)n * w[b].ms;
    w[b].W = w[b].Q + (size_t)n * w[b].ms;
    w[b].H = w[b].W + (size_t)n * w[b].ms;
    w[b].VH = w[b].H + (size_t)w[b].ms * w[b].ms;
    w[b].lsub = w[b].VH + (size_t)w[b].ms * w[b].ms;
    w[b].misc = w[b].lsub + w[b].ms;
  }
  // problems small enough for Jacobi on the whole matrix
  {
    JacBatch jb{};
    int nj = 0;
    size_t smem = 0;
    for (int b = 0; b < count; ++b) {
      if (w[b].ms != pr[b].n) continue;
      const int n = pr[b].n;
      k_copy_rows<<<64, 256, 0, s>>>(pr[b].G, w[b].H, n);
      TK_LAUNCH("k_copy_rows");
      jb.p[nj++] = JacProb{w[b].H, n, w[b].lsub, w[b].VH, (int*)(w[b].misc + 8)};
      smem = std::max(smem, jacobi_smem(n));
    }
    if (nj) {
      k_jacobi<<<nj, kJacobiThreads, smem, s>>>(jb);
      TK_LAUNCH("k_jacobi");
    }
    for (int b = 0; b < count; ++b) {
      if (w[b].ms != pr[b].n) continue;
      const int n = pr[b].n, m = pr[b].m;
      TK_CUDA(cudaMemcpy2DAsync(pr[b].V, sizeof(double) * m, w[b].VH, sizeof(double) * n, sizeof(double) * m, n,
                                cudaMemcpyDeviceToDevice, s));
      TK_CUDA(cudaMemcpyAsync(pr[b].lam, w[b].lsub, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    }
  }
  // the others: two passes of subspace iteration, then Rayleigh-Ritz
  int idx[2], nr = 0;
  for (int b = 0; b < count; ++b)
    if (w[b].ms != pr[b].n) idx[nr++] = b;
  if (nr == 0) return;
  for (int t = 0; t < nr; ++t) {
    const int b = idx[t];
    k_random<<<64, 256, 0, s>>>(w[b].Y, (long long)pr[b].n * w[b].ms, 0x1711068740ull + (unsigned)pr[b].n);
    TK_LAUNCH("k_random");
  }
  for (int pass = 0; pass < 2; ++pass) {
    QrBatch qb{};
    size_t smem = 0;
    bool shared = true;
    for (int t = 0; t < nr; ++t) {
      const int b = idx[t], n = pr[b].n, ms = w[b].ms;
      const double* src = (pass == 0) ? w[b].Y : w[b].Q;
      GemmDesc d{n, ms, n, 1, pr[b].G, 0, n, 1, src, 0, 1, n, w[b].W, 0, 1, n};
      gemm_f64(d, s);
      TK_CUDA(cudaMemcpyAsync(w[b].Y, w[b].W, sizeof(double) * (size_t)n * ms, cudaMemcpyDeviceToDevice, s));
      qb.p[t] = QrProb{w[b].Y, w[b].Q, n, ms};
      const size_t need = 2ull * n * ms * sizeof(double);
      smem = std::max(smem, need);
      if (need > kQrSmemMax) shared = false;
    }
    if (shared)
      k_householder_qr<true><<<nr, 256, smem, s>>>(qb);
    else
      k_householder_qr<false><<<nr, 256, 0, s>>>(qb);
    TK_LAUNCH("k_householder_qr");
  }
  JacBatch jb{};
  size_t smem = 0;
  for (int t = 0; t < nr; ++t) {
    const int b = idx[t], n = pr[b].n, ms = w[b].ms;
    GemmDesc d1{n, ms, n, 1, pr[b].G, 0, n, 1, w[b].Q, 0, 1, n, w[b].W, 0, 1, n};
    gemm_f64(d1, s);
    GemmDesc d2{ms, ms, n, 1, w[b].Q, 0, n, 1, w[b].W, 0, 1, n, w[b].H, 0, ms, 1};
    gemm_f64(d2, s);
    jb.p[t] = JacProb{w[b].H, ms, w[b].lsub, w[b].VH, (int*)(w[b].misc + 8)};
    smem = std::max(smem, jacobi_smem(ms));
  }
  k_jacobi<<<nr, kJacobiThreads, smem, s>>>(jb);
  TK_LAUNCH("k_jacobi");
  for (int t = 0; t < nr; ++t) {
    const int b = idx[t], n = pr[b].n, ms = w[b].ms, m = pr[b].m;
    // leading m Ritz vectors V = Q V_H[:, :m] (row-major n x m)
    GemmDesc d3{n, m, ms, 1, w[b].Q, 0, 1, n, w[b].VH, 0, ms, 1, pr[b].V, 0, m, 1};
    gemm_f64(d3, s);
    TK_CUDA(cudaMemcpyAsync(pr[b].lam, w[b].lsub, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  }
}

void sym_eig_topm(const double* G, int n, int m, double* lam, double* V, double* trace_out, double* scratch,
                  cudaStream_t s) {
  if (m < 1 || m > kMaxM || m > n) fail(TK_EINVAL, "sym_eig: need 1 <= m <= min(n, 96)");
  double* scr = scratch;
  double* misc = scratch + one_problem_doubles(n, m) - 64;
  k_trace<<<1, 32, 0, s>>>(G, n, trace_out ? trace_out : misc);
  TK_LAUNCH("k_trace");
  EigProb p{G, n, m, lam, V, scr};
  eig_batch(&p, 1, s);
  k_canonical_sign<<<m, 256, 0, s>>>(V, n, m);
  TK_LAUNCH("k_canonical_sign");
}

void sym_eig_topm_persym(const double* G, int n, int m, double* lam, double* V, double* trace_out, int* flag,
                         double* scratch, cudaStream_t s) {
  if (m < 1 || m > kMaxM || m > n) fail(TK_EINVAL, "sym_eig: need 1 <= m <= min(n, 96)");
  const int ho = n / 2, he = n - ho;
  const int me = std::min(he, (m + 1) / 2 + 4), mo = std::min(ho, (m + 1) / 2 + 4);
  double* Ge = scratch;
  double* Go = Ge + (size_t)he * he;
  double* le = Go + (size_t)ho * ho;
  double* lo = le + me;
  double* Ve = lo + mo;
  double* Vo = Ve + (size_t)he * me;
  double* s0 = Vo + (size_t)ho * mo;
  double* s1 = s0 + one_problem_doubles(he, me);
  k_trace<<<1, 32, 0, s>>>(G, n, trace_out);
  TK_LAUNCH("k_trace");
  k_persym_split<<<64, 256, 0, s>>>(G, n, Ge, Go);
  TK_LAUNCH("k_persym_split");
  EigProb p[2] = {{Ge, he, me, le, Ve, s0}, {Go, ho, mo, lo, Vo, s1}};
  eig_batch(p, 2, s);
  k_persym_merge<<<1, 256, 0, s>>>(le, Ve, me, lo, Vo, mo, n, m, lam, V, flag);
  TK_LAUNCH("k_persym_merge");
  k_canonical_sign<<<m, 256, 0, s>>>(V, n, m);
  TK_LAUNCH("k_canonical_sign");
}

// ---------------------------------------------------------------------------
// B instances with the same n and m (G: [b][n][n]).  Every step is one launch
// over all instances: the subspace products are batched GEMMs, QR and Jacobi
// run one CTA per instance, and each instance starts from the same random
// block, so an instance's eigenpairs do not depend on the batch around it.
// ---------------------------------------------------------------------------
namespace {

struct EigGroup {
  int n, m, ms;
  const double* G;
  double *Y, *Q, *W, *H, *VH, *lsub;
  double *lam, *V;
};

size_t group_doubles(int n, int m, int B) {
  const int ms = subspace_cols(n, m);
  return (size_t)B * (3ull * n * ms + 2ull * ms * ms + ms) + 1024;
}

EigGroup carve_group(double* p, const double* G, int n, int m, int B, double* lam, double* V) {
  EigGroup g;
  g.n = n;
  g.m = m;
  g.ms = subspace_cols(n, m);
  g.G = G;
  g.lam = lam;
  g.V = V;
  auto take = [&](size_t k) {
    double* q = p;
    p += (k + 31) & ~size_t(31);
    return q;
  };
  g.Y = take((size_t)B * n * g.ms);
  g.Q = take((size_t)B * n * g.ms);
  g.W = take((size_t)B * n * g.ms);
  g.H = take((size_t)B * g.ms * g.ms);
  g.VH = take((size_t)B * g.ms * g.ms);
  g.lsub = take((size_t)B * g.ms);
  return g;
}

// The FP32 start (with the trace folded in) serves the subspace path when
// its shared-memory image fits.
bool uses_start32(int n, int ms) {
  return ms != n && n <= 256 && start32_smem(n, ms) <= kStart32SmemMax && gomega32_smem(n, ms) <= kStart32SmemMax;
}

// trace: written by the FP32 start kernel when that path runs (the caller
// computes it otherwise).
void solve_group(const EigGroup& g, int B, double* trace, cudaStream_t s, Profiler* pf, const RankArgs* rank,
                 double u_data) {
  const int n = g.n, ms = g.ms, m = g.m;
  if (ms == n) {
    // whole matrices: Jacobi directly
    TK_CUDA(cudaMemcpyAsync(g.H, g.G, sizeof(double) * (size_t)B * n * n, cudaMemcpyDeviceToDevice, s));
  } else {
    const unsigned long long seed = 0x1711068740ull + (unsigned)n;
    const size_t need = 2ull * n * ms * sizeof(double);
    auto qr = [&]() {
      if (pf) pf->begin(TK_STAGE_QR, s);
      // the scalars go to H's storage, which the Rayleigh-Ritz step fills later
      if (!qr64_batch(g.Y, g.H, g.Q, n, ms, B, (long long)ms * ms, s)) {
        if (need <= kQrSmemMax)
          k_householder_qr_strided<true><<<B, 256, need, s>>>(g.Y, g.Q, n, ms, (long long)n * ms);
        else
          k_householder_qr_strided<false><<<B, 256, 0, s>>>(g.Y, g.Q, n, ms, (long long)n * ms);
        TK_LAUNCH("k_householder_qr_strided");
      }
      if (pf) pf->end(s);
    };
    auto power = [&](const double* src) {  // Y = G src
      GemmDesc d{n, ms, n, B, g.G, (long long)n * n, n, 1, src, (long long)n * ms, 1, n,
                 g.Y, (long long)n * ms, 1, n};
      d.fixed_order = 1;
      if (pf) pf->begin(TK_STAGE_EIG_GEMM, s);
      gemm_f64(d, s);
      if (pf) pf->end(s);
    };
    if (uses_start32(n, ms)) {
      // FP32 pass from the random block, then one FP64 pass
      // (Y's storage holds the FP32 product until the FP64 pass writes it)
      if (pf) pf->begin(TK_STAGE_START, s);
      start32_launch(g.G, n, ms, B, seed, g.Q, trace, reinterpret_cast<float*>(g.Y), s);
      if (pf) pf->end(s);
      power(g.Q);
      qr();
    } else {
      // two FP64 passes from the random block
      k_random_rep<<<(unsigned)std::min<long long>(((long long)B * n * ms + 255) / 256, 1024), 256, 0, s>>>(
          g.W, (long long)n * ms, B, seed);
      TK_LAUNCH("k_random_rep");
      power(g.W);
      qr();
      power(g.Q);
      qr();
    }
    GemmDesc d1{n, ms, n, B, g.G, (long long)n * n, n, 1, g.Q, (long long)n * ms, 1, n,
                g.W, (long long)n * ms, 1, n};
    d1.fixed_order = 1;
    if (pf) pf->begin(TK_STAGE_EIG_GEMM, s);
    gemm_f64(d1, s);
    GemmDesc d2{ms, ms, n, B, g.Q, (long long)n * ms, n, 1, g.W, (long long)n * ms, 1, n,
                g.H, (long long)ms * ms, ms, 1};
    d2.fixed_order = 1;
    gemm_f64(d2, s);
    if (pf) pf->end(s);
  }
  if (pf) pf->begin(TK_STAGE_JACOBI, s);
  launch_pdl("k_jacobi_strided", k_jacobi_strided, dim3(B), dim3(kJacobiThreads), jacobi_smem(ms), s, g.H, ms, g.lsub, g.VH,
             rank ? *rank : RankArgs{}, m, trace,
                                                    u_data);
  if (pf) pf->end(s);
  if (ms == n) {
    // first m columns of V_H (n x n) into V (n x m)
    TK_CUDA(cudaMemcpy2DAsync(g.V, sizeof(double) * m, g.VH, sizeof(double) * ms, sizeof(double) * m,
                              (size_t)B * n, cudaMemcpyDeviceToDevice, s));
  } else {
    GemmDesc d3{n, m, ms, B, g.Q, (long long)n * ms, 1, n, g.VH, (long long)ms * ms, ms, 1,
                g.V, (long long)n * m, m, 1};
    d3.fixed_order = 1;
    if (pf) pf->begin(TK_STAGE_EIG_GEMM, s);
    gemm_f64(d3, s);
    if (pf) pf->end(s);
  }
  TK_CUDA(cudaMemcpy2DAsync(g.lam, sizeof(double) * m, g.lsub, sizeof(double) * ms, sizeof(double) * m, B,
                            cudaMemcpyDeviceToDevice, s));
}

}  // namespace

size_t sym_eig_batch_scratch_doubles(int n, int m, int B) { return group_doubles(n, m, B) + 4096; }

void sym_eig_batch(const double* G, int n, int m, int B, double* lam, double* V, double* trace, double* scratch,
                   cudaStream_t s, Profiler* pf, const RankArgs* rank, bool signs, double u_data) {
  if (m < 1 || m > kMaxM || m > n) fail(TK_EINVAL, "sym_eig: need 1 <= m <= min(n, 96)");
  if (B < 1) return;
  set_attrs();
  const EigGroup g = carve_group(scratch, G, n, m, B, lam, V);
  if (!uses_start32(n, g.ms)) {
    k_trace<<<B, 32, 0, s>>>(G, n, trace);
    TK_LAUNCH("k_trace");
  }
  solve_group(g, B, trace, s, pf, rank, u_data);
  if (!signs) return;
  k_canonical_sign<<<dim3(m, B), 256, 0, s>>>(V, n, m);
  TK_LAUNCH("k_canonical_sign");
}

void rank_rule_batch(const double* lam, int m, const double* trace, const double* normF2, const double* eps,
                     const int* rmax, const int* rfix, double u_eff, int n_eig, int n_flag, int B, int* out,
                     cudaStream_t s) {
  k_rank_batch<<<(B + 3) / 4, 128, 0, s>>>(lam, m, trace, normF2, eps, rmax, rfix, u_eff, n_eig, n_flag, B, out);
  TK_LAUNCH("k_rank_batch");
}

void rank_rule(const double* lam, int m, const double* trace, const double* normF2, double eps,
               int rmax, int rfix, double u_eff, int n, int* rank_out, cudaStream_t s) {
  k_rank<<<1, 32, 0, s>>>(lam, m, trace, normF2, eps, rmax, rfix, u_eff, n, rank_out);
  TK_LAUNCH("k_rank");
}

}  // namespace tk
