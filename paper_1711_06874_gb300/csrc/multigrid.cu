// Multigrid Tucker (Sec. 3.2): the factors found on one grid of a dyadic
// hierarchy carried to the next finer grid as the start of its Tucker-ALS
// sweeps.  Each column of U_k is a function sampled at the coarse points of
// axis k; it is sampled at the fine points by linear interpolation between
// the two coarse points around each one (continued linearly past the
// outermost pair), and the interpolated columns are then orthonormalised.
//
// Only the span of the started factors matters to the sweeps that follow:
// the update of mode k depends on the other two factors through the Gram of
// F_(k) (U_l (x) U_m), which an orthogonal change of basis inside U_l or U_m
// leaves unchanged, and the starting U_1 is never read.  So any orthonormal
// basis of the interpolated columns' span serves; this one is classical
// Gram-Schmidt applied twice (one re-orthogonalisation pass), in FP64.
//
// Work: n_f r^2 multiply-adds per mode (n_f <= 1024, r <= 88), a few
// microseconds next to a sweep.  One CTA per mode; the factor stays in
// global memory (L1/L2 resident), each row owned by one thread in the
// update phases.
#include <cuda_runtime.h>

#include "tk_internal.h"

namespace tk {
namespace {

constexpr int kProlongThreads = 512;
constexpr int kProlongWarps = kProlongThreads / 32;

struct ProlongMode {
  const double* Uc;  // n_c x r, row-major
  double* Uf;        // n_f x r, row-major
  int nc, nf, r;
};

struct ProlongDesc {
  ProlongMode m[3];
  int vertex;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fine point i in units of the coarse spacing, measured from the first
// coarse point, from the grids of Sec. 3.7 (Eq. grid_points):
//  cell-centred, n_f = 2 n_c: x_f(i) - x_c(0) = (i/2 - 1/4) h_c;
//  vertex, n_f - 1 = 2 (n_c - 1): x_f(i) - x_c(0) = (i/2) h_c.
// Both are exact in binary floating point.
__device__ __forceinline__ double coarse_position(int i, int vertex) {
  return vertex ? 0.5 * (double)i : 0.5 * (double)i - 0.25;
}

__global__ void __launch_bounds__(kProlongThreads) k_prolong_orth(ProlongDesc d) {
  TK_PDL_ENTRY();
  __shared__ double dots[kMgMaxRank];
  __shared__ double part[kProlongWarps];
  __shared__ double scale;
  // a select, not an indexed read of the parameter array (which would copy it to local memory)
  const ProlongMode md = blockIdx.x == 0 ? d.m[0] : (blockIdx.x == 1 ? d.m[1] : d.m[2]);
  const int nc = md.nc, nf = md.nf, r = md.r;
  double* U = md.Uf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // 1. interpolation; 2 <= n_c keeps j and j + 1 inside the coarse factor
  const long long total = (long long)nf * r;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = (int)(e / r), c = (int)(e % r);
    const double p = coarse_position(i, d.vertex);
    const int j = min(max((int)floor(p), 0), nc - 2);
    const double t = p - (double)j;
    U[e] = (1.0 - t) * md.Uc[(size_t)j * r + c] + t * md.Uc[(size_t)(j + 1) * r + c];
  }
  __syncthreads();

  // 2. classical Gram-Schmidt, twice per column
  for (int c = 0; c < r; ++c) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = warp; q < c; q += kProlongWarps) {
        double s = 0.0;
        for (int i = lane; i < nf; i += 32) s += U[(size_t)i * r + q] * U[(size_t)i * r + c];
        s = warp_sum(s);
        if (lane == 0) dots[q] = s;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        double v = U[(size_t)i * r + c];
        for (int q = 0; q < c; ++q) v -= dots[q] * U[(size_t)i * r + q];
        U[(size_t)i * r + c] = v;
      }
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      const double v = U[(size_t)i * r + c];
      s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) part[warp] = s;
    __syncthreads();
    if (warp == 0) {
      double v = lane < kProlongWarps ? part[lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) scale = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf; i += blockDim.x) U[(size_t)i * r + c] *= scale;
    __syncthreads();
  }
}

}  // namespace

void mg_prolong_orth(const double* const Uc[3], const int nc[3], double* const Uf[3], const int nf[3],
                     const int r[3], int vertex, cudaStream_t s) {
  ProlongDesc d{};
  for (int a = 0; a < 3; ++a) {
    if (nc[a] < 2 || nf[a] < nc[a] || r[a] < 1 || r[a] > kMgMaxRank)
      fail(TK_EINVAL, "multigrid prolongation: need 2 <= n_c <= n_f and 1 <= r <= 96");
    if (vertex ? (nf[a] - 1 != 2 * (nc[a] - 1)) : (nf[a] != 2 * nc[a]))
      fail(TK_EINVAL, "multigrid prolongation: the fine grid is not the dyadic refinement of the coarse one");
    d.m[a] = ProlongMode{Uc[a], Uf[a], nc[a], nf[a], r[a]};
  }
  d.vertex = vertex;
  launch_pdl("k_prolong_orth", k_prolong_orth, dim3(3), dim3(kProlongThreads), 0, s, d);
}

}  // namespace tk
