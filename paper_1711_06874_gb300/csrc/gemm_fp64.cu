// FP64 contractions on the CUDA cores: the plain path's Gram (Sec. 3.2:
// G_k = A_(k) A_(k)^T, read in place from F for every unfolding), and a
// strided batched GEMM used by the eigensolver, the TTM chain of the core
// (Sec. 3.1: B = F x_1 U1^T x_2 U2^T x_3 U3^T) and the reconstruction error of
// Eq. (FNorm).  64 x 64 output tiles, 16-deep K steps staged in shared memory,
// 4 x 4 outputs per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "tk_internal.h"

namespace tk {

namespace {

constexpr int TB = 64;   // tile edge
constexpr int KS = 16;   // K step
constexpr int NT = 256;  // threads per block

// Address of A_(mode)(row, c) inside F (n1 x n2 x n3 row-major).
struct Unfold {
  int mode;
  int n1, n2, n3;
  __device__ __forceinline__ long long at(int row, long long c) const {
    if (mode == 0) return (long long)row * n2 * n3 + c;
    if (mode == 1) {
      const long long i = c / n3, l = c - i * n3;
      return (i * n2 + row) * n3 + l;
    }
    return c * n3 + row;
  }
};

// Tile loader for the unfolding: fills S[KS][TB] with A(r0 + r, c0 + k).
__device__ __forceinline__ void load_unfold_tile(const double* __restrict__ F, const Unfold& u,
                                                 int nrows, long long K, int r0, long long c0,
                                                 double (*S)[TB + 1]) {
  const int t = threadIdx.x;
  if (u.mode == 2) {
    // rows are contiguous: 16 threads cover 64 rows of one c
    const int kk = t >> 4, rq = (t & 15) * 4;
    const long long c = c0 + kk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + rq + q;
      S[kk][rq + q] = (r < nrows && c < K) ? __ldg(F + u.at(r, c)) : 0.0;
    }
  } else {
    const int r = t >> 2, kq = (t & 3) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long c = c0 + kq + q;
      S[kq + q][r] = (r0 + r < nrows && c < K) ? __ldg(F + u.at(r0 + r, c)) : 0.0;
    }
  }
}

// One (tile pair, K split) of the Gram; partial 64 x 64 block to P.
__global__ void __launch_bounds__(NT) k_gram_f64(const double* __restrict__ F, Unfold u, int nrows,
                                                  long long K, long long kc, int ntiles,
                                                  double* __restrict__ P) {
  __shared__ double As[KS][TB + 1];
  __shared__ double Bs[KS][TB + 1];
  // tile pair (ti <= tj) from the linear index
  int t = blockIdx.x, ti = 0;
  while (t >= ntiles - ti) {
    t -= ntiles - ti;
    ++ti;
  }
  const int tj = ti + t;
  const int split = blockIdx.y;
  const long long kb = (long long)split * kc;
  const long long ke = (kb + kc < K) ? kb + kc : K;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (long long c0 = kb; c0 < ke; c0 += KS) {
    load_unfold_tile(F, u, nrows, ke, ti * TB, c0, As);
    load_unfold_tile(F, u, nrows, ke, tj * TB, c0, Bs);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty * 4 + q];
        b[q] = Bs[k][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  const int npairs = ntiles * (ntiles + 1) / 2;
  double* out = P + ((long long)split * npairs + blockIdx.x) * TB * TB;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(ty * 4 + p) * TB + tx * 4 + q] = acc[p][q];
}

// Sum the K splits in index order and write both triangles of G.
__global__ void k_gram_reduce(const double* __restrict__ P, int nsplit, int ntiles, int n,
                              double* __restrict__ G) {
  const int npairs = ntiles * (ntiles + 1) / 2;
  const long long total = (long long)npairs * TB * TB;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int pr = (int)(e / (TB * TB));
    const int rc = (int)(e % (TB * TB));
    int t = pr, ti = 0;
    while (t >= ntiles - ti) {
      t -= ntiles - ti;
      ++ti;
    }
    const int tj = ti + t;
    const int gi = ti * TB + rc / TB, gj = tj * TB + rc % TB;
    if (gi >= n || gj >= n) continue;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += P[((long long)sp * npairs + pr) * TB * TB + rc];
    G[(long long)gi * n + gj] = s;
    G[(long long)gj * n + gi] = s;
  }
}

struct GramPlan {
  int ntiles, npairs, nsplit;
  long long K, kc;
};

GramPlan gram_plan(const int n[3], int mode) {
  GramPlan p;
  const int nr = n[mode];
  p.K = (long long)n[0] * n[1] * n[2] / nr;
  p.ntiles = (nr + TB - 1) / TB;
  p.npairs = p.ntiles * (p.ntiles + 1) / 2;
  const long long want = std::max<long long>(1, (4LL * 152 + p.npairs - 1) / p.npairs);
  const long long maxs = std::max<long long>(1, p.K / 256);
  p.nsplit = (int)std::min(want, maxs);
  p.kc = ((p.K + p.nsplit - 1) / p.nsplit + KS - 1) / KS * KS;
  p.nsplit = (int)((p.K + p.kc - 1) / p.kc);
  return p;
}

}  // namespace

size_t gram_f64_scratch_doubles(const int n[3], int mode) {
  const GramPlan p = gram_plan(n, mode);
  return (size_t)p.nsplit * p.npairs * TB * TB;
}

void gram_f64(const double* F, const int n[3], int mode, double* G, double* scratch,
              cudaStream_t s) {
  const GramPlan p = gram_plan(n, mode);
  Unfold u{mode, n[0], n[1], n[2]};
  dim3 grid(p.npairs, p.nsplit);
  k_gram_f64<<<grid, NT, 0, s>>>(F, u, n[mode], p.K, p.kc, p.ntiles, scratch);
  TK_LAUNCH("k_gram_f64");
  const long long total = (long long)p.npairs * TB * TB;
  k_gram_reduce<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(
      scratch, p.nsplit, p.ntiles, n[mode], G);
  TK_LAUNCH("k_gram_reduce");
}

// ---------------------------------------------------------------------------
// Allocation-free FP64 Gram (tk_gram_noalloc).
//
// Same kernels and arithmetic as gram_f64, but the split-K partial sums live
// in a fixed file-scope device array instead of caller- or library-allocated
// memory, for callers that must not allocate device memory.  Every GPU that
// loads the library holds this array (8 MiB) until the process exits.  In
// host code `g_gram_scratch` only names a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernel.  The partial blocks are written
// in full before they are read, so nothing needs clearing between calls; two
// calls whose work overlaps on the GPU share the array and race.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;  // 8 MiB
static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

}  // namespace tk

extern "C" int tk_gram_noalloc(const double* F, const int32_t n[3], int mode, double* G, void* stream) {
  using namespace tk;
  if (!F || !G || !n || mode < 0 || mode > 2) return TK_EINVAL;
  int nn[3] = {n[0], n[1], n[2]};
  for (int a = 0; a < 3; ++a)
    if (nn[a] < 1 || nn[a] > 1024) return TK_EINVAL;  // n outside [1, 1024]
  GramPlan p = gram_plan(nn, mode);
  const size_t per_split = (size_t)p.npairs * TB * TB;
  if (per_split > kNoAllocScratchDoubles) return TK_EINVAL;  // cannot happen for n <= 1024
  if ((size_t)p.nsplit * per_split > kNoAllocScratchDoubles) {
    // fewer, longer K splits so that the partial sums fit the fixed array
    const long long cap = (long long)(kNoAllocScratchDoubles / per_split);
    p.kc = ((p.K + cap - 1) / cap + KS - 1) / KS * KS;
    p.nsplit = (int)((p.K + p.kc - 1) / p.kc);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TK_ECUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_gram_scratch) != cudaSuccess || !addr) {
        cudaGetLastError();
        return TK_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(addr);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Unfold u{mode, nn[0], nn[1], nn[2]};
  k_gram_f64<<<dim3(p.npairs, p.nsplit), NT, 0, s>>>(F, u, nn[mode], p.K, p.kc, p.ntiles, scratch);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TK_ECUDA;
  const long long total = (long long)p.npairs * TB * TB;
  k_gram_reduce<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(
      scratch, p.nsplit, p.ntiles, nn[mode], G);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TK_ECUDA;
  return TK_OK;
}

namespace tk {

// ---------------------------------------------------------------------------
// Strided batched GEMM.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ void load_a_tile(const GemmDesc& d, const double* A, int i0, int k0,
                                            double (*S)[TB + 1]) {
  const int t = threadIdx.x;
  if (d.sAk == 1) {
    const int i = t >> 2, kq = (t & 3) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + kq + q;
      S[kq + q][i] = (i0 + i < d.M && k < d.K) ? A[(long long)(i0 + i) * d.sAi + k] : 0.0;
    }
  } else {
    const int kk = t >> 4, iq = (t & 15) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + iq + q, k = k0 + kk;
      S[kk][iq + q] = (i < d.M && k < d.K) ? A[(long long)i * d.sAi + (long long)k * d.sAk] : 0.0;
    }
  }
}

__device__ __forceinline__ void load_b_tile(const GemmDesc& d, const double* B, int k0, int j0,
                                            double (*S)[TB + 1]) {
  const int t = threadIdx.x;
  if (d.sBk == 1 && d.sBj != 1) {
    const int j = t >> 2, kq = (t & 3) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + kq + q;
      S[kq + q][j] = (j0 + j < d.N && k < d.K) ? B[k + (long long)(j0 + j) * d.sBj] : 0.0;
    }
  } else {
    const int kk = t >> 4, jq = (t & 15) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + jq + q, k = k0 + kk;
      S[kk][jq + q] = (j < d.N && k < d.K) ? B[(long long)k * d.sBk + (long long)j * d.sBj] : 0.0;
    }
  }
}

template <bool kErr>
__global__ void __launch_bounds__(NT) k_gemm_f64(GemmDesc d, const double* __restrict__ R,
                                                  double* __restrict__ partials) {
  __shared__ double As[KS][TB + 1];
  __shared__ double Bs[KS][TB + 1];
  const int b = blockIdx.z;
  const double* A = d.A + (long long)b * d.sAb;
  const double* B = d.B + (long long)b * d.sBb;
  const int i0 = blockIdx.y * TB, j0 = blockIdx.x * TB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < d.K; k0 += KS) {
    load_a_tile(d, A, i0, k0, As);
    load_b_tile(d, B, k0, j0, Bs);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      double a[4], bb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty * 4 + q];
        bb[q] = Bs[k][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bb[q], acc[p][q]);
    }
    __syncthreads();
  }
  if (!kErr) {
    double* C = d.C + (long long)b * d.sCb;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
        if (i < d.M && j < d.N) C[(long long)i * d.sCi + (long long)j * d.sCj] = acc[p][q];
      }
  } else {
    const double* Rb = R + (long long)b * d.sCb;
    double ds = 0.0, dc = 0.0, fs = 0.0, fc = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
        if (i < d.M && j < d.N) {
          const double r = Rb[(long long)i * d.sCi + (long long)j * d.sCj];
          const double e = r - acc[p][q];
          double t = ds + e * e;
          dc += (fabs(ds) >= e * e) ? (ds - t) + e * e : (e * e - t) + ds;
          ds = t;
          t = fs + r * r;
          fc += (fabs(fs) >= r * r) ? (fs - t) + r * r : (r * r - t) + fs;
          fs = t;
        }
      }
    __shared__ double red[4][NT];
    red[0][threadIdx.x] = ds;
    red[1][threadIdx.x] = dc;
    red[2][threadIdx.x] = fs;
    red[3][threadIdx.x] = fc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
      for (int t = 0; t < NT; ++t) {
        double v = red[0][t], tt = s0 + v;
        c0 += (fabs(s0) >= fabs(v)) ? (s0 - tt) + v : (v - tt) + s0;
        s0 = tt;
        c0 += red[1][t];
        v = red[2][t];
        tt = s1 + v;
        c1 += (fabs(s1) >= fabs(v)) ? (s1 - tt) + v : (v - tt) + s1;
        s1 = tt;
        c1 += red[3][t];
      }
      const long long blin = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partials[4 * blin + 0] = s0;
      partials[4 * blin + 1] = c0;
      partials[4 * blin + 2] = s1;
      partials[4 * blin + 3] = c1;
    }
  }
}

__global__ void k_err_final(const double* part, long long nparts, double* out) {
  if (threadIdx.x != 0) return;
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (long long b = 0; b < nparts; ++b) {
    double v = part[4 * b], t = s0 + v;
    c0 += (fabs(s0) >= fabs(v)) ? (s0 - t) + v : (v - t) + s0;
    s0 = t;
    c0 += part[4 * b + 1];
    v = part[4 * b + 2];
    t = s1 + v;
    c1 += (fabs(s1) >= fabs(v)) ? (s1 - t) + v : (v - t) + s1;
    s1 = t;
    c1 += part[4 * b + 3];
  }
  out[0] = s0 + c0;
  out[1] = s1 + c1;
}

dim3 gemm_grid(const GemmDesc& d) { return dim3((d.N + TB - 1) / TB, (d.M + TB - 1) / TB, d.batch); }

}  // namespace

void gemm_f64(const GemmDesc& d, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  k_gemm_f64<false><<<gemm_grid(d), NT, 0, s>>>(d, nullptr, nullptr);
  TK_LAUNCH("k_gemm_f64");
}

size_t gemm_err_partials(const GemmDesc& d) {
  const dim3 g = gemm_grid(d);
  return 4ull * g.x * g.y * g.z;
}

void gemm_f64_err(const GemmDesc& d, const double* R, double* partials, double* out_dev,
                  cudaStream_t s) {
  const dim3 g = gemm_grid(d);
  k_gemm_f64<true><<<g, NT, 0, s>>>(d, R, partials);
  TK_LAUNCH("k_gemm_f64_err");
  k_err_final<<<1, 32, 0, s>>>(partials, (long long)g.x * g.y * g.z, out_dev);
  TK_LAUNCH("k_err_final");
}

}  // namespace tk
