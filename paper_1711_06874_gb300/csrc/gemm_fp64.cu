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
// blockIdx.z: instance of a batch (tensor F + z sF, partials P + z nsplit npairs 64^2).
__global__ void __launch_bounds__(NT) k_gram_f64(const double* __restrict__ F, Unfold u, int nrows,
                                                  long long K, long long kc, int ntiles,
                                                  double* __restrict__ P, long long sF) {
  __shared__ double As[KS][TB + 1];
  __shared__ double Bs[KS][TB + 1];
  F += (long long)blockIdx.z * sF;
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
  double* out = P + (((long long)blockIdx.z * gridDim.y + split) * npairs + blockIdx.x) * TB * TB;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(ty * 4 + p) * TB + tx * 4 + q] = acc[p][q];
}

// Sum the K splits in index order and write both triangles of G, for B
// instances (G + b n^2).
__global__ void k_gram_reduce(const double* __restrict__ P, int nsplit, int ntiles, int n, int B,
                              double* __restrict__ G) {
  const int npairs = ntiles * (ntiles + 1) / 2;
  const long long per = (long long)npairs * TB * TB;
  const long long total = per * B;
  for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < total;
       e0 += (long long)gridDim.x * blockDim.x) {
    const long long b = e0 / per;
    const long long e = e0 - b * per;
    const double* Pb = P + b * nsplit * per;
    double* Gb = G + b * n * n;
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
    for (int sp = 0; sp < nsplit; ++sp) s += Pb[((long long)sp * npairs + pr) * TB * TB + rc];
    Gb[(long long)gi * n + gj] = s;
    Gb[(long long)gj * n + gi] = s;
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

size_t gram_f64_scratch_doubles(const int n[3], int mode, int B) {
  const GramPlan p = gram_plan(n, mode);
  return (size_t)B * p.nsplit * p.npairs * TB * TB;
}

// The plan depends on the shape only, so each instance's Gram is the same
// whatever the batch around it.
void gram_f64_batch(const double* F, const int n[3], int mode, int B, double* G, double* scratch,
                    cudaStream_t s) {
  const GramPlan p = gram_plan(n, mode);
  Unfold u{mode, n[0], n[1], n[2]};
  dim3 grid(p.npairs, p.nsplit, B);
  k_gram_f64<<<grid, NT, 0, s>>>(F, u, n[mode], p.K, p.kc, p.ntiles, scratch, (long long)n[0] * n[1] * n[2]);
  TK_LAUNCH("k_gram_f64");
  const long long total = (long long)p.npairs * TB * TB * B;
  k_gram_reduce<<<(unsigned)std::min<long long>((total + 255) / 256, 8192), 256, 0, s>>>(
      scratch, p.nsplit, p.ntiles, n[mode], B, G);
  TK_LAUNCH("k_gram_reduce");
}

void gram_f64(const double* F, const int n[3], int mode, double* G, double* scratch,
              cudaStream_t s) {
  gram_f64_batch(F, n, mode, 1, G, scratch, s);
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
  k_gram_f64<<<dim3(p.npairs, p.nsplit), NT, 0, s>>>(F, u, nn[mode], p.K, p.kc, p.ntiles, scratch, 0);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TK_ECUDA;
  const long long total = (long long)p.npairs * TB * TB;
  k_gram_reduce<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(
      scratch, p.nsplit, p.ntiles, nn[mode], 1, G);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TK_ECUDA;
  return TK_OK;
}

namespace tk {

// ---------------------------------------------------------------------------
// Strided batched GEMM.  Tile shapes (BM x BN, 16-deep K steps, 256 threads
// as 16 x 16, each thread BM/16 x BN/16 outputs) are picked from the output
// shape so that rank-sized dimensions do not waste a 64-wide tile; products
// with few outputs use one warp per output instead.
// ---------------------------------------------------------------------------
namespace {

template <int BM, int BN>
__device__ __forceinline__ void load_tiles(const GemmDesc& d, const double* A, const double* B, int i0, int j0, int k0,
                                           double (*As)[BM + 1], double (*Bs)[BN + 1]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < BM / 16; ++q) {
    const int e = t + 256 * q;
    int i, k;
    if (d.sAk == 1) {
      i = e / KS;
      k = e % KS;
    } else {
      k = e / BM;
      i = e % BM;
    }
    const int gi = i0 + i, gk = k0 + k;
    As[k][i] = (gi < d.M && gk < d.K) ? A[(long long)gi * d.sAi + (long long)gk * d.sAk] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < BN / 16; ++q) {
    const int e = t + 256 * q;
    int j, k;
    if (d.sBj == 1) {
      k = e / BN;
      j = e % BN;
    } else {
      j = e / KS;
      k = e % KS;
    }
    const int gj = j0 + j, gk = k0 + k;
    Bs[k][j] = (gj < d.N && gk < d.K) ? B[(long long)gk * d.sBk + (long long)gj * d.sBj] : 0.0;
  }
}

__device__ __forceinline__ void neum(double& s, double& c, double x) {
  const double t = s + x;
  c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
  s = t;
}

// Reference values of the error epilogue: an array in C's layout, or (for
// the cubic isotropic grid) the distinct-value table, F(ij, l) = T[q(s)] with
// s = a_i^2 + a_j^2 + a_l^2, a = 2 idx - (n - 1), row ij = i n + j.
struct ErrRef {
  const double* R;
  const double* T;
  int n;
  int even;
  __device__ __forceinline__ double at(const GemmDesc& d, const double* Rb, int i, int j) const {
    if (T == nullptr) return Rb[(long long)i * d.sCi + (long long)j * d.sCj];
    const int ai = 2 * (i / n) - (n - 1), aj = 2 * (i % n) - (n - 1), al = 2 * j - (n - 1);
    const int sq = ai * ai + aj * aj + al * al;
    return __ldg(T + (even ? (sq - 3) >> 3 : sq >> 2));
  }
};

// Operand offsets of batch entry z (outer index z / batch2, inner z % batch2;
// A's outer index through amap when given); returns C's offset.
__device__ __forceinline__ long long batch_offsets(const GemmDesc& d, long long z, const double*& A,
                                                   const double*& B) {
  const long long b1 = z / d.batch2, b2 = z - b1 * d.batch2;
  const long long ia = d.amap ? (long long)d.amap[b1] : b1;
  A = d.A + ia * d.sAb + b2 * d.sAb2;
  B = d.B + b1 * d.sBb + b2 * d.sBb2;
  return b1 * d.sCb + b2 * d.sCb2;
}

template <int BM, int BN, bool kErr>
__global__ void __launch_bounds__(NT) k_gemm_f64(GemmDesc d, ErrRef ref, double* __restrict__ partials) {
  TK_PDL_ENTRY();
  constexpr int RM = BM / 16, RN = BN / 16;
  __shared__ double As[KS][BM + 1];
  __shared__ double Bs[KS][BN + 1];
  const double* A;
  const double* B;
  const long long coff = batch_offsets(d, blockIdx.z, A, B);
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[RM][RN];
#pragma unroll
  for (int p = 0; p < RM; ++p)
#pragma unroll
    for (int q = 0; q < RN; ++q) acc[p][q] = 0.0;
  for (int k0 = 0; k0 < d.K; k0 += KS) {
    load_tiles<BM, BN>(d, A, B, i0, j0, k0, As, Bs);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      double a[RM], bb[RN];
#pragma unroll
      for (int p = 0; p < RM; ++p) a[p] = As[k][ty * RM + p];
#pragma unroll
      for (int q = 0; q < RN; ++q) bb[q] = Bs[k][tx * RN + q];
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RN; ++q) acc[p][q] = fma(a[p], bb[q], acc[p][q]);
    }
    __syncthreads();
  }
  if (!kErr) {
    double* C = d.C + coff;
#pragma unroll
    for (int p = 0; p < RM; ++p)
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        const int i = i0 + ty * RM + p, j = j0 + tx * RN + q;
        if (i < d.M && j < d.N) C[(long long)i * d.sCi + (long long)j * d.sCj] = acc[p][q];
      }
  } else {
    const double* Rb = ref.R ? ref.R + coff : nullptr;
    // plain FP64 sums over this thread's outputs; compensation starts at the tree
    double ds = 0.0, dc = 0.0, fs = 0.0, fc = 0.0;
#pragma unroll
    for (int p = 0; p < RM; ++p)
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        const int i = i0 + ty * RM + p, j = j0 + tx * RN + q;
        if (i < d.M && j < d.N) {
          const double r = ref.at(d, Rb, i, j);
          const double e = r - acc[p][q];
          ds = fma(e, e, ds);
          fs = fma(r, r, fs);
        }
      }
    // fixed-shape tree over the block's threads, compensation carried along
    __shared__ double red[4][NT];
    red[0][threadIdx.x] = ds;
    red[1][threadIdx.x] = dc;
    red[2][threadIdx.x] = fs;
    red[3][threadIdx.x] = fc;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        double s0 = red[0][threadIdx.x], c0 = red[1][threadIdx.x] + red[1][threadIdx.x + w];
        neum(s0, c0, red[0][threadIdx.x + w]);
        double s1 = red[2][threadIdx.x], c1 = red[3][threadIdx.x] + red[3][threadIdx.x + w];
        neum(s1, c1, red[2][threadIdx.x + w]);
        red[0][threadIdx.x] = s0;
        red[1][threadIdx.x] = c0;
        red[2][threadIdx.x] = s1;
        red[3][threadIdx.x] = c1;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const long long blin = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partials[4 * blin + 0] = red[0][0];
      partials[4 * blin + 1] = red[1][0];
      partials[4 * blin + 2] = red[2][0];
      partials[4 * blin + 3] = red[3][0];
    }
  }
}

// Sum of (R - C)^2 and R^2 partials: 1024 threads, each a Neumaier sum over a
// fixed stride of blocks, then a fixed tree.
__global__ void __launch_bounds__(1024) k_err_final(const double* part, long long nparts, double* out) {
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (long long b = threadIdx.x; b < nparts; b += blockDim.x) {
    neum(s0, c0, part[4 * b]);
    c0 += part[4 * b + 1];
    neum(s1, c1, part[4 * b + 2]);
    c1 += part[4 * b + 3];
  }
  __shared__ double red[4][1024];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = c0;
  red[2][threadIdx.x] = s1;
  red[3][threadIdx.x] = c1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a0 = red[0][threadIdx.x], a1 = red[1][threadIdx.x] + red[1][threadIdx.x + w];
      neum(a0, a1, red[0][threadIdx.x + w]);
      double b0 = red[2][threadIdx.x], b1 = red[3][threadIdx.x] + red[3][threadIdx.x + w];
      neum(b0, b1, red[2][threadIdx.x + w]);
      red[0][threadIdx.x] = a0;
      red[1][threadIdx.x] = a1;
      red[2][threadIdx.x] = b0;
      red[3][threadIdx.x] = b1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0] + red[1][0];
    out[1] = red[2][0] + red[3][0];
  }
}

// k_err_final for instance blockIdx.x of a batch (nparts partials each).
__global__ void __launch_bounds__(1024) k_err_final_batch(const double* part, long long nparts, double* out) {
  part += (long long)blockIdx.x * 4 * nparts;
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (long long b = threadIdx.x; b < nparts; b += blockDim.x) {
    neum(s0, c0, part[4 * b]);
    c0 += part[4 * b + 1];
    neum(s1, c1, part[4 * b + 2]);
    c1 += part[4 * b + 3];
  }
  __shared__ double red[4][1024];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = c0;
  red[2][threadIdx.x] = s1;
  red[3][threadIdx.x] = c1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a0 = red[0][threadIdx.x], a1 = red[1][threadIdx.x] + red[1][threadIdx.x + w];
      neum(a0, a1, red[0][threadIdx.x + w]);
      double b0 = red[2][threadIdx.x], b1 = red[3][threadIdx.x] + red[3][threadIdx.x + w];
      neum(b0, b1, red[2][threadIdx.x + w]);
      red[0][threadIdx.x] = a0;
      red[1][threadIdx.x] = a1;
      red[2][threadIdx.x] = b0;
      red[3][threadIdx.x] = b1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = red[0][0] + red[1][0];
    out[2 * blockIdx.x + 1] = red[2][0] + red[3][0];
  }
}

// One warp per output element; lanes stride over K, fixed shuffle tree.
__global__ void k_gemm_warp(GemmDesc d) {
  const long long per_batch = (long long)d.M * d.N;
  const long long total = per_batch * d.batch;
  const int lane = threadIdx.x & 31;
  for (long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; o < total;
       o += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long b = o / per_batch;
    const long long r = o - b * per_batch;
    const int i = (int)(r / d.N), j = (int)(r % d.N);
    const double* A;
    const double* B;
    const long long coff = batch_offsets(d, b, A, B);
    A += (long long)i * d.sAi;
    B += (long long)j * d.sBj;
    double acc = 0.0;
    for (int k = lane; k < d.K; k += 32) acc = fma(A[(long long)k * d.sAk], B[(long long)k * d.sBk], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) d.C[coff + (long long)i * d.sCi + (long long)j * d.sCj] = acc;
  }
}

// L lanes per output: lane q sums the terms k = q (mod L) as one FMA chain in
// k order, and the L chains are added in a fixed xor tree.  L = 32 for
// K >= 128 (short chains: these shapes are the large-n, few-instance,
// latency-bound solves) and L = 4 below (two additions of overhead per output:
// an FP64 warp instruction holds a sub-partition's FP64 unit for about 64
// cycles whatever the number of active lanes, which counts in large batches).
template <int L>
__global__ void k_gemm_lanes(GemmDesc d) {
  TK_PDL_ENTRY();
  const long long per_batch = (long long)d.M * d.N;
  const long long total = per_batch * d.batch;
  const int q = threadIdx.x & (L - 1);
  for (long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / L;
       o - (long long)((threadIdx.x & 31) / L) < total; o += ((long long)gridDim.x * blockDim.x) / L) {
    // every lane of a warp runs the shuffles: outputs past the end add zeros
    const bool live = o < total;
    double acc = 0.0;
    long long coff = 0;
    int i = 0, j = 0;
    if (live) {
      const long long b = o / per_batch;
      const long long r = o - b * per_batch;
      i = (int)(r / d.N);
      j = (int)(r % d.N);
      const double* A;
      const double* B;
      coff = batch_offsets(d, b, A, B);
      A += (long long)i * d.sAi;
      B += (long long)j * d.sBj;
      int k = q;
      // four terms per pass, loads first, FMAs in k order
      for (; k + 3 * L < d.K; k += 4 * L) {
        double a[4], bb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = A[(long long)(k + u * L) * d.sAk];
          bb[u] = B[(long long)(k + u * L) * d.sBk];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = fma(a[u], bb[u], acc);
      }
      for (; k < d.K; k += L) acc = fma(A[(long long)k * d.sAk], B[(long long)k * d.sBk], acc);
    }
#pragma unroll
    for (int off = 1; off < L; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (live && q == 0) d.C[coff + (long long)i * d.sCi + (long long)j * d.sCj] = acc;
  }
}

// Output tiles (BM x BN); every one sums each output in the same k order.
struct TileShape {
  int bm, bn;
};
constexpr TileShape kTiles[] = {{64, 64}, {128, 32}, {256, 16}, {32, 64}, {64, 32}, {128, 16}, {16, 128},
                                {32, 32}, {64, 16}, {16, 64}, {16, 16}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

// Largest tile that still fills a wave of CTAs with little padding; with too
// few outputs for a wave, the tile giving the most CTAs.
int pick_tile(const GemmDesc& d) {
  auto ctas = [&](int t) {
    return (long long)((d.M + kTiles[t].bm - 1) / kTiles[t].bm) * ((d.N + kTiles[t].bn - 1) / kTiles[t].bn) *
           d.batch;
  };
  auto waste = [&](int t) {
    const double pm = (double)((d.M + kTiles[t].bm - 1) / kTiles[t].bm) * kTiles[t].bm;
    const double pn = (double)((d.N + kTiles[t].bn - 1) / kTiles[t].bn) * kTiles[t].bn;
    return pm * pn / ((double)d.M * d.N);
  };
  for (int t = 0; t < kNumTiles; ++t)
    if (ctas(t) >= 152 && waste(t) <= 1.34) return t;
  int best = kNumTiles - 1;
  for (int t = 0; t < kNumTiles; ++t)
    if (waste(t) <= 2.0 && ctas(t) > ctas(best)) best = t;
  return best;
}

template <int BM, int BN>
dim3 grid_of(const GemmDesc& d) {
  return dim3((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, d.batch);
}

template <int BM, int BN, bool kErr>
void launch(const GemmDesc& d, const ErrRef& R, double* partials, cudaStream_t s) {
  launch_pdl("k_gemm_f64", k_gemm_f64<BM, BN, kErr>, dim3(grid_of<BM, BN>(d)), dim3(NT), 0, s, d, R, partials);
}

template <int I, bool kErr>
dim3 dispatch_at(int t, const GemmDesc& d, const ErrRef& R, double* partials, cudaStream_t s, bool run) {
  if constexpr (I < kNumTiles) {
    if (t == I) {
      if (run) launch<kTiles[I].bm, kTiles[I].bn, kErr>(d, R, partials, s);
      return grid_of<kTiles[I].bm, kTiles[I].bn>(d);
    }
    return dispatch_at<I + 1, kErr>(t, d, R, partials, s, run);
  } else {
    return dim3(0, 0, 0);
  }
}

template <bool kErr>
dim3 dispatch(const GemmDesc& d, const ErrRef& R, double* partials, cudaStream_t s, bool run) {
  return dispatch_at<0, kErr>(pick_tile(d), d, R, partials, s, run);
}

}  // namespace

void gemm_f64(const GemmDesc& d, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return;
  const dim3 g = dispatch<false>(d, ErrRef{}, nullptr, s, false);
  const long long ctas = (long long)g.x * g.y * g.z;
  const long long outs = (long long)d.M * d.N * d.batch;
  // fixed-order products: several lanes per output for small per-entry shapes
  // (their number set by K), tiles otherwise; the choice depends on the per-entry shape alone (never on
  // the batch), so an entry's result does not either
  if (d.fixed_order) {
    if (!d.tiles_only && (long long)d.M * d.N <= 4096 && d.K >= 32) {
      const int L = d.K >= 128 ? 32 : 4;
      const long long threads = (long long)L * outs;
      const unsigned blocks = (unsigned)std::min<long long>((threads + 255) / 256, 8192);
      if (L == 4)
        launch_pdl("k_gemm_lanes", k_gemm_lanes<4>, dim3(blocks), dim3(256), 0, s, d);
      else
        launch_pdl("k_gemm_lanes", k_gemm_lanes<32>, dim3(blocks), dim3(256), 0, s, d);
      return;
    }
    dispatch<false>(d, ErrRef{}, nullptr, s, true);
    return;
  }
  // one warp per output when the outputs are few
  const bool warp = ctas < 76 && outs <= (1LL << 18);
  if (warp) {
    // few tiles: one warp per output keeps every SM busy
    const long long warps = outs;
    const unsigned blocks = (unsigned)std::min<long long>((warps + 7) / 8, 4096);
    k_gemm_warp<<<blocks, 256, 0, s>>>(d);
    TK_LAUNCH("k_gemm_warp");
    return;
  }
  dispatch<false>(d, ErrRef{}, nullptr, s, true);
}

// ---------------------------------------------------------------------------
// Second TTM of the isotropic core, T2(a, k, c) = sum_i V(i, a) T1(i, k, c).
// F is symmetric under permutations of its indices and the three modes share
// V, so T2(a, k, c) = sum_{i,l} V(i, a) V(l, c) F(i, k, l) = T2(c, k, a): only
// a <= c is formed and mirrored (R (R + 1) / 2 of the R^2 pairs).  One CTA per
// (k, instance) holds V and T1(:, k, :) in shared memory; each output is four
// FMA chains over interleaved i (i = q mod 4), added in a fixed order.
namespace {

constexpr int kTtm2Threads = 256;

__global__ void __launch_bounds__(kTtm2Threads) k_ttm2_sym(const double* __restrict__ V, const double* __restrict__ T1,
                                                          double* __restrict__ T2, int h, int R) {
  TK_PDL_ENTRY();
  extern __shared__ double sm2[];
  double* Vs = sm2;          // [i][a]
  double* Ts = sm2 + h * R;  // [i][c]
  const int k = blockIdx.x, pos = blockIdx.y;
  V += (size_t)pos * h * R;
  T1 += (size_t)pos * h * h * R;
  T2 += (size_t)pos * R * h * R;
  // both operands in 16-byte asynchronous copies, all in flight at once: V
  // whole, T1(:, k, :) as h runs of R values (R a multiple of 4, so every run
  // starts on a 16-byte boundary)
  const int vp = h * R / 2, rp = R / 2;
  for (int e = threadIdx.x; e < 2 * vp; e += blockDim.x) {
    const double* src;
    double* dst;
    if (e < vp) {
      src = V + 2 * e;
      dst = Vs + 2 * e;
    } else {
      const int f = e - vp, i = f / rp, q = f - i * rp;
      src = T1 + ((size_t)i * h + k) * R + 2 * q;
      dst = Ts + (size_t)i * R + 2 * q;
    }
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int npairs = R * (R + 1) / 2;
  const int items = 4 * npairs, span = (items + 31) & ~31;  // whole warps in every pass
  for (int t = threadIdx.x; t < span; t += blockDim.x) {
    const bool valid = t < items;
    const int p = valid ? t >> 2 : 0, q = t & 3;
    // pair p -> (a, c), a <= c, row by row
    int a = 0, rem = p;
    while (rem >= R - a) {
      rem -= R - a;
      ++a;
    }
    const int c = a + rem;
    double acc = 0.0;
    if (valid)
      for (int i = q; i < h; i += 4) acc = fma(Vs[i * R + a], Ts[i * R + c], acc);
    // the four chains of an output sit in four adjacent lanes: a fixed tree
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (valid && q == 0) {
      T2[((size_t)a * h + k) * R + c] = acc;
      T2[((size_t)c * h + k) * R + a] = acc;
    }
  }
}

}  // namespace

size_t ttm2_sym_smem(int h, int R) { return sizeof(double) * 2 * (size_t)h * R; }

bool ttm2_sym_supported(int h, int R) { return R % 4 == 0 && ttm2_sym_smem(h, R) <= 96 * 1024; }

void ttm2_sym_batch(const double* V, const double* T1, double* T2, int h, int R, int cnt, cudaStream_t s) {
  if (!ttm2_sym_supported(h, R)) fail(TK_EINVAL, "ttm2_sym: shape out of range");
  if ((((uintptr_t)V | (uintptr_t)T1) & 15) != 0) fail(TK_EINVAL, "ttm2_sym: operands not 16-byte aligned");
  once_per_device((const void*)&k_ttm2_sym, [] {
    TK_CUDA(cudaFuncSetAttribute(k_ttm2_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
  });
  launch_pdl("k_ttm2_sym", k_ttm2_sym, dim3(h, cnt), dim3(kTtm2Threads), ttm2_sym_smem(h, R), s, V, T1, T2, h, R);
}

// ---------------------------------------------------------------------------
// Error of a rank-K product against a reference: sum (R - X)^2 and sum R^2
// with X = W Ut^T (W: M x K, ld K; Ut: N x K, ld K; R: M x N row-major) for a
// small K.  Each CTA takes 64 rows and 128 columns; W's rows and Ut's rows
// (transposed) sit in shared memory; every thread forms 32 outputs as K-long
// FMA chains and accumulates the two sums; the block partials go through the
// same fixed-order final sum as the GEMM epilogue.
// ---------------------------------------------------------------------------
namespace {

constexpr int kErrRows = 64, kErrCols = 128;

__global__ void __launch_bounds__(256) k_err_lowrank(const double* __restrict__ W, const double* __restrict__ Ut,
                                                     const double* __restrict__ R, int M, int N, int K,
                                                     double* __restrict__ partials, long long sW, long long sU,
                                                     long long sR, const int* __restrict__ amap) {
  extern __shared__ double es[];
  // instance blockIdx.z of a batch
  W += (long long)blockIdx.z * sW;
  Ut += (long long)blockIdx.z * sU;
  R += (amap ? (long long)amap[blockIdx.z] : (long long)blockIdx.z) * sR;
  partials += (long long)blockIdx.z * 4 * gridDim.x * gridDim.y;
  double* Ws = es;                   // [64][K]
  double* Us = es + kErrRows * K;    // [K][128]
  const int m0 = blockIdx.y * kErrRows, n0 = blockIdx.x * kErrCols;
  for (int e = threadIdx.x; e < kErrRows * K; e += blockDim.x) {
    const int i = e / K, k = e - i * K;
    Ws[e] = (m0 + i < M) ? W[(long long)(m0 + i) * K + k] : 0.0;
  }
  for (int e = threadIdx.x; e < kErrCols * K; e += blockDim.x) {
    const int c = e / K, k = e - c * K;
    Us[k * kErrCols + c] = (n0 + c < N) ? Ut[(long long)(n0 + c) * K + k] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x & (kErrCols - 1), r0 = threadIdx.x >> 7;  // 2 row phases
  double ds = 0.0, fs = 0.0;
  if (n0 + c < N) {
    // four rows at a time: independent FMA chains
    for (int i = r0; i < kErrRows; i += 8) {
      const double* w0 = Ws + i * K;
      double x[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < K; ++k) {
        const double u = Us[k * kErrCols + c];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = fma(w0[2 * q * K + k], u, x[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + i + 2 * q;
        if (row < M) {
          const double r = R[(long long)row * N + n0 + c];
          const double e = r - x[q];
          ds = fma(e, e, ds);
          fs = fma(r, r, fs);
        }
      }
    }
  }
  // fixed-shape tree over the block, compensation carried along
  __shared__ double red[4][256];
  red[0][threadIdx.x] = ds;
  red[1][threadIdx.x] = 0.0;
  red[2][threadIdx.x] = fs;
  red[3][threadIdx.x] = 0.0;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double s0 = red[0][threadIdx.x], c0 = red[1][threadIdx.x] + red[1][threadIdx.x + w];
      neum(s0, c0, red[0][threadIdx.x + w]);
      double s1 = red[2][threadIdx.x], c1 = red[3][threadIdx.x] + red[3][threadIdx.x + w];
      neum(s1, c1, red[2][threadIdx.x + w]);
      red[0][threadIdx.x] = s0;
      red[1][threadIdx.x] = c0;
      red[2][threadIdx.x] = s1;
      red[3][threadIdx.x] = c1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long blin = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partials[4 * blin + 0] = red[0][0];
    partials[4 * blin + 1] = red[1][0];
    partials[4 * blin + 2] = red[2][0];
    partials[4 * blin + 3] = red[3][0];
  }
}

}  // namespace

size_t err_lowrank_partials(int M, int N) {
  return 4ull * ((N + kErrCols - 1) / kErrCols) * ((M + kErrRows - 1) / kErrRows);
}

void err_lowrank_f64(const double* W, const double* Ut, const double* R, int M, int N, int K, double* partials,
                     double* out_dev, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)(kErrRows + kErrCols) * K;
  if (K < 1 || smem > 200 * 1024) fail(TK_EINVAL, "err_lowrank: K out of range");
  once_per_device((const void*)&k_err_lowrank, [] {
    TK_CUDA(cudaFuncSetAttribute(k_err_lowrank, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  const dim3 grid((N + kErrCols - 1) / kErrCols, (M + kErrRows - 1) / kErrRows);
  k_err_lowrank<<<grid, 256, smem, s>>>(W, Ut, R, M, N, K, partials, 0, 0, 0, nullptr);
  TK_LAUNCH("k_err_lowrank");
  k_err_final<<<1, 1024, 0, s>>>(partials, (long long)grid.x * grid.y, out_dev);
  TK_LAUNCH("k_err_final");
}

void err_lowrank_batch(const double* W, long long sW, const double* Ut, long long sU, const double* R, long long sR,
                       const int* amap, int M, int N, int K, int B, double* partials, double* out_dev,
                       cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)(kErrRows + kErrCols) * K;
  if (K < 1 || smem > 200 * 1024) fail(TK_EINVAL, "err_lowrank: K out of range");
  once_per_device((const void*)&k_err_lowrank, [] {
    TK_CUDA(cudaFuncSetAttribute(k_err_lowrank, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  });
  const dim3 grid((N + kErrCols - 1) / kErrCols, (M + kErrRows - 1) / kErrRows, B);
  k_err_lowrank<<<grid, 256, smem, s>>>(W, Ut, R, M, N, K, partials, sW, sU, sR, amap);
  TK_LAUNCH("k_err_lowrank");
  k_err_final_batch<<<B, 1024, 0, s>>>(partials, (long long)grid.x * grid.y, out_dev);
  TK_LAUNCH("k_err_final_batch");
}

size_t gemm_err_partials(const GemmDesc& d) {
  const dim3 g = dispatch<true>(d, ErrRef{}, nullptr, nullptr, false);
  return 4ull * g.x * g.y * g.z;
}

void gemm_f64_err(const GemmDesc& d, const double* R, const double* table, int table_n, double* partials,
                  double* out_dev, cudaStream_t s) {
  ErrRef ref{R, table, table_n, table_n % 2 == 0};
  const dim3 g = dispatch<true>(d, ref, partials, s, true);
  k_err_final<<<1, 1024, 0, s>>>(partials, (long long)g.x * g.y * g.z, out_dev);
  TK_LAUNCH("k_err_final");
}

}  // namespace tk
