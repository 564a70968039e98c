// (a) Sampling the covariance on the grid: the collocation tensor of Sec. 3.7,
//     F[i1][i2][i3] = C(x_i1, x_i2, x_i3), with C of Sec. 2.2 (Matern), the
//     p-Slater function of Eq. (exp_p) or the Gaussian limit.
//
// Distinct-value table.  On both grid kinds the coordinate of index i is
// x_i = h (2i - (n-1)) with h = b/n (cell-centred) or b/(n-1) (vertex), so on
// a cubic grid with isotropic ell, r^2 = h^2 s with the integer
// s = a_i^2 + a_j^2 + a_k^2, a = 2i - (n-1).  For even n every a is odd and
// s = 3 (mod 8); for odd n every a is even and s = 0 (mod 4).  The kernel is
// therefore evaluated once per admissible s (about n^2 / 3 values instead of
// n^3), and the tensor is a gather from that table.  Anisotropic ell or a
// non-cubic grid use the per-point kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "nu_consts.h"
#include "slices.cuh"
#include "tk_internal.h"

namespace tk {

KernelDev make_kernel_dev(const tk_kernel& k) {
  KernelDev d{};
  d.kind = k.kind;
  d.sigma2 = k.sigma2;
  d.p = k.p;
  for (int a = 0; a < 3; ++a) d.inv_ell[a] = 1.0 / k.ell[a];
  d.sqrt2nu = (k.kind == TK_MATERN) ? std::sqrt(2.0 * k.nu) : 0.0;
  d.nuc = make_nu_consts(k.kind == TK_MATERN || k.kind == TK_MATERN_SD ? k.nu : 0.5);
  return d;
}

GridDev make_grid_dev(const tk_grid& g) {
  GridDev d{};
  for (int a = 0; a < 3; ++a) {
    const int n = g.n[a];
    const double b = g.b[a];
    if (g.kind == TK_VERTEX) {
      d.ax[a].dx = 2.0 * b / (double)(n - 1);
      d.ax[a].x0 = -b;
    } else {
      d.ax[a].dx = 2.0 * b / (double)n;
      d.ax[a].x0 = -b + 0.5 * d.ax[a].dx;
    }
    d.ax[a].n = n;
  }
  return d;
}

bool table_applicable(const tk_kernel& k, const tk_grid& g) {
  return g.n[0] == g.n[1] && g.n[1] == g.n[2] && g.b[0] == g.b[1] && g.b[1] == g.b[2] &&
         k.ell[0] == k.ell[1] && k.ell[1] == k.ell[2];
}

// Covariance as a function of the scaled squared distance r_A^2.
__device__ __forceinline__ double cov_value(const KernelDev& k, double ra2) {
  const double ra = sqrt(ra2);
  if (k.kind == TK_MATERN) return tk_matern_z(k.nuc, k.sigma2, k.sqrt2nu * ra);
  if (k.kind == TK_SLATER_P) return (ra2 == 0.0) ? k.sigma2 : k.sigma2 * exp(-pow(ra, k.p));
  // Eq. (SD_matern), d = 3: sigma2 (alpha^2 + r_A^2)^-(nu + 3/2)
  if (k.kind == TK_MATERN_SD) return k.sigma2 * exp(-(k.nuc.nu + 1.5) * log(fma(k.p, k.p, ra2)));
  return k.sigma2 * exp(-ra2);
}

static inline long long table_size(int n) {
  if (n % 2 == 0) return (3LL * (n - 1) * (n - 1) - 3) / 8 + 1;
  const long long h = (n - 1) / 2;
  return 3 * h * h + 1;
}

void set_table_split(KernelDev& d, const tk_grid& g) {
  d.tsplit = 0;
  if (d.kind != TK_MATERN) return;
  const int n = g.n[0];
  const double hstep = (g.kind == TK_VERTEX) ? g.b[0] / (double)(n - 1) : g.b[0] / (double)n;
  const double zs = d.sqrt2nu * hstep * d.inv_ell[0];  // z = zs sqrt(s) for table entry s
  if (!(zs > 0.0)) return;
  const double thr = (1.5 / zs) * (1.5 / zs);         // s beyond which z > 1.5
  const double qb = (n % 2 == 0) ? std::floor((thr - 3.0) / 8.0) + 1.0 : std::floor(thr / 4.0) + 1.0;
  const double Q = (double)table_size(n);
  d.tsplit = (long long)std::min(std::max(qb, 0.0), Q);
}

size_t eval_scratch_doubles(const tk_kernel& k, const tk_grid& g) {
  return table_applicable(k, g) ? (size_t)table_size(g.n[0]) : 0;
}

// T[q] = C(h sqrt(s) / ell) with s = 8q + 3 (even n) or s = 4q (odd n).
__global__ void k_table(KernelDev k, double hs, int even, long long Q, double* T) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Q;
       q += (long long)gridDim.x * blockDim.x) {
    const double s = even ? (double)(8 * q + 3) : (double)(4 * q);
    T[q] = cov_value(k, hs * hs * s);
  }
}

// Sum of squares of one row across the block, fixed tree (deterministic).
__device__ __forceinline__ double block_row_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// F[i][j][l] = T[q(s)], one block per (i, j) row at a time (grid-stride),
// threads along l.  Each block sums the squares of everything it wrote and
// leaves one partial per block in part[blockIdx.x].
__global__ void k_gather(const double* __restrict__ T, int n, int even, double* __restrict__ F,
                         double* __restrict__ part) {
  __shared__ double red[32];
  const long long rows = (long long)n * n;
  double sq = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int i = (int)(row / n), j = (int)(row % n);
    const int ai = 2 * i - (n - 1), aj = 2 * j - (n - 1);
    const int sij = ai * ai + aj * aj;
    double* out = F + row * n;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      const int al = 2 * l - (n - 1);
      const int s = sij + al * al;
      const double v = __ldg(T + (even ? (s - 3) >> 3 : s >> 2));
      out[l] = v;
      sq = fma(v, v, sq);
    }
  }
  const double t = block_row_sum(sq, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Per-point evaluation for anisotropic ell or non-cubic grids (block sums of
// squares as in k_gather).
__global__ void k_eval_general(KernelDev k, GridDev g, double* __restrict__ F, double* __restrict__ part) {
  __shared__ double red[32];
  const int n1 = g.ax[0].n, n2 = g.ax[1].n, n3 = g.ax[2].n;
  const long long rows = (long long)n1 * n2;
  double sq = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int i = (int)(row / n2), j = (int)(row % n2);
    const double u = (g.ax[0].x0 + i * g.ax[0].dx) * k.inv_ell[0];
    const double v = (g.ax[1].x0 + j * g.ax[1].dx) * k.inv_ell[1];
    const double uv = u * u + v * v;
    for (int l = threadIdx.x; l < n3; l += blockDim.x) {
      const double w = (g.ax[2].x0 + l * g.ax[2].dx) * k.inv_ell[2];
      const double val = cov_value(k, uv + w * w);
      F[row * n3 + l] = val;
      sq = fma(val, val, sq);
    }
  }
  const double t = block_row_sum(sq, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// |F|^2 = sum of the row sums: 1024 threads, Neumaier over a fixed stride,
// then a fixed tree.
__global__ void __launch_bounds__(1024) k_rowsq_final(const double* __restrict__ rowsq, long long rows,
                                                      double* out) {
  __shared__ double rs[1024], rc[1024];
  double s = 0.0, c = 0.0;
  for (long long r = threadIdx.x; r < rows; r += blockDim.x) {
    const double x = rowsq[r], t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a = rs[threadIdx.x], ac = rc[threadIdx.x] + rc[threadIdx.x + w];
      const double x = rs[threadIdx.x + w], t = a + x;
      ac += (fabs(a) >= fabs(x)) ? (a - t) + x : (x - t) + a;
      rs[threadIdx.x] = t;
      rc[threadIdx.x] = ac;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = rs[0] + rc[0];
}

// Blocks of the tensor-writing kernels: a fixed count (so the partial sums of
// squares, one per block, are reduced in a fixed order), or fewer for tiny grids.
static constexpr int kEvalBlocks = 1216;  // 8 per SM
static unsigned eval_blocks(long long rows) { return (unsigned)(rows < kEvalBlocks ? rows : kEvalBlocks); }

bool eval_table_f64(const tk_kernel& kh, const tk_grid& gh, double* table, cudaStream_t s) {
  if (!table_applicable(kh, gh)) return false;
  const KernelDev k = make_kernel_dev(kh);
  const int n = gh.n[0];
  const long long Q = table_size(n);
  const double h = (gh.kind == TK_VERTEX) ? gh.b[0] / (double)(n - 1) : gh.b[0] / (double)n;
  const int tb = 64;
  const long long nb = (Q + tb - 1) / tb;
  k_table<<<(unsigned)(nb < 8192 ? nb : 8192), tb, 0, s>>>(k, h * k.inv_ell[0], n % 2 == 0, Q, table);
  TK_LAUNCH("k_table");
  return true;
}

void eval_tensor_f64(const tk_kernel& kh, const tk_grid& gh, double* F, double* table,
                     cudaStream_t s, double* rowsq, double* normF2) {
  const KernelDev k = make_kernel_dev(kh);
  const GridDev g = make_grid_dev(gh);
  if (table_applicable(kh, gh)) {
    const int n = gh.n[0];
    const long long Q = table_size(n);
    const double h = (gh.kind == TK_VERTEX) ? gh.b[0] / (double)(n - 1) : gh.b[0] / (double)n;
    const int even = (n % 2 == 0);
    const int tb = 64;
    const long long nb = (Q + tb - 1) / tb;
    k_table<<<(unsigned)(nb < 8192 ? nb : 8192), tb, 0, s>>>(k, h * k.inv_ell[0], even, Q, table);
    TK_LAUNCH("k_table");
    const long long rows = (long long)n * n;
    k_gather<<<eval_blocks(rows), n < 256 ? 128 : 256, 0, s>>>(table, n, even, F, rowsq);
    TK_LAUNCH("k_gather");
  } else {
    const long long rows = (long long)gh.n[0] * gh.n[1];
    k_eval_general<<<eval_blocks(rows), 128, 0, s>>>(k, g, F, rowsq);
    TK_LAUNCH("k_eval_general");
  }
  if (normF2) {
    k_rowsq_final<<<1, 1024, 0, s>>>(rowsq, (long long)eval_blocks((long long)gh.n[0] * gh.n[1]), normF2);
    TK_LAUNCH("k_rowsq_final");
  }
}

size_t eval_rowsq_doubles(const tk_grid&) { return kEvalBlocks; }

// ---------------------------------------------------------------------------
// Folded tensor.  Every covariance here depends on the coordinates only
// through x_a^2 / ell_a^2, and every grid is symmetric about 0 (x_{n-1-i} =
// -x_i), so F is unchanged by reversing any axis.  Octant index i of axis a is
// grid index c_a + i (c_a = floor(n_a / 2), 0 <= i < h_a = ceil(n_a / 2)) and
// stands for w_i grid points: 1 for the centre of an odd axis, else 2.  The
// weighted octant Fh(i, j, l) = sqrt(w_i w_j w_l) F(c_1 + i, c_2 + j, c_3 + l)
// has the same |.|_F as F.  B instances share one grid.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fold_scale(int twos) {
  // sqrt(2^twos) for twos = 0..3 (sqrt 2 correctly rounded)
  const double r2 = 1.4142135623730951;
  return (twos == 3) ? 2.0 * r2 : (twos == 2) ? 2.0 : (twos == 1) ? r2 : 1.0;
}

// Distinct values of instance blockIdx.y, times `scale` (one rounding, the
// same as scaling each gathered value).
// The table of instance blockIdx.y.  Values are taken in chunks of 32
// consecutive q (one warp, similar arguments and so similar cost); small q
// (small arguments: long recurrences) cost several times more than large q, so
// chunks go to the W warps of the instance in snake order (round r gives chunk
// r W + p to warp p for even r and to warp W - 1 - p for odd r), and warp p is
// warp p / gridDim.x of block p % gridDim.x, so that consecutive chunks (the
// most expensive ones first) land on different SMs: an SM's FP64 pipe is
// shared by all of its warps.  Every value depends on its q alone, so the
// assignment does not change any result.
constexpr int kTableWarps = 4;  // warps per block

// With counts set (the multiplicity of each entry among the octant's points),
// each chunk c also writes part[b][c] = sum of T[q]^2 counts[q] over its 32
// entries (a fixed warp tree of Neumaier pairs): the |F|^2 partials, one slot
// per chunk in a stride of table_parts(Q) slots (the unused last slot zero).
__global__ void __launch_bounds__(32 * kTableWarps) k_table_b(const KernelDev* __restrict__ kd, double hstep,
                                                             int even, long long Q, double* T, double scale,
                                                             const int* __restrict__ counts, double* part) {
  TK_PDL_ENTRY();
  const int b = blockIdx.y;
  const KernelDev& k = kd[b];
  const double hs = hstep * k.inv_ell[0];
  T += (size_t)b * Q;
  const long long W = (long long)gridDim.x * kTableWarps;
  const long long w = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int lane = threadIdx.x & 31;
  // chunks of 32 entries on each side of tsplit (Temme's range, then the
  // Miller recurrence's), so that no warp runs both branches
  const long long qb = k.tsplit < 0 ? 0 : (k.tsplit > Q ? Q : k.tsplit);
  const long long nchA = (qb + 31) / 32;
  const long long nch = nchA + (Q - qb + 31) / 32;
  const long long stride = (Q + 31) / 32 + 1;
  if (counts != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    for (long long c = nch; c < stride; ++c) part[(size_t)b * stride + c] = 0.0;
  for (long long r = 0; r * W < nch; ++r) {
    const long long c = r * W + ((r & 1) ? W - 1 - w : w);
    if (c >= nch) continue;
    const long long q = ((c < nchA) ? 32 * c : qb + 32 * (c - nchA)) + lane;
    const bool live = q < ((c < nchA) ? qb : Q);
    double v = 0.0;
    if (live) {
      const double s = even ? (double)(8 * q + 3) : (double)(4 * q);
      v = cov_value(k, hs * hs * s);
      v = (scale == 1.0) ? v : v * scale;
      T[q] = v;
    }
    if (counts != nullptr) {
      double sm = live ? v * v * (double)__ldg(counts + q) : 0.0, cm = 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, sm, o), xc = __shfl_xor_sync(0xffffffffu, cm, o);
        const double u = sm + x;
        cm += xc + ((fabs(sm) >= fabs(x)) ? (sm - u) + x : (x - u) + sm);
        sm = u;
      }
      if (lane == 0) part[(size_t)b * stride + c] = sm + cm;
    }
  }
}

// Blocks per instance of k_table_b: one warp per SM sub-partition for a
// single instance, fewer per instance in a batch (about four chunks per warp).
static unsigned table_blocks(long long Q, int B) {
  const long long nch = (Q + 31) / 32;
  const long long want = (B == 1) ? 152 : (nch + 4 * kTableWarps - 1) / (4 * kTableWarps);
  return (unsigned)std::max<long long>(1, std::min<long long>(want, (nch + kTableWarps - 1) / kTableWarps));
}

// Octant of the cubic isotropic grid from the distinct-value table: octant
// index i has a = 2 i + 1 (even n) or a = 2 i (odd n).
__global__ void k_gather_oct(const double* __restrict__ T, long long Q, int n, int h, double* __restrict__ F,
                             double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const double* Tb = T + (size_t)b * Q;
  double* Fb = F + (size_t)b * h * h * h;
  const int even = (n % 2 == 0);
  const long long rows = (long long)h * h;
  double sq = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int i = (int)(row / h), j = (int)(row % h);
    const int ai = 2 * i + even, aj = 2 * j + even;
    const int sij = ai * ai + aj * aj;
    const int tij = even ? 3 : (i > 0) + (j > 0);
    double* out = Fb + row * h;
    for (int l = threadIdx.x; l < h; l += blockDim.x) {
      const int al = 2 * l + even;
      const int s = sij + al * al;
      const double v = __ldg(Tb + (even ? (s - 3) >> 3 : s >> 2)) * fold_scale(even ? 3 : tij + (l > 0));
      out[l] = v;
      sq = fma(v, v, sq);
    }
  }
  const double t = block_row_sum(sq, red);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = t;
}

__global__ void k_eval_oct(const KernelDev* __restrict__ kd, GridDev g, double* __restrict__ F,
                           double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const KernelDev& k = kd[b];
  const int h1 = (g.ax[0].n + 1) / 2, h2 = (g.ax[1].n + 1) / 2, h3 = (g.ax[2].n + 1) / 2;
  const int c1 = g.ax[0].n / 2, c2 = g.ax[1].n / 2, c3 = g.ax[2].n / 2;
  const int o1 = g.ax[0].n & 1, o2 = g.ax[1].n & 1, o3 = g.ax[2].n & 1;
  double* Fb = F + (size_t)b * h1 * h2 * h3;
  const long long rows = (long long)h1 * h2;
  double sq = 0.0;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int i = (int)(row / h2), j = (int)(row % h2);
    const double u = (g.ax[0].x0 + (c1 + i) * g.ax[0].dx) * k.inv_ell[0];
    const double v = (g.ax[1].x0 + (c2 + j) * g.ax[1].dx) * k.inv_ell[1];
    const double uv = u * u + v * v;
    const int tij = (!o1 || i > 0) + (!o2 || j > 0);
    for (int l = threadIdx.x; l < h3; l += blockDim.x) {
      const double w = (g.ax[2].x0 + (c3 + l) * g.ax[2].dx) * k.inv_ell[2];
      const double val = cov_value(k, uv + w * w) * fold_scale(tij + (!o3 || l > 0));
      Fb[row * h3 + l] = val;
      sq = fma(val, val, sq);
    }
  }
  const double t = block_row_sum(sq, red);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = t;
}

// |Fh|^2 of instance blockIdx.x from its nparts block partials.
__global__ void __launch_bounds__(256) k_parts_final(const double* __restrict__ part, int nparts,
                                                     double* __restrict__ out) {
  norm_parts_block(part + (size_t)blockIdx.x * nparts, nparts, out + blockIdx.x);
}

// Blocks per instance: a function of the shape alone (about 8 rows each).
static unsigned oct_blocks(const tk_grid& g) {
  const long long rows = (long long)((g.n[0] + 1) / 2) * ((g.n[1] + 1) / 2);
  return (unsigned)std::max<long long>(1, std::min<long long>(rows / 8, kEvalBlocks));
}

// One block per octant row i (mode-1 unfolding, K = h^2 columns (j, l)) of
// instance blockIdx.y: values from the table, the row's largest magnitude and
// sum of squares (first pass), then its six BF16 slices (second pass, values
// recomputed from the table instead of stored).
__global__ void __launch_bounds__(1024) k_gather_slice(const double* __restrict__ T, long long Q, int n, int h,
                                                      long long Kp, int* __restrict__ rowexp,
                                                      __nv_bfloat16* __restrict__ S, double* __restrict__ part) {
  TK_PDL_ENTRY();
  // For even n every octant point stands for 8 grid points and the table
  // already holds 2 sqrt(2) C; for odd n the weight varies and is applied here.
  __shared__ unsigned long long redm[32];
  __shared__ double reds[32];
  __shared__ int eshared;
  const int i = blockIdx.x, b = blockIdx.y;
  const double* Tb = T + (size_t)b * Q;
  const int even = (n % 2 == 0);
  const int ai = 2 * i + even;
  const int ti = even ? 1 : (i > 0);
  const int K = h * h;
  auto value = [&](int j, int l) {
    const int aj = 2 * j + even, al = 2 * l + even;
    const int sq = ai * ai + aj * aj + al * al;
    const double t = __ldg(Tb + (even ? (sq - 3) >> 3 : sq >> 2));
    return even ? t : t * fold_scale(ti + (j > 0) + (l > 0));
  };
  // column c = j h + l advances by blockDim.x per iteration: (j, l) advance
  // by the quotient and remainder of that stride (no division in the loops)
  const int dj = (int)blockDim.x / h, dl = (int)blockDim.x - dj * h;
  const int j0 = (int)threadIdx.x / h, l0 = (int)threadIdx.x - j0 * h;
  // largest |value| by its bits (the order of non-negative doubles), sum of squares
  unsigned long long mx = 0;
  double ss = 0.0;
  for (int c = threadIdx.x, j = j0, l = l0; c < K; c += blockDim.x) {
    const double v = value(j, l);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    mx = bits > mx ? bits : mx;
    ss = fma(v, v, ss);
    j += dj;
    l += dl;
    if (l >= h) {
      l -= h;
      ++j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long om = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = om > mx ? om : mx;
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if ((threadIdx.x & 31) == 0) {
    redm[threadIdx.x >> 5] = mx;
    reds[threadIdx.x >> 5] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = redm[w] > m ? redm[w] : m;
      t += reds[w];
    }
    int e = -1000;
    const double mv = __longlong_as_double((long long)m);
    if (mv > 0.0) frexp(mv, &e);
    eshared = e;
    rowexp[(size_t)b * h + i] = e;
    part[(size_t)b * h + i] = t;
  }
  __syncthreads();
  const int e = eshared;
  const size_t plane = (size_t)h * Kp;
  __nv_bfloat16* Sb = S + (size_t)b * kSlices * plane + (size_t)i * Kp;
  for (int c = threadIdx.x, j = j0, l = l0; c < Kp; c += blockDim.x) {
    int d[kSlices] = {0, 0, 0, 0, 0, 0};
    if (c < K && e > -1000) slice_digits(value(j, l), e, d);
#pragma unroll
    for (int s2 = 0; s2 < kSlices; ++s2) Sb[s2 * plane + c] = slice_value(d[s2], s2);
    j += dj;
    l += dl;
    if (l >= h) {
      l -= h;
      ++j;
    }
  }
}

__global__ void __launch_bounds__(1024) k_gather_slice2(const double* __restrict__ T, long long Q, int n, int h,
                                                      long long Kp, int* __restrict__ rowexp,
                                                      __nv_bfloat16* __restrict__ S, double* __restrict__ part) {
  TK_PDL_ENTRY();
  // For even n every octant point stands for 8 grid points and the table
  // already holds 2 sqrt(2) C; for odd n the weight varies and is applied here.
  __shared__ unsigned long long redm[32];
  __shared__ double reds[32];
  __shared__ int eshared;
  const int i = blockIdx.x, b = blockIdx.y;
  const double* Tb = T + (size_t)b * Q;
  const int even = (n % 2 == 0);
  const int ai = 2 * i + even;
  const int ti = even ? 1 : (i > 0);
  const int K = h * h;
  auto value = [&](int j, int l) {
    const int aj = 2 * j + even, al = 2 * l + even;
    const int sq = ai * ai + aj * aj + al * al;
    const double t = __ldg(Tb + (even ? (sq - 3) >> 3 : sq >> 2));
    return even ? t : t * fold_scale(ti + (j > 0) + (l > 0));
  };
  // h even: each thread takes column pairs (c, c + 1) = (j h + l, j h + l + 1)
  // of one row j; the pair index advances by blockDim.x per iteration, (j, l)
  // by the quotient and remainder of that stride (no division in the loops)
  const int step = 2 * (int)blockDim.x;
  const int dj = step / h, dl = step - dj * h;
  const int j0 = 2 * (int)threadIdx.x / h, l0 = 2 * (int)threadIdx.x - j0 * h;
  // largest |value| by its bits (the order of non-negative doubles), sum of
  // squares in pair order
  unsigned long long mx = 0;
  double ss = 0.0;
  for (int c = 2 * threadIdx.x, j = j0, l = l0; c < K; c += step) {
    const double v0 = value(j, l), v1 = value(j, l + 1);
    const unsigned long long b0 = (unsigned long long)__double_as_longlong(v0) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long b1 = (unsigned long long)__double_as_longlong(v1) & 0x7FFFFFFFFFFFFFFFull;
    mx = b0 > mx ? b0 : mx;
    mx = b1 > mx ? b1 : mx;
    ss = fma(v0, v0, ss);
    ss = fma(v1, v1, ss);
    j += dj;
    l += dl;
    if (l >= h) {
      l -= h;
      ++j;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long om = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = om > mx ? om : mx;
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if ((threadIdx.x & 31) == 0) {
    redm[threadIdx.x >> 5] = mx;
    reds[threadIdx.x >> 5] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = redm[w] > m ? redm[w] : m;
      t += reds[w];
    }
    int e = -1000;
    const double mv = __longlong_as_double((long long)m);
    if (mv > 0.0) frexp(mv, &e);
    eshared = e;
    rowexp[(size_t)b * h + i] = e;
    part[(size_t)b * h + i] = t;
  }
  __syncthreads();
  const int e = eshared;
  const size_t plane = (size_t)h * Kp;
  __nv_bfloat16* Sb = S + (size_t)b * kSlices * plane + (size_t)i * Kp;
  for (int c = 2 * threadIdx.x, j = j0, l = l0; c < Kp; c += step) {
    int d0[kSlices] = {0, 0, 0, 0, 0, 0}, d1[kSlices] = {0, 0, 0, 0, 0, 0};
    if (c < K && e > -1000) {
      slice_digits(value(j, l), e, d0);
      slice_digits(value(j, l + 1), e, d1);
    }
    // both columns of a slice in one 4-byte store (c even, Kp even)
#pragma unroll
    for (int s2 = 0; s2 < kSlices; ++s2)
      *reinterpret_cast<__nv_bfloat162*>(Sb + s2 * plane + c) =
          __halves2bfloat162(slice_value(d0[s2], s2), slice_value(d1[s2], s2));
    j += dj;
    l += dl;
    if (l >= h) {
      l -= h;
      ++j;
    }
  }
}

void eval_octant_slices(const KernelDev* kd, const tk_grid& g, int B, double* table, int* rowexp, void* S,
                        long long Kp, double* part, double* normF2, cudaStream_t s, Profiler* pf) {
  const int n = g.n[0], h = (n + 1) / 2;
  const long long Q = table_size(n);
  const double hstep = (g.kind == TK_VERTEX) ? g.b[0] / (double)(n - 1) : g.b[0] / (double)n;
  if (pf) pf->begin(TK_STAGE_TABLE, s);
  // even n: the table holds the octant values 2 sqrt(2) C directly
  launch_pdl("k_table_b", k_table_b, dim3(table_blocks(Q, B), B), dim3(32 * kTableWarps), 0, s, kd, hstep, n % 2 == 0,
             Q, table, n % 2 == 0 ? 2.8284271247461903 : 1.0, (const int*)nullptr, (double*)nullptr);
  if (pf) pf->end(s);
  // rows of h^2 values: wide blocks for long rows (a function of the shape
  // alone, so that each instance's sums do not depend on the batch)
  const int threads = (h >= 128) ? 1024 : 256;
  if (h % 2 == 0)
    launch_pdl("k_gather_slice2", k_gather_slice2, dim3(h, B), dim3(threads), 0, s, table, Q, n, h, Kp, rowexp,
               (__nv_bfloat16*)S, part);
  else
    launch_pdl("k_gather_slice", k_gather_slice, dim3(h, B), dim3(threads), 0, s, table, Q, n, h, Kp, rowexp,
               (__nv_bfloat16*)S, part);
  if (normF2 != nullptr) {
    k_parts_final<<<B, 256, 0, s>>>(part, h, normF2);
    TK_LAUNCH("k_parts_final");
  }
}

// counts[q] += 1 for every octant point (i, j, l) of an even grid, q its table
// entry (a = 2 index + 1, q = (a_i^2 + a_j^2 + a_l^2 - 3) / 8).
__global__ void k_table_counts(int h, int* __restrict__ counts) {
  const long long total = (long long)h * h * h;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ((long long)h * h));
    const int rem = (int)(e - (long long)i * h * h);
    const int j = rem / h, l = rem - j * h;
    const int ai = 2 * i + 1, aj = 2 * j + 1, al = 2 * l + 1;
    atomicAdd(counts + ((ai * ai + aj * aj + al * al - 3) >> 3), 1);
  }
}

// The six BF16 slices of octant row blockIdx.x of instance blockIdx.y (even
// n, h a multiple of 8), eight consecutive columns (one table row j) a thread
// and item: the eight gathers first, then the digits, then six 16-byte
// stores.  The row exponent: row i holds the table entries q >= q_min(i) =
// ((2i + 1)^2 - 1) / 8 = i (i + 1) / 2 (its entry j = l = 0), and every
// covariance here decreases with the radius, so its largest entry is
// T[q_min(i)]: e is the binary exponent of T[q_min(i)] (1 + 2^-40), the
// factor keeping 2^e above the row even where neighbouring entries of a flat
// table agree to the last bits.  Block i also writes it to rowexp.
__global__ void __launch_bounds__(1024) k_gather_slice8(const double* __restrict__ T, long long Q, int h, long long Kp,
                                                       int* __restrict__ rowexp, __nv_bfloat16* __restrict__ S) {
  TK_PDL_ENTRY();
  const int i = blockIdx.x, b = blockIdx.y;
  const double* Tb = T + (size_t)b * Q;
  int e = -1000;
  {
    const double top = fabs(__ldg(Tb + (long long)i * (i + 1) / 2)) * (1.0 + 0x1p-40);
    if (top > 0.0) frexp(top, &e);
  }
  if (threadIdx.x == 0) rowexp[(size_t)b * h + i] = e;
  const int ai = 2 * i + 1;
  const long long K = (long long)h * h;
  const size_t plane = (size_t)h * Kp;
  __nv_bfloat16* Sb = S + (size_t)b * kSlices * plane + (size_t)i * Kp;
  for (long long g = threadIdx.x; 8 * g < Kp; g += blockDim.x) {
    const long long c = 8 * g;
    uint32_t w[kSlices][4];
    if (c < K && e > -1000) {
      const int j = (int)(c / h), l0 = (int)(c - (long long)j * h);
      const int aj = 2 * j + 1;
      const int base = ai * ai + aj * aj - 3;
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int al = 2 * (l0 + u) + 1;
        v[u] = __ldg(Tb + ((base + al * al) >> 3));
      }
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        int d0[kSlices], d1[kSlices];
        slice_digits(v[u], e, d0);
        slice_digits(v[u + 1], e, d1);
#pragma unroll
        for (int s2 = 0; s2 < kSlices; ++s2) {
          const __nv_bfloat162 pr = __halves2bfloat162(slice_value(d0[s2], s2), slice_value(d1[s2], s2));
          w[s2][u >> 1] = *reinterpret_cast<const uint32_t*>(&pr);
        }
      }
    } else {
#pragma unroll
      for (int s2 = 0; s2 < kSlices; ++s2) w[s2][0] = w[s2][1] = w[s2][2] = w[s2][3] = 0u;
    }
#pragma unroll
    for (int s2 = 0; s2 < kSlices; ++s2)
      *reinterpret_cast<uint4*>(Sb + s2 * plane + c) = make_uint4(w[s2][0], w[s2][1], w[s2][2], w[s2][3]);
  }
}

MultCache::~MultCache() {
  for (auto& kv : counts)
    if (kv.second) cudaFree(kv.second);
}

const int* table_counts(MultCache& cache, int n, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(cache.mu);
  auto it = cache.counts.find(n);
  if (it != cache.counts.end()) return it->second;
  if (n % 2 != 0) fail(TK_EINVAL, "table_counts: even n only");
  const long long Q = table_size(n);
  int* c = nullptr;
  TK_CUDA(cudaMalloc(&c, sizeof(int) * (size_t)Q));
  TK_CUDA(cudaMemsetAsync(c, 0, sizeof(int) * (size_t)Q, s));
  const int h = n / 2;
  const long long total = (long long)h * h * h;
  k_table_counts<<<(unsigned)std::min<long long>((total + 255) / 256, 8192), 256, 0, s>>>(h, c);
  TK_LAUNCH("k_table_counts");
  TK_CUDA(cudaStreamSynchronize(s));  // other streams of the context read it next
  cache.counts[n] = c;
  return c;
}

void eval_octant_slices8(const KernelDev* kd, const tk_grid& g, int B, double* table, int* rowexp, void* S,
                         long long Kp, double* part, const int* counts, cudaStream_t s, Profiler* pf) {
  const int n = g.n[0], h = n / 2;
  if (n % 2 != 0 || h % 8 != 0) fail(TK_EINVAL, "eval_octant_slices8: even n, h a multiple of 8");
  const long long Q = table_size(n);
  const double hstep = (g.kind == TK_VERTEX) ? g.b[0] / (double)(n - 1) : g.b[0] / (double)n;
  if (pf) pf->begin(TK_STAGE_TABLE, s);
  // even n: the table holds the octant values 2 sqrt(2) C directly
  launch_pdl("k_table_b", k_table_b, dim3(table_blocks(Q, B), B), dim3(32 * kTableWarps), 0, s, kd, hstep, 1, Q,
             table, 2.8284271247461903, counts, part);
  if (pf) pf->end(s);
  // one thread per group of eight columns, up to 1024 a row
  const long long groups = (long long)h * h / 8;
  const unsigned threads = (unsigned)std::min<long long>(1024, (groups + 31) / 32 * 32);
  launch_pdl("k_gather_slice8", k_gather_slice8, dim3(h, B), dim3(threads), 0, s, (const double*)table, Q, h, Kp,
             rowexp, (__nv_bfloat16*)S);
}

size_t eval_octant_parts(const tk_grid& g) { return oct_blocks(g); }
long long table_parts(int n) { return (table_size(n) + 31) / 32 + 1; }
long long table_entries(int n) { return table_size(n); }

void eval_octant_f64(const KernelDev* kd, bool tab, const tk_grid& g, int B, double* Fh, double* table,
                     double* part, double* normF2, cudaStream_t s, Profiler* pf) {
  const unsigned nb = oct_blocks(g);
  const int h3 = (g.n[2] + 1) / 2;
  const int threads = h3 < 128 ? 64 : 128;
  if (tab) {
    const int n = g.n[0];
    const long long Q = table_size(n);
    const double hstep = (g.kind == TK_VERTEX) ? g.b[0] / (double)(n - 1) : g.b[0] / (double)n;
    if (pf) pf->begin(TK_STAGE_TABLE, s);
    launch_pdl("k_table_b", k_table_b, dim3(table_blocks(Q, B), B), dim3(32 * kTableWarps), 0, s, kd, hstep,
               n % 2 == 0, Q, table, 1.0, (const int*)nullptr, (double*)nullptr);
    if (pf) pf->end(s);
    k_gather_oct<<<dim3(nb, B), threads, 0, s>>>(table, Q, n, (n + 1) / 2, Fh, part);
    TK_LAUNCH("k_gather_oct");
  } else {
    k_eval_oct<<<dim3(nb, B), threads, 0, s>>>(kd, make_grid_dev(g), Fh, part);
    TK_LAUNCH("k_eval_oct");
  }
  k_parts_final<<<B, 256, 0, s>>>(part, (int)nb, normF2);
  TK_LAUNCH("k_parts_final");
}

// ---------------------------------------------------------------------------
// |x|^2: each thread keeps a Neumaier pair over a fixed slice; blocks reduce
// in a fixed tree; one block sums the block partials in index order.  The
// result does not depend on scheduling.
// ---------------------------------------------------------------------------
static constexpr int kNormBlocks = 608;  // 4 x 152 SMs
static constexpr int kNormThreads = 256;

size_t norm2_scratch_doubles(size_t) { return 2 * kNormBlocks; }

__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

__global__ void k_norm2_partial(const double* __restrict__ x, long long len, double* part) {
  double s = 0.0, c = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = x[t];
    neumaier(s, c, v * v);
  }
  __shared__ double ss[kNormThreads], sc[kNormThreads];
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a = ss[threadIdx.x], ac = sc[threadIdx.x];
      neumaier(a, ac, ss[threadIdx.x + w]);
      ac += sc[threadIdx.x + w];
      ss[threadIdx.x] = a;
      sc[threadIdx.x] = ac;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ss[0];
    part[2 * blockIdx.x + 1] = sc[0];
  }
}

__global__ void k_norm2_final(const double* part, int nparts, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nparts; ++b) {
      neumaier(s, c, part[2 * b]);
      c += part[2 * b + 1];
    }
    out[0] = s + c;
  }
}

void norm2_f64(const double* x, size_t len, double* out_dev, double* scratch, cudaStream_t s) {
  k_norm2_partial<<<kNormBlocks, kNormThreads, 0, s>>>(x, (long long)len, scratch);
  TK_LAUNCH("k_norm2_partial");
  k_norm2_final<<<1, 32, 0, s>>>(scratch, kNormBlocks, out_dev);
  TK_LAUNCH("k_norm2_final");
}

}  // namespace tk
