// (e) Error of the Tucker approximation during a solve on the sliced path,
// |F - X| / |F| of Sec. 3.2 on the weighted octant (|F - X| = |Fh - Xh|):
//   Xh = B x_1 V x_2 V x_3 V,  V the octant factor that the three modes of an
//   isotropic problem share,
// with Fh read back from the exact BF16 slices the Gram used,
//   Fh(i, j, l) = 2^e_i sum_s S_s(i, j h + l).
//
// GB300 has little FP64 throughput (an FP64 warp instruction holds a sub-
// partition's FP64 unit for about 64 cycles), so the products run in
// float-float arithmetic on the FP32 pipes: every FP64 operand becomes
// hi + lo (two floats, split from the FP64 bits with integer operations), a
// product of two floats is split exactly (a b = p + e, e = fma(a, b, -p)),
// and sums carry their rounding error (Knuth's two-sum where a pair is formed,
// Kahan's compensated sum along the rank).  Per entry the reconstruction is
// accurate to about 2^-44 of the entry; the residual, formed from the three
// exact partial sums of the slices, to about 2^-23 of itself; its squares
// are summed in FP32 per thread and block and in FP64 across blocks.  The
// reported relative error carries about six correct digits.
//
// Symmetry.  The kernel serves the isotropic solve on a cubic grid, where
// F(i, j, l) depends on x_i^2 + x_j^2 + x_l^2 only and the three modes share
// one factor, so F and X (hence the residual) are invariant under every
// permutation of (i, j, l).  The sum runs over the orbit representatives
// i <= j <= l, each weighted by its orbit's size (6 for three distinct
// indices, 3 for two equal, 1 for three equal): about h^3 / 6 entries
// instead of h^3.  (X is symmetric up to the rounding of its FP64 core, and
// the slices up to 2^-48 of their row's largest entry; both move E by far
// less than the digits it carries.)
//
// Three launches.  k_err_w1: W1(i) = B x_1 V(i, :) (R x R) for every octant
// row i, one CTA per row.  k_err_sliced: one CTA per (row i, block of 8 or 16
// rows j) of one instance, blocks wholly below i having nothing to do; it
// forms W2(j, c) = sum_b V(j, b) W1(i, b, c) in shared memory, then each
// thread takes columns l >= j: X = sum_c V(l, c) W2(j, c), and the CTA writes
// its partial sum.  k_err_final: the partials of each instance in a fixed
// order.  (One kernel that computed W1 in every CTA and let the last CTA sum
// the partials spent most of its time in the redundant W1 and in the
// device-wide fences and the contended counter.)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "slices.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kJB = 16;  // most rows j per CTA (16, or 8 when h is not a multiple of 16)
constexpr int kErrThreads = 128;
constexpr int kMaxR = 32;  // padded rank handled here

struct FF {
  float hi, lo;
};

// a + b = s + e exactly (Knuth's two-sum).
// (The _rn intrinsics keep the compiler from fusing these into FMAs.)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += x y for float-float x, y: the leading product exactly (p + e), the
// cross terms in FP32 (about 2^-48 of the product), x.lo y.lo dropped.
__device__ __forceinline__ void ff_fma(FF& acc, const FF x, const FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.hi, -p);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e + fmaf(x.hi, y.lo, x.lo * y.hi);
}

// hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ FF ff_norm(FF a) {
  const float s = __fadd_rn(a.hi, a.lo);
  return FF{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// An FP64 value as hi + lo from its bits (no FP64 instruction): hi keeps the
// top 24 significand bits, lo the next 24 (rounded).  Values whose exponent
// lies outside about [-100, 100] are outside the range this kernel is used
// for (the caller checks sigma2).
__device__ __forceinline__ FF ff_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int fe = ex - 1023 + 127;
  if (ex == 0 || fe <= 0) return FF{__uint_as_float(sign), __uint_as_float(sign)};
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
  // remainder: significand bits 0..28, worth 2^(ex - 1075) each
  const unsigned rem = (unsigned)(b & 0x1FFFFFFFull);
  const int le = ex - 1075 + 127;  // exponent field of 2^(ex - 1075)
  float lo = 0.0f;
  if (rem != 0 && le > 0) lo = __uint2float_rn(rem) * __uint_as_float((unsigned)le << 23);
  return FF{hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only), and the
// wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct ErrSlicedArgs {
  const __nv_bfloat16* S;  // bucket: [b][6][h][Kp]
  long long Kp;
  const int* rowexp;       // bucket: [b][h]
  const double* normF2;    // bucket: [b]
  int h, R;
  const double* V;         // group: [pos][h][R]
  const double* B;         // group: [pos][R][R][R]
  const int* amap;         // group position -> bucket instance
  const int* rk;           // rank of bucket instance b at rk[b * rk_stride] (<= R)
  int rk_stride;
  int jbs;                 // rows j per CTA
  FF* W1;                  // group: [pos][h][kR][kR]
  FF* VF;                  // group: [pos][h][kR], V in float-float (zero past the rank)
  double* partials;        // group: [pos][h][h / jbs]
  double* esum;            // group: [pos][2]
};

// The instance's rank: the sums run over the rank's columns only, so the
// zero padding up to R does not change any bit.
__device__ __forceinline__ int err_rank(const ErrSlicedArgs& a, int b) {
  return min(a.rk[(size_t)b * a.rk_stride], a.R);
}

// X(j, l) = sum_{c < r} V(l, c) W2(j, c) in float-float: the leading products
// exact (p + e) and summed with Kahan's compensation, the small terms summed
// plainly (two short chains).
// The loop has no branch (columns from r on are zero in vl and w2 and their
// compensated steps are selected away), so two calls interleave.
template <int kR>
__device__ __forceinline__ FF x_entry(const FF (&vl)[kR], const FF* w2, int r) {
  float S = 0.0f, comp = 0.0f, le = 0.0f, lx = 0.0f;
#pragma unroll
  for (int c = 0; c < kR; ++c) {
    const FF w = w2[c];
    const float p = __fmul_rn(vl[c].hi, w.hi);
    le += fmaf(vl[c].hi, w.hi, -p);
    lx = fmaf(vl[c].hi, w.lo, lx);
    lx = fmaf(vl[c].lo, w.hi, lx);
    const float y = __fsub_rn(p, comp);
    const float t = __fadd_rn(S, y);
    const float cn = __fsub_rn(__fsub_rn(t, S), y);
    const bool take = c < r;
    S = take ? t : S;
    comp = take ? cn : comp;
  }
  return ff_norm(FF{S, __fsub_rn(le + lx, comp)});
}

// The residual Fh - Xh at one entry in units of 2^e_i, from the six slices at
// sp (run apart) and X scaled by sc.
__device__ __forceinline__ float residual(const FF x, const __nv_bfloat16* sp, int run, float sc) {
  // sums of two slices are exact: 8-bit digits eight binary places apart (a
  // zero row's slices are zero)
  const float A = __bfloat162float(sp[0]) + __bfloat162float(sp[run]);
  const float Bv = __bfloat162float(sp[2 * run]) + __bfloat162float(sp[3 * run]);
  const float Cv = __bfloat162float(sp[4 * run]) + __bfloat162float(sp[5 * run]);
  const float xh = x.hi * sc, xl = x.lo * sc;
  const float p1 = __fsub_rn(A, xh);  // exact while xh is within a factor 2 of A
  float p2h, p2l;
  two_sum(Bv, -xl, p2h, p2l);
  return (p1 + p2h) + (p2l + Cv);
}

// W1(i, b, c) = sum_a V(i, a) B(a, b, c): one CTA per (row i, instance), one
// thread per (b, c).
template <int kR>
__global__ void __launch_bounds__(kR * kR) k_err_w1(ErrSlicedArgs a) {
  TK_PDL_ENTRY();
  __shared__ FF Vi[kR];
  const int h = a.h, R = a.R;
  const int i = blockIdx.x, pos = blockIdx.y;
  const int r = err_rank(a, a.amap[pos]);
  const double* V = a.V + (size_t)pos * h * R;
  const double* Bc = a.B + (size_t)pos * R * R * R;
  if (threadIdx.x < kR) {
    const FF v = ((int)threadIdx.x < r) ? ff_from_double(V[(size_t)i * R + threadIdx.x]) : FF{0.0f, 0.0f};
    Vi[threadIdx.x] = v;
    a.VF[((size_t)pos * h + i) * kR + threadIdx.x] = v;  // for k_err_sliced: converted once
  }
  __syncthreads();
  const int bb = threadIdx.x / kR, c = threadIdx.x - bb * kR;
  FF acc{0.0f, 0.0f};
  if (bb < r && c < r) {
    // eight entries of the column of B in flight at once, then their products
    for (int a0 = 0; a0 < r; a0 += 8) {
      double bv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) bv[q] = (a0 + q < r) ? __ldg(Bc + ((size_t)(a0 + q) * R + bb) * R + c) : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (a0 + q < r) ff_fma(acc, Vi[a0 + q], ff_from_double(bv[q]));
    }
  }
  a.W1[((size_t)pos * h + i) * kR * kR + threadIdx.x] = ff_norm(acc);
}

// |Fh - Xh|^2 of each instance: its partials in a fixed order (a strided
// sum per thread, then a fixed tree), with |Fh|^2 beside it.
__global__ void __launch_bounds__(kErrThreads) k_err_final(ErrSlicedArgs a, int nparts) {
  TK_PDL_ENTRY();
  __shared__ double redd[kErrThreads];
  const int pos = blockIdx.x;
  const double* parts = a.partials + (size_t)pos * nparts;
  double sum = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) sum += parts[t];
  redd[threadIdx.x] = sum;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) redd[threadIdx.x] += redd[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.esum[2 * pos] = redd[0];
    a.esum[2 * pos + 1] = a.normF2[a.amap[pos]];
  }
}

template <int kR>
__global__ void __launch_bounds__(kErrThreads) k_err_sliced(ErrSlicedArgs a) {
  TK_PDL_ENTRY();
  __shared__ FF W1s[kR * kR];     // W1(i, b, c)
  __shared__ FF Vj[kJB * kR];     // V(j0 + jj, b)
  __shared__ FF W2s[kJB * kR];    // W2(j0 + jj, c)
  __shared__ float red[kErrThreads / 32];
  const int h = a.h;
  const int jb = blockIdx.x, i = blockIdx.y, pos = blockIdx.z;
  const int JB = a.jbs;
  const int j0 = jb * JB;
  const int b = a.amap[pos];
  const int r = err_rank(a, b);
  const int jlo = max(i - j0, 0);  // first row of the block with j >= i
  float acc2 = 0.0f;
  bool zero_row = false;
  int ei = 0;
  extern __shared__ __align__(16) unsigned char dyn[];
  __nv_bfloat16* Ss = reinterpret_cast<__nv_bfloat16*>(dyn);  // [6][JB rows j][h columns l]
  if (jlo < JB) {  // uniform over the CTA
    // the block's slices (six contiguous runs of JB h values) staged in shared
    // memory first, so that the rows j do not wait on the memory one by one
    const size_t plane = (size_t)h * a.Kp;
    const __nv_bfloat16* Srow = a.S + (size_t)b * kSlices * plane + (size_t)i * a.Kp + (size_t)j0 * h;
    const int run = JB * h, pieces = run / 8;
    for (int e = threadIdx.x; e < kSlices * pieces; e += blockDim.x) {
      const int sl = e / pieces, q = e - sl * pieces;
      cp_async16(Ss + (size_t)sl * run + 8 * q, Srow + (size_t)sl * plane + 8 * q);
    }
    const FF* W1 = a.W1 + ((size_t)pos * h + i) * kR * kR;
    for (int e = threadIdx.x; e < kR * kR; e += blockDim.x) W1s[e] = W1[e];
    const FF* VF = a.VF + (size_t)pos * h * kR;
    for (int e = threadIdx.x; e < JB * kR; e += blockDim.x) Vj[e] = VF[(size_t)j0 * kR + e];
    __syncthreads();
    // W2(j, c) = sum_b V(j, b) W1(i, b, c), rows j >= i
    for (int e = jlo * kR + threadIdx.x; e < JB * kR; e += blockDim.x) {
      const int jj = e / kR, c = e - jj * kR;
      FF acc{0.0f, 0.0f};
      for (int bb = 0; bb < r; ++bb) ff_fma(acc, Vj[jj * kR + bb], W1s[bb * kR + c]);
      W2s[e] = ff_norm(acc);
    }
    __syncthreads();
    ei = a.rowexp[(size_t)b * h + i];
    zero_row = ei <= -1000;
    // residual in units of 2^e_i (exact power-of-two scaling in FP32)
    const float sc = zero_row ? 1.0f : __int_as_float((127 - ei) << 23);
    cp_async_wait_all();
    __syncthreads();
    for (int l = threadIdx.x; l < h; l += blockDim.x) {
      const int jend = min(JB, l - j0 + 1);  // rows j <= l
      if (jend <= jlo) continue;
      FF vl[kR];
#pragma unroll
      for (int c = 0; c < kR; ++c) vl[c] = VF[(size_t)l * kR + c];
      // two rows j at a time (independent chains), accumulated in row order;
      // each entry weighted by the size of its orbit (i <= j <= l here)
      int jj = jlo;
      for (; jj + 1 < jend; jj += 2) {
        const FF x0 = x_entry<kR>(vl, W2s + jj * kR, r);
        const FF x1 = x_entry<kR>(vl, W2s + (jj + 1) * kR, r);
        const float r0 = residual(x0, Ss + jj * h + l, run, sc);
        const float r1 = residual(x1, Ss + (jj + 1) * h + l, run, sc);
        const int j = j0 + jj;
        const float w0 = (i == j) ? ((j == l) ? 1.0f : 3.0f) : ((j == l) ? 3.0f : 6.0f);
        const float w1 = (i == j + 1) ? ((j + 1 == l) ? 1.0f : 3.0f) : ((j + 1 == l) ? 3.0f : 6.0f);
        acc2 = fmaf(r0 * w0, r0, acc2);
        acc2 = fmaf(r1 * w1, r1, acc2);
      }
      if (jj < jend) {
        const FF x0 = x_entry<kR>(vl, W2s + jj * kR, r);
        const float r0 = residual(x0, Ss + jj * h + l, run, sc);
        const int j = j0 + jj;
        const float w0 = (i == j) ? ((j == l) ? 1.0f : 3.0f) : ((j == l) ? 3.0f : 6.0f);
        acc2 = fmaf(r0 * w0, r0, acc2);
      }
    }
  }
  // fixed tree: warp shuffles, then the warps in order
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kErrThreads / 32; ++w) t += red[w];
    // back to absolute units: times 2^(2 e_i), a power of two built from its
    // bits (|e_i| stays far inside the FP64 exponent range here)
    const double scale = __longlong_as_double((long long)(1023 + 2 * ei) << 52);
    a.partials[(size_t)pos * h * (h / JB) + (size_t)i * (h / JB) + jb] = zero_row ? (double)t : (double)t * scale;
  }
}

}  // namespace

// Rows j per CTA (0: h is not a multiple of 8).  Few rows per CTA keep each
// warp's serial chain short: the kernel is bound by the latency of that chain
// (slice loads, the compensated sum along the rank), not by its instructions.
static int err_rows(int h) { return (h % 16 == 0 && h <= 256) ? 16 : h % 8 == 0 ? 8 : 0; }

// Compiled padded ranks: the smallest of 8, 12, 16, 24, 32 that holds R.
static int err_kr(int R) { return R <= 8 ? 8 : R <= 12 ? 12 : R <= 16 ? 16 : R <= 24 ? 24 : 32; }

bool err_sliced_supported(int h, int R) { return err_rows(h) > 0 && R >= 1 && R <= kMaxR; }

size_t err_sliced_scratch_bytes(int h, int R, int cnt) {
  const int kr = err_kr(R);
  return carve_bytes<double>((size_t)cnt * h * (h / 8)) + carve_bytes<FF>((size_t)cnt * h * kr * kr) +
         carve_bytes<FF>((size_t)cnt * h * kr) + 1024;
}

constexpr size_t kErrSmemMax = 100 * 1024;  // staged slices: 6 JB h BF16 values

template <int kR>
static void err_launch(const ErrSlicedArgs& a, int cnt, cudaStream_t s) {
  once_per_device((const void*)&k_err_sliced<kR>, [] {
    TK_CUDA(cudaFuncSetAttribute(k_err_sliced<kR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kErrSmemMax));
  });
  const size_t smem = sizeof(__nv_bfloat16) * kSlices * (size_t)a.jbs * a.h;
  launch_pdl("k_err_w1", k_err_w1<kR>, dim3(a.h, cnt), dim3(kR * kR), 0, s, a);
  launch_pdl("k_err_sliced", k_err_sliced<kR>, dim3(a.h / a.jbs, a.h, cnt), dim3(kErrThreads), smem, s, a);
  launch_pdl("k_err_final", k_err_final, dim3(cnt), dim3(kErrThreads), 0, s, a, a.h * (a.h / a.jbs));
}

void err_sliced_batch(const SliceView& sv, const double* normF2, const double* V, const double* Bcore, int h, int R,
                      int cnt, const int* amap, const int* rk, int rk_stride, void* scratch, double* esum,
                      cudaStream_t s) {
  if (!err_sliced_supported(h, R)) fail(TK_EINVAL, "err_sliced: shape out of range");
  // 16-byte copies of the slice runs: aligned base and row offsets
  if (sv.Kp % 8 != 0 || ((uintptr_t)sv.S & 15) != 0) fail(TK_EINVAL, "err_sliced: slices not 16-byte aligned");
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  const int jbs = err_rows(h);
  double* parts = (double*)base;
  const int kr = err_kr(R);
  FF* w1 = (FF*)(base + carve_bytes<double>((size_t)cnt * h * (h / 8)));
  FF* vf = (FF*)((char*)w1 + carve_bytes<FF>((size_t)cnt * h * kr * kr));
  ErrSlicedArgs a{(const __nv_bfloat16*)sv.S, sv.Kp, sv.rowexp, normF2, h, R, V, Bcore, amap, rk, rk_stride, jbs, w1,
                  vf, parts, esum};
  switch (err_kr(R)) {
    case 8: err_launch<8>(a, cnt, s); break;
    case 12: err_launch<12>(a, cnt, s); break;
    case 16: err_launch<16>(a, cnt, s); break;
    case 24: err_launch<24>(a, cnt, s); break;
    default: err_launch<32>(a, cnt, s); break;
  }
}

}  // namespace tk
