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
// One CTA per (row i, block of 32, 16 or 8 rows j) of one instance: it forms
// W1(i) = B x_1 V(i, :) (R x R) and the block W2(j, c) =
// sum_b V(j, b) W1(i, b, c) in shared memory, then each thread takes columns
// l: X = sum_c V(l, c) W2(j, c).  The last CTA of an instance to finish sums
// the instance's block partials in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "slices.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kJB = 32;  // largest block of rows j per CTA (32, 16 or 8, dividing h)
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

struct ErrSlicedArgs {
  const __nv_bfloat16* S;  // bucket: [b][6][h][Kp]
  long long Kp;
  const int* rowexp;       // bucket: [b][h]
  const double* normF2;    // bucket: [b]
  int h, R;
  const double* V;         // group: [pos][h][R]
  const double* B;         // group: [pos][R][R][R]
  const int* amap;         // group position -> bucket instance
  int jbs;                 // rows j per CTA
  double* partials;        // group: [pos][h][h / jbs]
  int* counters;           // group: [pos], zero on entry
  double* esum;            // group: [pos][2]
};

template <int kR>
__global__ void __launch_bounds__(kErrThreads) k_err_sliced(ErrSlicedArgs a) {
  __shared__ FF Vi[kR];           // V(i, a)
  __shared__ FF W1s[kR * kR];     // W1(i, b, c)
  __shared__ FF Vj[kJB * kR];     // V(j0 + jj, b)
  __shared__ FF W2s[kJB * kR];    // W2(j0 + jj, c)
  __shared__ float red[kErrThreads / 32];
  __shared__ double redd[kErrThreads];
  __shared__ int last;
  const int h = a.h, R = a.R;
  const int jb = blockIdx.x, i = blockIdx.y, pos = blockIdx.z;
  const int JB = a.jbs;
  const int j0 = jb * JB;
  const int b = a.amap[pos];
  const double* V = a.V + (size_t)pos * h * R;
  const double* Bc = a.B + (size_t)pos * R * R * R;
  for (int e = threadIdx.x; e < kR; e += blockDim.x) Vi[e] = (e < R) ? ff_from_double(V[(size_t)i * R + e]) : FF{0, 0};
  for (int e = threadIdx.x; e < JB * kR; e += blockDim.x) {
    const int jj = e / kR, c = e - jj * kR;
    Vj[e] = (c < R) ? ff_from_double(V[(size_t)(j0 + jj) * R + c]) : FF{0.0f, 0.0f};
  }
  __syncthreads();
  // W1(i, b, c) = sum_a V(i, a) B(a, b, c)
  for (int e = threadIdx.x; e < kR * kR; e += blockDim.x) {
    const int bb = e / kR, c = e - bb * kR;
    FF acc{0.0f, 0.0f};
    if (bb < R && c < R)
      for (int aa = 0; aa < R; ++aa) ff_fma(acc, Vi[aa], ff_from_double(Bc[((size_t)aa * R + bb) * R + c]));
    W1s[e] = ff_norm(acc);
  }
  __syncthreads();
  // W2(j, c) = sum_b V(j, b) W1(i, b, c)
  for (int e = threadIdx.x; e < JB * kR; e += blockDim.x) {
    const int jj = e / kR, c = e - jj * kR;
    FF acc{0.0f, 0.0f};
    for (int bb = 0; bb < R; ++bb) ff_fma(acc, Vj[jj * kR + bb], W1s[bb * kR + c]);
    W2s[e] = ff_norm(acc);
  }
  __syncthreads();
  const int ei = a.rowexp[(size_t)b * h + i];
  const bool zero_row = ei <= -1000;
  // residual in units of 2^e_i (exact power-of-two scaling in FP32)
  const float sc = zero_row ? 1.0f : __int_as_float((127 - ei) << 23);
  const size_t plane = (size_t)h * a.Kp;
  const __nv_bfloat16* Srow = a.S + (size_t)b * kSlices * plane + (size_t)i * a.Kp + (size_t)j0 * h;
  float acc2 = 0.0f;
  for (int l = threadIdx.x; l < h; l += blockDim.x) {
    FF vl[kR];
#pragma unroll
    for (int c = 0; c < kR; ++c) vl[c] = (c < R) ? ff_from_double(V[(size_t)l * R + c]) : FF{0.0f, 0.0f};
#pragma unroll 1
    for (int jj = 0; jj < JB; ++jj) {
      // X = sum_c V(l, c) W2(j, c): leading products exact (p + e) and summed
      // with Kahan's compensation, the small terms summed plainly.  A zero
      // product leaves the compensated pair as it is (a Kahan step with 0
      // would renormalise it), so the zero-padded columns beyond the rank do
      // not change any bit: the result does not depend on the padding R.
      float S = 0.0f, comp = 0.0f, lo = 0.0f;
#pragma unroll
      for (int c = 0; c < kR; ++c) {
        if (c < R) {
          const FF w = W2s[jj * kR + c];
          const float p = __fmul_rn(vl[c].hi, w.hi);
          const float e = fmaf(vl[c].hi, w.hi, -p);
          const float y = __fsub_rn(p, comp);
          const float t = __fadd_rn(S, y);
          const float cn = __fsub_rn(__fsub_rn(t, S), y);
          const bool nz = p != 0.0f;
          S = nz ? t : S;
          comp = nz ? cn : comp;
          lo += e + fmaf(vl[c].hi, w.lo, vl[c].lo * w.hi);
        }
      }
      const FF x = ff_norm(FF{S, __fsub_rn(lo, comp)});
      const __nv_bfloat16* sp = Srow + (size_t)jj * h + l;
      float A = 0.0f, Bv = 0.0f, Cv = 0.0f;
      if (!zero_row) {
        // sums of two slices are exact: 8-bit digits eight binary places apart
        A = __bfloat162float(sp[0]) + __bfloat162float(sp[plane]);
        Bv = __bfloat162float(sp[2 * plane]) + __bfloat162float(sp[3 * plane]);
        Cv = __bfloat162float(sp[4 * plane]) + __bfloat162float(sp[5 * plane]);
      }
      const float xh = x.hi * sc, xl = x.lo * sc;
      const float p1 = __fsub_rn(A, xh);  // exact while xh is within a factor 2 of A
      float p2h, p2l;
      two_sum(Bv, -xl, p2h, p2l);
      const float r = (p1 + p2h) + (p2l + Cv);
      acc2 = fmaf(r, r, acc2);
    }
  }
  // fixed tree: warp shuffles, then the warps in order
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
  __syncthreads();
  const int nparts = h * (h / JB);
  double* parts = a.partials + (size_t)pos * nparts;
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kErrThreads / 32; ++w) t += red[w];
    parts[(size_t)i * (h / JB) + jb] = zero_row ? (double)t : ldexp((double)t, 2 * ei);
    __threadfence();
    last = (atomicAdd(a.counters + pos, 1) == nparts - 1);
  }
  __syncthreads();
  if (!last) return;
  // the instance's last block: its partials in a fixed order
  __threadfence();
  double sum = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) sum += __ldcg(parts + t);
  redd[threadIdx.x] = sum;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) redd[threadIdx.x] += redd[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.esum[2 * pos] = redd[0];
    a.esum[2 * pos + 1] = a.normF2[b];
    a.counters[pos] = 0;
  }
}

}  // namespace

// Rows j per CTA: the largest of 32, 16, 8 that divides h (0: none).
static int err_rows(int h) { return h % 32 == 0 ? 32 : h % 16 == 0 ? 16 : h % 8 == 0 ? 8 : 0; }

bool err_sliced_supported(int h, int R) { return err_rows(h) > 0 && R >= 1 && R <= kMaxR; }

size_t err_sliced_scratch_bytes(int h, int R, int cnt) {
  (void)R;
  return carve_bytes<double>((size_t)cnt * h * (h / 8)) + carve_bytes<int>((size_t)cnt) + 1024;
}

void err_sliced_batch(const SliceView& sv, const double* normF2, const double* V, const double* Bcore, int h, int R,
                      int cnt, const int* amap, void* scratch, double* esum, cudaStream_t s) {
  if (!err_sliced_supported(h, R)) fail(TK_EINVAL, "err_sliced: shape out of range");
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  const int jbs = err_rows(h);
  double* parts = (double*)base;
  int* counters = (int*)(base + carve_bytes<double>((size_t)cnt * h * (h / 8)));
  TK_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * cnt, s));
  ErrSlicedArgs a{(const __nv_bfloat16*)sv.S, sv.Kp, sv.rowexp, normF2, h, R, V, Bcore, amap, jbs, parts, counters,
                  esum};
  const dim3 grid(h / jbs, h, cnt);
  if (R <= 16)
    k_err_sliced<16><<<grid, kErrThreads, 0, s>>>(a);
  else
    k_err_sliced<32><<<grid, kErrThreads, 0, s>>>(a);
  TK_LAUNCH("k_err_sliced");
}

}  // namespace tk
