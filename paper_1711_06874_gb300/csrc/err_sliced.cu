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
// hi + lo (two floats, about 48 significant bits), a product of two floats
// is split exactly (a b = p + e, e = fma(a, b, -p)) and sums keep their
// rounding error (the two-sum of Knuth; Dekker's splitting into float pairs).
// Per entry the reconstruction is accurate to about 2^-44 of the entry; the
// residual, formed from the three exact partial sums of the slices, to about
// 2^-23 of itself; its squares are summed in FP32 per thread and block and in
// FP64 across blocks.  The reported relative error carries about six
// correct digits.
//
// One CTA per (row i, block of 8 rows j) of one instance: it forms the
// 8 x R block W2(j, c) = sum_b V(j, b) W1(i, b, c) of W2 = B x_1 V x_2 V in
// shared memory, then each thread takes columns l: X = sum_c V(l, c) W2(j, c).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "slices.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kJB = 8;         // rows j per CTA
constexpr int kErrThreads = 128;
constexpr int kMaxR = 32;      // padded rank handled here

struct FF {
  float hi, lo;
};

// a + b = s + e exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += x y for float-float x, y: the leading product exactly (p + e), the
// cross terms in FP32 (about 2^-48 of the product), x.lo y.lo dropped.
__device__ __forceinline__ void ff_fma(FF& acc, const FF x, const FF y) {
  const float p = x.hi * y.hi;
  const float e = fmaf(x.hi, y.hi, -p);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e + fmaf(x.hi, y.lo, x.lo * y.hi);
}

// hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ FF ff_norm(FF a) {
  const float s = a.hi + a.lo;
  return FF{s, a.lo - (s - a.hi)};
}

// x = hi + lo for an FP64 value (about 48 bits kept).
__global__ void k_ff_split(const double* __restrict__ x, long long n, FF* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double v = x[t];
    const float hi = __double2float_rn(v);
    out[t] = FF{hi, __double2float_rn(v - (double)hi)};
  }
}

struct ErrSlicedArgs {
  const __nv_bfloat16* S;  // bucket: [b][6][h][Kp]
  long long Kp;
  const int* rowexp;       // bucket: [b][h]
  int h, R;
  const FF* V;             // group: [pos][h][R]
  const FF* W1;            // group: [pos][h][R][R]
  const int* amap;         // group position -> bucket instance
  double* partials;        // group: [pos][h][h / kJB]
};

template <int kR>
__global__ void __launch_bounds__(kErrThreads) k_err_sliced(ErrSlicedArgs a) {
  __shared__ FF W1s[kR * kR];     // W1(i, b, c)
  __shared__ FF Vj[kJB * kR];     // V(j0 + jj, b)
  __shared__ FF W2s[kJB * kR];    // W2(j0 + jj, c)
  __shared__ float red[kErrThreads / 32];
  const int h = a.h, R = a.R;
  const int jb = blockIdx.x, i = blockIdx.y, pos = blockIdx.z;
  const int j0 = jb * kJB;
  const int b = a.amap[pos];
  const FF* V = a.V + (size_t)pos * h * R;
  for (int e = threadIdx.x; e < kR * kR; e += blockDim.x) {
    const int bb = e / kR, c = e - bb * kR;
    W1s[e] = (bb < R && c < R) ? a.W1[(((size_t)pos * h + i) * R + bb) * R + c] : FF{0.0f, 0.0f};
  }
  for (int e = threadIdx.x; e < kJB * kR; e += blockDim.x) {
    const int jj = e / kR, c = e - jj * kR;
    Vj[e] = (c < R) ? V[(size_t)(j0 + jj) * R + c] : FF{0.0f, 0.0f};
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kJB * kR; e += blockDim.x) {
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
    for (int c = 0; c < kR; ++c) vl[c] = (c < R) ? V[(size_t)l * R + c] : FF{0.0f, 0.0f};
#pragma unroll 1
    for (int jj = 0; jj < kJB; ++jj) {
      FF x{0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < kR; ++c)
        if (c < R) ff_fma(x, vl[c], W2s[jj * kR + c]);
      const __nv_bfloat16* sp = Srow + (size_t)jj * h + l;
      float A = 0.0f, Bv = 0.0f, Cv = 0.0f;
      if (!zero_row) {
        // sums of two slices are exact: 8-bit digits eight binary places apart
        A = __bfloat162float(sp[0]) + __bfloat162float(sp[plane]);
        Bv = __bfloat162float(sp[2 * plane]) + __bfloat162float(sp[3 * plane]);
        Cv = __bfloat162float(sp[4 * plane]) + __bfloat162float(sp[5 * plane]);
      }
      const float xh = x.hi * sc, xl = x.lo * sc;
      const float p1 = A - xh;  // exact while xh is within a factor 2 of A
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
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kErrThreads / 32; ++w) t += red[w];
    const double v = zero_row ? (double)t : ldexp((double)t, 2 * ei);
    a.partials[((size_t)pos * h + i) * (h / kJB) + jb] = v;
  }
}

// esum[2 pos] = sum of the partials of position pos (fixed order),
// esum[2 pos + 1] = |Fh|^2 of its instance.
__global__ void k_err_sliced_final(const double* __restrict__ partials, int nparts, const double* __restrict__ normF2,
                                   const int* __restrict__ amap, double* __restrict__ esum) {
  __shared__ double red[256];
  const int pos = blockIdx.x;
  partials += (size_t)pos * nparts;
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += partials[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    esum[2 * pos] = red[0];
    esum[2 * pos + 1] = normF2[amap[pos]];
  }
}

}  // namespace

bool err_sliced_supported(int h, int R) { return h % kJB == 0 && R >= 1 && R <= kMaxR; }

size_t err_sliced_scratch_bytes(int h, int R, int cnt) {
  return carve_bytes<FF>((size_t)cnt * h * R) + carve_bytes<FF>((size_t)cnt * h * R * R) +
         carve_bytes<double>((size_t)cnt * h * (h / kJB)) + 1024;
}

void err_sliced_batch(const SliceView& sv, const double* normF2, const double* V, const double* W1, int h, int R,
                      int cnt, const int* amap, void* scratch, double* esum, cudaStream_t s) {
  if (!err_sliced_supported(h, R)) fail(TK_EINVAL, "err_sliced: shape out of range");
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  FF* Vff = (FF*)base;
  FF* W1ff = (FF*)(base + carve_bytes<FF>((size_t)cnt * h * R));
  double* parts = (double*)((char*)W1ff + carve_bytes<FF>((size_t)cnt * h * R * R));
  const long long nV = (long long)cnt * h * R, nW = (long long)cnt * h * R * R;
  k_ff_split<<<(unsigned)std::min<long long>((nV + 255) / 256, 1024), 256, 0, s>>>(V, nV, Vff);
  TK_LAUNCH("k_ff_split");
  k_ff_split<<<(unsigned)std::min<long long>((nW + 255) / 256, 2048), 256, 0, s>>>(W1, nW, W1ff);
  TK_LAUNCH("k_ff_split");
  ErrSlicedArgs a{(const __nv_bfloat16*)sv.S, sv.Kp, sv.rowexp, h, R, Vff, W1ff, amap, parts};
  const dim3 grid(h / kJB, h, cnt);
  if (R <= 16)
    k_err_sliced<16><<<grid, kErrThreads, 0, s>>>(a);
  else
    k_err_sliced<32><<<grid, kErrThreads, 0, s>>>(a);
  TK_LAUNCH("k_err_sliced");
  k_err_sliced_final<<<cnt, 256, 0, s>>>(parts, h * (h / kJB), normF2, amap, esum);
  TK_LAUNCH("k_err_sliced_final");
}

}  // namespace tk
