// Exact BF16 slicing of FP64 values (after Ozaki, Ogita, Oishi and Rump's
// error-free splitting), shared by the tensor-core Gram and TTM kernels.
//
// A value x of a row (or column) whose largest magnitude is below 2^e is
// written as x 2^(7 - e) = sum_{s<6} d_s 2^(-8s) + O(2^-41), |d_s| <= 128, by
// rounding x 2^(47 - e) to an integer T with integer operations on the FP64
// bits and cutting T into balanced base-256 digits; slice s stores
// d_s 2^(-7-8s), exact in BF16.  A product of slices s and t has weight
// w = s + t; the 21 pairs with w <= 5 are kept.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

namespace tk {
namespace {

constexpr int kSlices = 6;
constexpr int kMaxWeight = 5;  // pairs with s + t <= 5 are kept (21 pairs)

// Slice pairs (s, t) with s + t <= kMaxWeight, in order of weight.
constexpr int kPairs = 21;
__constant__ int kPairS[kPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
__constant__ int kPairT[kPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};
static_assert(kPairs == (kMaxWeight + 1) * (kMaxWeight + 2) / 2, "pair table covers s + t <= kMaxWeight");

// Balanced base-256 digits of x 2^(7 - e): T = round(|x| 2^(47 - e)) from the
// FP64 bits with integer operations (|x| < 2^e, so T < 2^47), then digits from
// the bottom: x 2^(7 - e) = sum_s d_s 2^(-8s) + O(2^-41), |d_s| <= 128.
static_assert(kSlices == 6, "slice_digits cuts T into 3 + 3 digits");
__device__ __forceinline__ void slice_digits(double xv, int e, int (&d)[kSlices]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(xv);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long T = 0;
  if (ex != 0 && e > -1000) {
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int rs = 1028 + e - ex;  // right shift of the 53-bit mantissa, >= 6
    if (rs < 64) T = (long long)((mant + (1ull << (rs - 1))) >> rs);
    if (bits >> 63) T = -T;
  }
  // in 32-bit arithmetic: T = hi 2^24 + lo with lo balanced in [-2^23, 2^23);
  // the three low digits come from lo (their carry goes to hi), the other
  // three from hi; the same digits as cutting T from the bottom in 64 bits
  const int lo = (int)((T + 0x800000) & 0xFFFFFF) - 0x800000;
  int hi = (int)((T - lo) >> 24);
  int t = lo;
#pragma unroll
  for (int s = kSlices - 1; s >= 3; --s) {
    const int r = ((t + 128) & 255) - 128;
    d[s] = r;
    t = (t - r) >> 8;
  }
  hi += t;
#pragma unroll
  for (int s = 2; s >= 1; --s) {
    const int r = ((hi + 128) & 255) - 128;
    d[s] = r;
    hi = (hi - r) >> 8;
  }
  d[0] = hi;
}

__device__ __forceinline__ __nv_bfloat16 slice_value(int d, int s) {
  return __float2bfloat16_rn(__int2float_rn(d) * __int_as_float((127 - 7 - 8 * s) << 23));  // d 2^(-7-8s)
}


// The CUDA driver API entry cuTensorMapEncodeTiled, looked up once per process.
inline PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace
}  // namespace tk
