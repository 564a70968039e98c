// (b) Gram G = A A^T of an unfolding A = F_(k) (Sec. 3.2) on the tcgen05
// tensor cores with FP64-class accuracy, from exact BF16 slices.
//
// Slicing (after Ozaki, Ogita, Oishi and Rump's error-free splitting).  Each
// row i of A is scaled by 2^-e_i with e_i the binary exponent of its largest
// entry, so every scaled entry x lies in (-1, 1).  x 2^47 is rounded to an
// integer and cut into balanced base-256 digits, x = sum_{s<6} d_s 2^(-7-8s)
// + O(2^-48) with |d_s| <= 128, using integer operations on the FP64 bits;
// slice s stores d_s 2^(-7-8s): at most 8 significant bits, exact in BF16.
//
// Products.  slice_s(i) slice_t(j) = d d' 2^(-14-8(s+t)) is exact, and the
// pairs of equal weight w = s + t share an accumulator in TMEM:
//   w = 0 .. 3   -> four exact FP32 accumulators: every partial sum is an
//                   integer multiple of 2^(-14-8w) of at most 2^24 of those
//                   units while (w+1) * 256 * 2^14 <= 2^24, i.e. for 256-deep
//                   K chunks (the tensor core's FP32 sums are exact there);
//   w = 4, 5     -> one FP32 accumulator each; the tensor core truncates,
//                   which costs about 2^-17 of terms that are 2^-32 and 2^-40
//                   of the leading one;
//   w >= 6       -> dropped (2^-48 of the leading term).
// The six B slices of a stage sit one after the other in shared memory, so
// B_0 .. B_{5-s} read as one operand of 64 (6 - s) rows: one MMA per A slice
// s (two where N would pass 256) forms every pair (s, t) at once into the
// accumulators w = s .. 5, which lie side by side in TMEM -- 8 MMAs per
// 16-deep K step instead of 21, each reading the A slice once.
// Every 256-deep K chunk the epilogue warps move the six accumulators into a
// 64-bit integer accumulator in units of 2^-44 (exact for w <= 3), so the
// chunk sums carry no rounding; the split-K partials stay 64-bit integers and
// are summed exactly (in two 32-bit halves), so each entry of G is the
// correctly rounded value of the integer sum times 2^(e_i + e_j - 44), the
// same for any split of K.
//
// Kernel layout (one CTA per 128 x 64 block of G touching its upper triangle,
// and one K range):
//   warp 0       TMA producer: 6 slices x 128 rows (A) and 6 x 64 rows (B) x
//                32 K per stage, SWIZZLE_64B, three stages;
//   warp 1       TMEM owner (6 accumulators of 64 columns) and the
//                single-thread tcgen05.mma issuer (8 MMAs x 2 K steps);
//   warps 2..17  epilogue: TMEM -> registers -> int64, one TMEM lane quadrant
//                and one 16-column group each.
// Every mbarrier wait is bounded; on a timeout the kernel raises a flag, lets
// in-flight copies and MMAs finish (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "slices.cuh"
#include "tc_common.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kTM = 128;               // rows of a block of G (M)
constexpr int kTN = 64;                // columns of a block of G (N)
constexpr int kAcc = 6;                // accumulators: w = 0 .. 5
constexpr int kKB = 32;                // K per stage (64-byte rows, SWIZZLE_64B)
constexpr int kChunkBlocks = 8;        // 8 x 32 = 256 K per exact chunk
constexpr int kStages = 3;                             // stages of A and B tiles
constexpr int kSliceBytesA = kTM * kKB * 2;            // 8 KB
constexpr int kSliceBytesB = kTN * kKB * 2;            // 4 KB
constexpr int kOperandBytesA = kSlices * kSliceBytesA;  // 48 KB
constexpr int kOperandBytesB = kSlices * kSliceBytesB;  // 24 KB
constexpr int kStageBytes = kOperandBytesA + kOperandBytesB;  // 72 KB
constexpr int kThreads = 576;                          // 18 warps
constexpr int kEpiWarps = 16;
constexpr int kEpiCols = kTN / 4;                      // 16 columns per epilogue warp
constexpr size_t kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;

static_assert(kAcc * kTN <= 512, "accumulators fit in TMEM");

// Row exponents: e_i with max_c |A(i,c)| < 2^e_i (frexp), -1000 for a zero row.
__device__ __forceinline__ long long unfold_at(int mode, int n1, int n2, int n3, int row, long long c) {
  if (mode == 0) return (long long)row * n2 * n3 + c;
  if (mode == 1) {
    const long long i = c / n3, l = c - i * n3;
    return (i * n2 + row) * n3 + l;
  }
  return c * n3 + row;
}

// blockIdx.z: instance (F + z sF, rowmax_bits + z n_mode).
__global__ void k_rowmax(const double* __restrict__ F, int mode, int n1, int n2, int n3, long long K,
                         unsigned long long* __restrict__ rowmax_bits, long long sF) {
  F += (long long)blockIdx.z * sF;
  rowmax_bits += (size_t)blockIdx.z * (mode == 0 ? n1 : mode == 1 ? n2 : n3);
  // grid: (row blocks of 32 rows for mode 2 / one row for modes 0,1, K chunks)
  if (mode == 2) {
    const int row = blockIdx.x * 32 + (threadIdx.x & 31);
    const int nrows = n3;
    double m = 0.0;
    if (row < nrows)
      for (long long c = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5); c < K;
           c += (long long)gridDim.y * (blockDim.x >> 5))
        m = fmax(m, fabs(F[c * n3 + row]));
    if (row < nrows) atomicMax(rowmax_bits + row, (unsigned long long)__double_as_longlong(m));
  } else {
    const int row = blockIdx.x;
    double m = 0.0;
    for (long long c = blockIdx.y * (long long)blockDim.x + threadIdx.x; c < K;
         c += (long long)gridDim.y * blockDim.x)
      m = fmax(m, fabs(F[unfold_at(mode, n1, n2, n3, row, c)]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rowmax_bits + row, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_rowexp(const unsigned long long* __restrict__ rowmax_bits, int nrows, int* __restrict__ rowexp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
    const double m = __longlong_as_double((long long)rowmax_bits[i]);
    int e = -1000;
    if (m > 0.0) frexp(m, &e);
    rowexp[i] = e;
  }
}

// Slices of one unfolding, written K-major: S[s][row][c], row stride Kp (a
// multiple of 32, zero padded).  32 x 32 tiles through shared memory so that
// both the read of F and the write of S are coalesced for every mode.
// blockIdx.z: instance (F + z sF, rowexp + z nrows, S + z 6 nrows Kp).
__global__ void k_slice(const double* __restrict__ F, int mode, int n1, int n2, int n3, int nrows, long long K,
                        long long Kp, const int* __restrict__ rowexp, __nv_bfloat16* __restrict__ S, long long sF) {
  __shared__ double tile[32][33];
  F += (long long)blockIdx.z * sF;
  rowexp += (size_t)blockIdx.z * nrows;
  S += (size_t)blockIdx.z * kSlices * nrows * Kp;
  const int r0 = blockIdx.y * 32;
  const long long c0 = (long long)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  // load: for mode 2 rows are contiguous in F, otherwise columns are
  for (int q = ty; q < 32; q += 8) {
    int row;
    long long c;
    if (mode == 2) {
      row = r0 + tx;
      c = c0 + q;
    } else {
      row = r0 + q;
      c = c0 + tx;
    }
    double v = 0.0;
    if (row < nrows && c < K) v = F[unfold_at(mode, n1, n2, n3, row, c)];
    if (mode == 2)
      tile[tx][q] = v;  // [row][c]
    else
      tile[q][tx] = v;
  }
  __syncthreads();
  const size_t plane = (size_t)nrows * Kp;
  for (int q = ty; q < 32; q += 8) {
    const int row = r0 + q;
    const long long c = c0 + tx;
    if (row >= nrows || c >= Kp) continue;
    int d[kSlices];
    slice_digits(tile[q][tx], rowexp[row], d);
    const size_t base = (size_t)row * Kp + c;
#pragma unroll
    for (int s = 0; s < kSlices; ++s) S[s * plane + base] = slice_value(d[s], s);
  }
}

struct TcArgs {
  int nrows;
  int nrt, nct;           // row tiles (of 128) and column tiles (of 64)
  int nblocks;            // blocks of G touching the upper triangle
  int nsplit;             // K splits per instance
  int kblocks_per_split;  // k-blocks (of 32) per CTA
  int kblocks_total;
  long long* partials;    // [instance][split][block][128][64], units of 2^-44
  int* err;
};

// Block b (in row-major order over blocks with i*128 < (j+1)*64) -> (i, j).
__host__ __device__ __forceinline__ void block_of(int b, int nrt, int nct, int& bi, int& bj) {
  for (int i = 0; i < nrt; ++i) {
    const int j0 = (i * kTM) / kTN;
    const int cnt = nct - j0;
    if (b < cnt) {
      bi = i;
      bj = j0 + b;
      return;
    }
    b -= cnt;
  }
  bi = nrt;
  bj = nct;
}

__host__ __device__ __forceinline__ int block_count(int nrt, int nct) {
  int c = 0;
  for (int i = 0; i < nrt; ++i) {
    const int j0 = (i * kTM) / kTN;
    c += (nct > j0) ? nct - j0 : 0;
  }
  return c;
}

// Index of block (i, j) in that order.
__device__ __forceinline__ int block_index(int i, int j, int nct) {
  int b = 0;
  for (int r = 0; r < i; ++r) b += nct - (r * kTM) / kTN;
  return b + j - (i * kTM) / kTN;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapB, TcArgs args) {
  TK_PDL_ENTRY();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + kStages * kStageBytes);
  uint64_t* full = bars;                 // [kStages]
  uint64_t* empty = bars + kStages;      // [kStages]
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* drain = acc_full + 2;
  uint32_t* tmem_slot = (uint32_t*)(acc_full + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int inst = blockIdx.z;  // instance of a batch (one slice tensor each)
  int bi, bj;
  block_of(blockIdx.x, args.nrt, args.nct, bi, bj);
  const int kb0 = blockIdx.y * args.kblocks_per_split;
  const int kb1 = min(kb0 + args.kblocks_per_split, args.kblocks_total);
  const int nkb = kb1 - kb0;
  const int nchunks = (nkb + kChunkBlocks - 1) / kChunkBlocks;
  const int nst = kStages;
  const int sstride = kStageBytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, kEpiWarps);
    tc::mbar_init(drain, 1);
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int k = 0; k < nkb; ++k) {
        const int st = k % nst;
        const uint32_t use = k / nst;
        if (k >= nst && !tc::mbar_wait(&empty[st], (use - 1) & 1, args.err)) break;
        unsigned char* sa = smem + st * sstride;
        tc::mbar_expect_tx(&full[st], kStageBytes);
        tc::tma_load_4d(sa, &tmapA, &full[st], (kb0 + k) * kKB, bi * kTM, 0, inst);
        tc::tma_load_4d(sa + kOperandBytesA, &tmapB, &full[st], (kb0 + k) * kKB, bj * kTN, 0, inst);
        issued = k + 1;
      }
      // copies still in flight must land before the CTA exits
      for (int k = max(0, issued - nst); k < issued; ++k)
        tc::mbar_wait(&full[k % nst], (k / nst) & 1, args.err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      int k = 0;
      for (int ch = 0; ch < nchunks && ok; ++ch) {
        if (ch > 0 && !tc::mbar_wait(acc_empty, (ch - 1) & 1, args.err)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const int kend = min(nkb, (ch + 1) * kChunkBlocks);
        for (int k0 = k; k < kend; ++k) {
          const int st = k % nst;
          if (!tc::mbar_wait(&full[st], (k / nst) & 1, args.err)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          unsigned char* sa = smem + st * sstride;
          unsigned char* sb = sa + kOperandBytesA;
          // descriptors of slice 0; slice s and K step kk add (s * slice bytes + kk * 32 B) / 16
          const uint64_t da0 = tc::smem_desc(sa, 512, tc::kSwizzle64B);
          const uint64_t db0 = tc::smem_desc(sb, 512, tc::kSwizzle64B);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            // the chunk's first K step starts the accumulators: the two MMAs of
            // A slice 0 write every w = 0 .. 5 before any other MMA adds to it
            const uint32_t acc_on = (k == k0 && kk == 0) ? 0u : 1u;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              // (A slice, first B slice, B slices): accumulators w = s + t0 ..
              const int sl = e < 2 ? 0 : (e < 4 ? 1 : e - 2);
              const int t0 = (e == 1 || e == 3) ? 4 : 0;
              const int nt = e == 0 || e == 2 || e == 4 ? 4 : (e == 1 ? 2 : (e == 3 ? 1 : 6 - sl));
              const uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN * nt);
              const uint32_t dt = tmem + (uint32_t)((sl + t0) * kTN);
              const uint64_t da = da0 + (uint64_t)(sl * (kSliceBytesA >> 4) + 2 * kk);
              const uint64_t db = db0 + (uint64_t)(t0 * (kSliceBytesB >> 4) + 2 * kk);
              tc::mma_bf16(dt, da, db, idesc, sl == 0 ? acc_on : 1u);
            }
          }
          tc::mma_commit(&empty[st]);  // frees the stage once these MMAs finish
        }
        if (ok) tc::mma_commit(acc_full);
      }
      // every MMA issued must finish before TMEM is released
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, args.err);
    }
  } else {
    // ---------------- epilogue: TMEM -> int64 ----------------
    const int q = warp & 3;             // TMEM lane quadrant of this warp
    const int grp = (warp - 2) >> 2;    // 16-column group
    const int row = q * 32 + lane;
    long long V[kEpiCols];
#pragma unroll
    for (int j = 0; j < kEpiCols; ++j) V[j] = 0;
    bool ok = true;
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + grp * kEpiCols;
    for (int ch = 0; ch < nchunks; ++ch) {
      if (!tc::mbar_wait(acc_full, ch & 1, args.err)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      // w = 0..3 are integer multiples of 2^(-14-8w): exact into units of
      // 2^-44; the w = 4 and w = 5 accumulators are rounded to that unit
#pragma unroll
      for (int h = 0; h < kEpiCols / 8; ++h) {
        uint32_t r[8];
        tc::tmem_ld8(base + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 16384.0f) * (1LL << 30);
        tc::tmem_ld8(base + kTN + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 4194304.0f) * (1LL << 22);
        tc::tmem_ld8(base + 2 * kTN + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 1073741824.0f) * (1LL << 14);
        tc::tmem_ld8(base + 3 * kTN + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 274877906944.0f) * (1LL << 6);
        tc::tmem_ld8(base + 4 * kTN + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 17592186044416.0f);
        tc::tmem_ld8(base + 5 * kTN + h * 8, r);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          V[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * 17592186044416.0f);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(acc_empty);
    }
    if (ok) {
      long long* out = args.partials +
                       (((size_t)inst * args.nsplit + blockIdx.y) * args.nblocks + blockIdx.x) * kTM * kTN +
                       (size_t)row * kTN + grp * kEpiCols;
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) out[j] = V[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// G_b[gi][gj] = G_b[gj][gi] = 2^(e_gi + e_gj - 44) sum_split P[b][split][block(gi, gj)][..],
// gi <= gj, for every instance b (row exponents rowexp[b * n + i]).  The
// integer partials (each below 2^62) are summed exactly as high and low
// 32-bit halves and rounded to FP64 once.  SG lanes share one entry, each
// summing every SG-th split, and combine their integer sums by shuffles
// (exact, so the result does not depend on SG).
// The last B blocks (with norm.part set) sum the instances' |F|^2 partials
// instead (the grid-stride loop spans the first nred blocks).
template <int SG>
__global__ void k_tc_reduce(const long long* __restrict__ P, int nsplit, int nct, int nblocks, int n, int B,
                            const int* __restrict__ rowexp, double* __restrict__ G, int nred, NormParts norm) {
  TK_PDL_ENTRY();
  if ((int)blockIdx.x >= nred) {
    const int b = blockIdx.x - nred;
    norm_parts_block(norm.part + (size_t)b * norm.nparts, norm.nparts, norm.normF2 + b);
    return;
  }
  const long long per = (long long)n * n;
  const long long total = per * B;
  const int g = threadIdx.x % SG;
  const long long stride = (long long)nred * blockDim.x / SG;
  for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / SG; e - (threadIdx.x % 32) / SG < total;
       e += stride) {
    // every lane of a warp runs the shuffles: lanes past the end add zeros
    const bool live = e < total;
    const int b = live ? (int)(e / per) : 0;
    const long long r = live ? e - (long long)b * per : 0;
    const int gi = (int)(r / n), gj = (int)(r % n);
    const bool want = live && gi <= gj;
    long long hi = 0, lo = 0;
    if (want) {
      const int bi = gi / kTM, bj = gj / kTN;
      const int blk = block_index(bi, bj, nct);
      const size_t off = (size_t)(gi - bi * kTM) * kTN + (gj - bj * kTN);
      const long long* src = P + ((size_t)b * nsplit * nblocks + blk) * kTM * kTN + off;
      const size_t sstride = (size_t)nblocks * kTM * kTN;
#pragma unroll 4
      for (int sp = g; sp < nsplit; sp += SG) {
        const long long v = src[sp * sstride];
        hi += v >> 32;           // floor(v / 2^32)
        lo += v & 0xFFFFFFFFLL;  // v - 2^32 floor(v / 2^32), in [0, 2^32)
      }
    }
#pragma unroll
    for (int o = SG / 2; o > 0; o >>= 1) {
      hi += __shfl_xor_sync(0xffffffffu, hi, o);
      lo += __shfl_xor_sync(0xffffffffu, lo, o);
    }
    if (want && g == 0) {
      hi += lo >> 32;
      lo &= 0xFFFFFFFFLL;
      const double sum = fma((double)hi, 4294967296.0, (double)lo);  // one rounding
      const int ei = rowexp[(size_t)b * n + gi], ej = rowexp[(size_t)b * n + gj];
      const double v = (ei > -1000 && ej > -1000) ? ldexp(sum, ei + ej - 44) : 0.0;
      double* Gb = G + (size_t)b * per;
      Gb[(long long)gi * n + gj] = v;
      Gb[(long long)gj * n + gi] = v;
    }
  }
}

struct TcPlan {
  int nrows, nrt, nct, nblocks, nsplit, kb_per_split, kb_total;
  long long K, Kp;
};

TcPlan tc_plan(const int n[3], int mode, int sm_count, int B = 1) {
  TcPlan p;
  p.nrows = n[mode];
  p.K = (long long)n[0] * n[1] * n[2] / p.nrows;
  p.Kp = (p.K + kKB - 1) / kKB * kKB;
  p.kb_total = (int)(p.Kp / kKB);
  p.nrt = (p.nrows + kTM - 1) / kTM;
  p.nct = (p.nrows + kTN - 1) / kTN;
  p.nblocks = block_count(p.nrt, p.nct);
  // about one wave of CTAs; splits of whole 256-deep chunks, at most 256 chunks
  // each so that the int64 sums stay below 2^62
  const int chunks = (p.kb_total + kChunkBlocks - 1) / kChunkBlocks;
  int want = std::max(1, sm_count / (p.nblocks * B));
  want = std::max(want, (chunks + 255) / 256);
  want = std::min(want, chunks);
  const int chunks_per_split = (chunks + want - 1) / want;
  p.kb_per_split = chunks_per_split * kChunkBlocks;
  p.nsplit = (p.kb_total + p.kb_per_split - 1) / p.kb_per_split;
  return p;
}

// ---------------------------------------------------------------------------
// Autotuning of the K split.  The Gram does not depend on how K is split
// (exact integer chunk sums), so the split is free to pick for speed alone.
// The default plan aims at one wave of CTAs; when tuning is on, the first
// launch of a (SMs, rows, K, instances) shape also times 2, 4 and 8 times as
// many chunks per CTA (fewer CTAs, longer pipelines; never more partial sums
// than the default, so the scratch sizing holds) with CUDA events and keeps
// the fastest.  Choices live in a process-wide table, optionally read from and
// written to a JSON file ({"<key>": chunks per split, ...}).
// ---------------------------------------------------------------------------
struct TuneTable {
  std::mutex mu;
  bool on = false;
  std::string path;
  std::map<std::string, int> cps;  // chunks per split
};
TuneTable& tune_table() {
  static TuneTable t;
  return t;
}

// Batch sizes share a choice within powers of two.
std::string tune_key(int sm_count, const TcPlan& p, int B) {
  int bb = 1;
  while (bb < B) bb <<= 1;
  return "sm" + std::to_string(sm_count) + "/gram_tc/rows" + std::to_string(p.nrows) + "/K" + std::to_string(p.K) +
         "/B" + std::to_string(bb);
}

void tune_save_locked(const TuneTable& t) {
  if (t.path.empty()) return;
  const std::string tmp = t.path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : t.cps)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < t.cps.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), t.path.c_str());
}

// Entries of the form "key": integer (the format tune_save_locked writes).
void tune_load_locked(TuneTable& t) {
  if (t.path.empty()) return;
  FILE* f = std::fopen(t.path.c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t colon = text.find(':', end);
    if (colon == std::string::npos) break;
    const int v = std::atoi(text.c_str() + colon + 1);
    if (v > 0) t.cps[key] = v;
    pos = text.find_first_of(",}", colon);
    if (pos == std::string::npos) break;
  }
}

TcPlan with_chunks_per_split(TcPlan p, int cps) {
  const int chunks = (p.kb_total + kChunkBlocks - 1) / kChunkBlocks;
  cps = std::max(1, std::min(cps, std::min(chunks, 256)));
  p.kb_per_split = cps * kChunkBlocks;
  p.nsplit = (p.kb_total + p.kb_per_split - 1) / p.kb_per_split;
  return p;
}

// Slices of B instances, [b][s][row][Kp] bf16: dims (Kp, nrows, 6, B).
CUtensorMap slice_map(PFN_cuTensorMapEncodeTiled_v12000 enc, void* S, long long Kp, int nrows, int B,
                      int box_rows) {
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)nrows, (cuuint64_t)kSlices, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * nrows, (cuuint64_t)Kp * 2 * nrows * kSlices};
  cuuint32_t box[4] = {kKB, (cuuint32_t)box_rows, kSlices, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, S, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(TK_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return map;
}

// The tensor-core Gram and its reduction over B instances whose slices are
// at S ([b][s][row][Kp]) and row exponents at rowexp ([b][row]).
void run_tc_gram(const TcPlan& p, int B, __nv_bfloat16* S, const int* rowexp, long long* P, double* G, int* err,
                 cudaStream_t s, Profiler* pf, NormParts norm = NormParts{nullptr, 0, nullptr}) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encode_fn();
  if (!enc) fail(TK_ECUDA, "cuTensorMapEncodeTiled is not available");
  const CUtensorMap mapA = slice_map(enc, S, p.Kp, p.nrows, B, kTM);
  const CUtensorMap mapB = slice_map(enc, S, p.Kp, p.nrows, B, kTN);
  once_per_device((const void*)&k_gram_tc, [] {
    TK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  });
  TcPlan q = p;
  {
    TuneTable& t = tune_table();
    std::lock_guard<std::mutex> lock(t.mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (t.on && cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
      const std::string key = tune_key(152, p, B);
      auto it = t.cps.find(key);
      if (it == t.cps.end()) {
        const int c0 = p.kb_per_split / kChunkBlocks;
        int best = c0;
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        TK_CUDA(cudaEventCreate(&e0));
        TK_CUDA(cudaEventCreate(&e1));
        for (int f = 1; f <= 8; f *= 2) {
          const TcPlan c = with_chunks_per_split(p, c0 * f);
          if (f > 1 && c.nsplit == with_chunks_per_split(p, c0 * f / 2).nsplit) break;
          TcArgs ca{c.nrows, c.nrt, c.nct, c.nblocks, c.nsplit, c.kb_per_split, c.kb_total, P, err};
          float ms = 0.0f;
          for (int rep = 0; rep < 4; ++rep) {  // one warm-up, three timed
            TK_CUDA(cudaEventRecord(e0, s));
            launch_pdl("k_gram_tc", k_gram_tc, dim3(c.nblocks, c.nsplit, B), dim3(kThreads), kSmemBytes, s, mapA,
                       mapB, ca);
            TK_CUDA(cudaEventRecord(e1, s));
            TK_CUDA(cudaEventSynchronize(e1));
            float t_ms = 0.0f;
            TK_CUDA(cudaEventElapsedTime(&t_ms, e0, e1));
            if (rep > 0) ms += t_ms;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best = c0 * f;
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        it = t.cps.emplace(key, best).first;
        tune_save_locked(t);
      }
      q = with_chunks_per_split(p, it->second);
      if (q.nsplit > p.nsplit) q = p;  // a stored choice never needs more partials than reserved
    }
  }
  TcArgs a{q.nrows, q.nrt, q.nct, q.nblocks, q.nsplit, q.kb_per_split, q.kb_total, P, err};
  if (pf) pf->begin(TK_STAGE_GRAM_TC, s);
  launch_pdl("k_gram_tc", k_gram_tc, dim3(q.nblocks, q.nsplit, B), dim3(kThreads), kSmemBytes, s, mapA, mapB, a);
  if (pf) pf->end(s);
  const long long total = (long long)q.nrows * q.nrows * B;
  const int extra = norm.part != nullptr ? B : 0;
  if (q.nsplit >= 8) {
    const int nred = (int)std::min<long long>((8 * total + 255) / 256, 8192);
    launch_pdl("k_tc_reduce", k_tc_reduce<8>, dim3((unsigned)(nred + extra)), dim3(256), 0, s, P, q.nsplit, q.nct,
               q.nblocks, q.nrows, B, rowexp, G, nred, norm);
  } else {
    const int nred = (int)std::min<long long>((total + 255) / 256, 8192);
    launch_pdl("k_tc_reduce", k_tc_reduce<1>, dim3((unsigned)(nred + extra)), dim3(256), 0, s, P, q.nsplit, q.nct,
               q.nblocks, q.nrows, B, rowexp, G, nred, norm);
  }
}

}  // namespace

void gram_tune_config(bool on, const char* path) {
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lock(t.mu);
  t.on = on;
  if (path != nullptr) {  // a new cache file: its choices replace the ones held
    t.path = path;
    t.cps.clear();
    tune_load_locked(t);
  }
}

int gram_tune_entries() {
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lock(t.mu);
  return (int)t.cps.size();
}

size_t gram_sliced_scratch_bytes(const int n[3], int mode, int B) {
  const TcPlan p = tc_plan(n, mode, 152, B);
  size_t b = 0;
  b += carve_bytes<unsigned long long>((size_t)B * p.nrows);                   // row max bits
  b += carve_bytes<int>((size_t)B * p.nrows);                                  // row exponents
  b += carve_bytes<__nv_bfloat16>((size_t)B * kSlices * p.nrows * p.Kp);       // slices
  b += carve_bytes<long long>((size_t)B * p.nsplit * p.nblocks * kTM * kTN);  // partials
  return b + 4096;
}

void gram_sliced_batch(const double* F, const int n[3], int mode, int B, double* G, void* scratch, int* err,
                       cudaStream_t s, Profiler* pf) {
  // one plan (for 152 SMs and this batch) fixes both the scratch layout and
  // the grid; G does not depend on it (exact integer sums over K)
  const TcPlan p = tc_plan(n, mode, 152, B);
  const long long sF = (long long)n[0] * n[1] * n[2];
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    char* q = base + off;
    off += (bytes + 255) & ~size_t(255);
    return q;
  };
  unsigned long long* rowmax = (unsigned long long*)carve(sizeof(unsigned long long) * B * p.nrows);
  int* rowexp = (int*)carve(sizeof(int) * (size_t)B * p.nrows);
  __nv_bfloat16* S = (__nv_bfloat16*)carve(sizeof(__nv_bfloat16) * (size_t)B * kSlices * p.nrows * p.Kp);
  long long* P = (long long*)carve(sizeof(long long) * (size_t)B * p.nsplit * p.nblocks * kTM * kTN);

  TK_CUDA(cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * B * p.nrows, s));
  if (mode == 2) {
    dim3 g((p.nrows + 31) / 32, (unsigned)std::min<long long>(1024, (p.K + 7) / 8), B);
    k_rowmax<<<g, 256, 0, s>>>(F, mode, n[0], n[1], n[2], p.K, rowmax, sF);
  } else {
    dim3 g(p.nrows, (unsigned)std::min<long long>(64, (p.K + 255) / 256), B);
    k_rowmax<<<g, 256, 0, s>>>(F, mode, n[0], n[1], n[2], p.K, rowmax, sF);
  }
  TK_LAUNCH("k_rowmax");
  k_rowexp<<<(B * p.nrows + 255) / 256, 256, 0, s>>>(rowmax, B * p.nrows, rowexp);
  TK_LAUNCH("k_rowexp");
  {
    dim3 g((unsigned)(p.Kp / 32), (p.nrows + 31) / 32, B);
    k_slice<<<g, 256, 0, s>>>(F, mode, n[0], n[1], n[2], p.nrows, p.K, p.Kp, rowexp, S, sF);
    TK_LAUNCH("k_slice");
  }
  run_tc_gram(p, B, S, rowexp, P, G, err, s, pf);
}

// The Gram from slices already written into the scratch (by a sampling
// kernel that sliced the mode-1 rows while it evaluated them).
void gram_sliced_prepared(const int n[3], int B, double* G, void* scratch, int* err, cudaStream_t s,
                          Profiler* pf, NormParts norm) {
  const TcPlan p = tc_plan(n, 0, 152, B);
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    char* q = base + off;
    off += (bytes + 255) & ~size_t(255);
    return q;
  };
  carve(sizeof(unsigned long long) * B * p.nrows);
  int* rowexp = (int*)carve(sizeof(int) * (size_t)B * p.nrows);
  __nv_bfloat16* S = (__nv_bfloat16*)carve(sizeof(__nv_bfloat16) * (size_t)B * kSlices * p.nrows * p.Kp);
  long long* P = (long long*)carve(sizeof(long long) * (size_t)B * p.nsplit * p.nblocks * kTM * kTN);
  run_tc_gram(p, B, S, rowexp, P, G, err, s, pf, norm);
}

SliceView gram_slices_view(void* scratch, const int n[3], int mode, int B) {
  const TcPlan p = tc_plan(n, mode, 152, B);
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    char* q = base + off;
    off += (bytes + 255) & ~size_t(255);
    return q;
  };
  carve(sizeof(unsigned long long) * B * p.nrows);
  SliceView v;
  v.rowexp = (const int*)carve(sizeof(int) * (size_t)B * p.nrows);
  v.S = carve(sizeof(__nv_bfloat16) * (size_t)B * kSlices * p.nrows * p.Kp);
  v.nrows = p.nrows;
  v.Kp = p.Kp;
  return v;
}

void gram_sliced_bf16(const double* F, const int n[3], int mode, double* G, void* scratch, int* err,
                      cudaStream_t s) {
  gram_sliced_batch(F, n, mode, 1, G, scratch, err, s);
}

}  // namespace tk
