// (d) First product of the TTM chain of the core (Sec. 3.1, 3.2):
// T1 = Fh x_3 U_3^T, a (h1 h2) x h3 by h3 x R product, on the tcgen05 tensor
// cores with FP64-class accuracy.  The A operand reuses the exact BF16 slices
// of Fh that the mode-1 Gram made (rows i scaled by 2^-e_i; viewed with rows
// (i, k) and K = l when the slice row length equals h2 h3); the B operand is
// U_3 sliced per column c (scale 2^-f_c).  The 21 slice pairs with s + t <= 5
// go to FP32 TMEM accumulators per weight w = s + t (w = 0..3 exact; w = 4, 5
// apart for Np <= 64, where one MMA per A slice covers its B slices 0 .. 5 - s
// as in the Gram, and merged for Np = 96, one MMA per pair) over 256-deep
// chunks, moved to int64 in units of 2^-44 as in the Gram, and the output is
// that integer times 2^(e_i + f_c - 44): no rounding but the slices' own, the
// same for any batch.
//
// A CTA streams a run of consecutive (instance, 128-row tile) pairs of the
// group (about one run per SM): warp 0 issues the TMA loads (6 slices x 128
// rows of A, 6 x Np rows of B per 32-deep K block, two stages, the ring
// running on across tiles, so the next tile's loads overlap this tile's
// drain), warp 1 owns TMEM and issues the MMAs, warps 2..17 drain TMEM (one
// lane quadrant and Np/4 columns each) and write each tile's rows.  Bounded
// waits as in the Gram.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "slices.cuh"
#include "tc_common.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kTM = 128;       // rows (i, k) per CTA
constexpr int kKB = 32;        // K per stage
constexpr int kChunkBlocks = 8;  // 256-deep exact chunks
constexpr int kStages = 2;
constexpr int kMaxNp = 96;     // padded output columns (multiple of 32)
constexpr int kAcc = 5;
constexpr int kSliceBytesA = kTM * kKB * 2;                        // 8 KB
constexpr int kOperandBytesA = kSlices * kSliceBytesA;             // 48 KB
constexpr int kMaxOperandBytesB = kSlices * kMaxNp * kKB * 2;      // 36 KB
constexpr int kStageBytes = kOperandBytesA + kMaxOperandBytesB;    // 84 KB
constexpr int kThreads = 576;
constexpr int kEpiWarps = 16;
constexpr size_t kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
static_assert(kAcc * kMaxNp <= 512, "accumulators fit in TMEM");

struct TtmArgs {
  int M;           // rows h1 h2
  int h1, h2, h3;  // octant extents (K = h3)
  int R, Np;       // output columns and their padding
  int nkb;         // K blocks of 32
  int ntiles;      // row tiles of kTM per instance
  int tiles_per_cta;  // consecutive (instance, tile) pairs a CTA streams
  int Bg;             // instances of the group
  const int* amap;    // group instance -> bucket instance
  const int* rowexp;  // bucket: [b][h1]
  const int* colexp;  // group: [j][Np]
  double* T1;         // group: [j][M][R]
  int* err;
};

// Column slices of U (Up: [j][h3][R] FP64) -> colexp [j][Np], BS [j][6][Np][h3]
// BF16; padding columns c >= R are zero.
__global__ void k_bslice(const double* __restrict__ Up, int h3, int R, int Np, int* __restrict__ colexp,
                         __nv_bfloat16* __restrict__ BS) {
  TK_PDL_ENTRY();
  __shared__ double red[32];
  const int c = blockIdx.x, j = blockIdx.y;
  const double* U = Up + (size_t)j * h3 * R;
  const size_t plane = (size_t)Np * h3;
  __nv_bfloat16* out = BS + (size_t)j * kSlices * plane + (size_t)c * h3;
  double m = 0.0;
  if (c < R)
    for (int l = threadIdx.x; l < h3; l += blockDim.x) m = fmax(m, fabs(U[(size_t)l * R + c]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double v = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
  int e = -1000;
  if (v > 0.0) frexp(v, &e);
  for (int l = threadIdx.x; l < h3; l += blockDim.x) {
    int d[kSlices] = {0, 0, 0, 0, 0, 0};
    if (c < R && e > -1000) slice_digits(U[(size_t)l * R + c], e, d);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) out[s * plane + l] = slice_value(d[s], s);
  }
  if (threadIdx.x == 0) colexp[(size_t)j * Np + c] = e;
}

// kE: columns per epilogue warp, Np / 4 (8, 16 or 24), so that the
// epilogue's registers are sized for the group's padding
template <int kE>
__global__ void __launch_bounds__(kThreads, 1)
    k_ttm_tc(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapB, TtmArgs args) {
  TK_PDL_ENTRY();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + kStages * kStageBytes);
  uint64_t* full = bars;           // [kStages]
  uint64_t* empty = bars + 2;      // [kStages]
  uint64_t* acc_full = bars + 4;   // [2]: per accumulator set
  uint64_t* acc_empty = bars + 6;  // [2]
  uint64_t* drain = bars + 8;
  uint32_t* tmem_slot = (uint32_t*)(bars + 10);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's run of (instance, tile) pairs u = j ntiles + tile
  const int u0 = blockIdx.x * args.tiles_per_cta;
  const int u1 = min(args.Bg * args.ntiles, u0 + args.tiles_per_cta);
  const int Np = args.Np;
  const int sliceB = Np * kKB * 2;  // bytes of one B slice per stage
  const int stage_tx = kOperandBytesA + kSlices * sliceB;
  const int nkb = args.nkb;
  const int nchunks = (nkb + kChunkBlocks - 1) / kChunkBlocks;
  // two accumulator sets in TMEM when they fit: the MMAs of one round then
  // run while the epilogue drains the previous round
  // Np <= 64: six accumulators (w = 4 and 5 apart) side by side, so that one
  // MMA per A slice s covers the B slices 0 .. 5 - s (they lie one after the
  // other in shared memory: N = Np (6 - s), split at 256); Np = 96: five
  // accumulators (w = 4, 5 merged) and one MMA per slice pair
  const bool wide = 6 * Np <= 512;
  const int nacc = wide ? 6 : kAcc;
  const int acc_cols = nacc * Np;
  const int nbuf = (2 * acc_cols <= 512) ? 2 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kEpiWarps);
    }
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
      int g = 0, issued = 0;  // stage uses, over all tiles of the run
      bool ok = true;
      for (int u = u0; u < u1 && ok; ++u) {
        const int j = u / args.ntiles, row0 = (u - j * args.ntiles) * kTM;
        const int inst = args.amap[j];
        for (int k = 0; k < nkb; ++k, ++g) {
          const int st = g % kStages;
          const uint32_t use = g / kStages;
          if (g >= kStages && !tc::mbar_wait(&empty[st], (use - 1) & 1, args.err)) {
            ok = false;
            break;
          }
          unsigned char* sa = smem + st * kStageBytes;
          tc::mbar_expect_tx(&full[st], stage_tx);
          tc::tma_load_4d(sa, &tmapA, &full[st], k * kKB, row0, 0, inst);
          tc::tma_load_4d(sa + kOperandBytesA, &tmapB, &full[st], k * kKB, 0, 0, j);
          issued = g + 1;
        }
      }
      for (int q = max(0, issued - kStages); q < issued; ++q)
        tc::mbar_wait(&full[q % kStages], (q / kStages) & 1, args.err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, Np);
      bool ok = true;
      int g = 0, gc = 0;  // stage uses and accumulator rounds over the run
      for (int u = u0; u < u1 && ok; ++u) {
        int k = 0;
        for (int ch = 0; ch < nchunks && ok; ++ch, ++gc) {
          // round gc uses set gc % nbuf, drained (gc / nbuf) times before
          const int ab = gc % nbuf, ause = gc / nbuf;
          if (ause > 0 && !tc::mbar_wait(&acc_empty[ab], (ause - 1) & 1, args.err)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t tset = tmem + ab * acc_cols;
          const int kend = min(nkb, (ch + 1) * kChunkBlocks);
          uint32_t first_mask = (1u << kAcc) - 1;
          for (; k < kend; ++k, ++g) {
            const int st = g % kStages;
            if (!tc::mbar_wait(&full[st], (g / kStages) & 1, args.err)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            unsigned char* sa = smem + st * kStageBytes;
            unsigned char* sb = sa + kOperandBytesA;
            const uint64_t da0 = tc::smem_desc(sa, 512, tc::kSwizzle64B);
            const uint64_t db0 = tc::smem_desc(sb, 512, tc::kSwizzle64B);
            if (wide) {
              const int ppm = 256 / Np;  // B slices per MMA
#pragma unroll 1
              for (int kk = 0; kk < 2; ++kk) {
                // the chunk's first K step starts the accumulators: A slice 0's
                // MMAs write every w = 0 .. 5 before any other MMA adds to it
                const uint32_t acc_on = (first_mask != 0 && kk == 0) ? 0u : 1u;
#pragma unroll 1
                for (int sl = 0; sl < kSlices; ++sl) {
                  for (int t0 = 0; t0 < kSlices - sl; t0 += ppm) {
                    const int nt = min(ppm, kSlices - sl - t0);
                    const uint32_t dt = tset + (uint32_t)((sl + t0) * Np);
                    const uint64_t da = da0 + (uint64_t)(sl * (kSliceBytesA >> 4) + 2 * kk);
                    const uint64_t db = db0 + (uint64_t)(t0 * (sliceB >> 4) + 2 * kk);
                    tc::mma_bf16(dt, da, db, tc::idesc_bf16_f32(kTM, nt * Np), sl == 0 ? acc_on : 1u);
                  }
                }
              }
              first_mask = 0;
            } else {
#pragma unroll 1
              for (int pidx = 0; pidx < kPairs; ++pidx) {
                const int s = kPairS[pidx], t = kPairT[pidx];
                const int acc = (s + t < 4) ? s + t : 4;
                const uint32_t dt = tset + acc * Np;
                const uint32_t accum = ((first_mask >> acc) & 1u) ? 0u : 1u;
                first_mask &= ~(1u << acc);
                const uint64_t da = da0 + (uint64_t)(s * (kSliceBytesA >> 4));
                const uint64_t db = db0 + (uint64_t)(t * (sliceB >> 4));
                tc::mma_bf16(dt, da, db, idesc, accum);
                tc::mma_bf16(dt, da + 2, db + 2, idesc, 1u);
              }
            }
            tc::mma_commit(&empty[st]);
          }
          if (ok) tc::mma_commit(&acc_full[ab]);
        }
      }
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, args.err);
    }
  } else {
    // ---------------- epilogue: TMEM -> int64 -> FP64, per tile ----------------
    const int q = warp & 3;           // TMEM lane quadrant
    const int grp = (warp - 2) >> 2;  // column group
    const int cpg = Np / 4;           // 8, 16 or 24 columns
    const int row = q * 32 + lane;
    const uint32_t base0 = tmem + ((uint32_t)(q * 32) << 16) + grp * cpg;
    bool ok = true;
    int gc = 0;
    int jprev = -1;
    int fx[kE];  // column exponents of this warp's columns, per instance
    for (int u = u0; u < u1 && ok; ++u) {
      // this tile's scales, read before the accumulators are waited for (the
      // L2 round trips overlap the MMAs instead of following the drain)
      const int j = u / args.ntiles;
      const int grow = (u - j * args.ntiles) * kTM + row;
      const int inst = args.amap[j];
      const int e = (grow < args.M) ? args.rowexp[(size_t)inst * args.h1 + grow / args.h2] : -1000;
      if (j != jprev) {
        const int* fexp = args.colexp + (size_t)j * Np;
#pragma unroll
        for (int c = 0; c < kE; ++c) {
          const int col = grp * cpg + c;
          fx[c] = (c < cpg && col < args.R) ? fexp[col] : -1000;
        }
        jprev = j;
      }
      long long V[kE];
#pragma unroll
      for (int c = 0; c < kE; ++c) V[c] = 0;
      for (int ch = 0; ch < nchunks; ++ch, ++gc) {
        const int ab = gc % nbuf;
        if (!tc::mbar_wait(&acc_full[ab], (gc / nbuf) & 1, args.err)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t base = base0 + ab * acc_cols;
#pragma unroll
        for (int hh = 0; hh < kE / 8; ++hh) {
          if (hh * 8 < cpg) {
            uint32_t r[8];
            tc::tmem_ld8(base + hh * 8, r);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 16384.0f) * (1LL << 30);
            tc::tmem_ld8(base + Np + hh * 8, r);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 4194304.0f) * (1LL << 22);
            tc::tmem_ld8(base + 2 * Np + hh * 8, r);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 1073741824.0f) * (1LL << 14);
            tc::tmem_ld8(base + 3 * Np + hh * 8, r);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 274877906944.0f) * (1LL << 6);
            tc::tmem_ld8(base + 4 * Np + hh * 8, r);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 17592186044416.0f);
            if (wide) {
              tc::tmem_ld8(base + 5 * Np + hh * 8, r);
#pragma unroll
              for (int c = 0; c < 8; ++c)
                V[hh * 8 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * 17592186044416.0f);
            }
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[ab]);
      }
      if (!ok) break;
      if (grow < args.M) {
        double* out = args.T1 + ((size_t)j * args.M + grow) * args.R;
#pragma unroll
        for (int c = 0; c < kE; ++c) {
          const int col = grp * cpg + c;
          if (c < cpg && col < args.R) {
            const int f = fx[c];
            out[col] = (e > -1000 && f > -1000) ? tc::i64_scaled(V[c], e + f - 44) : 0.0;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

template <int kE>
void ttm_attrs() {
  TK_CUDA(cudaFuncSetAttribute(k_ttm_tc<kE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
}

CUtensorMap map4d(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* base, cuuint64_t d0, cuuint64_t d1,
                  cuuint64_t d2, cuuint64_t d3, cuuint64_t s1, cuuint64_t s2, cuuint64_t s3, cuuint32_t b1) {
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  cuuint64_t dims[4] = {d0, d1, d2, d3};
  cuuint64_t strides[3] = {s1, s2, s3};
  cuuint32_t box[4] = {kKB, b1, (cuuint32_t)kSlices, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(TK_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return map;
}

int padded_cols(int R) { return (R + 31) / 32 * 32; }

}  // namespace

size_t ttm_sliced_scratch_bytes(int h3, int R, int Bg) {
  const int Np = padded_cols(R);
  return carve_bytes<int>((size_t)Bg * Np) + carve_bytes<__nv_bfloat16>((size_t)Bg * kSlices * Np * h3) + 4096;
}

void ttm_mode3_sliced(const SliceView& sv, const int h[3], const int* amap, int Bg, int Btot, const double* Up, int R,
                      double* T1, void* scratch, int* err, cudaStream_t s) {
  const int h1 = h[0], h2 = h[1], h3 = h[2];
  const int Np = padded_cols(R);
  if (Np > kMaxNp || h3 % 8 != 0 || sv.Kp != (long long)h2 * h3 || sv.nrows != h1)
    fail(TK_EINVAL, "sliced TTM: unsupported shape");
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  int* colexp = (int*)base;
  __nv_bfloat16* BS = (__nv_bfloat16*)(base + carve_bytes<int>((size_t)Bg * Np));
  launch_pdl("k_bslice", k_bslice, dim3(Np, Bg), dim3(128), 0, s, Up, h3, R, Np, colexp, BS);
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encode_fn();
  if (!enc) fail(TK_ECUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t M = (cuuint64_t)h1 * h2;
  // A: the Gram's slices [b][s][i][h2 h3] viewed as [b][s][(i, k)][l]
  const CUtensorMap mapA = map4d(enc, sv.S, h3, M, kSlices, Btot, (cuuint64_t)h3 * 2, M * h3 * 2,
                                 M * h3 * 2 * kSlices, kTM);
  // B: [j][s][c][l]
  const CUtensorMap mapB = map4d(enc, BS, h3, Np, kSlices, Bg, (cuuint64_t)h3 * 2, (cuuint64_t)Np * h3 * 2,
                                 (cuuint64_t)Np * h3 * 2 * kSlices, Np);
  const auto kern = Np == 32 ? k_ttm_tc<8> : Np == 64 ? k_ttm_tc<16> : k_ttm_tc<24>;
  once_per_device((const void*)kern, Np == 32 ? ttm_attrs<8> : Np == 64 ? ttm_attrs<16> : ttm_attrs<24>);
  // about one run of consecutive (instance, tile) pairs per SM
  static const int sms = [] {
    int d = 0, v = 0;
    if (cudaGetDevice(&d) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
      cudaGetLastError();
      v = 152;
    }
    return std::max(v, 1);
  }();
  const int ntiles = (int)((M + kTM - 1) / kTM);
  const long long total = (long long)ntiles * Bg;
  const int tpc = (int)std::max<long long>(1, (total + sms - 1) / sms);
  const unsigned nctas = (unsigned)((total + tpc - 1) / tpc);
  TtmArgs a{(int)M, h1, h2, h3, R, Np, (h3 + kKB - 1) / kKB, ntiles, tpc, Bg, amap, sv.rowexp, colexp, T1, err};
  launch_pdl("k_ttm_tc", kern, dim3(nctas), dim3(kThreads), kSmemBytes, s, mapA, mapB, a);
}

}  // namespace tk
