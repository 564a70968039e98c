// (b) Gram G = A A^T of an unfolding A = F_(k) (Sec. 3.2) on the tcgen05
// tensor cores from a two-term split of each entry and three products with
// FP32 accumulation: the BF16x3 variant (kind::f16) and the TF32x3 variant
// (kind::tf32).
//
// Each entry is rounded to FP32, x, and written as x = hi + lo + d, with hi
// the BF16 (or TF32) rounding of x and lo that of x - hi (exact in FP32).
// Then x_i x_j ~ hi_i hi_j + hi_i lo_j + lo_i hi_j: the lo lo term and d are
// dropped, which leaves about 2^-16 (BF16, 8 + 8 significant bits) or 2^-21
// (TF32, 11 + 11 bits) of each product, and the tensor core sums the three
// products over the K range of a CTA in its FP32 accumulator.  The K splits'
// FP32 partials are added in FP64.  Unlike the exact slices of the sliced
// Gram, these variants carry FP32-class error in G (about u lambda_1), so the
// eigenvectors, and the error E, are resolved only down to sqrt(u) of the
// largest singular value: they serve the comparison of precisions, and the
// rank rule flags an eps below their accuracy.
//
// Kernel layout (one CTA per 128 x 64 block of G touching its upper triangle,
// one K range and one instance):
//   warp 0     TMA producer: 2 planes x 128 rows (A) and 2 x 64 rows (B) x
//              64 bytes of K per stage (32 BF16 or 16 TF32 values), SWIZZLE_64B;
//   warp 1     TMEM owner (one FP32 accumulator of 64 columns) and the
//              single-thread tcgen05.mma issuer (3 pairs x 2 K steps a stage);
//   warps 2-5  epilogue: TMEM -> registers -> FP32 partials, one TMEM lane
//              quadrant each.
// Every mbarrier wait is bounded; on a timeout the kernel raises a flag, lets
// in-flight copies and MMAs finish (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "slices.cuh"
#include "tc_common.cuh"
#include "tk_internal.h"

namespace tk {

namespace {

constexpr int kTM = 128;                 // rows of a block of G (M)
constexpr int kTN = 64;                  // columns of a block of G (N)
constexpr int kRowBytes = 64;            // K bytes per stage row (SWIZZLE_64B)
constexpr int kPlanes = 2;               // hi, lo
constexpr int kStages = 6;
constexpr int kPlaneBytesA = kTM * kRowBytes;            // 8 KB
constexpr int kPlaneBytesB = kTN * kRowBytes;            // 4 KB
constexpr int kOperandBytesA = kPlanes * kPlaneBytesA;   // 16 KB
constexpr int kOperandBytesB = kPlanes * kPlaneBytesB;   // 8 KB
constexpr int kStageBytes = kOperandBytesA + kOperandBytesB;
constexpr int kThreads = 192;                            // 6 warps
constexpr size_t kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kTmemCols = 64;

// the three products kept: (hi, hi), (hi, lo), (lo, hi)
constexpr int kNP = 3;
__constant__ int kP3A[kNP] = {0, 0, 1};
__constant__ int kP3B[kNP] = {0, 1, 0};

template <bool kTF32>
struct Elem;
template <>
struct Elem<false> {
  using T = __nv_bfloat16;
  static constexpr int kPerRow = kRowBytes / 2;  // 32 values a stage row
};
template <>
struct Elem<true> {
  using T = float;
  static constexpr int kPerRow = kRowBytes / 4;  // 16 values a stage row
};

// Index into F (row-major n1 x n2 x n3) of entry (row, c) of the mode-k unfolding.
__device__ __forceinline__ long long unfolding_index(int mode, int n1, int n2, int n3, int row, long long c) {
  (void)n1;
  if (mode == 0) return (long long)row * n2 * n3 + c;
  if (mode == 1) {
    const long long i = c / n3, l = c - i * n3;
    return (i * n2 + row) * n3 + l;
  }
  return c * n3 + row;
}

// TF32 rounding of a finite float: round to nearest on the 13 dropped bits
// (ties away from zero), by integer operations on the bit pattern.
__device__ __forceinline__ float round_tf32(float x) {
  unsigned u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

template <bool kTF32>
__device__ __forceinline__ void split2(double v, typename Elem<kTF32>::T& hi, typename Elem<kTF32>::T& lo) {
  const float x = (float)v;
  if constexpr (kTF32) {
    const float h = round_tf32(x);
    hi = h;
    lo = round_tf32(x - h);  // x - h is exact in FP32
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = h;
    lo = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// Planes of one unfolding, K-major: P[b][plane][row][Kp] (zero past K).  32 x
// 32 tiles through shared memory keep both the read of F and the write of the
// planes coalesced for every mode.  blockIdx.z: instance.
template <bool kTF32>
__global__ void k_split2(const double* __restrict__ F, int mode, int n1, int n2, int n3, int nrows, long long K,
                         long long Kp, typename Elem<kTF32>::T* __restrict__ P, long long sF) {
  using T = typename Elem<kTF32>::T;
  __shared__ double tile[32][33];
  F += (long long)blockIdx.z * sF;
  P += (size_t)blockIdx.z * kPlanes * nrows * Kp;
  const int r0 = blockIdx.y * 32;
  const long long c0 = (long long)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
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
    if (row < nrows && c < K) v = F[unfolding_index(mode, n1, n2, n3, row, c)];
    if (mode == 2)
      tile[tx][q] = v;
    else
      tile[q][tx] = v;
  }
  __syncthreads();
  const size_t plane = (size_t)nrows * Kp;
  for (int q = ty; q < 32; q += 8) {
    const int row = r0 + q;
    const long long c = c0 + tx;
    if (row >= nrows || c >= Kp) continue;
    T hi, lo;
    split2<kTF32>(tile[q][tx], hi, lo);
    const size_t at = (size_t)row * Kp + c;
    P[at] = hi;
    P[plane + at] = lo;
  }
}

struct S3Args {
  int nrt, nct, nblocks, nsplit, kb_per_split, kb_total;
  float* partials;  // [instance][split][block][128][64]
  int* err;
};

// Block b (row-major over blocks with i 128 < (j + 1) 64) -> (i, j).
__host__ __device__ __forceinline__ void block_ij(int b, int nrt, int nct, int& bi, int& bj) {
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

__host__ __device__ __forceinline__ int blocks_upper(int nrt, int nct) {
  int c = 0;
  for (int i = 0; i < nrt; ++i) {
    const int j0 = (i * kTM) / kTN;
    c += (nct > j0) ? nct - j0 : 0;
  }
  return c;
}

__device__ __forceinline__ int block_at(int i, int j, int nct) {
  int b = 0;
  for (int r = 0; r < i; ++r) b += nct - (r * kTM) / kTN;
  return b + j - (i * kTM) / kTN;
}

// Instruction descriptor: D = FP32, A = B = BF16 (kind::f16) or TF32
// (kind::tf32), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_split3(bool tf32, int M, int N) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <bool kTF32>
__device__ __forceinline__ void mma_split3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  if constexpr (kTF32) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    tc::mma_bf16(d_tmem, adesc, bdesc, idesc, accumulate);
  }
}

template <bool kTF32>
__global__ void __launch_bounds__(kThreads, 1)
    k_gram_split3(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapB, S3Args args) {
  TK_PDL_ENTRY();
  constexpr int kKE = Elem<kTF32>::kPerRow;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + kStages * kStageBytes);
  uint64_t* full = bars;              // [kStages]
  uint64_t* empty = bars + kStages;   // [kStages]
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* drain = acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(acc_full + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int inst = blockIdx.z;
  int bi, bj;
  block_ij(blockIdx.x, args.nrt, args.nct, bi, bj);
  const int kb0 = blockIdx.y * args.kb_per_split;
  const int kb1 = min(kb0 + args.kb_per_split, args.kb_total);
  const int nkb = max(0, kb1 - kb0);
  // one row block holds every row: the B rows are rows of the A tile
  const bool b_in_a = args.nrt == 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(drain, 1);
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int k = 0; k < nkb; ++k) {
        const int st = k % kStages;
        const uint32_t use = k / kStages;
        if (k >= kStages && !tc::mbar_wait(&empty[st], (use - 1) & 1, args.err)) break;
        unsigned char* sa = smem + st * kStageBytes;
        tc::mbar_expect_tx(&full[st], b_in_a ? kOperandBytesA : kStageBytes);
        tc::tma_load_4d(sa, &tmapA, &full[st], (kb0 + k) * kKE, bi * kTM, 0, inst);
        if (!b_in_a) tc::tma_load_4d(sa + kOperandBytesA, &tmapB, &full[st], (kb0 + k) * kKE, bj * kTN, 0, inst);
        issued = k + 1;
      }
      for (int k = max(0, issued - kStages); k < issued; ++k)
        tc::mbar_wait(&full[k % kStages], (k / kStages) & 1, args.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_split3(kTF32, kTM, kTN);
      bool ok = true;
      for (int k = 0; k < nkb; ++k) {
        const int st = k % kStages;
        if (!tc::mbar_wait(&full[st], (k / kStages) & 1, args.err)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        unsigned char* sa = smem + st * kStageBytes;
        unsigned char* sb = b_in_a ? sa + bj * kTN * kRowBytes : sa + kOperandBytesA;
        const int planeB = b_in_a ? kPlaneBytesA : kPlaneBytesB;
        const uint64_t da0 = tc::smem_desc(sa, 512, tc::kSwizzle64B);
        const uint64_t db0 = tc::smem_desc(sb, 512, tc::kSwizzle64B);
#pragma unroll
        for (int p = 0; p < kNP; ++p) {
          const uint64_t da = da0 + (uint64_t)(kP3A[p] * (kPlaneBytesA >> 4));
          const uint64_t db = db0 + (uint64_t)(kP3B[p] * (planeB >> 4));
          // two MMAs of 32 bytes of K each (16 BF16 or 8 TF32 values)
          mma_split3<kTF32>(tmem, da, db, idesc, (k > 0 || p > 0) ? 1u : 0u);
          mma_split3<kTF32>(tmem, da + 2, db + 2, idesc, 1u);
        }
        tc::mma_commit(&empty[st]);
      }
      if (ok && nkb > 0) tc::mma_commit(acc_full);
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, args.err);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quadrant this warp may read
    const int row = q * 32 + lane;
    float* out = args.partials +
                 (((size_t)inst * args.nsplit + blockIdx.y) * args.nblocks + blockIdx.x) * kTM * kTN +
                 (size_t)row * kTN;
    if (nkb == 0) {
      for (int j = 0; j < kTN; ++j) out[j] = 0.0f;
    } else if (tc::mbar_wait(acc_full, 0, args.err)) {
      tc::fence_after_sync();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll
      for (int h = 0; h < kTN / 32; ++h) {
        uint32_t r[32];
        tc::tmem_ld32(base + h * 32, r);
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(out + h * 32 + j) =
              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                          __uint_as_float(r[j + 3]));
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
}

// G_b[gi][gj] = G_b[gj][gi] = sum over the K splits of the FP32 partials, in
// FP64 and split order, for gi <= gj.
__global__ void k_split3_reduce(const float* __restrict__ P, int nsplit, int nct, int nblocks, int n, int B,
                                double* __restrict__ G) {
  TK_PDL_ENTRY();
  const long long per = (long long)n * n;
  const long long total = per * B;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / per);
    const long long r = e - (long long)b * per;
    const int gi = (int)(r / n), gj = (int)(r % n);
    if (gi > gj) continue;
    const int bi = gi / kTM, bj = gj / kTN;
    const int blk = block_at(bi, bj, nct);
    const float* src = P + ((size_t)b * nsplit * nblocks + blk) * kTM * kTN + (size_t)(gi - bi * kTM) * kTN +
                       (gj - bj * kTN);
    const size_t stride = (size_t)nblocks * kTM * kTN;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += (double)src[sp * stride];
    double* Gb = G + (size_t)b * per;
    Gb[(long long)gi * n + gj] = s;
    Gb[(long long)gj * n + gi] = s;
  }
}

struct S3Plan {
  int nrows, nrt, nct, nblocks, nsplit, kb_per_split, kb_total;
  long long K, Kp;
};

S3Plan s3_plan(const int n[3], int mode, int B, bool tf32) {
  const int ke = tf32 ? Elem<true>::kPerRow : Elem<false>::kPerRow;
  S3Plan p;
  p.nrows = n[mode];
  p.K = (long long)n[0] * n[1] * n[2] / p.nrows;
  p.Kp = (p.K + ke - 1) / ke * ke;
  p.kb_total = (int)(p.Kp / ke);
  p.nrt = (p.nrows + kTM - 1) / kTM;
  p.nct = (p.nrows + kTN - 1) / kTN;
  p.nblocks = blocks_upper(p.nrt, p.nct);
  // about one wave of CTAs over 152 SMs
  int want = std::max(1, 152 / (p.nblocks * B));
  want = std::min(want, p.kb_total);
  p.kb_per_split = (p.kb_total + want - 1) / want;
  p.nsplit = (p.kb_total + p.kb_per_split - 1) / p.kb_per_split;
  return p;
}

CUtensorMap plane_map(PFN_cuTensorMapEncodeTiled_v12000 enc, void* P, long long Kp, int nrows, int B, int box_rows,
                      bool tf32) {
  const int es = tf32 ? 4 : 2;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  cuuint64_t dims[4] = {(cuuint64_t)Kp, (cuuint64_t)nrows, (cuuint64_t)kPlanes, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * es, (cuuint64_t)Kp * es * nrows, (cuuint64_t)Kp * es * nrows * kPlanes};
  cuuint32_t box[4] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)box_rows, kPlanes, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, P, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(TK_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return map;
}

template <bool kTF32>
void run_split3(const double* F, const int n[3], int mode, int B, double* G, void* scratch, int* err, cudaStream_t s,
                Profiler* pf) {
  using T = typename Elem<kTF32>::T;
  const S3Plan p = s3_plan(n, mode, B, kTF32);
  const long long sF = (long long)n[0] * n[1] * n[2];
  char* base = (char*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255);
  T* P = (T*)base;
  const size_t pbytes = ((sizeof(T) * (size_t)B * kPlanes * p.nrows * p.Kp) + 255) & ~size_t(255);
  float* part = (float*)(base + pbytes);
  {
    dim3 g((unsigned)((p.Kp + 31) / 32), (p.nrows + 31) / 32, B);
    k_split2<kTF32><<<g, 256, 0, s>>>(F, mode, n[0], n[1], n[2], p.nrows, p.K, p.Kp, P, sF);
    TK_LAUNCH("k_split2");
  }
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encode_fn();
  if (!enc) fail(TK_ECUDA, "cuTensorMapEncodeTiled is not available");
  const CUtensorMap mapA = plane_map(enc, P, p.Kp, p.nrows, B, kTM, kTF32);
  const CUtensorMap mapB = plane_map(enc, P, p.Kp, p.nrows, B, kTN, kTF32);
  once_per_device((const void*)&k_gram_split3<kTF32>, [] {
    TK_CUDA(cudaFuncSetAttribute(k_gram_split3<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
  });
  S3Args a{p.nrt, p.nct, p.nblocks, p.nsplit, p.kb_per_split, p.kb_total, part, err};
  if (pf) pf->begin(TK_STAGE_GRAM_TC, s);
  launch_pdl("k_gram_split3", k_gram_split3<kTF32>, dim3(p.nblocks, p.nsplit, B), dim3(kThreads), kSmemBytes, s,
             mapA, mapB, a);
  if (pf) pf->end(s);
  const long long total = (long long)p.nrows * p.nrows * B;
  launch_pdl("k_split3_reduce", k_split3_reduce, dim3((unsigned)std::min<long long>((total + 255) / 256, 8192)),
             dim3(256), 0, s, (const float*)part, p.nsplit, p.nct, p.nblocks, p.nrows, B, G);
}

}  // namespace

bool is_split3(int precision) { return precision == TK_BF16X3 || precision == TK_TF32X3; }

size_t gram_split3_scratch_bytes(const int n[3], int mode, int B, int precision) {
  const bool tf32 = precision == TK_TF32X3;
  const S3Plan p = s3_plan(n, mode, B, tf32);
  const size_t es = tf32 ? 4 : 2;
  size_t b = ((es * (size_t)B * kPlanes * p.nrows * p.Kp) + 255) & ~size_t(255);
  b += carve_bytes<float>((size_t)B * p.nsplit * p.nblocks * kTM * kTN);
  return b + 4096;
}

void gram_split3_batch(const double* F, const int n[3], int mode, int B, double* G, void* scratch, int* err,
                       cudaStream_t s, Profiler* pf, int precision) {
  if (precision == TK_TF32X3)
    run_split3<true>(F, n, mode, B, G, scratch, err, s, pf);
  else if (precision == TK_BF16X3)
    run_split3<false>(F, n, mode, B, G, scratch, err, s, pf);
  else
    fail(TK_EINVAL, "gram_split3: precision is not a three-product split");
}

}  // namespace tk
