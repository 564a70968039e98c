// Internal declarations shared by the translation units of libtucker_matern.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tucker_matern.h"
#include "bessel.cuh"

namespace tk {

struct Profiler;
struct MultCache;

// Error raised inside the library and turned into a status at the C-ABI.
struct Error {
  int status;
  std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
// Counts the library's kernel launches (diagnostics, tk_kernel_launches).
void count_launch();
void count_launches(unsigned long long k);  // k kernels of a replayed graph
#define TK_CUDA(call) ::tk::check_cuda((call), #call)

// Programmatic dependent launch.  A kernel of the solve's chain is launched
// with programmatic stream serialisation and starts with TK_PDL_ENTRY(): it
// waits there until the previous kernel on the stream has finished and its
// writes are visible, so its launch may be processed while the previous grid
// drains (a no-op for a kernel launched without the attribute).  Kernels of
// many CTAs do not let their dependents start early: CTAs of the next kernel
// parked on the wait cost more than the overlap gained (measured on the
// n = 256 solve).  The eigensolver chain's kernels that run on a few SMs
// (one CTA per instance and a single instance) do, with
// TK_PDL_EARLY_IF_SMALL() after TK_PDL_ENTRY(): the next kernel's launch is
// then processed while they run on otherwise idle SMs, and its CTAs still
// wait for this grid to finish before they read anything.
#define TK_PDL_ENTRY() asm volatile("griddepcontrol.wait;" ::: "memory")
#define TK_PDL_EARLY_IF_SMALL()                                  \
  do {                                                           \
    if (gridDim.x * gridDim.y * gridDim.z <= 32)                 \
      asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
  } while (0)
#define TK_LAUNCH(what) (::tk::count_launch(), ::tk::check_cuda(cudaGetLastError(), what))

// Launches kernel k (which must begin with TK_PDL_ENTRY()) on stream s with
// programmatic stream serialisation allowed; counts it like TK_LAUNCH.
template <typename... KArgs, typename... Args>
void launch_pdl(const char* what, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  check_cuda(cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...), what);
  count_launch();
}

// Runs fn once for each (key, current CUDA device) pair, thread-safe; for
// per-device settings such as a kernel's shared-memory limit.
void once_per_device(const void* key, void (*fn)());

// Device workspace owned by a context: grows, never shrinks until destroyed.
struct Workspace {
  char* base = nullptr;
  size_t bytes = 0;
  size_t used = 0;
  void reserve(size_t need, cudaStream_t s);
  void reset() { used = 0; }
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t nb = count * sizeof(T);
    if (off + nb > bytes) fail(TK_ENOMEM, "workspace carve past its reservation");
    used = off + nb;
    return reinterpret_cast<T*>(base + off);
  }
  void release();
};

// Pinned host staging for the engine's small transfers (parameters,
// descriptors, ranks), so that they are truly asynchronous; grows, never
// shrinks.  Its owner must synchronise its stream before reusing it.
struct HostPinned {
  char* p = nullptr;
  size_t bytes = 0;
  char* reserve(size_t need);
  ~HostPinned();
};

// Instantiated CUDA graphs of whole solves, one per (bucket key, batch size,
// error path).  A graph is valid only for the placement it was captured with:
// the bases of the two device workspaces and of the pinned staging, whose
// layout the capture baked into its kernels' arguments and copies.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  const void* bases[3] = {};
  unsigned long long kernels = 0;  // kernel nodes, for the launch count
  int seen = 0;                    // plain runs of this plan so far
};
struct GraphCache {
  std::map<std::vector<double>, SolveGraph> graphs;
  // per bucket plan (any batch size): whether the last batch needed no more
  // eigenpairs than the first pass computes (batches above the small-batch
  // size then run their second phase speculatively)
  std::map<std::vector<double>, bool> spec_ok;
  void release();
  ~GraphCache() { release(); }
};

// A second stream with two events, for work that overlaps the solve.
struct SideStream {
  int device = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  void ensure(int dev);
  ~SideStream();
};

// Device memory shared by the results of one batched solve; freed with the
// last of them.
struct DeviceBlock {
  int device = 0;
  void* ptr = nullptr;
  size_t bytes = 0;
  ~DeviceBlock();
};

// Bytes of a carve of `count` T after 256-byte alignment (for sizing).
template <class T>
inline size_t carve_bytes(size_t count) {
  return ((count * sizeof(T)) + 255) & ~size_t(255);
}

// Parameters of the sampled function in device-friendly form.
struct KernelDev {
  int kind;
  double sigma2;
  double p;
  double inv_ell[3];
  double sqrt2nu;
  long long tsplit;  // distinct-value table: first entry past Temme's range (0: none)
  tk_nu_consts nuc;
};

// Axis coordinates x_i = x0 + i * dx (both grid kinds).
struct AxisDev {
  int n;
  double x0, dx;
};

struct GridDev {
  AxisDev ax[3];
};

KernelDev make_kernel_dev(const tk_kernel& k);
// For the distinct-value table of the cubic isotropic grid g: the first
// entry whose Matern argument exceeds Temme's range (z > 1.5), where the
// table's warps start a new chunk so that none runs both branches.
void set_table_split(KernelDev& d, const tk_grid& g);
GridDev make_grid_dev(const tk_grid& g);
bool table_applicable(const tk_kernel& k, const tk_grid& g);

// ---- stage launchers (all enqueue on `s`, no synchronisation) ----
// (a) collocation tensor, FP64.  rowsq (n1 n2 doubles) receives the sum of
// squares of every (i1, i2) row; when normF2 is given, |F|^2 is written there.
void eval_tensor_f64(const tk_kernel& k, const tk_grid& g, double* F, double* table_scratch,
                     cudaStream_t s, double* rowsq, double* normF2);
size_t eval_rowsq_doubles(const tk_grid& g);
size_t eval_scratch_doubles(const tk_kernel& k, const tk_grid& g);
// Only the distinct-value table (when table_applicable); returns false otherwise.
bool eval_table_f64(const tk_kernel& k, const tk_grid& g, double* table, cudaStream_t s);

// Weighted octant of the folded tensor for B instances sharing grid g
// (Fh + b h1 h2 h3, h_a = ceil(n_a / 2)): Fh(i, j, l) = sqrt(w_i w_j w_l)
// F(c_1 + i, c_2 + j, c_3 + l), c_a = floor(n_a / 2), w = 1 at the centre of an
// odd axis and 2 elsewhere.  kd: device array of B kernels.  tab: every kernel
// is isotropic and the grid cubic, so the distinct-value table (B x
// table_entries(n) doubles at `table`) is used.  part: B x eval_octant_parts(g)
// doubles; normF2[b] receives |Fh_b|^2 = |F_b|^2.
size_t eval_octant_parts(const tk_grid& g);
long long table_entries(int n);
void eval_octant_f64(const KernelDev* kd, bool tab, const tk_grid& g, int B, double* Fh, double* table,
                     double* part, double* normF2, cudaStream_t s, Profiler* pf = nullptr);

// |F|^2 with compensated per-thread sums and a fixed-order final sum.
size_t norm2_scratch_doubles(size_t len);
void norm2_f64(const double* x, size_t len, double* out_dev, double* scratch, cudaStream_t s);

// (b) Gram in FP64 on the CUDA cores (split-K partials in scratch).  The batch
// form takes B tensors F + b n1 n2 n3 and writes G + b n_mode^2.
size_t gram_f64_scratch_doubles(const int n[3], int mode, int B = 1);
void gram_f64(const double* F, const int n[3], int mode, double* G, double* scratch, cudaStream_t s);
void gram_f64_batch(const double* F, const int n[3], int mode, int B, double* G, double* scratch,
                    cudaStream_t s);

// (b) Gram from exact BF16 slices on the tcgen05 tensor cores.  `err` (device
// int) is raised if a bounded wait inside the kernel ran out.  The batch form
// takes B tensors F + b n1 n2 n3 and writes G + b n_mode^2; each G is the same
// whatever the batch.
size_t gram_sliced_scratch_bytes(const int n[3], int mode, int B = 1);
void gram_sliced_bf16(const double* F, const int n[3], int mode, double* G, void* scratch, int* err,
                      cudaStream_t s);
void gram_sliced_batch(const double* F, const int n[3], int mode, int B, double* G, void* scratch, int* err,
                       cudaStream_t s, Profiler* pf = nullptr);
// Where gram_sliced_batch left the slices of its last call in `scratch`:
// S = [b][6][nrows][Kp] BF16 planes, rowexp = [b][nrows] row exponents.
struct SliceView {
  const int* rowexp;
  const void* S;
  int nrows;
  long long Kp;
};
SliceView gram_slices_view(void* scratch, const int n[3], int mode, int B);
// Autotuning of the sliced Gram's K split (process-wide): on/off, and the
// JSON cache file to read now and to write after each new choice (NULL: keep
// the current file, "" : none).  gram_tune_entries: choices held.
void gram_tune_config(bool on, const char* path);
int gram_tune_entries();
// |F|^2 partials of an instance summed by one CTA of 256 threads (strided
// Neumaier sums, then a fixed tree): out = sum of p[0 .. nparts).
struct NormParts {
  const double* part;  // [b][nparts]
  int nparts;
  double* normF2;      // [b]
};
#ifdef __CUDACC__
// One CTA of 256 threads: *out = sum of p[0 .. nparts), strided Neumaier sums
// then a fixed tree (the same bits whichever kernel runs it).
__device__ inline void norm_parts_block(const double* p, int nparts, double* out) {
  __shared__ double rs[256], rc[256];
  double sm = 0.0, c = 0.0;
  for (int r = threadIdx.x; r < nparts; r += blockDim.x) {
    const double x = p[r], t = sm + x;
    c += (fabs(sm) >= fabs(x)) ? (sm - t) + x : (x - t) + sm;
    sm = t;
  }
  rs[threadIdx.x] = sm;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double a = rs[threadIdx.x], ac = rc[threadIdx.x] + rc[threadIdx.x + w];
      const double x = rs[threadIdx.x + w], t = a + x;
      ac += (fabs(a) >= fabs(x)) ? (a - t) + x : (x - t) + a;
      rs[threadIdx.x] = t;
      rc[threadIdx.x] = ac;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = rs[0] + rc[0];
}
#endif
// The mode-1 Gram of B tensors whose slices and row exponents were already
// written where gram_slices_view(scratch, n, 0, B) points.  With norm.part
// set, the Gram's reduction kernel also sums each instance's |F|^2 partials.
void gram_sliced_prepared(const int n[3], int B, double* G, void* scratch, int* err, cudaStream_t s,
                          Profiler* pf = nullptr, NormParts norm = NormParts{nullptr, 0, nullptr});
// One-pass sampling and slicing for cubic isotropic grids with even n and
// h = n / 2 a multiple of 8: the distinct-value table, with the |F|^2
// partials of its chunks from the multiplicity of each entry (part:
// [b][table_parts(n)], summed by the Gram's reduction as
// NormParts{part, table_parts(n), normF2}), then the six BF16 slices of every
// row in one pass, eight columns a thread, the row exponent from the row's
// first table entry (its largest: every covariance here decreases with the
// radius).
long long table_parts(int n);
void eval_octant_slices8(const KernelDev* kd, const tk_grid& g, int B, double* table, int* rowexp, void* S,
                         long long Kp, double* part, const int* counts, cudaStream_t s, Profiler* pf = nullptr);
// The multiplicities of the table entries of an even n, cached in `cache`;
// synchronises s the first time for an n (not inside a stream capture).
const int* table_counts(MultCache& cache, int n, cudaStream_t s);
// Sampling fused with the mode-1 slicing for cubic isotropic grids: the
// distinct-value table, then per octant row i the values Fh(i, j, l) (never
// stored), their largest magnitude (row exponent), their BF16 slices and
// their sum of squares; normF2[b] = |F_b|^2.  rowexp: [b][h]; S: [b][6][h][Kp]
// (zero beyond h^2); part: B x h doubles.
// With normF2 == nullptr the partials are left for the Gram's reduction
// (gram_sliced_prepared with NormParts{part, h, normF2}).
void eval_octant_slices(const KernelDev* kd, const tk_grid& g, int B, double* table, int* rowexp, void* S,
                        long long Kp, double* part, double* normF2, cudaStream_t s, Profiler* pf = nullptr);
// (d) First TTM (mode 3) of Bg instances on the tensor cores from the mode-1
// Gram slices of the bucket (Fh of instance amap[j] with h = (h1, h2, h3),
// h3 % 8 == 0 and Kp == h2 h3): T1[j][(i, k)][c] = sum_l Fh[(i, k)][l]
// Up[j][l][c] for c < R (Up: [j][h3][R] FP64).  scratch: ttm_sliced_scratch_bytes.
size_t ttm_sliced_scratch_bytes(int h3, int R, int Bg);
void ttm_mode3_sliced(const SliceView& sv, const int h[3], const int* amap, int Bg, int Btot, const double* Up, int R,
                      double* T1, void* scratch, int* err, cudaStream_t s);
// unit roundoff of the Gram of each precision (for the eps-unreachable flag)
inline double gram_u_eff(int precision) {
  switch (precision) {
    case TK_FP64: return 0x1p-53;
    case TK_BF16X3: return 0x1p-16;
    case TK_TF32X3: return 0x1p-21;
    default: return 0x1p-48;
  }
}
// (b) Gram from a two-term BF16 or TF32 split and three products with FP32
// accumulation on the tensor cores (TK_BF16X3, TK_TF32X3), B instances of F
// ([b][n1 n2 n3] FP64), G: [b][n_mode][n_mode].
bool is_split3(int precision);
size_t gram_split3_scratch_bytes(const int n[3], int mode, int B, int precision);
void gram_split3_batch(const double* F, const int n[3], int mode, int B, double* G, void* scratch, int* err,
                       cudaStream_t s, Profiler* pf, int precision);

// Canonical-to-Tucker (Sec. 3.4): the reduced HOSVD of the canonical tensor
// (c, U_1, U_2, U_3) (device; U_l n_l x R row-major) and `sweeps` Tucker-ALS
// sweeps in the canonical format; returns a new result (factors, core, |A|^2,
// the last update's eigenvalues).  hist_out (host, 3 sweeps, may be NULL)
// receives |B|^2 after each mode update.  Synchronises s.
tk_result* c2t_solve(tk_ctx* ctx, int R, const double* c, const double* const U[3], const int n[3], double eps,
                     const int rmax[3], const int rfix[3], int sweeps, double* hist_out, cudaStream_t s);

// General strided batched FP64 GEMM: C[z](i,j) = sum_k A[z](i,k) B[z](k,j).
// Batch entry z = b1 batch2 + b2 has operand offsets b1 s_b + b2 s_b2 (A's b1
// replaced by amap[b1] when amap is given).  Every output is one FMA chain in
// k order (or, for few outputs, a fixed split of k over several lanes);
// fixed_order = 1 makes that choice from the per-entry shape alone, so that
// each entry's result does not depend on the batch it is part of; tiles_only
// keeps one k-order chain per output for every shape, so that an output does
// not depend on the size of its matrix either.
struct GemmDesc {
  int M, N, K, batch;
  const double* A;
  long long sAb, sAi, sAk;
  const double* B;
  long long sBb, sBk, sBj;
  double* C;
  long long sCb, sCi, sCj;
  int batch2 = 1;
  long long sAb2 = 0, sBb2 = 0, sCb2 = 0;
  const int* amap = nullptr;
  int fixed_order = 0;
  int tiles_only = 0;  // fixed order on tiles whatever the shape
};
void gemm_f64(const GemmDesc& d, cudaStream_t s);
// Second TTM of an isotropic core (F symmetric under index permutations, one
// factor for all modes), for cnt instances: T2 [pos][a][k][c] =
// sum_i V [pos][i][a] T1 [pos][i][k][c] with V h x R, T1 h x h x R; the pairs
// a <= c are formed and mirrored.  Each output is a fixed-order sum.
bool ttm2_sym_supported(int h, int R);
void ttm2_sym_batch(const double* V, const double* T1, double* T2, int h, int R, int cnt, cudaStream_t s);
// Same product, but instead of storing C accumulates sum (R - C)^2 and sum R^2
// over all entries against the reference R (same layout as C); per-block
// partials go to `partials` (2 * gridsize doubles), then a fixed-order sum
// writes out_dev[0] = |R - C|^2, out_dev[1] = |R|^2.
size_t gemm_err_partials(const GemmDesc& d);
// With table != nullptr the reference is read from the distinct-value table
// of the cubic isotropic grid with table_n points per axis (R unused).
void gemm_f64_err(const GemmDesc& d, const double* R, const double* table, int table_n, double* partials,
                  double* out_dev, cudaStream_t s);

// sum (R - W Ut^T)^2 and sum R^2 for a small inner dimension K (W: M x K,
// Ut: N x K, R: M x N); out_dev[0], out_dev[1] as gemm_f64_err.
size_t err_lowrank_partials(int M, int N);
void err_lowrank_f64(const double* W, const double* Ut, const double* R, int M, int N, int K, double* partials,
                     double* out_dev, cudaStream_t s);
// The same for B entries: W + b sW, Ut + b sU, R + amap[b] sR; partials
// [b][err_lowrank_partials(M, N)], out_dev [b][2].
void err_lowrank_batch(const double* W, long long sW, const double* Ut, long long sU, const double* R, long long sR,
                       const int* amap, int M, int N, int K, int B, double* partials, double* out_dev,
                       cudaStream_t s);

// Error during a solve on the sliced path (isotropic, octant side h): the
// octant residual against the Gram's slices sv, in float-float arithmetic, for
// the cnt instances of one rank group (padded rank R <= 32, h a multiple of 8).
// The octant tensor must be symmetric under permutations of its three indices
// (an isotropic kernel on a cubic grid, one factor for all modes): the sum runs
// over i <= j <= l with orbit weights.
// V [pos][h][R] the shared factor, Bcore [pos][R][R][R] the padded core;
// esum [pos][2] = (|Fh - Xh|^2, |Fh|^2) with |Fh|^2 from normF2[amap[pos]].
bool err_sliced_supported(int h, int R);
size_t err_sliced_scratch_bytes(int h, int R, int cnt);
// rk: the rank of bucket instance b at rk[b * rk_stride] (the sums run over
// the rank's columns of the zero-padded factor and core).
void err_sliced_batch(const SliceView& sv, const double* normF2, const double* V, const double* Bcore, int h, int R,
                      int cnt, const int* amap, const int* rk, int rk_stride, void* scratch, double* esum,
                      cudaStream_t s);

// (c) leading m eigenpairs of a symmetric PSD matrix, FP64.
size_t sym_eig_scratch_doubles(int n, int m);
void sym_eig_topm(const double* G, int n, int m, double* lam, double* V, double* trace_out,
                  double* scratch, cudaStream_t s);
// Same, for a persymmetric G (G(i,j) = G(n-1-i, n-1-j)): the even and odd
// halves are solved side by side; *safe (device int) receives how many of the
// leading pairs are certainly exact (a rank above it needs sym_eig_topm).
// Same scratch size.
void sym_eig_topm_persym(const double* G, int n, int m, double* lam, double* V, double* trace_out, int* safe,
                         double* scratch, cudaStream_t s);
// B instances with the same n and m: G [b][n][n] -> lam [b][m], V [b][n][m]
// (canonical signs unless signs = false), trace [b].  Each instance's result is the same whatever
// the batch.
// With rank (optional), the Jacobi kernel also applies the truncation rule
// to each instance's m eigenvalues and trace (as rank_rule_batch, with
// rank->out + 4 b receiving instance b's results), saving a launch.
struct RankArgs {
  const double* normF2;  // [b]
  const double* eps;     // [b]
  const int* rmax;       // [b]
  const int* rfix;       // [b]
  double u_eff;
  int n_eig, n_flag;
  int* out;              // [b][4]
};
size_t sym_eig_batch_scratch_doubles(int n, int m, int B);
// signs = false leaves the eigenvectors' signs as the solver produced them
// (for callers that fix the signs themselves, such as the factor unfolding).
// u_data: relative accuracy of G (gram_u_eff of its precision); the Jacobi
// rotations stop at that level.
void sym_eig_batch(const double* G, int n, int m, int B, double* lam, double* V, double* trace, double* scratch,
                   cudaStream_t s, Profiler* pf = nullptr, const RankArgs* rank = nullptr, bool signs = true,
                   double u_data = 0x1p-53);
// Tucker-ALS (Sec. 3.2): `sweeps` sweeps over modes 1, 2, 3 updating U[k]
// (device, n_k x r_k row-major) in place, then B (r1 r2 r3).  lam_log gets
// the r_k leading eigenvalues of each update's Gram at
// lam_log[(sweep * 3 + k) * kAlsLamStride].  Buffer sizes (doubles) in the
// order of AlsBuffers come from als_sizes.
constexpr int kAlsBuffers = 6;
constexpr int kAlsLamStride = 96;
struct AlsBuffers {
  double *T1, *Y, *W, *G, *eig_scr, *trace;
};
void als_sizes(const int n[3], const int r[3], size_t out[kAlsBuffers]);
void als_f64(const double* F, const int n[3], double* const U[3], const int r[3], int sweeps, double* B,
             double* lam_log, const AlsBuffers& w, int sm_count, cudaStream_t s);

// Multigrid Tucker (Sec. 3.2): the factors Uc[k] (device, nc_k x r_k) of a
// grid, linearly interpolated to the next finer grid of the dyadic hierarchy
// (cell-centred n_f = 2 n_c, vertex n_f - 1 = 2 (n_c - 1)) and orthonormalised,
// into Uf[k] (device, nf_k x r_k).  One launch for the three modes.
constexpr int kMgMaxRank = 96;
void mg_prolong_orth(const double* const Uc[3], const int nc[3], double* const Uf[3], const int nf[3],
                     const int r[3], int vertex, cudaStream_t s);

// rank rule for B instances: out [b * 4 + 0..2] as rank_rule, with eps [b],
// rmax [b], rfix [b]; n_eig is the order of the eigenproblems, n_flag the n
// of the precision flag.
void rank_rule_batch(const double* lam, int m, const double* trace, const double* normF2, const double* eps,
                     const int* rmax, const int* rfix, double u_eff, int n_eig, int n_flag, int B, int* out,
                     cudaStream_t s);
// rank rule on device; writes for one mode rank_out[0] = rank, [1] = flags,
// [2] = rank before the cap (m + 1 when more than the m computed pairs are needed).
void rank_rule(const double* lam, int m, const double* trace, const double* normF2, double eps,
               int rmax, int rfix, double u_eff, int n, int* rank_out, cudaStream_t s);

// ---- batched engine (engine.cu) ----
struct Profiler;
struct SolveReq {
  tk_kernel k;
  tk_grid g;
  tk_opts o;
};
// The three Grams are equal by symmetry (cubic grid, isotropic kernel, equal
// caps) and the options allow solving one of them.
bool shortcut_ok(const tk_kernel& k, const tk_grid& g, const tk_opts& o);
// The solve may run on the weighted octant (reflection symmetry).
bool fold_applicable(const tk_grid& g, const tk_opts& o);
// Requests with equal keys are solved together; every field fixes a launch
// shape or a summation order, so a request's result does not depend on the
// others in its batch.
struct BucketKey {
  int n[3];
  double b[3];
  int kind, precision, nmodes, tab, m[3], err, fz;  // fz: fused sampling and slicing allowed
  bool operator<(const BucketKey& o) const;
  bool operator==(const BucketKey& o) const;
};
BucketKey bucket_key(const SolveReq& r);
// Argument checks of a solve request (TK_OK or TK_EINVAL), no side effects.
int validate_request(const tk_kernel* k, const tk_grid* g, const tk_opts* o);
// Upper bound of the device bytes one request adds to a batch (workspaces
// and results), for admission.
size_t bucket_bytes_per_instance(const BucketKey& key);
// Solves B requests of one bucket (fold_applicable for all), enqueued on s;
// synchronises s once (small batches whose ranks phase A covers) or twice
// (ranks, then results).  outs[b] receives new results.  graphs (optional):
// where repeated solves of one plan are replayed from.
void solve_bucket(tk_ctx* ctx, Workspace& pre, Workspace& post, HostPinned& pin, SideStream& side,
                  GraphCache* graphs, Profiler* pf, const SolveReq* req, int B, tk_result** outs, cudaStream_t s);

}  // namespace tk

namespace tk {
// Per-stage device time of a context, from CUDA events recorded around each
// stage when profiling is on (tk_profile_enable).
struct Profiler {
  bool on = false;
  double ms[TK_NSTAGES] = {};
  long long calls[TK_NSTAGES] = {};
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<size_t> open;  // pending entries begun and not yet ended (stages nest)
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void begin(int stage, cudaStream_t s);
  void end(cudaStream_t s);
  void collect();  // after the stream is synchronised
  void reset();
  void release();
};
}  // namespace tk

namespace tk {
// Multiplicities of the distinct-value table of an even cubic grid (how many
// octant points share each table entry), one device array per n, kept for
// the context's life.
struct MultCache {
  std::mutex mu;
  std::map<int, int*> counts;  // n -> [table entries]
  ~MultCache();
};
}  // namespace tk

struct tk_ctx {
  int device = 0;
  std::mutex mu;
  tk::MultCache mult;  // table multiplicities (|F|^2 of the one-pass slicing)
  tk::Workspace ws;   // stages before the rank decision
  tk::Workspace ws2;  // stages after it (sized from the ranks)
  tk::HostPinned pin; // staging of the engine's small transfers
  tk::HostPinned pin_out; // staging of tk_result_copy
  tk::SideStream side; // overlapped independent sampling (with_error)
  tk::GraphCache graphs; // replayed solves
  std::string last_error;
  int sm_count = 0;
  tk::Profiler prof;
  std::mutex server_mu;
  std::shared_ptr<struct tk_server> server;  // serving loop, when started
};

struct tk_result {
  tk_ctx* ctx = nullptr;
  int n[3] = {0, 0, 0};
  int r[3] = {0, 0, 0};
  int m[3] = {0, 0, 0};
  uint32_t flags[3] = {0, 0, 0};
  double* U[3] = {nullptr, nullptr, nullptr};   // device, n_k x r_k
  double* Uh[3] = {nullptr, nullptr, nullptr};  // folded solves: device, ceil(n_k/2) x r_k octant factors
  double* core = nullptr;                       // device, r1 r2 r3
  std::vector<double> lam[3];                   // host, m_k leading eigenvalues
  double normF2 = 0.0;
  int precision = 0;
  int fold = 0;
  int has_error = 0;
  double rel_error = 0.0;  // when has_error
  std::shared_ptr<tk::DeviceBlock> mem;  // when set, owns U, Uh and core (shared by a batch)
};
