// Internal declarations shared by the translation units of libtucker_matern.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tucker_matern.h"
#include "bessel.cuh"

namespace tk {

// Error raised inside the library and turned into a status at the C-ABI.
struct Error {
  int status;
  std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
// Counts the library's kernel launches (diagnostics, tk_kernel_launches).
void count_launch();
#define TK_CUDA(call) ::tk::check_cuda((call), #call)
#define TK_LAUNCH(what) (::tk::count_launch(), ::tk::check_cuda(cudaGetLastError(), what))

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

// |F|^2 with compensated per-thread sums and a fixed-order final sum.
size_t norm2_scratch_doubles(size_t len);
void norm2_f64(const double* x, size_t len, double* out_dev, double* scratch, cudaStream_t s);

// (b) Gram in FP64 on the CUDA cores (split-K partials in scratch).
size_t gram_f64_scratch_doubles(const int n[3], int mode);
void gram_f64(const double* F, const int n[3], int mode, double* G, double* scratch, cudaStream_t s);

// (b) Gram from exact BF16 slices on the tcgen05 tensor cores.  `err` (device
// int) is raised if a bounded wait inside the kernel ran out.
size_t gram_sliced_scratch_bytes(const int n[3], int mode);
void gram_sliced_bf16(const double* F, const int n[3], int mode, double* G, void* scratch, int* err,
                      cudaStream_t s);
// Gram (mode 1) of B cubic isotropic tensors given by their distinct-value
// tables (T + b * tq, n points per axis), without writing F; G: [b][n][n].
size_t gram_sliced_table_scratch_bytes(int n, int B);
void gram_sliced_table(const double* T, long long tq, int n, int B, double* G, void* scratch, int* err,
                       cudaStream_t s);
// unit roundoff of the Gram of each precision (for the eps-unreachable flag)
inline double gram_u_eff(int precision) { return precision == TK_FP64 ? 0x1p-53 : 0x1p-48; }

// General strided batched FP64 GEMM: C[b](i,j) = sum_k A[b](i,k) B[b](k,j)
struct GemmDesc {
  int M, N, K, batch;
  const double* A;
  long long sAb, sAi, sAk;
  const double* B;
  long long sBb, sBk, sBj;
  double* C;
  long long sCb, sCi, sCj;
};
void gemm_f64(const GemmDesc& d, cudaStream_t s);
// Same product, but instead of storing C accumulates sum (R - C)^2 and sum R^2
// over all entries against the reference R (same layout as C); per-block
// partials go to `partials` (2 * gridsize doubles), then a fixed-order sum
// writes out_dev[0] = |R - C|^2, out_dev[1] = |R|^2.
size_t gemm_err_partials(const GemmDesc& d);
// With table != nullptr the reference is read from the distinct-value table
// of the cubic isotropic grid with table_n points per axis (R unused).
void gemm_f64_err(const GemmDesc& d, const double* R, const double* table, int table_n, double* partials,
                  double* out_dev, cudaStream_t s);

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
// B instances with the same n and m: G [b][n][n] -> lam [b][m], V [b][n][m],
// trace [b], safe [b * 4] (certain leading pairs per instance).
size_t sym_eig_persym_batch_scratch_doubles(int n, int m, int B);
void sym_eig_persym_batch(const double* G, int n, int m, int B, double* lam, double* V, double* trace, int* safe,
                          double* scratch, cudaStream_t s);
// rank rule for B instances: out [b * 4 + 0..2] as rank_rule, eps [b], rmax [b]
void rank_rule_batch(const double* lam, int m, const double* trace, const double* normF2, const double* eps,
                     const int* rmax, int rfix, double u_eff, int n, int B, int* out, cudaStream_t s);
// rank rule on device; writes for one mode rank_out[0] = rank, [1] = flags,
// [2] = rank before the cap (m + 1 when more than the m computed pairs are needed).
void rank_rule(const double* lam, int m, const double* trace, const double* normF2, double eps,
               int rmax, int rfix, double u_eff, int n, int* rank_out, cudaStream_t s);

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
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void begin(int stage, cudaStream_t s);
  void end(cudaStream_t s);
  void collect();  // after the stream is synchronised
  void reset();
  void release();
};
}  // namespace tk

struct tk_ctx {
  int device = 0;
  std::mutex mu;
  tk::Workspace ws;
  std::string last_error;
  int sm_count = 0;
  tk::Profiler prof;
};

struct tk_result {
  tk_ctx* ctx = nullptr;
  int n[3] = {0, 0, 0};
  int r[3] = {0, 0, 0};
  int m[3] = {0, 0, 0};
  uint32_t flags[3] = {0, 0, 0};
  double* U[3] = {nullptr, nullptr, nullptr};  // device, n_k x r_k
  double* core = nullptr;                      // device, r1 r2 r3
  std::vector<double> lam[3];                  // host, m_k leading eigenvalues
  double normF2 = 0.0;
  int precision = 0;
};
