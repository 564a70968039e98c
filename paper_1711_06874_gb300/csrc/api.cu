// C-ABI of libtucker_matern: argument checks, workspace planning, and the
// order of the stages of the HOSVD (Sec. 3.2): sample F, |F|^2, Gram per
// mode, leading eigenpairs and rank per mode, then the core by chained TTMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>

#include "tk_internal.h"

namespace tk {

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    fail(TK_ECUDA, m);
  }
}

// Growth is stream-ordered (cudaFreeAsync / cudaMallocAsync on the stream of
// the work that uses the workspace), so it never synchronises the device.
void Workspace::reserve(size_t need, cudaStream_t s) {
  used = 0;
  if (need <= bytes) return;
  if (base) {
    check_cuda(cudaFreeAsync(base, s), "cudaFreeAsync(workspace)");
    base = nullptr;
    bytes = 0;
  }
  const size_t want = std::max(need, bytes + bytes / 4);
  if (cudaMallocAsync((void**)&base, want, s) != cudaSuccess) {
    cudaGetLastError();
    base = nullptr;
    if (cudaMallocAsync((void**)&base, need, s) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      fail(TK_ENOMEM, "cannot allocate device workspace of " + std::to_string(need) + " bytes");
    }
    bytes = need;
  } else {
    bytes = want;
  }
}

void once_per_device(const void* key, void (*fn)()) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({key, dev})) return;
  fn();
  done.insert({key, dev});
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  check_cuda(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

void Profiler::begin(int stage, cudaStream_t s) {
  if (!on) return;
  Pending p{stage, get(), get()};
  check_cuda(cudaEventRecord(p.a, s), "cudaEventRecord");
  open.push_back(pending.size());
  pending.push_back(p);
}

void Profiler::end(cudaStream_t s) {
  if (!on || open.empty()) return;
  check_cuda(cudaEventRecord(pending[open.back()].b, s), "cudaEventRecord");
  open.pop_back();
}

void Profiler::collect() {
  for (auto& p : pending) {
    float ms_ = 0.f;
    if (cudaEventElapsedTime(&ms_, p.a, p.b) == cudaSuccess) {
      ms[p.stage] += ms_;
      calls[p.stage] += 1;
    } else {
      cudaGetLastError();
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  open.clear();
}

void Profiler::reset() {
  for (int i = 0; i < TK_NSTAGES; ++i) {
    ms[i] = 0.0;
    calls[i] = 0;
  }
}

void Profiler::release() {
  collect();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

void Workspace::release() {
  if (base) cudaFreeAsync(base, 0);
  base = nullptr;
  bytes = used = 0;
}

}  // namespace tk

using namespace tk;

namespace {

constexpr int kMaxN = 1024;
constexpr int kMaxRank = 88;

template <class Fn>
int guard(tk_ctx* ctx, Fn&& fn) {
  try {
    fn();
    return TK_OK;
  } catch (const Error& e) {
    if (ctx) ctx->last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->last_error = "host allocation failed";
    return TK_ENOMEM;
  } catch (...) {
    if (ctx) ctx->last_error = "unexpected exception";
    return TK_ECUDA;
  }
}

void check_kernel(const tk_kernel* k) {
  if (!k) fail(TK_EINVAL, "kernel is NULL");
  if (k->kind < TK_MATERN || k->kind > TK_MATERN_SD) fail(TK_EINVAL, "unknown kernel kind");
  for (int a = 0; a < 3; ++a)
    if (!(k->ell[a] > 0.0) || !std::isfinite(k->ell[a])) fail(TK_EINVAL, "ell must be > 0");
  if (!(k->sigma2 > 0.0) || !std::isfinite(k->sigma2)) fail(TK_EINVAL, "sigma2 must be > 0");
  if (k->kind == TK_MATERN && (!(k->nu > 0.0) || !(k->nu <= 50.0)))
    fail(TK_EINVAL, "nu must be in (0, 50]");
  if (k->kind == TK_SLATER_P && (!(k->p > 0.0) || !(k->p <= 8.0))) fail(TK_EINVAL, "p must be in (0, 8]");
  if (k->kind == TK_MATERN_SD && (!(k->nu > 0.0) || !(k->nu <= 50.0)))
    fail(TK_EINVAL, "nu must be in (0, 50]");
  if (k->kind == TK_MATERN_SD && (!(k->p > 0.0) || !std::isfinite(k->p))) fail(TK_EINVAL, "alpha (p) must be > 0");
}

void check_grid(const tk_grid* g) {
  if (!g) fail(TK_EINVAL, "grid is NULL");
  if (g->kind != TK_CELL_CENTRED && g->kind != TK_VERTEX) fail(TK_EINVAL, "unknown grid kind");
  for (int a = 0; a < 3; ++a) {
    if (g->n[a] < 2 || g->n[a] > kMaxN) fail(TK_EINVAL, "n must be in [2, 1024]");
    if (!(g->b[a] > 0.0) || !std::isfinite(g->b[a])) fail(TK_EINVAL, "b must be > 0");
  }
}

void check_opts(const tk_opts* o) {
  if (!o) fail(TK_EINVAL, "opts is NULL");
  if (!(o->eps >= 0.0) || !std::isfinite(o->eps)) fail(TK_EINVAL, "eps must be >= 0");
  for (int a = 0; a < 3; ++a) {
    if (o->rmax[a] < 1 || o->rmax[a] > kMaxRank) fail(TK_EINVAL, "rmax must be in [1, 88]");
    if (o->rfix[a] < 0 || o->rfix[a] > kMaxRank) fail(TK_EINVAL, "rfix must be in [0, 88]");
  }
  if (o->precision < TK_FP64 || o->precision > TK_TF32X3) fail(TK_EINVAL, "unknown precision");
  if (o->reflect_fold != 0 && o->reflect_fold != 1) fail(TK_EINVAL, "reflect_fold must be 0 or 1");
  if (o->with_error != 0 && o->with_error != 1) fail(TK_EINVAL, "with_error must be 0 or 1");
  if (o->fused_eval != 0 && o->fused_eval != 1) fail(TK_EINVAL, "fused_eval must be 0 or 1");
  if (o->reserved[0] != 0) fail(TK_EINVAL, "reserved fields must be zero");
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

int tk::validate_request(const tk_kernel* k, const tk_grid* g, const tk_opts* o) {
  try {
    check_kernel(k);
    check_grid(g);
    check_opts(o);
  } catch (const Error& e) {
    return e.status;
  }
  return TK_OK;
}

namespace {

void set_device(tk_ctx* ctx) { TK_CUDA(cudaSetDevice(ctx->device)); }

// Eigenpairs computed for mode a: the rank cap (or fixed rank), at most n.
// The eigensolver adds its own margin columns to the subspace.
int subspace_m(const tk_opts& o, int n, int a) {
  return std::min(std::max(o.rmax[a], o.rfix[a]), n);
}

// TTM chain of Sec. 3.1/3.2 (mode 3, then 2, then 1), FP64 GEMMs.
// U_k: n_k x r_k with leading dimension ld_k (row-major).
void ttm_core_f64(const double* F, const int n[3], const double* U1, int ld1, const double* U2,
                  int ld2, const double* U3, int ld3, const int r[3], double* T1, double* T2,
                  double* B, cudaStream_t s) {
  const int n1 = n[0], n2 = n[1], n3 = n[2], r1 = r[0], r2 = r[1], r3 = r[2];
  // T1[ij][c] = sum_l F[ij][l] U3[l][c]
  GemmDesc a{n1 * n2, r3, n3, 1, F, 0, n3, 1, U3, 0, ld3, 1, T1, 0, r3, 1};
  gemm_f64(a, s);
  // T2[i][b][c] = sum_j U2[j][b] T1[i][j][c]
  GemmDesc b{r2, r3, n2, n1, U2, 0, 1, ld2, T1, (long long)n2 * r3, r3, 1, T2, (long long)r2 * r3, r3, 1};
  gemm_f64(b, s);
  // B[a][bc] = sum_i U1[i][a] T2[i][bc]
  GemmDesc c{r1, r2 * r3, n1, 1, U1, 0, 1, ld1, T2, 0, (long long)r2 * r3, 1, B, 0, (long long)r2 * r3, 1};
  gemm_f64(c, s);
}

size_t ttm_scratch_doubles(const int n[3], const int r[3]) {
  return (size_t)n[0] * n[1] * r[2] + (size_t)n[0] * r[1] * r[2];
}

// W2 (n1 n2 x r3) = B x_1 U1 x_2 U2, the reconstruction up to the last mode.
void recon_w2(const double* B, const int r[3], const double* U1, int ld1, const double* U2, int ld2,
              const int n[3], double* W1, double* W2, cudaStream_t s) {
  const int n1 = n[0], n2 = n[1], r1 = r[0], r2 = r[1], r3 = r[2];
  // W1[i][bc] = sum_a U1[i][a] B[a][bc]
  GemmDesc a{n1, r2 * r3, r1, 1, U1, 0, ld1, 1, B, 0, (long long)r2 * r3, 1, W1, 0, (long long)r2 * r3, 1};
  gemm_f64(a, s);
  // W2[i][j][c] = sum_b U2[j][b] W1[i][b][c]
  GemmDesc b{n2, r3, r2, n1, U2, 0, ld2, 1, W1, (long long)r2 * r3, r3, 1, W2, (long long)n2 * r3, r3, 1};
  gemm_f64(b, s);
}

}  // namespace

extern "C" {

const char* tk_version(void) { return "tucker_matern 0.1 (sm_103a)"; }

const char* tk_strerror(int status) {
  switch (status) {
    case TK_OK: return "ok";
    case TK_EINVAL: return "invalid argument";
    case TK_ENOMEM: return "out of memory";
    case TK_ECUDA: return "CUDA error";
    case TK_ETIMEOUT: return "device wait timed out";
    case TK_EBUSY: return "not ready";
    case TK_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

const char* tk_last_error(const tk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

void tk_default_opts(tk_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps = 1e-6;
  for (int a = 0; a < 3; ++a) o->rmax[a] = 32;
  o->precision = TK_SLICED_BF16;
  o->isotropic_shortcut = 1;
  o->reflect_fold = 1;
  o->fused_eval = 1;
}

int tk_create(tk_ctx** out, int device) {
  if (!out) return TK_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return TK_ECUDA;
  }
  if (device < 0 || device >= count) return TK_EINVAL;
  tk_ctx* ctx = new (std::nothrow) tk_ctx();
  if (!ctx) return TK_ENOMEM;
  ctx->device = device;
  int rc = guard(ctx, [&] {
    TK_CUDA(cudaSetDevice(device));
    TK_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  });
  if (rc != TK_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return TK_OK;
}

void tk_destroy(tk_ctx* ctx) {
  if (!ctx) return;
  tk_serve_stop(ctx);  // no-op when not serving
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->graphs.release();
  ctx->prof.release();
  ctx->ws.release();
  ctx->ws2.release();
  delete ctx;
}

void tk_result_free(tk_result* res) {
  if (!res) return;
  if (res->mem) {  // a block shared with the other results of its batch
    delete res;
    return;
  }
  if (res->ctx) cudaSetDevice(res->ctx->device);
  for (int a = 0; a < 3; ++a)
    if (res->U[a]) cudaFree(res->U[a]);
  if (res->core) cudaFree(res->core);
  delete res;
}

}  // extern "C"

namespace {

// The unfolded solve on the whole tensor (reflect_fold = 0, or a fixed rank
// above the even eigenvectors): Gram per mode, persymmetric eigensolve, rank,
// core by the TTM chain.  Returns a new result.
tk_result* tucker_full(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts,
                       cudaStream_t s) {
  tk_result* res = nullptr;
  try {
    const tk_opts& o = *opts;
    const int* n = grid->n;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    const bool one = shortcut_ok(*kernel, *grid, o);
    const int nmodes = one ? 1 : 3;
    int m[3];
    for (int a = 0; a < 3; ++a) m[a] = subspace_m(o, n[a], a);
    const bool sliced = (o.precision == TK_SLICED_BF16);
    size_t gram_scr = 0, eig_scr = 0;
    for (int a = 0; a < nmodes; ++a) {
      gram_scr = std::max(gram_scr, sliced                     ? (gram_sliced_scratch_bytes(n, a) + 7) / 8
                                    : is_split3(o.precision) ? (gram_split3_scratch_bytes(n, a, 1, o.precision) + 7) / 8
                                                             : gram_f64_scratch_doubles(n, a));
      eig_scr = std::max(eig_scr, sym_eig_scratch_doubles(n[a], m[a]));
    }
    int rcap[3];
    for (int a = 0; a < 3; ++a) rcap[a] = std::max(o.rmax[a], o.rfix[a]);
    // workspace layout: one list of sizes drives both the reservation and the carves
    const size_t sz[8] = {N,
                          std::max<size_t>(1, eval_scratch_doubles(*kernel, *grid)),
                          eval_rowsq_doubles(*grid),
                          std::max<size_t>(1, gram_scr),
                          eig_scr,
                          64,
                          ttm_scratch_doubles(n, rcap),
                          0};
    size_t need = carve_bytes<int>(64);
    for (int i = 0; i < 7; ++i) need += carve_bytes<double>(sz[i]);
    for (int a = 0; a < 3; ++a)
      need += carve_bytes<double>((size_t)n[a] * n[a]) + carve_bytes<double>((size_t)n[a] * m[a]) +
              carve_bytes<double>(m[a]);
    ctx->ws.reserve(need, s);
    Workspace& ws = ctx->ws;
    double* F = ws.take<double>(sz[0]);
    double* table = ws.take<double>(sz[1]);
    double* nscr = ws.take<double>(sz[2]);
    double* gscr = ws.take<double>(sz[3]);
    double* escr = ws.take<double>(sz[4]);
    double* small = ws.take<double>(sz[5]);  // [0] |F|^2, [1..3] traces
    double* ttm = ws.take<double>(sz[6]);
    int* ranks_dev = ws.take<int>(64);  // [0..5] ranks and flags, [8] timeout flag
    TK_CUDA(cudaMemsetAsync(ranks_dev, 0, sizeof(int) * 64, s));
    double *G[3], *V[3], *lam[3];
    for (int a = 0; a < 3; ++a) {
      G[a] = ws.take<double>((size_t)n[a] * n[a]);
      V[a] = ws.take<double>((size_t)n[a] * m[a]);
      lam[a] = ws.take<double>(m[a]);
    }
    Profiler& pf = ctx->prof;
    pf.begin(TK_STAGE_EVAL, s);
    eval_tensor_f64(*kernel, *grid, F, table, s, nscr, small);  // |F|^2 to small[0]
    pf.end(s);
    // Gram, then the leading eigenpairs in two phases: first 16 pairs (enough
    // whenever the rank is below 16), then the full rank cap only for the
    // modes whose rank rule asks for more than the pairs computed.
    int mA[3];
    for (int a = 0; a < 3; ++a) mA[a] = (o.rfix[a] > 0) ? m[a] : std::min(m[a], 16);
    for (int a = 0; a < nmodes; ++a) {
      pf.begin(TK_STAGE_GRAM, s);
      if (sliced)
        gram_sliced_bf16(F, n, a, G[a], gscr, ranks_dev + 16, s);
      else if (is_split3(o.precision))
        gram_split3_batch(F, n, a, 1, G[a], gscr, ranks_dev + 16, s, nullptr, o.precision);
      else
        gram_f64(F, n, a, G[a], gscr, s);
      pf.end(s);
      pf.begin(TK_STAGE_EIG, s);
      // every G_k here is persymmetric (symmetric grid, even covariance)
      sym_eig_topm_persym(G[a], n[a], mA[a], lam[a], V[a], small + 1 + a, ranks_dev + 4 * a + 3, escr, s);
      pf.end(s);
      pf.begin(TK_STAGE_RANK, s);
      rank_rule(lam[a], mA[a], small + 1 + a, small, o.eps, o.rmax[a], o.rfix[a], gram_u_eff(o.precision),
                n[a], ranks_dev + 4 * a, s);
      pf.end(s);
    }
    int hr[20];
    double hsmall[4];
    TK_CUDA(cudaMemcpyAsync(hr, ranks_dev, sizeof(int) * 20, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    if (hr[16] != 0) fail(TK_ETIMEOUT, "a bounded wait in the tensor-core Gram ran out");
    bool again = false;
    for (int a = 0; a < nmodes; ++a) {
      // the rank needs more pairs than are certain: more than computed, or
      // beyond the pairs the split guarantees
      const int needed = o.rfix[a] > 0 ? o.rfix[a] : hr[4 * a + 2];
      if ((mA[a] < m[a] && hr[4 * a + 2] > mA[a]) || needed > hr[4 * a + 3]) {
        pf.begin(TK_STAGE_EIG, s);
        sym_eig_topm(G[a], n[a], m[a], lam[a], V[a], small + 1 + a, escr, s);
        pf.end(s);
        pf.begin(TK_STAGE_RANK, s);
        rank_rule(lam[a], m[a], small + 1 + a, small, o.eps, o.rmax[a], o.rfix[a], gram_u_eff(o.precision),
                  n[a], ranks_dev + 4 * a, s);
        pf.end(s);
        mA[a] = m[a];
        again = true;
      }
    }
    if (again) {
      TK_CUDA(cudaMemcpyAsync(hr, ranks_dev, sizeof(int) * 20, cudaMemcpyDeviceToHost, s));
    }
    TK_CUDA(cudaMemcpyAsync(hsmall, small, sizeof(double) * 1, cudaMemcpyDeviceToHost, s));
    res = new tk_result();
    res->ctx = ctx;
    res->precision = o.precision;
    for (int a = 0; a < 3; ++a) {
      res->n[a] = n[a];
      res->m[a] = mA[one ? 0 : a];
      res->lam[a].resize(res->m[a]);
    }
    for (int a = 0; a < nmodes; ++a)
      TK_CUDA(cudaMemcpyAsync(res->lam[a].data(), lam[a], sizeof(double) * mA[a], cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; ++a) {
      const int src = one ? 0 : a;
      res->r[a] = hr[4 * src];
      res->flags[a] = (uint32_t)hr[4 * src + 1];
      if (one && a > 0) res->lam[a] = res->lam[0];
    }
    res->normF2 = hsmall[0];
    const int* r = res->r;
    for (int a = 0; a < 3; ++a) {
      TK_CUDA(cudaMalloc(&res->U[a], sizeof(double) * (size_t)n[a] * r[a]));
      const int src = one ? 0 : a;
      // first r columns of V (n x m, ld m) into U (n x r, ld r)
      TK_CUDA(cudaMemcpy2DAsync(res->U[a], sizeof(double) * r[a], V[src], sizeof(double) * mA[src],
                                sizeof(double) * r[a], n[a], cudaMemcpyDeviceToDevice, s));
    }
    TK_CUDA(cudaMalloc(&res->core, sizeof(double) * (size_t)r[0] * r[1] * r[2]));
    double* T1 = ttm;
    double* T2 = ttm + (size_t)n[0] * n[1] * r[2];
    pf.begin(TK_STAGE_CORE, s);
    ttm_core_f64(F, n, res->U[0], r[0], res->U[1], r[1], res->U[2], r[2], r, T1, T2, res->core, s);
    pf.end(s);
    TK_CUDA(cudaStreamSynchronize(s));
    pf.collect();
  } catch (...) {
    if (res) tk_result_free(res);
    throw;
  }
  return res;
}

// One solve: the folded engine (a batch of one) when it applies.
tk_result* solve_one(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts,
                     cudaStream_t s) {
  if (!fold_applicable(*grid, *opts)) return tucker_full(ctx, kernel, grid, opts, s);
  SolveReq rq{*kernel, *grid, *opts};
  tk_result* res = nullptr;
  solve_bucket(ctx, ctx->ws, ctx->ws2, ctx->pin, ctx->side, &ctx->graphs, &ctx->prof, &rq, 1, &res, s);
  return res;
}

}  // namespace

extern "C" {

int tk_tucker(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts,
              tk_result** out, void* stream) {
  if (!ctx || !out) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  tk_result* res = nullptr;
  int rc = guard(ctx, [&] {
    check_kernel(kernel);
    check_grid(grid);
    check_opts(opts);
    set_device(ctx);
    res = solve_one(ctx, kernel, grid, opts, as_stream(stream));
  });
  if (rc != TK_OK) {
    if (res) tk_result_free(res);
    return rc;
  }
  *out = res;
  return TK_OK;
}

int tk_batch(tk_ctx* ctx, int count, const tk_kernel* kernels, const tk_grid* grids, const tk_opts* opts,
             tk_result** outs, void* stream) {
  if (!ctx || count < 0 || (count > 0 && (!kernels || !grids || !opts || !outs))) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  for (int i = 0; i < count; ++i) outs[i] = nullptr;
  int rc = guard(ctx, [&] {
    for (int i = 0; i < count; ++i) {
      check_kernel(kernels + i);
      check_grid(grids + i);
      check_opts(opts + i);
    }
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    std::map<BucketKey, std::vector<int>> buckets;
    for (int i = 0; i < count; ++i) {
      if (!fold_applicable(grids[i], opts[i])) {
        outs[i] = tucker_full(ctx, kernels + i, grids + i, opts + i, s);
        continue;
      }
      buckets[bucket_key(SolveReq{kernels[i], grids[i], opts[i]})].push_back(i);
    }
    for (auto& kv : buckets) {
      const std::vector<int>& idx = kv.second;
      // chunks that fit in about half of the free device memory
      size_t free_b = 0, total_b = 0;
      TK_CUDA(cudaMemGetInfo(&free_b, &total_b));
      const size_t per = bucket_bytes_per_instance(kv.first);
      const size_t fit = std::max<size_t>(1, (free_b / 2) / std::max<size_t>(per, 1));
      const int chunk = (int)std::min<size_t>(idx.size(), std::min<size_t>(fit, 4096));
      for (size_t c0 = 0; c0 < idx.size(); c0 += chunk) {
        const int cnt = (int)std::min<size_t>(chunk, idx.size() - c0);
        std::vector<SolveReq> rq(cnt);
        std::vector<tk_result*> rs(cnt, nullptr);
        for (int j = 0; j < cnt; ++j) {
          const int i = idx[c0 + j];
          rq[j] = SolveReq{kernels[i], grids[i], opts[i]};
        }
        solve_bucket(ctx, ctx->ws, ctx->ws2, ctx->pin, ctx->side, &ctx->graphs, &ctx->prof, rq.data(), cnt, rs.data(), s);
        for (int j = 0; j < cnt; ++j) outs[idx[c0 + j]] = rs[j];
      }
    }
  });
  if (rc != TK_OK) {
    for (int i = 0; i < count; ++i) {
      if (outs[i]) tk_result_free(outs[i]);
      outs[i] = nullptr;
    }
  }
  return rc;
}

int tk_ranks(const tk_result* res, int32_t r[3], uint32_t flags[3]) {
  if (!res || !r) return TK_EINVAL;
  for (int a = 0; a < 3; ++a) {
    r[a] = res->r[a];
    if (flags) flags[a] = res->flags[a];
  }
  return TK_OK;
}

int tk_factor(const tk_result* res, int mode, double* dst, int on_device, void* stream) {
  if (!res || !dst || mode < 0 || mode > 2) return TK_EINVAL;
  return guard(res->ctx, [&] {
    set_device(res->ctx);
    cudaStream_t s = as_stream(stream);
    TK_CUDA(cudaMemcpyAsync(dst, res->U[mode], sizeof(double) * (size_t)res->n[mode] * res->r[mode],
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_core(const tk_result* res, double* dst, int on_device, void* stream) {
  if (!res || !dst) return TK_EINVAL;
  return guard(res->ctx, [&] {
    set_device(res->ctx);
    cudaStream_t s = as_stream(stream);
    TK_CUDA(cudaMemcpyAsync(dst, res->core, sizeof(double) * (size_t)res->r[0] * res->r[1] * res->r[2],
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_result_copy(const tk_result* res, double* U1, double* U2, double* U3, double* core, void* stream) {
  if (!res || !res->ctx) return TK_EINVAL;
  tk_ctx* ctx = res->ctx;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    double* dst[4] = {U1, U2, U3, core};
    const double* src[4] = {res->U[0], res->U[1], res->U[2], res->core};
    size_t cnt[4];
    for (int a = 0; a < 3; ++a) cnt[a] = (size_t)res->n[a] * res->r[a];
    cnt[3] = (size_t)res->r[0] * res->r[1] * res->r[2];
    // the span of device memory holding what is asked for (one block per
    // result: one copy), each distinct source staged once
    const double* lo = nullptr;
    const double* hi = nullptr;
    for (int q = 0; q < 4; ++q) {
      if (!dst[q] || !src[q] || cnt[q] == 0) continue;
      if (!lo || src[q] < lo) lo = src[q];
      if (!hi || src[q] + cnt[q] > hi) hi = src[q] + cnt[q];
    }
    if (!lo) return;
    const size_t span = (size_t)(hi - lo);
    // one staged copy only within the result's own block of device memory
    const char* b0 = res->mem ? static_cast<const char*>(res->mem->ptr) : nullptr;
    const bool in_block = b0 && (const char*)lo >= b0 && (const char*)hi <= b0 + res->mem->bytes;
    if (!in_block || span > (size_t)64 << 20) {
      // separate allocations, or a span above 512 MB: copy each part
      for (int q = 0; q < 4; ++q)
        if (dst[q] && src[q] && cnt[q])
          TK_CUDA(cudaMemcpyAsync(dst[q], src[q], sizeof(double) * cnt[q], cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      return;
    }
    double* stage = reinterpret_cast<double*>(ctx->pin_out.reserve(sizeof(double) * span));
    TK_CUDA(cudaMemcpyAsync(stage, lo, sizeof(double) * span, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < 4; ++q)
      if (dst[q] && src[q] && cnt[q]) std::memcpy(dst[q], stage + (src[q] - lo), sizeof(double) * cnt[q]);
  });
}

int tk_eigenvalues(const tk_result* res, int mode, double* dst, int count, int* written) {
  if (!res || !dst || mode < 0 || mode > 2 || count < 0) return TK_EINVAL;
  const int k = std::min<int>(count, (int)res->lam[mode].size());
  std::memcpy(dst, res->lam[mode].data(), sizeof(double) * k);
  if (written) *written = k;
  return TK_OK;
}

int tk_result_rel_error(const tk_result* res, double* rel_error) {
  if (!res || !rel_error || !res->has_error) return TK_EINVAL;
  *rel_error = res->rel_error;
  return TK_OK;
}

int tk_norm2(const tk_result* res, double* normF2) {
  if (!res || !normF2) return TK_EINVAL;
  *normF2 = res->normF2;
  return TK_OK;
}

int tk_reconstruct(tk_ctx* ctx, const tk_result* res, double* dst, void* stream) {
  if (!ctx || !res || !dst) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    const int* n = res->n;
    const int* r = res->r;
    const size_t w1 = (size_t)n[0] * r[1] * r[2], w2 = (size_t)n[0] * n[1] * r[2];
    ctx->ws.reserve(carve_bytes<double>(w1) + carve_bytes<double>(w2), s);
    double* W1 = ctx->ws.take<double>(w1);
    double* W2 = ctx->ws.take<double>(w2);
    recon_w2(res->core, r, res->U[0], r[0], res->U[1], r[1], n, W1, W2, s);
    GemmDesc d{n[0] * n[1], n[2], r[2], 1, W2, 0, r[2], 1, res->U[2], 0, 1, r[2], dst, 0, n[2], 1};
    gemm_f64(d, s);
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_rel_error(tk_ctx* ctx, const tk_result* res, const tk_kernel* kernel, const tk_grid* grid,
                 double* out, void* stream) {
  if (!ctx || !res || !out) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    check_kernel(kernel);
    check_grid(grid);
    for (int a = 0; a < 3; ++a)
      if (grid->n[a] != res->n[a]) fail(TK_EINVAL, "grid does not match the result");
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    const int* r = res->r;
    if (res->fold) {
      // |F - X| = |Fh - Xh| on the weighted octant: Xh from the core and the
      // octant factors, Fh resampled; Xh is never stored
      int h[3];
      for (int a = 0; a < 3; ++a) h[a] = (res->n[a] + 1) / 2;
      const size_t H = (size_t)h[0] * h[1] * h[2];
      const bool tab = table_applicable(*kernel, *grid);
      const size_t Q = tab ? (size_t)table_entries(grid->n[0]) : 1;
      const size_t w1 = (size_t)h[0] * r[1] * r[2], w2 = (size_t)h[0] * h[1] * r[2];
      const size_t parts = err_lowrank_partials(h[0] * h[1], h[2]);
      const size_t np = eval_octant_parts(*grid);
      ctx->ws.reserve(carve_bytes<KernelDev>(1) + carve_bytes<double>(H) + carve_bytes<double>(Q) +
                          carve_bytes<double>(w1) + carve_bytes<double>(w2) + carve_bytes<double>(parts) +
                          carve_bytes<double>(8) + carve_bytes<double>(np) + 4096,
                      s);
      KernelDev* kd = ctx->ws.take<KernelDev>(1);
      double* Fh = ctx->ws.take<double>(H);
      double* table = ctx->ws.take<double>(Q);
      double* W1 = ctx->ws.take<double>(w1);
      double* W2 = ctx->ws.take<double>(w2);
      double* part = ctx->ws.take<double>(parts);
      double* sums = ctx->ws.take<double>(8);
      double* opart = ctx->ws.take<double>(np);
      const KernelDev kh = make_kernel_dev(*kernel);
      TK_CUDA(cudaMemcpyAsync(kd, &kh, sizeof(KernelDev), cudaMemcpyHostToDevice, s));
      ctx->prof.begin(TK_STAGE_ERROR, s);
      eval_octant_f64(kd, tab, *grid, 1, Fh, table, opart, sums + 4, s);
      recon_w2(res->core, r, res->Uh[0], r[0], res->Uh[1], r[1], h, W1, W2, s);
      // X = W2 Uh3^T (inner dimension r3), against Fh
      err_lowrank_f64(W2, res->Uh[2], Fh, h[0] * h[1], h[2], r[2], part, sums, s);
      ctx->prof.end(s);
      double hs[2];
      TK_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      ctx->prof.collect();
      *out = std::sqrt(hs[0] / hs[1]);
      return;
    }
    const int* n = res->n;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    const size_t w1 = (size_t)n[0] * r[1] * r[2], w2 = (size_t)n[0] * n[1] * r[2];
    GemmDesc d{n[0] * n[1], n[2], r[2], 1, nullptr, 0, r[2], 1, res->U[2], 0, 1, r[2], nullptr, 0, n[2], 1};
    const size_t parts = gemm_err_partials(d);
    ctx->ws.reserve(carve_bytes<double>(N) + carve_bytes<double>(eval_scratch_doubles(*kernel, *grid) + 1) +
                        carve_bytes<double>(w1) + carve_bytes<double>(w2) + carve_bytes<double>(parts) +
                        carve_bytes<double>(8) + carve_bytes<double>(eval_rowsq_doubles(*grid)),
                    s);
    double* rowsq = ctx->ws.take<double>(eval_rowsq_doubles(*grid));
    double* F = ctx->ws.take<double>(N);
    double* table = ctx->ws.take<double>(eval_scratch_doubles(*kernel, *grid) + 1);
    double* W1 = ctx->ws.take<double>(w1);
    double* W2 = ctx->ws.take<double>(w2);
    double* part = ctx->ws.take<double>(parts);
    double* sums = ctx->ws.take<double>(8);
    ctx->prof.begin(TK_STAGE_ERROR, s);
    // F is resampled: the distinct-value table feeds the error epilogue
    // directly on cubic isotropic grids, otherwise F is written out first
    const bool tab = eval_table_f64(*kernel, *grid, table, s);
    if (!tab) eval_tensor_f64(*kernel, *grid, F, table, s, rowsq, nullptr);
    recon_w2(res->core, r, res->U[0], r[0], res->U[1], r[1], n, W1, W2, s);
    d.A = W2;
    gemm_f64_err(d, tab ? nullptr : F, tab ? table : nullptr, n[0], part, sums, s);
    ctx->prof.end(s);
    double h[2];
    TK_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    ctx->prof.collect();
    *out = std::sqrt(h[0] / h[1]);
  });
}

int tk_eval(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, double* F, void* stream) {
  if (!ctx || !F) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    check_kernel(kernel);
    check_grid(grid);
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    ctx->ws.reserve(carve_bytes<double>(eval_scratch_doubles(*kernel, *grid) + 1) +
                        carve_bytes<double>(eval_rowsq_doubles(*grid)),
                    s);
    double* table = ctx->ws.take<double>(eval_scratch_doubles(*kernel, *grid) + 1);
    double* rowsq = ctx->ws.take<double>(eval_rowsq_doubles(*grid));
    eval_tensor_f64(*kernel, *grid, F, table, s, rowsq, nullptr);
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_gram(tk_ctx* ctx, const double* F, const int32_t n[3], int mode, int precision, double* G,
            void* stream) {
  if (!ctx || !F || !G || !n || mode < 0 || mode > 2) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    int nn[3] = {n[0], n[1], n[2]};
    for (int a = 0; a < 3; ++a)
      if (nn[a] < 1 || nn[a] > kMaxN) fail(TK_EINVAL, "n must be in [1, 1024]");
    if (precision < TK_FP64 || precision > TK_TF32X3) fail(TK_EINVAL, "unknown precision");
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    if (is_split3(precision)) {
      const size_t b = gram_split3_scratch_bytes(nn, mode, 1, precision);
      ctx->ws.reserve(carve_bytes<char>(b) + carve_bytes<int>(4), s);
      char* scr = ctx->ws.take<char>(b);
      int* err = ctx->ws.take<int>(4);
      TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int) * 4, s));
      gram_split3_batch(F, nn, mode, 1, G, scr, err, s, nullptr, precision);
      int h = 0;
      TK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      if (h != 0) fail(TK_ETIMEOUT, "a bounded wait in the tensor-core Gram ran out");
    } else if (precision == TK_FP64) {
      ctx->ws.reserve(carve_bytes<double>(gram_f64_scratch_doubles(nn, mode)), s);
      double* scr = ctx->ws.take<double>(gram_f64_scratch_doubles(nn, mode));
      gram_f64(F, nn, mode, G, scr, s);
      TK_CUDA(cudaStreamSynchronize(s));
    } else {
      const size_t b = gram_sliced_scratch_bytes(nn, mode);
      ctx->ws.reserve(carve_bytes<char>(b) + carve_bytes<int>(4), s);
      char* scr = ctx->ws.take<char>(b);
      int* err = ctx->ws.take<int>(4);
      TK_CUDA(cudaMemsetAsync(err, 0, sizeof(int) * 4, s));
      gram_sliced_bf16(F, nn, mode, G, scr, err, s);
      int h = 0;
      TK_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      if (h != 0) fail(TK_ETIMEOUT, "a bounded wait in the tensor-core Gram ran out");
    }
  });
}

int tk_sym_eig(tk_ctx* ctx, const double* G, int n, int m, double* lam, double* V, void* stream) {
  if (!ctx || !G || !lam || !V) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    if (n < 1 || n > kMaxN || m < 1 || m > std::min(n, 96)) fail(TK_EINVAL, "need 1 <= m <= min(n, 96)");
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    ctx->ws.reserve(carve_bytes<double>(sym_eig_scratch_doubles(n, m)), s);
    double* scr = ctx->ws.take<double>(sym_eig_scratch_doubles(n, m));
    sym_eig_topm(G, n, m, lam, V, nullptr, scr, s);
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_ttm_core(tk_ctx* ctx, const double* F, const int32_t n[3], const double* U1, const double* U2,
                const double* U3, const int32_t r[3], int precision, double* B, void* stream) {
  if (!ctx || !F || !n || !U1 || !U2 || !U3 || !r || !B) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    int nn[3] = {n[0], n[1], n[2]}, rr[3] = {r[0], r[1], r[2]};
    for (int a = 0; a < 3; ++a) {
      if (nn[a] < 1 || nn[a] > kMaxN) fail(TK_EINVAL, "n must be in [1, 1024]");
      if (rr[a] < 1 || rr[a] > nn[a]) fail(TK_EINVAL, "need 1 <= r <= n");
    }
    if (precision != TK_FP64) fail(TK_EINVAL, "only TK_FP64 is available through this entry point");
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    ctx->ws.reserve(carve_bytes<double>((size_t)nn[0] * nn[1] * rr[2]) +
                        carve_bytes<double>((size_t)nn[0] * rr[1] * rr[2]),
                    s);
    double* T1 = ctx->ws.take<double>((size_t)nn[0] * nn[1] * rr[2]);
    double* T2 = ctx->ws.take<double>((size_t)nn[0] * rr[1] * rr[2]);
    ttm_core_f64(F, nn, U1, rr[0], U2, rr[1], U3, rr[2], rr, T1, T2, B, s);
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_als(tk_ctx* ctx, const double* F, const int32_t n[3], double* U1, double* U2, double* U3, const int32_t r[3],
           int sweeps, double* B, double* core_norm2, void* stream) {
  if (!ctx || !F || !n || !U1 || !U2 || !U3 || !r || !B) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    int nn[3] = {n[0], n[1], n[2]}, rr[3] = {r[0], r[1], r[2]};
    for (int a = 0; a < 3; ++a) {
      if (nn[a] < 1 || nn[a] > kMaxN) fail(TK_EINVAL, "n must be in [1, 1024]");
      if (rr[a] < 1 || rr[a] > std::min(nn[a], kAlsLamStride)) fail(TK_EINVAL, "need 1 <= r <= min(n, 96)");
    }
    for (int a = 0; a < 3; ++a)
      if ((long long)rr[a] > (long long)rr[(a + 1) % 3] * rr[(a + 2) % 3])
        fail(TK_EINVAL, "r is not a multilinear rank (r_k > r_m r_l)");
    if (sweeps < 0 || sweeps > 64) fail(TK_EINVAL, "need 0 <= sweeps <= 64");
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    size_t sz[kAlsBuffers];
    als_sizes(nn, rr, sz);
    const size_t nlam = (size_t)std::max(sweeps, 1) * 3 * kAlsLamStride;
    size_t total = carve_bytes<double>(nlam);
    for (int i = 0; i < kAlsBuffers; ++i) total += carve_bytes<double>(std::max<size_t>(sz[i], 1));
    ctx->ws.reserve(total, s);
    double* buf[kAlsBuffers];
    for (int i = 0; i < kAlsBuffers; ++i) buf[i] = ctx->ws.take<double>(std::max<size_t>(sz[i], 1));
    double* lam_log = ctx->ws.take<double>(nlam);
    const AlsBuffers w{buf[0], buf[1], buf[2], buf[3], buf[4], buf[5]};
    double* const U[3] = {U1, U2, U3};
    als_f64(F, nn, U, rr, sweeps, B, lam_log, w, ctx->sm_count, s);
    if (core_norm2 && sweeps > 0) {
      std::vector<double> h(nlam);
      TK_CUDA(cudaMemcpyAsync(h.data(), lam_log, sizeof(double) * nlam, cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      for (int t = 0; t < 3 * sweeps; ++t) {
        const int k = t % 3;
        double acc = 0.0;  // descending eigenvalues, summed from the smallest kept one
        for (int i = rr[k] - 1; i >= 0; --i) acc += h[(size_t)t * kAlsLamStride + i];
        core_norm2[t] = acc;
      }
    }
    TK_CUDA(cudaStreamSynchronize(s));
  });
}

int tk_multigrid(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts, int levels,
                 int sweeps, tk_result** out, void* stream) {
  if (!ctx || !out) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  tk_result* coarse = nullptr;
  tk_result* res = nullptr;
  int rc = guard(ctx, [&] {
    check_kernel(kernel);
    check_grid(grid);
    check_opts(opts);
    if (levels < 0 || levels > 8) fail(TK_EINVAL, "need 0 <= levels <= 8");
    if (sweeps < 1 || sweeps > 64) fail(TK_EINVAL, "need 1 <= sweeps <= 64");
    const bool vertex = (grid->kind == TK_VERTEX);
    // g[0] is the coarsest grid, g[levels] the requested one
    std::vector<tk_grid> g((size_t)levels + 1);
    g[levels] = *grid;
    for (int lv = levels; lv > 0; --lv) {
      tk_grid c = g[lv];
      for (int a = 0; a < 3; ++a) {
        const int nf = g[lv].n[a];
        if (vertex ? (nf % 2 == 0) : (nf % 2 != 0))
          fail(TK_EINVAL, vertex ? "multigrid on a vertex grid needs odd n at every refined level"
                                 : "multigrid on a cell-centred grid needs even n at every refined level");
        c.n[a] = vertex ? (nf - 1) / 2 + 1 : nf / 2;
      }
      check_grid(&c);
      g[lv - 1] = c;
    }
    set_device(ctx);
    cudaStream_t s = as_stream(stream);
    coarse = solve_one(ctx, kernel, &g[0], opts, s);
    int r[3];
    for (int a = 0; a < 3; ++a) r[a] = coarse->r[a];
    for (int a = 0; a < 3; ++a) {
      if (r[a] > std::min(kAlsLamStride, kMgMaxRank)) fail(TK_EINVAL, "coarse rank above 96");
      if ((long long)r[a] > (long long)r[(a + 1) % 3] * r[(a + 2) % 3])
        fail(TK_EINVAL, "the coarse ranks are not a multilinear rank (r_k > r_m r_l)");
    }
    const int* nfin = grid->n;
    const size_t Nf = (size_t)nfin[0] * nfin[1] * nfin[2];
    // second workspace: F of the grid being refined (the finest is largest),
    // |F|^2, and two factor sets that alternate between grids
    size_t need = carve_bytes<double>(Nf) + carve_bytes<double>(1);
    for (int set = 0; set < 2; ++set)
      for (int a = 0; a < 3; ++a) need += carve_bytes<double>((size_t)nfin[a] * r[a]);
    ctx->ws2.reserve(need, s);
    double* F = ctx->ws2.take<double>(Nf);
    double* normF2 = ctx->ws2.take<double>(1);
    double* Uset[2][3];
    for (int set = 0; set < 2; ++set)
      for (int a = 0; a < 3; ++a) Uset[set][a] = ctx->ws2.take<double>((size_t)nfin[a] * r[a]);
    for (int a = 0; a < 3; ++a)
      TK_CUDA(cudaMemcpyAsync(Uset[0][a], coarse->U[a], sizeof(double) * (size_t)g[0].n[a] * r[a],
                              cudaMemcpyDeviceToDevice, s));
    res = new tk_result();
    res->ctx = ctx;
    res->precision = TK_FP64;
    for (int a = 0; a < 3; ++a) {
      res->n[a] = nfin[a];
      res->r[a] = r[a];
      res->m[a] = r[a];
      res->flags[a] = coarse->flags[a];
      TK_CUDA(cudaMalloc(&res->U[a], sizeof(double) * (size_t)nfin[a] * r[a]));
    }
    TK_CUDA(cudaMalloc(&res->core, sizeof(double) * (size_t)r[0] * r[1] * r[2]));
    const size_t nlam = (size_t)sweeps * 3 * kAlsLamStride;
    std::vector<double> lam_h(nlam);
    int cur = 0;
    for (int lv = 0; lv <= levels; ++lv) {
      if (lv > 0) {
        const double* const from[3] = {Uset[cur][0], Uset[cur][1], Uset[cur][2]};
        mg_prolong_orth(from, g[lv - 1].n, Uset[1 - cur], g[lv].n, r, vertex ? 1 : 0, s);
        cur = 1 - cur;
      }
      const tk_grid& gl = g[lv];
      ctx->ws.reserve(carve_bytes<double>(eval_scratch_doubles(*kernel, gl) + 1) +
                          carve_bytes<double>(eval_rowsq_doubles(gl)),
                      s);
      double* table = ctx->ws.take<double>(eval_scratch_doubles(*kernel, gl) + 1);
      double* rowsq = ctx->ws.take<double>(eval_rowsq_doubles(gl));
      eval_tensor_f64(*kernel, gl, F, table, s, rowsq, lv == levels ? normF2 : nullptr);
      size_t sz[kAlsBuffers];
      als_sizes(gl.n, r, sz);
      size_t total = carve_bytes<double>(nlam);
      for (int i = 0; i < kAlsBuffers; ++i) total += carve_bytes<double>(std::max<size_t>(sz[i], 1));
      ctx->ws.reserve(total, s);
      double* buf[kAlsBuffers];
      for (int i = 0; i < kAlsBuffers; ++i) buf[i] = ctx->ws.take<double>(std::max<size_t>(sz[i], 1));
      double* lam_log = ctx->ws.take<double>(nlam);
      const AlsBuffers w{buf[0], buf[1], buf[2], buf[3], buf[4], buf[5]};
      double* const U[3] = {Uset[cur][0], Uset[cur][1], Uset[cur][2]};
      als_f64(F, gl.n, U, r, sweeps, res->core, lam_log, w, ctx->sm_count, s);
      if (lv == levels)
        TK_CUDA(cudaMemcpyAsync(lam_h.data(), lam_log, sizeof(double) * nlam, cudaMemcpyDeviceToHost, s));
    }
    for (int a = 0; a < 3; ++a)
      TK_CUDA(cudaMemcpyAsync(res->U[a], Uset[cur][a], sizeof(double) * (size_t)nfin[a] * r[a],
                              cudaMemcpyDeviceToDevice, s));
    double nrm = 0.0;
    TK_CUDA(cudaMemcpyAsync(&nrm, normF2, sizeof(double), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    res->normF2 = nrm;
    for (int k = 0; k < 3; ++k) {
      const double* l = lam_h.data() + (size_t)((sweeps - 1) * 3 + k) * kAlsLamStride;
      res->lam[k].assign(l, l + r[k]);
    }
  });
  if (coarse) tk_result_free(coarse);
  if (rc != TK_OK) {
    if (res) tk_result_free(res);
    return rc;
  }
  *out = res;
  return TK_OK;
}

int tk_c2t(tk_ctx* ctx, int R, const double* c, const double* U1, const double* U2, const double* U3,
           const int32_t n[3], double eps, const int32_t rmax[3], const int32_t rfix[3], int sweeps,
           tk_result** out, double* core_norm2, void* stream) {
  if (!ctx || !out || !c || !U1 || !U2 || !U3 || !n) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  tk_result* res = nullptr;
  int rc = guard(ctx, [&] {
    if (R < 1 || R > 4096) fail(TK_EINVAL, "need 1 <= R <= 4096");
    int nn[3], rm[3], rf[3];
    for (int a = 0; a < 3; ++a) {
      nn[a] = n[a];
      if (nn[a] < 1 || nn[a] > kMaxN) fail(TK_EINVAL, "n must be in [1, 1024]");
      rm[a] = rmax ? rmax[a] : std::min(std::min(nn[a], R), 96);
      rf[a] = rfix ? rfix[a] : 0;
      if (rm[a] < 1 || rm[a] > 96) fail(TK_EINVAL, "need 1 <= rmax <= 96");
      if (rf[a] < 0 || rf[a] > 96) fail(TK_EINVAL, "need 0 <= rfix <= 96");
    }
    if (!(eps >= 0.0) || !std::isfinite(eps)) fail(TK_EINVAL, "eps must be >= 0");
    if (sweeps < 0 || sweeps > 64) fail(TK_EINVAL, "need 0 <= sweeps <= 64");
    set_device(ctx);
    const double* const U[3] = {U1, U2, U3};
    res = c2t_solve(ctx, R, c, U, nn, eps, rm, rf, sweeps, core_norm2, as_stream(stream));
  });
  if (rc != TK_OK) return rc;
  *out = res;
  return TK_OK;
}

int tk_tune(tk_ctx* ctx, int on, const char* cache_path, int* entries) {
  if (!ctx || (on != 0 && on != 1)) return TK_EINVAL;
  return guard(ctx, [&] {
    gram_tune_config(on != 0, cache_path);
    if (entries) *entries = gram_tune_entries();
  });
}

int tk_profile_enable(tk_ctx* ctx, int on) {
  if (!ctx) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  return guard(ctx, [&] {
    set_device(ctx);
    ctx->prof.collect();
    ctx->prof.reset();
    ctx->prof.on = (on != 0);
  });
}

int tk_profile_read(tk_ctx* ctx, double ms[TK_NSTAGES], int64_t calls[TK_NSTAGES]) {
  if (!ctx || !ms || !calls) return TK_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  for (int i = 0; i < TK_NSTAGES; ++i) {
    ms[i] = ctx->prof.ms[i];
    calls[i] = ctx->prof.calls[i];
  }
  return TK_OK;
}

uint64_t tk_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
