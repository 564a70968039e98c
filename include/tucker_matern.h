/*
 * tucker_matern.h -- C-ABI of the GB300 (sm_103a) library that computes the
 * Tucker (HOSVD) approximation of Matern, p-Slater and Gaussian covariance
 * functions sampled on an n1 x n2 x n3 axis-parallel grid, after
 * Litvinenko, Keyes, Khoromskaia, Khoromskij, Matthies, "Tucker tensor
 * analysis of Matern functions in spatial statistics" (arXiv:1711.06874).
 *
 * Conventions for every entry point
 *  - Return value: TK_OK (0) or a positive tk_status code.  Nothing throws
 *    across this interface.  tk_last_error(ctx) gives a message for the last
 *    failure on that context.
 *  - Invalid arguments return TK_EINVAL before any work is enqueued and
 *    leave outputs untouched.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; entry points that must return host
 *    values (ranks, error norms) synchronise that stream before returning.
 *  - Arrays are row-major, FP64 unless stated.  "device" pointers are CUDA
 *    global-memory addresses on the context's device; "host" pointers are
 *    ordinary CPU memory.  The caller owns every pointer it passes; the
 *    library owns tk_ctx and tk_result and everything inside them.
 *  - A context serialises the calls made on it; use one context per host
 *    thread for concurrency.
 */
#ifndef TUCKER_MATERN_H
#define TUCKER_MATERN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TK_OK = 0,
  TK_EINVAL = 1,   /* argument out of range */
  TK_ENOMEM = 2,   /* device or host allocation failed */
  TK_ECUDA = 3,    /* a CUDA call failed (message in tk_last_error) */
  TK_ETIMEOUT = 4, /* a bounded device wait ran out; results are invalid */
  TK_EBUSY = 5,    /* serving: the ticket is not finished yet */
  TK_ENOTFOUND = 6 /* serving: unknown ticket */
} tk_status;

/* Covariance kinds.
 *  TK_MATERN   Sec. 2.2, Eq. (Matern): C = sigma2 2^(1-nu)/Gamma(nu) z^nu K_nu(z),
 *              z = sqrt(2 nu) r_A, with the anisotropic distance of Sec. 2.2,
 *              r_A^2 = sum_a x_a^2 / ell_a^2 (A = diag(1/ell_a^2)).
 *  TK_SLATER_P Sec. 3.7, Eq. (exp_p): C = sigma2 exp(-r_A^p).
 *  TK_GAUSSIAN the nu -> infinity limit of Sec. 2.2: C = sigma2 exp(-r_A^2);
 *              a rank-one tensor (Sec. 4.4).
 *  TK_MATERN_SD the 3D spectral density of the Matern covariance, Sec. 3.7,
 *              Eq. (SD_matern) with d = 3: f = sigma2 / (alpha^2 + r_A^2)^(nu + 3/2),
 *              alpha > 0 given in the field p (the paper's constant C is sigma2). */
typedef enum { TK_MATERN = 0, TK_SLATER_P = 1, TK_GAUSSIAN = 2, TK_MATERN_SD = 3 } tk_kind;

/* Grid kinds.  Coordinates of axis a, 0-based index i:
 *  TK_CELL_CENTRED x_i = -b_a + (i + 1/2) 2 b_a / n_a
 *  TK_VERTEX       x_i = -b_a + i 2 b_a / (n_a - 1)   (Sec. 3.7, Eq. (grid_points)) */
typedef enum { TK_CELL_CENTRED = 0, TK_VERTEX = 1 } tk_grid_kind;

/* Arithmetic of the Gram G_k = F_(k) F_(k)^T (Sec. 3.2) and of the core.  The
 * eigensolve and the rank decision are FP64 in every mode.
 *  TK_FP64        FP64 on the CUDA cores (the plain path).
 *  TK_SLICED_BF16 Gram as exact products of 8-bit BF16 slices on the tcgen05
 *                 tensor cores, FP32 chunk sums promoted to FP64 (FP64-class).
 *  TK_BF16X3      Gram on the tcgen05 tensor cores from a two-term BF16 split
 *                 of each (FP32-rounded) entry, x ~ hi + lo, with the three
 *                 products hi hi + hi lo + lo hi summed in FP32 (about 2^-16
 *                 of each product).  Core by the FP64 TTM chain.
 *  TK_TF32X3      the same with a two-term TF32 split (kind::tf32, about 2^-21).
 * The two split variants have FP32-class Grams: their eigenvectors, and E, are
 * resolved only to about the square root of that accuracy, and the rank rule
 * flags (TK_EPS_UNREACHABLE_AT_PRECISION) an eps below it. */
typedef enum { TK_FP64 = 0, TK_SLICED_BF16 = 1, TK_BF16X3 = 2, TK_TF32X3 = 3 } tk_precision;

/* Result flags, per mode. */
enum {
  TK_RANK_CAPPED = 1u,                 /* the eps rule wanted more than rmax */
  TK_EPS_UNREACHABLE_AT_PRECISION = 2u, /* eps^2 |F|^2 / 3 is below 10 u_eff n |F|^2 */
  TK_SOLVED_AGAIN_IN_FP64 = 4u         /* a TK_SLICED_BF16 solve with with_error = 1 whose E came
                                          out above eps (ranks from the eps rule, none capped) was
                                          solved again with the FP64 Gram: this is that result */
};

typedef struct {
  int32_t kind;     /* tk_kind */
  double nu;        /* Matern smoothness, > 0 */
  double ell[3];    /* per-axis length scale, > 0 */
  double sigma2;    /* variance, > 0 */
  double p;         /* p-Slater exponent, or alpha of TK_MATERN_SD; > 0 */
} tk_kernel;

typedef struct {
  int32_t n[3];     /* grid points per axis, 2 <= n <= 1024 */
  double b[3];      /* half-width of the box [-b, b], > 0 */
  int32_t kind;     /* tk_grid_kind */
} tk_grid;

typedef struct {
  double eps;       /* relative Frobenius tolerance, >= 0 (Task 1, Sec. 2.1) */
  int32_t rmax[3];  /* rank caps, 1 <= rmax <= 88 */
  int32_t rfix[3];  /* > 0: use this rank for the mode instead of the eps rule */
  int32_t precision;          /* tk_precision */
  int32_t isotropic_shortcut; /* 1: when the three Grams are equal by symmetry
                                 (equal n, b, ell), form and solve one of them */
  int32_t reflect_fold;       /* 1: solve on the weighted octant.  The covariance
                                 depends on each x_a only through x_a^2 and the
                                 grid is symmetric about 0, so F is unchanged by
                                 reversing an axis; the odd eigenvectors of each
                                 G_k then have eigenvalue 0 and the factors, core
                                 and eigenvalues follow from the octant tensor
                                 sqrt(w_i w_j w_l) F (w = grid points an octant
                                 index stands for: 1 at the centre of an odd axis,
                                 else 2).  Skipped when rfix_k > ceil(n_k / 2). */
  int32_t with_error;         /* 1 (folded solves): also compute E = |F - X|_F / |F|_F
                                 of Eq. (FNorm) as tk_rel_error does, from a second,
                                 independent sampling of F that runs on a side
                                 stream while the eigenpairs are computed; read it
                                 with tk_result_rel_error */
  int32_t fused_eval;         /* 1 (tk_default_opts): on the sliced path of a cubic
                                 isotropic grid, sample F and cut its BF16 slices
                                 in one kernel, so the octant tensor is never
                                 stored; 0: sample the FP64 octant tensor into
                                 device memory first, then slice it (the
                                 materialised path, kept for comparison) */
  int32_t reserved[1];        /* must be zero */
} tk_opts;

typedef struct tk_ctx tk_ctx;
typedef struct tk_result tk_result;

const char* tk_strerror(int status);
const char* tk_last_error(const tk_ctx* ctx);
/* Version string of the library build. */
const char* tk_version(void);

/* Creates a context on CUDA device `device` (TK_EINVAL if out of range). */
int tk_create(tk_ctx** ctx, int device);
/* Frees the context and its workspace; results created on it must be freed first. */
void tk_destroy(tk_ctx* ctx);
/* Default options: eps 1e-6, rmax 32, rfix 0, TK_SLICED_BF16, shortcut, fold
 * and fused_eval on. */
void tk_default_opts(tk_opts* opts);

/* ---------------------------------------------------------------------------
 * Whole solve: Task 1 of Sec. 2.1 by the HOSVD of Sec. 3.2.
 *   (a) sample C on the grid (collocation tensor, Sec. 3.7),
 *   (b) form G_k = F_(k) F_(k)^T for the three unfoldings (Fig. Unfolding),
 *   (c) take the leading eigenvectors of each G_k as the factor U_k, the rank
 *       r_k being the smallest r whose discarded eigenvalue sum is
 *       <= eps^2 |F|^2 / 3 (capped at rmax), sign fixed so that the entry of
 *       largest magnitude among the first ceil(n_k/2) is positive,
 *   (d) core B = F x_1 U_1^T x_2 U_2^T x_3 U_3^T (Sec. 3.1, 3.2), mode 3 first.
 * On TK_OK *out owns device copies of U_k (n_k x r_k) and B (r1 x r2 x r3).
 * Synchronises `stream` once to read the three ranks.
 * ------------------------------------------------------------------------- */
int tk_tucker(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts,
              tk_result** out, void* stream);

/* Ranks and flags of a result (host arrays of 3): the Tucker rank
 * (r1, r2, r3) of Sec. 3.1. */
int tk_ranks(const tk_result* res, int32_t r[3], uint32_t flags[3]);
/* Factor U_mode of the Tucker format (Sec. 3.1: the orthonormal side matrix
 * V^(l) of mode l; Sec. 3.2: the leading left singular vectors of the
 * unfolding), n_mode x r_mode, row-major, orthonormal columns, into dst.
 * on_device: 1 = dst is device memory, 0 = host memory.  TK_EINVAL for a
 * mode outside 0..2. */
int tk_factor(const tk_result* res, int mode, double* dst, int on_device, void* stream);
/* Core B of the Tucker format (Sec. 3.1, the core tensor beta of the
 * decomposition; Sec. 3.2, B = F x_1 U_1^T x_2 U_2^T x_3 U_3^T), r1 x r2 x r3
 * row-major, into dst (on_device as tk_factor). */
int tk_core(const tk_result* res, double* dst, int on_device, void* stream);
/* The whole decomposition of Sec. 3.2 (U_1, U_2, U_3 and B, layouts as
 * tk_factor and tk_core) into host memory with one device-to-host copy and
 * one synchronisation of `stream`: the result's factors and core are staged
 * together in pinned memory owned by the context, then copied out.  Any of
 * the four destinations may be NULL (not copied).  Thread-safe with respect
 * to other calls on the same context. */
int tk_result_copy(const tk_result* res, double* U1, double* U2, double* U3, double* core, void* stream);
/* Leading eigenvalues of G_mode (descending) computed by the solve; writes
 * min(count, available) values to the host array dst and returns that number
 * through *written. */
int tk_eigenvalues(const tk_result* res, int mode, double* dst, int count, int* written);
/* |F|^2 of the sampled tensor (compensated FP64 sum), host scalar. */
int tk_norm2(const tk_result* res, double* normF2);
/* E computed during the solve (opts.with_error = 1); TK_EINVAL otherwise. */
int tk_result_rel_error(const tk_result* res, double* rel_error);

/* The Tucker tensor of Sec. 3.1, X = B x_1 U_1 x_2 U_2 x_3 U_3 (the
 * rank-(r1, r2, r3) approximation whose error Eq. (FNorm) measures), into dst
 * (device, n1 n2 n3 FP64, row-major, caller-owned). */
int tk_reconstruct(tk_ctx* ctx, const tk_result* res, double* dst, void* stream);
/* Eq. (FNorm): |F - X|_F / |F|_F by direct subtraction with compensated FP64
 * sums, where F is resampled from (kernel, grid) and X is never stored.
 * Writes the host scalar *out; synchronises `stream`. */
int tk_rel_error(tk_ctx* ctx, const tk_result* res, const tk_kernel* kernel, const tk_grid* grid,
                 double* out, void* stream);
void tk_result_free(tk_result* res);

/* ---------------------------------------------------------------------------
 * Batched solve: `count` independent instances of tk_tucker (the parameter
 * sweeps behind the likelihood of Sec. 2.3, Eq. (like)); instance i uses
 * kernels[i], grids[i], opts[i] (host arrays).  Instances that share a grid,
 * precision, rank caps and isotropy are solved together, every stage one
 * launch over all of them, in chunks that fit the free device memory; each
 * result is bitwise the one that instance gets in any other batch, alone
 * included.  On TK_OK outs[i] (host array of count) receives a result for
 * every i, each freed with tk_result_free; on failure every outs[i] is NULL.
 * Synchronises `stream`.
 * ------------------------------------------------------------------------- */
int tk_batch(tk_ctx* ctx, int count, const tk_kernel* kernels, const tk_grid* grids, const tk_opts* opts,
             tk_result** outs, void* stream);

/* ---------------------------------------------------------------------------
 * Serving (no counterpart in the paper): a request loop with continuous
 * batching on the context's device.  Worker threads, each with its own CUDA
 * stream, take the oldest queued request together with every queued request
 * of the same shape (grid, precision, rank caps; any kernel and eps) that the
 * memory budget admits, and solve them as one tk_batch-style batch; requests
 * arriving meanwhile form the next batches, so work from several batches
 * overlaps on the device.  Results (factors, cores) stay in device memory
 * until taken.  A request's result is bitwise the one tk_tucker returns for it
 * alone.  Requests need reflect_fold = 1 and rfix_k <= ceil(n_k / 2).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t workers;      /* concurrent batches (streams), 1..8; default 2 */
  int32_t max_batch;    /* most requests per batch, 1..4096; default 256 */
  double mem_fraction;  /* share of the device memory free at start (and at
                           each admission) that batches may plan for,
                           (0, 0.95]; default 0.8 */
  int32_t reserved[4];  /* must be zero */
} tk_serve_opts;

typedef struct {
  uint64_t submitted, completed, failed;  /* requests */
  uint64_t batches, max_batch_seen;       /* batches launched, largest one */
  uint64_t bytes_budget, bytes_peak;      /* admission budget, largest planned in-flight bytes */
  uint64_t queued, in_flight_batches;     /* now */
} tk_serve_stats;

void tk_default_serve_opts(tk_serve_opts* opts);
/* Starts the loop (TK_EINVAL if already serving or opts out of range). */
int tk_serve_start(tk_ctx* ctx, const tk_serve_opts* opts);
/* Finishes every queued request, stops the workers and frees the results
 * not taken (TK_EINVAL if not serving).  tk_destroy calls it. */
int tk_serve_stop(tk_ctx* ctx);
/* Queues one solve (host structs, copied); *ticket identifies it.  Returns
 * at once; TK_EINVAL for invalid arguments or when not serving. */
int tk_submit(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts, uint64_t* ticket);
/* Takes the result of a ticket, waiting up to wait_s seconds (0: no wait).
 * TK_EBUSY: not finished yet; TK_ENOTFOUND: unknown or already taken ticket.
 * Otherwise the ticket is consumed: TK_OK with *out the result (free it with
 * tk_result_free) and *latency_s (may be NULL) the seconds from tk_submit to
 * the end of its batch; or the status of a failed solve with *out NULL. */
int tk_poll(tk_ctx* ctx, uint64_t ticket, tk_result** out, double* latency_s, double wait_s);
int tk_serve_read_stats(tk_ctx* ctx, tk_serve_stats* out);

/* ---------------------------------------------------------------------------
 * Stage entry points (one step of the path each, device buffers in and out).
 * ------------------------------------------------------------------------- */
/* Collocation tensor F (device, n1 n2 n3 FP64) of Sec. 3.7. */
int tk_eval(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, double* F, void* stream);
/* Gram G = F_(mode) F_(mode)^T (device, n_mode x n_mode FP64) of the device
 * tensor F (n[0] n[1] n[2] FP64), in the arithmetic `precision`. */
int tk_gram(tk_ctx* ctx, const double* F, const int32_t n[3], int mode, int precision, double* G,
            void* stream);
/* Leading m eigenpairs of the symmetric PSD device matrix G (n x n):
 * lam (device, m, descending) and V (device, n x m, orthonormal columns,
 * canonical signs).  1 <= m <= min(n, 96). */
int tk_sym_eig(tk_ctx* ctx, const double* G, int n, int m, double* lam, double* V, void* stream);
/* Core B (device, r1 r2 r3) = F x_1 U1^T x_2 U2^T x_3 U3^T for the device
 * tensor F (n[0] n[1] n[2]) and device factors U_k (n_k x r_k). */
int tk_ttm_core(tk_ctx* ctx, const double* F, const int32_t n[3], const double* U1,
                const double* U2, const double* U3, const int32_t r[3], int precision, double* B,
                void* stream);

/* Tucker-ALS (Sec. 3.2): `sweeps` alternating sweeps refining the orthonormal
 * factors U_k (device, n_k x r_k row-major, updated in place; the HOSVD's
 * factors are the usual start) of the device tensor F (n[0] n[1] n[2] FP64,
 * row-major, last index fastest).  A sweep visits modes 1, 2, 3 in order;
 * mode k forms the single-hole tensor Y_k = F x_{m != k} U_m^T (the other
 * modes mapped into their current subspaces) and replaces U_k by the r_k
 * leading left singular vectors of Y_k's mode-k unfolding, computed in FP64
 * as the leading eigenvectors of that unfolding's Gram (canonical signs as
 * tk_sym_eig's).  B (device, r1 r2 r3) = F x_1 U1^T x_2 U2^T x_3 U3^T with the
 * final factors (sweeps = 0: the core of the given factors).
 * core_norm2 (host, 3 * sweeps doubles, may be NULL) receives the sum of the
 * r_k leading eigenvalues after each mode update, i.e. |B|^2 for the factors
 * of that moment; in exact arithmetic it never decreases.
 * Needs 1 <= n_k <= 1024, 1 <= r_k <= min(n_k, 96), r_k <= r_m r_l for the
 * other two modes (a multilinear rank), 0 <= sweeps <= 64; TK_EINVAL
 * otherwise.  The covariance tensors of this library have fast-decaying
 * unfolding spectra, which the subspace eigensolver relies on for n_k > 32.
 * Synchronous with respect to `stream`. */
int tk_als(tk_ctx* ctx, const double* F, const int32_t n[3], double* U1, double* U2, double* U3,
           const int32_t r[3], int sweeps, double* B, double* core_norm2, void* stream);

/* Multigrid Tucker (Sec. 3.2): the HOSVD (as tk_tucker, with `opts`) only on
 * the coarsest of levels + 1 dyadically refined grids, the finest being
 * `grid`; each coarser grid has half the cells per axis over the same box
 * (cell-centred n -> n / 2, vertex n -> (n - 1) / 2 + 1).  On every grid,
 * coarsest first, the current factors start `sweeps` Tucker-ALS sweeps on
 * that grid's collocation tensor (as tk_als); between grids each factor
 * column is carried to the finer grid by linear interpolation between the
 * two coarse points around each fine point (continued linearly past the
 * outermost ones) and the columns are orthonormalised.  The ranks and flags
 * are the coarse HOSVD's.
 * On TK_OK *out owns device copies of the finest grid's U_k (n_k x r_k) and
 * B (r1 x r2 x r3), read as any result (tk_factor, tk_core, tk_result_copy,
 * tk_reconstruct, tk_rel_error); tk_norm2 gives |F|^2 of the finest tensor
 * and tk_eigenvalues the r_k eigenvalues of mode k's last update.
 * Needs 0 <= levels <= 8 and 1 <= sweeps <= 64, every level's grid valid
 * (n >= 2; cell-centred: even n at every grid but the coarsest; vertex: odd
 * n likewise) and the coarse ranks a multilinear rank (r_k <= r_m r_l);
 * TK_EINVAL otherwise.  Holds one FP64 tensor of the finest grid in the
 * context's workspace.  Synchronous with respect to `stream`. */
int tk_multigrid(tk_ctx* ctx, const tk_kernel* kernel, const tk_grid* grid, const tk_opts* opts, int levels,
                 int sweeps, tk_result** out, void* stream);

/* Canonical-to-Tucker (Sec. 3.4): the Tucker approximation of a tensor given
 * in the canonical format of Eq. (Can_Contr),
 *   A(i1, i2, i3) = sum_{k<R} c_k U1[i1][k] U2[i2][k] U3[i3][k],
 * without forming or unfolding A.  c (device, R) are the weights and U_l
 * (device, n_l x R row-major) the side matrices (unit columns are the usual
 * normalisation; the rule below holds for any).  The initial factors come
 * from the reduced HOSVD: Z_l spans the r_l leading left singular vectors of
 * U_l alone (computed as the leading eigenvectors of U_l U_l^T in FP64), r_l
 * being the smallest r whose discarded singular values satisfy
 * (sum_{k>=r} s_k^2)^(1/2) <= eps |A| / (3 |c|) (so that the RHOSVD bound
 * |A - A_r| <= |c| sum_l (sum_{k>=r_l} s_{l,k}^2)^(1/2) gives E <= eps), capped
 * at rmax_l (TK_RANK_CAPPED) and replaced by rfix_l where rfix_l > 0.  A
 * discarded sum_k s_k^2 at or below n_l u |U_l|_F^2 (u = 2^-53, the rounding
 * level of the FP64 Gram's eigenvalues) counts as zero, and a tolerance below
 * that level sets TK_EPS_UNREACHABLE_AT_PRECISION.  Then
 * `sweeps` Tucker-ALS sweeps (modes 1, 2, 3 in order), each mode's single-hole
 * unfolding U_l diag(c) (W_m (.) W_q)^T formed from the side matrices
 * (W_j = Z_j^T U_j, (.) the Khatri-Rao product); Z_l becomes its r_l leading
 * left singular vectors (eigenvectors of its FP64 Gram, signs as tk_tucker's).
 * The core B = sum_k c_k W1[:, k] o W2[:, k] o W3[:, k].
 * rmax, rfix: host arrays of 3 or NULL (rmax: min(n_l, R, 96); rfix: 0),
 * 1 <= rmax <= 96, 0 <= rfix <= 96.  Needs 1 <= R <= 4096, 1 <= n_l <= 1024,
 * eps >= 0, 0 <= sweeps <= 64 and the ranks a multilinear rank (r_l <= r_m r_q);
 * TK_EINVAL otherwise.  On TK_OK *out owns device copies of the Z_l (n_l x r_l)
 * and B (r1 x r2 x r3), read as any result; tk_norm2 gives |A|^2 (from the
 * side matrices' Grams) and tk_eigenvalues the r_l squared singular values of
 * mode l's last update.  core_norm2 (host, 3 sweeps doubles, may be NULL)
 * receives |B|^2 after each mode update.  tk_rel_error does not apply (A is
 * not a sampled covariance).  Synchronous with respect to `stream`. */
int tk_c2t(tk_ctx* ctx, int R, const double* c, const double* U1, const double* U2, const double* U3,
           const int32_t n[3], double eps, const int32_t rmax[3], const int32_t rfix[3], int sweeps,
           tk_result** out, double* core_norm2, void* stream);

/* Allocation-free variant of tk_gram with precision TK_FP64 (no counterpart
 * in the paper).  Some callers cannot allocate device memory: code embedded in
 * a host application whose own allocator has reserved the GPU's memory,
 * real-time loops that must not pay cudaMalloc's latency or its implicit
 * synchronisation, and plugins that are only handed pointers.  This entry
 * point takes no context, performs no cudaMalloc, cudaFree or other
 * allocation, and keeps its split-K partial sums in a fixed 8 MiB device
 * array that every GPU loading this library holds until the process exits;
 * n[a] must lie in [1, 1024] (TK_EINVAL otherwise), which always fits.
 * F (device, n[0] n[1] n[2] FP64) and G (device, n_mode x n_mode FP64) are the
 * caller's; the result equals tk_gram's up to rounding: when tk_gram's K
 * split would need more partial sums than the array holds, fewer and longer
 * splits are taken, which changes the summation order.  Runs on the current
 * CUDA device and only enqueues on `stream` (no synchronisation).  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  Calls share the array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU race. */
int tk_gram_noalloc(const double* F, const int32_t n[3], int mode, double* G, void* stream);

/* Autotuning (no counterpart in the paper) of the K split of the sliced
 * tensor-core Gram.  Its result does not depend on the split (exact integer
 * chunk sums), so the split is chosen for speed alone: with on = 1, the first
 * Gram of each (SM count, rows, K, instances rounded up to a power of two)
 * shape, outside stream capture,
 * also times 2, 4 and 8 times as many 256-deep chunks per CTA as the default
 * plan (which aims at one wave of CTAs) with CUDA events on the solve's
 * stream, which it synchronises, and keeps the fastest for every later call.
 * The choices are process-wide.  cache_path (may be NULL: keep the current
 * file and choices; "": none, and forget the choices) names a JSON file of
 * {"<shape key>": chunks per CTA} whose choices replace the ones held now and
 * which is rewritten after every new choice.  *entries (may be NULL) receives
 * the number of choices held.  on = 0 stops tuning and uses the default plan. */
int tk_tune(tk_ctx* ctx, int on, const char* cache_path, int* entries);

/* ---------------------------------------------------------------------------
 * Diagnostics (no counterpart in the paper): per-stage device time and the
 * number of kernels the library launched.
 * ------------------------------------------------------------------------- */
typedef enum {
  TK_STAGE_EVAL = 0,  /* sampling F (table + gather, or per point) */
  TK_STAGE_NORM = 1,  /* |F|^2 when not read off the Gram trace (tk_tucker reads the trace) */
  TK_STAGE_GRAM = 2,  /* Gram matrices, all modes */
  TK_STAGE_EIG = 3,   /* eigenpairs, all modes */
  TK_STAGE_RANK = 4,  /* rank rule and factor extraction */
  TK_STAGE_CORE = 5,  /* TTM chain */
  TK_STAGE_ERROR = 6, /* tk_rel_error */
  /* single kernels inside the stages above (their time is also in the stage) */
  TK_STAGE_TABLE = 7,   /* K_nu distinct-value table */
  TK_STAGE_GRAM_TC = 8, /* tensor-core Gram kernel (slices excluded) */
  TK_STAGE_QR = 9,      /* FP64 Householder QR of the eigensolver */
  TK_STAGE_JACOBI = 10, /* Jacobi of the Rayleigh-Ritz matrix */
  TK_STAGE_START = 11,  /* FP32 start block of the eigensolver (G Omega, its QR, Q0) */
  TK_STAGE_EIG_GEMM = 12, /* the eigensolver's FP64 products (G Q0, G Q, Q^T G Q, Q V_H) */
  TK_NSTAGES = 13
} tk_stage;
/* on = 1 starts recording CUDA events around every stage of later calls on
 * this context and zeroes the totals; on = 0 stops. */
int tk_profile_enable(tk_ctx* ctx, int on);
/* Accumulated device milliseconds and call counts per stage (host arrays of
 * TK_NSTAGES), for the calls made since profiling was enabled. */
int tk_profile_read(tk_ctx* ctx, double ms[TK_NSTAGES], int64_t calls[TK_NSTAGES]);
/* Kernels launched by the library in this process so far. */
uint64_t tk_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_MATERN_H */
