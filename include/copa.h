/*
 * copa.h — C ABI of the GB300 implementation of the per-iteration hot path of COPA,
 * constrained PARAFAC2 fitted by AO-ADMM (Afshar et al., arXiv 1803.04572).
 *
 * Model (Sec. 2 "Original PARAFAC2 model", Sec. 3.1): every subject k holds a sparse
 * I_k x J slice X_k ~ Q_k H S_k V^T with S_k = diag(W(k,:)), Q_k^T Q_k = I. One outer
 * iteration of Algorithm 1 is
 *   (a) the Procrustes step Q_k = polar(X_k V S_k H^T) (Eq. 5),
 *   (b) the projection Y_k = Q_k^T X_k,
 *   (c) the MTTKRPs of Y for H, W and V,
 *   (d) per factor an ADMM inner loop with a cached Cholesky of G + rho I, a proximal
 *       operator and the dual update (Eq. 8 update rules, Sec. 3.3).
 *
 * Conventions shared by every call
 *   - All array pointers are DEVICE pointers unless a name ends in _host. They are
 *     owned by the caller, must stay valid until the work queued on the handle's
 *     stream has finished, and are never freed by the library.
 *   - Matrices are dense row-major: H is R x R, V is J x R, W is K x R (row k holds the
 *     diagonal of S_k), per-subject R x R blocks are stored one after another.
 *   - "real" arrays are float in COPA_PREC_MIXED handles and double in COPA_PREC_FP64
 *     handles (the precision chosen at copa_create). Gram matrices (G, U^T U) and
 *     scalars are always double.
 *   - Calls are asynchronous on the handle's stream unless documented otherwise.
 *     Errors found on the host are returned at once; errors found by a kernel are
 *     written to a device status word and returned by the next call that
 *     synchronises (copa_sync, copa_fit, copa_fit_host, copa_smooth_plan).
 *   - A handle is not thread-safe. Different handles may be used from different
 *     threads.
 */
#ifndef COPA_H
#define COPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  COPA_OK = 0,
  COPA_ERR_INVALID_ARG = 1, /* a size, pointer, index or option is out of range */
  COPA_ERR_OOM = 2,         /* the library could not allocate its workspace */
  COPA_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  COPA_ERR_NUMERIC = 4,     /* a non-positive Cholesky pivot or a non-finite value */
  COPA_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  COPA_ERR_UNSUPPORTED = 6, /* the request is valid but not implemented (e.g. R > 128) */
  COPA_ERR_COMM = 7         /* the caller's all-reduce callback reported a failure */
} copa_status_t;

typedef enum { COPA_PREC_MIXED = 0, COPA_PREC_FP64 = 1 } copa_precision_t;

/* Proximal operator applied to a factor (Sec. 3.3): none, max(0,v), soft threshold
 * sign(v) max(|v| - lambda/rho, 0), hard threshold (v if v^2 > 2 lambda / rho else 0). */
typedef enum { COPA_C_NONE = 0, COPA_C_NONNEG = 1, COPA_C_L1 = 2, COPA_C_L0 = 3 } copa_constraint_t;

/* Element type of the nonzero values of X. BF16 is accepted only for values that are
 * integers of magnitude <= 256 (exact in bf16; checked by copa_validate). */
typedef enum { COPA_VAL_F32 = 0, COPA_VAL_F64 = 1, COPA_VAL_BF16 = 2 } copa_val_dtype_t;

typedef enum { COPA_MODE_H = 0, COPA_MODE_V = 1, COPA_MODE_W = 2 } copa_mode_t;

/* Segmented per-subject CSR storage of {X_k} (device arrays, caller-owned, read-only).
 * Rows of subject k are subj_ptr[k] .. subj_ptr[k+1]-1; nonzeros of row i are
 * row_ptr[i] .. row_ptr[i+1]-1 with 0 <= col_idx < J, strictly increasing in a row. */
typedef struct {
  int64_t K;
  int32_t J;
  int64_t S;                /* total rows = subj_ptr[K] */
  int64_t nnz;              /* total nonzeros = row_ptr[S] */
  const int64_t* subj_ptr;  /* K+1 */
  const int64_t* row_ptr;   /* S+1 */
  const int32_t* col_idx;   /* nnz */
  const void* vals;         /* nnz, element type val_dtype */
  int32_t val_dtype;        /* copa_val_dtype_t */
} copa_tensor_t;

/* Result of the Procrustes step (caller-owned device buffers).
 * Q holds Q_k for every subject explicitly, row i of Q being row (i - subj_ptr[k]) of
 * Q_k for the subject k owning visit i; Y_k = Q_k^T X_k stays implicit: the MTTKRPs use
 * T_k = Q_k^T X_k V (= Y_k V) and Q itself. */
typedef struct {
  void* Q;         /* real[S*R], required: the orthonormal factors Q_k, stacked by rows */
  void* T;         /* real[K*R*R], required: T_k = Q_k^T X_k V, row-major R x R */
  void* Pi;        /* real[K*R*R], optional (NULL): Pi_k = Q_k^T Q_k (a projector) */
  int32_t* rank;   /* int32[K], optional (NULL): number of kept singular values */
} copa_procrustes_out_t;

typedef struct {
  int32_t R;               /* target rank, 1 <= R <= 128 */
  int32_t n_outer;         /* outer iterations (Algorithm 1, fixed count) */
  int32_t n_inner;         /* ADMM iterations per factor update (fixed count) */
  int32_t c_H, c_W, c_V;   /* copa_constraint_t per factor */
  double lam_H, lam_W, lam_V; /* regularisation weights of the l1 / l0 constraints */
  double tau;              /* Procrustes rank cut: keep eigenvalues > tau * max (1e-8) */
  double x_norm2;          /* sum_k ||X_k||^2 of the ORIGINAL data when X is a smoothed
                              projection (Sec. 3.3.1); <= 0 means: use ||X||^2 */
  int32_t use_graph;       /* 1: capture one outer iteration in a CUDA graph and replay */
  /* Convergence tests of Algorithm 1 (the paper names them without defining them; <= 0
   * keeps the fixed counts above). eps_inner > 0: each factor's ADMM stops after the first
   * iteration with ||Zbar - Z||_F <= eps ||Zbar||_F and ||Zbar - Zbar_prev||_F <= eps ||Zbar||_F
   * (norms over the whole factor; n_inner is then the cap). eps_fit > 0: the outer loop
   * stops after the first iteration t >= 2 with |FIT_t - FIT_{t-1}| <= eps_fit (n_outer is
   * the cap). copa_fit_stats reports the counts that ran. */
  double eps_inner;
  double eps_fit;
} copa_options_t;

typedef struct copa_ctx* copa_handle_t;

/* Create a handle bound to `device` and to `stream` (a cudaStream_t, NULL = legacy
 * default stream). The library allocates its workspace lazily on that device. */
copa_status_t copa_create(copa_handle_t* handle, int device, void* stream, int32_t precision);
copa_status_t copa_destroy(copa_handle_t handle);
/* Human-readable description of the last error on this handle (never NULL). */
const char* copa_last_error(copa_handle_t handle);
/* Wait for the handle's stream and return the first device-side error, if any. */
copa_status_t copa_sync(copa_handle_t handle);

/* Check X on the device: monotone pointer arrays, 0 <= col < J, strictly increasing
 * columns in each row, BF16 values integral and <= 256 in magnitude. Synchronises.
 * Returns COPA_ERR_INVALID_ARG with a message naming the first violation. */
copa_status_t copa_validate(copa_handle_t handle, const copa_tensor_t* X);

/* A handle keeps data derived from the tensors it has been called with, keyed by their
 * device addresses and sizes: the schedule of subjects by I_k, the offsets and the
 * Jacobi rotations of the warm start (the previous iteration's rotations start the next
 * one), the column-sorted copy of X and the nonzero -> row maps of the V mode, and the
 * choice of copa_tune. A tensor whose device arrays were rewritten in place, or a new
 * tensor at the addresses of a freed one with the same sizes, looks unchanged to those
 * keys: call copa_forget_tensor before the next call with it. It waits for the handle's
 * stream, then drops every such datum (they are rebuilt on the next call, and the next
 * fit starts its Procrustes sweeps cold). copa_fit_host needs no such call: it compares
 * the uploaded tensor with the previous one itself. */
copa_status_t copa_forget_tensor(copa_handle_t handle);

/* (a)+(b), Eq. 5 and Algorithm 1's per-subject loop, for every subject at once:
 * A_k = X_k V S_k H^T = B D C^T (thin SVD) and Q_k = B C^T over the singular values with
 * sigma^2 > tau * sigma_max^2 (tau = 1e-8 in the paper's reading used here). Computed by
 * one-sided Jacobi on the rows of A_k (I_k <= R) or of the R factor of a Householder QR
 * of A_k (I_k > R), never forming A_k^T A_k. Writes Q (S x R), T_k = Q_k^T X_k V and, on
 * request, Pi_k and rank_k. If F_H is not NULL it also returns the mode-1 MTTKRP
 * F_H = sum_k T_k S_k (R x R, real), which is (c) for H, fused. H: R x R, V: J x R,
 * W: K x R (S_k = diag(W(k,:))). Shared memory bounds R: <= 96 in COPA_PREC_MIXED,
 * <= 64 in COPA_PREC_FP64 (COPA_ERR_UNSUPPORTED above). */
copa_status_t copa_procrustes(copa_handle_t handle, const copa_tensor_t* X, int32_t R,
                              const void* H, const void* V, const void* W, double tau,
                              copa_procrustes_out_t* out, void* F_H);

/* Diagnostic (no counterpart in the paper): the number of multiply-adds the last
 * copa_procrustes launch on this handle performed, as tallied by the kernel from the
 * rows, rotations and products it executed (the algorithmic work behind the roofline
 * figure of the benchmark). Synchronises; writes 0 before the first launch. */
copa_status_t copa_procrustes_work(copa_handle_t handle, double* fma_host);

/* Test hook (no counterpart in the paper). COPA_DEBUG_TC_FORCE_TIMEOUT_NS = value > 0 makes
 * the first bounded wait of every later launch of the tensor-core V-mode kernel (FP32
 * handles, copa_mttkrp(COPA_MODE_V) and copa_fit) wait on an mbarrier that nothing arrives
 * at, for `value` ns, instead of on its first MMA batch: the kernel then takes its timeout
 * path (status COPA_ERR_TIMEOUT, reported by the next synchronising call; it waits for the
 * MMAs it issued, frees its tensor memory and returns), so that this path can be tested
 * without a fault. 0 switches it off. value must be in [0, 1e9]; other keys return
 * COPA_ERR_INVALID_ARG. The results of an affected call are undefined. */
enum { COPA_DEBUG_TC_FORCE_TIMEOUT_NS = 1 };
copa_status_t copa_debug_set(copa_handle_t handle, int32_t key, int64_t value);

/* Diagnostic (no counterpart in the paper): the number of kernels the last copa_fit call
 * on this handle launched (the kernel nodes of the captured iteration graph times n_outer,
 * plus set-up kernels), or -1 if unknown (use_graph = 0). */
copa_status_t copa_fit_launches(copa_handle_t handle, int64_t* launches_host);

/* (c) The MTTKRPs of Y = {Q_k^T X_k} (Sec. 2, Algorithm 1 "F = Y_(n)(Khatri-Rao)"),
 * from the Procrustes output `st` (computed with some V_p; T_k = Q_k^T X_k V_p):
 *   COPA_MODE_H: F (R x R) = sum_k T_k diag(W(k,:))               uses st->T, W
 *   COPA_MODE_W: F (K x R), F(k,s) = sum_r H(r,s) T_k(r,s)         uses st->T, H
 *   COPA_MODE_V: F (J x R) = sum_k X_k^T Q_k H diag(W(k,:))        uses X, st->Q, H, W
 *                if UtU is not NULL it also returns U^T U = sum_k S_k H^T Q_k^T Q_k H S_k
 *                (R x R double), the Gram of the rows of Q_k H S_k (FIT and gradient).
 * Pointers a mode does not use may be NULL. F is overwritten. */
copa_status_t copa_mttkrp(copa_handle_t handle, int32_t mode, const copa_tensor_t* X,
                          int32_t R, const copa_procrustes_out_t* st, const void* H,
                          const void* W, void* F, double* UtU);

/* Column Gram G = A^T A (R x R, double) of a rows x R real matrix (Algorithm 1: the
 * factor Grams whose Hadamard products give G for each mode). */
copa_status_t copa_gram(copa_handle_t handle, const void* A, int64_t rows, int32_t R,
                        double* G);

/* Column Gram without any allocation (no counterpart in the paper; a deployment aid).
 * Some callers cannot allocate device memory while they run this: their device memory
 * is reserved up front by their own pool, or the implicit device synchronisation of
 * cudaMalloc/cudaFree would stall other work they have in flight. This call computes the
 * same G = A^T A as copa_gram but needs no handle and no workspace: its per-block partial
 * sums go to a fixed 1 MiB array that libcopa keeps in device memory (every GPU that
 * loads the library holds it until the process exits). It allocates nothing and calls no
 * allocating routine.
 *   stream:     cudaStream_t to enqueue on (NULL = legacy default stream)
 *   a_is_double: 0 if A is float, 1 if A is double
 *   A:          rows x R row-major (device), G: R x R double (device, overwritten)
 * Runs on the calling thread's current device. R > 90 returns COPA_ERR_UNSUPPORTED,
 * other bad sizes or NULL pointers COPA_ERR_INVALID_ARG. The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, no allocation); make that first
 * call before any stream capture. That address is cached for the life of the process,
 * which assumes the device's primary context is never reset (no cudaDeviceReset while
 * the library is loaded). A CUDA error already pending on the calling thread when the
 * call starts is left in place and the call returns COPA_ERR_CUDA without launching. All calls share the one array, which keeps the last
 * call's contents: calls that may overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. Asynchronous: launch errors are returned at
 * once, execution errors surface at the caller's next synchronisation. */
copa_status_t copa_gram_noalloc(void* stream, int32_t a_is_double, const void* A, int64_t rows,
                                int32_t R, double* G);

/* (d) One factor update by ADMM (Algorithm 1 inner loop; Eq. 8 update rules):
 * G = Ga .* Gb (R x R double, Hadamard product of two Grams; Gb may be NULL meaning
 * G = Ga), rho = trace(G)/R, L = chol(G + rho I) (FP64), then n_inner times, row-wise
 *   z = (G + rho I)^{-1} (f + rho (zbar + d)),  zbar = prox_c(z - d),  d = d + zbar - z.
 * F, Zbar, D are rows x R real; Zbar and D are updated in place. rho_out (double[1],
 * device, may be NULL) receives rho. Returns COPA_ERR_NUMERIC (at the next sync) if
 * G + rho I is not positive definite. */
copa_status_t copa_admm_step(copa_handle_t handle, const void* F, const double* Ga,
                             const double* Gb, int32_t n_inner, int32_t constraint,
                             double lambda, void* Zbar, void* D, int64_t rows, int32_t R,
                             double* rho_out);

/* (c)+(d) fused for W (a warp per subject, all inner iterations in registers):
 * F_W(k,:) = diag(H^T T_k) then the ADMM row update of W with G = Ga .* Gb. */
copa_status_t copa_admm_w_fused(copa_handle_t handle, const copa_procrustes_out_t* st,
                                const void* H, const double* Ga, const double* Gb,
                                int32_t n_inner, int32_t constraint, double lambda,
                                void* Wbar, void* DW, int64_t K, int32_t R,
                                double* rho_out);

/* FIT (Sec. 4.1) of the model (Q_k from `st`, H, V, W) from the pieces of the V-mode
 * MTTKRP: with F_V and U^T U computed by copa_mttkrp(COPA_MODE_V) at (H, W),
 *   sum_k ||X_k - Q_k H S_k V^T||^2 = ||X||^2 - 2 <V, F_V> + <V^T V, U^T U>,
 * FIT = 1 - (x_norm2 - ||X||^2 + that) / x_norm2 (x_norm2 <= 0: x_norm2 = ||X||^2).
 * Writes fit (double[1], device). */
copa_status_t copa_fit_value(copa_handle_t handle, const copa_tensor_t* X, int32_t R,
                             const void* V, const void* F_V, const double* UtU,
                             double x_norm2, double* fit);

/* Algorithm 1: n_outer outer iterations from the given state. H, V, W hold the initial
 * auxiliary factors on entry and the fitted ones on return; DH, DV, DW (same shapes)
 * hold the scaled duals (zero for a cold start) and are updated. fit_history_host
 * (double[n_outer], HOST, may be NULL) receives the FIT after every iteration.
 * st (may be NULL) receives the last iteration's Procrustes output (Q and T; Pi and rank
 * if given), from which the paper's outputs U_k = Q_k H follow. Synchronises. */
copa_status_t copa_fit(copa_handle_t handle, const copa_tensor_t* X, const copa_options_t* opt,
                       void* H, void* V, void* W, void* DH, void* DV, void* DW,
                       double* fit_history_host, copa_procrustes_out_t* st);

/* Subject sharding (Sec. 3.2: the Procrustes loop runs over subjects independently; every
 * other step touches the subjects only through sums). A fit over K subjects can be split
 * into shards of contiguous subjects, one per GPU: a shard holds its subjects' slices X_k
 * and rows of W and D_W; H, V, D_H, D_V are replicated. Each shard runs copa_fit on its own
 * subjects; the partial sums F_H, W^T W, F_V, U^T U and ||X||^2 are completed by an
 * all-reduce (sum over shards) that the caller supplies, after which the H and V updates
 * see identical inputs on every shard and the FIT is that of the whole tensor.
 *
 * copa_partition (host only, no GPU needed): contiguous shards balanced by nonzeros.
 * subj_ptr_host (K+1) and row_ptr_host (S+1) are X's HOST pointer arrays; bounds_host
 * (nshards+1) receives the first subject of every shard, bounds[0] = 0, bounds[nshards] = K,
 * non-decreasing: shard p holds subjects bounds[p] .. bounds[p+1]-1, and bounds[p] is the
 * subject boundary whose nonzero prefix is closest to p * nnz / nshards. Returns
 * COPA_ERR_INVALID_ARG for NULL arrays, K < 0 or nshards < 1. */
copa_status_t copa_partition(const int64_t* subj_ptr_host, const int64_t* row_ptr_host, int64_t K,
                             int32_t nshards, int64_t* bounds_host);

/* The all-reduce of a sharded fit. Called by copa_fit on the calling thread with `count`
 * doubles at buf (the device buffer registered below); it must leave in buf[0..count) the
 * elementwise sum of buf over all shards, either before it returns or enqueued on `stream`
 * (the handle's cudaStream_t; work the library enqueues after the call waits for it). It
 * returns 0 on success; anything else fails the fit with COPA_ERR_COMM. Every shard makes
 * the same sequence of calls with the same counts. */
typedef int32_t (*copa_allreduce_fn)(double* buf, int64_t count, void* stream, void* user);

/* Registers (fn != NULL) or clears (fn == NULL) the all-reduce of this handle. While one is
 * registered, copa_fit and copa_fit_host run as one shard of a sharded fit: X holds the
 * shard's subjects, W and D_W their rows, the FIT history is the whole tensor's. Outer
 * iterations are then launched eagerly (use_graph is ignored: the callback runs on the
 * host between steps). buf (device, caller-owned) must hold at least
 * J * R + 2 * R * R doubles for the fits that follow (checked at copa_fit). */
copa_status_t copa_set_allreduce(copa_handle_t handle, copa_allreduce_fn fn, void* user, double* buf,
                                 int64_t capacity);

/* The plain per-subject FP64 form of Algorithm 1 (a comparison form: the method as
 * written, without this library's batching, fusion or precision choices). Same arguments
 * and results as copa_fit (fixed counts; eps_*, use_graph and the sharding hook are not
 * used) on an FP64 handle: one block per subject forms A_k = X_k V S_k H^T in global memory,
 * the FP64 Gram A_k^T A_k (or A_k A_k^T when I_k < R) and its eigendecomposition by cyclic
 * Jacobi, and Q_k = A_k C Lambda^{-1/2}_+ C^T (or C Lambda^{-1/2}_+ C^T A_k) over the
 * eigenvalues above tau times the largest (Eq. 5 with the truncated SVD of Algorithm 1);
 * Y_k = Q_k^T X_k is materialised over the distinct columns of every X_k; the MTTKRPs read Y;
 * each ADMM inner iteration is its own launch; the host waits for every outer iteration.
 * R <= 64 and J <= 65536 (COPA_ERR_UNSUPPORTED otherwise, and on a mixed handle). Uses
 * (2 S + 1) R + (distinct (subject, column) pairs) R doubles of workspace. Synchronises. */
copa_status_t copa_fit_plain(copa_handle_t handle, const copa_tensor_t* X, const copa_options_t* opt,
                             void* H, void* V, void* W, void* DH, void* DV, void* DW,
                             double* fit_history_host);

/* Launch-schedule autotuner (no counterpart in the paper). The schedule of one outer
 * iteration has three knobs that depend on the rank, the precision and the distribution of
 * subject sizes I_k:
 *   split          subjects with I_k > split take the tall-subject Procrustes kernels (QR,
 *                  Jacobi on R_A, second pass), the others the warp-per-subject kernel;
 *                  1 <= split <= min(R, 32) (default min(R, 32));
 *   blocks_per_sm  cap on the resident blocks per SM of those persistent kernels (0 = as
 *                  many as fit, the default);
 *   fv_path        F_V (mixed precision) by the row-order kernel with the sums in L2 (2,
 *                  the default; R a multiple of 4, 2, or R <= 32), by the row-order kernel
 *                  with shared-memory sums (0; J x 32 floats must fit), or over the
 *                  column-sorted copy of X (1). A path that does not apply falls back to
 *                  the next in that order.
 * copa_tune times the candidates (every split in {min(R,32), 24, 16, 8} below min(R,32) with
 * blocks_per_sm in {0, 2}; then the F_V kernels that apply) on X with the factors H, V, W, with CUDA
 * events on the handle's stream, and keeps the fastest: in a process-wide table keyed by
 * copa_tune_key(R, precision, size histogram) and on the handle, whose later calls on the
 * same X (same subj_ptr, K, S) and R use it. A key already in the table is applied without
 * timing unless force != 0. out (HOST, may be NULL) receives the choice, ms the measured
 * time of one Procrustes step plus one V mode with it. Synchronises. */
typedef struct {
  int32_t split;
  int32_t blocks_per_sm;
  int32_t fv_path;
  float ms;
} copa_tune_t;
copa_status_t copa_tune(copa_handle_t handle, const copa_tensor_t* X, int32_t R, const void* H,
                        const void* V, const void* W, int32_t force, copa_tune_t* out);
/* The table's key (host only, no GPU): a hash of R, precision and the share of subjects in
 * each power-of-two size class of I_k (0, 1, 2-3, 4-7, ...) rounded to 1/64, so that
 * tensors drawn from the same size distribution share it. subj_ptr_host has K+1 entries. */
copa_status_t copa_tune_key(const int64_t* subj_ptr_host, int64_t K, int32_t R, int32_t precision,
                            uint64_t* key);
/* Table access (host only): lookup sets *found (0/1) and, if found, *out; store inserts or
 * replaces (split >= 1, blocks_per_sm >= 0, fv_path 0, 1 or 2, else COPA_ERR_INVALID_ARG). */
copa_status_t copa_tune_lookup(uint64_t key, int32_t* found, copa_tune_t* out);
copa_status_t copa_tune_store(uint64_t key, const copa_tune_t* choice);

/* Hyperparameter sweeps (Sec. 4.2 tunes the regularisation weight and the basis over a
 * grid): G independent fits of the same X (device, resident once) with their own options,
 * factors and duals, run concurrently on G streams that the library creates and keeps
 * with the handle (each with its own workspace). opts[g], H[g], V[g], W[g], DH[g], DV[g],
 * DW[g] are those of copa_fit for fit g; all fits share R and n_outer (constraints,
 * lambdas, n_inner, tau, eps_* may differ). fit_history_host (HOST, G x n_outer, may be
 * NULL) receives each fit's FIT history as a row. The fits start after the work already
 * queued on the handle's stream, and work queued there after the call sees their results.
 * Synchronises. 1 <= G <= 64; not for a shard of a sharded fit. copa_fit_stats is not
 * updated by this call. */
copa_status_t copa_fit_batch(copa_handle_t handle, const copa_tensor_t* X, int32_t G,
                             const copa_options_t* opts, void* const* H, void* const* V, void* const* W,
                             void* const* DH, void* const* DV, void* const* DW, double* fit_history_host);

/* The iteration counts of the last copa_fit / copa_fit_host call on this handle:
 * n_outer_run_host (int32[1]) the outer iterations run (< n_outer if eps_fit stopped the
 * loop; FIT history entries past it are NaN), inner_host (int32[3 * n_outer], may be NULL)
 * the ADMM iterations of H, W, V (update order) in each outer iteration (n_inner each with
 * fixed counts, 0 past n_outer_run). */
copa_status_t copa_fit_stats(copa_handle_t handle, int32_t* n_outer_run_host, int32_t* inner_host);

/* copa_fit on HOST buffers: copies X (arrays given as host pointers in X_host) and the
 * state to the device, runs copa_fit, copies H, V, W, the duals and the FIT history
 * back. Device memory is owned by the handle and reused across calls. The uploaded X is
 * compared byte for byte, on the device, with the one the previous call uploaded: if it
 * is the same, the data derived from it (see copa_forget_tensor) carry over, so that
 * successive calls continue one fit (warm start included); otherwise they are rebuilt.
 * Synchronises. */
copa_status_t copa_fit_host(copa_handle_t handle, const copa_tensor_t* X_host,
                            const copa_options_t* opt, void* H_host, void* V_host,
                            void* W_host, void* DH_host, void* DV_host, void* DW_host,
                            double* fit_history_host);

/* Pipelined input for copa_fit_host (no counterpart in the paper): queues the copy of the
 * four arrays of a HOST tensor (pinned memory, or the copy is synchronous) into device
 * buffers of the handle (allocated here) and returns. The next copa_fit_host call issues
 * the queued copies on a copy stream of the handle's own, behind its own host-to-device
 * copies, so that they run while its kernels do; a later copa_fit_host call whose X_host
 * names the same four host pointers with the same K, J, S, nnz and val_dtype as the oldest
 * queued copy takes it (its stream waits for the copy) instead of copying X itself (if the
 * oldest was not issued yet, that call copies X itself). At most two copies are queued; a
 * copa_fit_host call whose X_host does not match the oldest waits for the issued ones and
 * discards them all. The copy reads the arrays while it runs: the caller must not write
 * them until the copa_fit_host call that takes (or discards) the copy has returned, or the
 * handle is destroyed. A NULL X_host or array, negative sizes, an unknown val_dtype and a
 * third queued copy return COPA_ERR_INVALID_ARG; COPA_ERR_OOM if the buffers cannot be
 * allocated. The contents are checked by the copa_fit_host call that takes the copy, as
 * for its own copies. */
copa_status_t copa_stage_host(copa_handle_t handle, const copa_tensor_t* X_host);

/* Smoothness on U_k (Sec. 3.3.1), set-up step. For every subject, the B-spline basis of
 * the given degree with n_basis functions on [t_1, t_{I_k}] (the first and last visit day;
 * days (double[S], device) must be non-decreasing within a subject; boundary knots
 * repeated degree+1 times; Cox-de Boor recursion) is evaluated at the visit days,
 * M_k = C_k D P^T, and C_k keeps the left singular vectors with sigma^2 > 1e-10
 * sigma_max^2 (r_k of them; if t_1 = t_{I_k} the basis is the constant function). The
 * n_basis - degree - 1 interior knots follow knot_rule: COPA_KNOTS_UNIFORM spaces them
 * equally in days, COPA_KNOTS_QUANTILE puts them at the quantiles j / (n_basis - degree)
 * of the subject's visit days (linear interpolation between order statistics), i.e.
 * where the visits are (the paper estimates the knots from the data and builds the
 * functions on days so that uneven gaps are respected). The projected slices
 * X'_k = C_k^T X_k are r_k x J, stored as CSR over the columns X_k uses.
 * copa_smooth_plan returns the sizes of X' (S' rows, nnz' nonzeros) and synchronises;
 * copa_smooth_project fills X' (caller-allocated device arrays in Xp: subj_ptr K+1,
 * row_ptr S'+1, col_idx nnz', vals nnz' of type Xp->val_dtype = F32 or F64). The
 * optional C (double[S * n_basis], device, may be NULL) receives C_k padded with zero
 * columns to n_basis. */
enum { COPA_KNOTS_UNIFORM = 0, COPA_KNOTS_QUANTILE = 1 };
copa_status_t copa_smooth_plan(copa_handle_t handle, const copa_tensor_t* X,
                               const double* days, int32_t n_basis, int32_t degree,
                               int32_t knot_rule, int64_t* S_out_host, int64_t* nnz_out_host);
copa_status_t copa_smooth_project(copa_handle_t handle, const copa_tensor_t* X,
                                  const double* days, int32_t n_basis, int32_t degree,
                                  int32_t knot_rule, copa_tensor_t* Xp, double* C);

/* The output factor of Algorithm 1 (Sec. 3.3.1): U_k = Q_k H, or U_k = C_k Q_k H when the
 * fit ran on the smoothed projection. Q (S_fit x R, real) holds Q_k of every subject
 * stacked by rows with offsets subj_ptr_fit (K+1, device: those of the tensor the fit ran
 * on), as copa_procrustes or copa_fit's state returns it; H is R x R.
 *   C == NULL: U (S_fit x R, real) gets u_i = q_i H.
 *   C != NULL: C (S x n_basis double, device) as copa_smooth_project returns it (C_k padded
 *     with zero columns to n_basis), subj_ptr (K+1, device) the ORIGINAL X's row offsets;
 *     U (S x R, real) gets, for visit row i of subject k,
 *     u_i = sum_{q < r_k} C[i, q] (Q_k H)(q, :) with r_k = subj_ptr_fit[k+1] - subj_ptr_fit[k].
 * With C it uses S_fit x R reals of the handle's workspace. Asynchronous. */
copa_status_t copa_factor_U(copa_handle_t handle, int64_t K, int32_t R, const int64_t* subj_ptr_fit,
                            int64_t S_fit, const void* Q, const void* H, const int64_t* subj_ptr,
                            const double* C, int32_t n_basis, int64_t S, void* U);

/* Reconstruction loss L = sum_k ||X_k - Q_k H S_k V^T||_F^2 (no 1/2) with Q_k fixed (from
 * `st`, which must include Pi and come from copa_procrustes at the same H, V, W) and its
 * gradient: dL/dH = -2 (F_H - sum_k Pi_k H S_k V^T V S_k), dL/dV = -2 (F_V - V U^T U),
 * dL/dW(k,r) = -2 [(H^T T_k)(r,r) - (H^T Pi_k H S_k V^T V)(r,r)]. loss is double[1]
 * (device); gH (R x R), gV (J x R), gW (K x R) are real and overwritten. */
copa_status_t copa_loss_grad(copa_handle_t handle, const copa_tensor_t* X, int32_t R,
                             const copa_procrustes_out_t* st, const void* H, const void* V,
                             const void* W, double* loss, void* gH, void* gV, void* gW);

#ifdef __cplusplus
}
#endif
#endif /* COPA_H */
