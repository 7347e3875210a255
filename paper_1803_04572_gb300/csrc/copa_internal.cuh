// Internal declarations shared by the CUDA translation units of libcopa.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "copa.h"

namespace copa {

constexpr int kMaxR = 96;          // largest rank the shared-memory kernels hold
constexpr int kMaxBasis = 16;      // largest spline basis (smoothing set-up)

// Device status word layout (int32[4] in the workspace): [0] = first error code,
// [1..3] = details (subject index, etc.). Kernels never trap; they record and return.
__device__ __forceinline__ void set_status(int* st, int code, int info = 0) {
  if (atomicCAS(st, 0, code) == 0) st[1] = info;
}

// Read-only view of X on the device.
struct TensorView {
  int64_t K;
  int32_t J;
  int64_t S;
  int64_t nnz;
  const int64_t* subj_ptr;
  const int64_t* row_ptr;
  const int32_t* col;
  const void* vals;
  int32_t dtype;
};

__device__ __forceinline__ double load_val(const TensorView& X, int64_t i) {
  if (X.dtype == COPA_VAL_BF16) {
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X.vals)[i]);
  } else if (X.dtype == COPA_VAL_F32) {
    return (double)__ldg(reinterpret_cast<const float*>(X.vals) + i);
  }
  return __ldg(reinterpret_cast<const double*>(X.vals) + i);
}

__device__ __forceinline__ float load_valf(const TensorView& X, int64_t i) {
  if (X.dtype == COPA_VAL_BF16) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X.vals)[i]);
  } else if (X.dtype == COPA_VAL_F32) {
    return __ldg(reinterpret_cast<const float*>(X.vals) + i);
  }
  return (float)__ldg(reinterpret_cast<const double*>(X.vals) + i);
}

template <typename Real>
__device__ __forceinline__ Real load_x(const TensorView& X, int64_t i);
template <>
__device__ __forceinline__ float load_x<float>(const TensorView& X, int64_t i) {
  return load_valf(X, i);
}
template <>
__device__ __forceinline__ double load_x<double>(const TensorView& X, int64_t i) {
  return load_val(X, i);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Proximal operators of Sec. 3.3 (v = z - d). Shared by every ADMM kernel.
template <typename Real>
__device__ __forceinline__ Real prox(Real v, int c, Real lam_over_rho) {
  switch (c) {
    case COPA_C_NONNEG:
      return v > Real(0) ? v : Real(0);
    case COPA_C_L1: {
      Real a = fabs(v) - lam_over_rho;
      if (a <= Real(0)) return Real(0);
      return v > Real(0) ? a : -a;
    }
    case COPA_C_L0:
      return (v * v > Real(2) * lam_over_rho) ? v : Real(0);
    default:
      return v;
  }
}

}  // namespace copa

// The handle. Workspace buffers grow on demand and are reused.
struct copa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = COPA_PREC_MIXED;
  std::string err;
  int* d_status = nullptr;       // int32[4] device status word
  int num_sms = 0;
  // generic workspace slots
  void* slot_ptr[20] = {nullptr};
  size_t slot_bytes[20] = {0};
  // cached per-tensor schedule (subjects ordered by decreasing I_k)
  const int64_t* sched_key = nullptr;
  int64_t sched_K = 0;
  int64_t sched_S = 0;
  // copa_fit_host device copies: [0..3] X as the last call left it, [4..9] the state,
  // [10..13] the X arrays of the current call before the comparison, [14] a flag,
  // [15..18] and [19..22] the two sets of copa_stage_host copies
  static constexpr int kHostSlots = 23;
  void* host_slot_ptr[kHostSlots] = {nullptr};
  size_t host_slot_bytes[kHostSlots] = {0};
  // copa_stage_host: pending copies of host tensors, oldest first; each names its slot set
  // (0: [15..18], 1: [19..22]) and, once issued on copy_stream, has stage_ev[set] recorded
  // after its copies
  struct StagedX {
    int set = 0;
    bool issued = false;
    const void* src[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t K = -1, J = -1, S = -1, nnz = -1;
    int vdt = -1;
  };
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  cudaEvent_t stage_go = nullptr;   // recorded on `stream` after a copa_fit_host call's own copies
  StagedX staged[2];
  int n_staged = 0;
  bool host_x_valid = false;   // [0..3] hold the X of the last copa_fit_host call
  int64_t host_K = -1, host_J = -1, host_S = -1, host_nnz = -1;
  int host_vdt = -1;
  // CUDA graph of one outer iteration
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_key = 0;
  // cached warm-start offsets (per tensor and rank)
  const int64_t* warm_key = nullptr;
  int64_t warm_K = 0, warm_S = 0, warm_total = 0;
  int warm_R = 0;
  int warm_prec = -1;
  bool warm_valid = false;   // the buffer holds the rotations of a finished iteration
  // kernels launched by the last copa_fit call (graph nodes x iterations + set-up), -1 unknown
  int64_t fit_launches = -1;
  int64_t setup_launches = 0;
  // cached column-sorted copy of X
  const int32_t* csc_key = nullptr;
  int64_t csc_nnz = -1, csc_S = -1;
  int csc_J = 0, csc_prec = -1;
  // iteration counts of the last copa_fit (copa_fit_stats)
  int32_t last_n_run = 0;
  std::vector<int32_t> last_inner;
  // the fit enqueued last (results collected by finish_fit)
  const int* pend_it = nullptr;
  const double* pend_hist = nullptr;
  const int* pend_counts = nullptr;
  int pend_n_outer = 0, pend_n_inner = 0;
  bool pend_adaptive = false;
  int64_t pend_per_iter = -1;
  cudaGraphExec_t pend_exec = nullptr;   // replayed graph of that fit, destroyed by finish_fit
  // autotuned schedule (copa_tune): used by the calls on the tensor, rank and precision it
  // was tuned for
  bool tune_valid = false;
  const int64_t* tune_ptr = nullptr;
  int64_t tune_K = -1, tune_S = -1;
  int tune_R = 0;
  int tune_split = 0, tune_bps = 0, tune_fv = 0;
  // batched fits (copa_fit_batch): one child handle, with its own stream, per fit
  std::vector<copa_ctx*> children;
  cudaEvent_t batch_ev = nullptr;
  // sharded fit: the caller's all-reduce (copa_set_allreduce), NULL when not sharded
  copa_allreduce_fn red_fn = nullptr;
  void* red_user = nullptr;
  double* red_buf = nullptr;
  int64_t red_cap = 0;
  // test hook: > 0 makes the first mbarrier wait of the tensor-core V-mode kernel run out
  // after this many ns on an mbarrier that nothing arrives at (copa_debug_set)
  int64_t dbg_tc_force_ns = 0;
  // cached nonzero -> row and row -> subject maps (row-order F_V path)
  const int32_t* rmap_key = nullptr;
  int64_t rmap_nnz = -1, rmap_S = -1, rmap_K = -1;
};

namespace copa {

enum Slot {
  SLOT_ORDER = 0,      // int64[K] subject schedule
  SLOT_SCHED_TMP = 1,  // histogram / counters
  SLOT_PARTIAL = 2,    // per-warp or per-block FP64 partial sums
  SLOT_COUNTER = 3,    // int32 work counters
  SLOT_FIT_Q = 4,      // copa_fit: Q (S x R)
  SLOT_FIT_T = 5,      // copa_fit: T
  SLOT_FIT_SMALL = 6,  // copa_fit: F_H, F_V, Grams, Ginv, rho, UtU, fit values
  SLOT_GINV = 7,       // Ginv + rho for standalone ADMM calls
  SLOT_SMOOTH = 8,     // smoothing set-up temporaries
  SLOT_MISC = 9,
  SLOT_PI = 10,
  SLOT_WARM = 11,      // copa_fit: per-subject Jacobi rotations kept between iterations
  SLOT_WARM_OFF = 12,  // int64[K+1] offsets of the min(I_k,R)^2 blocks
  SLOT_CSC = 13,       // column-sorted copy of X (pointers, row indices, values)
  SLOT_UVEC = 14,      // u_i = q_i H S_k for every visit row (S x R)
  SLOT_ROWMAP = 15,    // int32 nonzero -> row map and int32 row -> subject map
  SLOT_FV_PART = 16,   // per-CTA partial sums of F_V (row-order path)
  SLOT_FIT_FW = 17,    // copa_fit: F_W (K x R) for the early-stopping W update
};
copa_status_t get_warm_offsets(copa_ctx* h, const TensorView& X, int R, const int64_t** woff,
                               int64_t* total);

// The schedule knobs of the Procrustes and V-mode launches: subjects with I_k > split take
// the tall-subject kernels; bps caps the resident blocks per SM of the persistent
// Procrustes kernels (0: as many as fit); fv selects the F_V kernel: 2 (default) row order
// with the sums in L2, 0 row order with shared-memory sums, 1 the column-sorted copy (each
// falls back to the next that applies). Defaults unless copa_tune chose them for (X, R).
struct TuneChoice {
  int split, bps, fv;
  bool pair;   // two subjects of I_k <= 16 per warp in the warp-per-subject Procrustes path
};
inline TuneChoice active_tune(const copa_ctx* h, const TensorView& X, int R) {
  TuneChoice c{R < 32 ? R : 32, 0, 2, true};
  if (h->tune_valid && h->tune_ptr == X.subj_ptr && h->tune_K == X.K && h->tune_S == X.S && h->tune_R == R) {
    c.split = h->tune_split;
    c.bps = h->tune_bps;
    c.fv = h->tune_fv;
  }
  return c;
}

copa_status_t ws_get(copa_ctx* h, int slot, size_t bytes, void** out);
// Drops everything the handle (and its batch children) derived from a tensor's contents:
// subject schedule, warm-start offsets and rotations, column-sorted copy, row maps, tuned
// schedule. The caches are keyed by device address and sizes, which a tensor rewritten in
// place (or a new one at a freed one's address) does not change.
void forget_tensor_caches(copa_ctx* h);
copa_status_t fail(copa_ctx* h, copa_status_t code, const std::string& msg);
copa_status_t cuda_check(copa_ctx* h, cudaError_t e, const char* what);
TensorView view_of(const copa_tensor_t* X);
copa_status_t check_tensor_args(copa_ctx* h, const copa_tensor_t* X);
copa_status_t get_schedule(copa_ctx* h, const TensorView& X, const int64_t** order);
// Device pointer to the number of subjects with I_k > thr (0 <= thr < 2047), which is the
// length of the prefix of the schedule (decreasing I_k) that holds them. Valid after
// get_schedule for the same tensor, until the next get_schedule for another tensor.
const int* schedule_count_above(copa_ctx* h, int thr);

// ---- launchers (host functions, enqueue on h->stream) ----
template <typename Real>
copa_status_t launch_procrustes(copa_ctx* h, const TensorView& X, int R, const Real* H,
                                const Real* V, const Real* W, double tau, Real* Q, Real* T,
                                Real* Pi, int32_t* rank, Real* F_H, Real* Uw = nullptr,
                                const int64_t* woff = nullptr, bool warm_in = false,
                                const int* epoch = nullptr);
template <typename Real>
size_t procrustes_smem(int R);
template <typename Real>
copa_status_t launch_mttkrp_h(copa_ctx* h, int64_t K, int R, const Real* T, const Real* W,
                              Real* F);
template <typename Real>
copa_status_t launch_mttkrp_v(copa_ctx* h, const TensorView& X, int R, const Real* Q,
                              const Real* H, const Real* W, Real* F, double* UtU,
                              bool reuse_csc = false);
// V-mode tile products on the tensor cores (FP32 path, k_vmode_tc.cu): U = (Q H) .* W(k(i),:)
// and the UtU partials (two per CTA, *nparts). Supported for R % 4 == 0, R <= 48 and
// 16-byte aligned Q, W, U.
bool uvec_tc_supported(int R, const void* Q, const void* W, const void* U);
copa_status_t launch_uvec_tc(copa_ctx* h, int64_t S, int R, const float* Q, const float* H, const float* W,
                             const int32_t* rsubj, float* U, double* utu_part, int64_t* nparts, bool size_only);
template <typename Real>
copa_status_t launch_mttkrp_w(copa_ctx* h, int64_t K, int R, const Real* T, const Real* H,
                              Real* F);
template <typename Real>
copa_status_t launch_gram(copa_ctx* h, const Real* A, int64_t rows, int R, double* G);
template <typename Real>
copa_status_t launch_chol(copa_ctx* h, const double* Ga, const double* Gb, int R, Real* Ginv,
                          double* rho_dev);
template <typename Real>
copa_status_t launch_admm_rows(copa_ctx* h, const Real* F, const Real* Ginv,
                               const double* rho_dev, int n_inner, int c, double lam,
                               Real* Zbar, Real* D, int64_t rows, int R);
// Early-stopping form of the row ADMM: at most max_inner launches of one iteration each,
// with the residual test of the method after each (see k_admm_check); the number of
// iterations run goes to counts[*it * 3 + mode].
template <typename Real>
copa_status_t launch_admm_adaptive(copa_ctx* h, const Real* F, const Real* Ginv, const double* rho_dev,
                                   int max_inner, int c, double lam, Real* Zbar, Real* D, int64_t rows, int R,
                                   double eps, double* acc, int* done, int* counts, const int* it, int mode);
template <typename Real>
copa_status_t launch_admm_w(copa_ctx* h, const Real* T, const Real* H, const Real* Ginv,
                            const double* rho_dev, int n_inner, int c, double lam, Real* Wbar,
                            Real* DW, int64_t K, int R);
template <typename Real>
// VtV (R x R, FP64) receives V^T V, which the FIT needs.
copa_status_t launch_fit_value(copa_ctx* h, int64_t J, int R, const Real* V, const Real* F_V,
                               const double* UtU, const double* xn2_dev, double x_norm2,
                               double* fit, double* VtV);
template <typename Real>
copa_status_t launch_loss_grad(copa_ctx* h, const TensorView& X, int R, const Real* Q,
                               const Real* T, const Real* Pi, const Real* H, const Real* V,
                               const Real* W, double* loss, Real* gH, Real* gV, Real* gW);
copa_status_t launch_validate(copa_ctx* h, const TensorView& X);
copa_status_t launch_xnorm2(copa_ctx* h, const TensorView& X, double* out);

}  // namespace copa
