// The C ABI of libcopa: handle and workspace management, argument checks, the subject
// schedule, X validation and the orchestration of whole outer iterations (Algorithm 1)
// on one stream, optionally captured once into a CUDA graph and replayed.
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "copa_internal.cuh"

using namespace copa;

namespace copa {

copa_status_t fail(copa_ctx* h, copa_status_t code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

copa_status_t cuda_check(copa_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return COPA_OK;
  return fail(h, COPA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

copa_status_t ws_get(copa_ctx* h, int slot, size_t bytes, void** out) {
  if (bytes == 0) bytes = 16;
  if (h->slot_bytes[slot] < bytes) {
    if (h->slot_ptr[slot]) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->slot_ptr[slot]);
      h->slot_ptr[slot] = nullptr;
      h->slot_bytes[slot] = 0;
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&h->slot_ptr[slot], want) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, COPA_ERR_OOM, "workspace allocation of " + std::to_string(want) + " bytes failed");
    }
    h->slot_bytes[slot] = want;
  }
  if (out) *out = h->slot_ptr[slot];
  return COPA_OK;
}

void forget_tensor_caches(copa_ctx* h) {
  h->sched_key = nullptr;
  h->sched_K = h->sched_S = 0;
  h->warm_key = nullptr;
  h->warm_valid = false;
  h->csc_key = nullptr;
  h->csc_nnz = h->csc_S = -1;
  h->rmap_key = nullptr;
  h->rmap_nnz = h->rmap_S = h->rmap_K = -1;
  h->tune_valid = false;
  h->tune_ptr = nullptr;
  h->host_x_valid = false;
  for (copa_ctx* c : h->children) forget_tensor_caches(c);
}

// The same for the caches keyed by one tensor's subj_ptr / col_idx addresses only.
static void forget_caches_of(copa_ctx* h, const void* subj_ptr, const void* col) {
  if (!subj_ptr && !col) return;
  if (h->sched_key == subj_ptr) h->sched_key = nullptr;
  if (h->warm_key == subj_ptr) {
    h->warm_key = nullptr;
    h->warm_valid = false;
  }
  if (h->tune_ptr == subj_ptr) {
    h->tune_valid = false;
    h->tune_ptr = nullptr;
  }
  if (h->csc_key == col) h->csc_key = nullptr;
  if (h->rmap_key == col) h->rmap_key = nullptr;
  for (copa_ctx* c : h->children) forget_caches_of(c, subj_ptr, col);
}

TensorView view_of(const copa_tensor_t* X) {
  TensorView v;
  v.K = X->K; v.J = X->J; v.S = X->S; v.nnz = X->nnz;
  v.subj_ptr = X->subj_ptr; v.row_ptr = X->row_ptr; v.col = X->col_idx; v.vals = X->vals;
  v.dtype = X->val_dtype;
  return v;
}

copa_status_t check_tensor_args(copa_ctx* h, const copa_tensor_t* X) {
  if (!X) return fail(h, COPA_ERR_INVALID_ARG, "X is NULL");
  if (X->K < 0 || X->J < 1 || X->S < 0 || X->nnz < 0)
    return fail(h, COPA_ERR_INVALID_ARG, "X: negative K, S, nnz or J < 1");
  if (X->val_dtype != COPA_VAL_F32 && X->val_dtype != COPA_VAL_F64 && X->val_dtype != COPA_VAL_BF16)
    return fail(h, COPA_ERR_INVALID_ARG, "X: unknown val_dtype");
  if (!X->subj_ptr || !X->row_ptr || (X->nnz > 0 && (!X->col_idx || !X->vals)))
    return fail(h, COPA_ERR_INVALID_ARG, "X: NULL array");
  return COPA_OK;
}

namespace {

constexpr int kBuckets = 2048;

__global__ void k_sched_hist(const int64_t* __restrict__ subj_ptr, int64_t K, int* __restrict__ hist) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += gridDim.x * (int64_t)blockDim.x) {
    int64_t sz = subj_ptr[k + 1] - subj_ptr[k];
    if (sz > kBuckets - 1) sz = kBuckets - 1;
    atomicAdd(hist + (kBuckets - 1 - sz), 1);
  }
}

__global__ void k_sched_scan(int* __restrict__ hist, int* __restrict__ offs) {
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < kBuckets; ++b) { offs[b] = acc; acc += hist[b]; hist[b] = 0; }
  }
}

__global__ void k_sched_scatter(const int64_t* __restrict__ subj_ptr, int64_t K, const int* __restrict__ offs,
                                int* __restrict__ cursor, int64_t* __restrict__ order) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += gridDim.x * (int64_t)blockDim.x) {
    int64_t sz = subj_ptr[k + 1] - subj_ptr[k];
    if (sz > kBuckets - 1) sz = kBuckets - 1;
    const int b = kBuckets - 1 - (int)sz;
    order[offs[b] + atomicAdd(cursor + b, 1)] = k;
  }
}

__global__ void k_validate(TensorView X, int* __restrict__ status) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = gridDim.x * (int64_t)blockDim.x;
  if (tid == 0) {
    if (X.subj_ptr[0] != 0 || X.subj_ptr[X.K] != X.S) set_status(status, 101, 0);
    if (X.row_ptr[0] != 0 || X.row_ptr[X.S] != X.nnz) set_status(status, 102, 0);
  }
  for (int64_t k = tid; k < X.K; k += nt)
    if (X.subj_ptr[k + 1] < X.subj_ptr[k]) set_status(status, 103, (int)k);
  for (int64_t i = tid; i < X.S; i += nt) {
    const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
    if (b < a) { set_status(status, 104, (int)i); continue; }
    for (int64_t t = a; t < b; ++t) {
      const int32_t c = X.col[t];
      if (c < 0 || c >= X.J) set_status(status, 105, (int)i);
      if (t > a && c <= X.col[t - 1]) set_status(status, 106, (int)i);
    }
  }
  if (X.dtype == COPA_VAL_BF16) {
    for (int64_t t = tid; t < X.nnz; t += nt) {
      const float v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X.vals)[t]);
      if (!(fabsf(v) <= 256.0f) || v != rintf(v)) set_status(status, 107, (int)t);
    }
  }
}

// Sets *flag if any byte of a[q] differs from b[q] (q < 4; n[q] bytes each; both
// cudaMalloc'd, hence 16-byte aligned).
struct ByteCmp {
  const unsigned char* a[4];
  const unsigned char* b[4];
  int64_t n[4];
};

__global__ void k_bytes_differ(ByteCmp c, int* __restrict__ flag) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = gridDim.x * (int64_t)blockDim.x;
  bool diff = false;
  for (int q = 0; q < 4; ++q) {
    const int64_t n16 = c.n[q] >> 4;
    const uint4* a = reinterpret_cast<const uint4*>(c.a[q]);
    const uint4* b = reinterpret_cast<const uint4*>(c.b[q]);
    for (int64_t i = tid; i < n16; i += nt) {
      const uint4 x = __ldcs(a + i), y = __ldcs(b + i);
      diff |= (x.x != y.x) | (x.y != y.y) | (x.z != y.z) | (x.w != y.w);
    }
    for (int64_t i = (n16 << 4) + tid; i < c.n[q]; i += nt) diff |= c.a[q][i] != c.b[q][i];
  }
  if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_xnorm2(TensorView X, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < X.nnz; t += gridDim.x * (int64_t)blockDim.x) {
    const double v = load_val(X, t);
    acc += v * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

__global__ void k_warm_sizes(const int64_t* __restrict__ subj_ptr, int64_t K, int R, int64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += gridDim.x * (int64_t)blockDim.x) {
    const int64_t ik = subj_ptr[k + 1] - subj_ptr[k];
    out[k] = ik <= R ? ik * ik : 0;   // tall subjects keep no rotation between iterations
  }
}

// exclusive scan of n values in place into out[0..n] (single block)
__global__ void k_scan_inplace(int64_t* __restrict__ v, int64_t n) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (n + nt - 1) / nt;
  const int64_t a = tid * per, b = min(n, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += v[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int64_t acc = 0;
    for (int i = 0; i < nt; ++i) { const int64_t x = part[i]; part[i] = acc; acc += x; }
    v[n] = acc;
  }
  __syncthreads();
  s = part[tid];
  for (int64_t i = a; i < b; ++i) { const int64_t x = v[i]; v[i] = s; s += x; }
}

// Packs the partial sums of a shard into one FP64 buffer for the all-reduce:
// out = [a (na reals, widened) | b (nb doubles) | c (nc doubles)], and back.
template <typename Real>
__global__ void k_pack_sums(const Real* __restrict__ a, int64_t na, const double* __restrict__ b, int64_t nb,
                            const double* __restrict__ c, int64_t nc, double* __restrict__ out) {
  const int64_t n = na + nb + nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += gridDim.x * (int64_t)blockDim.x)
    out[e] = e < na ? (double)a[e] : (e < na + nb ? b[e - na] : c[e - na - nb]);
}

template <typename Real>
__global__ void k_unpack_sums(const double* __restrict__ in, Real* __restrict__ a, int64_t na, double* __restrict__ b,
                              int64_t nb, double* __restrict__ c, int64_t nc) {
  const int64_t n = na + nb + nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += gridDim.x * (int64_t)blockDim.x) {
    if (e < na) a[e] = (Real)in[e];
    else if (e < na + nb) b[e - na] = in[e];
    else c[e - na - nb] = in[e];
  }
}

// Records the FIT of outer iteration *it, advances the counters and, with eps_fit > 0,
// raises *stop once the FIT changed by at most eps_fit (from the second iteration on).
__global__ void k_store_fit(const double* __restrict__ fit, double* __restrict__ hist, int* __restrict__ it,
                            int* __restrict__ epoch, int* __restrict__ stop, double eps_fit) {
  const int i = *it;
  const double f = *fit;
  hist[i] = f;
  if (eps_fit > 0.0 && i >= 1 && fabs(f - hist[i - 1]) <= eps_fit) *stop = 1;
  *it = i + 1;
  *epoch += 1;
}

// Sets the condition of the conditional node that wraps one outer iteration in the
// replayed graph: run the iteration unless the outer loop has converged.
__global__ void k_cond_set(cudaGraphConditionalHandle ch, const int* __restrict__ stop) {
  cudaGraphSetConditional(ch, *stop ? 0u : 1u);
}

}  // namespace

copa_status_t get_schedule(copa_ctx* h, const TensorView& X, const int64_t** order) {
  copa_status_t st;
  if (h->sched_key == X.subj_ptr && h->sched_K == X.K && h->sched_S == X.S && h->slot_ptr[SLOT_ORDER]) {
    *order = reinterpret_cast<const int64_t*>(h->slot_ptr[SLOT_ORDER]);
    return COPA_OK;
  }
  int64_t* ord = nullptr;
  int* tmp = nullptr;
  if ((st = ws_get(h, SLOT_ORDER, sizeof(int64_t) * (X.K + 1), (void**)&ord)) != COPA_OK) return st;
  if ((st = ws_get(h, SLOT_SCHED_TMP, sizeof(int) * 3 * kBuckets, (void**)&tmp)) != COPA_OK) return st;
  if ((st = cuda_check(h, cudaMemsetAsync(tmp, 0, sizeof(int) * 3 * kBuckets, h->stream), "memset")) != COPA_OK)
    return st;
  if (X.K > 0) {
    const int blocks = (int)std::min<int64_t>((X.K + 255) / 256, 4096);
    k_sched_hist<<<blocks, 256, 0, h->stream>>>(X.subj_ptr, X.K, tmp);
    k_sched_scan<<<1, 32, 0, h->stream>>>(tmp, tmp + kBuckets);
    k_sched_scatter<<<blocks, 256, 0, h->stream>>>(X.subj_ptr, X.K, tmp + kBuckets, tmp, ord);
    if ((st = cuda_check(h, cudaGetLastError(), "schedule kernels")) != COPA_OK) return st;
    h->setup_launches += 3;
  }
  h->sched_key = X.subj_ptr;
  h->sched_K = X.K;
  h->sched_S = X.S;
  *order = ord;
  return COPA_OK;
}

const int* schedule_count_above(copa_ctx* h, int thr) {
  // the scan left offs[b] = number of subjects in buckets before b (bucket b holds I_k =
  // kBuckets - 1 - b), i.e. offs[kBuckets - 1 - thr] subjects have I_k > thr
  return reinterpret_cast<const int*>(h->slot_ptr[SLOT_SCHED_TMP]) + kBuckets + (kBuckets - 1 - thr);
}

copa_status_t get_warm_offsets(copa_ctx* h, const TensorView& X, int R, const int64_t** woff, int64_t* total) {
  copa_status_t st;
  if (h->warm_key == X.subj_ptr && h->warm_K == X.K && h->warm_S == X.S && h->warm_R == R &&
      h->slot_ptr[SLOT_WARM_OFF]) {
    *woff = reinterpret_cast<const int64_t*>(h->slot_ptr[SLOT_WARM_OFF]);
    *total = h->warm_total;
    return COPA_OK;
  }
  int64_t* off = nullptr;
  if ((st = ws_get(h, SLOT_WARM_OFF, sizeof(int64_t) * (X.K + 1), (void**)&off)) != COPA_OK) return st;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.K + 255) / 256, 4096));
  k_warm_sizes<<<blocks, 256, 0, h->stream>>>(X.subj_ptr, X.K, R, off);
  k_scan_inplace<<<1, 1024, 0, h->stream>>>(off, X.K);
  if ((st = cuda_check(h, cudaGetLastError(), "warm offsets")) != COPA_OK) return st;
  h->setup_launches += 2;
  int64_t tot = 0;
  if ((st = cuda_check(h, cudaMemcpyAsync(&tot, off + X.K, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream),
                       "D2H")) != COPA_OK)
    return st;
  if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync")) != COPA_OK) return st;
  h->warm_key = X.subj_ptr;
  h->warm_K = X.K;
  h->warm_S = X.S;
  h->warm_R = R;
  h->warm_total = tot;
  h->warm_valid = false;
  *woff = off;
  *total = tot;
  return COPA_OK;
}

copa_status_t launch_validate(copa_ctx* h, const TensorView& X) {
  const int64_t work = std::max<int64_t>(std::max<int64_t>(X.K, X.S), X.nnz);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)h->num_sms * 8));
  k_validate<<<blocks, 256, 0, h->stream>>>(X, h->d_status);
  return cuda_check(h, cudaGetLastError(), "k_validate");
}

copa_status_t launch_xnorm2(copa_ctx* h, const TensorView& X, double* out) {
  copa_status_t st;
  if ((st = cuda_check(h, cudaMemsetAsync(out, 0, sizeof(double), h->stream), "memset")) != COPA_OK) return st;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.nnz + 255) / 256, (int64_t)h->num_sms * 4));
  k_xnorm2<<<blocks, 256, 0, h->stream>>>(X, out);
  h->setup_launches += 1;
  return cuda_check(h, cudaGetLastError(), "k_xnorm2");
}

// Sum over the shards of a sharded fit (no-op without a registered all-reduce):
// [a (na reals) | b (nb doubles) | c (nc doubles)] are packed into the caller's buffer,
// reduced by the caller's callback and unpacked in place.
template <typename Real>
copa_status_t shard_allreduce(copa_ctx* h, Real* a, int64_t na, double* b, int64_t nb, double* c, int64_t nc) {
  if (!h->red_fn) return COPA_OK;
  const int64_t n = na + nb + nc;
  if (n > h->red_cap) return fail(h, COPA_ERR_INVALID_ARG, "all-reduce buffer too small");
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
  k_pack_sums<Real><<<blocks, 256, 0, h->stream>>>(a, na, b, nb, c, nc, h->red_buf);
  copa_status_t st;
  if ((st = cuda_check(h, cudaGetLastError(), "k_pack_sums")) != COPA_OK) return st;
  const int32_t rc = h->red_fn(h->red_buf, n, reinterpret_cast<void*>(h->stream), h->red_user);
  if (rc != 0) return fail(h, COPA_ERR_COMM, "all-reduce callback returned " + std::to_string(rc));
  k_unpack_sums<Real><<<blocks, 256, 0, h->stream>>>(h->red_buf, a, na, b, nb, c, nc);
  return cuda_check(h, cudaGetLastError(), "k_unpack_sums");
}

}  // namespace copa

// =====================================================================================
// C ABI
// =====================================================================================

static copa_status_t sync_status(copa_ctx* h) {
  copa_status_t st = cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  if (st != COPA_OK) return st;
  int hs[4] = {0, 0, 0, 0};
  if ((st = cuda_check(h, cudaMemcpy(hs, h->d_status, sizeof(hs), cudaMemcpyDeviceToHost), "status read")) != COPA_OK)
    return st;
  if (hs[0] == 0) return COPA_OK;
  cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, h->stream);
  cudaStreamSynchronize(h->stream);
  const int code = hs[0];
  if (code == COPA_ERR_NUMERIC)
    return fail(h, COPA_ERR_NUMERIC, "G + rho I is not positive definite or not finite");
  if (code == COPA_ERR_TIMEOUT)
    return fail(h, COPA_ERR_TIMEOUT,
                std::string("a bounded device wait gave up (site ") + std::to_string(hs[1]) + ")" +
                    (hs[2] == 3 ? "; the work in flight did not finish either: do not use this handle further"
                                : ""));
  static const char* what[] = {"subj_ptr[0] != 0 or subj_ptr[K] != S", "row_ptr[0] != 0 or row_ptr[S] != nnz",
                               "subj_ptr decreases at subject", "row_ptr decreases at row",
                               "column index out of [0, J) in row", "columns not strictly increasing in row",
                               "bf16 value not an integer of magnitude <= 256 at nonzero"};
  if (code >= 101 && code <= 107)
    return fail(h, COPA_ERR_INVALID_ARG, std::string("X invalid: ") + what[code - 101] + " " + std::to_string(hs[1]));
  return fail(h, (copa_status_t)code, "device error " + std::to_string(code) + " info " + std::to_string(hs[1]));
}

#define CHECK_H(h) \
  if (!(h)) return COPA_ERR_INVALID_ARG
#define TRY(x)                           \
  do {                                   \
    copa_status_t _s = (x);              \
    if (_s != COPA_OK) return _s;        \
  } while (0)

static copa_status_t check_R(copa_ctx* h, int R) {
  if (R < 1) return fail(h, COPA_ERR_INVALID_ARG, "R must be >= 1");
  if (R > kMaxR) return fail(h, COPA_ERR_UNSUPPORTED, "R must be <= 96");
  return COPA_OK;
}

static copa_status_t set_dev(copa_ctx* h) { return cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice"); }

extern "C" {

copa_status_t copa_create(copa_handle_t* handle, int device, void* stream, int32_t precision) {
  if (!handle) return COPA_ERR_INVALID_ARG;
  *handle = nullptr;
  if (precision != COPA_PREC_MIXED && precision != COPA_PREC_FP64) return COPA_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return COPA_ERR_CUDA;
  }
  copa_ctx* h = new copa_ctx();
  h->device = device;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->precision = precision;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&h->d_status, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int) * 4) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return COPA_ERR_CUDA;
  }
  *handle = h;
  return COPA_OK;
}

static void release_ctx(copa_ctx* h, bool own_stream) {
  cudaStreamSynchronize(h->stream);
  for (copa_ctx* c : h->children) release_ctx(c, true);
  h->children.clear();
  if (h->batch_ev) cudaEventDestroy(h->batch_ev);
  if (h->pend_exec) cudaGraphExecDestroy(h->pend_exec);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  for (int i = 0; i < 20; ++i)
    if (h->slot_ptr[i]) cudaFree(h->slot_ptr[i]);
  if (h->copy_stream) {   // staged copies still in flight read host memory: end them first
    cudaStreamSynchronize(h->copy_stream);
    cudaStreamDestroy(h->copy_stream);
  }
  for (cudaEvent_t e : h->stage_ev)
    if (e) cudaEventDestroy(e);
  if (h->stage_go) cudaEventDestroy(h->stage_go);
  for (int i = 0; i < copa_ctx::kHostSlots; ++i)
    if (h->host_slot_ptr[i]) cudaFree(h->host_slot_ptr[i]);
  cudaFree(h->d_status);
  if (own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

copa_status_t copa_destroy(copa_handle_t h) {
  CHECK_H(h);
  cudaSetDevice(h->device);
  release_ctx(h, false);
  return COPA_OK;
}

const char* copa_last_error(copa_handle_t h) {
  if (!h) return "invalid handle";
  return h->err.c_str();
}

copa_status_t copa_sync(copa_handle_t h) {
  CHECK_H(h);
  TRY(set_dev(h));
  return sync_status(h);
}

copa_status_t copa_validate(copa_handle_t h, const copa_tensor_t* X) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, X));
  TRY(launch_validate(h, view_of(X)));
  return sync_status(h);
}

copa_status_t copa_forget_tensor(copa_handle_t h) {
  CHECK_H(h);
  TRY(set_dev(h));
  // work already queued may still read the caches: let it finish first
  TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  forget_tensor_caches(h);
  return COPA_OK;
}

copa_status_t copa_procrustes(copa_handle_t h, const copa_tensor_t* X, int32_t R, const void* H,
                              const void* V, const void* W, double tau, copa_procrustes_out_t* out,
                              void* F_H) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, X));
  TRY(check_R(h, R));
  if (!H || !V || !W || !out || !out->Q || !out->T)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_procrustes: NULL H, V, W, Q or T");
  if (!(tau >= 0.0 && tau < 1.0)) return fail(h, COPA_ERR_INVALID_ARG, "tau must be in [0, 1)");
  const TensorView v = view_of(X);
  if (h->precision == COPA_PREC_MIXED)
    return launch_procrustes<float>(h, v, R, (const float*)H, (const float*)V, (const float*)W, tau,
                                    (float*)out->Q, (float*)out->T, (float*)out->Pi, out->rank,
                                    (float*)F_H);
  return launch_procrustes<double>(h, v, R, (const double*)H, (const double*)V, (const double*)W, tau,
                                   (double*)out->Q, (double*)out->T, (double*)out->Pi, out->rank,
                                   (double*)F_H);
}

copa_status_t copa_debug_set(copa_handle_t h, int32_t key, int64_t value) {
  CHECK_H(h);
  if (key == COPA_DEBUG_TC_FORCE_TIMEOUT_NS) {
    if (value < 0 || value > 1000000000LL)
      return fail(h, COPA_ERR_INVALID_ARG, "copa_debug_set: timeout must be in [0, 1e9] ns");
    h->dbg_tc_force_ns = value;
    return COPA_OK;
  }
  return fail(h, COPA_ERR_INVALID_ARG, "copa_debug_set: unknown key");
}

copa_status_t copa_fit_launches(copa_handle_t h, int64_t* launches_host) {
  CHECK_H(h);
  if (!launches_host) return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_launches: NULL output");
  *launches_host = h->fit_launches;
  return COPA_OK;
}

copa_status_t copa_procrustes_work(copa_handle_t h, double* fma_host) {
  CHECK_H(h);
  TRY(set_dev(h));
  if (!fma_host) return fail(h, COPA_ERR_INVALID_ARG, "copa_procrustes_work: NULL output");
  *fma_host = 0.0;
  if (!h->slot_ptr[SLOT_COUNTER]) return COPA_OK;
  TRY(sync_status(h));
  unsigned long long v = 0;
  TRY(cuda_check(h, cudaMemcpy(&v, reinterpret_cast<char*>(h->slot_ptr[SLOT_COUNTER]) + 8, sizeof(v),
                               cudaMemcpyDeviceToHost), "counter read"));
  *fma_host = (double)v;
  return COPA_OK;
}

copa_status_t copa_mttkrp(copa_handle_t h, int32_t mode, const copa_tensor_t* X, int32_t R,
                          const copa_procrustes_out_t* st, const void* H, const void* W, void* F,
                          double* UtU) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_R(h, R));
  if (!st || !F) return fail(h, COPA_ERR_INVALID_ARG, "copa_mttkrp: NULL state or F");
  const bool mixed = h->precision == COPA_PREC_MIXED;
  if (mode == COPA_MODE_H) {
    if (!X || !st->T || !W) return fail(h, COPA_ERR_INVALID_ARG, "copa_mttkrp(H): needs X (for K), T, W");
    if (mixed) return launch_mttkrp_h<float>(h, X->K, R, (const float*)st->T, (const float*)W, (float*)F);
    return launch_mttkrp_h<double>(h, X->K, R, (const double*)st->T, (const double*)W, (double*)F);
  }
  if (mode == COPA_MODE_W) {
    if (!X || !st->T || !H) return fail(h, COPA_ERR_INVALID_ARG, "copa_mttkrp(W): needs X (for K), T, H");
    if (mixed) return launch_mttkrp_w<float>(h, X->K, R, (const float*)st->T, (const float*)H, (float*)F);
    return launch_mttkrp_w<double>(h, X->K, R, (const double*)st->T, (const double*)H, (double*)F);
  }
  if (mode == COPA_MODE_V) {
    TRY(check_tensor_args(h, X));
    if (!st->Q || !H || !W) return fail(h, COPA_ERR_INVALID_ARG, "copa_mttkrp(V): needs Q, H, W");
    const TensorView v = view_of(X);
    if (mixed)
      return launch_mttkrp_v<float>(h, v, R, (const float*)st->Q, (const float*)H, (const float*)W, (float*)F, UtU);
    return launch_mttkrp_v<double>(h, v, R, (const double*)st->Q, (const double*)H, (const double*)W, (double*)F,
                                   UtU);
  }
  return fail(h, COPA_ERR_INVALID_ARG, "copa_mttkrp: mode must be 0 (H), 1 (V) or 2 (W)");
}

copa_status_t copa_gram(copa_handle_t h, const void* A, int64_t rows, int32_t R, double* G) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_R(h, R));
  if (!A || !G || rows < 0) return fail(h, COPA_ERR_INVALID_ARG, "copa_gram: bad arguments");
  if (h->precision == COPA_PREC_MIXED) return launch_gram<float>(h, (const float*)A, rows, R, G);
  return launch_gram<double>(h, (const double*)A, rows, R, G);
}

static copa_status_t check_admm(copa_ctx* h, int n_inner, int c, double lam, int R) {
  TRY(check_R(h, R));
  if (n_inner < 0) return fail(h, COPA_ERR_INVALID_ARG, "n_inner must be >= 0");
  if (c < COPA_C_NONE || c > COPA_C_L0) return fail(h, COPA_ERR_INVALID_ARG, "unknown constraint");
  if (!(lam >= 0.0)) return fail(h, COPA_ERR_INVALID_ARG, "lambda must be >= 0");
  return COPA_OK;
}

copa_status_t copa_admm_step(copa_handle_t h, const void* F, const double* Ga, const double* Gb,
                             int32_t n_inner, int32_t c, double lambda, void* Zbar, void* D,
                             int64_t rows, int32_t R, double* rho_out) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_admm(h, n_inner, c, lambda, R));
  if (!F || !Ga || !Zbar || !D || rows < 0) return fail(h, COPA_ERR_INVALID_ARG, "copa_admm_step: bad arguments");
  void* ginv = nullptr;
  TRY(ws_get(h, SLOT_GINV, sizeof(double) * ((size_t)R * (R + 1) + 2), &ginv));
  double* rho = rho_out ? rho_out : reinterpret_cast<double*>(ginv) + (size_t)R * (R + 1);
  if (h->precision == COPA_PREC_MIXED) {
    TRY(launch_chol<float>(h, Ga, Gb, R, (float*)ginv, rho));
    return launch_admm_rows<float>(h, (const float*)F, (const float*)ginv, rho, n_inner, c, lambda,
                                   (float*)Zbar, (float*)D, rows, R);
  }
  TRY(launch_chol<double>(h, Ga, Gb, R, (double*)ginv, rho));
  return launch_admm_rows<double>(h, (const double*)F, (const double*)ginv, rho, n_inner, c, lambda,
                                  (double*)Zbar, (double*)D, rows, R);
}

copa_status_t copa_admm_w_fused(copa_handle_t h, const copa_procrustes_out_t* st, const void* H,
                                const double* Ga, const double* Gb, int32_t n_inner, int32_t c,
                                double lambda, void* Wbar, void* DW, int64_t K, int32_t R,
                                double* rho_out) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_admm(h, n_inner, c, lambda, R));
  if (!st || !st->T || !H || !Ga || !Wbar || !DW || K < 0)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_admm_w_fused: bad arguments");
  void* ginv = nullptr;
  TRY(ws_get(h, SLOT_GINV, sizeof(double) * ((size_t)R * (R + 1) + 2), &ginv));
  double* rho = rho_out ? rho_out : reinterpret_cast<double*>(ginv) + (size_t)R * (R + 1);
  if (h->precision == COPA_PREC_MIXED) {
    TRY(launch_chol<float>(h, Ga, Gb, R, (float*)ginv, rho));
    return launch_admm_w<float>(h, (const float*)st->T, (const float*)H, (const float*)ginv, rho, n_inner,
                                c, lambda, (float*)Wbar, (float*)DW, K, R);
  }
  TRY(launch_chol<double>(h, Ga, Gb, R, (double*)ginv, rho));
  return launch_admm_w<double>(h, (const double*)st->T, (const double*)H, (const double*)ginv, rho, n_inner,
                               c, lambda, (double*)Wbar, (double*)DW, K, R);
}

copa_status_t copa_fit_value(copa_handle_t h, const copa_tensor_t* X, int32_t R, const void* V,
                             const void* F_V, const double* UtU, double x_norm2, double* fit) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, X));
  TRY(check_R(h, R));
  if (!V || !F_V || !UtU || !fit) return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_value: NULL argument");
  double* xn2 = nullptr;
  TRY(ws_get(h, SLOT_PI, sizeof(double) * (4 + (size_t)R * R), (void**)&xn2));
  const TensorView v = view_of(X);
  TRY(launch_xnorm2(h, v, xn2));
  if (h->precision == COPA_PREC_MIXED)
    return launch_fit_value<float>(h, X->J, R, (const float*)V, (const float*)F_V, UtU, xn2, x_norm2, fit,
                                   xn2 + 4);
  return launch_fit_value<double>(h, X->J, R, (const double*)V, (const double*)F_V, UtU, xn2, x_norm2, fit,
                                  xn2 + 4);
}

}  // extern "C"

// =====================================================================================
// Whole outer iterations
// =====================================================================================

namespace {

template <typename Real>
struct FitBufs {
  Real* Uw;
  const int64_t* woff;
  int* epoch;   // outer iterations since the warm-start buffer was laid out (schedules re-orthonormalisation)
  Real* Q;
  Real* T;
  Real* Pi;
  int32_t* rank;
  Real* FH;
  Real* FV;
  Real* Ginv;
  double* gH;
  double* gV;
  double* gW;
  double* UtU;
  double* rho;
  double* xn2;
  double* fitv;
  double* hist;
  int* it;
  int* stop;      // outer loop converged (eps_fit)
  int* counts;    // int[3 * n_outer]: inner iterations run for H, W, V
  int* done;      // inner loop converged (eps_inner), per mode
  double* acc;    // residual sums of the current inner iteration
  Real* FW;       // F_W (K x R) for the early-stopping W update
};

template <typename Real>
copa_status_t one_iteration(copa_ctx* h, const TensorView& X, const copa_options_t* o, Real* H, Real* V,
                            Real* W, Real* DH, Real* DV, Real* DW, const FitBufs<Real>& b, bool warm_in,
                            bool first) {
  const int R = o->R;
  // (a)+(b) Procrustes, with the H-mode MTTKRP fused
  TRY(launch_procrustes<Real>(h, X, R, H, V, W, o->tau, b.Q, b.T, b.Pi, b.rank, b.FH, b.Uw, b.woff, warm_in,
                              b.epoch));
  // H: G = W^T W .* V^T V (V^T V of the current V is left by the previous iteration's FIT
  // within one copa_fit call)
  TRY(launch_gram<Real>(h, W, X.K, R, b.gW));
  if (first) TRY(launch_gram<Real>(h, V, X.J, R, b.gV));
  // sharded fit: F_H and W^T W summed over the shards (H is then updated identically)
  TRY(shard_allreduce<Real>(h, b.FH, (int64_t)R * R, b.gW, (int64_t)R * R, nullptr, 0));
  const bool adaptive = o->eps_inner > 0.0;
  TRY(launch_chol<Real>(h, b.gW, b.gV, R, b.Ginv, b.rho + 0));
  if (adaptive)
    TRY(launch_admm_adaptive<Real>(h, b.FH, b.Ginv, b.rho + 0, o->n_inner, o->c_H, o->lam_H, H, DH, R, R,
                                   o->eps_inner, b.acc, b.done, b.counts, b.it, 0));
  else
    TRY(launch_admm_rows<Real>(h, b.FH, b.Ginv, b.rho + 0, o->n_inner, o->c_H, o->lam_H, H, DH, R, R));
  // W: G = H^T H .* V^T V, F_W fused into the ADMM (or computed first for early stopping,
  // whose residual test needs every row after each iteration)
  TRY(launch_gram<Real>(h, H, R, R, b.gH));
  TRY(launch_chol<Real>(h, b.gH, b.gV, R, b.Ginv, b.rho + 1));
  if (adaptive) {
    TRY(launch_mttkrp_w<Real>(h, X.K, R, b.T, H, b.FW));
    TRY(launch_admm_adaptive<Real>(h, b.FW, b.Ginv, b.rho + 1, o->n_inner, o->c_W, o->lam_W, W, DW, X.K, R,
                                   o->eps_inner, b.acc, b.done, b.counts, b.it, 1));
  } else {
    TRY(launch_admm_w<Real>(h, b.T, H, b.Ginv, b.rho + 1, o->n_inner, o->c_W, o->lam_W, W, DW, X.K, R));
  }
  // V: G = H^T H .* W^T W; F_V = sum_k X_k^T Q_k H S_k
  TRY(launch_gram<Real>(h, W, X.K, R, b.gW));
  TRY(launch_mttkrp_v<Real>(h, X, R, b.Q, H, W, b.FV, b.UtU, /*reuse_csc=*/!first));
  // sharded fit: F_V, W^T W and U^T U summed over the shards (V is then updated identically)
  TRY(shard_allreduce<Real>(h, b.FV, (int64_t)X.J * R, b.gW, (int64_t)R * R, b.UtU, (int64_t)R * R));
  TRY(launch_chol<Real>(h, b.gH, b.gW, R, b.Ginv, b.rho + 2));
  if (adaptive)
    TRY(launch_admm_adaptive<Real>(h, b.FV, b.Ginv, b.rho + 2, o->n_inner, o->c_V, o->lam_V, V, DV, X.J, R,
                                   o->eps_inner, b.acc, b.done, b.counts, b.it, 2));
  else
    TRY(launch_admm_rows<Real>(h, b.FV, b.Ginv, b.rho + 2, o->n_inner, o->c_V, o->lam_V, V, DV, X.J, R));
  // FIT of (Q_k, H, W, V) after the iteration
  TRY(launch_fit_value<Real>(h, X.J, R, V, b.FV, b.UtU, b.xn2, o->x_norm2, b.fitv, b.gV));
  k_store_fit<<<1, 1, 0, h->stream>>>(b.fitv, b.hist, b.it, b.epoch, b.stop, o->eps_fit);
  return cuda_check(h, cudaGetLastError(), "k_store_fit");
}

// Waits for the fit enqueued last on this handle and collects its results: the device
// status, the iteration counts (copa_fit_stats) and the FIT history.
copa_status_t finish_fit(copa_ctx* h, double* hist_host) {
  const copa_status_t sst = sync_status(h);
  if (h->pend_exec) {
    cudaGraphExecDestroy(h->pend_exec);
    h->pend_exec = nullptr;
  }
  TRY(sst);
  const int n_outer = h->pend_n_outer;
  int32_t n_run = 0;
  if (n_outer > 0) TRY(cuda_check(h, cudaMemcpy(&n_run, h->pend_it, sizeof(int), cudaMemcpyDeviceToHost), "D2H"));
  h->last_n_run = n_run;
  h->last_inner.assign(3 * (size_t)std::max(0, n_outer), 0);
  if (h->pend_adaptive && n_outer > 0) {
    TRY(cuda_check(h, cudaMemcpy(h->last_inner.data(), h->pend_counts, sizeof(int) * 3 * n_outer,
                                 cudaMemcpyDeviceToHost), "D2H"));
  } else {
    for (int i = 0; i < 3 * n_run; ++i) h->last_inner[i] = h->pend_n_inner;
  }
  if (h->pend_per_iter >= 0) h->fit_launches = h->setup_launches + h->pend_per_iter * n_outer;
  if (hist_host && n_outer > 0) {
    TRY(cuda_check(h, cudaMemcpy(hist_host, h->pend_hist, sizeof(double) * n_run, cudaMemcpyDeviceToHost),
                   "history D2H"));
    for (int i = n_run; i < n_outer; ++i) hist_host[i] = std::numeric_limits<double>::quiet_NaN();
  }
  return COPA_OK;
}

// Enqueues a whole fit on h->stream (set-up, the first iteration eagerly, the others as
// graph replays) and, if finish, waits for it (finish_fit). Without finish the results
// are collected by a later finish_fit on the same handle.
template <typename Real>
copa_status_t fit_impl(copa_ctx* h, const copa_tensor_t* Xc, const copa_options_t* o, Real* H, Real* V,
                       Real* W, Real* DH, Real* DV, Real* DW, double* hist_host, copa_procrustes_out_t* st,
                       bool finish = true) {
  const TensorView X = view_of(Xc);
  const int R = o->R;
  const size_t KRR = (size_t)X.K * R * R;
  FitBufs<Real> b{};
  if (st && st->Q && st->T) {
    b.Q = (Real*)st->Q;
    b.T = (Real*)st->T;
    b.Pi = (Real*)st->Pi;
    b.rank = st->rank;
  } else {
    TRY(ws_get(h, SLOT_FIT_Q, sizeof(Real) * (size_t)X.S * R + 16, (void**)&b.Q));
    TRY(ws_get(h, SLOT_FIT_T, sizeof(Real) * KRR, (void**)&b.T));
  }
  auto rnd = [](size_t bytes) { return (bytes + 255) & ~size_t(255); };
  const size_t nsmall = 4 * rnd(sizeof(double) * R * R) + rnd(sizeof(double) * 4) + 2 * rnd(sizeof(double)) +
                        rnd(sizeof(double) * std::max(1, o->n_outer)) + rnd(sizeof(int)) +
                        rnd(sizeof(Real) * R * R) + rnd(sizeof(Real) * (size_t)X.J * R) +
                        rnd(sizeof(Real) * R * (R + 1)) + 2 * rnd(sizeof(int)) +
                        rnd(sizeof(int) * 3 * std::max(1, o->n_outer)) + rnd(sizeof(double) * 4);
  char* p = nullptr;
  TRY(ws_get(h, SLOT_FIT_SMALL, nsmall, (void**)&p));
  auto take = [&](size_t bytes) {
    char* r = p;
    p += rnd(bytes);
    return r;
  };
  b.gH = (double*)take(sizeof(double) * R * R);
  b.gV = (double*)take(sizeof(double) * R * R);
  b.gW = (double*)take(sizeof(double) * R * R);
  b.UtU = (double*)take(sizeof(double) * R * R);
  b.rho = (double*)take(sizeof(double) * 4);
  b.xn2 = (double*)take(sizeof(double));
  b.fitv = (double*)take(sizeof(double));
  b.hist = (double*)take(sizeof(double) * std::max(1, o->n_outer));
  b.it = (int*)take(sizeof(int));
  b.FH = (Real*)take(sizeof(Real) * R * R);
  b.FV = (Real*)take(sizeof(Real) * (size_t)X.J * R);
  b.Ginv = (Real*)take(sizeof(Real) * R * (R + 1));
  b.stop = (int*)take(sizeof(int));
  b.done = (int*)take(sizeof(int));
  b.counts = (int*)take(sizeof(int) * 3 * std::max(1, o->n_outer));
  b.acc = (double*)take(sizeof(double) * 4);
  b.FW = nullptr;
  if (o->eps_inner > 0.0) TRY(ws_get(h, SLOT_FIT_FW, sizeof(Real) * (size_t)std::max<int64_t>(X.K, 1) * R,
                                     (void**)&b.FW));
  TRY(cuda_check(h, cudaMemsetAsync(b.stop, 0, sizeof(int), h->stream), "memset"));
  TRY(cuda_check(h, cudaMemsetAsync(b.counts, 0, sizeof(int) * 3 * std::max(1, o->n_outer), h->stream), "memset"));
  h->fit_launches = -1;
  h->setup_launches = 0;
  int64_t per_iter = -1;
  TRY(cuda_check(h, cudaMemsetAsync(b.it, 0, sizeof(int), h->stream), "memset"));
  TRY(launch_xnorm2(h, X, b.xn2));
  if (h->red_fn) {
    if (h->red_cap < (int64_t)X.J * R + 2 * (int64_t)R * R)
      return fail(h, COPA_ERR_INVALID_ARG, "all-reduce buffer smaller than J * R + 2 R^2 doubles");
    TRY(shard_allreduce<Real>(h, (Real*)nullptr, 0, b.xn2, 1, nullptr, 0));
  }
  {
    int64_t wtot = 0;
    TRY(get_warm_offsets(h, X, R, &b.woff, &wtot));
    const size_t ub = (sizeof(Real) * (size_t)(wtot + 1) + 15) & ~size_t(15);
    TRY(ws_get(h, SLOT_WARM, ub + 16, (void**)&b.Uw));
    b.epoch = reinterpret_cast<int*>(reinterpret_cast<char*>(b.Uw) + ub);
    if (!(h->warm_valid && h->warm_prec == h->precision))
      TRY(cuda_check(h, cudaMemsetAsync(b.epoch, 0, sizeof(int), h->stream), "memset"));
  }
  if (o->n_outer > 0) {
    // the first iteration runs eagerly: it sizes every workspace buffer
    TRY(one_iteration<Real>(h, X, o, H, V, W, DH, DV, DW, b, h->warm_valid && h->warm_prec == h->precision, true));
    h->warm_valid = true;
    h->warm_prec = h->precision;
  }
  if (o->n_outer > 1) {
    if (o->use_graph && !h->red_fn) {
      // Capture on a private stream (the caller's may be the legacy default stream, which
      // cannot be captured); capturing enqueues nothing, the replays go to h->stream. With
      // eps_fit > 0 the iteration is the body of a conditional (if) node whose condition a
      // small kernel sets from the device's stop flag before it, so that the replays after
      // convergence do nothing and the host never waits.
      const bool cond = o->eps_fit > 0.0;
      cudaGraph_t graph = nullptr, body = nullptr;
      cudaStream_t orig = h->stream, cap = nullptr;
      TRY(cuda_check(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate"));
      cudaError_t ce = cudaSuccess;
      if (cond) {
        cudaGraphConditionalHandle ch = 0;
        ce = cudaGraphCreate(&graph, 0);
        if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&ch, graph, 1, 0);
        if (ce == cudaSuccess) ce = cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0,
                                                                  cudaStreamCaptureModeRelaxed);
        if (ce == cudaSuccess) {
          k_cond_set<<<1, 1, 0, cap>>>(ch, b.stop);
          ce = cudaGetLastError();
          cudaGraph_t g2 = nullptr;
          const cudaError_t ce2 = cudaStreamEndCapture(cap, &g2);
          if (ce == cudaSuccess) ce = ce2;
        }
        cudaGraphNode_t kn = nullptr;
        size_t nk = 1;
        if (ce == cudaSuccess) ce = cudaGraphGetNodes(graph, &kn, &nk);
        if (ce == cudaSuccess && nk != 1) ce = cudaErrorUnknown;
        if (ce == cudaSuccess) {
          cudaGraphNodeParams cp = {};
          cp.type = cudaGraphNodeTypeConditional;
          cp.conditional.handle = ch;
          cp.conditional.type = cudaGraphCondTypeIf;
          cp.conditional.size = 1;
          cudaGraphNode_t cn = nullptr;
          ce = cudaGraphAddNode(&cn, graph, &kn, nullptr, 1, &cp);
          if (ce == cudaSuccess) body = cp.conditional.phGraph_out[0];
        }
        if (ce == cudaSuccess)
          ce = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      } else {
        ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
      }
      copa_status_t cs = COPA_OK;
      if (ce == cudaSuccess) {
        h->stream = cap;
        cs = one_iteration<Real>(h, X, o, H, V, W, DH, DV, DW, b, true, false);
        h->stream = orig;
        cudaGraph_t got = nullptr;
        ce = cudaStreamEndCapture(cap, &got);
        if (!cond) graph = got;
        else body = got;
      }
      cudaStreamDestroy(cap);
      if (cs != COPA_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (cs != COPA_OK) return cs;
        TRY(cuda_check(h, ce, "graph capture"));
      }
      {
        cudaGraph_t counted = cond ? body : graph;
        size_t nn = 0;
        if (cudaGraphGetNodes(counted, nullptr, &nn) == cudaSuccess && nn > 0) {
          std::vector<cudaGraphNode_t> nodes(nn);
          if (cudaGraphGetNodes(counted, nodes.data(), &nn) == cudaSuccess) {
            per_iter = cond ? 1 : 0;
            for (size_t q = 0; q < nn; ++q) {
              cudaGraphNodeType ty;
              if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++per_iter;
            }
          }
        }
      }
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      TRY(cuda_check(h, ce, "GraphInstantiate"));
      for (int it = 1; it < o->n_outer; ++it) {
        ce = cudaGraphLaunch(exec, h->stream);
        if (ce != cudaSuccess) break;
      }
      // destroyed by finish_fit once the stream has drained (the launches stay in flight
      // meanwhile, so that fits on other streams can be enqueued behind them)
      h->pend_exec = exec;
      TRY(cuda_check(h, ce, "GraphLaunch"));
    } else {
      for (int it = 1; it < o->n_outer; ++it) {
        if (o->eps_fit > 0.0) {   // the eager loop asks the device whether to go on
          int stop = 0;
          TRY(cuda_check(h, cudaMemcpyAsync(&stop, b.stop, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "D2H"));
          TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
          if (stop) break;
        }
        TRY(one_iteration<Real>(h, X, o, H, V, W, DH, DV, DW, b, true, false));
      }
    }
  }
  h->pend_it = b.it;
  h->pend_hist = b.hist;
  h->pend_counts = b.counts;
  h->pend_n_outer = o->n_outer;
  h->pend_n_inner = o->n_inner;
  h->pend_adaptive = o->eps_inner > 0.0;
  h->pend_per_iter = per_iter;
  if (!finish) return COPA_OK;
  return finish_fit(h, hist_host);
}

copa_status_t check_options(copa_ctx* h, const copa_options_t* o) {
  if (!o) return fail(h, COPA_ERR_INVALID_ARG, "options NULL");
  TRY(check_R(h, o->R));
  if (o->n_outer < 0 || o->n_inner < 0) return fail(h, COPA_ERR_INVALID_ARG, "negative iteration count");
  for (int c : {o->c_H, o->c_W, o->c_V})
    if (c < COPA_C_NONE || c > COPA_C_L0) return fail(h, COPA_ERR_INVALID_ARG, "unknown constraint");
  if (!(o->lam_H >= 0 && o->lam_W >= 0 && o->lam_V >= 0)) return fail(h, COPA_ERR_INVALID_ARG, "negative lambda");
  if (!(o->tau >= 0.0 && o->tau < 1.0)) return fail(h, COPA_ERR_INVALID_ARG, "tau must be in [0, 1)");
  if (!(o->eps_inner >= 0.0) || !(o->eps_fit >= 0.0))
    return fail(h, COPA_ERR_INVALID_ARG, "eps_inner and eps_fit must be >= 0");
  if (h->red_fn && o->eps_inner > 0.0)
    return fail(h, COPA_ERR_UNSUPPORTED,
                "eps_inner in a sharded fit (the W residuals would need an all-reduce per inner iteration)");
  return COPA_OK;
}

}  // namespace

extern "C" {

copa_status_t copa_fit(copa_handle_t h, const copa_tensor_t* X, const copa_options_t* opt, void* H, void* V,
                       void* W, void* DH, void* DV, void* DW, double* fit_history_host,
                       copa_procrustes_out_t* st) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, X));
  TRY(check_options(h, opt));
  if (!H || !V || !W || !DH || !DV || !DW) return fail(h, COPA_ERR_INVALID_ARG, "copa_fit: NULL factor or dual");
  if (h->precision == COPA_PREC_MIXED)
    return fit_impl<float>(h, X, opt, (float*)H, (float*)V, (float*)W, (float*)DH, (float*)DV, (float*)DW,
                           fit_history_host, st);
  return fit_impl<double>(h, X, opt, (double*)H, (double*)V, (double*)W, (double*)DH, (double*)DV, (double*)DW,
                          fit_history_host, st);
}

copa_status_t copa_fit_batch(copa_handle_t h, const copa_tensor_t* X, int32_t G, const copa_options_t* opts,
                             void* const* H, void* const* V, void* const* W, void* const* DH, void* const* DV,
                             void* const* DW, double* fit_history_host) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, X));
  if (G < 1 || G > 64 || !opts || !H || !V || !W || !DH || !DV || !DW)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_batch: need 1 <= G <= 64 and non-NULL arrays");
  if (h->red_fn) return fail(h, COPA_ERR_UNSUPPORTED, "copa_fit_batch: not for a shard of a sharded fit");
  for (int g = 0; g < G; ++g) {
    TRY(check_options(h, &opts[g]));
    if (opts[g].R != opts[0].R || opts[g].n_outer != opts[0].n_outer)
      return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_batch: every fit must have the same R and n_outer");
    if (!H[g] || !V[g] || !W[g] || !DH[g] || !DV[g] || !DW[g])
      return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_batch: NULL factor or dual");
  }
  while ((int)h->children.size() < G) {
    copa_ctx* c = new copa_ctx();
    c->device = h->device;
    c->precision = h->precision;
    c->num_sms = h->num_sms;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&c->d_status, sizeof(int) * 4) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int) * 4) != cudaSuccess) {
      cudaGetLastError();
      if (c->stream) cudaStreamDestroy(c->stream);
      if (c->d_status) cudaFree(c->d_status);
      delete c;
      return fail(h, COPA_ERR_CUDA, "copa_fit_batch: could not create a stream for a fit");
    }
    h->children.push_back(c);
  }
  if (!h->batch_ev) TRY(cuda_check(h, cudaEventCreateWithFlags(&h->batch_ev, cudaEventDisableTiming), "event"));
  for (int g = 0; g < G; ++g) h->children[g]->num_sms = h->num_sms;
  // every fit starts after the work already queued on the handle's stream
  TRY(cuda_check(h, cudaEventRecord(h->batch_ev, h->stream), "cudaEventRecord"));
  for (int g = 0; g < G; ++g)
    TRY(cuda_check(h, cudaStreamWaitEvent(h->children[g]->stream, h->batch_ev, 0), "cudaStreamWaitEvent"));
  const bool mixed = h->precision == COPA_PREC_MIXED;
  copa_status_t first = COPA_OK;
  int enq = 0;
  for (; enq < G; ++enq) {
    copa_ctx* c = h->children[enq];
    const copa_status_t st =
        mixed ? fit_impl<float>(c, X, &opts[enq], (float*)H[enq], (float*)V[enq], (float*)W[enq], (float*)DH[enq],
                                (float*)DV[enq], (float*)DW[enq], nullptr, nullptr, false)
              : fit_impl<double>(c, X, &opts[enq], (double*)H[enq], (double*)V[enq], (double*)W[enq],
                                 (double*)DH[enq], (double*)DV[enq], (double*)DW[enq], nullptr, nullptr, false);
    if (st != COPA_OK) {
      first = fail(h, st, "copa_fit_batch: fit " + std::to_string(enq) + ": " + c->err);
      break;
    }
  }
  // collect every enqueued fit (also after an error, so that nothing is left running)
  for (int g = 0; g < enq; ++g) {
    copa_ctx* c = h->children[g];
    const copa_status_t st =
        finish_fit(c, fit_history_host ? fit_history_host + (size_t)g * std::max(0, opts[0].n_outer) : nullptr);
    if (st != COPA_OK && first == COPA_OK) first = fail(h, st, "copa_fit_batch: fit " + std::to_string(g) + ": " + c->err);
  }
  // later work on the handle's stream sees the fits' results
  for (int g = 0; g < enq; ++g) {
    TRY(cuda_check(h, cudaEventRecord(h->batch_ev, h->children[g]->stream), "cudaEventRecord"));
    TRY(cuda_check(h, cudaStreamWaitEvent(h->stream, h->batch_ev, 0), "cudaStreamWaitEvent"));
  }
  return first;
}

copa_status_t copa_fit_stats(copa_handle_t h, int32_t* n_outer_run_host, int32_t* inner_host) {
  CHECK_H(h);
  if (!n_outer_run_host) return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_stats: NULL output");
  *n_outer_run_host = h->last_n_run;
  if (inner_host)
    for (size_t i = 0; i < h->last_inner.size(); ++i) inner_host[i] = h->last_inner[i];
  return COPA_OK;
}

copa_status_t copa_partition(const int64_t* subj_ptr, const int64_t* row_ptr, int64_t K, int32_t nshards,
                             int64_t* bounds) {
  if (!subj_ptr || !row_ptr || !bounds || K < 0 || nshards < 1) return COPA_ERR_INVALID_ARG;
  // nonzero prefix at subject boundary k: row_ptr[subj_ptr[k]] (non-decreasing in k)
  auto pre = [&](int64_t k) { return row_ptr[subj_ptr[k]]; };
  const int64_t N = pre(K);
  bounds[0] = 0;
  bounds[nshards] = K;
  int64_t lo = 0;
  for (int32_t p = 1; p < nshards; ++p) {
    // target p * N / nshards without overflow
    const long double target = (long double)N * p / nshards;
    int64_t a = lo, b = K;   // smallest k in [lo, K] with pre(k) >= target
    while (a < b) {
      const int64_t m = a + (b - a) / 2;
      if ((long double)pre(m) >= target) b = m;
      else a = m + 1;
    }
    int64_t k = a;
    if (k > lo && target - (long double)pre(k - 1) < (long double)pre(k) - target) k -= 1;
    bounds[p] = k;
    lo = k;
  }
  return COPA_OK;
}

copa_status_t copa_set_allreduce(copa_handle_t h, copa_allreduce_fn fn, void* user, double* buf, int64_t capacity) {
  CHECK_H(h);
  if (fn && (!buf || capacity < 1)) return fail(h, COPA_ERR_INVALID_ARG, "copa_set_allreduce: NULL buffer");
  h->red_fn = fn;
  h->red_user = fn ? user : nullptr;
  h->red_buf = fn ? buf : nullptr;
  h->red_cap = fn ? capacity : 0;
  return COPA_OK;
}

namespace {

// Bytes of the four arrays of a tensor (subj_ptr, row_ptr, col_idx, vals).
void tensor_bytes(const copa_tensor_t* X, size_t out[4]) {
  const size_t vs = X->val_dtype == COPA_VAL_F64 ? 8 : (X->val_dtype == COPA_VAL_F32 ? 4 : 2);
  out[0] = sizeof(int64_t) * (X->K + 1);
  out[1] = sizeof(int64_t) * (X->S + 1);
  out[2] = sizeof(int32_t) * X->nnz;
  out[3] = vs * X->nnz;
}

// Device buffer of at least `bytes` (+16) in host slot i; a smaller one is replaced.
copa_status_t host_slot(copa_ctx* h, int i, size_t bytes) {
  if (h->host_slot_bytes[i] < bytes + 16) {
    if (h->host_slot_ptr[i]) cudaFree(h->host_slot_ptr[i]);
    h->host_slot_ptr[i] = nullptr;
    h->host_slot_bytes[i] = 0;
    if (cudaMalloc(&h->host_slot_ptr[i], bytes + 16) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, COPA_ERR_OOM, "device allocation for the copies of host arrays failed");
    }
    h->host_slot_bytes[i] = bytes + 16;
  }
  return COPA_OK;
}

bool staged_matches(const copa_ctx::StagedX& s, const copa_tensor_t* X) {
  return s.K == X->K && s.J == X->J && s.S == X->S && s.nnz == X->nnz && s.vdt == X->val_dtype &&
         s.src[0] == X->subj_ptr && s.src[1] == X->row_ptr && s.src[2] == X->col_idx && s.src[3] == X->vals;
}

// Waits for every pending staged copy that was issued and forgets them all (their buffers
// stay allocated).
copa_status_t drop_staged(copa_ctx* h) {
  for (int q = 0; q < h->n_staged; ++q)
    if (h->staged[q].issued)
      TRY(cuda_check(h, cudaEventSynchronize(h->stage_ev[h->staged[q].set]), "cudaEventSynchronize"));
  h->n_staged = 0;
  return COPA_OK;
}

// Issues the copies of the pending staged tensors not issued yet, on the copy stream after
// the work queued so far on the handle's stream (a copa_fit_host call's own copies), so
// that they take the host link after those and run beside the call's kernels.
copa_status_t issue_staged(copa_ctx* h) {
  bool first = true;
  for (int q = 0; q < h->n_staged; ++q) {
    copa_ctx::StagedX& e = h->staged[q];
    if (e.issued) continue;
    if (first) {
      TRY(cuda_check(h, cudaEventRecord(h->stage_go, h->stream), "cudaEventRecord"));
      TRY(cuda_check(h, cudaStreamWaitEvent(h->copy_stream, h->stage_go, 0), "cudaStreamWaitEvent"));
      first = false;
    }
    const size_t vs = e.vdt == COPA_VAL_F64 ? 8 : (e.vdt == COPA_VAL_F32 ? 4 : 2);
    const size_t sizes[4] = {sizeof(int64_t) * (e.K + 1), sizeof(int64_t) * (e.S + 1), sizeof(int32_t) * e.nnz,
                             vs * e.nnz};
    for (int i = 0; i < 4; ++i)
      if (sizes[i])
        TRY(cuda_check(h, cudaMemcpyAsync(h->host_slot_ptr[15 + 4 * e.set + i], e.src[i], sizes[i],
                                          cudaMemcpyHostToDevice, h->copy_stream),
                       "H2D"));
    TRY(cuda_check(h, cudaEventRecord(h->stage_ev[e.set], h->copy_stream), "cudaEventRecord"));
    e.issued = true;
  }
  return COPA_OK;
}

}  // namespace

copa_status_t copa_stage_host(copa_handle_t h, const copa_tensor_t* Xh) {
  CHECK_H(h);
  TRY(set_dev(h));
  TRY(check_tensor_args(h, Xh));
  if (h->n_staged >= 2) return fail(h, COPA_ERR_INVALID_ARG, "copa_stage_host: two copies are queued already");
  if (!h->copy_stream)
    TRY(cuda_check(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate"));
  if (!h->stage_go)
    TRY(cuda_check(h, cudaEventCreateWithFlags(&h->stage_go, cudaEventDisableTiming), "cudaEventCreate"));
  // the set that the pending copy (if any) does not use; its buffers are free: a set is
  // reused only after copa_fit_host took its copy (and synchronised) or dropped it
  const int set = h->n_staged == 1 ? 1 - h->staged[0].set : 0;
  if (!h->stage_ev[set])
    TRY(cuda_check(h, cudaEventCreateWithFlags(&h->stage_ev[set], cudaEventDisableTiming), "cudaEventCreate"));
  size_t sizes[4];
  tensor_bytes(Xh, sizes);
  const void* src[4] = {Xh->subj_ptr, Xh->row_ptr, Xh->col_idx, Xh->vals};
  for (int i = 0; i < 4; ++i) TRY(host_slot(h, 15 + 4 * set + i, sizes[i]));
  copa_ctx::StagedX& e = h->staged[h->n_staged++];
  e.set = set;
  e.issued = false;
  for (int i = 0; i < 4; ++i) e.src[i] = src[i];
  e.K = Xh->K;
  e.J = Xh->J;
  e.S = Xh->S;
  e.nnz = Xh->nnz;
  e.vdt = Xh->val_dtype;
  return COPA_OK;
}

copa_status_t copa_fit_host(copa_handle_t h, const copa_tensor_t* Xh, const copa_options_t* opt, void* H_host,
                            void* V_host, void* W_host, void* DH_host, void* DV_host, void* DW_host,
                            double* fit_history_host) {
  CHECK_H(h);
  TRY(set_dev(h));
  if (!Xh) return fail(h, COPA_ERR_INVALID_ARG, "X is NULL");
  // First (before any check can fail, so that a caller can track the pending copies): if
  // the oldest copy staged by copa_stage_host is of this X (same host arrays and sizes), it
  // leaves the queue, and if it was issued, its buffers become slots 10..13 (the stream
  // waits for its copies) and X is not copied again; otherwise every pending copy is
  // waited for (where issued) and discarded.
  bool took = false;
  if (h->n_staged > 0) {
    if (staged_matches(h->staged[0], Xh)) {
      const int set = h->staged[0].set;
      if (h->staged[0].issued) {   // not issued yet: this call copies X itself
        TRY(cuda_check(h, cudaStreamWaitEvent(h->stream, h->stage_ev[set], 0), "cudaStreamWaitEvent"));
        for (int q = 0; q < 4; ++q) {
          std::swap(h->host_slot_ptr[10 + q], h->host_slot_ptr[15 + 4 * set + q]);
          std::swap(h->host_slot_bytes[10 + q], h->host_slot_bytes[15 + 4 * set + q]);
        }
        took = true;
      }
      h->staged[0] = h->staged[1];
      --h->n_staged;
    } else {
      TRY(drop_staged(h));
    }
  }
  TRY(check_tensor_args(h, Xh));
  TRY(check_options(h, opt));
  if (!H_host || !V_host || !W_host || !DH_host || !DV_host || !DW_host)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_host: NULL factor or dual");
  const size_t es = h->precision == COPA_PREC_MIXED ? sizeof(float) : sizeof(double);
  const int R = opt->R;
  size_t sizes[10];
  tensor_bytes(Xh, sizes);
  sizes[4] = es * R * R;
  sizes[5] = es * (size_t)Xh->J * R;
  sizes[6] = es * (size_t)Xh->K * R;
  sizes[7] = es * R * R;
  sizes[8] = es * (size_t)Xh->J * R;
  sizes[9] = es * (size_t)Xh->K * R;
  const void* src[10] = {Xh->subj_ptr, Xh->row_ptr, Xh->col_idx, Xh->vals, H_host, V_host, W_host,
                         DH_host,      DV_host,     DW_host};
  // X goes to the staging slots 10..13 and is compared on the device with the copy in
  // slots 0..3 that the last call left there: the handle's caches derived from X (subject
  // schedule, warm-start rotations, column-sorted copy) are keyed by device address, so
  // they carry over to this call only if the contents are unchanged.
  for (int i = took ? 4 : 0; i < 10; ++i) {
    const int d = i < 4 ? 10 + i : i;
    TRY(host_slot(h, d, sizes[i]));
    if (sizes[i])
      TRY(cuda_check(h, cudaMemcpyAsync(h->host_slot_ptr[d], src[i], sizes[i], cudaMemcpyHostToDevice, h->stream),
                     "H2D"));
  }
  TRY(issue_staged(h));   // the next calls' tensors, behind this call's own copies
  bool same = h->host_x_valid && h->host_K == Xh->K && h->host_J == Xh->J && h->host_S == Xh->S &&
              h->host_nnz == Xh->nnz && h->host_vdt == Xh->val_dtype;
  for (int i = 0; i < 4 && same; ++i) same = h->host_slot_bytes[i] >= sizes[i] + 16;
  if (same) {
    TRY(host_slot(h, 14, sizeof(int)));
    int* flag = reinterpret_cast<int*>(h->host_slot_ptr[14]);
    TRY(cuda_check(h, cudaMemsetAsync(flag, 0, sizeof(int), h->stream), "memset"));
    ByteCmp c;
    int64_t most = 0;
    for (int q = 0; q < 4; ++q) {
      c.a[q] = reinterpret_cast<const unsigned char*>(h->host_slot_ptr[q]);
      c.b[q] = reinterpret_cast<const unsigned char*>(h->host_slot_ptr[10 + q]);
      c.n[q] = (int64_t)sizes[q];
      most = std::max<int64_t>(most, c.n[q] >> 4);
    }
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((most + 255) / 256, (int64_t)h->num_sms * 8));
    k_bytes_differ<<<blocks, 256, 0, h->stream>>>(c, flag);
    TRY(cuda_check(h, cudaGetLastError(), "k_bytes_differ"));
    int differ = 1;
    TRY(cuda_check(h, cudaMemcpyAsync(&differ, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "D2H"));
    TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    same = differ == 0;
  }
  if (!same) {   // the staged copy becomes the resident one; nothing derived from either is kept
    TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    for (int q : {0, 10})
      forget_caches_of(h, h->host_slot_ptr[q], h->host_slot_ptr[q + 2]);
    for (int q = 0; q < 4; ++q) {
      std::swap(h->host_slot_ptr[q], h->host_slot_ptr[10 + q]);
      std::swap(h->host_slot_bytes[q], h->host_slot_bytes[10 + q]);
    }
    h->host_x_valid = true;
    h->host_K = Xh->K;
    h->host_J = Xh->J;
    h->host_S = Xh->S;
    h->host_nnz = Xh->nnz;
    h->host_vdt = Xh->val_dtype;
  }
  void* dst[10];
  for (int i = 0; i < 10; ++i) dst[i] = h->host_slot_ptr[i];
  copa_tensor_t Xd = *Xh;
  Xd.subj_ptr = (const int64_t*)dst[0];
  Xd.row_ptr = (const int64_t*)dst[1];
  Xd.col_idx = (const int32_t*)dst[2];
  Xd.vals = dst[3];
  TRY(copa_fit(h, &Xd, opt, dst[4], dst[5], dst[6], dst[7], dst[8], dst[9], fit_history_host, nullptr));
  for (int i = 4; i < 10; ++i)
    TRY(cuda_check(h, cudaMemcpyAsync(const_cast<void*>(src[i]), dst[i], sizes[i], cudaMemcpyDeviceToHost, h->stream),
                   "D2H"));
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

}  // extern "C"
