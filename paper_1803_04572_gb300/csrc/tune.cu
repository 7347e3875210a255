// Autotuner of the launch schedule (no counterpart in the paper; a property of this
// implementation): which subjects take the tall-subject Procrustes kernels, how many
// blocks per SM the persistent Procrustes kernels keep resident, and which F_V kernel the
// V mode uses. Candidates are timed once per (rank, precision, subject-size histogram) with
// CUDA events on the handle's stream; the choice goes to a process-wide table keyed by a
// hash of those three, so that another handle or another tensor of the same shape reuses
// it without timing again.
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "copa_internal.cuh"

namespace copa {
namespace {

std::mutex g_tune_mu;
std::map<uint64_t, copa_tune_t> g_tune_table;

// FNV-1a over 64-bit words
uint64_t fnv(uint64_t h, uint64_t v) {
  for (int b = 0; b < 8; ++b) {
    h ^= (v >> (8 * b)) & 0xffu;
    h *= 1099511628211ull;
  }
  return h;
}

void apply(copa_ctx* h, const TensorView& X, int R, const copa_tune_t& c) {
  h->tune_valid = true;
  h->tune_ptr = X.subj_ptr;
  h->tune_K = X.K;
  h->tune_S = X.S;
  h->tune_R = R;
  h->tune_split = c.split;
  h->tune_bps = c.blocks_per_sm;
  h->tune_fv = c.fv_path;
  h->warm_valid = false;   // the subjects' assignment to the kernels may have changed
}

// Average duration (ms) of `reps` calls of f after one untimed call.
template <typename F>
copa_status_t time_ms(copa_ctx* h, int reps, F f, float* ms) {
  copa_status_t st;
  if ((st = f()) != COPA_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((st = cuda_check(h, cudaEventCreate(&e0), "cudaEventCreate")) != COPA_OK) return st;
  if ((st = cuda_check(h, cudaEventCreate(&e1), "cudaEventCreate")) != COPA_OK) {
    cudaEventDestroy(e0);
    return st;
  }
  cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps && st == COPA_OK; ++r) st = f();
  cudaEventRecord(e1, h->stream);
  if (st == COPA_OK) st = cuda_check(h, cudaEventSynchronize(e1), "cudaEventSynchronize");
  float t = 0.f;
  if (st == COPA_OK) st = cuda_check(h, cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return st;
}

template <typename Real>
copa_status_t tune_impl(copa_ctx* h, const TensorView& X, int R, const Real* H, const Real* V, const Real* W,
                        copa_tune_t* best) {
  copa_status_t st;
  Real *Q = nullptr, *T = nullptr, *F = nullptr;
  if ((st = ws_get(h, SLOT_FIT_Q, sizeof(Real) * (size_t)X.S * R + 16, (void**)&Q)) != COPA_OK) return st;
  if ((st = ws_get(h, SLOT_FIT_T, sizeof(Real) * (size_t)X.K * R * R + 16, (void**)&T)) != COPA_OK) return st;
  if ((st = ws_get(h, SLOT_FIT_FW, sizeof(Real) * ((size_t)X.J * R + 16), (void**)&F)) != COPA_OK) return st;
  const int top = std::min(R, 32);
  std::vector<int> splits = {top};
  for (int s : {24, 16, 8})
    if (s < top) splits.push_back(s);
  best->ms = INFINITY;
  const int reps = 2;
  for (int split : splits) {
    for (int bps : {0, 2}) {
      const copa_tune_t c{split, bps, 0, 0.f};
      apply(h, X, R, c);
      float ms = 0.f;
      if ((st = time_ms(h, reps, [&] {
             return launch_procrustes<Real>(h, X, R, H, V, W, 1e-8, Q, T, nullptr, nullptr, nullptr);
           }, &ms)) != COPA_OK)
        return st;
      if (ms < best->ms) {
        *best = c;
        best->ms = ms;
      }
    }
  }
  // the F_V kernel (FP32): row order with shared-memory sums (J x 32 floats), over the
  // column-sorted copy, or row order with the sums in L2
  best->fv_path = 2;
  if (std::is_same<Real, float>::value) {
    float t_path[3] = {INFINITY, INFINITY, INFINITY};
    const int n_fv = 3;
    for (int fv = 0; fv < n_fv; ++fv) {
      copa_tune_t c = *best;
      c.fv_path = fv;
      apply(h, X, R, c);
      if ((st = time_ms(h, reps, [&] {
             return launch_mttkrp_v<Real>(h, X, R, Q, H, W, F, nullptr, /*reuse_csc=*/true);
           }, &t_path[fv])) != COPA_OK)
        return st;
    }
    for (int fv = 0; fv < n_fv; ++fv)
      if (t_path[fv] < t_path[best->fv_path]) best->fv_path = fv;
    best->ms += t_path[best->fv_path];
  }
  return COPA_OK;
}

}  // namespace
}  // namespace copa

using namespace copa;

extern "C" copa_status_t copa_tune_key(const int64_t* subj_ptr_host, int64_t K, int32_t R, int32_t precision,
                                       uint64_t* key) {
  if (!subj_ptr_host || K < 0 || !key || R < 1) return COPA_ERR_INVALID_ARG;
  // share of the subjects in each power-of-two size class (I_k = 0, 1, 2-3, 4-7, ...), in
  // 1/64 steps, so that tensors drawn from the same distribution share a key
  int64_t cnt[64] = {0};
  for (int64_t k = 0; k < K; ++k) {
    const int64_t ik = subj_ptr_host[k + 1] - subj_ptr_host[k];
    int b = 0;
    while (b < 63 && (ik >> b) > 0) ++b;
    ++cnt[b];
  }
  uint64_t hsh = 1469598103934665603ull;
  hsh = fnv(hsh, (uint64_t)R);
  hsh = fnv(hsh, (uint64_t)precision);
  for (int b = 0; b < 64; ++b) {
    const uint64_t q = K > 0 ? (uint64_t)std::llround(64.0 * (double)cnt[b] / (double)K) : 0;
    hsh = fnv(hsh, q);
  }
  *key = hsh;
  return COPA_OK;
}

extern "C" copa_status_t copa_tune_lookup(uint64_t key, int32_t* found, copa_tune_t* out) {
  if (!found) return COPA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_table.find(key);
  *found = it != g_tune_table.end();
  if (*found && out) *out = it->second;
  return COPA_OK;
}

extern "C" copa_status_t copa_tune_store(uint64_t key, const copa_tune_t* choice) {
  if (!choice || choice->split < 1 || choice->blocks_per_sm < 0 || choice->fv_path < 0 || choice->fv_path > 2)
    return COPA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_table[key] = *choice;
  return COPA_OK;
}

extern "C" copa_status_t copa_tune(copa_handle_t h, const copa_tensor_t* X, int32_t R, const void* H, const void* V,
                                   const void* W, int32_t force, copa_tune_t* out) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t st;
  if ((st = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return st;
  if ((st = check_tensor_args(h, X)) != COPA_OK) return st;
  if (R < 1 || R > kMaxR) return fail(h, R < 1 ? COPA_ERR_INVALID_ARG : COPA_ERR_UNSUPPORTED, "copa_tune: R");
  if (!H || !V || !W) return fail(h, COPA_ERR_INVALID_ARG, "copa_tune: NULL factor");
  std::vector<int64_t> sp((size_t)X->K + 1);
  if ((st = cuda_check(h, cudaMemcpyAsync(sp.data(), X->subj_ptr, sizeof(int64_t) * sp.size(), cudaMemcpyDeviceToHost,
                                          h->stream), "D2H")) != COPA_OK)
    return st;
  if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync")) != COPA_OK) return st;
  uint64_t key = 0;
  copa_tune_key(sp.data(), X->K, R, h->precision, &key);
  const TensorView v = view_of(X);
  copa_tune_t c{};
  int32_t found = 0;
  copa_tune_lookup(key, &found, &c);
  if (!found || force) {
    st = h->precision == COPA_PREC_MIXED
             ? tune_impl<float>(h, v, R, (const float*)H, (const float*)V, (const float*)W, &c)
             : tune_impl<double>(h, v, R, (const double*)H, (const double*)V, (const double*)W, &c);
    if (st != COPA_OK) {
      h->tune_valid = false;
      return st;
    }
    copa_tune_store(key, &c);
  }
  apply(h, v, R, c);
  if (out) *out = c;
  return copa_sync(h);
}
