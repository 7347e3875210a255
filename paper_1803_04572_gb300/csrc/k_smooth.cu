// Smoothness on U_k (Sec. 3.3.1): per subject, the spline basis M_k (I_k x l) evaluated
// at the visit days, C_k = its left singular vectors (rank cut sigma^2 > 1e-10 sigma_max^2)
// and the projected slice X'_k = C_k^T X_k, run once before the fit. PARAFAC2 on X'
// gives the same H, S_k, V; U_k = C_k Q_k H afterwards (proof in Sec. 3.3.1).
//
// Basis: clamped B-splines of degree d with l functions on [t_1, t_n] (the first and last
// visit day; days are non-decreasing within a subject): knots t_1 repeated d+1 times,
// l-d-1 interior knots, t_n repeated d+1 times. The interior knots are either equally
// spaced in days (COPA_KNOTS_UNIFORM) or placed at the quantiles j/(l-d) of the subject's
// visit days, interpolating linearly between order statistics (COPA_KNOTS_QUANTILE: many
// knots where visits cluster, few across long gaps; Sec. 3.3.1 leaves the knots to be
// estimated). The values of the recursion of Sec. 3.3.1 at a day t are computed with the
// triangular scheme on the last non-empty knot span that starts at or before t (half-open
// spans; the last non-empty one is closed at t_n).
// C_k = M_k Z Lambda^{-1/2} from the FP64 Jacobi eigendecomposition M_k^T M_k = Z Lambda Z^T.
#include "copa_internal.cuh"

namespace copa {

namespace {

constexpr double kTauBasis = 1e-10;
constexpr int kMaxJWords = 8192;   // column bitmap of X_k in shared memory: J <= 262144

struct SmoothArgs {
  TensorView X;
  const double* days;
  int l, d, rule;
  int* r_out;          // K: rank r_k
  int64_t* c_out;      // K: distinct columns c_k
  double* Zs;          // K x l x l: Z Lambda^{-1/2} on the kept eigenpairs (columns >= r_k zero)
};

// knots of the clamped basis of the subject with visit rows r0 .. r1-1 (l + d + 1 of them)
__device__ inline void make_knots(const double* days, int64_t r0, int64_t r1, int l, int d, int rule, double* kn) {
  const double t1 = days[r0], tn = days[r1 - 1];
  const int nint = l - d - 1;
  for (int i = 0; i < l + d + 1; ++i) {
    if (i <= d) {
      kn[i] = t1;
    } else if (i >= l) {
      kn[i] = tn;
    } else {
      const double p = (double)(i - d) / (double)(nint + 1);
      if (rule == COPA_KNOTS_QUANTILE) {
        const double hq = (double)(r1 - r0 - 1) * p;
        const int64_t j = (int64_t)floor(hq);
        const int64_t j1 = min(j + 1, r1 - r0 - 1);
        kn[i] = days[r0 + j] + (hq - (double)j) * (days[r0 + j1] - days[r0 + j]);
      } else {
        kn[i] = t1 + (tn - t1) * p;
      }
    }
  }
}

// all l basis values at t (out[0..l-1]); t in [kn[0], kn[l+d]], kn[0] < kn[l+d]
__device__ inline void basis_at(double t, int l, int d, const double* kn, double* out) {
  for (int b = 0; b < l; ++b) out[b] = 0.0;
  int mu = d;   // the last non-empty span [kn[m], kn[m+1]) with kn[m] <= t
  for (int m = d; m < l; ++m)
    if (kn[m] <= t && kn[m] < kn[m + 1]) mu = m;
  double N[kMaxBasis], left[kMaxBasis], right[kMaxBasis];
  N[0] = 1.0;
  for (int j = 1; j <= d; ++j) {
    left[j] = t - kn[mu + 1 - j];
    right[j] = kn[mu + j] - t;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      const double den = right[r + 1] + left[j - r];
      const double temp = den > 0.0 ? N[r] / den : 0.0;
      N[r] = saved + right[r + 1] * temp;
      saved = left[j - r] * temp;
    }
    N[j] = saved;
  }
  for (int j = 0; j <= d; ++j) out[mu - d + j] = N[j];
}

// Basis row of visit i of a subject (handles the constant-basis special case).
__device__ inline void basis_row(const double* days, int64_t r0, int64_t r1, int64_t i, int l, int d, int rule,
                                 double* out, int* lb) {
  const double t1 = days[r0], tn = days[r1 - 1];
  if (!(tn > t1)) {
    *lb = 1;
    out[0] = 1.0;
    return;
  }
  *lb = l;
  double kn[2 * kMaxBasis + 1];
  make_knots(days, r0, r1, l, d, rule, kn);
  basis_at(days[i], l, d, kn, out);
}

// Cyclic Jacobi on a small symmetric matrix (n <= kMaxBasis), single thread, FP64.
__device__ void jacobi_small(double* A, double* Z, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Z[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? dg : off) += A[i * n + j] * A[i * n + j];
    if (dg == 0.0 || off <= 1e-30 * dg) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = fabs(theta) > 1e150 ? 0.5 / theta
                                               : copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double a = A[p * n + k], b = A[q * n + k];
          A[p * n + k] = c * a - s * b;
          A[q * n + k] = s * a + c * b;
        }
        for (int k = 0; k < n; ++k) {
          double a = A[k * n + p], b = A[k * n + q];
          A[k * n + p] = c * a - s * b;
          A[k * n + q] = s * a + c * b;
          a = Z[k * n + p];
          b = Z[k * n + q];
          Z[k * n + p] = c * a - s * b;
          Z[k * n + q] = s * a + c * b;
        }
        A[p * n + q] = A[q * n + p] = 0.0;
      }
  }
}

// column bitmap of subject k in per-warp shared memory; returns c_k
__device__ int64_t build_bitmap(const TensorView& X, int64_t r0, int64_t r1, uint32_t* bm, int* pre, int nw) {
  const int lane = threadIdx.x & 31;
  for (int w = lane; w < nw; w += 32) bm[w] = 0u;
  __syncwarp();
  for (int64_t t = X.row_ptr[r0] + lane; t < X.row_ptr[r1]; t += 32) {
    const int c = X.col[t];
    atomicOr(bm + (c >> 5), 1u << (c & 31));
  }
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    for (int w = 0; w < nw; ++w) { pre[w] = acc; acc += __popc(bm[w]); }
    pre[nw] = acc;
  }
  __syncwarp();
  return pre[nw];
}

__global__ void k_smooth_plan(SmoothArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nw = (a.X.J + 31) / 32;
  const int l = a.l;
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)warp * (2 * nw + 2);
  int* pre = reinterpret_cast<int*>(bm + nw);
  double* B = reinterpret_cast<double*>(smem_raw + (size_t)nwarps * (2 * nw + 2) * 4) +
              (size_t)warp * (3 * l * l + l);
  double* Z = B + l * l;
  double* row = Z + l * l;
  const int64_t wid = blockIdx.x * (int64_t)nwarps + warp, nwt = (int64_t)gridDim.x * nwarps;
  for (int64_t k = wid; k < a.X.K; k += nwt) {
    const int64_t r0 = a.X.subj_ptr[k], r1 = a.X.subj_ptr[k + 1];
    const int64_t ck = build_bitmap(a.X, r0, r1, bm, pre, nw);
    if (lane == 0) {
      int r = 0;
      double* Zk = a.Zs + k * l * l;
      for (int e = 0; e < l * l; ++e) Zk[e] = 0.0;
      if (r1 > r0) {
        int lb = l;
        for (int e = 0; e < l * l; ++e) B[e] = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
          basis_row(a.days, r0, r1, i, l, a.d, a.rule, row, &lb);
          for (int p = 0; p < lb; ++p)
            for (int q = 0; q < lb; ++q) B[p * lb + q] += row[p] * row[q];
        }
        jacobi_small(B, Z, lb);
        double lmax = 0.0;
        for (int p = 0; p < lb; ++p) lmax = fmax(lmax, B[p * lb + p]);
        for (int p = 0; p < lb; ++p) {
          const double lp = B[p * lb + p];
          if (lmax > 0.0 && lp > kTauBasis * lmax) {
            for (int q = 0; q < lb; ++q) Zk[q * l + r] = Z[q * lb + p] / sqrt(lp);
            ++r;
          }
        }
      }
      a.r_out[k] = r;
      a.c_out[k] = ck;
    }
    __syncwarp();
  }
}

__global__ void k_scan_sizes(const int* __restrict__ r, const int64_t* __restrict__ c, int64_t K,
                             int64_t* __restrict__ row_off, int64_t* __restrict__ nz_off) {
  // single block: exclusive scans of r_k and r_k c_k (K + 1 entries each)
  __shared__ int64_t part_r[1024], part_n[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (K + nt - 1) / nt;
  const int64_t k0 = tid * per, k1 = min(K, k0 + per);
  int64_t sr = 0, sn = 0;
  for (int64_t k = k0; k < k1; ++k) { sr += r[k]; sn += (int64_t)r[k] * c[k]; }
  part_r[tid] = sr;
  part_n[tid] = sn;
  __syncthreads();
  if (tid == 0) {
    int64_t ar = 0, an = 0;
    for (int i = 0; i < nt; ++i) {
      const int64_t x = part_r[i], y = part_n[i];
      part_r[i] = ar; part_n[i] = an;
      ar += x; an += y;
    }
    row_off[K] = ar;
    nz_off[K] = an;
  }
  __syncthreads();
  sr = part_r[tid];
  sn = part_n[tid];
  for (int64_t k = k0; k < k1; ++k) {
    row_off[k] = sr;
    nz_off[k] = sn;
    sr += r[k];
    sn += (int64_t)r[k] * c[k];
  }
}

template <typename Out>
__global__ void k_smooth_project(SmoothArgs a, const int64_t* __restrict__ row_off,
                                 const int64_t* __restrict__ nz_off, int64_t* __restrict__ subj_ptr,
                                 int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                 Out* __restrict__ vals, double* __restrict__ Cout) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nw = (a.X.J + 31) / 32;
  const int l = a.l;
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw) + (size_t)warp * (2 * nw + 2);
  int* pre = reinterpret_cast<int*>(bm + nw);
  double* crow = reinterpret_cast<double*>(smem_raw + (size_t)nwarps * (2 * nw + 2) * 4) + (size_t)warp * 2 * kMaxBasis;
  double* brow = crow + kMaxBasis;
  const int64_t wid = blockIdx.x * (int64_t)nwarps + warp, nwt = (int64_t)gridDim.x * nwarps;
  for (int64_t k = wid; k < a.X.K; k += nwt) {
    const int64_t r0 = a.X.subj_ptr[k], r1 = a.X.subj_ptr[k + 1];
    const int64_t ck = build_bitmap(a.X, r0, r1, bm, pre, nw);
    const int rk = a.r_out[k];
    const int64_t ro = row_off[k], no = nz_off[k];
    if (lane == 0) subj_ptr[k] = ro;
    if (k == a.X.K - 1 && lane == 0) {
      subj_ptr[a.X.K] = row_off[a.X.K];
      row_ptr[row_off[a.X.K]] = nz_off[a.X.K];
    }
    for (int q = 0; q < rk; ++q) {
      if (lane == 0) row_ptr[ro + q] = no + (int64_t)q * ck;
      for (int w = 0; w < nw; ++w) {
        uint32_t bits = bm[w];
        int base = pre[w];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          if ((base & 31) == lane) {
            col[no + (int64_t)q * ck + base] = w * 32 + b;
            vals[no + (int64_t)q * ck + base] = Out(0);
          }
          ++base;
        }
      }
    }
    __syncwarp();
    const double* Zk = a.Zs + k * l * l;
    for (int64_t i = r0; i < r1; ++i) {
      int lb = l;
      if (lane == 0) {
        basis_row(a.days, r0, r1, i, l, a.d, a.rule, brow, &lb);
        for (int q = 0; q < kMaxBasis; ++q) crow[q] = 0.0;
        for (int q = 0; q < rk; ++q) {
          double acc = 0.0;
          for (int p = 0; p < lb; ++p) acc += brow[p] * Zk[p * l + q];
          crow[q] = acc;
        }
        if (Cout)
          for (int q = 0; q < l; ++q) Cout[i * l + q] = crow[q];
      }
      __syncwarp();
      for (int64_t t = a.X.row_ptr[i] + lane; t < a.X.row_ptr[i + 1]; t += 32) {
        const int c = a.X.col[t];
        const int pos = pre[c >> 5] + __popc(bm[c >> 5] & ((1u << (c & 31)) - 1u));
        const double x = load_val(a.X, t);
        for (int q = 0; q < rk; ++q) {
          Out* v = vals + no + (int64_t)q * ck + pos;
          *v = Out((double)*v + crow[q] * x);
        }
      }
      __syncwarp();
    }
  }
}

copa_status_t run_plan(copa_ctx* h, const copa_tensor_t* X, const double* days, int l, int d, int rule,
                       SmoothArgs* a, int64_t** row_off, int64_t** nz_off, size_t* smem_plan) {
  if (l < 1 || l > kMaxBasis || d < 0 || d >= l)
    return fail(h, COPA_ERR_INVALID_ARG, "smoothing: need 1 <= n_basis <= 16 and 0 <= degree < n_basis");
  if (rule != COPA_KNOTS_UNIFORM && rule != COPA_KNOTS_QUANTILE)
    return fail(h, COPA_ERR_INVALID_ARG, "smoothing: unknown knot rule");
  if (!days) return fail(h, COPA_ERR_INVALID_ARG, "smoothing: days is NULL");
  const int nw = (X->J + 31) / 32;
  if (nw > kMaxJWords) return fail(h, COPA_ERR_UNSUPPORTED, "smoothing: J too large");
  const int64_t K = X->K;
  const size_t bytes = sizeof(int) * (K + 1) + sizeof(int64_t) * (K + 1) * 3 + sizeof(double) * (size_t)K * l * l + 1024;
  char* p = nullptr;
  copa_status_t st;
  if ((st = ws_get(h, SLOT_SMOOTH, bytes, (void**)&p)) != COPA_OK) return st;
  a->X = view_of(X);
  a->days = days;
  a->l = l;
  a->d = d;
  a->rule = rule;
  a->c_out = reinterpret_cast<int64_t*>(p);
  *row_off = a->c_out + (K + 1);
  *nz_off = *row_off + (K + 1);
  a->Zs = reinterpret_cast<double*>(*nz_off + (K + 1));
  a->r_out = reinterpret_cast<int*>(a->Zs + (size_t)K * l * l);
  const int warps = 4;
  *smem_plan = (size_t)warps * (2 * nw + 2) * 4 + (size_t)warps * (3 * l * l + l) * sizeof(double) + 64;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_smooth_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)*smem_plan), "attr")) != COPA_OK)
    return st;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((K + warps - 1) / warps, (int64_t)h->num_sms * 8));
  if (K > 0) k_smooth_plan<<<blocks, 32 * warps, *smem_plan, h->stream>>>(*a);
  k_scan_sizes<<<1, 1024, 0, h->stream>>>(a->r_out, a->c_out, K, *row_off, *nz_off);
  return cuda_check(h, cudaGetLastError(), "k_smooth_plan");
}

}  // namespace
}  // namespace copa

using namespace copa;

extern "C" copa_status_t copa_smooth_plan(copa_handle_t h, const copa_tensor_t* X, const double* days,
                                          int32_t n_basis, int32_t degree, int32_t knot_rule, int64_t* S_out,
                                          int64_t* nnz_out) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t st;
  if ((st = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return st;
  if ((st = check_tensor_args(h, X)) != COPA_OK) return st;
  if (!S_out || !nnz_out) return fail(h, COPA_ERR_INVALID_ARG, "copa_smooth_plan: NULL output");
  SmoothArgs a;
  int64_t *ro, *no;
  size_t smem;
  if ((st = run_plan(h, X, days, n_basis, degree, knot_rule, &a, &ro, &no, &smem)) != COPA_OK) return st;
  if ((st = cuda_check(h, cudaMemcpyAsync(S_out, ro + X->K, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream),
                       "D2H")) != COPA_OK)
    return st;
  if ((st = cuda_check(h, cudaMemcpyAsync(nnz_out, no + X->K, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream),
                       "D2H")) != COPA_OK)
    return st;
  return copa_sync(h);
}

extern "C" copa_status_t copa_smooth_project(copa_handle_t h, const copa_tensor_t* X, const double* days,
                                             int32_t n_basis, int32_t degree, int32_t knot_rule, copa_tensor_t* Xp,
                                             double* C) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t st;
  if ((st = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return st;
  if ((st = check_tensor_args(h, X)) != COPA_OK) return st;
  if (!Xp || !Xp->subj_ptr || !Xp->row_ptr || (Xp->nnz > 0 && (!Xp->col_idx || !Xp->vals)))
    return fail(h, COPA_ERR_INVALID_ARG, "copa_smooth_project: NULL output array");
  if (Xp->val_dtype != COPA_VAL_F32 && Xp->val_dtype != COPA_VAL_F64)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_smooth_project: output values must be F32 or F64");
  SmoothArgs a;
  int64_t *ro, *no;
  size_t smem;
  if ((st = run_plan(h, X, days, n_basis, degree, knot_rule, &a, &ro, &no, &smem)) != COPA_OK) return st;
  const int warps = 4;
  const int nw = (X->J + 31) / 32;
  const size_t smem2 = (size_t)warps * (2 * nw + 2) * 4 + (size_t)warps * 2 * kMaxBasis * sizeof(double) + 64;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((X->K + warps - 1) / warps, (int64_t)h->num_sms * 8));
  auto* sp = const_cast<int64_t*>(Xp->subj_ptr);
  auto* rp = const_cast<int64_t*>(Xp->row_ptr);
  auto* cp = const_cast<int32_t*>(Xp->col_idx);
  if (X->K == 0) {
    cudaMemsetAsync(sp, 0, sizeof(int64_t), h->stream);
    cudaMemsetAsync(rp, 0, sizeof(int64_t), h->stream);
  } else if (Xp->val_dtype == COPA_VAL_F32) {
    cudaFuncSetAttribute(k_smooth_project<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    k_smooth_project<float><<<blocks, 32 * warps, smem2, h->stream>>>(a, ro, no, sp, rp, cp,
                                                                      (float*)const_cast<void*>(Xp->vals), C);
  } else {
    cudaFuncSetAttribute(k_smooth_project<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    k_smooth_project<double><<<blocks, 32 * warps, smem2, h->stream>>>(a, ro, no, sp, rp, cp,
                                                                       (double*)const_cast<void*>(Xp->vals), C);
  }
  if ((st = cuda_check(h, cudaGetLastError(), "k_smooth_project")) != COPA_OK) return st;
  return copa_sync(h);
}

// =====================================================================================
// The paper's output factor U_k = Q_k H, or C_k Q_k H after a fit on the smoothed
// projection (Algorithm 1 output; Sec. 3.3.1).
// =====================================================================================

namespace copa {
namespace {

constexpr int kUThreads = 256;

// Y[i, :] = Q[i, :] H for rows, a warp per row, H in shared memory (R x R)
template <typename Real>
__global__ void __launch_bounds__(kUThreads) k_times_H(int64_t rows, int R, const Real* __restrict__ Q,
                                                       const Real* __restrict__ H, Real* __restrict__ Y) {
  extern __shared__ unsigned char smem_raw[];
  Real* Hs = reinterpret_cast<Real*>(smem_raw);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Hs[e] = H[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < rows; i += nw) {
    const Real* q = Q + i * R;
    for (int c = lane; c < R; c += 32) {
      Real acc = Real(0);
      for (int r = 0; r < R; ++r) acc += q[r] * Hs[r * R + c];
      Y[i * R + c] = acc;
    }
  }
}

// U[i, :] = sum_{q < r_k} C[i, q] Y[sp_fit[k] + q, :] for every original visit row i of
// subject k (r_k = sp_fit[k+1] - sp_fit[k]), a warp per row
template <typename Real>
__global__ void __launch_bounds__(kUThreads) k_basis_combine(int64_t K, int64_t S, int R, int nb,
                                                             const int64_t* __restrict__ sp,
                                                             const int64_t* __restrict__ sp_fit,
                                                             const double* __restrict__ C,
                                                             const Real* __restrict__ Y, Real* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < S; i += nw) {
    int64_t lo = 0, hi = K;   // the subject k with sp[k] <= i < sp[k+1]
    while (hi - lo > 1) {
      const int64_t m = (lo + hi) >> 1;
      if (sp[m] <= i) lo = m;
      else hi = m;
    }
    const int64_t k = lo;
    const int64_t f0 = sp_fit[k];
    const int rk = (int)min(sp_fit[k + 1] - f0, (int64_t)nb);
    for (int c = lane; c < R; c += 32) {
      double acc = 0.0;
      for (int q = 0; q < rk; ++q) acc += C[i * nb + q] * (double)Y[(f0 + q) * R + c];
      U[i * R + c] = (Real)acc;
    }
  }
}

template <typename Real>
copa_status_t launch_factor_U(copa_ctx* h, int64_t K, int R, const int64_t* sp_fit, int64_t S_fit, const Real* Q,
                              const Real* H, const int64_t* sp, const double* C, int nb, int64_t S, Real* U) {
  copa_status_t st;
  const size_t smem = sizeof(Real) * (size_t)R * R;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_times_H<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "attr")) != COPA_OK)
    return st;
  auto grid = [&](int64_t rows) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)h->num_sms * 8));
  };
  if (!C) {
    if (S_fit > 0) k_times_H<Real><<<grid(S_fit), kUThreads, smem, h->stream>>>(S_fit, R, Q, H, U);
    return cuda_check(h, cudaGetLastError(), "k_times_H");
  }
  Real* Y = nullptr;
  if ((st = ws_get(h, SLOT_MISC, sizeof(Real) * (size_t)std::max<int64_t>(S_fit, 1) * R, (void**)&Y)) != COPA_OK)
    return st;
  if (S_fit > 0) k_times_H<Real><<<grid(S_fit), kUThreads, smem, h->stream>>>(S_fit, R, Q, H, Y);
  if (S > 0) k_basis_combine<Real><<<grid(S), kUThreads, 0, h->stream>>>(K, S, R, nb, sp, sp_fit, C, Y, U);
  return cuda_check(h, cudaGetLastError(), "k_basis_combine");
}

}  // namespace
}  // namespace copa

extern "C" copa_status_t copa_factor_U(copa_handle_t h, int64_t K, int32_t R, const int64_t* subj_ptr_fit,
                                       int64_t S_fit, const void* Q, const void* H, const int64_t* subj_ptr,
                                       const double* C, int32_t n_basis, int64_t S, void* U) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t st;
  if ((st = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return st;
  if (R < 1 || R > kMaxR) return fail(h, R < 1 ? COPA_ERR_INVALID_ARG : COPA_ERR_UNSUPPORTED, "copa_factor_U: R");
  if (K < 0 || S_fit < 0 || !Q || !H || !U || !subj_ptr_fit)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_factor_U: bad arguments");
  if (C && (!subj_ptr || S < 0 || n_basis < 1 || n_basis > kMaxBasis))
    return fail(h, COPA_ERR_INVALID_ARG, "copa_factor_U: C needs subj_ptr, S >= 0 and 1 <= n_basis <= 16");
  if (h->precision == COPA_PREC_MIXED)
    return launch_factor_U<float>(h, K, R, subj_ptr_fit, S_fit, (const float*)Q, (const float*)H, subj_ptr, C,
                                  n_basis, S, (float*)U);
  return launch_factor_U<double>(h, K, R, subj_ptr_fit, S_fit, (const double*)Q, (const double*)H, subj_ptr, C,
                                 n_basis, S, (double*)U);
}
