// Procrustes step of COPA (Sec. 3.1, Eq. solv_Q; Algorithm 1 per-subject loop) for all
// subjects in one persistent launch, one warp per subject, dynamic scheduling over a
// largest-first subject order.
//
// Per subject k (P_k = X_k V, S_k = diag(w_k), E_k = S_k H^T, A_k = P_k E_k):
//   G_k   = P_k^T P_k                       FP64, accumulated from FP32/FP64 rows p_i
//   M_k   = E_k^T G_k E_k = H S_k G_k S_k H^T   (= A_k^T A_k)
//   M_k   = C diag(lambda) C^T               FP64 cyclic Jacobi, parallel pair order
//   Omega = sum_{lambda_i > tau lambda_max} lambda_i^{-1/2} c_i c_i^T
//   Gamma = E_k Omega   (Q_k = A_k Omega = P_k Gamma)
//   T_k   = Gamma^T G_k (= Q_k^T X_k V),  Pi_k = Omega M_k Omega = sum_kept c_i c_i^T
//   F_H  += T_k S_k     (mode-1 MTTKRP, Algorithm 1, fused; per-warp FP64 partials)
// Q_k = B C^T of the truncated SVD A_k = B D C^T equals A_k Omega: the left singular
// vectors are B = A_k C D^{-1} on the kept part.
#include "copa_internal.cuh"

namespace copa {

namespace {

constexpr int kMaxSweeps = 24;

struct ProcLayout {
  int R, n2, ld, m, ldh, npk;
  size_t doubles;  // dynamic shared memory in doubles
};

__host__ __device__ inline ProcLayout proc_layout(int R) {
  ProcLayout L;
  L.R = R;
  L.n2 = R + (R & 1);     // even size for the round-robin pairing (one zero dummy)
  L.ld = L.n2 + 1;        // odd stride: conflict-free column access of doubles
  L.m = L.n2 / 2;         // disjoint rotations per round
  L.ldh = R + 1;
  L.npk = R * (R + 1) / 2;
  size_t d = 0;
  d += (size_t)R * L.ldh;            // H (double)
  d += L.ld;                         // p / scratch vector
  d += 3 * (size_t)L.n2 * L.ld;      // G, A, C
  d += 2 * (size_t)L.m;              // (c, s) per pair
  d += (size_t)L.m;                  // (p, q) per pair as two ints
  d += ((size_t)L.npk * 2 + 7) / 8;  // packed upper-triangle pair table (uint16)
  L.doubles = d;
  return L;
}

// Element at round-robin position `pos` in round `round` (position 0 is fixed).
__device__ __forceinline__ int rr_elem(int pos, int round, int n2) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (n2 - 1));
}

template <typename Real>
__global__ void __launch_bounds__(32) k_procrustes(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V,
    const Real* __restrict__ W, double tau, Real* __restrict__ Gamma, Real* __restrict__ T,
    Real* __restrict__ Pi, int32_t* __restrict__ rank, double* __restrict__ fh_partial,
    const int64_t* __restrict__ order, int* __restrict__ counter, int* __restrict__ status) {
  extern __shared__ double smem[];
  const ProcLayout L = proc_layout(R);
  const int n2 = L.n2, ld = L.ld, m = L.m, ldh = L.ldh;
  const int lane = threadIdx.x;
  double* Hs = smem;
  double* p = Hs + (size_t)R * ldh;
  double* G = p + ld;
  double* A = G + (size_t)n2 * ld;
  double* C = A + (size_t)n2 * ld;
  double* cs = C + (size_t)n2 * ld;
  int* pq = reinterpret_cast<int*>(cs + 2 * m);
  uint16_t* pk = reinterpret_cast<uint16_t*>(pq + 2 * m);

  for (int i = lane; i < R * R; i += 32) Hs[(i / R) * ldh + (i % R)] = (double)H[i];
  for (int r = 0, e = 0; r < R; ++r)
    for (int s = r; s < R; ++s, ++e)
      if ((e & 31) == lane) pk[e] = (uint16_t)((r << 8) | s);
  double* fh = fh_partial ? fh_partial + (size_t)blockIdx.x * R * R : nullptr;
  if (fh)
    for (int i = lane; i < R * R; i += 32) fh[i] = 0.0;
  __syncwarp();

  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= X.K) break;
    const int64_t k = order ? order[idx] : idx;
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];

    // ---- G_k = sum_i p_i^T p_i (upper triangle, FP64) ----
    for (int e = lane; e < n2 * ld; e += 32) G[e] = 0.0;
    __syncwarp();
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
      for (int r = lane; r < R; r += 32) {
        Real acc = Real(0);
        for (int64_t t = a; t < b; ++t)
          acc += load_x<Real>(X, t) * __ldg(V + (int64_t)__ldg(X.col + t) * R + r);
        p[r] = (double)acc;
      }
      __syncwarp();
      for (int e = lane; e < L.npk; e += 32) {
        const int r = pk[e] >> 8, s = pk[e] & 255;
        G[r * ld + s] = fma(p[r], p[s], G[r * ld + s]);
      }
      __syncwarp();
    }
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, s = e - r * R;
      if (r > s) G[r * ld + s] = G[s * ld + r];
    }
    for (int r = lane; r < R; r += 32) p[r] = (double)W[k * R + r];
    __syncwarp();

    // ---- M = H (S G S) H^T: A <- (S G S) H^T, C <- H A, A <- sym(C), C <- I ----
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, u = e - r * R;
      double acc = 0.0;
      for (int s = 0; s < R; ++s) acc = fma(G[r * ld + s] * p[s], Hs[u * ldh + s], acc);
      A[r * ld + u] = acc * p[r];
    }
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) {
      const int t = e / R, u = e - t * R;
      double acc = 0.0;
      for (int r = 0; r < R; ++r) acc = fma(Hs[t * ldh + r], A[r * ld + u], acc);
      C[t * ld + u] = acc;
    }
    __syncwarp();
    for (int e = lane; e < n2 * n2; e += 32) {
      const int t = e / n2, u = e - t * n2;
      A[t * ld + u] = (t < R && u < R) ? 0.5 * (C[t * ld + u] + C[u * ld + t]) : 0.0;
    }
    __syncwarp();
    for (int e = lane; e < n2 * n2; e += 32) {
      const int t = e / n2, u = e - t * n2;
      C[t * ld + u] = (t == u) ? 1.0 : 0.0;
    }
    __syncwarp();

    // ---- cyclic Jacobi, n2 - 1 rounds of m disjoint rotations per sweep. A pair is
    // rotated only if |a_pq| > 1e-15 sqrt(|a_pp a_qq|) (relative threshold, which keeps
    // small eigenvalues accurate); the sweeps stop after one without any rotation. ----
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      int nrot = 0;
      for (int round = 0; round < n2 - 1; ++round) {
        for (int j = lane; j < m; j += 32) {
          int pp = rr_elem(j, round, n2), qq = rr_elem(n2 - 1 - j, round, n2);
          if (pp > qq) { const int tmp = pp; pp = qq; qq = tmp; }
          const double app = A[pp * ld + pp], aqq = A[qq * ld + qq], apq = A[pp * ld + qq];
          double c = 1.0, s = 0.0;
          if (apq != 0.0 && fabs(apq) > 1e-15 * sqrt(fabs(app) * fabs(aqq))) {
            const double theta = (aqq - app) / (2.0 * apq);
            double t;
            if (fabs(theta) > 1e150) t = 0.5 / theta;
            else t = copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            ++nrot;
          }
          cs[2 * j] = c; cs[2 * j + 1] = s;
          pq[2 * j] = pp; pq[2 * j + 1] = qq;
        }
        __syncwarp();
        for (int e = lane; e < m * n2; e += 32) {          // rows p, q of J^T A
          const int j = e / n2, col = e - j * n2;
          const double c = cs[2 * j], s = cs[2 * j + 1];
          if (s == 0.0) continue;
          const int pp = pq[2 * j], qq = pq[2 * j + 1];
          const double a = A[pp * ld + col], b = A[qq * ld + col];
          A[pp * ld + col] = c * a - s * b;
          A[qq * ld + col] = s * a + c * b;
        }
        __syncwarp();
        for (int e = lane; e < m * n2; e += 32) {          // columns p, q of (J^T A) J, C J
          const int j = e / n2, row = e - j * n2;
          const double c = cs[2 * j], s = cs[2 * j + 1];
          if (s == 0.0) continue;
          const int pp = pq[2 * j], qq = pq[2 * j + 1];
          double a = A[row * ld + pp], b = A[row * ld + qq];
          A[row * ld + pp] = c * a - s * b;
          A[row * ld + qq] = s * a + c * b;
          a = C[row * ld + pp]; b = C[row * ld + qq];
          C[row * ld + pp] = c * a - s * b;
          C[row * ld + qq] = s * a + c * b;
        }
        __syncwarp();
        for (int j = lane; j < m; j += 32) {
          if (cs[2 * j + 1] != 0.0) {
            A[pq[2 * j] * ld + pq[2 * j + 1]] = 0.0;
            A[pq[2 * j + 1] * ld + pq[2 * j]] = 0.0;
          }
        }
        __syncwarp();
      }
      if (warp_sum(nrot) == 0) break;
    }

    // ---- kept eigenpairs: lambda_i > tau * lambda_max ----
    double lmax = 0.0;
    for (int i = lane; i < R; i += 32) lmax = fmax(lmax, A[i * ld + i]);
    lmax = warp_max(lmax);
    int kept = 0;
    for (int i = lane; i < R; i += 32) {
      const double li = A[i * ld + i];
      const bool keep = lmax > 0.0 && li > tau * lmax;
      p[i] = keep ? 1.0 / sqrt(li) : 0.0;
      kept += keep ? 1 : 0;
    }
    kept = warp_sum(kept);
    if (rank && lane == 0) rank[k] = kept;
    __syncwarp();

    // ---- Omega -> A;  Pi (optional) -> global ----
    for (int e = lane; e < R * R; e += 32) {
      const int t = e / R, u = e - t * R;
      double acc = 0.0, pacc = 0.0;
      for (int i = 0; i < R; ++i) {
        const double ci = C[t * ld + i] * C[u * ld + i];
        acc = fma(ci, p[i], acc);
        pacc += (p[i] > 0.0) ? ci : 0.0;
      }
      A[t * ld + u] = acc;
      if (Pi) Pi[k * R * R + e] = (Real)pacc;
    }
    __syncwarp();
    for (int r = lane; r < R; r += 32) p[r] = (double)W[k * R + r];
    __syncwarp();
    // ---- Gamma = S H^T Omega -> C and global ----
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, u = e - r * R;
      double acc = 0.0;
      for (int t = 0; t < R; ++t) acc = fma(Hs[t * ldh + r], A[t * ld + u], acc);
      acc *= p[r];
      C[r * ld + u] = acc;
      Gamma[k * R * R + e] = (Real)acc;
    }
    __syncwarp();
    // ---- T = Gamma^T G -> global; F_H partial += T S ----
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, s = e - r * R;
      double acc = 0.0;
      for (int t = 0; t < R; ++t) acc = fma(C[t * ld + r], G[t * ld + s], acc);
      T[k * R * R + e] = (Real)acc;
      if (fh) fh[e] += acc * p[s];
    }
    __syncwarp();
  }
}

template <typename Real>
__global__ void k_reduce_partials(const double* __restrict__ part, int nparts, int n,
                                  Real* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nparts; ++q) acc += part[(size_t)q * n + e];
    out[e] = (Real)acc;
  }
}

}  // namespace

template <typename Real>
copa_status_t launch_procrustes(copa_ctx* h, const TensorView& X, int R, const Real* H,
                                const Real* V, const Real* W, double tau, Real* Gamma, Real* T,
                                Real* Pi, int32_t* rank, Real* F_H) {
  if (R < 1 || R > kMaxR) return fail(h, COPA_ERR_UNSUPPORTED, "Procrustes: R must be in [1, 80]");
  const ProcLayout L = proc_layout(R);
  const size_t smem = L.doubles * sizeof(double);
  if (smem > 227 * 1024) return fail(h, COPA_ERR_UNSUPPORTED, "Procrustes: R too large for shared memory");
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_procrustes<Real>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  int per_sm = 0;
  if ((st = cuda_check(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_procrustes<Real>,
                                                                        32, smem),
                       "occupancy")) != COPA_OK)
    return st;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)h->num_sms * per_sm;
  if (blocks > X.K) blocks = X.K > 0 ? X.K : 1;
  const int64_t* order = nullptr;
  if ((st = get_schedule(h, X, &order)) != COPA_OK) return st;
  int* counter = nullptr;
  if ((st = ws_get(h, SLOT_COUNTER, 64, (void**)&counter)) != COPA_OK) return st;
  double* part = nullptr;
  if (F_H) {
    if ((st = ws_get(h, SLOT_PARTIAL, (size_t)blocks * R * R * sizeof(double), (void**)&part)) != COPA_OK)
      return st;
  }
  if ((st = cuda_check(h, cudaMemsetAsync(counter, 0, sizeof(int), h->stream), "memset")) != COPA_OK)
    return st;
  k_procrustes<Real><<<(unsigned)blocks, 32, smem, h->stream>>>(
      X, R, H, V, W, tau, Gamma, T, Pi, rank, part, order, counter, h->d_status);
  if ((st = cuda_check(h, cudaGetLastError(), "k_procrustes launch")) != COPA_OK) return st;
  if (F_H) {
    k_reduce_partials<Real><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, (int)blocks, R * R, F_H);
    if ((st = cuda_check(h, cudaGetLastError(), "k_reduce_partials launch")) != COPA_OK) return st;
  }
  return COPA_OK;
}

template copa_status_t launch_procrustes<float>(copa_ctx*, const TensorView&, int, const float*,
                                                const float*, const float*, double, float*,
                                                float*, float*, int32_t*, float*);
template copa_status_t launch_procrustes<double>(copa_ctx*, const TensorView&, int, const double*,
                                                 const double*, const double*, double, double*,
                                                 double*, double*, int32_t*, double*);

}  // namespace copa
