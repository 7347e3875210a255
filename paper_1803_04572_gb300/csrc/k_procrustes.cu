// Procrustes step of COPA (Sec. 3.1, Eq. solv_Q; Algorithm 1 per-subject loop) and the
// fused mode-1 MTTKRP, for all subjects in one persistent launch: one warp per subject,
// dynamic scheduling over a largest-first subject order.
//
// For subject k: P_k = X_k V (I_k x R), E_k = S_k H^T, A_k = P_k E_k. With the thin SVD
// A_k = B D C^T, the update is Q_k = B C^T over the singular values kept by the rank
// cut sigma_i^2 > tau sigma_max^2. It is computed without forming A_k^T A_k (which would
// square the condition number) by one-sided (Hestenes) Jacobi on row vectors:
//   * I_k <= R ("wide"): rotate the I_k rows of A_k until they are orthogonal,
//     Z = U A_k with U orthogonal (accumulated). Then A_k = U^T Z = U^T Sigma C^T, and
//     Q_k = U^T C_K^T (kept columns), a product of orthonormal factors.
//   * I_k > R ("tall"): a blocked Householder QR of the streamed rows gives
//     A_k = Q_A R_A (R_A upper triangular R x R); Hestenes on the rows of R_A gives
//     Sigma and C, so Omega = C_K Sigma_K^{-1} C_K^T and Q_k = A_k Omega (rows recomputed
//     in a second pass over X_k, which also accumulates T_k = sum_i q_i^T p_i).
// Outputs per subject: Q_k rows (S x R), T_k = Q_k^T P_k (= Y_k V, R x R), optionally
// Pi_k = Q_k^T Q_k = C_K C_K^T and the rank |K|; and F_H = sum_k T_k S_k through per-warp
// FP64 partial sums. The same code runs in float (mixed) or double (plain FP64).
#include "copa_internal.cuh"

namespace copa {

namespace {

constexpr int kMaxSweeps = 30;

template <typename Real>
struct Tol;
template <>
struct Tol<float> {
  static __device__ __forceinline__ float v() { return 1e-6f; }
};
template <>
struct Tol<double> {
  static __device__ __forceinline__ double v() { return 1e-14; }
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }

struct Lay {
  int R, ld, npk, np;   // np: max pairs per round
  size_t Hs, Es, Zb, Pb, Ub, pv, av, al, vb, misc, cs, pq, pk, total;  // in Real units
};

template <typename Real>
__host__ __device__ inline Lay lay_of(int R) {
  Lay L;
  L.R = R;
  L.ld = (R & 1) ? R + 2 : R + 1;   // odd leading dimension
  L.npk = R * (R + 1) / 2;
  L.np = R / 2 + 1;
  size_t o = 0;
  const size_t m = (size_t)R * L.ld;
  L.Hs = o; o += m;
  L.Es = o; o += m;
  L.Zb = o; o += 2 * m;
  L.Pb = o; o += m;
  L.Ub = o; o += m;
  L.pv = o; o += R;
  L.av = o; o += R;
  L.al = o; o += R;
  L.vb = o; o += R + 1;
  L.misc = o; o += 8;
  L.cs = o; o += 2 * L.np;
  L.pq = o; o += (2 * L.np * sizeof(int) + sizeof(Real) - 1) / sizeof(Real);
  L.pk = o; o += (L.npk * sizeof(uint16_t) + sizeof(Real) - 1) / sizeof(Real);
  L.total = o;
  return L;
}

__device__ __forceinline__ int rr_elem(int pos, int round, int n2) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (n2 - 1));
}

// Householder QR update of the stacked [R_A (R x R, rows 0..R-1 of Z); block (nb rows,
// rows R..R+nb-1 of Z)]: afterwards Z[0..R-1] holds the new R factor and the block is 0.
template <typename Real>
__device__ void tsqr_block(Real* Z, int ld, int R, int nb, Real* vb, Real* misc) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < R; ++j) {
    if (lane == (j & 31)) {
      const Real x0 = Z[j * ld + j];
      Real ss = Real(0);
      for (int i = 0; i < nb; ++i) {
        const Real v = Z[(R + i) * ld + j];
        ss += v * v;
      }
      Real tau = Real(0);
      if (ss > Real(0)) {
        const Real nrm = sqrt(x0 * x0 + ss);
        const Real beta = x0 >= Real(0) ? -nrm : nrm;
        tau = (beta - x0) / beta;
        const Real scale = Real(1) / (x0 - beta);
        for (int i = 0; i < nb; ++i) {
          vb[i] = Z[(R + i) * ld + j] * scale;
          Z[(R + i) * ld + j] = Real(0);
        }
        Z[j * ld + j] = beta;
      }
      misc[0] = tau;
    }
    __syncwarp();
    const Real tau = misc[0];
    if (tau != Real(0)) {
      for (int c = j + 1 + ((lane - (j + 1)) & 31); c < R; c += 32) {
        Real w = Z[j * ld + c];
        for (int i = 0; i < nb; ++i) w += vb[i] * Z[(R + i) * ld + c];
        w *= tau;
        Z[j * ld + c] -= w;
        for (int i = 0; i < nb; ++i) Z[(R + i) * ld + c] -= vb[i] * w;
      }
    }
    __syncwarp();
  }
}

template <typename Real>
__global__ void __launch_bounds__(32) k_procrustes(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V,
    const Real* __restrict__ W, double tau_rank, Real* __restrict__ Q, Real* __restrict__ T,
    Real* __restrict__ Pi, int32_t* __restrict__ rank, double* __restrict__ fh_partial,
    const int64_t* __restrict__ order, int* __restrict__ counter,
    unsigned long long* __restrict__ fma_count) {
  extern __shared__ unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const Lay L = lay_of<Real>(R);
  const int ld = L.ld;
  const int lane = threadIdx.x;
  Real* Hs = sm + L.Hs;   // H[t][r] at t*ld + r
  Real* Es = sm + L.Es;   // E[r][t] = w_r H[t][r]
  Real* Zb = sm + L.Zb;   // rows 0..R-1: A_k rows / R_A / c_j; rows R..2R-1: block, B, T
  Real* Pb = sm + L.Pb;   // wide: p rows; tall: Omega
  Real* Ub = sm + L.Ub;   // wide: U
  Real* pv = sm + L.pv;
  Real* av = sm + L.av;
  Real* al = sm + L.al;
  Real* vb = sm + L.vb;
  Real* misc = sm + L.misc;
  Real* cs = sm + L.cs;
  int* pq = reinterpret_cast<int*>(sm + L.pq);
  uint16_t* pk = reinterpret_cast<uint16_t*>(sm + L.pk);
  const Real tol = Tol<Real>::v();
  // work tally (lane 0): multiply-adds the algorithm performs, for the roofline
  unsigned long long fma = 0;

  for (int i = lane; i < R * R; i += 32) Hs[(i / R) * ld + (i % R)] = H[i];
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
    const int Ik = (int)(r1 - r0 < (int64_t)R + 1 ? r1 - r0 : (int64_t)R + 1);
    const bool wide = Ik <= R;
    const int m = wide ? Ik : R;
    const unsigned long long nnzk = (unsigned long long)(X.row_ptr[r1] - X.row_ptr[r0]);
    const unsigned long long ik = (unsigned long long)(r1 - r0), RR = (unsigned long long)R * R;
    // rows: p_i and a_i; tall: Householder QR (~R^2 per row) and the second pass
    fma += nnzk * R + ik * RR;
    if (!wide) fma += ik * RR + nnzk * R + 3 * ik * RR + 2 * RR * R;
    else fma += 2ull * m * m * R + 2ull * RR * m;
    fma += 2ull * m * R;   // norms and normalisation

    // ---- E = S_k H^T; clear R_A (tall) or nothing (wide) and G ----
    for (int r = lane; r < R; r += 32) al[r] = W[k * R + r];
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, t = e - r * R;
      Es[r * ld + t] = al[r] * Hs[t * ld + r];
      if (!wide) Zb[r * ld + t] = Real(0);
    }
    __syncwarp();

    // ---- pass 1 over the rows: p_i, a_i = p_i E; wide: keep both; tall: G, TSQR ----
    int nb = 0;
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
      for (int r = lane; r < R; r += 32) {
        Real acc = Real(0);
        for (int64_t t = a; t < b; ++t)
          acc += load_x<Real>(X, t) * __ldg(V + (int64_t)__ldg(X.col + t) * R + r);
        pv[r] = acc;
      }
      __syncwarp();
      const int row = wide ? (int)(i - r0) : R + nb;
      for (int t = lane; t < R; t += 32) {
        Real acc = Real(0);
        for (int r = 0; r < R; ++r) acc += pv[r] * Es[r * ld + t];
        Zb[row * ld + t] = acc;
        if (wide) Pb[row * ld + t] = pv[t];
      }
      __syncwarp();
      if (!wide && ++nb == R) {
        tsqr_block<Real>(Zb, ld, R, nb, vb, misc);
        nb = 0;
      }
    }
    if (!wide && nb > 0) tsqr_block<Real>(Zb, ld, R, nb, vb, misc);

    // ---- Hestenes one-sided Jacobi on rows 0..m-1 of Zb (U accumulated if wide) ----
    if (wide)
      for (int e = lane; e < m * m; e += 32) Ub[(e / m) * ld + (e % m)] = (e / m == e % m) ? Real(1) : Real(0);
    __syncwarp();
    const int n2 = m + (m & 1);
    for (int sweep = 0; sweep < kMaxSweeps && n2 > 1; ++sweep) {
      int nrot = 0, ntest = 0;
      for (int round = 0; round < n2 - 1; ++round) {
        for (int pj = lane; pj < n2 / 2; pj += 32) {
          int ii = rr_elem(pj, round, n2), jj = rr_elem(n2 - 1 - pj, round, n2);
          if (ii > jj) { const int tmp = ii; ii = jj; jj = tmp; }
          if (jj >= m) continue;
          ++ntest;
          Real* zi = Zb + ii * ld;
          Real* zj = Zb + jj * ld;
          Real aa = Real(0), bb = Real(0), gg = Real(0);
          for (int t = 0; t < R; ++t) {
            const Real x = zi[t], y = zj[t];
            aa += x * x;
            bb += y * y;
            gg += x * y;
          }
          if (gg != Real(0) && fabs(gg) > tol * sqrt(aa * bb)) {
            const Real zeta = (bb - aa) / (Real(2) * gg);
            Real tt;
            if (fabs(zeta) > Real(1e15)) tt = Real(0.5) / zeta;
            else tt = (zeta >= Real(0) ? Real(1) : Real(-1)) / (fabs(zeta) + sqrt(Real(1) + zeta * zeta));
            const Real c = rsqrt_(Real(1) + tt * tt), s = c * tt;
            for (int t = 0; t < R; ++t) {
              const Real x = zi[t], y = zj[t];
              zi[t] = c * x - s * y;
              zj[t] = s * x + c * y;
            }
            if (wide) {
              Real* ui = Ub + ii * ld;
              Real* uj = Ub + jj * ld;
              for (int t = 0; t < m; ++t) {
                const Real x = ui[t], y = uj[t];
                ui[t] = c * x - s * y;
                uj[t] = s * x + c * y;
              }
            }
            ++nrot;
          }
        }
        __syncwarp();
      }
      const int tot_rot = warp_sum(nrot), tot_test = warp_sum(ntest);
      fma += (unsigned long long)tot_test * 3 * R + (unsigned long long)tot_rot * 4 * (R + (wide ? m : 0));
      if (tot_rot == 0) break;
    }

    // ---- singular values, rank cut, normalised right singular vectors c_j ----
    Real amax = Real(0);
    for (int j = lane; j < m; j += 32) {
      Real acc = Real(0);
      for (int t = 0; t < R; ++t) acc += Zb[j * ld + t] * Zb[j * ld + t];
      al[j] = acc;
      amax = acc > amax ? acc : amax;
    }
    amax = warp_max(amax);
    int kept = 0;
    for (int j = lane; j < m; j += 32) {
      const bool keep = amax > Real(0) && (double)al[j] > tau_rank * (double)amax;
      al[j] = keep ? rsqrt_(al[j]) : Real(0);   // 1 / sigma_j, 0 if dropped
      kept += keep ? 1 : 0;
    }
    kept = warp_sum(kept);
    if (rank && lane == 0) rank[k] = kept;
    __syncwarp();
    for (int e = lane; e < m * R; e += 32) {
      const int j = e / R, t = e - j * R;
      Zb[j * ld + t] *= al[j];
    }
    __syncwarp();

    Real* Tk = T + k * R * R;
    if (wide) {
      // Q rows: q_i = sum_j U[j][i] c_j
      for (int e = lane; e < m * R; e += 32) {
        const int i = e / R, t = e - i * R;
        Real acc = Real(0);
        for (int j = 0; j < m; ++j) acc += Ub[j * ld + i] * Zb[j * ld + t];
        Q[(r0 + i) * R + t] = acc;
      }
      // B = U P -> rows R.. of Zb
      for (int e = lane; e < m * R; e += 32) {
        const int j = e / R, s = e - j * R;
        Real acc = Real(0);
        for (int i = 0; i < m; ++i) acc += Ub[j * ld + i] * Pb[i * ld + s];
        Zb[(R + j) * ld + s] = acc;
      }
      __syncwarp();
      for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, s = e - r * R;
        Real acc = Real(0), pacc = Real(0);
        for (int j = 0; j < m; ++j) {
          acc += Zb[j * ld + r] * Zb[(R + j) * ld + s];
          pacc += Zb[j * ld + r] * Zb[j * ld + s];
        }
        Tk[e] = acc;
        if (Pi) Pi[k * R * R + e] = pacc;
        if (fh) fh[e] += (double)acc * (double)W[k * R + s];
      }
      __syncwarp();
    } else {
      // Omega = sum_j c_j c_j^T / sigma_j -> Pb; Pi -> global; clear the T accumulator
      for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, t = e - r * R;
        Real acc = Real(0), pacc = Real(0);
        for (int j = 0; j < R; ++j) {
          const Real cc = Zb[j * ld + r] * Zb[j * ld + t];
          acc += cc * al[j];
          pacc += cc;
        }
        Pb[r * ld + t] = acc;
        if (Pi) Pi[k * R * R + e] = pacc;
        Zb[(R + r) * ld + t] = Real(0);
      }
      __syncwarp();
      // pass 2: q_i = (p_i E) Omega, T_k += q_i^T p_i
      for (int64_t i = r0; i < r1; ++i) {
        const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
        for (int r = lane; r < R; r += 32) {
          Real acc = Real(0);
          for (int64_t t = a; t < b; ++t)
            acc += load_x<Real>(X, t) * __ldg(V + (int64_t)__ldg(X.col + t) * R + r);
          pv[r] = acc;
        }
        __syncwarp();
        for (int t = lane; t < R; t += 32) {
          Real acc = Real(0);
          for (int r = 0; r < R; ++r) acc += pv[r] * Es[r * ld + t];
          av[t] = acc;
        }
        __syncwarp();
        for (int t = lane; t < R; t += 32) {
          Real acc = Real(0);
          for (int r = 0; r < R; ++r) acc += av[r] * Pb[r * ld + t];
          Q[i * R + t] = acc;
          al[t] = acc;
        }
        __syncwarp();
        for (int e = lane; e < R * R; e += 32) {
          const int r = e / R, s = e - r * R;
          Zb[(R + r) * ld + s] += al[r] * pv[s];
        }
        __syncwarp();
      }
      for (int e = lane; e < R * R; e += 32) {
        const int r = e / R, s = e - r * R;
        const Real acc = Zb[(R + r) * ld + s];
        Tk[e] = acc;
        if (fh) fh[e] += (double)acc * (double)W[k * R + s];
      }
      __syncwarp();
    }
  }
  if (fma_count && lane == 0) atomicAdd(fma_count, fma);
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
size_t procrustes_smem(int R) {
  return lay_of<Real>(R).total * sizeof(Real);
}

template <typename Real>
copa_status_t launch_procrustes(copa_ctx* h, const TensorView& X, int R, const Real* H,
                                const Real* V, const Real* W, double tau, Real* Q, Real* T,
                                Real* Pi, int32_t* rank, Real* F_H) {
  const size_t smem = procrustes_smem<Real>(R);
  if (R < 1 || smem > 227 * 1024)
    return fail(h, COPA_ERR_UNSUPPORTED, "Procrustes: R too large for shared memory at this precision");
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
  unsigned long long* fma_count = reinterpret_cast<unsigned long long*>(counter + 2);
  double* part = nullptr;
  if (F_H) {
    if ((st = ws_get(h, SLOT_PARTIAL, (size_t)blocks * R * R * sizeof(double), (void**)&part)) != COPA_OK)
      return st;
  }
  if ((st = cuda_check(h, cudaMemsetAsync(counter, 0, 16, h->stream), "memset")) != COPA_OK)
    return st;
  k_procrustes<Real><<<(unsigned)blocks, 32, smem, h->stream>>>(X, R, H, V, W, tau, Q, T, Pi, rank, part,
                                                               order, counter, fma_count);
  if ((st = cuda_check(h, cudaGetLastError(), "k_procrustes launch")) != COPA_OK) return st;
  if (F_H) {
    k_reduce_partials<Real><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, (int)blocks, R * R, F_H);
    if ((st = cuda_check(h, cudaGetLastError(), "k_reduce_partials launch")) != COPA_OK) return st;
  }
  return COPA_OK;
}

template size_t procrustes_smem<float>(int);
template size_t procrustes_smem<double>(int);
template copa_status_t launch_procrustes<float>(copa_ctx*, const TensorView&, int, const float*,
                                                const float*, const float*, double, float*,
                                                float*, float*, int32_t*, float*);
template copa_status_t launch_procrustes<double>(copa_ctx*, const TensorView&, int, const double*,
                                                 const double*, const double*, double, double*,
                                                 double*, double*, int32_t*, double*);

}  // namespace copa
