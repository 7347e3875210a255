// MTTKRPs on the implicit Y (Algorithm 1, "F = Y_(n)(Khatri-Rao of the others)"), the
// factor Grams, rho and the cached Cholesky of G + rho I, the ADMM inner loops with the
// proximal operators of Sec. 3.3 (Eq. 8 update rules), and the FIT of Sec. 4.1.
//
// With Q_k from k_procrustes.cu and T_k = Q_k^T X_k V (Y_k = Q_k^T X_k never formed):
//   F_H = sum_k Y_k V S_k        = sum_k T_k S_k
//   F_W(k,s) = (H^T Y_k V)(s,s)  = sum_r H(r,s) T_k(r,s)
//   F_V = sum_k Y_k^T H S_k      = sum_k X_k^T (Q_k H S_k)
// so only F_V streams X again: u_i = q_i H S_k for every visit, then F_V = X^T U over a
// column-sorted copy of X; U^T U = sum_i u_i^T u_i comes with the first step.
#include <mutex>

#include <type_traits>

#include "copa_internal.cuh"

namespace copa {

namespace {

constexpr int kRegs = (kMaxR + 31) / 32;   // per-lane slots of an R-vector

// ------------------------------------------------------------------------------------
// F_H = sum_k T_k S_k: blocks reduce chunks of subjects, then a final FP64 reduction
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_mttkrp_h(int64_t K, int R, const Real* __restrict__ T,
                           const Real* __restrict__ W, double* __restrict__ part) {
  const int n = R * R;
  const int64_t per = (K + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = blockIdx.x * per, k1 = min(K, k0 + per);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int s = e % R;
    Real acc = Real(0);
    for (int64_t k = k0; k < k1; ++k) acc += T[k * n + e] * W[k * R + s];
    part[(size_t)blockIdx.x * n + e] = (double)acc;
  }
}

template <typename Real>
__global__ void k_reduce_rows(const double* __restrict__ part, int nparts, int n,
                              Real* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nparts; ++q) acc += part[(size_t)q * n + e];
    out[e] = (Real)acc;
  }
}

// ------------------------------------------------------------------------------------
// F_W(k,s) = sum_r H(r,s) T_k(r,s): a warp per subject, lanes over s
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_mttkrp_w(int64_t K, int R, const Real* __restrict__ T,
                           const Real* __restrict__ H, Real* __restrict__ F) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
  for (int64_t k = wid; k < K; k += nw) {
    for (int s = lane; s < R; s += 32) {
      Real acc = Real(0);
      for (int r = 0; r < R; ++r) acc += H[r * R + s] * T[k * R * R + r * R + s];
      F[k * R + s] = acc;
    }
  }
}

// ------------------------------------------------------------------------------------
// F_V as a gather: F_V = sum_k X_k^T U_k with U_k = Q_k H S_k.
//  1. k_uvec: u_i = q_i H S_k for every visit row (warp per subject, largest first),
//     written to U (S x R); U^T U = sum_i u_i^T u_i accumulated in registers, each lane
//     owning a 5 x 10 tile of the R x R result (R <= 40; packed shared-memory sums above).
//  2. k_spmm_csc: F_V(j,:) = sum_{i in column j} x_ij u_i over a column-sorted copy of X
//     (built once per tensor); each warp takes a fixed chunk of nonzeros, so hot
//     columns are split evenly, and flushes one atomic add per (chunk, column).
// ------------------------------------------------------------------------------------
constexpr int kTR = 5, kTC = 10;   // U^T U register tile per lane (8 x 4 tiles cover 40 x 40)
constexpr int kUNT = 256;          // threads per block of k_uvec
constexpr int kChunk = 256;        // nonzeros per warp in k_spmm_csc

template <typename Real, bool kTiles>
__global__ void __launch_bounds__(kUNT) k_uvec(
    TensorView X, int R, const Real* __restrict__ Q, const Real* __restrict__ H,
    const Real* __restrict__ W, Real* __restrict__ U, double* __restrict__ utu_part,
    const int64_t* __restrict__ order, int* __restrict__ counter) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kUNT / 32;
  const int npk = R * (R + 1) / 2;
  Real* Hs = reinterpret_cast<Real*>(smem_raw);                      // R x R
  Real* wv = Hs + R * R + (size_t)warp * (2 * R + (kTiles ? 0 : npk));
  Real* uv = wv + R;
  Real* uacc = uv + R;                                               // packed U^T U (no tiles)
  uint16_t* pk = reinterpret_cast<uint16_t*>(Hs + R * R + (size_t)nw * (2 * R + (kTiles ? 0 : npk)));
  for (int e = threadIdx.x; e < R * R; e += kUNT) Hs[e] = H[e];
  if (!kTiles) {
    for (int e = threadIdx.x; e < npk; e += kUNT) {
      int r = 0, rem = e;
      while (rem >= R - r) { rem -= R - r; ++r; }
      pk[e] = (uint16_t)((r << 8) | (r + rem));
    }
    for (int e = lane; e < npk; e += 32) uacc[e] = Real(0);
  }
  __syncthreads();
  const int tr = lane >> 2, tc = lane & 3;
  Real acc[kTiles ? kTR : 1][kTiles ? kTC : 1];
#pragma unroll
  for (int a = 0; a < (kTiles ? kTR : 1); ++a)
#pragma unroll
    for (int b = 0; b < (kTiles ? kTC : 1); ++b) acc[a][b] = Real(0);

  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= X.K) break;
    const int64_t k = order ? order[idx] : idx;
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    for (int s = lane; s < R; s += 32) wv[s] = W[k * R + s];
    __syncwarp();
    for (int64_t i = r0; i < r1; ++i) {
      const Real* qi = Q + i * R;
      for (int s = lane; s < R; s += 32) {
        Real a0 = Real(0), a1 = Real(0);
        int r = 0;
        for (; r + 1 < R; r += 2) {
          a0 += __ldg(qi + r) * Hs[r * R + s];
          a1 += __ldg(qi + r + 1) * Hs[(r + 1) * R + s];
        }
        if (r < R) a0 += __ldg(qi + r) * Hs[r * R + s];
        const Real u = (a0 + a1) * wv[s];
        uv[s] = u;
        U[i * R + s] = u;
      }
      __syncwarp();
      if (utu_part) {
        if (kTiles) {
#pragma unroll
          for (int aa = 0; aa < kTR; ++aa) {
            const int r = tr * kTR + aa;
            const Real ur = r < R ? uv[r] : Real(0);
#pragma unroll
            for (int bb = 0; bb < kTC; ++bb) {
              const int s = tc * kTC + bb;
              if (s < R) acc[aa][bb] += ur * uv[s];
            }
          }
        } else {
          for (int e = lane; e < npk; e += 32) {
            const int r = pk[e] >> 8, s = pk[e] & 255;
            uacc[e] += uv[r] * uv[s];
          }
        }
      }
      __syncwarp();
    }
  }
  if (utu_part) {
    double* up = utu_part + ((size_t)blockIdx.x * nw + warp) * R * R;
    if (kTiles) {
#pragma unroll
      for (int aa = 0; aa < kTR; ++aa)
#pragma unroll
        for (int bb = 0; bb < kTC; ++bb) {
          const int r = tr * kTR + aa, s = tc * kTC + bb;
          if (r < R && s < R) up[r * R + s] = (double)acc[aa][bb];
        }
    } else {
      for (int e = lane; e < npk; e += 32) {
        const int r = pk[e] >> 8, s = pk[e] & 255;
        up[r * R + s] = (double)uacc[e];
        if (r != s) up[s * R + r] = (double)uacc[e];
      }
    }
  }
}

// Compensated (two-float) accumulation of FP32 addends: hi + lo carries the sum to about
// twice the float precision (Knuth's TwoSum per addend) at a few float operations, where a
// float-to-double conversion and a double add per addend would run on the FP64 unit
// (1/58 of the FP32 rate on this part). The FP64 path accumulates in double directly.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x, bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}
__device__ __forceinline__ void two_sum_add(double& hi, double& lo, double x) {
  hi += x;
  (void)lo;
}

// Tiled form of step 1 for R <= 48: a block takes kVT consecutive visit rows at a time
// (rows of any subjects; the subject of a row comes from the row -> subject map), forms
// the kVT x R tile of U = (Q H) .* W(k(i), :) as a small GEMM from shared memory (a thread
// owns 4 rows x NC columns), writes the tile out coalesced, and adds the tile's Gram to
// U^T U: four groups of 64 threads take 32 rows each, a thread owning an NC x NC block,
// summed in FP32 within a tile and across tiles as a compensated float pair (double at the end).
constexpr int kVT = 128;    // rows per tile
constexpr int kVNT = 256;   // threads per block

template <typename Real, int NC>   // NC = ceil(R / 8)
__global__ void __launch_bounds__(kVNT, 2) k_uvec_tiled(int64_t S, int R, const Real* __restrict__ Q,
                                                       const Real* __restrict__ H, const Real* __restrict__ W,
                                                       const int32_t* __restrict__ row_subj, Real* __restrict__ U,
                                                       double* __restrict__ utu_part) {
  constexpr int HL = 8 * NC;   // padded row length of H in shared memory
  extern __shared__ unsigned char smem_raw[];
  Real* Hs = reinterpret_cast<Real*>(smem_raw);   // Hs[r * HL + c] = H(r, c), zero-padded
  Real* Ts = Hs + HL * HL;                        // kVT x ld: Q rows, then U rows
  const int ld = R + 1;
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;                            // GEMM mapping
  const int g = tid >> 6, gp = (tid >> 3) & 7, gq = tid & 7;        // Gram mapping
  for (int e = tid; e < HL * HL; e += kVNT) {
    const int r = e / HL, c = e - r * HL;
    Hs[e] = (r < R && c < R) ? H[r * R + c] : Real(0);
  }
  Real ghi[NC][NC], glo[NC][NC];   // this thread's U^T U block, compensated
#pragma unroll
  for (int a = 0; a < NC; ++a)
#pragma unroll
    for (int b = 0; b < NC; ++b) ghi[a][b] = glo[a][b] = Real(0);

  for (int64_t i0 = (int64_t)blockIdx.x * kVT; i0 < S; i0 += (int64_t)gridDim.x * kVT) {
    const int nrow = (int)min((int64_t)kVT, S - i0);
    __syncthreads();   // the previous tile's Gram reads are done (and Hs is filled)
    const Real* qt = Q + i0 * R;
    for (int e = tid; e < kVT * R; e += kVNT) {
      const int i = e / R, c = e - i * R;
      Ts[i * ld + c] = i < nrow ? qt[e] : Real(0);
    }
    __syncthreads();
    Real acc[4][NC];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < NC; ++b) acc[a][b] = Real(0);
#pragma unroll 2
    for (int r = 0; r < R; ++r) {
      Real qa[4], hb[NC];
#pragma unroll
      for (int a = 0; a < 4; ++a) qa[a] = Ts[(ty * 4 + a) * ld + r];
#pragma unroll
      for (int b = 0; b < NC; ++b) hb[b] = Hs[r * HL + tx * NC + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) acc[a][b] += qa[a] * hb[b];
    }
    __syncthreads();   // every read of the Q tile is done
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ty * 4 + a;
      const int64_t k = i < nrow ? (int64_t)row_subj[i0 + i] : -1;
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        const int c = tx * NC + b;
        if (c < R) Ts[i * ld + c] = k >= 0 ? acc[a][b] * W[k * R + c] : Real(0);
      }
    }
    __syncthreads();
    Real* ut = U + i0 * R;
    for (int e = tid; e < nrow * R; e += kVNT) {
      const int i = e / R, c = e - i * R;
      ut[e] = Ts[i * ld + c];
    }
    if (utu_part) {
      Real sacc[NC][NC];
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) sacc[a][b] = Real(0);
      for (int i = g * (kVT / 4); i < (g + 1) * (kVT / 4); ++i) {
        Real ua[NC], ub[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          const int c = gp * NC + a;
          ua[a] = c < R ? Ts[i * ld + c] : Real(0);
        }
#pragma unroll
        for (int b = 0; b < NC; ++b) {
          const int c = gq * NC + b;
          ub[b] = c < R ? Ts[i * ld + c] : Real(0);
        }
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
          for (int b = 0; b < NC; ++b) sacc[a][b] += ua[a] * ub[b];
      }
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) two_sum_add(ghi[a][b], glo[a][b], sacc[a][b]);
    }
  }
  if (utu_part) {
    double* up = utu_part + ((size_t)blockIdx.x * 4 + g) * R * R;
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int b = 0; b < NC; ++b) {
        const int r = gp * NC + a, c = gq * NC + b;
        if (r < R && c < R) up[r * R + c] = (double)ghi[a][b] + (double)glo[a][b];
      }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_spmm_csc(int64_t nnz, int J, int R, const int64_t* __restrict__ cptr,
                                                  const int32_t* __restrict__ crow, const Real* __restrict__ cval,
                                                  const Real* __restrict__ U, Real* __restrict__ F) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (nnz + kChunk - 1) / kChunk;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwt = (gridDim.x * (int64_t)blockDim.x) >> 5;
  for (int64_t c = wid; c < nchunks; c += nwt) {
    const int64_t e0 = c * kChunk, e1 = min(nnz, e0 + kChunk);
    // column holding e0: last j with cptr[j] <= e0
    int lo = 0, hi = J;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (cptr[mid] <= e0) lo = mid; else hi = mid;
    }
    int j = lo;
    int64_t jend = cptr[j + 1];
    Real a0 = Real(0), a1 = Real(0), a2 = Real(0);
    for (int64_t b0 = e0; b0 < e1; b0 += 32) {
      const int n = (int)min((int64_t)32, e1 - b0);
      int row = 0;
      Real x = Real(0);
      if (lane < n) {
        row = __ldg(crow + b0 + lane);
        x = __ldg(cval + b0 + lane);
      }
      for (int q = 0; q < n; ++q) {
        const int64_t e = b0 + q;
        while (e >= jend) {   // column boundary: flush and move on
          if (a0 != Real(0) && lane < R) atomicAdd(F + (int64_t)j * R + lane, a0);
          if (a1 != Real(0) && lane + 32 < R) atomicAdd(F + (int64_t)j * R + lane + 32, a1);
          if (a2 != Real(0) && lane + 64 < R) atomicAdd(F + (int64_t)j * R + lane + 64, a2);
          a0 = a1 = a2 = Real(0);
          ++j;
          jend = cptr[j + 1];
        }
        const int rq = __shfl_sync(0xffffffffu, row, q);
        const Real xq = __shfl_sync(0xffffffffu, x, q);
        const Real* ur = U + (int64_t)rq * R;
        if (lane < R) a0 += xq * __ldg(ur + lane);
        if (lane + 32 < R) a1 += xq * __ldg(ur + lane + 32);
        if (lane + 64 < R) a2 += xq * __ldg(ur + lane + 64);
      }
    }
    if (a0 != Real(0) && lane < R) atomicAdd(F + (int64_t)j * R + lane, a0);
    if (a1 != Real(0) && lane + 32 < R) atomicAdd(F + (int64_t)j * R + lane + 32, a1);
    if (a2 != Real(0) && lane + 64 < R) atomicAdd(F + (int64_t)j * R + lane + 64, a2);
  }
}

// column-sorted copy of X: histogram of columns, exclusive scan, scatter (row index and
// value of every nonzero; the order inside a column is arbitrary). Code frequencies are
// heavy-tailed, so both passes aggregate before touching a shared counter: the histogram
// counts in shared memory per block (J <= kHistSmem), the scatter claims positions once
// per (warp, column) with the lanes that hold the same column.
constexpr int kHistSmem = 12288;

__global__ void k_csc_hist(TensorView X, int64_t* __restrict__ cnt) {
  __shared__ unsigned int sh[kHistSmem];
  const bool local = X.J <= kHistSmem;
  if (local) {
    for (int j = threadIdx.x; j < X.J; j += blockDim.x) sh[j] = 0u;
    __syncthreads();
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < X.nnz; t += gridDim.x * (int64_t)blockDim.x) {
    const int c = X.col[t];
    if (local) atomicAdd(sh + c, 1u);
    else atomicAdd(reinterpret_cast<unsigned long long*>(cnt + c), 1ull);
  }
  if (local) {
    __syncthreads();
    for (int j = threadIdx.x; j < X.J; j += blockDim.x)
      if (sh[j]) atomicAdd(reinterpret_cast<unsigned long long*>(cnt + j), (unsigned long long)sh[j]);
  }
}

// one visit row per lane; the lanes step through their rows' nonzeros together
template <typename Real>
__global__ void k_csc_scatter(TensorView X, const int64_t* __restrict__ cptr, int64_t* __restrict__ cur,
                              int32_t* __restrict__ crow, Real* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = gridDim.x * (int64_t)blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < X.S; base += stride) {
    const int64_t i = base + lane;
    int64_t t = 0, e = 0;
    if (i < X.S) { t = X.row_ptr[i]; e = X.row_ptr[i + 1]; }
    while (true) {
      const bool act = t < e;
      const unsigned amask = __ballot_sync(0xffffffffu, act);
      if (amask == 0u) break;
      if (act) {
        const int c = X.col[t];
        const unsigned peers = __match_any_sync(amask, c);
        const int leader = __ffs(peers) - 1;
        unsigned long long pos0 = 0;
        if (lane == leader) pos0 = atomicAdd(reinterpret_cast<unsigned long long*>(cur + c), (unsigned long long)__popc(peers));
        pos0 = __shfl_sync(peers, pos0, leader);
        const int64_t pos = cptr[c] + (int64_t)pos0 + __popc(peers & ((1u << lane) - 1u));
        crow[pos] = (int32_t)i;
        cval[pos] = load_x<Real>(X, t);
        ++t;
      }
    }
  }
}

// Row-ordered form (every column lists its visit rows in ascending order up to a
// permutation inside 32-row steps; the order depends only on X, so F_V is summed in a fixed
// order and the gathers of a column walk U forward), for J <= kHistSmem: the visit rows
// are cut into nb contiguous ranges, one warp each. k_csc_count counts the columns of
// every range into rel[j * nb + b]; k_csc_colscan turns each column's counts into offsets
// over the ranges and its total; k_csc_place walks every range again, 32 rows at a time
// (lane = row, the rows' q-th nonzeros together), and puts each nonzero after the ones of
// its column already placed (ranks among equal columns from __match_any_sync, a
// shared-memory cursor per column).
__device__ __forceinline__ void csc_range(int64_t S, int nb, int b, int64_t* lo, int64_t* hi) {
  *lo = S * b / nb;
  *hi = S * (b + 1) / nb;
}

__global__ void __launch_bounds__(32) k_csc_count(TensorView X, int nb, int* __restrict__ rel) {
  extern __shared__ int cnt[];   // J counters
  const int lane = threadIdx.x, b = blockIdx.x;
  for (int j = lane; j < X.J; j += 32) cnt[j] = 0;
  __syncwarp();
  int64_t lo, hi;
  csc_range(X.S, nb, b, &lo, &hi);
  const int64_t t1 = X.row_ptr[hi];
  for (int64_t t = X.row_ptr[lo] + lane; t < t1; t += 32) atomicAdd(&cnt[X.col[t]], 1);
  __syncwarp();
  for (int j = lane; j < X.J; j += 32) rel[(int64_t)j * nb + b] = cnt[j];
}

// one warp per column: exclusive scan of its range counts in place, column total -> tot[j]
__global__ void k_csc_colscan(int J, int nb, int* __restrict__ rel, int64_t* __restrict__ tot) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= J) return;
  int* r = rel + (int64_t)j * nb;
  int run = 0;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int v = b0 + lane < nb ? r[b0 + lane] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += n;
    }
    if (b0 + lane < nb) r[b0 + lane] = run + incl - v;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) tot[j] = run;
}

template <typename Real>
__global__ void __launch_bounds__(32) k_csc_place(TensorView X, int nb, const int* __restrict__ rel,
                                                  const int64_t* __restrict__ cptr, int32_t* __restrict__ crow,
                                                  Real* __restrict__ cval) {
  extern __shared__ int cur[];   // J cursors
  const int lane = threadIdx.x, b = blockIdx.x;
  for (int j = lane; j < X.J; j += 32) cur[j] = 0;
  __syncwarp();
  int64_t lo, hi;
  csc_range(X.S, nb, b, &lo, &hi);
  for (int64_t i0 = lo; i0 < hi; i0 += 32) {
    const int64_t i = i0 + lane;
    int64_t t = 0, e = 0;
    if (i < hi) {
      t = X.row_ptr[i];
      e = X.row_ptr[i + 1];
    }
    int len = (int)(e - t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    for (int q = 0; q < len; ++q, ++t) {
      const bool act = t < e;
      const unsigned amask = __ballot_sync(0xffffffffu, act);
      int c = 0;
      unsigned peers = 0u;
      if (act) {
        c = X.col[t];
        peers = __match_any_sync(amask, c);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int64_t pos = cptr[c] + rel[(int64_t)c * nb + b] + cur[c] + rank;
        crow[pos] = (int32_t)i;
        cval[pos] = load_x<Real>(X, t);
      }
      __syncwarp();
      if (act && (peers >> lane) == 1u) cur[c] += __popc(peers);   // highest lane of its group
      __syncwarp();
    }
  }
}

// subject of every visit row
__global__ void k_row_subject(const int64_t* __restrict__ subj_ptr, int64_t K, int32_t* __restrict__ rs) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += gridDim.x * (int64_t)blockDim.x)
    for (int64_t i = subj_ptr[k]; i < subj_ptr[k + 1]; ++i) rs[i] = (int32_t)k;
}

__global__ void k_scan_cols(int64_t* __restrict__ v, int n) {
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int j = 0; j < n; ++j) { const int64_t x = v[j]; v[j] = acc; acc += x; }
    v[n] = acc;
  }
}

// ------------------------------------------------------------------------------------
// Column Gram G = A^T A of a rows x R matrix: block partials (FP64) then reduction
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_gram(const Real* __restrict__ A, int64_t rows, int R, double* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  Real* tile = reinterpret_cast<Real*>(smem_raw);   // 64 x R
  const int npk = R * (R + 1) / 2;
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = min(rows, i0 + per);
  double acc_d[8];
  int er[8], es[8];
  int nl = 0;
  for (int e = threadIdx.x; e < npk && nl < 8; e += blockDim.x, ++nl) {
    int r = 0, rem = e;
    while (rem >= R - r) { rem -= R - r; ++r; }
    er[nl] = r; es[nl] = r + rem; acc_d[nl] = 0.0;
  }
  for (int64_t c0 = i0; c0 < i1; c0 += 64) {
    const int nrow = (int)min((int64_t)64, i1 - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < nrow * R; t += blockDim.x) tile[t] = A[c0 * R + t];
    __syncthreads();
    for (int q = 0; q < nl; ++q) {
      Real acc = Real(0);
      for (int i = 0; i < nrow; ++i) acc += tile[i * R + er[q]] * tile[i * R + es[q]];
      acc_d[q] += (double)acc;
    }
  }
  for (int q = 0; q < nl; ++q) {
    part[(size_t)blockIdx.x * R * R + er[q] * R + es[q]] = acc_d[q];
    part[(size_t)blockIdx.x * R * R + es[q] * R + er[q]] = acc_d[q];
  }
}

// ------------------------------------------------------------------------------------
// G = Ga .* Gb, rho = tr(G)/R, L = chol(G + rho I) (FP64), Ginv = L^{-T} L^{-1}
// One block; Ginv is stored with leading dimension R + 1 for conflict-free reads.
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_chol(const double* __restrict__ Ga, const double* __restrict__ Gb, int R,
                       Real* __restrict__ Ginv, double* __restrict__ rho_out,
                       int* __restrict__ status) {
  extern __shared__ double sm[];
  double* A = sm;             // R x R, becomes L (lower)
  double* Li = A + R * R;     // R x R, L^{-1} (lower)
  __shared__ double rho_s;
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < R * R; e += nt) A[e] = Ga[e] * (Gb ? Gb[e] : 1.0);
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < R; ++i) tr += A[i * R + i];
    rho_s = tr / R;
    bad = !(rho_s > 0.0) || !isfinite(rho_s);
  }
  __syncthreads();
  for (int i = tid; i < R; i += nt) A[i * R + i] += rho_s;
  __syncthreads();
  // right-looking Cholesky
  for (int j = 0; j < R; ++j) {
    if (tid == 0) {
      const double d = A[j * R + j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      A[j * R + j] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double ljj = A[j * R + j];
    for (int i = j + 1 + tid; i < R; i += nt) A[i * R + j] /= ljj;
    __syncthreads();
    for (int e = tid; e < (R - j - 1) * (R - j - 1); e += nt) {
      const int i = j + 1 + e / (R - j - 1), c = j + 1 + e % (R - j - 1);
      if (c <= i) A[i * R + c] -= A[i * R + j] * A[c * R + j];
    }
    __syncthreads();
  }
  // L^{-1}: column c solves L x = e_c by forward substitution (one thread per column)
  for (int c = tid; c < R; c += nt) {
    for (int i = 0; i < R; ++i) {
      double acc = (i == c) ? 1.0 : 0.0;
      for (int t = c; t < i; ++t) acc -= A[i * R + t] * Li[t * R + c];
      Li[i * R + c] = (i < c) ? 0.0 : acc / A[i * R + i];
    }
  }
  __syncthreads();
  // Ginv = Li^T Li
  for (int e = tid; e < R * R; e += nt) {
    const int r = e / R, s = e % R;
    double acc = 0.0;
    for (int t = max(r, s); t < R; ++t) acc += Li[t * R + r] * Li[t * R + s];
    Ginv[r * (R + 1) + s] = (Real)acc;
  }
  if (tid == 0) {
    *rho_out = rho_s;
    if (bad) set_status(status, COPA_ERR_NUMERIC, 1);
  }
}

// ADMM row loop shared by H, V and the fused W kernel. f, zb, d hold the lane's
// components (s = lane + 32 q); bv is a per-warp shared R-vector.
template <typename Real>
__device__ __forceinline__ void admm_row(int R, const Real* __restrict__ Gi, Real rho,
                                         Real lam_over_rho, int c, int n_inner, const Real* f,
                                         Real* zb, Real* d, Real* bv) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < n_inner; ++it) {
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      if (s < R) bv[s] = f[q] + rho * (zb[q] + d[q]);
    }
    __syncwarp();
    Real z[kRegs];
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      Real acc = Real(0);
      if (s < R)
        for (int t = 0; t < R; ++t) acc += Gi[s * (R + 1) + t] * bv[t];
      z[q] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const Real nz = prox<Real>(z[q] - d[q], c, lam_over_rho);
      d[q] = d[q] + nz - z[q];
      zb[q] = nz;
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_admm_rows(const Real* __restrict__ F,
                                                   const Real* __restrict__ Ginv,
                                                   const double* __restrict__ rho_dev, int n_inner,
                                                   int c, double lam, Real* __restrict__ Zbar,
                                                   Real* __restrict__ D, int64_t rows, int R) {
  extern __shared__ unsigned char smem_raw[];
  Real* Gi = reinterpret_cast<Real*>(smem_raw);          // R x (R+1)
  Real* bvall = Gi + R * (R + 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* bv = bvall + warp * R;
  for (int e = threadIdx.x; e < R * (R + 1); e += blockDim.x) Gi[e] = Ginv[e];
  __syncthreads();
  const double rho = *rho_dev;
  const Real lor = (Real)(lam / rho);
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
  for (int64_t i = wid; i < rows; i += nw) {
    Real f[kRegs], zb[kRegs], d[kRegs];
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      f[q] = s < R ? F[i * R + s] : Real(0);
      zb[q] = s < R ? Zbar[i * R + s] : Real(0);
      d[q] = s < R ? D[i * R + s] : Real(0);
    }
    admm_row<Real>(R, Gi, (Real)rho, lor, c, n_inner, f, zb, d, bv);
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      if (s < R) { Zbar[i * R + s] = zb[q]; D[i * R + s] = d[q]; }
    }
    __syncwarp();
  }
}

// One inner ADMM iteration over all rows (the early-stopping form of the update): a warp
// per row does z = (G + rho I)^{-1} (f + rho (zbar + d)), zbar' = prox(z - d),
// d' = d + zbar' - z, and the grid sums ||zbar' - z||^2, ||zbar'||^2, ||zbar' - zbar||^2 into
// acc[0..2] (FP64 atomics, one per block). Returns at once once *done is set.
template <typename Real>
__global__ void __launch_bounds__(256) k_admm_iter(const Real* __restrict__ F, const Real* __restrict__ Ginv,
                                                   const double* __restrict__ rho_dev, int c, double lam,
                                                   Real* __restrict__ Zbar, Real* __restrict__ D, int64_t rows,
                                                   int R, const int* __restrict__ done, double* __restrict__ acc) {
  if (*done) return;
  extern __shared__ unsigned char smem_raw[];
  Real* Gi = reinterpret_cast<Real*>(smem_raw);          // R x (R+1)
  Real* bvall = Gi + R * (R + 1);
  __shared__ double red[3][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* bv = bvall + warp * R;
  for (int e = threadIdx.x; e < R * (R + 1); e += blockDim.x) Gi[e] = Ginv[e];
  __syncthreads();
  const double rho = *rho_dev;
  const Real rr = (Real)rho, lor = (Real)(lam / rho);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
  for (int64_t i = wid; i < rows; i += nw) {
    Real zb[kRegs], d[kRegs];
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int sc = lane + 32 * q;
      const Real f = sc < R ? F[i * R + sc] : Real(0);
      zb[q] = sc < R ? Zbar[i * R + sc] : Real(0);
      d[q] = sc < R ? D[i * R + sc] : Real(0);
      if (sc < R) bv[sc] = f + rr * (zb[q] + d[q]);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int sc = lane + 32 * q;
      if (sc < R) {
        Real z = Real(0);
        for (int t = 0; t < R; ++t) z += Gi[sc * (R + 1) + t] * bv[t];
        const Real nz = prox<Real>(z - d[q], c, lor);
        const Real dn = d[q] + nz - z;
        s0 += (double)(nz - z) * (double)(nz - z);
        s1 += (double)nz * (double)nz;
        s2 += (double)(nz - zb[q]) * (double)(nz - zb[q]);
        Zbar[i * R + sc] = nz;
        D[i * R + sc] = dn;
      }
    }
    __syncwarp();
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; red[2][warp] = s2; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    atomicAdd(acc + threadIdx.x, t);
  }
}

// After an inner iteration: counts it for (outer iteration *it, mode) and sets *done when
// ||zbar - z||^2 <= eps^2 ||zbar||^2 and ||zbar - zbar_prev||^2 <= eps^2 ||zbar||^2; clears
// the sums for the next iteration.
__global__ void k_admm_check(double* __restrict__ acc, double eps2, int* __restrict__ done,
                             int* __restrict__ counts, const int* __restrict__ it, int mode) {
  if (*done) return;
  counts[*it * 3 + mode] += 1;
  if (acc[0] <= eps2 * acc[1] && acc[2] <= eps2 * acc[1]) *done = 1;
  acc[0] = acc[1] = acc[2] = 0.0;
}

__global__ void k_admm_reset(double* __restrict__ acc, int* __restrict__ done, int* __restrict__ counts,
                             const int* __restrict__ it, int mode) {
  acc[0] = acc[1] = acc[2] = 0.0;
  *done = 0;
  counts[*it * 3 + mode] = 0;
}

// F_W(k,:) = diag(H^T T_k) fused with the W ADMM (all inner iterations in registers).
template <typename Real>
__global__ void __launch_bounds__(256) k_admm_w(const Real* __restrict__ T,
                                                const Real* __restrict__ H,
                                                const Real* __restrict__ Ginv,
                                                const double* __restrict__ rho_dev, int n_inner,
                                                int c, double lam, Real* __restrict__ Wbar,
                                                Real* __restrict__ DW, int64_t K, int R) {
  extern __shared__ unsigned char smem_raw[];
  Real* Gi = reinterpret_cast<Real*>(smem_raw);          // R x (R+1)
  Real* Hs = Gi + R * (R + 1);                            // R x R
  Real* bvall = Hs + R * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* bv = bvall + warp * R;
  for (int e = threadIdx.x; e < R * (R + 1); e += blockDim.x) Gi[e] = Ginv[e];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Hs[e] = H[e];
  __syncthreads();
  const double rho = *rho_dev;
  const Real lor = (Real)(lam / rho);
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
  for (int64_t k = wid; k < K; k += nw) {
    const Real* Tk = T + k * R * R;
    Real f[kRegs], zb[kRegs], d[kRegs];
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      Real acc = Real(0);
      if (s < R)
        for (int r = 0; r < R; ++r) acc += Hs[r * R + s] * Tk[r * R + s];
      f[q] = acc;
      zb[q] = s < R ? Wbar[k * R + s] : Real(0);
      d[q] = s < R ? DW[k * R + s] : Real(0);
    }
    admm_row<Real>(R, Gi, (Real)rho, lor, c, n_inner, f, zb, d, bv);
#pragma unroll
    for (int q = 0; q < kRegs; ++q) {
      const int s = lane + 32 * q;
      if (s < R) { Wbar[k * R + s] = zb[q]; DW[k * R + s] = d[q]; }
    }
    __syncwarp();
  }
}

// W update for R <= 48, batched: a block takes kWS subjects at once and runs every inner
// iteration as one small GEMM Z = (G + rho I)^{-1} B over the tile (B = F_W + rho (Wbar + D),
// a row per subject), so Ginv is read from shared memory once per tile and iteration
// instead of once per subject. A thread owns NC components of two subjects (state in
// registers); Ginv and B sit in shared memory with 16-byte aligned, zero-padded rows, read
// with vector loads along the contraction. F_W(k, s) = sum_r H(r, s) T_k(r, s) comes
// first, one warp per subject with coalesced (FP32, R % 4 == 0: float4 streaming) reads of
// T_k.
constexpr int kWS = 64;      // subjects per block
constexpr int kWNTH = 256;   // threads per block

// 16-byte loads from shared memory (4 floats or 2 doubles)
template <typename Real>
struct V16;
template <>
struct V16<float> {
  static constexpr int n = 4;
  static __device__ __forceinline__ void ld(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct V16<double> {
  static constexpr int n = 2;
  static __device__ __forceinline__ void ld(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
};

// Shared memory of k_admm_w_tiled: Ginv (R rows, stride RP + VN), B (kWS subject rows, same
// stride), H (R x R), F_W (R x (kWS + 1)); RP = R rounded up to the vector width VN.
template <typename Real>
__host__ __device__ inline int wt_rp(int R) {
  constexpr int VN = 16 / (int)sizeof(Real);
  return (R + VN - 1) / VN * VN;
}
template <typename Real>
__host__ __device__ inline size_t wt_smem_elems(int R) {
  constexpr int VN = 16 / (int)sizeof(Real);
  const int ld = wt_rp<Real>(R) + VN;
  return (size_t)R * ld + (size_t)kWS * ld + (size_t)R * R + (size_t)R * (kWS + 1);
}

template <typename Real, int NC>
__global__ void __launch_bounds__(kWNTH) k_admm_w_tiled(const Real* __restrict__ T, const Real* __restrict__ H,
                                                        const Real* __restrict__ Ginv,
                                                        const double* __restrict__ rho_dev, int n_inner, int c,
                                                        double lam, Real* __restrict__ Wbar, Real* __restrict__ DW,
                                                        int64_t K, int R) {
  using Vl = V16<Real>;
  constexpr int VN = Vl::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int RP = wt_rp<Real>(R), ld = RP + VN;
  Real* Gs = reinterpret_cast<Real*>(smem_raw);   // R x ld: Ginv, zero-padded
  Real* Bq = Gs + R * ld;                          // kWS x ld: B, row per subject, zero-padded
  Real* Hs = Bq + kWS * ld;                        // R x R
  constexpr int ldw = kWS + 1;                     // odd stride: conflict-free columns
  Real* Fs = Hs + R * R;                           // R x ldw: F_W
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sr = tid & 7, kc = tid >> 3;           // components sr*NC.., subjects 2kc, 2kc+1
  for (int e = tid; e < R * ld; e += kWNTH) {
    const int r = e / ld, t = e - r * ld;
    Gs[e] = t < R ? Ginv[r * (R + 1) + t] : Real(0);
  }
  for (int e = tid; e < kWS * ld; e += kWNTH) Bq[e] = Real(0);
  for (int e = tid; e < R * R; e += kWNTH) Hs[e] = H[e];
  const double rho = *rho_dev;
  const Real rr = (Real)rho, lor = (Real)(lam / rho);
  for (int64_t k0 = (int64_t)blockIdx.x * kWS; k0 < K; k0 += (int64_t)gridDim.x * kWS) {
    const int nk = (int)min((int64_t)kWS, K - k0);
    __syncthreads();   // Gs/Hs ready; the previous tile's reads of Fs/Bs are done
    if (std::is_same<Real, float>::value && R % 4 == 0) {
      // FP32, R % 4 == 0: lanes take float4 slices of 32 / (R / 4) rows of T_k at a time
      // (independent streaming loads), then add up the row groups by shuffles
      const int q4 = R >> 2, per = 32 / q4, rg = lane / q4, c4 = lane - rg * q4;
      for (int q = warp; q < kWS; q += kWNTH / 32) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < nk && rg < per) {
          const float4* T4 = reinterpret_cast<const float4*>(T + (k0 + q) * R * R);
          const float4* H4 = reinterpret_cast<const float4*>(Hs);
#pragma unroll 4
          for (int r = rg; r < R; r += per) {
            const float4 t = __ldcs(T4 + r * q4 + c4), hv = H4[r * q4 + c4];
            acc.x += t.x * hv.x;
            acc.y += t.y * hv.y;
            acc.z += t.z * hv.z;
            acc.w += t.w * hv.w;
          }
        }
        for (int o = 1; o < per; ++o) {
          const int src = min(lane + o * q4, 31);
          const float ax = __shfl_sync(0xffffffffu, acc.x, src), ay = __shfl_sync(0xffffffffu, acc.y, src),
                      az = __shfl_sync(0xffffffffu, acc.z, src), aw = __shfl_sync(0xffffffffu, acc.w, src);
          if (rg == 0) {
            acc.x += ax;
            acc.y += ay;
            acc.z += az;
            acc.w += aw;
          }
        }
        if (rg == 0) {
          Fs[(4 * c4) * ldw + q] = (Real)acc.x;
          Fs[(4 * c4 + 1) * ldw + q] = (Real)acc.y;
          Fs[(4 * c4 + 2) * ldw + q] = (Real)acc.z;
          Fs[(4 * c4 + 3) * ldw + q] = (Real)acc.w;
        }
      }
    } else {
      for (int q = warp; q < kWS; q += kWNTH / 32) {
        for (int s = lane; s < R; s += 32) {
          Real acc = Real(0);
          if (q < nk) {
            const Real* Tk = T + (k0 + q) * R * R;
            for (int r = 0; r < R; ++r) acc += Hs[r * R + s] * Tk[r * R + s];
          }
          Fs[s * ldw + q] = acc;
        }
      }
    }
    __syncthreads();
    Real f[NC][2], zb[NC][2], d[NC][2];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int s = sr * NC + a, q = 2 * kc + b;
        const bool in = s < R && q < nk;
        f[a][b] = in ? Fs[s * ldw + q] : Real(0);
        zb[a][b] = in ? Wbar[(k0 + q) * R + s] : Real(0);
        d[a][b] = in ? DW[(k0 + q) * R + s] : Real(0);
      }
    for (int it = 0; it < n_inner; ++it) {
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int s = sr * NC + a;
          if (s < R) Bq[(2 * kc + b) * ld + s] = f[a][b] + rr * (zb[a][b] + d[a][b]);
        }
      __syncthreads();
      Real z[NC][2];
#pragma unroll
      for (int a = 0; a < NC; ++a) z[a][0] = z[a][1] = Real(0);
      for (int t = 0; t < RP; t += VN) {
        Real b0[VN], b1[VN];
        Vl::ld(Bq + (2 * kc) * ld + t, b0);
        Vl::ld(Bq + (2 * kc + 1) * ld + t, b1);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          const int s = sr * NC + a;
          Real g[VN];
          if (s < R) {
            Vl::ld(Gs + s * ld + t, g);
          } else {
#pragma unroll
            for (int v = 0; v < VN; ++v) g[v] = Real(0);
          }
#pragma unroll
          for (int v = 0; v < VN; ++v) {
            z[a][0] += g[v] * b0[v];
            z[a][1] += g[v] * b1[v];
          }
        }
      }
      __syncthreads();   // every read of B is done before the next iteration writes it
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const Real nz = prox<Real>(z[a][b] - d[a][b], c, lor);
          d[a][b] = d[a][b] + nz - z[a][b];
          zb[a][b] = nz;
        }
    }
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int s = sr * NC + a, q = 2 * kc + b;
        if (s < R && q < nk) {
          Wbar[(k0 + q) * R + s] = zb[a][b];
          DW[(k0 + q) * R + s] = d[a][b];
        }
      }
  }
}

// ------------------------------------------------------------------------------------
// FIT = 1 - (x_norm2 - ||X||^2 + ||X||^2 - 2 <V, F_V> + <V^T V, U^T U>) / x_norm2
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void k_fit_value(int64_t J, int R, const Real* __restrict__ V, const Real* __restrict__ FV,
                            const double* __restrict__ VtV, const double* __restrict__ UtU,
                            const double* __restrict__ xn2_dev, double x_norm2, double* __restrict__ fit) {
  __shared__ double red[2][256];
  double cross = 0.0, model = 0.0;
  for (int64_t e = threadIdx.x; e < J * R; e += blockDim.x) cross += (double)V[e] * (double)FV[e];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) model += VtV[e] * UtU[e];
  red[0][threadIdx.x] = cross;
  red[1][threadIdx.x] = model;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double xx = *xn2_dev;
    const double resid = xx - 2.0 * red[0][0] + red[1][0];
    const double xn = x_norm2 > 0.0 ? x_norm2 : xx;
    fit[0] = 1.0 - (xn - xx + resid) / xn;
  }
}

}  // namespace

// ---------------------------------- launchers ----------------------------------------

static int grid_for(copa_ctx* h, int64_t work_items, int per_block, int cap_per_sm = 8) {
  int64_t blocks = (work_items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)h->num_sms * cap_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <typename Real>
copa_status_t launch_mttkrp_h(copa_ctx* h, int64_t K, int R, const Real* T, const Real* W, Real* F) {
  const int blocks = grid_for(h, K, 512, 4);
  double* part = nullptr;
  copa_status_t st;
  if ((st = ws_get(h, SLOT_PARTIAL, (size_t)blocks * R * R * sizeof(double), (void**)&part)) != COPA_OK)
    return st;
  k_mttkrp_h<Real><<<blocks, 256, 0, h->stream>>>(K, R, T, W, part);
  k_reduce_rows<Real><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, blocks, R * R, F);
  return cuda_check(h, cudaGetLastError(), "k_mttkrp_h");
}

template <typename Real>
copa_status_t launch_mttkrp_w(copa_ctx* h, int64_t K, int R, const Real* T, const Real* H, Real* F) {
  k_mttkrp_w<Real><<<grid_for(h, K, 8, 16), 256, 0, h->stream>>>(K, R, T, H, F);
  return cuda_check(h, cudaGetLastError(), "k_mttkrp_w");
}

// The column-sorted copy is rebuilt unless `reuse` (copa_fit builds it once per call and
// reuses it for the later iterations of the same call, where X cannot change).
// Column-sorted copy of X and the row -> subject map, in SLOT_CSC:
//   int64 ptr[J+1], int64 cursor[J+1], int32 rows[nnz], Real vals[nnz] (16-byte aligned),
//   int32 row_subj[S] (16-byte aligned).
template <typename Real>
static copa_status_t get_csc(copa_ctx* h, const TensorView& X, bool reuse, const int64_t** cptr,
                             const int32_t** crow, const Real** cval, const int32_t** rsubj) {
  copa_status_t st;
  const int prec = sizeof(Real) == 8 ? 1 : 0;
  auto al16 = [](uintptr_t v) { return (v + 15) & ~uintptr_t(15); };
  auto layout = [&](char* p, int64_t** ptr, int32_t** rows, Real** vals, int32_t** rs) {
    *ptr = reinterpret_cast<int64_t*>(p);
    *rows = reinterpret_cast<int32_t*>(*ptr + 2 * ((size_t)X.J + 1));
    *vals = reinterpret_cast<Real*>(al16(reinterpret_cast<uintptr_t>(*rows + X.nnz)));
    *rs = reinterpret_cast<int32_t*>(al16(reinterpret_cast<uintptr_t>(*vals + X.nnz)));
  };
  int64_t* ptr = nullptr;
  int32_t* rows = nullptr;
  Real* vals = nullptr;
  int32_t* rs = nullptr;
  if (!(reuse && h->csc_key == X.col && h->csc_nnz == X.nnz && h->csc_J == X.J && h->csc_prec == prec &&
        h->csc_S == X.S && h->slot_ptr[SLOT_CSC])) {
    // stable build: J fits the shared-memory counters and every count fits an int
    const bool stable = X.J <= kHistSmem && X.nnz < (int64_t)INT32_MAX;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(8192, X.S / 64));
    const size_t rel_bytes = stable ? sizeof(int) * (size_t)X.J * nb + 16 : 0;
    const size_t bytes = sizeof(int64_t) * 2 * ((size_t)X.J + 1) + sizeof(int32_t) * (size_t)X.nnz +
                         sizeof(Real) * (size_t)X.nnz + sizeof(int32_t) * (size_t)X.S + 64 + rel_bytes;
    char* p = nullptr;
    if ((st = ws_get(h, SLOT_CSC, bytes, (void**)&p)) != COPA_OK) return st;
    layout(p, &ptr, &rows, &vals, &rs);
    int64_t* cur = ptr + X.J + 1;
    if ((st = cuda_check(h, cudaMemsetAsync(ptr, 0, sizeof(int64_t) * 2 * ((size_t)X.J + 1), h->stream),
                         "memset")) != COPA_OK)
      return st;
    if (stable) {
      int* rel = reinterpret_cast<int*>(al16(reinterpret_cast<uintptr_t>(rs + X.S)));
      const size_t jsm = sizeof(int) * (size_t)X.J;
      k_csc_count<<<nb, 32, jsm, h->stream>>>(X, nb, rel);
      k_csc_colscan<<<(X.J + 7) / 8, 256, 0, h->stream>>>(X.J, nb, rel, ptr);
      k_scan_cols<<<1, 32, 0, h->stream>>>(ptr, X.J);
      k_csc_place<Real><<<nb, 32, jsm, h->stream>>>(X, nb, rel, ptr, rows, vals);
      h->setup_launches += 1;
    } else {
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.nnz + 255) / 256, (int64_t)h->num_sms * 8));
      k_csc_hist<<<blocks, 256, 0, h->stream>>>(X, ptr);
      k_scan_cols<<<1, 32, 0, h->stream>>>(ptr, X.J);
      const int rblocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.S + 255) / 256, (int64_t)h->num_sms * 16));
      k_csc_scatter<Real><<<rblocks, 256, 0, h->stream>>>(X, ptr, cur, rows, vals);
    }
    const int kblocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.K + 255) / 256, (int64_t)h->num_sms * 16));
    k_row_subject<<<kblocks, 256, 0, h->stream>>>(X.subj_ptr, X.K, rs);
    if ((st = cuda_check(h, cudaGetLastError(), "csc build")) != COPA_OK) return st;
    h->setup_launches += 4;
    h->csc_key = X.col;
    h->csc_nnz = X.nnz;
    h->csc_J = X.J;
    h->csc_S = X.S;
    h->csc_prec = prec;
  } else {
    layout(reinterpret_cast<char*>(h->slot_ptr[SLOT_CSC]), &ptr, &rows, &vals, &rs);
  }
  *cptr = ptr;
  *crow = rows;
  *cval = vals;
  *rsubj = rs;
  return COPA_OK;
}

template <typename Real>
static copa_status_t launch_uvec_tiled(copa_ctx* h, int64_t S, int R, const Real* Q, const Real* H, const Real* W,
                                       const int32_t* rsubj, Real* U, double* UtU_part_or_null, int64_t* nparts,
                                       bool size_only) {
  const int nc = (R + 7) / 8;
  void (*kern)(int64_t, int, const Real*, const Real*, const Real*, const int32_t*, Real*, double*) = nullptr;
  switch (nc) {
    case 1: kern = k_uvec_tiled<Real, 1>; break;
    case 2: kern = k_uvec_tiled<Real, 2>; break;
    case 3: kern = k_uvec_tiled<Real, 3>; break;
    case 4: kern = k_uvec_tiled<Real, 4>; break;
    case 5: kern = k_uvec_tiled<Real, 5>; break;
    case 6: kern = k_uvec_tiled<Real, 6>; break;
    default: return fail(h, COPA_ERR_UNSUPPORTED, "tiled U: R > 48");
  }
  const size_t smem = sizeof(Real) * ((size_t)64 * nc * nc + (size_t)kVT * (R + 1));
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kVNT, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)h->num_sms * per_sm;
  const int64_t need = (S + kVT - 1) / kVT;
  if (blocks > need) blocks = std::max<int64_t>(need, 1);
  *nparts = blocks * 4;
  if (size_only) return COPA_OK;
  kern<<<(unsigned)blocks, kVNT, smem, h->stream>>>(S, R, Q, H, W, rsubj, U, UtU_part_or_null);
  return cuda_check(h, cudaGetLastError(), "k_uvec_tiled");
}

// ---- F_V = X^T U in row order (FP32 path) ----
// The nonzeros of X are taken in their stored (row) order, split evenly over the CTAs (one
// per SM). A CTA keeps its own copy of 32 columns of F_V (J x 32 floats in shared memory)
// per pass and adds x_ij u_i(c) into it by shared-memory atomics: a warp takes 32 nonzeros
// at a time (column, value and row loaded by the lanes, then broadcast by shuffles), each
// lane adding one column, or several nonzeros per step when a pass is narrower than 32
// columns. U is read in row order (consecutive nonzeros share rows), so it streams from
// memory about once per pass, where the column-order form gathered a row of U per
// nonzero. The per-CTA copies go to FP32 partials that k_reduce_fv adds in FP64.
constexpr int kSRT = 1024;   // threads per CTA

__global__ void k_nz_row(const int64_t* __restrict__ row_ptr, int64_t S, int32_t* __restrict__ nzrow) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S; i += gridDim.x * (int64_t)blockDim.x)
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) nzrow[p] = (int32_t)i;
}

__global__ void __launch_bounds__(kSRT, 1) k_spmm_rows(TensorView X, int R, const float* __restrict__ U,
                                                       const int32_t* __restrict__ nzrow, float* __restrict__ part) {
  extern __shared__ float Fs[];   // J x 32: this CTA's sums of columns c0 .. c0 + 31 of F_V
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kSRT / 32;
  const int64_t per = (X.nnz + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = min(X.nnz, (int64_t)blockIdx.x * per), p1 = min(X.nnz, p0 + per);
  const int npass = (R + 31) / 32;
  for (int pass = 0; pass < npass; ++pass) {
    const int c0 = 32 * pass, w = min(32, R - c0);
    // lanes per nonzero: the pass width rounded up to a power of two
    const int lw = w > 16 ? 32 : (w > 8 ? 16 : (w > 4 ? 8 : (w > 2 ? 4 : (w > 1 ? 2 : 1))));
    const int per_step = 32 / lw, sub = lane / lw, c = lane - sub * lw;
    for (int e = threadIdx.x; e < X.J * 32; e += kSRT) Fs[e] = 0.f;
    __syncthreads();
    // Chunks of 32 nonzeros, software-pipelined: the column, value and row of chunk n + 2
    // are loaded, and the U lines of chunk n + 1 prefetched into L1, while chunk n is added.
    constexpr int64_t step = (int64_t)nw * 32;
    auto load = [&](int64_t b, int& j, float& x, int& i) {
      const int64_t p = b + lane;
      const bool v = p < p1;
      j = v ? __ldg(X.col + p) : 0;
      x = v ? load_valf(X, p) : 0.f;
      i = v ? __ldg(nzrow + p) : 0;
    };
    const int64_t first = p0 + (int64_t)warp * 32;
    int jj, ii, j1, i1;
    float xx, x1;
    load(first, jj, xx, ii);
    load(first + step, j1, x1, i1);
    for (int64_t base = first; base < p1; base += step) {
      int j2, i2;
      float x2;
      load(base + 2 * step, j2, x2, i2);
      if (base + step + lane < p1 && c0 < R)   // this lane's nonzero of the next chunk: its U line
        asm volatile("prefetch.global.L1 [%0];" ::"l"(U + (int64_t)i1 * R + c0));
      const int cnt = (int)min((int64_t)32, p1 - base);
#pragma unroll 4
      for (int q = 0; q < 32; q += per_step) {
        const int src = q + sub;   // < 32
        const int j = __shfl_sync(kFull, jj, src);
        const float x = __shfl_sync(kFull, xx, src);
        const int i = __shfl_sync(kFull, ii, src);
        if (src < cnt && c < w) atomicAdd(&Fs[j * 32 + c], x * __ldg(U + (int64_t)i * R + c0 + c));
      }
      jj = j1; xx = x1; ii = i1;
      j1 = j2; x1 = x2; i1 = i2;
    }
    __syncthreads();
    float* pp = part + ((size_t)blockIdx.x * npass + pass) * (size_t)X.J * 32;
    for (int e = threadIdx.x; e < X.J * 32; e += kSRT) pp[e] = Fs[e];
    __syncthreads();
  }
}

template <typename Real>
__global__ void k_reduce_fv(const float* __restrict__ part, int nblocks, int npass, int J, int R,
                            Real* __restrict__ F) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J * R; e += gridDim.x * blockDim.x) {
    const int j = e / R, c = e - j * R, pass = c >> 5, cc = c & 31;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += (double)part[((size_t)b * npass + pass) * (size_t)J * 32 + j * 32 + cc];
    F[e] = (Real)acc;
  }
}

// F_V in row order with the sums kept in L2 instead of shared memory: the lanes of a warp
// take VW-wide slices of the U rows of 32 / (R / VW) nonzeros at a time (VW the largest of
// 4, 2, 1 dividing R) and add x u_i into a partial copy of F_V (FP32, one per group of
// CTAs, small enough to stay in L2) with vector reductions, so that every column of U is
// read in one pass, whatever J is.
constexpr int kRedT = 512;   // threads per CTA
template <int VW> struct RedVec;
template <> struct RedVec<4> {
  static __device__ __forceinline__ void add(float* dst, const float* src, float x) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(src));
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(x * u.x), "f"(x * u.y),
                 "f"(x * u.z), "f"(x * u.w)
                 : "memory");
  }
};
template <> struct RedVec<2> {
  static __device__ __forceinline__ void add(float* dst, const float* src, float x) {
    const float2 u = __ldg(reinterpret_cast<const float2*>(src));
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(x * u.x), "f"(x * u.y) : "memory");
  }
};
template <> struct RedVec<1> {
  static __device__ __forceinline__ void add(float* dst, const float* src, float x) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(dst), "f"(x * __ldg(src)) : "memory");
  }
};

template <int VW>
__global__ void __launch_bounds__(kRedT) k_spmm_rows_red(TensorView X, int R, const float* __restrict__ U,
                                                           const int32_t* __restrict__ nzrow, float* __restrict__ part,
                                                           int nparts) {
  constexpr unsigned kFull = 0xffffffffu;
  constexpr int nw = kRedT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qv = R / VW, per = 32 / qv;   // lanes per nonzero (<= 32), nonzeros per step
  const int sub = lane / qv, cv = lane - sub * qv;
  const bool act = sub < per;
  const int64_t per_cta = (X.nnz + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = min(X.nnz, (int64_t)blockIdx.x * per_cta), p1 = min(X.nnz, p0 + per_cta);
  float* Fp = part + (size_t)(blockIdx.x % nparts) * (size_t)X.J * R;
  constexpr int64_t step = (int64_t)nw * 32;
  for (int64_t base = p0 + (int64_t)warp * 32; base < p1; base += step) {
    const int64_t p = base + lane;
    const bool v = p < p1;
    const int jj = v ? __ldg(X.col + p) : 0;
    const float xx = v ? load_valf(X, p) : 0.f;
    const int ii = v ? __ldg(nzrow + p) : 0;
    const int cnt = (int)min((int64_t)32, p1 - base);
#pragma unroll 2
    for (int q = 0; q < cnt; q += per) {
      const int src = q + sub;
      const int j = __shfl_sync(kFull, jj, src & 31);
      const float x = __shfl_sync(kFull, xx, src & 31);
      const int i = __shfl_sync(kFull, ii, src & 31);
      if (act && src < cnt) RedVec<VW>::add(Fp + (int64_t)j * R + VW * cv, U + (int64_t)i * R + VW * cv, x);
    }
  }
}

static int red_width(int R) { return R % 4 == 0 ? 4 : (R % 2 == 0 ? 2 : 1); }

// F(e) = sum over the nparts partial copies of element e, in FP64.
template <typename Real>
__global__ void k_reduce_fv_red(const float* __restrict__ part, int nparts, int64_t n, Real* __restrict__ F) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += gridDim.x * (int64_t)blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += (double)part[(size_t)b * n + e];
    F[e] = (Real)acc;
  }
}

static bool spmm_red_applies(int R, const TensorView& X) {
  return R <= 32 * red_width(R) && X.nnz < (int64_t)INT32_MAX && X.S < (int64_t)INT32_MAX;
}

// Shared memory the row-order F_V kernel needs (J x 32 floats); the path is taken when it fits.
static size_t spmm_rows_smem(int J) { return sizeof(float) * 32 * (size_t)J; }
static bool spmm_rows_fits(const copa_ctx* h, const TensorView& X) {
  (void)h;
  return spmm_rows_smem(X.J) <= (size_t)200 * 1024 && X.nnz < (int64_t)INT32_MAX && X.S < (int64_t)INT32_MAX;
}

// Nonzero -> row and row -> subject maps in SLOT_ROWMAP, rebuilt unless `reuse` and the
// tensor is the one they were built for.
static copa_status_t get_rowmaps(copa_ctx* h, const TensorView& X, bool reuse, const int32_t** nzrow,
                                 const int32_t** rsubj) {
  copa_status_t st;
  const size_t off = ((sizeof(int32_t) * (size_t)X.nnz + 15) & ~size_t(15));
  if (!(reuse && h->rmap_key == X.col && h->rmap_nnz == X.nnz && h->rmap_S == X.S && h->rmap_K == X.K &&
        h->slot_ptr[SLOT_ROWMAP])) {
    char* p = nullptr;
    if ((st = ws_get(h, SLOT_ROWMAP, off + sizeof(int32_t) * (size_t)X.S + 16, (void**)&p)) != COPA_OK) return st;
    int32_t* nz = reinterpret_cast<int32_t*>(p);
    int32_t* rs = reinterpret_cast<int32_t*>(p + off);
    const int rblocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.S + 255) / 256, (int64_t)h->num_sms * 16));
    k_nz_row<<<rblocks, 256, 0, h->stream>>>(X.row_ptr, X.S, nz);
    const int kblocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.K + 255) / 256, (int64_t)h->num_sms * 16));
    k_row_subject<<<kblocks, 256, 0, h->stream>>>(X.subj_ptr, X.K, rs);
    if ((st = cuda_check(h, cudaGetLastError(), "row maps")) != COPA_OK) return st;
    h->setup_launches += 2;
    h->rmap_key = X.col;
    h->rmap_nnz = X.nnz;
    h->rmap_S = X.S;
    h->rmap_K = X.K;
  }
  const char* p = reinterpret_cast<const char*>(h->slot_ptr[SLOT_ROWMAP]);
  *nzrow = reinterpret_cast<const int32_t*>(p);
  *rsubj = reinterpret_cast<const int32_t*>(p + off);
  return COPA_OK;
}

template <typename Real>
copa_status_t launch_mttkrp_v(copa_ctx* h, const TensorView& X, int R, const Real* Q, const Real* H,
                              const Real* W, Real* F, double* UtU, bool reuse_csc) {
  if (R > kMaxR) return fail(h, COPA_ERR_UNSUPPORTED, "mttkrp V: R too large");
  copa_status_t st;
  const int64_t* cptr = nullptr;
  const int32_t* crow = nullptr;
  const Real* cval = nullptr;
  const int32_t* rsubj = nullptr;
  const int32_t* nzrow = nullptr;
  // F_V in row order (FP32, when J x 32 floats fit in shared memory), else over the
  // column-sorted copy of X
  bool rows_fv = false, red_fv = false;
  if constexpr (std::is_same<Real, float>::value) {
    const int fv = active_tune(h, X, R).fv;
    red_fv = fv == 2 && spmm_red_applies(R, X);
    rows_fv = !red_fv && spmm_rows_fits(h, X) && fv != 1;
  }
  if (rows_fv || red_fv) {
    if ((st = get_rowmaps(h, X, reuse_csc, &nzrow, &rsubj)) != COPA_OK) return st;
  } else if ((st = get_csc<Real>(h, X, reuse_csc, &cptr, &crow, &cval, &rsubj)) != COPA_OK) {
    return st;
  }
  Real* U = nullptr;
  if ((st = ws_get(h, SLOT_UVEC, sizeof(Real) * ((size_t)X.S * R + 16), (void**)&U)) != COPA_OK) return st;
  if (!rows_fv && !red_fv &&
      (st = cuda_check(h, cudaMemsetAsync(F, 0, sizeof(Real) * (size_t)X.J * R, h->stream), "memset F")) != COPA_OK)
    return st;
  double* part = nullptr;
  int64_t nparts = 0;
  bool tensor = false;   // FP32: the tensor-core tile kernel where its layout applies
  if constexpr (std::is_same<Real, float>::value) tensor = uvec_tc_supported(R, Q, W, U);
  if (tensor) {
    if constexpr (std::is_same<Real, float>::value) {
      if ((st = launch_uvec_tc(h, X.S, R, Q, H, W, rsubj, U, nullptr, &nparts, true)) != COPA_OK) return st;
      if (UtU && (st = ws_get(h, SLOT_PARTIAL, (size_t)nparts * R * R * sizeof(double), (void**)&part)) != COPA_OK)
        return st;
      if ((st = launch_uvec_tc(h, X.S, R, Q, H, W, rsubj, U, part, &nparts, false)) != COPA_OK) return st;
    }
  } else if (R <= 48) {
    if ((st = launch_uvec_tiled<Real>(h, X.S, R, Q, H, W, rsubj, U, nullptr, &nparts, true)) != COPA_OK) return st;
    if (UtU && (st = ws_get(h, SLOT_PARTIAL, (size_t)nparts * R * R * sizeof(double), (void**)&part)) != COPA_OK)
      return st;
    if ((st = launch_uvec_tiled<Real>(h, X.S, R, Q, H, W, rsubj, U, part, &nparts, false)) != COPA_OK) return st;
  } else {
    const int64_t* order = nullptr;
    if ((st = get_schedule(h, X, &order)) != COPA_OK) return st;
    int* counter = nullptr;
    if ((st = ws_get(h, SLOT_COUNTER, 64, (void**)&counter)) != COPA_OK) return st;
    if ((st = cuda_check(h, cudaMemsetAsync(counter + 1, 0, sizeof(int), h->stream), "memset")) != COPA_OK)
      return st;
    const bool tiles = R <= kTR * 8;
    const int nw = kUNT / 32;
    const int npk = R * (R + 1) / 2;
    const size_t smem = sizeof(Real) * ((size_t)R * R + (size_t)nw * (2 * R + (tiles ? 0 : npk))) +
                        (tiles ? 0 : sizeof(uint16_t) * npk) + 64;
    auto kern = tiles ? k_uvec<Real, true> : k_uvec<Real, false>;
    if ((st = cuda_check(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                         "cudaFuncSetAttribute")) != COPA_OK)
      return st;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kUNT, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)h->num_sms * per_sm;
    const int64_t need = (X.K + nw - 1) / nw;
    if (blocks > need) blocks = need > 0 ? need : 1;
    nparts = blocks * nw;
    if (UtU) {
      if ((st = ws_get(h, SLOT_PARTIAL, (size_t)nparts * R * R * sizeof(double), (void**)&part)) != COPA_OK)
        return st;
    }
    kern<<<(unsigned)blocks, kUNT, smem, h->stream>>>(X, R, Q, H, W, U, part, order, counter + 1);
    if ((st = cuda_check(h, cudaGetLastError(), "k_uvec")) != COPA_OK) return st;
  }
  if (red_fv) {
    if constexpr (std::is_same<Real, float>::value) {
      const int vw = red_width(R);
      auto kern = vw == 4 ? k_spmm_rows_red<4> : (vw == 2 ? k_spmm_rows_red<2> : k_spmm_rows_red<1>);
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRedT, 0);
      const int fblocks = h->num_sms * std::max(per_sm, 1);
      // partial copies: one per SM, fewer if that would exceed 64 MB
      const int64_t jr = (int64_t)X.J * R;
      const int nparts_fv = (int)std::max<int64_t>(1, std::min<int64_t>(h->num_sms, (64ll << 20) / (4 * jr)));
      float* fpart = nullptr;
      if ((st = ws_get(h, SLOT_FV_PART, sizeof(float) * (size_t)nparts_fv * jr + 16, (void**)&fpart)) != COPA_OK)
        return st;
      if ((st = cuda_check(h, cudaMemsetAsync(fpart, 0, sizeof(float) * (size_t)nparts_fv * jr, h->stream),
                           "memset")) != COPA_OK)
        return st;
      kern<<<fblocks, kRedT, 0, h->stream>>>(X, R, U, nzrow, fpart, nparts_fv);
      if ((st = cuda_check(h, cudaGetLastError(), "k_spmm_rows_red")) != COPA_OK) return st;
      const int rb = (int)std::max<int64_t>(1, std::min<int64_t>((jr + 255) / 256, 4096));
      k_reduce_fv_red<Real><<<rb, 256, 0, h->stream>>>(fpart, nparts_fv, jr, F);
      if ((st = cuda_check(h, cudaGetLastError(), "k_reduce_fv_red")) != COPA_OK) return st;
    }
  } else if (rows_fv) {
    if constexpr (std::is_same<Real, float>::value) {
      const int npass = (R + 31) / 32;
      const int fblocks = std::max(1, h->num_sms);
      float* fpart = nullptr;
      if ((st = ws_get(h, SLOT_FV_PART, sizeof(float) * (size_t)fblocks * npass * 32 * (size_t)X.J + 16,
                       (void**)&fpart)) != COPA_OK)
        return st;
      const size_t fsm = spmm_rows_smem(X.J);
      if ((st = cuda_check(h, cudaFuncSetAttribute(k_spmm_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm),
                           "cudaFuncSetAttribute")) != COPA_OK)
        return st;
      k_spmm_rows<<<fblocks, kSRT, fsm, h->stream>>>(X, R, U, nzrow, fpart);
      if ((st = cuda_check(h, cudaGetLastError(), "k_spmm_rows")) != COPA_OK) return st;
      const int rb = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)X.J * R + 255) / 256, 4096));
      k_reduce_fv<Real><<<rb, 256, 0, h->stream>>>(fpart, fblocks, npass, X.J, R, F);
      if ((st = cuda_check(h, cudaGetLastError(), "k_reduce_fv")) != COPA_OK) return st;
    }
  } else {
    const int64_t nchunks = (X.nnz + kChunk - 1) / kChunk;
    const int sblocks = (int)std::max<int64_t>(1, std::min<int64_t>((nchunks + 7) / 8, (int64_t)h->num_sms * 16));
    k_spmm_csc<Real><<<sblocks, 256, 0, h->stream>>>(X.nnz, X.J, R, cptr, crow, cval, U, F);
    if ((st = cuda_check(h, cudaGetLastError(), "k_spmm_csc")) != COPA_OK) return st;
  }
  if (UtU) {
    k_reduce_rows<double><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, (int)nparts, R * R, UtU);
    if ((st = cuda_check(h, cudaGetLastError(), "UtU reduce")) != COPA_OK) return st;
  }
  return COPA_OK;
}

template <typename Real>
copa_status_t launch_gram(copa_ctx* h, const Real* A, int64_t rows, int R, double* G) {
  const int npk = R * (R + 1) / 2;
  const int threads = npk <= 256 ? 256 : 512;
  if (npk > threads * 8) return fail(h, COPA_ERR_UNSUPPORTED, "gram: R too large");
  const int blocks = grid_for(h, rows, 2048, 2);
  double* part = nullptr;
  copa_status_t st;
  if ((st = ws_get(h, SLOT_MISC, (size_t)blocks * R * R * sizeof(double), (void**)&part)) != COPA_OK)
    return st;
  const size_t smem = sizeof(Real) * 64 * (size_t)R;
  k_gram<Real><<<blocks, threads, smem, h->stream>>>(A, rows, R, part);
  k_reduce_rows<double><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, blocks, R * R, G);
  return cuda_check(h, cudaGetLastError(), "k_gram");
}

template <typename Real>
copa_status_t launch_chol(copa_ctx* h, const double* Ga, const double* Gb, int R, Real* Ginv,
                          double* rho_dev) {
  const size_t smem = 2 * sizeof(double) * R * R;
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_chol<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  k_chol<Real><<<1, 128, smem, h->stream>>>(Ga, Gb, R, Ginv, rho_dev, h->d_status);
  return cuda_check(h, cudaGetLastError(), "k_chol");
}

template <typename Real>
copa_status_t launch_admm_rows(copa_ctx* h, const Real* F, const Real* Ginv, const double* rho_dev,
                               int n_inner, int c, double lam, Real* Zbar, Real* D, int64_t rows,
                               int R) {
  const size_t smem = sizeof(Real) * ((size_t)R * (R + 1) + 8 * (size_t)R);
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_admm_rows<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  k_admm_rows<Real><<<grid_for(h, rows, 8, 8), 256, smem, h->stream>>>(F, Ginv, rho_dev, n_inner, c, lam,
                                                                      Zbar, D, rows, R);
  return cuda_check(h, cudaGetLastError(), "k_admm_rows");
}

template <typename Real>
copa_status_t launch_admm_adaptive(copa_ctx* h, const Real* F, const Real* Ginv, const double* rho_dev,
                                   int max_inner, int c, double lam, Real* Zbar, Real* D, int64_t rows, int R,
                                   double eps, double* acc, int* done, int* counts, const int* it, int mode) {
  const size_t smem = sizeof(Real) * ((size_t)R * (R + 1) + 8 * (size_t)R);
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_admm_iter<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  k_admm_reset<<<1, 1, 0, h->stream>>>(acc, done, counts, it, mode);
  const int grid = grid_for(h, rows, 8, 8);
  for (int t = 0; t < max_inner; ++t) {
    k_admm_iter<Real><<<grid, 256, smem, h->stream>>>(F, Ginv, rho_dev, c, lam, Zbar, D, rows, R, done, acc);
    k_admm_check<<<1, 1, 0, h->stream>>>(acc, eps * eps, done, counts, it, mode);
  }
  return cuda_check(h, cudaGetLastError(), "k_admm_iter");
}

template <typename Real>
copa_status_t launch_admm_w(copa_ctx* h, const Real* T, const Real* H, const Real* Ginv,
                            const double* rho_dev, int n_inner, int c, double lam, Real* Wbar,
                            Real* DW, int64_t K, int R) {
  copa_status_t st;
  if (R <= 48) {
    void (*kern)(const Real*, const Real*, const Real*, const double*, int, int, double, Real*, Real*, int64_t,
                 int) = nullptr;
    switch ((R + 7) / 8) {
      case 1: kern = k_admm_w_tiled<Real, 1>; break;
      case 2: kern = k_admm_w_tiled<Real, 2>; break;
      case 3: kern = k_admm_w_tiled<Real, 3>; break;
      case 4: kern = k_admm_w_tiled<Real, 4>; break;
      case 5: kern = k_admm_w_tiled<Real, 5>; break;
      default: kern = k_admm_w_tiled<Real, 6>; break;
    }
    const size_t tsm = sizeof(Real) * wt_smem_elems<Real>(R);
    if ((st = cuda_check(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm),
                         "cudaFuncSetAttribute")) != COPA_OK)
      return st;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWNTH, tsm);
    const int64_t tiles = (K + kWS - 1) / kWS;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)h->num_sms * std::max(per_sm, 1)));
    kern<<<blocks, kWNTH, tsm, h->stream>>>(T, H, Ginv, rho_dev, n_inner, c, lam, Wbar, DW, K, R);
    return cuda_check(h, cudaGetLastError(), "k_admm_w_tiled");
  }
  const size_t smem = sizeof(Real) * ((size_t)R * (R + 1) + (size_t)R * R + 8 * (size_t)R);
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_admm_w<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  k_admm_w<Real><<<grid_for(h, K, 8, 8), 256, smem, h->stream>>>(T, H, Ginv, rho_dev, n_inner, c, lam,
                                                                 Wbar, DW, K, R);
  return cuda_check(h, cudaGetLastError(), "k_admm_w");
}

template <typename Real>
copa_status_t launch_fit_value(copa_ctx* h, int64_t J, int R, const Real* V, const Real* F_V,
                               const double* UtU, const double* xn2_dev, double x_norm2, double* fit,
                               double* VtV) {
  copa_status_t st;
  if ((st = launch_gram<Real>(h, V, J, R, VtV)) != COPA_OK) return st;   // V^T V over many blocks
  k_fit_value<Real><<<1, 256, 0, h->stream>>>(J, R, V, F_V, VtV, UtU, xn2_dev, x_norm2, fit);
  return cuda_check(h, cudaGetLastError(), "k_fit_value");
}

#define COPA_INST(Real)                                                                          \
  template copa_status_t launch_mttkrp_h<Real>(copa_ctx*, int64_t, int, const Real*, const Real*, \
                                               Real*);                                            \
  template copa_status_t launch_mttkrp_w<Real>(copa_ctx*, int64_t, int, const Real*, const Real*, \
                                               Real*);                                            \
  template copa_status_t launch_mttkrp_v<Real>(copa_ctx*, const TensorView&, int, const Real*,    \
                                               const Real*, const Real*, Real*, double*, bool);   \
  template copa_status_t launch_gram<Real>(copa_ctx*, const Real*, int64_t, int, double*);        \
  template copa_status_t launch_chol<Real>(copa_ctx*, const double*, const double*, int, Real*,   \
                                           double*);                                              \
  template copa_status_t launch_admm_rows<Real>(copa_ctx*, const Real*, const Real*,              \
                                                const double*, int, int, double, Real*, Real*,    \
                                                int64_t, int);                                    \
  template copa_status_t launch_admm_adaptive<Real>(copa_ctx*, const Real*, const Real*,          \
                                                    const double*, int, int, double, Real*, Real*, \
                                                    int64_t, int, double, double*, int*, int*,     \
                                                    const int*, int);                              \
  template copa_status_t launch_admm_w<Real>(copa_ctx*, const Real*, const Real*, const Real*,    \
                                             const double*, int, int, double, Real*, Real*,       \
                                             int64_t, int);                                       \
  template copa_status_t launch_fit_value<Real>(copa_ctx*, int64_t, int, const Real*, const Real*, \
                                                const double*, const double*, double, double*,    \
                                                double*);                                         \

COPA_INST(float)
COPA_INST(double)

}  // namespace copa


// =====================================================================================
// copa_gram_noalloc: the column Gram with its per-block partial sums in a fixed device
// array owned by the library instead of the handle's workspace, for callers that cannot
// allocate device memory. No counterpart in the paper.
// =====================================================================================

namespace copa {
namespace {

constexpr int kNoAllocMaxR = 90;                       // k_gram holds <= 8 entries/thread
constexpr size_t kNoAllocScratchDoubles = 131072;      // 1 MiB of block partials
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {nullptr};                 // resolved address per device

}  // namespace

}  // namespace copa

extern "C" copa_status_t copa_gram_noalloc(void* stream, int32_t a_is_double, const void* A, int64_t rows,
                                           int32_t R, double* G) {
  using namespace copa;
  if (!A || !G || rows < 0 || R < 1) return COPA_ERR_INVALID_ARG;
  if (R > kNoAllocMaxR) return COPA_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return COPA_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // host code cannot use the array's name as a device address: look it up once per
      // device, with that device current
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return COPA_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  const int npk = R * (R + 1) / 2;
  const int threads = npk <= 256 ? 256 : 512;
  int64_t blocks = (rows + 2047) / 2048;
  const int64_t cap = (int64_t)(kNoAllocScratchDoubles / ((size_t)R * R));
  if (blocks > cap) blocks = cap;
  if (blocks > 304) blocks = 304;
  if (blocks < 1) blocks = 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* part = reinterpret_cast<double*>(scratch);
  // every block writes its whole R x R partial, so nothing has to be cleared first
  // An error left pending by earlier, unrelated work is not this call's failure: refuse to
  // launch (and leave the error for its owner to collect) instead of clearing it.
  if (cudaPeekAtLastError() != cudaSuccess) return COPA_ERR_CUDA;
  if (a_is_double) {
    k_gram<double><<<(unsigned)blocks, threads, sizeof(double) * 64 * (size_t)R, st>>>(
        reinterpret_cast<const double*>(A), rows, R, part);
  } else {
    k_gram<float><<<(unsigned)blocks, threads, sizeof(float) * 64 * (size_t)R, st>>>(
        reinterpret_cast<const float*>(A), rows, R, part);
  }
  // the reduction must not run over the previous call's partials if the Gram did not launch
  if (cudaGetLastError() != cudaSuccess) return COPA_ERR_CUDA;
  k_reduce_rows<double><<<(R * R + 255) / 256, 256, 0, st>>>(part, (int)blocks, R * R, G);
  if (cudaGetLastError() != cudaSuccess) return COPA_ERR_CUDA;
  return COPA_OK;
}
