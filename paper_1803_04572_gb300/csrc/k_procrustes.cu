// Procrustes step of COPA (Sec. 3.1, Eq. 5; Algorithm 1 per-subject loop) and the
// fused mode-1 MTTKRP, for all subjects, over a largest-first subject order.
//
// For subject k: P_k = X_k V (I_k x R), E_k = S_k H^T, A_k = P_k E_k. With the thin SVD
// A_k = B D C^T, the update is Q_k = B C^T over the singular values kept by the rank
// cut sigma_i^2 > tau sigma_max^2. It is computed without forming A_k^T A_k (which would
// square the condition number) by one-sided (Hestenes) Jacobi on row vectors:
//   * "wide" (I_k rows rotated directly): Z = U A_k with U orthogonal (accumulated), then
//     A_k = U^T Z = U^T Sigma C^T and Q_k = U^T C_K^T (kept columns), a product of
//     orthonormal factors.
//   * "tall": a blocked Householder QR of the streamed rows gives A_k = Q_A R_A (R_A
//     upper triangular R x R); Hestenes on the rows of R_A gives Sigma and C, so
//     Omega = C_K Sigma_K^{-1} C_K^T and Q_k = A_k Omega (rows recomputed in a second pass
//     over X_k, which also accumulates T_k = sum_i q_i^T p_i).
// Outputs per subject: Q_k rows (S x R), T_k = Q_k^T P_k (= Y_k V, R x R), optionally
// Pi_k = Q_k^T Q_k = C_K C_K^T and the rank |K|; and F_H = sum_k T_k S_k through FP64
// partial sums. The same code runs in float (mixed) or double (plain FP64).
//
// Kernels (the lane-per-row ones exist for R <= 48 in float and R <= 16 in double):
//   * k_procrustes_warp: I_k <= min(R, 32), wide form, one warp per subject, lane = row.
//     Warm start (copa_fit): U of each subject is kept between outer iterations and the
//     next iteration starts the sweeps from U_prev A, which is nearly row-orthogonal once
//     the factors settle, so fewer sweeps are needed (same SVD up to rounding).
//   * k_tall_qr, k_tall_jacobi, k_tall_pass2: I_k > min(R, 32), tall form, one warp per
//     subject in each launch.
//   * k_procrustes: every subject, one 128-thread block per subject (both forms), for the
//     R and precisions the lane-per-row kernels do not cover.
#include <type_traits>

#include "copa_internal.cuh"

namespace copa {

namespace {

constexpr int kNT = 128;          // threads per CTA (one subject); 256 for R > 64
constexpr int kNWMax = 8;         // most warps per CTA (rows handled at once)
constexpr int kMaxSweeps = 30;
// After a sweep whose rotations all had |tan| below this, the next sweep would most likely
// only confirm convergence; the Jacobi kernels test every pair once from shared memory
// instead (same criterion) and stop if no pair needs a rotation.
constexpr double kTSmall = 1e-3;

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
// Tolerance of the Jacobi on the R factor of a tall subject (and of the block kernel).
// There Q_k = A_k Omega_k multiplies A_k by Omega_k = C Sigma^-1 C^T, so a residual cosine
// eps between two rows of the rotated R factor becomes an error of about eps kappa_k in
// Q_k; in a wide subject Q_k = U^T C_K is formed from the rotation itself and the same
// residual costs far less. In FP32 1e-7 sits at the rounding floor of the rotated rows;
// simulated on FP32 arithmetic at R = 40 it cut the error of Q_k eightfold against 1e-6
// for 13% more sweeps.
template <typename Real>
struct TolTall;
template <>
struct TolTall<float> {
  static __device__ __forceinline__ float v() { return 1e-7f; }
};
template <>
struct TolTall<double> {
  static __device__ __forceinline__ double v() { return 1e-14; }
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
// Square root for the rotation set-up and the rotation test: x * rsqrt(x) in float (the
// rotation is orthogonal to rounding whatever the last bits of its tangent are, since c
// and s are formed from it, and both lanes of a pair evaluate the same expression),
// IEEE in double.
__device__ __forceinline__ float sqrt_r(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

struct Lay {
  int R, ld;
  size_t Es, Zb, Pb, Ub, rv, al, vb, misc, total;  // in Real units
};

template <typename Real>
__host__ __device__ inline Lay lay_of(int R) {
  Lay L;
  L.R = R;
  L.ld = (R & 1) ? R + 2 : R + 1;   // odd leading dimension: conflict-free row/column access
  size_t o = 0;
  const size_t m = (size_t)R * L.ld;
  L.Es = o; o += m;
  L.Zb = o; o += 2 * m;
  L.Pb = o; o += m;
  L.Ub = o; o += m;
  L.rv = o; o += (size_t)kNWMax * 3 * R;   // per-warp p, a, q vectors of one row
  L.al = o; o += R;
  L.vb = o; o += R + 1;
  L.misc = o; o += 8 + kNWMax;
  L.total = o;
  return L;
}

__device__ __forceinline__ int rr_elem(int pos, int round, int n2) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (n2 - 1));
}

// Element at a round-robin position in the next round (position 0 stays at element 0).
__device__ __forceinline__ int rr_next(int e, int n2) { return e == 0 ? 0 : (e == n2 - 1 ? 1 : e + 1); }

__device__ __forceinline__ float fdiv_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_(double a, double b) { return a / b; }

// Jacobi rotation (c, s) that makes the pair with squared norms aa, bb and dot product gg
// orthogonal: x' = c x - s y, y' = s x + c y. Then |x'|^2 = aa - t gg and |y'|^2 = bb + t gg
// with t = s / c (returned in *t).
// The tangent is the smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (bb - aa) / (2 gg), in
// the form t = sign(h) gg / (|h| + sqrt(h^2 + gg^2)), h = (bb - aa) / 2, which needs one
// division fewer on the dependent path of a Jacobi round; where h^2 + gg^2 overflows it
// falls back to the form in zeta.
template <typename Real>
__device__ __forceinline__ void rotation_of(Real aa, Real bb, Real gg, Real* c, Real* s, Real* t = nullptr) {
  const Real h = Real(0.5) * (bb - aa);
  const Real q = h * h + gg * gg;
  Real tt;
  if (isfinite(q)) {
    tt = fdiv_(h >= Real(0) ? gg : -gg, fabs(h) + sqrt_r(q));
  } else {
    const Real zeta = fdiv_(bb - aa, Real(2) * gg);
    if (fabs(zeta) > Real(1e15)) tt = fdiv_(Real(0.5), zeta);
    else tt = fdiv_(zeta >= Real(0) ? Real(1) : Real(-1), fabs(zeta) + sqrt_r(Real(1) + zeta * zeta));
  }
  *c = rsqrt_(Real(1) + tt * tt);
  *s = *c * tt;
  if (t) *t = tt;
}

template <typename Real, int kR>
__device__ __forceinline__ Real sq_sum(const Real (&x)[kR]) {
  Real a4[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
  for (int t = 0; t < kR; ++t) a4[t & 3] += x[t] * x[t];
  return (a4[0] + a4[1]) + (a4[2] + a4[3]);
}

// One row of a pair split over two lanes (this lane's row x, the partner's in lane j).
// Rows are held scaled: the row is f * x, and n is its squared norm. The partner row is
// read with shuffles and both lanes form the same rotation (the same products summed in
// the same order, the same norms); each lane then updates only its own row, which in the
// scaled form is one multiply-add per component: x += m * x_partner with
// m = -+ t * f_partner / f, and f *= c (c >= 1/sqrt(2), so f stays far from underflow
// within a sweep). lo: this lane holds the pair's first row. Returns whether it rotated;
// tmx takes the largest |tan| of the rotations.
template <typename Real, int kR>
__device__ __forceinline__ bool pair_rotate(Real (&x)[kR], Real& f, Real& n, int j, bool lo, bool pair, Real tol,
                                            Real& tmx) {
  constexpr unsigned kFull = 0xffffffffu;
  Real xp[kR];
  Real g4[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    xp[t] = __shfl_sync(kFull, x[t], j);
    g4[t & 3] += x[t] * xp[t];
  }
  const Real fp = __shfl_sync(kFull, f, j), np = __shfl_sync(kFull, n, j);
  const Real gg = (f * fp) * ((g4[0] + g4[1]) + (g4[2] + g4[3]));
  const Real aa = lo ? n : np, bb = lo ? np : n;
  const bool rot = pair && gg != Real(0) && fabs(gg) > tol * sqrt_r(aa * bb);
  if (rot) {
    Real c, s, tt;
    rotation_of(aa, bb, gg, &c, &s, &tt);
    const Real m = (lo ? -tt : tt) * fdiv_(fp, f);
    tmx = fmax(tmx, fabs(tt));
#pragma unroll
    for (int t = 0; t < kR; ++t) x[t] += m * xp[t];
    f *= c;
    const Real n1 = lo ? n - tt * gg : n + tt * gg;
    n = n1 < Real(0.5) * n ? f * f * sq_sum<Real, kR>(x) : n1;
  }
  return rot;
}

constexpr int kEPL = 12;   // components per thread held in registers by the block Jacobi

template <typename Real>
__device__ __forceinline__ Real warp_sum_r(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// p_i = x_i V (lanes over components) for row i; the row's nonzeros are fetched 32 at a
// time by the lanes and broadcast, so that the V-row gathers of a row are independent.
template <typename Real>
__device__ __forceinline__ void row_times_v(const TensorView& X, int64_t i, int R, const Real* __restrict__ V,
                                            Real* __restrict__ pv) {
  const int lane = threadIdx.x & 31;
  const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
  Real acc0 = Real(0), acc1 = Real(0), acc2 = Real(0);
  for (int64_t c0 = a; c0 < b; c0 += 32) {
    const int n = (int)min((int64_t)32, b - c0);
    int col = 0;
    Real x = Real(0);
    if (lane < n) {
      col = __ldg(X.col + c0 + lane);
      x = load_x<Real>(X, c0 + lane);
    }
    for (int q = 0; q < n; ++q) {
      const int cq = __shfl_sync(0xffffffffu, col, q);
      const Real xq = __shfl_sync(0xffffffffu, x, q);
      const Real* vr = V + (int64_t)cq * R;
      if (lane < R) acc0 += xq * __ldg(vr + lane);
      if (lane + 32 < R) acc1 += xq * __ldg(vr + lane + 32);
      if (lane + 64 < R) acc2 += xq * __ldg(vr + lane + 64);
    }
  }
  if (lane < R) pv[lane] = acc0;
  if (lane + 32 < R) pv[lane + 32] = acc1;
  if (lane + 64 < R) pv[lane + 64] = acc2;
}

// out = p M (lanes over t); M[r][t] at r*ld + t
template <typename Real>
__device__ __forceinline__ void vec_times_mat(const Real* __restrict__ p, const Real* __restrict__ M, int ld,
                                              int R, Real* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < R; t += 32) {
    Real a0 = Real(0), a1 = Real(0);
    int r = 0;
    for (; r + 1 < R; r += 2) {
      a0 += p[r] * M[r * ld + t];
      a1 += p[r + 1] * M[(r + 1) * ld + t];
    }
    if (r < R) a0 += p[r] * M[r * ld + t];
    out[t] = a0 + a1;
  }
}

// Householder QR update of the stacked [R_A (R x R, rows 0..R-1 of Z); block (nb rows,
// rows R..R+nb-1 of Z)]: afterwards Z[0..R-1] holds the new R factor and the block is 0.
// Thread c owns column c; warp 0 forms each reflector.
template <typename Real, int NT>
__device__ void tsqr_block(Real* Z, int ld, int R, int nb, Real* vb, Real* misc) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int j = 0; j < R; ++j) {
    if (tid < 32) {
      Real ss = Real(0);
      for (int i = lane; i < nb; i += 32) {
        const Real v = Z[(R + i) * ld + j];
        ss += v * v;
      }
      ss = warp_sum_r(ss);
      const Real x0 = Z[j * ld + j];
      Real tau = Real(0), scale = Real(0), beta = x0;
      if (ss > Real(0)) {
        const Real nrm = sqrt(x0 * x0 + ss);
        beta = x0 >= Real(0) ? -nrm : nrm;
        tau = (beta - x0) / beta;
        scale = Real(1) / (x0 - beta);
      }
      __syncwarp();
      for (int i = lane; i < nb; i += 32) {
        vb[i] = Z[(R + i) * ld + j] * scale;
        if (tau != Real(0)) Z[(R + i) * ld + j] = Real(0);
      }
      if (lane == 0) {
        misc[0] = tau;
        Z[j * ld + j] = beta;
      }
    }
    __syncthreads();
    const Real tau = misc[0];
    if (tau != Real(0)) {
      for (int c = j + 1 + threadIdx.x; c < R; c += NT) {
        Real w0 = Z[j * ld + c], w1 = Real(0);
        int i = 0;
        for (; i + 1 < nb; i += 2) {
          w0 += vb[i] * Z[(R + i) * ld + c];
          w1 += vb[i + 1] * Z[(R + i + 1) * ld + c];
        }
        if (i < nb) w0 += vb[i] * Z[(R + i) * ld + c];
        const Real w = (w0 + w1) * tau;
        Z[j * ld + c] -= w;
        for (int q = 0; q < nb; ++q) Z[(R + q) * ld + c] -= vb[q] * w;
      }
    }
    __syncthreads();
  }
}

// A warm start reuses U from the previous outer iteration. Each rotation is orthogonal
// only to rounding, so U drifts from orthogonality by about 1e-7 per iteration; every
// kReorth-th iteration of a fit the loaded U is re-orthonormalised (modified Gram-Schmidt
// on its rows, two passes) before it is applied, which bounds the drift.
constexpr unsigned kReorth = 16;

// Modified Gram-Schmidt (two passes) on the rows of the m x m matrix U[r * ld + c], by the
// whole block; red[0] is shared scratch.
template <typename Real>
__device__ void mgs2_rows_block(Real* U, int m, int ld, Real* red) {
  const int tid = threadIdx.x;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < m; ++i) {
      if (tid < 32) {
        Real ss = Real(0);
        for (int c = tid; c < m; c += 32) ss += U[i * ld + c] * U[i * ld + c];
        ss = warp_sum(ss);
        if (tid == 0) red[0] = Real(1) / sqrt(ss);
      }
      __syncthreads();
      const Real inv = red[0];
      for (int c = tid; c < m; c += blockDim.x) U[i * ld + c] *= inv;
      __syncthreads();
      for (int r = i + 1 + tid; r < m; r += blockDim.x) {
        Real d = Real(0);
        for (int c = 0; c < m; ++c) d += U[r * ld + c] * U[i * ld + c];
        for (int c = 0; c < m; ++c) U[r * ld + c] -= d * U[i * ld + c];
      }
      __syncthreads();
    }
  }
}

// Block kernel, one 128-thread CTA per subject. Rows of X_k are handled four at a time,
// one per warp (lanes over the R components); the Jacobi pairs of a round are spread over
// the block with LP = 128 / pairs threads per pair (a power of two), each thread holding
// R / LP components of the two vectors and the pair's dot products reduced by shuffles;
// one barrier per round.
template <typename Real, int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 5 : 2) k_procrustes(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V,
    const Real* __restrict__ W, double tau_rank, Real* __restrict__ Q, Real* T,
    Real* __restrict__ Pi, int32_t* __restrict__ rank, double* __restrict__ fh_partial,
    const int64_t* __restrict__ order, int* __restrict__ counter,
    unsigned long long* __restrict__ fma_count, Real* __restrict__ Uw,
    const int64_t* __restrict__ woff, int warm_in, const int* __restrict__ epoch, const int* __restrict__ limit,
    const int* __restrict__ first) {
  extern __shared__ unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const Lay L = lay_of<Real>(R);
  const int ld = L.ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Real* Es = sm + L.Es;   // E[r][t] = w_r H[t][r]
  Real* Zb = sm + L.Zb;   // rows 0..R-1: A_k rows / R_A / c_j; rows R..2R-1: QR block, B
  Real* Pb = sm + L.Pb;   // wide: p rows; tall: Omega
  Real* Ub = sm + L.Ub;   // U (wide, or any subject with a warm-start buffer); tall: then T
  Real* pvw = sm + L.rv + (size_t)warp * 3 * R;   // this warp's p, a, q
  Real* avw = pvw + R;
  Real* qvw = avw + R;
  Real* al = sm + L.al;
  Real* vb = sm + L.vb;
  Real* misc = sm + L.misc;
  int* sidx = reinterpret_cast<int*>(misc + 8);
  const Real tol = TolTall<Real>::v();
  unsigned long long fma = 0;   // work tally (thread 0), for the roofline
  // subjects order[kbeg .. kend) are this kernel's; the others take the lane-per-row kernels
  const int64_t kend = limit ? min((int64_t)max(*limit, 0), X.K) : X.K;
  const int64_t kbeg = first ? min((int64_t)max(*first, 0), kend) : 0;

  double* fh = fh_partial ? fh_partial + (size_t)blockIdx.x * R * R : nullptr;
  if (fh)
    for (int i = tid; i < R * R; i += NT) fh[i] = 0.0;

  while (true) {
    __syncthreads();
    if (tid == 0) sidx[0] = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t idx = kbeg + sidx[0];
    if (idx >= kend) break;
    const int64_t k = order ? order[idx] : idx;
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    const int64_t Ik64 = r1 - r0;
    const bool wide = Ik64 <= R;
    const int m = wide ? (int)Ik64 : R;
    if (tid == 0) {
      const unsigned long long nnzk = (unsigned long long)(X.row_ptr[r1] - X.row_ptr[r0]);
      const unsigned long long ik = (unsigned long long)Ik64, RR = (unsigned long long)R * R;
      fma += 2ull * m * R;
      if (wide) fma += nnzk * R + ik * RR + 2ull * m * m * R + 2ull * RR * m;
      else fma += 2 * nnzk * R + 5 * ik * RR + 2 * RR * R;
    }

    // ---- E = S_k H^T; tall: clear R_A ----
    for (int e = tid; e < R * R; e += NT) {
      const int r = e / R, t = e - r * R;
      Es[r * ld + t] = W[k * R + r] * __ldg(H + t * R + r);
      if (!wide) Zb[r * ld + t] = Real(0);
    }
    __syncthreads();

    // ---- pass 1: rows four at a time, a_i = (x_i V) E; wide: keep p_i and a_i;
    //      tall: fill a QR block of up to R rows, then fold it into R_A ----
    int nb = 0;   // rows in the QR block (tall); always < R before a group
    for (int64_t g = r0; g < r1;) {
      int nrow = (int)min((int64_t)(NT / 32), r1 - g);
      if (!wide && nrow > R - nb) nrow = R - nb;   // the block holds at most R rows
      const int64_t i = g + warp;
      if (warp < nrow) {
        row_times_v<Real>(X, i, R, V, pvw);
        __syncwarp();
        const int row = wide ? (int)(i - r0) : R + nb + warp;
        vec_times_mat<Real>(pvw, Es, ld, R, Zb + row * ld);
        if (wide)
          for (int t = lane; t < R; t += 32) Pb[row * ld + t] = pvw[t];
      }
      __syncthreads();
      g += nrow;
      if (!wide) {
        nb += nrow;
        if (nb == R || g >= r1) {
          tsqr_block<Real, NT>(Zb, ld, R, nb, vb, misc);
          nb = 0;
        }
      }
    }

    // ---- Hestenes one-sided Jacobi on rows 0..m-1 of Zb. U (Z = U A) is accumulated for
    //      wide subjects (it gives Q) and whenever a warm-start buffer is given; a warm
    //      start begins from the previous outer iteration's U: Z = U_prev A. Tall subjects
    //      need only Sigma and C (the rows of Z), so they keep no U: accumulating it would
    //      cost more per sweep than a warm start saves in sweeps there. ----
    const bool accU = wide;
    Real* Uk = (wide && Uw) ? Uw + woff[k] : nullptr;
    if (accU) {
      for (int e = tid; e < m * m; e += NT) {
        const int r = e / m, t = e - r * m;
        Ub[r * ld + t] = (Uk && warm_in) ? Uk[e] : ((r == t) ? Real(1) : Real(0));
      }
      __syncthreads();
      if (Uk && warm_in && epoch && ((unsigned)__ldg(epoch) % kReorth) == 0u) mgs2_rows_block<Real>(Ub, m, ld, misc);
      if (Uk && warm_in) {
        for (int e = tid; e < m * R; e += NT) {
          const int i = e / R, t = e - i * R;
          Real acc = Real(0);
          for (int j = 0; j < m; ++j) acc += Ub[i * ld + j] * Zb[j * ld + t];
          Zb[(R + i) * ld + t] = acc;
        }
        __syncthreads();
        for (int e = tid; e < m * R; e += NT) {
          const int i = e / R, t = e - i * R;
          Zb[i * ld + t] = Zb[(R + i) * ld + t];
        }
        __syncthreads();
        if (tid == 0) fma += (unsigned long long)m * m * R;
      }
    }
    const int n2 = m + (m & 1);
    const int npairs = n2 / 2;
    int LP = 1;
    while (LP < 32 && npairs * LP * 2 <= NT) LP <<= 1;
    const int pj = tid / LP, sl = tid % LP;
    const bool act = pj < npairs;
    const bool few = (R + LP - 1) / LP <= kEPL && (m + LP - 1) / LP <= kEPL;
    for (int sweep = 0; sweep < kMaxSweeps && n2 > 1; ++sweep) {
      int nrot = 0;
      int e1 = act ? rr_elem(pj, 0, n2) : 0, e2 = act ? rr_elem(n2 - 1 - pj, 0, n2) : 0;
      for (int round = 0; round < n2 - 1; ++round) {
        bool rotated = false;
        const int ii = e1 < e2 ? e1 : e2, jj = e1 < e2 ? e2 : e1;
        e1 = rr_next(e1, n2);
        e2 = rr_next(e2, n2);
        const bool real_pair = act && jj < m;
        Real* zi = Zb + ii * ld;
        Real* zj = Zb + jj * ld;
        if (few) {
          // at most kEPL components per thread: keep them in registers for the update
          Real xi[kEPL], xj[kEPL];
          Real aa = Real(0), bb = Real(0), gg = Real(0);
#pragma unroll
          for (int q = 0; q < kEPL; ++q) {
            const int t = sl + q * LP;
            const bool in = real_pair && t < R;
            xi[q] = in ? zi[t] : Real(0);
            xj[q] = in ? zj[t] : Real(0);
            aa += xi[q] * xi[q];
            bb += xj[q] * xj[q];
            gg += xi[q] * xj[q];
          }
          for (int o = LP >> 1; o > 0; o >>= 1) {
            aa += __shfl_xor_sync(0xffffffffu, aa, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
            gg += __shfl_xor_sync(0xffffffffu, gg, o);
          }
          if (real_pair && gg != Real(0) && fabs(gg) > tol * sqrt(aa * bb)) {
            Real c, s;
            rotation_of(aa, bb, gg, &c, &s);
#pragma unroll
            for (int q = 0; q < kEPL; ++q) {
              const int t = sl + q * LP;
              if (t < R) {
                zi[t] = c * xi[q] - s * xj[q];
                zj[t] = s * xi[q] + c * xj[q];
              }
            }
            if (accU) {
              Real* ui = Ub + ii * ld;
              Real* uj = Ub + jj * ld;
#pragma unroll
              for (int q = 0; q < kEPL; ++q) {
                const int t = sl + q * LP;
                if (t < m) {
                  const Real x = ui[t], y = uj[t];
                  ui[t] = c * x - s * y;
                  uj[t] = s * x + c * y;
                }
              }
            }
            rotated = sl == 0;
          }
        } else {
          Real aa = Real(0), bb = Real(0), gg = Real(0);
          if (real_pair)
            for (int t = sl; t < R; t += LP) {
              const Real x = zi[t], y = zj[t];
              aa += x * x;
              bb += y * y;
              gg += x * y;
            }
          // reduce over the LP threads of the pair (aligned groups inside one warp)
          for (int o = LP >> 1; o > 0; o >>= 1) {
            aa += __shfl_xor_sync(0xffffffffu, aa, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
            gg += __shfl_xor_sync(0xffffffffu, gg, o);
          }
          if (real_pair && gg != Real(0) && fabs(gg) > tol * sqrt(aa * bb)) {
            Real c, s;
            rotation_of(aa, bb, gg, &c, &s);
            for (int t = sl; t < R; t += LP) {
              const Real x = zi[t], y = zj[t];
              zi[t] = c * x - s * y;
              zj[t] = s * x + c * y;
            }
            if (accU) {
              Real* ui = Ub + ii * ld;
              Real* uj = Ub + jj * ld;
              for (int t = sl; t < m; t += LP) {
                const Real x = ui[t], y = uj[t];
                ui[t] = c * x - s * y;
                uj[t] = s * x + c * y;
              }
            }
            rotated = sl == 0;
          }
        }
        nrot += __syncthreads_count(rotated);
      }
      if (tid == 0)
        fma += (unsigned long long)(m * (m - 1) / 2) * 3 * R + (unsigned long long)nrot * 4 * (R + (accU ? m : 0));
      if (nrot == 0) break;
    }
    if (Uk)
      for (int e = tid; e < m * m; e += NT) Uk[e] = Ub[(e / m) * ld + (e % m)];

    // ---- singular values, rank cut, normalised right singular vectors c_j ----
    for (int j = tid; j < m; j += NT) {
      Real acc = Real(0);
      for (int t = 0; t < R; ++t) acc += Zb[j * ld + t] * Zb[j * ld + t];
      al[j] = acc;
    }
    __syncthreads();
    if (tid < 32) {
      Real amax = Real(0);
      for (int j = lane; j < m; j += 32) amax = al[j] > amax ? al[j] : amax;
      amax = warp_max(amax);
      int kept = 0;
      for (int j = lane; j < m; j += 32) {
        const bool keep = amax > Real(0) && (double)al[j] > tau_rank * (double)amax;
        al[j] = keep ? rsqrt_(al[j]) : Real(0);   // 1 / sigma_j, 0 if dropped
        kept += keep ? 1 : 0;
      }
      kept = warp_sum(kept);
      if (rank && lane == 0) rank[k] = kept;
    }
    __syncthreads();
    for (int e = tid; e < m * R; e += NT) {
      const int j = e / R, t = e - j * R;
      Zb[j * ld + t] *= al[j];
    }
    __syncthreads();

    Real* Tk = T + k * R * R;
    if (wide) {
      // Q rows q_i = sum_j U[j][i] c_j; B = U P -> rows R.. of Zb
      for (int e = tid; e < m * R; e += NT) {
        const int i = e / R, t = e - i * R;
        Real acc = Real(0), bacc = Real(0);
        for (int j = 0; j < m; ++j) {
          acc += Ub[j * ld + i] * Zb[j * ld + t];
          bacc += Ub[i * ld + j] * Pb[j * ld + t];
        }
        Q[(r0 + i) * R + t] = acc;
        Zb[(R + i) * ld + t] = bacc;
      }
      __syncthreads();
      for (int e = tid; e < R * R; e += NT) {
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
    } else {
      // Omega = sum_j c_j c_j^T / sigma_j -> Pb; Pi -> global
      for (int e = tid; e < R * R; e += NT) {
        const int r = e / R, t = e - r * R;
        Real acc = Real(0), pacc = Real(0);
        for (int j = 0; j < R; ++j) {
          const Real cc = Zb[j * ld + r] * Zb[j * ld + t];
          acc += cc * al[j];
          pacc += cc;
        }
        Pb[r * ld + t] = acc;
        if (Pi) Pi[k * R * R + e] = pacc;
        Ub[r * ld + t] = Real(0);
      }
      __syncthreads();
      // pass 2, rows four at a time: q_i = (p_i E) Omega; T_k += q_i^T p_i
      for (int64_t g = r0; g < r1; g += (NT / 32)) {
        const int64_t i = g + warp;
        const int nrow = (int)min((int64_t)(NT / 32), r1 - g);
        if (warp < nrow) {
          row_times_v<Real>(X, i, R, V, pvw);
          __syncwarp();
          vec_times_mat<Real>(pvw, Es, ld, R, avw);
          __syncwarp();
          vec_times_mat<Real>(avw, Pb, ld, R, qvw);
          __syncwarp();
          for (int t = lane; t < R; t += 32) Q[i * R + t] = qvw[t];
        }
        __syncthreads();
        for (int e = tid; e < R * R; e += NT) {
          const int r = e / R, s = e - r * R;
          Real acc = Ub[r * ld + s];
          for (int w = 0; w < nrow; ++w) {
            const Real* base = sm + L.rv + (size_t)w * 3 * R;
            acc += base[2 * R + r] * base[s];
          }
          Ub[r * ld + s] = acc;
        }
        __syncthreads();
      }
      for (int e = tid; e < R * R; e += NT) {
        const int r = e / R, s = e - r * R;
        const Real acc = Ub[r * ld + s];
        Tk[e] = acc;
        if (fh) fh[e] += (double)acc * (double)W[k * R + s];
      }
    }
  }
  if (fma_count && tid == 0) atomicAdd(fma_count, fma);
}

// p = x_i V for the visit row i of this lane (components padded to kR with zeros): the
// row's column indices and values are fetched four at a time before their V rows, so that
// the dependent gathers of a row overlap. Returns the row's number of nonzeros.
template <typename Real, int kR>
__device__ __forceinline__ int row_p(const TensorView& X, int R, const Real* __restrict__ V, int64_t i, bool valid,
                                     Real* p) {
#pragma unroll
  for (int t = 0; t < kR; ++t) p[t] = Real(0);
  if (!valid) return 0;
  const int64_t a = X.row_ptr[i], b = X.row_ptr[i + 1];
  for (int64_t q0 = a; q0 < b; q0 += 4) {
    int c[4];
    Real x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = q0 + u < b;
      c[u] = in ? __ldg(X.col + q0 + u) : 0;
      x[u] = in ? load_x<Real>(X, q0 + u) : Real(0);
    }
    if constexpr (std::is_same<Real, float>::value && kR % 4 == 0) {
      if ((R & 3) == 0) {   // 16-byte rows of V: float4 loads
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4* vr = reinterpret_cast<const float4*>(V + (int64_t)c[u] * R);
#pragma unroll
          for (int t4 = 0; t4 < kR / 4; ++t4) {
            if (4 * t4 < R) {
              const float4 v = __ldg(vr + t4);
              p[4 * t4] += x[u] * v.x;
              p[4 * t4 + 1] += x[u] * v.y;
              p[4 * t4 + 2] += x[u] * v.z;
              p[4 * t4 + 3] += x[u] * v.w;
            }
          }
        }
        continue;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const Real* vr = V + (int64_t)c[u] * R;
#pragma unroll
      for (int t = 0; t < kR; ++t)
        if (t < R) p[t] += x[u] * __ldg(vr + t);
    }
  }
  return (int)(b - a);
}

// ---- warp-per-subject path for the many small subjects (I_k <= min(R, 32)) ----
// One warp per subject, lane i holding row i of A_k (then of Z = U A_k) and row i of U in
// registers, so that a Jacobi round needs no block barrier: the partner row is read with
// shuffles and both lanes of a pair compute the same rotation from the same three dot
// products. Pairs follow the circle method on n2 = m + (m & 1) positions: position n2-1
// meets position r in round r, every other position i meets (2r - i) mod (n2 - 1).
// Rows are zero-padded to kR components (R rounded up to a multiple of 8); padding stays 0
// under the rotations. Shared-memory rows have a 16-byte aligned stride, so that the
// warp-wide (broadcast) row reads are vector loads; the stride is chosen so that the
// lane-per-row vector stores of a quarter warp fall in distinct banks.
// Outputs are the same as the block path's wide branch. With kSeg = 16 a warp takes two
// subjects of I_k <= 16, one per half (lane = row within the half, partners and reductions
// inside the half); both halves run the rounds of the larger, the outputs go out one subject
// at a time. It runs the schedule's smallest subjects at half the instructions per subject.
constexpr int kWNT = 128;   // threads per block of the warp path (4 subjects at a time)

template <typename Real>
struct Vec16;   // 16-byte vector of Real
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int n = 4;
  static __device__ __forceinline__ void ld(const float* p, float* o) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ void st(float* p, const float* o) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int n = 2;
  static __device__ __forceinline__ void ld(const double* p, double* o) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
  static __device__ __forceinline__ void st(double* p, const double* o) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  }
};

template <typename Real, int kR>
struct WarpLay {
  static constexpr int kM = kR < 32 ? kR : 32;   // rows of a subject on this path
  static constexpr int VN = Vec16<Real>::n;
  static constexpr int ld = kR + VN;             // row stride of the row buffers
  static constexpr int ldu = kM + 1;             // U: odd stride, read by columns
  static constexpr int per_warp = 2 * kM * ld + kM * ldu + 2 * kR + VN;   // two W rows (paired subjects)
  static constexpr size_t bytes = sizeof(Real) * ((size_t)kR * kR + (kWNT / 32) * (size_t)per_warp) + 16;
  static_assert(kM * ld + kM * ldu >= kR * kR && kM * ld + kM * ldu >= kM * kR,
                "the B2 and U buffers stage T_k and the Q rows");
};

template <typename Real, int kR, int kSeg>
__global__ void __launch_bounds__(kWNT, 3) k_procrustes_warp(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V,
    const Real* __restrict__ W, double tau_rank, Real* __restrict__ Q, Real* __restrict__ T,
    Real* __restrict__ Pi, int32_t* __restrict__ rank,
    const int64_t* __restrict__ order, const int* __restrict__ first, const int* __restrict__ last,
    int* __restrict__ counter,
    unsigned long long* __restrict__ fma_count, Real* __restrict__ Uw,
    const int64_t* __restrict__ woff, int warm_in, const int* __restrict__ epoch, int* __restrict__ status) {
  using Lw = WarpLay<Real, kR>;
  using Vc = Vec16<Real>;
  constexpr int kM = Lw::kM, ld = Lw::ld, ldu = Lw::ldu, VN = Lw::VN;
  constexpr int kTR = kR / 8, kTC = kR / 4;   // T tile of a lane: 8 x 4 lanes cover kR x kR
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Hs = reinterpret_cast<Real*>(smem_raw);   // Hs[r * kR + t] = H(t, r), zero-padded
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // kSeg = 16: two subjects (I_k <= 16) per warp, one per half, lane = row within the half
  constexpr int kMs = kM < kSeg ? kM : kSeg;   // rows of a subject
  constexpr int kNS = 32 / kSeg;               // subjects per warp
  static_assert(kSeg == 32 || kM == 32, "paired subjects need 32 buffer rows");
  const int seg = lane / kSeg, sl = lane - seg * kSeg, sb = seg * kSeg;
  const unsigned segmask = kSeg == 32 ? kFull : (0xffffu << sb);
  Real* B1 = Hs + kR * kR + (size_t)warp * Lw::per_warp;   // A rows, then c_j rows
  Real* B2 = B1 + kM * ld;                                  // p rows, then b = U P rows
  Real* Us = B2 + kM * ld;                                  // U, for its transpose
  Real* Wb = Us + kM * ldu;                                 // the subjects' rows of W
  for (int e = threadIdx.x; e < kR * kR; e += kWNT) {
    const int r = e / kR, t = e - r * kR;
    Hs[e] = (t < R && r < R) ? H[t * R + r] : Real(0);
  }
  __syncthreads();
  const Real tol = Tol<Real>::v();
  // schedule positions [first, last) (last NULL: to the end)
  const int64_t k1 = last ? min((int64_t)max(*last, 0), X.K) : X.K;
  const int64_t k0 = min((int64_t)max(*first, 0), k1);
  const int tr = lane >> 2, tc = lane & 3;
  unsigned long long fma = 0;

  while (true) {
    int claim = 0;
    if (lane == 0) claim = atomicAdd(counter, kNS);
    const int64_t idx0 = k0 + __shfl_sync(kFull, claim, 0);
    if (idx0 >= k1) break;
    const int64_t idx = idx0 + seg;
    const bool has = idx < k1;   // a half without a subject runs on m = 0 and writes nothing
    const int64_t k = order[has ? idx : idx0];
    const int64_t r0 = X.subj_ptr[k];
    const int64_t ik = has ? X.subj_ptr[k + 1] - r0 : 0;
    if (ik > kMs && sl == 0)   // the schedule split guarantees I_k <= kMs; record and skip
      set_status(status, COPA_ERR_CUDA, (int)k);
    const bool out = has && ik <= kMs;
    const int m = out ? (int)ik : 0;
    const int mmax = kNS == 1 ? m : __reduce_max_sync(kFull, m);
    const Real* wk = W + k * R;
    Real* Wbs = Wb + seg * kR;
    for (int r = sl; r < kR; r += kSeg) Wbs[r] = r < R ? wk[r] : Real(0);

    // ---- p_i = x_i V (lane i); a_i = (p_i * w) H^T ----
    Real p[kR];
    const int nnz_row = row_p<Real, kR>(X, R, V, r0 + sl, sl < m, p);
    if (lane < kM) {
#pragma unroll
      for (int t = 0; t < kR; t += VN) Vc::st(B2 + lane * ld + t, p + t);
    }
    __syncwarp();
    Real z[kR];
#pragma unroll
    for (int t = 0; t < kR; ++t) z[t] = Real(0);
    if (sl < m) {
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const Real pw = B2[lane * ld + r] * Wbs[r];
#pragma unroll
        for (int t = 0; t < kR; t += VN) {
          Real hv[VN];
          Vc::ld(Hs + r * kR + t, hv);
#pragma unroll
          for (int q = 0; q < VN; ++q) z[t + q] += pw * hv[q];
        }
      }
    }

    // ---- U: identity, or the previous outer iteration's rotation (then Z = U_prev A) ----
    Real* Uk = Uw ? Uw + woff[k] : nullptr;
    const bool warm = Uk != nullptr && warm_in != 0;
    Real u[kMs];
#pragma unroll
    for (int j = 0; j < kMs; ++j) u[j] = (!warm && j == sl && sl < m) ? Real(1) : Real(0);
    if (warm) {
      if (lane < kM) {
#pragma unroll
        for (int t = 0; t < kR; t += VN) Vc::st(B1 + lane * ld + t, z + t);
      }
      // U_prev (m x m, contiguous) through Us: contiguous row copies, then lane = row
      for (int r = 0; r < mmax; ++r)
        if (r < m && sl < m) Us[(sb + r) * ldu + sl] = Uk[r * m + sl];
      __syncwarp();
      if (sl < m) {
#pragma unroll
        for (int j = 0; j < kMs; ++j)
          if (j < m) u[j] = Us[lane * ldu + j];
      }
      if (epoch && ((unsigned)__ldg(epoch) % kReorth) == 0u) {
        // modified Gram-Schmidt on the rows of U_prev (lane = row), two passes
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 1
          for (int i = 0; i < mmax; ++i) {
            const bool act = i < m;   // row i exists in this lane's subject
            Real ss = Real(0);
#pragma unroll
            for (int jj = 0; jj < kMs; ++jj) ss += u[jj] * u[jj];
            const Real si = __shfl_sync(kFull, ss, sb + i);
            const Real inv = act ? Real(1) / sqrt(si) : Real(0);
            Real d = Real(0);
#pragma unroll
            for (int jj = 0; jj < kMs; ++jj) {
              const Real ui = __shfl_sync(kFull, u[jj], sb + i) * inv;
              if (act && sl == i) u[jj] = ui;
              d += u[jj] * ui;
            }
            // (lane i's d is its own squared norm, 1; it does not update)
            const Real dd = act && sl > i && sl < m ? d : Real(0);
#pragma unroll
            for (int jj = 0; jj < kMs; ++jj) u[jj] -= dd * __shfl_sync(kFull, u[jj], sb + i);
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kR; ++t) z[t] = Real(0);
      if (sl < m) {
#pragma unroll
        for (int j = 0; j < kMs; ++j) {
          if (j < m) {
#pragma unroll
            for (int t = 0; t < kR; t += VN) {
              Real av[VN];
              Vc::ld(B1 + (sb + j) * ld + t, av);
#pragma unroll
              for (int q = 0; q < VN; ++q) z[t + q] += u[j] * av[q];
            }
          }
        }
      }
      __syncwarp();
    }

    // ---- Hestenes sweeps. The lane's rows of Z and U are held scaled by f (the rows are
    //      f z and f u), so that a rotation is one multiply-add per component (see
    //      pair_rotate); f is folded back at the start of every sweep. The squared row norm
    //      al is exact at the start of every sweep and for the rank cut; within a sweep a
    //      rotation updates it by -+ t * gamma, recomputed where it drops by half or more
    //      (so that its rounding stays relative). ----
    auto fold = [&](Real f) {
#pragma unroll
      for (int t = 0; t < kR; ++t) z[t] *= f;
#pragma unroll
      for (int jj = 0; jj < kMs; ++jj) u[jj] *= f;
    };
    Real al = Real(0), f = Real(1);
    const int n2 = m + (m & 1), n2max = mmax + (mmax & 1);
    unsigned long long nrot = 0;
    int sweeps = 0;
    for (int sweep = 0; sweep < kMaxSweeps && n2max > 1; ++sweep) {
      ++sweeps;
      bool any = false;
      Real tmx = Real(0);   // largest |tan| of this lane's rotations in the sweep
      fold(f);
      f = Real(1);
      al = sq_sum<Real, kR>(z);
      for (int rd = 0; rd < n2max - 1; ++rd) {
        int jl;   // partner row within the subject
        if (sl >= n2 || rd >= n2 - 1) jl = sl;
        else if (sl == n2 - 1) jl = rd;
        else if (sl == rd) jl = n2 - 1;
        else {
          jl = 2 * rd - sl;
          if (jl < 0) jl += n2 - 1;
          else if (jl >= n2 - 1) jl -= n2 - 1;
        }
        const int j = sb + jl;
        Real zp[kR];
        Real g[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int t = 0; t < kR; ++t) {
          zp[t] = __shfl_sync(kFull, z[t], j);
          g[t & 3] += z[t] * zp[t];
        }
        const Real be = __shfl_sync(kFull, al, j), fp = __shfl_sync(kFull, f, j);
        const bool lo = lane < j;
        const Real aa = lo ? al : be, bb = lo ? be : al;
        const Real gg = (f * fp) * ((g[0] + g[1]) + (g[2] + g[3]));
        const bool rot = j != lane && gg != Real(0) && fabs(gg) > tol * sqrt_r(aa * bb);
        const unsigned rmask = __ballot_sync(kFull, rot);
        if (rmask == 0u) continue;
        any = true;
        nrot += __popc(rmask) / 2;
        // lower row x, upper row y: x' = c x - s y, y' = s x + c y; in the scaled form
        // the own row takes -+ t (fp / f) times the partner's and the scale takes c
        Real mu = Real(0);
        if (rot) {
          Real c, s, tt;
          rotation_of(aa, bb, gg, &c, &s, &tt);
          mu = (lo ? -tt : tt) * fdiv_(fp, f);
          tmx = fmax(tmx, fabs(tt));
#pragma unroll
          for (int t = 0; t < kR; ++t) z[t] += mu * zp[t];
          f *= c;
          const Real al1 = lo ? al - tt * gg : al + tt * gg;
          al = al1 < Real(0.5) * al ? f * f * sq_sum<Real, kR>(z) : al1;
        }
        // U rows, in chunks of 8 entries up to m
#pragma unroll
        for (int c8 = 0; c8 < kMs; c8 += 8) {
          if (c8 < mmax) {
#pragma unroll
            for (int jj = c8; jj < c8 + 8; ++jj) {
              const Real up = __shfl_sync(kFull, u[jj], j);
              u[jj] += mu * up;
            }
          }
        }
      }
      if (!any) break;
      if (warp_max(tmx) < Real(kTSmall) && sweep + 1 < kMaxSweeps) {
        // confirm convergence without a sweep: rows (scales folded) and squared norms to
        // shared memory (B1 and Us are free during the sweeps), every pair tested once
        fold(f);
        f = Real(1);
        al = sq_sum<Real, kR>(z);
        if (lane < kM) {
#pragma unroll
          for (int t = 0; t < kR; t += VN) Vc::st(B1 + lane * ld + t, z + t);
          Us[lane] = al;
        }
        __syncwarp();
        bool bad = false;
        if (sl < m) {
#pragma unroll 1
          for (int jj = 0; jj < m; ++jj) {
            Real g4[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
            for (int t = 0; t < kR; t += VN) {
              Real rv[VN];
              Vc::ld(B1 + (sb + jj) * ld + t, rv);
#pragma unroll
              for (int q = 0; q < VN; ++q) g4[(t + q) & 3] += z[t + q] * rv[q];
            }
            const Real gg = (g4[0] + g4[1]) + (g4[2] + g4[3]);
            bad |= jj != sl && gg != Real(0) && fabs(gg) > tol * sqrt(al * Us[sb + jj]);
          }
        }
        __syncwarp();
        if (!__any_sync(kFull, bad)) {
          ++sweeps;   // the test stood in for the confirming sweep
          break;
        }
      }
    }
    fold(f);
    al = sq_sum<Real, kR>(z);

    // ---- rank cut; c_i = z_i / sigma_i for kept rows, 0 otherwise ----
    Real amax = al;   // largest squared row norm of the subject
#pragma unroll
    for (int o = kSeg / 2; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(kFull, amax, o));
    const bool keep = sl < m && amax > Real(0) && (double)al > tau_rank * (double)amax;
    const int kept = __popc(__ballot_sync(kFull, keep) & segmask);
    if (rank && sl == 0 && out) rank[k] = kept;
    const Real inv = keep ? rsqrt_(al) : Real(0);
    if (lane < kM) {
#pragma unroll
      for (int t = 0; t < kR; ++t) z[t] *= inv;
#pragma unroll
      for (int t = 0; t < kR; t += VN) Vc::st(B1 + lane * ld + t, z + t);
#pragma unroll
      for (int jj = 0; jj < kMs; ++jj) Us[lane * ldu + jj] = u[jj];
    }
    __syncwarp();
    if (Uk && out) {   // this iteration's U for the next one: contiguous row copies from Us
      for (int r = 0; r < m; ++r)
        if (sl < m) Uk[r * m + sl] = Us[(sb + r) * ldu + sl];
    }

    // ---- q_i = sum_j U(j, i) c_j and b_i = sum_j U(i, j) p_j ----
#pragma unroll
    for (int t = 0; t < kR; ++t) { z[t] = Real(0); p[t] = Real(0); }
    if (sl < m) {
#pragma unroll 1
      for (int jj = 0; jj < m; ++jj) {
        const Real uji = Us[(sb + jj) * ldu + sl], uij = Us[lane * ldu + jj];
#pragma unroll
        for (int t = 0; t < kR; t += VN) {
          Real cv[VN], pv[VN];
          Vc::ld(B1 + (sb + jj) * ld + t, cv);
          Vc::ld(B2 + (sb + jj) * ld + t, pv);
#pragma unroll
          for (int q = 0; q < VN; ++q) {
            z[t + q] += uji * cv[q];
            p[t + q] += uij * pv[q];
          }
        }
      }
    }
    __syncwarp();
    if (lane < kM) {
#pragma unroll
      for (int t = 0; t < kR; t += VN) Vc::st(B2 + lane * ld + t, p + t);
    }
    __syncwarp();

    // ---- T_k = sum_j c_j^T b_j (lane tile kTR x kTC), optional Pi_k, one subject at a
    //      time (the whole warp). With one subject per warp, T_k and the rows q_i go out
    //      through shared memory (the B2 and U buffers, free by then), so that the global
    //      stores are contiguous; with two, T_k and Pi_k go out from the tiles (rows of kTC
    //      contiguous values) and the q rows of both subjects through shared memory. ----
    Real* St = B2;   // staging: B2 and Us are adjacent and hold >= max(R * R, kM * R) values
#pragma unroll 1
    for (int s2 = 0; s2 < kNS; ++s2) {
      const int base = s2 * kSeg;
      const int ms = kNS == 1 ? m : __shfl_sync(kFull, m, base);
      const bool outs = kNS == 1 ? out : __shfl_sync(kFull, (int)out, base) != 0;
      const int64_t ks = kNS == 1 ? k : __shfl_sync(kFull, (long long)k, base);
      Real acc[kTR][kTC];
#pragma unroll
      for (int a = 0; a < kTR; ++a)
#pragma unroll
        for (int b = 0; b < kTC; ++b) acc[a][b] = Real(0);
      for (int jj = 0; jj < ms; ++jj) {
        Real cr[kTR], bs[kTC];
#pragma unroll
        for (int a = 0; a < kTR; ++a) cr[a] = B1[(base + jj) * ld + tr * kTR + a];
#pragma unroll
        for (int b = 0; b < kTC; ++b) bs[b] = B2[(base + jj) * ld + tc * kTC + b];
#pragma unroll
        for (int a = 0; a < kTR; ++a)
#pragma unroll
          for (int b = 0; b < kTC; ++b) acc[a][b] += cr[a] * bs[b];
      }
      Real* Tk = T + ks * R * R;
      if constexpr (kNS == 1) {
        __syncwarp();   // every lane is done reading B2
#pragma unroll
        for (int a = 0; a < kTR; ++a) {
          const int r = tr * kTR + a;
          if (r < R) {
#pragma unroll
            for (int b = 0; b < kTC; ++b) {
              const int s = tc * kTC + b;
              if (s < R) St[r * R + s] = acc[a][b];
            }
          }
        }
        __syncwarp();
        if (outs)
          for (int e = lane; e < R * R; e += 32) Tk[e] = St[e];
        __syncwarp();
      } else if (outs) {
#pragma unroll
        for (int a = 0; a < kTR; ++a) {
          const int r = tr * kTR + a;
          if (r < R) {
#pragma unroll
            for (int b = 0; b < kTC; ++b) {
              const int s = tc * kTC + b;
              if (s < R) Tk[r * R + s] = acc[a][b];
            }
          }
        }
      }
      if (Pi) {
#pragma unroll
        for (int a = 0; a < kTR; ++a)
#pragma unroll
          for (int b = 0; b < kTC; ++b) acc[a][b] = Real(0);
        for (int jj = 0; jj < ms; ++jj) {
          Real cr[kTR], cs[kTC];
#pragma unroll
          for (int a = 0; a < kTR; ++a) cr[a] = B1[(base + jj) * ld + tr * kTR + a];
#pragma unroll
          for (int b = 0; b < kTC; ++b) cs[b] = B1[(base + jj) * ld + tc * kTC + b];
#pragma unroll
          for (int a = 0; a < kTR; ++a)
#pragma unroll
            for (int b = 0; b < kTC; ++b) acc[a][b] += cr[a] * cs[b];
        }
        if (outs) {
          Real* Pk = Pi + ks * R * R;
#pragma unroll
          for (int a = 0; a < kTR; ++a) {
            const int r = tr * kTR + a;
            if (r < R) {
#pragma unroll
              for (int b = 0; b < kTC; ++b) {
                const int s = tc * kTC + b;
                if (s < R) Pk[r * R + s] = acc[a][b];
              }
            }
          }
        }
      }
    }
    // the q rows, contiguous in Q, through St
    __syncwarp();   // every lane is done reading B2
    if (sl < m) {
#pragma unroll
      for (int t = 0; t < kR; ++t)
        if (t < R) St[lane * R + t] = z[t];
    }
    __syncwarp();
#pragma unroll 1
    for (int s2 = 0; s2 < kNS; ++s2) {
      const int base = s2 * kSeg;
      const int ms = kNS == 1 ? m : __shfl_sync(kFull, m, base);
      const int64_t r0s = kNS == 1 ? r0 : __shfl_sync(kFull, (long long)r0, base);
      Real* Qk = Q + r0s * R;
      for (int e = lane; e < ms * R; e += 32) Qk[e] = St[base * R + e];
    }
    __syncwarp();
    if (fma_count) {
      int nz = nnz_row;
#pragma unroll
      for (int o = kSeg / 2; o > 0; o >>= 1) nz += __shfl_xor_sync(kFull, nz, o);
      if (sl == 0 && out) {
        const unsigned long long mm = (unsigned long long)m, RR = (unsigned long long)R * R;
        fma += (unsigned long long)nz * R + mm * RR + 2ull * mm * R + 2ull * mm * mm * R + 2ull * RR * mm;
        if (warm) fma += mm * mm * R;
        fma += (unsigned long long)sweeps * (mm * (mm > 0 ? mm - 1 : 0) / 2) * 3 * R + nrot / kNS * 4 * (R + mm);
      }
    }
  }
  if (fma_count && sl == 0) atomicAdd(fma_count, fma);
}

// ---- tall form (I_k > min(R, 32)), in three warp-per-subject launches ----
// k_tall_qr: the rows of A_k = X_k V S_k H^T are formed 32 at a time (lane = row) and
// folded into R_A by Householder reflections on the stacked [R_A; block] (lane = column,
// the block's columns in registers, each reflector broadcast by shuffles); R_A goes to
// T_k. k_tall_jacobi runs the one-sided Jacobi on the rows of R_A and leaves
// Omega = C_K Sigma_K^{-1} C_K^T in T_k. k_tall_pass2 (lane = row) recomputes the rows,
// writes q_i = a_i Omega and accumulates T_k = sum_i q_i^T p_i and the F_H partial sums.
// Same arithmetic as the block kernel's tall branch.
template <typename Real, int kR>
struct TallLay {
  static constexpr int VN = Vec16<Real>::n;
  static constexpr int ldb = kR + 1;    // row blocks: odd, so lane-per-row accesses are conflict-free
  static constexpr int ldr = kR + 1;    // R_A (read by columns)
  static constexpr int pad = (2 * 32 * ldb + VN - 1) / VN * VN;   // keeps Omega 16-byte aligned
  static constexpr int per_warp = pad + kR * kR + kR;             // pass 2: p and a/q blocks, Omega, W row
  static constexpr int per_warp_qr = (32 * ldb + kR * ldr + kR + VN - 1) / VN * VN;   // QR: row block, R_A, W row
  static constexpr size_t bytes = sizeof(Real) * ((size_t)kR * kR + (kWNT / 32) * (size_t)per_warp) + 16;
  static constexpr size_t qr_bytes = sizeof(Real) * ((size_t)kR * kR + (kWNT / 32) * (size_t)per_warp_qr) + 16;
  static_assert(2 * 32 * ldb >= kR * kR, "the two row blocks stage T_k");
};

// p_i = x_i V into the registers of the lane owning row i (rows past the block: 0), then
// a_i = (p_i * w) H^T from the p row kept in shared memory. Returns the row's nonzeros.
template <typename Real, int kR>
__device__ __forceinline__ int tall_row(const TensorView& X, int R, const Real* __restrict__ V, const Real* Hs,
                                        const Real* wk, int64_t i, bool valid, Real* prow, Real* z) {
  using Vc = Vec16<Real>;
  constexpr int VN = Vc::n;
  Real p[kR];
  const int nnz = row_p<Real, kR>(X, R, V, i, valid, p);
#pragma unroll
  for (int t = 0; t < kR; ++t) prow[t] = p[t];
#pragma unroll
  for (int t = 0; t < kR; ++t) z[t] = Real(0);
  if (valid) {
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      const Real pw = prow[r] * wk[r];
#pragma unroll
      for (int t = 0; t < kR; t += VN) {
        Real hv[VN];
        Vc::ld(Hs + r * kR + t, hv);
#pragma unroll
        for (int q = 0; q < VN; ++q) z[t + q] += pw * hv[q];
      }
    }
  }
  return nnz;
}

template <typename Real, int kR>
__device__ __forceinline__ void load_hs(const Real* __restrict__ H, int R, Real* Hs) {
  for (int e = threadIdx.x; e < kR * kR; e += kWNT) {
    const int r = e / kR, t = e - r * kR;
    Hs[e] = (t < R && r < R) ? H[t * R + r] : Real(0);   // Hs[r * kR + t] = H(t, r)
  }
}

// Four blocks per SM in FP32: the register cap of 128 costs no spills there (R = 40:
// 136 -> 128), its shared memory (4 x 54 KB) fits, and the extra resident warps hide more
// of the reflector chain's latency (measured: Procrustes step 70.2 -> 69.2 ms at
// K = 500k). The FP64 instantiations would spill at 128 and keep three.
template <typename Real, int kR>
__global__ void __launch_bounds__(kWNT, sizeof(Real) == 4 ? 4 : 3) k_tall_qr(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V, const Real* __restrict__ W,
    const int64_t* __restrict__ order, const int* __restrict__ count, int* __restrict__ counter,
    Real* __restrict__ T, unsigned long long* __restrict__ fma_count) {
  using Lt = TallLay<Real, kR>;
  constexpr int ldb = Lt::ldb, ldr = Lt::ldr;
  constexpr int kC2 = kR > 32 ? kR - 32 : 1;   // second columns (lanes 0 .. kR-33)
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Hs = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* Bs = Hs + kR * kR + (size_t)warp * Lt::per_warp_qr;   // 32 rows of A_k
  Real* Rs = Bs + 32 * ldb;                                     // R_A
  Real* Wb = Rs + kR * ldr;                                     // this subject's row of W
  load_hs<Real, kR>(H, R, Hs);
  __syncthreads();
  const int64_t nt = min((int64_t)max(*count, 0), X.K);
  unsigned long long fma = 0;

  while (true) {
    int claim = 0;
    if (lane == 0) claim = atomicAdd(counter, 1);
    const int64_t idx = __shfl_sync(kFull, claim, 0);
    if (idx >= nt) break;
    const int64_t k = order[idx];
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    const Real* wk = W + k * R;
    for (int r = lane; r < kR; r += 32) Wb[r] = r < R ? wk[r] : Real(0);
    for (int e = lane; e < kR * ldr; e += 32) Rs[e] = Real(0);
    __syncwarp();
    int nnzk = 0;
    for (int64_t g = r0; g < r1; g += 32) {
      const int nb = (int)min((int64_t)32, r1 - g);
      Real z[kR];
      nnzk += tall_row<Real, kR>(X, R, V, Hs, Wb, g + lane, lane < nb, Bs + lane * ldb, z);
#pragma unroll
      for (int t = 0; t < kR; ++t) Bs[lane * ldb + t] = z[t];
      __syncwarp();
      // block columns: c1 = lane, c2 = 32 + lane
      Real bc[32], bc2[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        bc[i] = lane < kR ? Bs[i * ldb + lane] : Real(0);
        bc2[i] = (kR > 32 && lane < kC2) ? Bs[i * ldb + 32 + lane] : Real(0);
      }
      __syncwarp();
      for (int j = 0; j < R; ++j) {
        const int jl = j & 31;
        const bool second = j >= 32;
        Real s4[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const Real v = second ? bc2[i] : bc[i];
          s4[i & 3] += v * v;
        }
        const Real ss = __shfl_sync(kFull, (s4[0] + s4[1]) + (s4[2] + s4[3]), jl);
        const Real x0 = Rs[j * ldr + j];
        Real tau = Real(0), scale = Real(0), beta = x0;
        if (ss > Real(0)) {
          // (FP32: x rsqrt(x) and approximate reciprocals, as in the rotation set-up; the
          // reflector is formed from them consistently, v = x / (x0 - beta) with tau from
          // the same beta)
          const Real nrm = sqrt_r(x0 * x0 + ss);
          beta = x0 >= Real(0) ? -nrm : nrm;
          tau = fdiv_(beta - x0, beta);
          scale = fdiv_(Real(1), x0 - beta);
        }
        if (tau != Real(0)) {
          Real v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = __shfl_sync(kFull, second ? bc2[i] : bc[i], jl) * scale;
          if (lane > j && lane < R) {
            Real d4[4] = {Rs[j * ldr + lane], Real(0), Real(0), Real(0)};
#pragma unroll
            for (int i = 0; i < 32; ++i) d4[i & 3] += v[i] * bc[i];
            const Real w = ((d4[0] + d4[1]) + (d4[2] + d4[3])) * tau;
            Rs[j * ldr + lane] -= w;
#pragma unroll
            for (int i = 0; i < 32; ++i) bc[i] -= w * v[i];
          }
          if (kR > 32 && 32 + lane > j && 32 + lane < R) {
            Real d4[4] = {Rs[j * ldr + 32 + lane], Real(0), Real(0), Real(0)};
#pragma unroll
            for (int i = 0; i < 32; ++i) d4[i & 3] += v[i] * bc2[i];
            const Real w = ((d4[0] + d4[1]) + (d4[2] + d4[3])) * tau;
            Rs[j * ldr + 32 + lane] -= w;
#pragma unroll
            for (int i = 0; i < 32; ++i) bc2[i] -= w * v[i];
          }
          if (lane == jl) {   // the block's column j is annihilated
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              if (second) bc2[i] = Real(0);
              else bc[i] = Real(0);
            }
          }
        }
        __syncwarp();
        if (lane == 0) Rs[j * ldr + j] = beta;
        __syncwarp();
      }
    }
    __syncwarp();
    Real* Tk = T + k * R * R;
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, t = e - r * R;
      Tk[e] = Rs[r * ldr + t];
    }
    __syncwarp();
    if (fma_count) {
      const int nz = __reduce_add_sync(kFull, nnzk);
      if (lane == 0) {
        const unsigned long long ik = (unsigned long long)(r1 - r0), RR = (unsigned long long)R * R;
        fma += (unsigned long long)nz * R + 2ull * ik * RR;
      }
    }
  }
  if (fma_count && lane == 0) atomicAdd(fma_count, fma);
}

template <typename Real, int kR>
__global__ void __launch_bounds__(kWNT, 3) k_tall_pass2(
    TensorView X, int R, const Real* __restrict__ H, const Real* __restrict__ V, const Real* __restrict__ W,
    const int64_t* __restrict__ order, const int* __restrict__ count, int* __restrict__ counter,
    Real* __restrict__ Q, Real* T, unsigned long long* __restrict__ fma_count) {
  using Lt = TallLay<Real, kR>;
  using Vc = Vec16<Real>;
  constexpr int ldb = Lt::ldb, VN = Lt::VN;
  constexpr int kTR = kR / 8, kTC = kR / 4;
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Hs = reinterpret_cast<Real*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* Bp = Hs + kR * kR + (size_t)warp * Lt::per_warp;   // p rows of a block
  Real* Ba = Bp + 32 * ldb;                                 // a rows, then q rows
  Real* Om = Bp + Lt::pad;                                  // Omega (kR x kR, zero-padded)
  Real* Wb = Om + kR * kR;                                  // this subject's row of W
  load_hs<Real, kR>(H, R, Hs);
  __syncthreads();
  const int64_t nt = min((int64_t)max(*count, 0), X.K);
  const int tr = lane >> 2, tc = lane & 3;
  unsigned long long fma = 0;

  while (true) {
    int claim = 0;
    if (lane == 0) claim = atomicAdd(counter, 1);
    const int64_t idx = __shfl_sync(kFull, claim, 0);
    if (idx >= nt) break;
    const int64_t k = order[idx];
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    const Real* wk = W + k * R;
    Real* Tk = T + k * R * R;
    // Omega was written by the previous launch: read it through L2
    for (int r = 0; r < kR; ++r)
      for (int t = lane; t < kR; t += 32) Om[r * kR + t] = (r < R && t < R) ? __ldcg(Tk + r * R + t) : Real(0);
    for (int r = lane; r < kR; r += 32) Wb[r] = r < R ? wk[r] : Real(0);
    __syncwarp();
    Real acc[kTR][kTC];
#pragma unroll
    for (int a = 0; a < kTR; ++a)
#pragma unroll
      for (int b = 0; b < kTC; ++b) acc[a][b] = Real(0);
    int nnzk = 0;
    for (int64_t g = r0; g < r1; g += 32) {
      const int nb = (int)min((int64_t)32, r1 - g);
      Real z[kR];
      nnzk += tall_row<Real, kR>(X, R, V, Hs, Wb, g + lane, lane < nb, Bp + lane * ldb, z);
#pragma unroll
      for (int t = 0; t < kR; ++t) Ba[lane * ldb + t] = z[t];
      // q_i = a_i Omega (own row of Ba, rows of Omega broadcast)
#pragma unroll
      for (int t = 0; t < kR; ++t) z[t] = Real(0);
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const Real ar = Ba[lane * ldb + r];
#pragma unroll
        for (int t = 0; t < kR; t += VN) {
          Real ov[VN];
          Vc::ld(Om + r * kR + t, ov);
#pragma unroll
          for (int q = 0; q < VN; ++q) z[t + q] += ar * ov[q];
        }
      }
#pragma unroll
      for (int t = 0; t < kR; ++t) Ba[lane * ldb + t] = z[t];
      __syncwarp();
      // the block's q rows are contiguous in Q: written row by row from shared memory
      for (int i = 0; i < nb; ++i)
        for (int t = lane; t < R; t += 32) Q[(g + i) * R + t] = Ba[i * ldb + t];
      // T_k += sum_i q_i^T p_i over the block (rows past nb are zero)
      for (int i = 0; i < nb; ++i) {
        Real qr[kTR], ps[kTC];
#pragma unroll
        for (int a = 0; a < kTR; ++a) qr[a] = Ba[i * ldb + tr * kTR + a];
#pragma unroll
        for (int b = 0; b < kTC; ++b) ps[b] = Bp[i * ldb + tc * kTC + b];
#pragma unroll
        for (int a = 0; a < kTR; ++a)
#pragma unroll
          for (int b = 0; b < kTC; ++b) acc[a][b] += qr[a] * ps[b];
      }
      __syncwarp();
    }
    // T_k through shared memory (the row blocks, free now), then contiguous stores
    Real* St = Bp;
#pragma unroll
    for (int a = 0; a < kTR; ++a) {
      const int r = tr * kTR + a;
      if (r < R) {
#pragma unroll
        for (int b = 0; b < kTC; ++b) {
          const int s = tc * kTC + b;
          if (s < R) St[r * R + s] = acc[a][b];
        }
      }
    }
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) Tk[e] = St[e];
    __syncwarp();
    if (fma_count) {
      const int nz = __reduce_add_sync(kFull, nnzk);
      if (lane == 0) {
        const unsigned long long ik = (unsigned long long)(r1 - r0), RR = (unsigned long long)R * R;
        fma += (unsigned long long)nz * R + 3ull * ik * RR;
      }
    }
  }
  if (fma_count && lane == 0) atomicAdd(fma_count, fma);
}

// k_tall_jacobi: warp per subject, the one-sided Jacobi on the rows of R_A (left in
// T_k by k_tall_qr) without block barriers. The n2 = R + (R & 1) rows sit two per lane
// (a "top" and a "bottom" row) in lanes 0 .. L - 1, L = n2 / 2. A sweep meets every pair
// once in two phases: (1) L rounds of top against bottom in the same lane, the bottoms
// moving one lane down the ring after each round (one shuffle per component, the same
// source rule in every lane); (2) the top-top and bottom-bottom pairs across lanes, the
// lanes paired by the circle method, each lane updating its own rows (pair_rotate).
// Rows are held scaled (row = f * x), so that a rotation costs one multiply-add per
// component and row; the scales are folded back at the start of every sweep.
// Omega_k = C_K Sigma_K^{-1} C_K^T goes back to T_k, with rank_k and, on request,
// Pi_k = C_K C_K^T.
template <typename Real, int kR>
struct TallJLay {
  static constexpr int ld = kR + 1;
  static constexpr int per_warp = (kR + 2) * ld + kR;   // c_j rows, 1/sigma_j
  static constexpr size_t bytes = sizeof(Real) * (kWNT / 32) * (size_t)per_warp + 16;
};

template <typename Real, int kR>
__global__ void __launch_bounds__(kWNT, 3) k_tall_jacobi(
    int64_t K, int R, double tau_rank, const int64_t* __restrict__ order, const int* __restrict__ count,
    int* __restrict__ counter, Real* T, Real* __restrict__ Pi, int32_t* __restrict__ rank,
    unsigned long long* __restrict__ fma_count) {
  using Lj = TallJLay<Real, kR>;
  constexpr int ld = Lj::ld;
  constexpr int kTR = kR / 8, kTC = kR / 4;
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* Cs = reinterpret_cast<Real*>(smem_raw) + (size_t)warp * Lj::per_warp;   // c_j rows
  Real* Is = Cs + (kR + 2) * ld;                                               // 1/sigma_j
  const Real tol = TolTall<Real>::v();
  const int n2 = R + (R & 1), L = n2 / 2;
  const bool own = lane < L;
  const int Le = L + (L & 1);   // circle-method positions of phase 2 (lane L is idle when L is odd)
  const int64_t nt = min((int64_t)max(*count, 0), K);
  const int tr = lane >> 2, tc = lane & 3;
  const int down = own ? (lane + 1 == L ? 0 : lane + 1) : lane;   // phase-1 bottom source
  unsigned long long fma = 0;

  while (true) {
    int claim = 0;
    if (lane == 0) claim = atomicAdd(counter, 1);
    const int64_t idx = __shfl_sync(kFull, claim, 0);
    if (idx >= nt) break;
    const int64_t k = order[idx];
    Real* Tk = T + k * R * R;
    Real top[kR], bot[kR];
    const int ra = lane, rb = L + lane;   // rows held at the start
#pragma unroll
    for (int t = 0; t < kR; ++t) {   // R_A was written by the previous launch: read it through L2
      top[t] = (own && ra < R && t < R) ? __ldcg(Tk + ra * R + t) : Real(0);
      bot[t] = (own && rb < R && t < R) ? __ldcg(Tk + rb * R + t) : Real(0);
    }
    Real na = Real(0), nb = Real(0), fa = Real(1), fb = Real(1);
    int sweeps = 0;
    unsigned long long nrot = 0;
    for (int sweep = 0; sweep < kMaxSweeps && n2 > 1; ++sweep) {
      ++sweeps;
      bool any = false;
      Real tmx = Real(0);   // largest |tan| of this lane's rotations in the sweep
      // fold the scales back; exact squared norms at the start of every sweep
#pragma unroll
      for (int t = 0; t < kR; ++t) {
        top[t] *= fa;
        bot[t] *= fb;
      }
      fa = fb = Real(1);
      na = sq_sum<Real, kR>(top);
      nb = sq_sum<Real, kR>(bot);
      // phase 1: top against bottom in each lane; the bottoms then move one lane down
      for (int rd = 0; rd < L; ++rd) {
        Real g4[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int t = 0; t < kR; ++t) g4[t & 3] += top[t] * bot[t];
        const Real gg = (fa * fb) * ((g4[0] + g4[1]) + (g4[2] + g4[3]));
        const bool rot = own && gg != Real(0) && fabs(gg) > tol * sqrt_r(na * nb);
        if (rot) {
          Real c, s, tt;
          rotation_of(na, nb, gg, &c, &s, &tt);
          // top' = c top - s bot, bot' = s top + c bot, in the scaled form
          const Real ma = tt * fdiv_(fb, fa), mb = tt * fdiv_(fa, fb);
          tmx = fmax(tmx, fabs(tt));
#pragma unroll
          for (int t = 0; t < kR; ++t) {
            const Real x = top[t], y = bot[t];
            top[t] = x - ma * y;
            bot[t] = y + mb * x;
          }
          fa *= c;
          fb *= c;
          // updated norms; recomputed where one of them drops by half or more, so that
          // rounding in the update stays small relative to the new norm
          const Real na1 = na - tt * gg, nb1 = nb + tt * gg;
          na = na1 < Real(0.5) * na ? fa * fa * sq_sum<Real, kR>(top) : na1;
          nb = nb1 < Real(0.5) * nb ? fb * fb * sq_sum<Real, kR>(bot) : nb1;
        }
        const unsigned rmask = __ballot_sync(kFull, rot);
        any |= rmask != 0u;
        if (lane == 0) nrot += __popc(rmask);
        if (rd + 1 < L) {
#pragma unroll
          for (int t = 0; t < kR; ++t) bot[t] = __shfl_sync(kFull, bot[t], down);
          fb = __shfl_sync(kFull, fb, down);
          nb = __shfl_sync(kFull, nb, down);
        }
      }
      // phase 2: tops against tops and bottoms against bottoms, lanes paired by the circle
      // method on Le positions (position Le - 1 meets r in round r, position i != r meets
      // (2r - i) mod (Le - 1))
      for (int rd = 0; rd < Le - 1; ++rd) {
        int j;
        if (lane >= Le) j = lane;
        else if (lane == Le - 1) j = rd;
        else if (lane == rd) j = Le - 1;
        else {
          j = 2 * rd - lane;
          if (j < 0) j += Le - 1;
          else if (j >= Le - 1) j -= Le - 1;
        }
        const bool pair = own && j < L && j != lane, lo = lane < j;
        const bool r1 = pair_rotate<Real, kR>(top, fa, na, j, lo, pair, tol, tmx);
        const bool r2 = pair_rotate<Real, kR>(bot, fb, nb, j, lo, pair, tol, tmx);
        const unsigned m1 = __ballot_sync(kFull, r1), m2 = __ballot_sync(kFull, r2);
        any |= (m1 | m2) != 0u;
        if (lane == 0) nrot += (__popc(m1) + __popc(m2)) / 2;
      }
      if (!any) break;
      if (warp_max(tmx) < Real(kTSmall) && sweep + 1 < kMaxSweeps) {
        // confirm convergence without a sweep: rows (scales folded) and squared norms to
        // shared memory (Cs and Is are free during the sweeps), every pair tested once
#pragma unroll
        for (int t = 0; t < kR; ++t) {
          top[t] *= fa;
          bot[t] *= fb;
        }
        fa = fb = Real(1);
        na = sq_sum<Real, kR>(top);
        nb = sq_sum<Real, kR>(bot);
        if (own) {
#pragma unroll
          for (int t = 0; t < kR; ++t) {
            Cs[lane * ld + t] = top[t];
            Cs[(L + lane) * ld + t] = bot[t];
          }
          Is[lane] = na;
          Is[L + lane] = nb;
        }
        __syncwarp();
        bool bad = false;
        if (own) {
#pragma unroll 1
          for (int jj = 0; jj < n2; ++jj) {
            Real ga[4] = {Real(0), Real(0), Real(0), Real(0)}, gb[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
            for (int t = 0; t < kR; ++t) {
              const Real r = Cs[jj * ld + t];
              ga[t & 3] += top[t] * r;
              gb[t & 3] += bot[t] * r;
            }
            const Real g1 = (ga[0] + ga[1]) + (ga[2] + ga[3]), g2 = (gb[0] + gb[1]) + (gb[2] + gb[3]);
            const Real nj = Is[jj];
            bad |= jj != lane && g1 != Real(0) && fabs(g1) > tol * sqrt(na * nj);
            bad |= jj != L + lane && g2 != Real(0) && fabs(g2) > tol * sqrt(nb * nj);
          }
        }
        __syncwarp();
        if (!__any_sync(kFull, bad)) {
          ++sweeps;   // the test stood in for the confirming sweep
          break;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kR; ++t) {   // exact squared norms for the rank cut
      top[t] *= fa;
      bot[t] *= fb;
    }
    na = sq_sum<Real, kR>(top);
    nb = sq_sum<Real, kR>(bot);

    // ---- rank cut; c_j = z_j / sigma_j, Omega = sum_j c_j c_j^T / sigma_j ----
    const Real amax = warp_max(own ? (na > nb ? na : nb) : Real(0));
    const bool ka = own && amax > Real(0) && (double)na > tau_rank * (double)amax;
    const bool kb = own && amax > Real(0) && (double)nb > tau_rank * (double)amax;
    const int kept = __popc(__ballot_sync(kFull, ka)) + __popc(__ballot_sync(kFull, kb));
    if (rank && lane == 0) rank[k] = kept;
    const Real sa = ka ? rsqrt_(na) : Real(0), sb = kb ? rsqrt_(nb) : Real(0);
    if (own) {
#pragma unroll
      for (int t = 0; t < kR; ++t) {
        Cs[lane * ld + t] = top[t] * sa;
        Cs[(L + lane) * ld + t] = bot[t] * sb;
      }
      Is[lane] = sa;
      Is[L + lane] = sb;
    }
    __syncwarp();
#pragma unroll 1
    for (int pass = 0; pass < (Pi ? 2 : 1); ++pass) {
      Real acc[kTR][kTC];
#pragma unroll
      for (int a = 0; a < kTR; ++a)
#pragma unroll
        for (int b = 0; b < kTC; ++b) acc[a][b] = Real(0);
      for (int j = 0; j < n2; ++j) {
        const Real w = pass == 0 ? Is[j] : Real(1);
        Real cr[kTR], cs[kTC];
#pragma unroll
        for (int a = 0; a < kTR; ++a) cr[a] = Cs[j * ld + tr * kTR + a] * w;
#pragma unroll
        for (int b = 0; b < kTC; ++b) cs[b] = Cs[j * ld + tc * kTC + b];
#pragma unroll
        for (int a = 0; a < kTR; ++a)
#pragma unroll
          for (int b = 0; b < kTC; ++b) acc[a][b] += cr[a] * cs[b];
      }
      Real* out = pass == 0 ? Tk : Pi + k * R * R;
#pragma unroll
      for (int a = 0; a < kTR; ++a) {
        const int r = tr * kTR + a;
        if (r < R) {
#pragma unroll
          for (int b = 0; b < kTC; ++b) {
            const int s = tc * kTC + b;
            if (s < R) out[r * R + s] = acc[a][b];
          }
        }
      }
    }
    __syncwarp();
    if (fma_count && lane == 0) {
      const unsigned long long RR = (unsigned long long)R * R, mm = (unsigned long long)R;
      fma += (unsigned long long)sweeps * (mm * (mm - 1) / 2) * 3 * R + nrot * 4ull * R + 2 * RR * R + 2 * mm * R;
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

// F_H = sum_k Y_k V S_k = sum_k T_k S_k (the MTTKRP of the H update, Sec. 3.1) from the stored
// T_k, for the lane-per-row path: block b takes a contiguous range of subjects, thread e
// the entries e, e + 512, ... of the R x R matrix (coalesced reads of T). In float every
// product is split exactly (p + e = T_k(r,s) w_k(s), by a fused multiply-add) and summed
// in a compensated pair; in double it is a plain sum. The per-block sums go to FP64
// partials, which k_reduce_partials adds in a fixed order.
constexpr int kFhThreads = 512, kFhE = 5;   // entries per thread: R*R <= 5 * 512 (R <= 48)
constexpr int kFhU = 8;                      // subjects whose T_k entries are loaded ahead

// (the _rn intrinsics keep the compiler from fusing the product into the sum)
__device__ __forceinline__ void fh_add(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b), pe = fmaf(a, b, -p);
  const float t = __fadd_rn(s, p), bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c += e + pe;
}
__device__ __forceinline__ void fh_add(double& s, double&, double a, double b) { s = fma(a, b, s); }

template <typename Real>
__global__ void __launch_bounds__(kFhThreads) k_fh_stream(int64_t K, int R, const Real* __restrict__ T,
                                                          const Real* __restrict__ W, double* __restrict__ part) {
  const int n = R * R;
  const int64_t per = (K + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = min(K, (int64_t)blockIdx.x * per), k1 = min(K, k0 + per);
  Real s[kFhE], c[kFhE];
  int col[kFhE];
#pragma unroll
  for (int j = 0; j < kFhE; ++j) {
    const int e = threadIdx.x + j * kFhThreads;
    col[j] = e < n ? e % R : 0;
    s[j] = c[j] = Real(0);
  }
  // kFhU subjects' loads are issued before their sums, so that enough reads are in flight
  int64_t k = k0;
  for (; k + kFhU <= k1; k += kFhU) {
    Real tv[kFhU][kFhE];
#pragma unroll
    for (int u = 0; u < kFhU; ++u)
#pragma unroll
      for (int j = 0; j < kFhE; ++j) {
        const int e = threadIdx.x + j * kFhThreads;
        tv[u][j] = e < n ? __ldcs(T + (k + u) * n + e) : Real(0);
      }
#pragma unroll
    for (int u = 0; u < kFhU; ++u)   // the W rows are shared by the block: L1 hits
#pragma unroll
      for (int j = 0; j < kFhE; ++j)
        if (threadIdx.x + j * kFhThreads < n) fh_add(s[j], c[j], tv[u][j], __ldg(W + (k + u) * R + col[j]));
  }
  for (; k < k1; ++k) {
#pragma unroll
    for (int j = 0; j < kFhE; ++j) {
      const int e = threadIdx.x + j * kFhThreads;
      if (e < n) fh_add(s[j], c[j], __ldcs(T + k * n + e), __ldg(W + k * R + col[j]));
    }
  }
#pragma unroll
  for (int j = 0; j < kFhE; ++j) {
    const int e = threadIdx.x + j * kFhThreads;
    if (e < n) part[(size_t)blockIdx.x * n + e] = (double)s[j] + (double)c[j];
  }
}

// The same sum in float4 units, for float with R % 4 == 0 and 16-byte aligned T and W: the
// four entries of a unit lie in one row of T_k, so they take one float4 of w_k as well.
// kFh4U subjects' units are loaded before their sums.
constexpr int kFh4Threads = 256, kFh4E = 3;   // units per thread: R*R/4 <= 3 * 256 (R <= 48)
constexpr int kFh4U = 4;

__global__ void __launch_bounds__(kFh4Threads) k_fh_stream4(int64_t K, int R, const float* __restrict__ T,
                                                            const float* __restrict__ W, double* __restrict__ part) {
  const int n4 = R * R / 4;
  const int64_t per = (K + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = min(K, (int64_t)blockIdx.x * per), k1 = min(K, k0 + per);
  float s[kFh4E][4], c[kFh4E][4];
  int col4[kFh4E];
#pragma unroll
  for (int j = 0; j < kFh4E; ++j) {
    const int e4 = threadIdx.x + j * kFh4Threads;
    col4[j] = e4 < n4 ? (4 * e4) % R / 4 : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s[j][q] = c[j][q] = 0.f;
  }
  const float4* T4 = reinterpret_cast<const float4*>(T);
  const float4* W4 = reinterpret_cast<const float4*>(W);
  const int r4 = R / 4;
  auto add4 = [&](int j, float4 t, float4 w) {
    fh_add(s[j][0], c[j][0], t.x, w.x);
    fh_add(s[j][1], c[j][1], t.y, w.y);
    fh_add(s[j][2], c[j][2], t.z, w.z);
    fh_add(s[j][3], c[j][3], t.w, w.w);
  };
  int64_t k = k0;
  for (; k + kFh4U <= k1; k += kFh4U) {
    float4 tv[kFh4U][kFh4E];
#pragma unroll
    for (int u = 0; u < kFh4U; ++u)
#pragma unroll
      for (int j = 0; j < kFh4E; ++j) {
        const int e4 = threadIdx.x + j * kFh4Threads;
        tv[u][j] = e4 < n4 ? __ldcs(T4 + (k + u) * n4 + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
    for (int u = 0; u < kFh4U; ++u)
#pragma unroll
      for (int j = 0; j < kFh4E; ++j)
        if (threadIdx.x + j * kFh4Threads < n4) add4(j, tv[u][j], __ldg(W4 + (k + u) * r4 + col4[j]));
  }
  for (; k < k1; ++k) {
#pragma unroll
    for (int j = 0; j < kFh4E; ++j) {
      const int e4 = threadIdx.x + j * kFh4Threads;
      if (e4 < n4) add4(j, __ldcs(T4 + k * n4 + e4), __ldg(W4 + k * r4 + col4[j]));
    }
  }
#pragma unroll
  for (int j = 0; j < kFh4E; ++j) {
    const int e4 = threadIdx.x + j * kFh4Threads;
    if (e4 < n4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) part[(size_t)blockIdx.x * R * R + 4 * e4 + q] = (double)s[j][q] + (double)c[j][q];
    }
  }
}

template <typename Real>
using WarpKernel = void (*)(TensorView, int, const Real*, const Real*, const Real*, double, Real*, Real*, Real*,
                            int32_t*, const int64_t*, const int*, const int*, int*, unsigned long long*, Real*,
                            const int64_t*, int, const int*, int*);
template <typename Real>
using TallQrKernel = void (*)(TensorView, int, const Real*, const Real*, const Real*, const int64_t*, const int*, int*,
                              Real*, unsigned long long*);
template <typename Real>
using TallJacobiKernel = void (*)(int64_t, int, double, const int64_t*, const int*, int*, Real*, Real*, int32_t*,
                                  unsigned long long*);
template <typename Real>
using TallPass2Kernel = void (*)(TensorView, int, const Real*, const Real*, const Real*, const int64_t*, const int*,
                                 int*, Real*, Real*, unsigned long long*);

// The lane-per-row kernels for one padded width kR.
template <typename Real>
struct RowKernels {
  WarpKernel<Real> small = nullptr;
  WarpKernel<Real> pair = nullptr;   // two subjects of I_k <= 16 per warp (kR >= 32)
  TallQrKernel<Real> qr = nullptr;
  TallJacobiKernel<Real> jac = nullptr;
  TallPass2Kernel<Real> pass2 = nullptr;
  size_t small_smem = 0, qr_smem = 0, jac_smem = 0, tall_smem = 0;
};

template <typename Real, int KR>
RowKernels<Real> row_kernels_of() {
  RowKernels<Real> r;
  r.small = k_procrustes_warp<Real, KR, 32>;
  if constexpr (KR >= 32) r.pair = k_procrustes_warp<Real, KR, 16>;
  r.qr = k_tall_qr<Real, KR>;
  r.jac = k_tall_jacobi<Real, KR>;
  r.jac_smem = TallJLay<Real, KR>::bytes;
  r.pass2 = k_tall_pass2<Real, KR>;
  r.small_smem = WarpLay<Real, KR>::bytes;
  r.qr_smem = TallLay<Real, KR>::qr_bytes;
  r.tall_smem = TallLay<Real, KR>::bytes;
  return r;
}

// Kernels for R padded to kr components; empty where the registers of a lane cannot hold
// a row (float: R <= 48, double: R <= 16).
template <typename Real>
RowKernels<Real> row_kernels_for(int kr);
template <>
RowKernels<float> row_kernels_for<float>(int kr) {
  switch (kr) {
    case 8: return row_kernels_of<float, 8>();
    case 16: return row_kernels_of<float, 16>();
    case 24: return row_kernels_of<float, 24>();
    case 32: return row_kernels_of<float, 32>();
    case 40: return row_kernels_of<float, 40>();
    case 48: return row_kernels_of<float, 48>();
    default: return RowKernels<float>{};
  }
}
template <>
RowKernels<double> row_kernels_for<double>(int kr) {
  switch (kr) {
    case 8: return row_kernels_of<double, 8>();
    case 16: return row_kernels_of<double, 16>();
    default: return RowKernels<double>{};
  }
}

// grid of a lane-per-row kernel: SMs x resident blocks (at most bps if bps > 0), no more
// than the subjects need
template <typename Kern>
copa_status_t row_grid(copa_ctx* h, Kern kern, size_t smem, int64_t K, int64_t* blocks, int bps) {
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  int per_sm = 0;
  if ((st = cuda_check(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWNT, smem), "occupancy")) !=
      COPA_OK)
    return st;
  if (bps > 0 && per_sm > bps) per_sm = bps;
  *blocks = (int64_t)h->num_sms * std::max(per_sm, 1);
  const int64_t need = (K + kWNT / 32 - 1) / (kWNT / 32);
  if (*blocks > need) *blocks = std::max<int64_t>(need, 1);
  return COPA_OK;
}

}  // namespace

template <typename Real>
size_t procrustes_smem(int R) {
  return lay_of<Real>(R).total * sizeof(Real);
}

// Launch order where the lane-per-row kernels exist for this R and precision: the subjects
// with I_k > min(R, 32) go through k_tall_qr (R_A -> T_k), k_tall_jacobi (Omega -> T_k) and
// k_tall_pass2 (Q rows, T_k, F_H); the others through k_procrustes_warp. Otherwise the
// block kernel k_procrustes takes every subject.
template <typename Real>
copa_status_t launch_procrustes(copa_ctx* h, const TensorView& X, int R, const Real* H,
                                const Real* V, const Real* W, double tau, Real* Q, Real* T,
                                Real* Pi, int32_t* rank, Real* F_H, Real* Uw, const int64_t* woff,
                                bool warm_in, const int* epoch) {
  const size_t smem = procrustes_smem<Real>(R);
  if (R < 1 || R > 2 * kNT || smem > 227 * 1024)
    return fail(h, COPA_ERR_UNSUPPORTED, "Procrustes: R too large for shared memory at this precision");
  copa_status_t st;
  // block kernel: 256 threads above R = 64, where one CTA fills an SM's shared memory and
  // the Jacobi pairs of a round need more threads (measured at K = 100k: R = 80 500 -> 334 ms
  // per outer iteration; R = 56 and the FP64 handle are faster with 128)
  const int nt = R > 64 ? 2 * kNT : kNT;
  auto block_kern = nt == kNT ? k_procrustes<Real, kNT> : k_procrustes<Real, 2 * kNT>;
  if ((st = cuda_check(h, cudaFuncSetAttribute(block_kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  int per_sm = 0;
  if ((st = cuda_check(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_kern, nt, smem),
                       "occupancy")) != COPA_OK)
    return st;
  if (per_sm < 1) per_sm = 1;
  const RowKernels<Real> rk = row_kernels_for<Real>((R + 7) / 8 * 8);
  const bool rows = rk.small != nullptr;
  int64_t blocks = 0;   // block kernel grid (only without the lane-per-row kernels)
  if (!rows) {
    blocks = (int64_t)h->num_sms * per_sm;
    if (blocks > X.K) blocks = X.K > 0 ? X.K : 1;
  }
  const TuneChoice tc = active_tune(h, X, R);
  int64_t sblocks = 0, qblocks = 0, jblocks = 0, pblocks = 0;
  if (rows) {
    if ((st = row_grid(h, rk.small, rk.small_smem, X.K, &sblocks, tc.bps)) != COPA_OK) return st;
    if ((st = row_grid(h, rk.qr, rk.qr_smem, X.K, &qblocks, tc.bps)) != COPA_OK) return st;
    if ((st = row_grid(h, rk.jac, rk.jac_smem, X.K, &jblocks, tc.bps)) != COPA_OK) return st;
    if ((st = row_grid(h, rk.pass2, rk.tall_smem, X.K, &pblocks, tc.bps)) != COPA_OK) return st;
  }
  const int64_t* order = nullptr;
  if ((st = get_schedule(h, X, &order)) != COPA_OK) return st;
  // I_k > split (min(R, 32) unless tuned lower) take the tall-subject kernels
  const int split = std::max(1, std::min(tc.split, std::min(R, 32)));
  const int* n_big = rows ? schedule_count_above(h, split) : nullptr;
  // subjects with I_k <= 16 (and <= the split), two to a warp where the rows allow it
  const bool pair = rows && rk.pair != nullptr && tc.pair;
  const int* n_small = pair ? schedule_count_above(h, std::min(16, split)) : nullptr;
  int64_t pair_blocks = 0;
  if (pair && (st = row_grid(h, rk.pair, rk.small_smem, (X.K + 1) / 2, &pair_blocks, tc.bps)) != COPA_OK) return st;
  int* counter = nullptr;
  if ((st = ws_get(h, SLOT_COUNTER, 64, (void**)&counter)) != COPA_OK) return st;
  unsigned long long* fma_count = reinterpret_cast<unsigned long long*>(counter + 2);
  // F_H partials: one per block of the block kernel, or one per block of k_fh_stream
  int64_t fblocks = 0;
  bool fh4 = false;   // float4 form of the F_H stream
  if constexpr (std::is_same<Real, float>::value)
    fh4 = R % 4 == 0 && (reinterpret_cast<uintptr_t>(T) & 15u) == 0 && (reinterpret_cast<uintptr_t>(W) & 15u) == 0;
  if (rows) {   // one wave of the F_H stream
    int fh_per_sm = 0;
    if ((st = cuda_check(h, fh4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fh_per_sm, k_fh_stream4, kFh4Threads, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fh_per_sm, k_fh_stream<Real>,
                                                                                kFhThreads, 0),
                         "occupancy")) != COPA_OK)
      return st;
    fblocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)h->num_sms * std::max(fh_per_sm, 1), X.K));
  }
  const int64_t nparts = rows ? fblocks : blocks;
  double* part = nullptr;
  if (F_H) {
    if ((st = ws_get(h, SLOT_PARTIAL, (size_t)nparts * R * R * sizeof(double), (void**)&part)) != COPA_OK)
      return st;
  }
  // counter[0]: block kernel, [2..3]: work tally, [4]: small subjects, [5]: tall QR, [6]: tall pass 2,
  // [7]: tall Jacobi
  if ((st = cuda_check(h, cudaMemsetAsync(counter, 0, 64, h->stream), "memset")) != COPA_OK)
    return st;
  if (rows) {
    rk.qr<<<(unsigned)qblocks, kWNT, rk.qr_smem, h->stream>>>(X, R, H, V, W, order, n_big, counter + 5, T, fma_count);
    if ((st = cuda_check(h, cudaGetLastError(), "k_tall_qr launch")) != COPA_OK) return st;
    rk.jac<<<(unsigned)jblocks, kWNT, rk.jac_smem, h->stream>>>(X.K, R, tau, order, n_big, counter + 7, T, Pi, rank,
                                                                  fma_count);
    if ((st = cuda_check(h, cudaGetLastError(), "k_tall_jacobi launch")) != COPA_OK) return st;
    rk.pass2<<<(unsigned)pblocks, kWNT, rk.tall_smem, h->stream>>>(X, R, H, V, W, order, n_big, counter + 6, Q, T,
                                                                     fma_count);
    if ((st = cuda_check(h, cudaGetLastError(), "k_tall_pass2 launch")) != COPA_OK) return st;
    rk.small<<<(unsigned)sblocks, kWNT, rk.small_smem, h->stream>>>(
        X, R, H, V, W, tau, Q, T, Pi, rank, order, n_big, n_small, counter + 4, fma_count, Uw, woff,
        warm_in ? 1 : 0, epoch, h->d_status);
    if ((st = cuda_check(h, cudaGetLastError(), "k_procrustes_warp launch")) != COPA_OK) return st;
    if (pair) {
      rk.pair<<<(unsigned)pair_blocks, kWNT, rk.small_smem, h->stream>>>(
          X, R, H, V, W, tau, Q, T, Pi, rank, order, n_small, nullptr, counter + 8, fma_count, Uw, woff,
          warm_in ? 1 : 0, epoch, h->d_status);
      if ((st = cuda_check(h, cudaGetLastError(), "k_procrustes_warp (paired) launch")) != COPA_OK) return st;
    }
    if (F_H && X.K > 0) {
      if constexpr (std::is_same<Real, float>::value) {
        if (fh4) k_fh_stream4<<<(unsigned)fblocks, kFh4Threads, 0, h->stream>>>(X.K, R, T, W, part);
        else k_fh_stream<Real><<<(unsigned)fblocks, kFhThreads, 0, h->stream>>>(X.K, R, T, W, part);
      } else {
        k_fh_stream<Real><<<(unsigned)fblocks, kFhThreads, 0, h->stream>>>(X.K, R, T, W, part);
      }
      if ((st = cuda_check(h, cudaGetLastError(), "F_H stream launch")) != COPA_OK) return st;
    }
  } else {
    block_kern<<<(unsigned)blocks, nt, smem, h->stream>>>(X, R, H, V, W, tau, Q, T, Pi, rank, part, order, counter,
                                                         fma_count, Uw, woff, warm_in ? 1 : 0, epoch, nullptr, nullptr);
    if ((st = cuda_check(h, cudaGetLastError(), "k_procrustes launch")) != COPA_OK) return st;
  }
  if (F_H) {
    k_reduce_partials<Real><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, (int)nparts, R * R, F_H);
    if ((st = cuda_check(h, cudaGetLastError(), "k_reduce_partials launch")) != COPA_OK) return st;
  }
  return COPA_OK;
}

template size_t procrustes_smem<float>(int);
template size_t procrustes_smem<double>(int);
template copa_status_t launch_procrustes<float>(copa_ctx*, const TensorView&, int, const float*,
                                                const float*, const float*, double, float*,
                                                float*, float*, int32_t*, float*, float*,
                                                const int64_t*, bool, const int*);
template copa_status_t launch_procrustes<double>(copa_ctx*, const TensorView&, int, const double*,
                                                 const double*, const double*, double, double*,
                                                 double*, double*, int32_t*, double*, double*,
                                                 const int64_t*, bool, const int*);

}  // namespace copa
