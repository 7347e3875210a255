// The plain per-subject FP64 form of one outer iteration: the comparison form of the
// method as written, without this library's batching, fusion or precision choices. One
// block per subject forms A_k = X_k V S_k H^T in global memory, its Gram (A_k^T A_k, or the
// dual A_k A_k^T when I_k < R), the Gram's eigendecomposition by cyclic Jacobi, and the
// pseudo-polar factor Q_k = A_k C Lambda^{-1/2}_+ C^T (or C Lambda^{-1/2}_+ C^T A_k), keeping
// eigenvalues above tau times the largest (Eq. 5 and the truncated SVD of Algorithm 1);
// Y_k = Q_k^T X_k is then materialised over the distinct columns of X_k; the three MTTKRPs
// (Sec. 2) read Y; every ADMM inner iteration is its own launch; the host drives the
// iteration step by step (no graph) and reads the FIT after each one. Everything in FP64.
#include <vector>

#include "copa_internal.cuh"

namespace copa {
namespace {

constexpr int kPT = 128;          // threads per block
constexpr int kPMaxR = 64;        // shared memory holds three m x m FP64 matrices, m <= 64
constexpr int kPMaxJWords = 2048; // column bitmap: J <= 65536
constexpr int kPSweeps = 40;

// Distinct columns of every subject: count (pass 0) or write the sorted list and the
// nonzero -> (subject, column) position map (pass 1). One block per subject.
__global__ void __launch_bounds__(kPT) k_plain_cols(TensorView X, int pass, int64_t* __restrict__ ccount,
                                                   const int64_t* __restrict__ yoff, int32_t* __restrict__ ycol,
                                                   int64_t* __restrict__ nz2y) {
  __shared__ uint32_t bm[kPMaxJWords];
  __shared__ int pre[kPMaxJWords + 1];
  const int nw = (X.J + 31) / 32;
  for (int64_t k = blockIdx.x; k < X.K; k += gridDim.x) {
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    const int64_t t0 = X.row_ptr[r0], t1 = X.row_ptr[r1];
    for (int w = threadIdx.x; w < nw; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      const int c = X.col[t];
      atomicOr(bm + (c >> 5), 1u << (c & 31));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < nw; ++w) { pre[w] = acc; acc += __popc(bm[w]); }
      pre[nw] = acc;
    }
    __syncthreads();
    if (pass == 0) {
      if (threadIdx.x == 0) ccount[k] = pre[nw];
    } else {
      const int64_t base = yoff[k];
      for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t bits = bm[w];
        int pos = pre[w];
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          ycol[base + pos++] = w * 32 + b;
        }
      }
      for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int c = X.col[t];
        nz2y[t] = base + pre[c >> 5] + __popc(bm[c >> 5] & ((1u << (c & 31)) - 1u));
      }
    }
    __syncthreads();
  }
}

// exclusive scan of n values into out[0..n] (one block)
__global__ void k_plain_scan(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t per = (n + nt - 1) / nt;
  const int64_t a = tid * per, b = min(n, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += in[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int64_t acc = 0;
    for (int i = 0; i < nt; ++i) { const int64_t x = part[i]; part[i] = acc; acc += x; }
    out[n] = acc;
  }
  __syncthreads();
  s = part[tid];
  for (int64_t i = a; i < b; ++i) { out[i] = s; s += in[i]; }
}

// Round-robin pairing of n2 (even) indices: pair j of round rd.
__device__ inline void rr_pair(int rd, int j, int n2, int* p, int* q) {
  // positions 0 .. n2-1; position n2-1 fixed, the others rotate
  const int a = j == 0 ? n2 - 1 : (rd + j) % (n2 - 1);
  const int b = (rd + n2 - 1 - j) % (n2 - 1);
  *p = min(a, b);
  *q = max(a, b);
}

// Procrustes for one subject per block (FP64). A (S x R) and Q (S x R) are global scratch
// and output; Pw (S x R) is scratch for P_k S_k.
__global__ void __launch_bounds__(kPT) k_plain_procrustes(TensorView X, int R, const double* __restrict__ H,
                                                         const double* __restrict__ V, const double* __restrict__ W,
                                                         double tau, double* __restrict__ Pw, double* __restrict__ A,
                                                         double* __restrict__ Q, int* __restrict__ status) {
  extern __shared__ double sm[];
  const int L = R;                       // leading dimension (m <= R)
  double* G = sm;                        // m x m, becomes diag(Lambda)
  double* Z = G + L * L;                 // eigenvectors (columns)
  double* M = Z + L * L;                 // C Lambda^{-1/2}_+ C^T
  __shared__ double cs[kPMaxR / 2][2];
  __shared__ int pq[kPMaxR / 2][2];
  __shared__ int any_rot;
  const int tid = threadIdx.x;
  for (int64_t k = blockIdx.x; k < X.K; k += gridDim.x) {
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    const int Ik = (int)(r1 - r0);
    if (Ik == 0) continue;
    const double* wk = W + k * R;
    // P_k S_k, then A_k = P_k S_k H^T, both materialised
    for (int e = tid; e < Ik * R; e += blockDim.x) {
      const int i = e / R, r = e - i * R;
      double acc = 0.0;
      for (int64_t t = X.row_ptr[r0 + i]; t < X.row_ptr[r0 + i + 1]; ++t) acc += load_val(X, t) * V[(int64_t)X.col[t] * R + r];
      Pw[(r0 + i) * R + r] = acc * wk[r];
    }
    __syncthreads();
    for (int e = tid; e < Ik * R; e += blockDim.x) {
      const int i = e / R, s = e - i * R;
      double acc = 0.0;
      for (int r = 0; r < R; ++r) acc += Pw[(r0 + i) * R + r] * H[s * R + r];
      A[(r0 + i) * R + s] = acc;
    }
    __syncthreads();
    const bool dual = Ik < R;
    const int m = dual ? Ik : R;
    // Gram: A^T A (m = R) or A A^T (m = I_k)
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int p = e / m, q = e - p * m;
      double acc = 0.0;
      if (dual) {
        for (int s = 0; s < R; ++s) acc += A[(r0 + p) * R + s] * A[(r0 + q) * R + s];
      } else {
        for (int i = 0; i < Ik; ++i) acc += A[(r0 + i) * R + p] * A[(r0 + i) * R + q];
      }
      G[p * L + q] = acc;
      Z[p * L + q] = p == q ? 1.0 : 0.0;
    }
    __syncthreads();
    // cyclic Jacobi, round-robin order: m/2 disjoint rotations per round
    const int n2 = m + (m & 1);
    for (int sweep = 0; sweep < kPSweeps && m > 1; ++sweep) {
      if (tid == 0) any_rot = 0;
      __syncthreads();
      for (int rd = 0; rd < n2 - 1; ++rd) {
        for (int j = tid; j < n2 / 2; j += blockDim.x) {
          int p, q;
          rr_pair(rd, j, n2, &p, &q);
          double c = 1.0, s = 0.0;
          if (q < m) {
            const double apq = G[p * L + q], app = G[p * L + p], aqq = G[q * L + q];
            if (apq != 0.0 && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
              const double th = (aqq - app) / (2.0 * apq);
              const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
              c = 1.0 / sqrt(t * t + 1.0);
              s = t * c;
              any_rot = 1;
            }
          }
          pq[j][0] = p;
          pq[j][1] = q;
          cs[j][0] = c;
          cs[j][1] = s;
        }
        __syncthreads();
        // rows p, q of G
        for (int e = tid; e < (n2 / 2) * m; e += blockDim.x) {
          const int j = e / m, col = e - j * m;
          const int p = pq[j][0], q = pq[j][1];
          if (q >= m) continue;
          const double c = cs[j][0], s = cs[j][1];
          const double gp = G[p * L + col], gq = G[q * L + col];
          G[p * L + col] = c * gp - s * gq;
          G[q * L + col] = s * gp + c * gq;
        }
        __syncthreads();
        // columns p, q of G and of Z
        for (int e = tid; e < (n2 / 2) * m; e += blockDim.x) {
          const int j = e / m, row = e - j * m;
          const int p = pq[j][0], q = pq[j][1];
          if (q >= m) continue;
          const double c = cs[j][0], s = cs[j][1];
          const double gp = G[row * L + p], gq = G[row * L + q];
          G[row * L + p] = c * gp - s * gq;
          G[row * L + q] = s * gp + c * gq;
          const double zp = Z[row * L + p], zq = Z[row * L + q];
          Z[row * L + p] = c * zp - s * zq;
          Z[row * L + q] = s * zp + c * zq;
        }
        __syncthreads();
      }
      if (!any_rot) break;
      __syncthreads();
    }
    // M = sum over kept eigenpairs of z z^T / sqrt(lambda)
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, G[i * L + i]);
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int p = e / m, q = e - p * m;
      double acc = 0.0;
      for (int i = 0; i < m; ++i) {
        const double li = G[i * L + i];
        if (lmax > 0.0 && li > tau * lmax) acc += Z[p * L + i] * Z[q * L + i] / sqrt(li);
      }
      M[p * L + q] = acc;
    }
    __syncthreads();
    // Q_k = A_k M (m = R) or M A_k (m = I_k)
    for (int e = tid; e < Ik * R; e += blockDim.x) {
      const int i = e / R, s = e - i * R;
      double acc = 0.0;
      if (dual) {
        for (int j = 0; j < Ik; ++j) acc += M[i * L + j] * A[(r0 + j) * R + s];
      } else {
        for (int r = 0; r < R; ++r) acc += A[(r0 + i) * R + r] * M[r * L + s];
      }
      Q[(r0 + i) * R + s] = acc;
    }
    __syncthreads();
  }
  (void)status;
}

// Y_k = Q_k^T X_k over the distinct columns of X_k: Y[yoff[k] + pos] (an R-vector) for the
// subject's pos-th column. One block per subject.
__global__ void __launch_bounds__(kPT) k_plain_Y(TensorView X, int R, const double* __restrict__ Q,
                                                 const int64_t* __restrict__ yoff, const int64_t* __restrict__ nz2y,
                                                 double* __restrict__ Y) {
  for (int64_t k = blockIdx.x; k < X.K; k += gridDim.x) {
    const int64_t r0 = X.subj_ptr[k], r1 = X.subj_ptr[k + 1];
    for (int64_t e = yoff[k] * R + threadIdx.x; e < yoff[k + 1] * R; e += blockDim.x) Y[e] = 0.0;
    __syncthreads();
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t t0 = X.row_ptr[i], t1 = X.row_ptr[i + 1];
      for (int64_t e = threadIdx.x; e < (t1 - t0) * R; e += blockDim.x) {
        const int64_t t = t0 + e / R;
        const int r = (int)(e % R);
        atomicAdd(Y + nz2y[t] * R + r, load_val(X, t) * Q[i * R + r]);
      }
    }
    __syncthreads();
  }
}

// F_H = sum_k Y_k V S_k (persistent blocks, R x R block sums in shared memory)
__global__ void __launch_bounds__(kPT) k_plain_fh(int64_t K, int R, const double* __restrict__ Y,
                                                  const int64_t* __restrict__ yoff, const int32_t* __restrict__ ycol,
                                                  const double* __restrict__ V, const double* __restrict__ W,
                                                  double* __restrict__ FH) {
  __shared__ double acc[kPMaxR * kPMaxR];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();
  for (int64_t k = blockIdx.x; k < K; k += gridDim.x) {
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const int r = e / R, s = e - r * R;
      double a = 0.0;
      for (int64_t p = yoff[k]; p < yoff[k + 1]; ++p) a += Y[p * R + r] * V[(int64_t)ycol[p] * R + s];
      acc[e] += a * W[k * R + s];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) atomicAdd(FH + e, acc[e]);
}

// F_W(k, s) = sum_r H(r, s) (Y_k V)(r, s); one block per subject
__global__ void __launch_bounds__(kPT) k_plain_fw(int64_t K, int R, const double* __restrict__ Y,
                                                  const int64_t* __restrict__ yoff, const int32_t* __restrict__ ycol,
                                                  const double* __restrict__ H, const double* __restrict__ V,
                                                  double* __restrict__ FW) {
  for (int64_t k = blockIdx.x; k < K; k += gridDim.x) {
    for (int s = threadIdx.x; s < R; s += blockDim.x) {
      double a = 0.0;
      for (int64_t p = yoff[k]; p < yoff[k + 1]; ++p) {
        double yh = 0.0;
        for (int r = 0; r < R; ++r) yh += H[r * R + s] * Y[p * R + r];
        a += yh * V[(int64_t)ycol[p] * R + s];
      }
      FW[k * R + s] = a;
    }
  }
}

// F_V(j, :) += Y_k(:, j)^T H S_k for every (subject, column) pair (global FP64 atomics)
__global__ void __launch_bounds__(kPT) k_plain_fv(int64_t K, int R, const double* __restrict__ Y,
                                                  const int64_t* __restrict__ yoff, const int32_t* __restrict__ ycol,
                                                  const double* __restrict__ H, const double* __restrict__ W,
                                                  double* __restrict__ FV) {
  for (int64_t k = blockIdx.x; k < K; k += gridDim.x) {
    const int64_t np = yoff[k + 1] - yoff[k];
    for (int64_t e = threadIdx.x; e < np * R; e += blockDim.x) {
      const int64_t p = yoff[k] + e / R;
      const int s = (int)(e % R);
      double a = 0.0;
      for (int r = 0; r < R; ++r) a += Y[p * R + r] * H[r * R + s];
      atomicAdd(FV + (int64_t)ycol[p] * R + s, a * W[k * R + s]);
    }
  }
}

// U^T U = sum_k (Q_k H S_k)^T (Q_k H S_k) (persistent blocks, shared block sums)
__global__ void __launch_bounds__(kPT) k_plain_utu(TensorView X, int R, const double* __restrict__ Q,
                                                   const double* __restrict__ H, const double* __restrict__ W,
                                                   double* __restrict__ UtU) {
  __shared__ double acc[kPMaxR * kPMaxR];
  __shared__ double u[kPMaxR];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();
  for (int64_t k = blockIdx.x; k < X.K; k += gridDim.x) {
    for (int64_t i = X.subj_ptr[k]; i < X.subj_ptr[k + 1]; ++i) {
      for (int s = threadIdx.x; s < R; s += blockDim.x) {
        double a = 0.0;
        for (int r = 0; r < R; ++r) a += Q[i * R + r] * H[r * R + s];
        u[s] = a * W[k * R + s];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < R * R; e += blockDim.x) acc[e] += u[e / R] * u[e % R];
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) atomicAdd(UtU + e, acc[e]);
}

}  // namespace
}  // namespace copa

using namespace copa;

extern "C" copa_status_t copa_fit_plain(copa_handle_t h, const copa_tensor_t* Xc, const copa_options_t* o, void* Hv,
                                        void* Vv, void* Wv, void* DHv, void* DVv, void* DWv,
                                        double* fit_history_host) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t st;
  if ((st = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return st;
  if ((st = check_tensor_args(h, Xc)) != COPA_OK) return st;
  if (h->precision != COPA_PREC_FP64)
    return fail(h, COPA_ERR_UNSUPPORTED, "copa_fit_plain: the plain form is FP64 (create the handle with COPA_PREC_FP64)");
  if (!o || o->R < 1 || o->n_outer < 0 || o->n_inner < 0)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_plain: bad options");
  if (o->R > kPMaxR) return fail(h, COPA_ERR_UNSUPPORTED, "copa_fit_plain: R <= 64");
  if (Xc->J > 32 * kPMaxJWords) return fail(h, COPA_ERR_UNSUPPORTED, "copa_fit_plain: J <= 65536");
  if (!Hv || !Vv || !Wv || !DHv || !DVv || !DWv) return fail(h, COPA_ERR_INVALID_ARG, "copa_fit_plain: NULL factor");
  const TensorView X = view_of(Xc);
  const int R = o->R;
  double *H = (double*)Hv, *V = (double*)Vv, *W = (double*)Wv, *DH = (double*)DHv, *DV = (double*)DVv,
         *DW = (double*)DWv;
  // set-up: the distinct columns of every subject (the layout of the explicit Y)
  int64_t *ccount = nullptr, *yoff = nullptr, *nz2y = nullptr;
  int32_t* ycol = nullptr;
  char* p = nullptr;
  const size_t nsetup = sizeof(int64_t) * (2 * (size_t)X.K + 2) + sizeof(int64_t) * ((size_t)X.nnz + 1) +
                        sizeof(int32_t) * ((size_t)X.nnz + 1) + 256;
  if ((st = ws_get(h, SLOT_CSC, nsetup, (void**)&p)) != COPA_OK) return st;
  ccount = reinterpret_cast<int64_t*>(p);
  yoff = ccount + X.K + 1;
  nz2y = yoff + X.K + 1;
  ycol = reinterpret_cast<int32_t*>(nz2y + X.nnz + 1);
  h->csc_key = nullptr;   // this slot no longer holds the column-sorted copy
  const int pgrid = (int)std::max<int64_t>(1, std::min<int64_t>(X.K, (int64_t)h->num_sms * 16));
  if (X.K > 0) {
    k_plain_cols<<<pgrid, kPT, 0, h->stream>>>(X, 0, ccount, nullptr, nullptr, nullptr);
    k_plain_scan<<<1, 1024, 0, h->stream>>>(ccount, X.K, yoff);
    k_plain_cols<<<pgrid, kPT, 0, h->stream>>>(X, 1, nullptr, yoff, ycol, nz2y);
  }
  if ((st = cuda_check(h, cudaGetLastError(), "k_plain_cols")) != COPA_OK) return st;
  int64_t npairs = 0;
  if (X.K > 0 &&
      (st = cuda_check(h, cudaMemcpyAsync(&npairs, yoff + X.K, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream),
                       "D2H")) != COPA_OK)
    return st;
  if ((st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync")) != COPA_OK) return st;
  // per-iteration buffers
  double *Pw = nullptr, *A = nullptr, *Q = nullptr, *Y = nullptr, *small = nullptr;
  const size_t SR = sizeof(double) * ((size_t)std::max<int64_t>(X.S, 1) * R);
  if ((st = ws_get(h, SLOT_FIT_Q, SR, (void**)&Q)) != COPA_OK) return st;
  if ((st = ws_get(h, SLOT_FIT_T, 2 * SR, (void**)&A)) != COPA_OK) return st;
  Pw = A + (size_t)std::max<int64_t>(X.S, 1) * R;
  if ((st = ws_get(h, SLOT_UVEC, sizeof(double) * ((size_t)std::max<int64_t>(npairs, 1) * R), (void**)&Y)) != COPA_OK)
    return st;
  const size_t nsm = (size_t)R * R * 6 + (size_t)X.J * R + (size_t)R * (R + 1) + (size_t)X.K * R + 16;
  if ((st = ws_get(h, SLOT_FIT_SMALL, sizeof(double) * nsm, (void**)&small)) != COPA_OK) return st;
  double *FH = small, *gH = FH + R * R, *gV = gH + R * R, *gW = gV + R * R, *UtU = gW + R * R, *Ginv = UtU + R * R,
         *FV = Ginv + R * (R + 1), *FW = FV + (size_t)X.J * R, *scal = FW + (size_t)X.K * R;
  double* rho = scal;        // [0..2]
  double* xn2 = scal + 4;
  double* fitv = scal + 5;
  if ((st = launch_xnorm2(h, X, xn2)) != COPA_OK) return st;
  const size_t psmem = sizeof(double) * 3 * (size_t)R * R;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_plain_procrustes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)psmem), "attr")) != COPA_OK)
    return st;
  auto admm = [&](const double* F, const double* Ga, const double* Gb, double* Z, double* D, int64_t rows, int c,
                  double lam, double* rh) -> copa_status_t {
    copa_status_t s2;
    if ((s2 = launch_chol<double>(h, Ga, Gb, R, Ginv, rh)) != COPA_OK) return s2;
    for (int it = 0; it < o->n_inner; ++it)   // one launch per inner iteration
      if ((s2 = launch_admm_rows<double>(h, F, Ginv, rh, 1, c, lam, Z, D, rows, R)) != COPA_OK) return s2;
    return COPA_OK;
  };
  for (int outer = 0; outer < o->n_outer; ++outer) {
    if (X.K > 0) {
      k_plain_procrustes<<<pgrid, kPT, psmem, h->stream>>>(X, R, H, V, W, o->tau, Pw, A, Q, h->d_status);
      k_plain_Y<<<pgrid, kPT, 0, h->stream>>>(X, R, Q, yoff, nz2y, Y);
    }
    if ((st = cuda_check(h, cudaGetLastError(), "k_plain_procrustes")) != COPA_OK) return st;
    // H
    if ((st = cuda_check(h, cudaMemsetAsync(FH, 0, sizeof(double) * R * R, h->stream), "memset")) != COPA_OK) return st;
    if (X.K > 0) k_plain_fh<<<pgrid, kPT, 0, h->stream>>>(X.K, R, Y, yoff, ycol, V, W, FH);
    if ((st = launch_gram<double>(h, W, X.K, R, gW)) != COPA_OK) return st;
    if ((st = launch_gram<double>(h, V, X.J, R, gV)) != COPA_OK) return st;
    if ((st = admm(FH, gW, gV, H, DH, R, o->c_H, o->lam_H, rho + 0)) != COPA_OK) return st;
    // W
    if (X.K > 0) k_plain_fw<<<pgrid, kPT, 0, h->stream>>>(X.K, R, Y, yoff, ycol, H, V, FW);
    if ((st = launch_gram<double>(h, H, R, R, gH)) != COPA_OK) return st;
    if ((st = admm(FW, gH, gV, W, DW, X.K, o->c_W, o->lam_W, rho + 1)) != COPA_OK) return st;
    // V
    if ((st = cuda_check(h, cudaMemsetAsync(FV, 0, sizeof(double) * (size_t)X.J * R, h->stream), "memset")) != COPA_OK)
      return st;
    if (X.K > 0) k_plain_fv<<<pgrid, kPT, 0, h->stream>>>(X.K, R, Y, yoff, ycol, H, W, FV);
    if ((st = launch_gram<double>(h, W, X.K, R, gW)) != COPA_OK) return st;
    if ((st = admm(FV, gH, gW, V, DV, X.J, o->c_V, o->lam_V, rho + 2)) != COPA_OK) return st;
    // FIT of (Q_k, H, W, V)
    if ((st = cuda_check(h, cudaMemsetAsync(UtU, 0, sizeof(double) * R * R, h->stream), "memset")) != COPA_OK) return st;
    if (X.K > 0) k_plain_utu<<<pgrid, kPT, 0, h->stream>>>(X, R, Q, H, W, UtU);
    if ((st = launch_fit_value<double>(h, X.J, R, V, FV, UtU, xn2, o->x_norm2, fitv, gV)) != COPA_OK) return st;
    if ((st = cuda_check(h, cudaGetLastError(), "plain iteration")) != COPA_OK) return st;
    double f = 0.0;
    if ((st = cuda_check(h, cudaMemcpyAsync(&f, fitv, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "D2H")) !=
        COPA_OK)
      return st;
    if ((st = copa_sync(h)) != COPA_OK) return st;
    if (fit_history_host) fit_history_host[outer] = f;
  }
  h->warm_valid = false;
  return COPA_OK;
}
