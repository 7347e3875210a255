// Gradient of the reconstruction loss L = sum_k ||X_k - Q_k H S_k V^T||_F^2 (no 1/2)
// with Q_k fixed, from the model of Sec. 2 / Eq. 1. With
// R_k = X_k - Q_k H S_k V^T, Phi = V^T V, Pi_k = Q_k^T Q_k, T_k = Q_k^T X_k V:
//   dL/dH      = -2 sum_k Q_k^T R_k V S_k = -2 (F_H - sum_k Pi_k H S_k Phi S_k)
//   dL/dV      = -2 sum_k R_k^T Q_k H S_k = -2 (F_V - V U^T U)
//   dL/dW(k,r) = -2 [(H^T T_k)(r,r) - (H^T Pi_k H S_k Phi)(r,r)]
//   L          = ||X||^2 - 2 <V, F_V> + <Phi, U^T U>
// F_V and U^T U come from the V-mode MTTKRP (k_factor.cu); the per-subject part runs
// here, a warp per subject, reusing T_k and Pi_k of the Procrustes step.
#include "copa_internal.cuh"

namespace copa {

namespace {

template <typename Real>
__global__ void __launch_bounds__(128) k_grad_subject(int64_t K, int R, const Real* __restrict__ T,
                                                      const Real* __restrict__ Pi, const Real* __restrict__ H,
                                                      const Real* __restrict__ W, const double* __restrict__ Phi,
                                                      Real* __restrict__ gW, double* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int ld = R + 1;
  Real* Hs = reinterpret_cast<Real*>(smem_raw);   // R x R
  Real* Ps = Hs + R * R;                           // R x R (Phi)
  Real* Z = Ps + R * R + (size_t)warp * (2 * R * ld + R);   // Pi_k H
  Real* B = Z + R * ld;                                      // H^T Pi_k H
  Real* wv = B + R * ld;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) { Hs[e] = H[e]; Ps[e] = (Real)Phi[e]; }
  double* acc = part + (size_t)(blockIdx.x * nwarps + warp) * R * R;
  for (int e = lane; e < R * R; e += 32) acc[e] = 0.0;
  __syncthreads();
  const int64_t wid = blockIdx.x * (int64_t)nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
  for (int64_t k = wid; k < K; k += nw) {
    const Real* Tk = T + k * R * R;
    const Real* Pk = Pi + k * R * R;
    for (int s = lane; s < R; s += 32) wv[s] = W[k * R + s];
    for (int e = lane; e < R * R; e += 32) {
      const int t = e / R, s = e - t * R;
      Real a = Real(0);
      for (int u = 0; u < R; ++u) a += Pk[t * R + u] * Hs[u * R + s];
      Z[t * ld + s] = a;
    }
    __syncwarp();
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, s = e - r * R;
      Real a = Real(0);
      for (int t = 0; t < R; ++t) a += Hs[t * R + r] * Z[t * ld + s];
      B[r * ld + s] = a;
    }
    __syncwarp();
    for (int r = lane; r < R; r += 32) {
      Real ht = Real(0), hp = Real(0);
      for (int t = 0; t < R; ++t) ht += Hs[t * R + r] * Tk[t * R + r];
      for (int s = 0; s < R; ++s) hp += B[r * ld + s] * wv[s] * Ps[s * R + r];
      gW[k * R + r] = Real(-2) * (ht - hp);
    }
    // acc += T_k S_k - Pi_k H S_k Phi S_k
    for (int e = lane; e < R * R; e += 32) {
      const int t = e / R, u = e - t * R;
      Real a = Real(0);
      for (int s = 0; s < R; ++s) a += Z[t * ld + s] * wv[s] * Ps[s * R + u];
      acc[e] += (double)(Tk[e] * wv[u] - a * wv[u]);
    }
    __syncwarp();
  }
}

template <typename Real>
__global__ void k_grad_h(const double* __restrict__ part, int nparts, int R, Real* __restrict__ gH) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * R; e += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < nparts; ++q) a += part[(size_t)q * R * R + e];
    gH[e] = (Real)(-2.0 * a);
  }
}

template <typename Real>
__global__ void k_grad_v(int64_t J, int R, const Real* __restrict__ V, const Real* __restrict__ FV,
                         const double* __restrict__ UtU, Real* __restrict__ gV) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < J * R; e += gridDim.x * (int64_t)blockDim.x) {
    const int64_t j = e / R;
    const int s = (int)(e - j * R);
    double a = 0.0;
    for (int r = 0; r < R; ++r) a += (double)V[j * R + r] * UtU[r * R + s];
    gV[e] = (Real)(-2.0 * ((double)FV[e] - a));
  }
}

// L = ||X||^2 - 2 <V, F_V> + <Phi, U^T U>
template <typename Real>
__global__ void k_loss(int64_t J, int R, const Real* __restrict__ V, const Real* __restrict__ FV,
                       const double* __restrict__ UtU, const double* __restrict__ Phi,
                       const double* __restrict__ xn2, double* __restrict__ loss) {
  __shared__ double red[256];
  double a = 0.0;
  for (int64_t e = threadIdx.x; e < J * R; e += blockDim.x) a -= 2.0 * (double)V[e] * (double)FV[e];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) a += Phi[e] * UtU[e];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = *xn2 + red[0];
}

}  // namespace

template <typename Real>
copa_status_t launch_loss_grad(copa_ctx* h, const TensorView& X, int R, const Real* Q, const Real* T,
                               const Real* Pi, const Real* H, const Real* V, const Real* W, double* loss,
                               Real* gH, Real* gV, Real* gW) {
  copa_status_t st;
  // scratch: Phi, UtU, xn2 (FP64) and F_V (Real) in SLOT_MISC2 layout
  char* p = nullptr;
  const size_t need = sizeof(double) * (2 * (size_t)R * R + 4) + sizeof(Real) * (size_t)X.J * R + 1024;
  if ((st = ws_get(h, SLOT_SMOOTH, need, (void**)&p)) != COPA_OK) return st;
  double* Phi = reinterpret_cast<double*>(p);
  double* UtU = Phi + R * R;
  double* xn2 = UtU + R * R;
  Real* FV = reinterpret_cast<Real*>(xn2 + 4);
  if ((st = launch_gram<Real>(h, V, X.J, R, Phi)) != COPA_OK) return st;
  if ((st = launch_mttkrp_v<Real>(h, X, R, Q, H, W, FV, UtU)) != COPA_OK) return st;
  if ((st = launch_xnorm2(h, X, xn2)) != COPA_OK) return st;
  const int warps = 4;
  const size_t smem = sizeof(Real) * (2 * (size_t)R * R + (size_t)warps * (2 * R * (R + 1) + R));
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_grad_subject<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "attr")) != COPA_OK)
    return st;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((X.K + warps - 1) / warps, (int64_t)h->num_sms * 4));
  double* part = nullptr;
  if ((st = ws_get(h, SLOT_PARTIAL, sizeof(double) * (size_t)blocks * warps * R * R, (void**)&part)) != COPA_OK)
    return st;
  k_grad_subject<Real><<<blocks, 32 * warps, smem, h->stream>>>(X.K, R, T, Pi, H, W, Phi, gW, part);
  k_grad_h<Real><<<(R * R + 255) / 256, 256, 0, h->stream>>>(part, blocks * warps, R, gH);
  const int vb = (int)std::max<int64_t>(1, std::min<int64_t>((X.J * R + 255) / 256, 1024));
  k_grad_v<Real><<<vb, 256, 0, h->stream>>>(X.J, R, V, FV, UtU, gV);
  k_loss<Real><<<1, 256, 0, h->stream>>>(X.J, R, V, FV, UtU, Phi, xn2, loss);
  return cuda_check(h, cudaGetLastError(), "loss/grad kernels");
}

template copa_status_t launch_loss_grad<float>(copa_ctx*, const TensorView&, int, const float*, const float*,
                                               const float*, const float*, const float*, const float*, double*,
                                               float*, float*, float*);
template copa_status_t launch_loss_grad<double>(copa_ctx*, const TensorView&, int, const double*, const double*,
                                                const double*, const double*, const double*, const double*,
                                                double*, double*, double*, double*);

}  // namespace copa

using namespace copa;

extern "C" copa_status_t copa_loss_grad(copa_handle_t h, const copa_tensor_t* X, int32_t R,
                                        const copa_procrustes_out_t* st, const void* H, const void* V,
                                        const void* W, double* loss, void* gH, void* gV, void* gW) {
  if (!h) return COPA_ERR_INVALID_ARG;
  copa_status_t s;
  if ((s = cuda_check(h, cudaSetDevice(h->device), "cudaSetDevice")) != COPA_OK) return s;
  if ((s = check_tensor_args(h, X)) != COPA_OK) return s;
  if (R < 1 || R > kMaxR) return fail(h, COPA_ERR_INVALID_ARG, "copa_loss_grad: R out of range");
  if (!st || !st->Q || !st->T || !st->Pi || !H || !V || !W || !loss || !gH || !gV || !gW)
    return fail(h, COPA_ERR_INVALID_ARG, "copa_loss_grad: NULL argument (Pi is required)");
  const TensorView v = view_of(X);
  if (h->precision == COPA_PREC_MIXED)
    return launch_loss_grad<float>(h, v, R, (const float*)st->Q, (const float*)st->T, (const float*)st->Pi,
                                   (const float*)H, (const float*)V, (const float*)W, loss, (float*)gH, (float*)gV,
                                   (float*)gW);
  return launch_loss_grad<double>(h, v, R, (const double*)st->Q, (const double*)st->T, (const double*)st->Pi,
                                  (const double*)H, (const double*)V, (const double*)W, loss, (double*)gH,
                                  (double*)gV, (double*)gW);
}
