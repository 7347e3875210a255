// V-mode tile products on the tensor cores (FP32 path): for 128 consecutive visit rows at a
// time, U = (Q H) .* W(k(i), :) and the tile's Gram U^T U (the MTTKRP for V of Sec. 3.1
// with the implicit Y_k, and the Gram that the V update and the FIT need), as tcgen05
// MMAs with the accumulators in tensor memory.
//
// Precision. The MMAs take TF32 operands; every FP32 operand x is split as
// x = x_hi + x_lo with x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a product is formed
// from three or four partial products (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi [+ A_lo B_lo]),
// which keeps about 2^-21 of relative accuracy per product: the accuracy of the FP32 path.
// Sums over the 40-odd terms of a row and over the 128 rows of a tile accumulate in FP32 in
// tensor memory; the tile Grams are summed across tiles as compensated float pairs and
// leave as FP64 partials.
//
// One CTA of 128 threads, persistent over tiles, one thread per row of a tile:
//   1. the Q tile is loaded (float4 per thread), split, and stored as the K-major A
//      operand (hi and lo copies); H^T (hi, lo) is the B operand, stored once;
//   2. thread 0 issues D1 = Q_hi [H_hi H_lo] and adds Q_lo H_hi to its first half (M = 128,
//      N = R rounded to 16, doubled for the first product; K = R rounded to 8) into tensor
//      memory and commits to an mbarrier;
//   3. each thread reads its row of D1, forms u_i = d_i .* w_k(i), stores it, and writes
//      u_i^T split in hi and lo into the A operand of the Gram: rows 0-63 hold U_hi^T and
//      rows 64-127 hold U_lo^T (the Q buffers are dead by then and are reused);
//   4. thread 0 issues D2 = [U_hi^T; U_lo^T] [U_hi^T; pad; U_lo^T]^T (M = 128, N = 64 + R
//      rounded to 16, K = 128 tile rows): the four blocks at rows r, 64 + r and columns
//      c, 64 + c add up to entry (r, c) of the tile's U^T U;
//   5. the threads owning lanes r < R and 64 + r read columns c and 64 + c and add them to
//      their compensated sums.
// Every wait on an mbarrier is bounded (1 s of wall time); a timeout records
// COPA_ERR_TIMEOUT in the status word, waits once more (bounded) for the MMAs in flight,
// frees the tensor memory and ends the kernel. If that second wait gives up as well, detail
// word 2 of the status is set to 3: the tensor memory was released while MMAs may still have
// been writing it, and the handle should not be used further. For tests of this path a
// launch can make its first wait run out on purpose: it then waits on an mbarrier that
// nothing arrives at (force_ns of wall time) instead of the first MMA commit.
#include "copa_internal.cuh"
#include "tc_sm100.cuh"

namespace copa {

namespace {

constexpr int kTM = 128;                        // rows per tile = threads per CTA
constexpr int kLBO = 144;                       // bytes between K-adjacent core matrices (conflict-free stores)
constexpr int kGChunks = kTM / 4;               // K chunks of the Gram operand
constexpr int kGSBO = kGChunks * kLBO;          // 4608
constexpr int kGBytes = (kTM / 8) * kGSBO;      // 73,728: the Gram's A operand, 128 rows
constexpr uint32_t kTmemCols = 256;             // D1 at column 0 (96 wide), D2 at column 128 (112 wide)
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr int kQPer = 12;                       // float4 chunks of a Q tile per thread (128 x 48 / 4 / 128)

struct TcLay {
  int KP, NP, nch, sbo, qbytes, hbytes, total;
};

__host__ __device__ inline TcLay tc_lay(int R) {
  TcLay L;
  L.KP = (R + 7) / 8 * 8;         // K of D1, a multiple of 8 (one MMA takes K = 8)
  L.NP = (R + 15) / 16 * 16;      // N of both MMAs (M = 128 needs N % 16 == 0)
  L.nch = L.KP / 4;
  L.sbo = L.nch * kLBO;
  L.qbytes = (kTM / 8) * L.sbo;   // one copy of the Q tile operand
  L.hbytes = (L.NP / 8) * L.sbo;  // one copy of the H^T operand
  // [Gram operand / Q hi, Q lo][H^T hi][H^T lo][2 mbarriers, tmem address]
  L.total = kGBytes + 2 * L.hbytes + 32;
  return L;
}

// Byte offset of element (row, k) in a K-major operand with stride-dimension offset sbo.
__device__ __forceinline__ int opnd_off(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tc::to_tf32(x);
  lo = tc::to_tf32(x - hi);
}

__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x), bp = __fsub_rn(s, hi);
  lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
}

}  // namespace

namespace {

__device__ __forceinline__ float4 split4(float4 x, float4& lo) {
  float4 hi;
  split_tf32(x.x, hi.x, lo.x);
  split_tf32(x.y, hi.y, lo.y);
  split_tf32(x.z, hi.z, lo.z);
  split_tf32(x.w, hi.w, lo.w);
  return hi;
}

// Requires R % 4 == 0, R <= 48, and 16-byte aligned Q, W and U.
__global__ void __launch_bounds__(kTM, 2) k_uvec_tc(int64_t S, int R, const float* __restrict__ Q,
                                                    const float* __restrict__ H, const float* __restrict__ W,
                                                    const int32_t* __restrict__ row_subj, float* __restrict__ U,
                                                    double* __restrict__ utu_part, int* __restrict__ status,
                                                    uint64_t force_ns) {
  const TcLay L = tc_lay(R);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* opg = smem;                  // the Gram's A operand (128 rows), aliasing the Q tile
  unsigned char* oqh = smem;                  // Q tile, hi
  unsigned char* oql = smem + L.qbytes;       // Q tile, lo
  unsigned char* ohh = smem + kGBytes;        // H^T, hi
  unsigned char* ohl = ohh + L.hbytes;        // H^T, lo
  uint64_t* bars = reinterpret_cast<uint64_t*>(ohl + L.hbytes);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar1 = tc::smem_u32(bars), bar2 = tc::smem_u32(bars + 1);
  const uint32_t bar_never = tc::smem_u32(bars + 2);   // nothing arrives here (timeout tests)

  for (int e = tid; e < L.NP * L.KP; e += kTM) {   // H^T: element (n, k) = H(k, n), zero-padded
    const int n = e / L.KP, k = e - n * L.KP;
    float hi, lo;
    split_tf32((n < R && k < R) ? H[k * R + n] : 0.f, hi, lo);
    *reinterpret_cast<float*>(ohh + opnd_off(n, k, L.sbo)) = hi;
    *reinterpret_cast<float*>(ohl + opnd_off(n, k, L.sbo)) = lo;
  }
  if (tid == 0) {
    tc::mbar_init(bar1, 1);
    tc::mbar_init(bar2, 1);
    tc::mbar_init(bar_never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(taddr_s), kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  const uint32_t d1 = tmem, d2 = tmem + 128;
  const uint32_t lane_sel = (uint32_t)(32 * warp) << 16;   // this warp's quarter of the lanes
  // D1: A = Q_hi against B = [H_hi^T; H_lo^T] (N = 2 NP, the two copies are adjacent), then
  // A = Q_lo against H_hi^T (N = NP). D2: A = [U_hi^T; U_lo^T] against B = the same rows
  // 0..64+NP-1 (N = 64 + NP: U_hi^T, padding, U_lo^T).
  const uint32_t id_d1a = tc::idesc_tf32(kTM, 2 * L.NP), id_d1b = tc::idesc_tf32(kTM, L.NP),
                 id_d2 = tc::idesc_tf32(kTM, 64 + L.NP);
  const int gr = tid & 63;   // Gram row read by this thread: rows 0-63 from U_hi^T, 64-127 from U_lo^T
  const bool grow = gr < R;
  float ghi[48], glo[48];
#pragma unroll
  for (int c = 0; c < 48; ++c) ghi[c] = glo[c] = 0.f;
  uint32_t ph = 0;
  bool failed = false;
  const int64_t ntiles = (S + kTM - 1) / kTM;
  // The next tile's Q chunks (kQPer float4 per thread) and row -> subject entry are loaded
  // one tile ahead, so that their latency overlaps the current tile's MMAs.
  float4 qn[kQPer];
  int32_t sn = 0;
  auto prefetch = [&](int64_t tt) {
    const int64_t j0 = tt * kTM;
    const int nr = tt < ntiles ? (int)min((int64_t)kTM, S - j0) : 0;
#pragma unroll
    for (int q = 0; q < kQPer; ++q) {
      const int e = tid + q * kTM, m = e / L.nch, c = e - m * L.nch;
      qn[q] = (e < kTM * L.nch && m < nr && 4 * c < R)
                  ? __ldcs(reinterpret_cast<const float4*>(Q + (j0 + m) * R) + c)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    sn = tid < nr ? __ldg(row_subj + j0 + tid) : 0;
  };
  prefetch(blockIdx.x);

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i0 = t * kTM;
    const int nrow = (int)min((int64_t)kTM, S - i0);
    // ---- 1. the Q tile as the A operand (hi, lo); this thread's W row ----
    const bool mine = tid < nrow;
    const int64_t ksub = mine ? (int64_t)sn : 0;
#pragma unroll
    for (int q = 0; q < kQPer; ++q) {
      const int e = tid + q * kTM, m = e / L.nch, c = e - m * L.nch;
      if (e < kTM * L.nch) {
        float4 lo;
        const float4 hi = split4(qn[q], lo);
        *reinterpret_cast<float4*>(oqh + opnd_off(m, 4 * c, L.sbo)) = hi;
        *reinterpret_cast<float4*>(oql + opnd_off(m, 4 * c, L.sbo)) = lo;
      }
    }
    prefetch(t + gridDim.x);
    float wv[48];
    {
      const int64_t k = ksub;
      const float4* wr = reinterpret_cast<const float4*>(W + k * R);
#pragma unroll
      for (int c4 = 0; c4 < 12; ++c4) {
        const float4 v = (mine && 4 * c4 < R) ? __ldg(wr + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
        wv[4 * c4] = v.x;
        wv[4 * c4 + 1] = v.y;
        wv[4 * c4 + 2] = v.z;
        wv[4 * c4 + 3] = v.w;
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // ---- 2. D1[:, 0:NP] = Q_hi H_hi + Q_lo H_hi, D1[:, NP:2NP] = Q_hi H_lo ----
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t qh = tc::smem_u32(oqh), ql = tc::smem_u32(oql), hh = tc::smem_u32(ohh);
      for (int ks = 0; ks < L.KP / 8; ++ks) {
        const uint32_t ko = ks * 2 * kLBO;
        tc::mma_tf32(d1, tc::smem_desc(qh + ko, kLBO, L.sbo), tc::smem_desc(hh + ko, kLBO, L.sbo), id_d1a, ks > 0);
        tc::mma_tf32(d1, tc::smem_desc(ql + ko, kLBO, L.sbo), tc::smem_desc(hh + ko, kLBO, L.sbo), id_d1b, true);
      }
      tc::mma_commit(bar1);
    }
    bool ok = force_ns ? tc::mbar_wait(bar_never, 0, force_ns) : tc::mbar_wait(bar1, ph, kWaitNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(status, COPA_ERR_TIMEOUT, 1);
      // the MMAs in flight, before the memory is released
      const bool drained = tc::mbar_wait(bar1, ph, kWaitNs);
      if (__syncthreads_or(!drained) && tid == 0) status[2] = 3;
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // ---- 3. u_i = d_i .* w_k(i): to U, and split into U_hi^T, U_lo^T (the Q tile is dead) ----
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (16 * j < L.NP) {
        float v[16], v2[16];
        tc::tmem_ld16(d1 + lane_sel + 16 * j, v);
        tc::tmem_ld16(d1 + lane_sel + L.NP + 16 * j, v2);
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = (16 * j + q < R) ? (v[q] + v2[q]) * wv[16 * j + q] : 0.f;
        if (mine) {
          float4* ur = reinterpret_cast<float4*>(U + (i0 + tid) * R);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (16 * j + 4 * q < R) ur[4 * j + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float hi, lo;
          split_tf32(v[q], hi, lo);
          *reinterpret_cast<float*>(opg + opnd_off(16 * j + q, tid, kGSBO)) = hi;
          *reinterpret_cast<float*>(opg + opnd_off(64 + 16 * j + q, tid, kGSBO)) = lo;
        }
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // ---- 4. D2 = [U_hi^T; U_lo^T] [U_hi^T; pad; U_lo^T]^T over the tile's rows ----
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t g = tc::smem_u32(opg);
      for (int ks = 0; ks < kTM / 8; ++ks) {
        const uint64_t ad = tc::smem_desc(g + ks * 2 * kLBO, kLBO, kGSBO);
        tc::mma_tf32(d2, ad, ad, id_d2, ks > 0);
      }
      tc::mma_commit(bar2);
    }
    ok = tc::mbar_wait(bar2, ph, kWaitNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) set_status(status, COPA_ERR_TIMEOUT, 2);
      const bool drained = tc::mbar_wait(bar2, ph, kWaitNs);
      if (__syncthreads_or(!drained) && tid == 0) status[2] = 3;
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // ---- 5. this thread's Gram row, into its compensated sums ----
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (16 * j < L.NP) {
        float v[16], v2[16];
        tc::tmem_ld16(d2 + lane_sel + 16 * j, v);        // x U_hi
        tc::tmem_ld16(d2 + lane_sel + 64 + 16 * j, v2);  // x U_lo
        tc::tmem_wait_ld();
        if (grow) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (16 * j + q < R) comp_add(ghi[16 * j + q], glo[16 * j + q], v[q] + v2[q]);
        }
      }
    }
    tc::fence_before_sync();
    ph ^= 1u;
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  if (utu_part && grow) {
    double* up = utu_part + ((size_t)blockIdx.x * 2 + (tid >> 6)) * R * R + (size_t)gr * R;
#pragma unroll
    for (int c = 0; c < 48; ++c)
      if (c < R) up[c] = failed ? 0.0 : (double)ghi[c] + (double)glo[c];
  }
}

}  // namespace

bool uvec_tc_supported(int R, const void* Q, const void* W, const void* U) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return R >= 4 && R <= 48 && R % 4 == 0 && al(Q) && al(W) && al(U);
}

// Grid: one wave of persistent CTAs; UtU partials: two per CTA (nparts).
copa_status_t launch_uvec_tc(copa_ctx* h, int64_t S, int R, const float* Q, const float* H, const float* W,
                             const int32_t* rsubj, float* U, double* utu_part, int64_t* nparts, bool size_only) {
  const TcLay L = tc_lay(R);
  copa_status_t st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_uvec_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total),
                       "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  if ((st = cuda_check(h, cudaFuncSetAttribute(k_uvec_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100),
                       "cudaFuncSetAttribute")) != COPA_OK)
    return st;
  // Two CTAs per SM (2 x 256 tensor-memory columns): shared memory (2 x 91 KB) and registers
  // (2 x 128 x 256) fit. (The occupancy query reported one for this kernel.)
  const int per_sm = 2;
  const int64_t ntiles = (S + kTM - 1) / kTM;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)h->num_sms * per_sm, ntiles));
  *nparts = blocks * 2;
  if (size_only) return COPA_OK;
  k_uvec_tc<<<(unsigned)blocks, kTM, L.total, h->stream>>>(S, R, Q, H, W, rsubj, U, utu_part, h->d_status,
                                                          (uint64_t)h->dbg_tc_force_ns);
  return cuda_check(h, cudaGetLastError(), "k_uvec_tc");
}

}  // namespace copa
