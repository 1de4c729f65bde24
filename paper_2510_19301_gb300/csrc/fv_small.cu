// fv_small.cu -- the exact forward pass (Sec. III-A) for small state
// spaces, K <= 128, on exact (vanilla) jobs: one CTA of KM threads per
// sequence (KM = 64 or 128, the class bound).
//
// Thread j owns target state j and keeps the column logA[:, j] in
// registers; delta_{t-1} sits in shared memory (double buffered) and every
// thread reads it as broadcast rows.  Per step the thread forms the K
// candidates fl(delta_{t-1}[i] + logA[i][j]) in ascending i, in four
// interleaved chains over quarters of the rows, keeping the first strictly
// larger candidate and its row; the quarters merge in row order, so ties
// keep the lowest row and the kept value is that row's candidate, as
// Sec. III-A's argmax rule and the oracle fix.  delta_t = fl(max + E_t[j]);
// psi_t[j] is the row.  The slot engine spends a few thousand cycles of
// merges, re-scans and barriers on every tick whatever K is; here a step
// costs about 4.5 instructions per candidate row, which is what a lone
// short-K sequence (a latency-bound decode) needs.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

__device__ __forceinline__ float small_emit(const DenseArgs& a, const Job& jb, int t, int j) {
  return a.emit == FV_EMIT_DENSE ? __ldg(a.E + jb.e_off + (int64_t)t * a.K + j)
                                 : __ldg(a.logB + (int64_t)j * a.V + __ldg(a.obs + jb.e_off + t));
}

template <int KM>
__global__ void __launch_bounds__(KM) small_fwd_kernel(DenseArgs a) {
  constexpr int Q = KM / 4;  // rows per chain
  __shared__ __align__(16) float sd[2][KM];
  if (a.hdr->status != 0) return;  // an earlier kernel recorded an error
  const int b = a.order[a.order_begin + blockIdx.x];
  const Job jb = a.jobs[b];
  const int K = a.K, T = jb.T, j = threadIdx.x;
  if (T < 1) return;
  const bool own = j < K;
  // rows and states beyond K are -inf, so they never win
  float A[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i) A[i] = (own && i < K) ? __ldg(a.logA + (int64_t)i * K + j) : -CUDART_INF_F;
  sd[0][j] = own ? __fadd_rn(__ldg(a.log_pi + j), small_emit(a, jb, 0, j)) : -CUDART_INF_F;
  float en = (own && T > 1) ? small_emit(a, jb, 1, j) : 0.f;
  __syncthreads();
  int cur = 0;
  for (int t = 1; t < T; ++t) {
    const float e = en;
    if (own && t + 1 < T) en = small_emit(a, jb, t + 1, j);  // one step ahead
    const float4* dv = reinterpret_cast<const float4*>(sd[cur]);
    float bq[4];
    int gq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bq[q] = -CUDART_INF_F;
      gq[q] = q * Q;
    }
#pragma unroll
    for (int i4 = 0; i4 < Q / 4; ++i4)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = q * Q + 4 * i4;
        const float4 x = dv[i / 4];
        float c = __fadd_rn(x.x, A[i]);
        if (c > bq[q]) { bq[q] = c; gq[q] = i; }
        c = __fadd_rn(x.y, A[i + 1]);
        if (c > bq[q]) { bq[q] = c; gq[q] = i + 1; }
        c = __fadd_rn(x.z, A[i + 2]);
        if (c > bq[q]) { bq[q] = c; gq[q] = i + 2; }
        c = __fadd_rn(x.w, A[i + 3]);
        if (c > bq[q]) { bq[q] = c; gq[q] = i + 3; }
      }
    float bv = bq[0];
    int g = gq[0];
#pragma unroll
    for (int q = 1; q < 4; ++q)
      if (bq[q] > bv) { bv = bq[q]; g = gq[q]; }
    if (own) a.psi[jb.aux_off + (int64_t)t * K + j] = (uint16_t)g;
    sd[cur ^ 1][j] = own ? __fadd_rn(bv, e) : -CUDART_INF_F;
    __syncthreads();
    cur ^= 1;
  }
  // termination: q_{T-1} = lowest argmax_j delta_{T-1}[j], score = delta_{T-1}[q]
  if (j < 32) {
    float v = sd[cur][j];
    int qi = j;
#pragma unroll
    for (int k = 1; k < KM / 32; ++k) {
      const float vk = sd[cur][j + 32 * k];
      if (vk > v) { v = vk; qi = j + 32 * k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oq = __shfl_xor_sync(0xffffffffu, qi, o);
      if (ov > v || (ov == v && oq < qi)) { v = ov; qi = oq; }
    }
    if (j == 0) {
      a.qlast[b] = qi;
      a.scores[b] = sd[cur][qi];
    }
  }
}

cudaError_t launch_small_forward(const DenseArgs& a, cudaStream_t st) {
  if (a.K > 128 || a.kind != kJobVanilla) return cudaErrorInvalidValue;
  if (a.order_count <= 0) return cudaSuccess;
  if (a.K <= 64)
    small_fwd_kernel<64><<<a.order_count, 64, 0, st>>>(a);
  else
    small_fwd_kernel<128><<<a.order_count, 128, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fv
