// fv_backward.cu -- path-count backward of the Viterbi score and the path
// log-likelihood (forward order of Sec. III-A).
//
// With every path q_b held fixed the score of sequence b is the linear
// function logpi[q_0] + sum_t (logA[q_{t-1}, q_t] + E_t[q_t]), so for
// L = sum_b g_b score_b:
//   dlog_pi[j]   = sum_b g_b [q_{b,0} = j]
//   dlogA[i][j]  = sum_b g_b #{t : (q_{b,t-1}, q_{b,t}) = (i, j)}
//   dE_b[t][j]   = g_b [q_{b,t} = j]
// Determinism: each parameter's terms fl(g_b * count) are added in
// ascending b starting from +0.  CTA r owns a range of "pairs" (the K*K
// transitions followed by the K start states) in shared memory and walks
// the batch in order; per sequence it counts the pairs with shared integer
// atomics (order-free) and then exactly one thread per touched pair
// (whoever takes the count with atomicExch) folds that sequence's term in.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

constexpr int kBwdThreads = 1024;

__global__ void __launch_bounds__(kBwdThreads) backward_pairs_kernel(const Job* jobs, int32_t n_seq, int32_t K,
                                                                     const int32_t* paths, const float* g,
                                                                     int64_t pairs_per_cta, float* dlogA,
                                                                     float* dlog_pi, const WsHeader* hdr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (hdr->status != 0) return;
  const int64_t KK = (int64_t)K * K, total = KK + K;
  const int64_t lo = (int64_t)blockIdx.x * pairs_per_cta;
  const int64_t hi = lo + pairs_per_cta < total ? lo + pairs_per_cta : total;
  if (lo >= hi) return;
  const int npr = (int)(hi - lo);
  float* acc = reinterpret_cast<float*>(smem_raw);
  int* cnt = reinterpret_cast<int*>(acc + pairs_per_cta);
  for (int x = threadIdx.x; x < npr; x += blockDim.x) {
    acc[x] = 0.0f;
    cnt[x] = 0;
  }
  __syncthreads();
  for (int b = 0; b < n_seq; ++b) {
    const Job jb = jobs[b];
    const int32_t* q = paths + jb.path_off;
    const float gb = g[b];
    // pair index of step t: t = 0 -> start state, t >= 1 -> transition
    for (int t = threadIdx.x; t < jb.T; t += blockDim.x) {
      const int qt = q[t];
      if ((unsigned)qt >= (unsigned)K) continue;
      int64_t pr;
      if (t == 0) {
        pr = KK + qt;
      } else {
        const int qp = q[t - 1];
        if ((unsigned)qp >= (unsigned)K) continue;
        pr = (int64_t)qp * K + qt;
      }
      if (pr >= lo && pr < hi) atomicAdd(&cnt[pr - lo], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < jb.T; t += blockDim.x) {
      const int qt = q[t];
      if ((unsigned)qt >= (unsigned)K) continue;
      int64_t pr;
      if (t == 0) {
        pr = KK + qt;
      } else {
        const int qp = q[t - 1];
        if ((unsigned)qp >= (unsigned)K) continue;
        pr = (int64_t)qp * K + qt;
      }
      if (pr >= lo && pr < hi) {
        const int c = atomicExch(&cnt[pr - lo], 0);
        if (c != 0) acc[pr - lo] = __fadd_rn(acc[pr - lo], __fmul_rn(gb, (float)c));
      }
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < npr; x += blockDim.x) {
    const int64_t pr = lo + x;
    if (pr < KK) dlogA[pr] = acc[x];
    else dlog_pi[pr - KK] = acc[x];
  }
}

// dE over the batch's emission rows: g_b on the path, +0 elsewhere.
__global__ void backward_emissions_kernel(const Job* jobs, int32_t b0, int32_t K, const int32_t* paths, const float* g,
                                          float* dE, const WsHeader* hdr) {
  if (hdr->status != 0) return;
  const int b = b0 + blockIdx.y;
  const Job jb = jobs[b];
  const int64_t n = (int64_t)jb.T * K;
  const float gb = g[b];
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(x / K), j = (int)(x % K);
    dE[jb.e_off + x] = (paths[jb.path_off + t] == j) ? gb : 0.0f;
  }
}

// Path log-likelihood straight from the batch arrays (no job table):
// s = fl(logpi[q0] + E_0[q0]); s = fl(fl(s + logA[q_{t-1}][q_t]) + E_t[q_t]);
// a state id outside [0, K) makes the score -inf.
__global__ void path_score_direct_kernel(ScoreArgs a, int32_t model, int32_t n_seq, const int32_t* T,
                                         const int32_t* model_idx, const int64_t* e_off, const int64_t* path_off,
                                         const int32_t* paths, float* scores) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_seq) return;
  if ((model_idx ? model_idx[b] : 0) != model) return;
  const int Tb = T[b];
  if (Tb < 1) {
    scores[b] = -CUDART_INF_F;
    return;
  }
  const int32_t* q = paths + path_off[b];
  const int64_t eo = e_off[b];
  auto emis = [&](int t, int j) -> float {
    if (a.emit == FV_EMIT_DENSE) return __ldg(a.E + eo + (int64_t)t * a.K + j);
    return __ldg(a.logB + (int64_t)j * a.V + __ldg(a.obs + eo + t));
  };
  auto csr_w = [&](int i, int j) -> float {
    float best = -CUDART_INF_F;
    for (int e = a.row_ptr[i]; e < a.row_ptr[i + 1]; ++e)
      if (a.col[e] == j) best = fmaxf(best, a.val[e]);
    return best;
  };
  int qp = q[0];
  if ((unsigned)qp >= (unsigned)a.K) {
    scores[b] = -CUDART_INF_F;
    return;
  }
  float s = __fadd_rn(__ldg(a.log_pi + qp), emis(0, qp));
  for (int t = 1; t < Tb; ++t) {
    const int qt = q[t];
    if ((unsigned)qt >= (unsigned)a.K) {
      scores[b] = -CUDART_INF_F;
      return;
    }
    const float w = a.trans == FV_TRANS_DENSE ? __ldg(a.logA + (int64_t)qp * a.K + qt) : csr_w(qp, qt);
    s = __fadd_rn(__fadd_rn(s, w), emis(t, qt));
    qp = qt;
  }
  scores[b] = s;
}

size_t backward_pairs_per_cta(int K, int* n_ctas) {
  const int64_t total = (int64_t)K * K + K;
  const int64_t cap = (200 * 1024) / 8;  // acc + cnt per pair in shared memory
  int64_t ctas = (total + cap - 1) / cap;
  // spread large problems over more CTAs (each walks the whole batch)
  if (ctas < 1) ctas = 1;
  const int64_t per = (total + ctas - 1) / ctas;
  *n_ctas = (int)ctas;
  return (size_t)per;
}

cudaError_t launch_backward(const Job* jobs, int32_t n_seq, int32_t K, const int32_t* paths, const float* g,
                            float* dlog_pi, float* dlogA, float* dE, int32_t max_T, const WsHeader* hdr,
                            cudaStream_t st) {
  if (n_seq <= 0) return cudaSuccess;
  int nct = 1;
  const size_t per = backward_pairs_per_cta(K, &nct);
  const size_t smem = per * 8;
  cudaError_t e =
      cudaFuncSetAttribute(backward_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  backward_pairs_kernel<<<nct, kBwdThreads, smem, st>>>(jobs, n_seq, K, paths, g, (int64_t)per, dlogA, dlog_pi,
                                                        hdr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t per_seq = (int64_t)max_T * K;
  int gx = (int)((per_seq + 255) / 256);
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  for (int b0 = 0; b0 < n_seq; b0 += 65535) {
    const int nb = n_seq - b0 < 65535 ? n_seq - b0 : 65535;
    backward_emissions_kernel<<<dim3(gx, nb), 256, 0, st>>>(jobs, b0, K, paths, g, dE, hdr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_path_score_direct(const ScoreArgs& a, int32_t model, int32_t n_seq, const int32_t* T,
                                     const int32_t* model_idx, const int64_t* e_off, const int64_t* path_off,
                                     const int32_t* paths, float* scores, cudaStream_t st) {
  if (n_seq <= 0) return cudaSuccess;
  path_score_direct_kernel<<<(n_seq + 127) / 128, 128, 0, st>>>(a, model, n_seq, T, model_idx, e_off, path_off,
                                                                 paths, scores);
  return cudaGetLastError();
}

}  // namespace fv
