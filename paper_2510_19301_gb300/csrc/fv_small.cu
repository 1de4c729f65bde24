// fv_small.cu -- the forward engine for small state spaces, K <= 128: a
// persistent grid of CTAs of KM threads (KM = 64 or 128, the class bound),
// each running one job at a time from the launch's counter, for every
// job kind of the slot engine: exact decoding with psi rows (Sec. III-A),
// the FLASH root pass with MidState, delta snapshots and ancestor maps at
// the division points, FLASH subtasks from the pruned start (Alg. 2,
// Sec. V-B.2), budget leaves and Checkpoint Viterbi passes.
//
// Target state j is owned by one thread (two for exact decoding, each with
// half of the rows) that keeps its part of the column logA[:, j] in
// registers; delta_{t-1} sits in shared memory (double buffered) and every
// thread reads it as broadcast rows.  Per step the thread forms its
// candidates fl(delta_{t-1}[i] + logA[i][j]) in ascending i, in four
// interleaved chains over quarters of the rows, keeping the first strictly
// larger candidate and its row; the quarters merge in row order, so ties
// keep the lowest row and the kept value is that row's candidate, as
// Sec. III-A's argmax rule and the oracle fix.  delta_t = fl(max + E_t[j]);
// psi_t[j] is the row.  The slot engine spends a few thousand cycles of
// merges, re-scans and barriers on every tick whatever K is; here a step
// costs about 4.5 instructions per candidate row, which is what a lone
// short-K sequence (a latency-bound decode) needs.  Emission scores are
// loaded four steps ahead (a discrete table is staged in shared memory as
// [symbol][state] when it fits), so a lone sequence does not wait on them.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

// emission score E_t[j]: the dense row, or logB[j][x_t] for discrete
// symbols (from shared memory, transposed to [symbol][state], when the
// table fits there)
constexpr int kSmallLogB = 48 * 1024;  // bytes of logB staged in shared memory at most
template <int KM>
__host__ __device__ inline bool small_stage_logB(const DenseArgs& a) {
  return a.emit != FV_EMIT_DENSE && (size_t)a.V * KM * sizeof(float) <= (size_t)kSmallLogB;
}
template <int KM>
__device__ __forceinline__ float small_emit(const DenseArgs& a, const Job& jb, int t, int j, const float* sB) {
  if (a.emit == FV_EMIT_DENSE) return __ldg(a.E + jb.e_off + (int64_t)t * a.K + j);
  const int x = __ldg(a.obs + jb.e_off + t);
  return sB ? sB[x * KM + j] : __ldg(a.logB + (int64_t)j * a.V + x);
}
constexpr int kSmallAhead = 4;  // emission scores loaded this many steps ahead
// TPC = threads per state: with two, each runs the argmax over half of the
// rows, the pair merges with one shuffle of adjacent lanes and the first
// writes.  Exact decoding always runs two; the other job kinds run two
// when the launch's jobs all fit the resident grid at once (a lone
// sequence's FLASH levels), else one (twice the jobs in flight: measured,
// two threads cut config 1's FLASH decode by 12% and slowed a 512-sequence
// K=64 FLASH batch by 45%).
// VAN: the exact-decoding instance (no MidState, snapshots or task lists,
// fewer registers); otherwise every job kind of the engines
template <int KM, bool VAN, int TPC>
__global__ void __launch_bounds__(KM * TPC, VAN ? (KM <= 64 ? 6 : 2) : (KM <= 64 ? 8 / TPC : 1)) small_fwd_kernel(DenseArgs a) {
  constexpr int RH = KM / TPC;  // rows per thread
  constexpr int Q = RH / 4;                      // rows per chain
  __shared__ __align__(16) float sd[2][KM];
  __shared__ uint16_t smid[2][KM];  // MidState_{t-1}, MidState_t
  __shared__ float ssnap[KM];       // sub jobs: delta_{tmid}
  extern __shared__ float sB_dyn[];
  if (a.hdr->status != 0) return;  // an earlier kernel recorded an error
  const int kind = VAN ? (int)kJobVanilla : a.kind, K = a.K, tid = threadIdx.x;
  const int j = tid / TPC, h = tid % TPC, r0 = h * RH;  // state, row share, its first row
  const bool own = j < K, lead = h == 0;
  // rows and states beyond K are -inf, so they never win; the model is the
  // same for every job of the launch, so the column stays in registers
  float A[RH];
  auto load_column = [&]() {
#pragma unroll
    for (int i = 0; i < RH; ++i)
      A[i] = (own && r0 + i < K) ? __ldg(a.logA + (int64_t)(r0 + i) * K + j) : -CUDART_INF_F;
  };
  if constexpr (!VAN) load_column();
  const float* sB = nullptr;
  if (small_stage_logB<KM>(a)) {
    for (int x = h; x < a.V; x += TPC) sB_dyn[x * KM + j] = own ? __ldg(a.logB + (int64_t)j * a.V + x) : 0.f;
    sB = sB_dyn;
  }
  // exact decoding: one job per CTA (grid = sequences); other kinds:
  // persistent, jobs drawn one at a time from the launch's counter, so
  // the column is loaded once for the many short tasks of a FLASH level
  __shared__ int s_k;
  const bool from_tasks = kind == kJobSub || kind == kJobLeaf;
  const int count = from_tasks ? *a.task_count : a.order_count;
  auto run_job = [&](const int k) {
    // ---- the job: a sequence (exact decoding, FLASH root pass) or a task
    // of the current list (FLASH subtask, budget or checkpoint leaf)
    int b, m, n, pad = 0, q_prev = 0, q_n = 0, Pe = 1;
    float s_prev = 0.f;
    if (!from_tasks) {
      b = a.order[a.order_begin + k];
      m = 0;
      n = a.jobs[b].T - 1;
    } else {
      const Task tk = a.tasks[(a.task_first ? *a.task_first : 0) + (int64_t)k];
      b = tk.b;
      m = tk.m;
      n = tk.n;
      pad = tk.pad;
    }
    const Job jb = a.jobs[b];
    const int T = jb.T;
    if (T < 1 || n < m) return;
    if constexpr (VAN) load_column();  // (one job per CTA)
    if (kind == kJobRoot || (kind == kJobLeaf && a.ckpt)) Pe = a.ckpt ? ckpt_count(T, a.P) : flash_pe(T, a.P);
    if (from_tasks && !a.ckpt) {
      // states revealed by earlier levels (clamped into [0, K))
      const int qn = a.paths[jb.path_off + n];
      q_n = (unsigned)qn < (unsigned)K ? qn : 0;
      if (m > 0) {
        const int qp = a.paths[jb.path_off + m - 1];
        q_prev = (unsigned)qp < (unsigned)K ? qp : 0;
        s_prev = a.sval[jb.aux_off + m - 1];
      }
    }
    if (!VAN && lead) {
      smid[0][j] = smid[1][j] = 0;
      ssnap[j] = -CUDART_INF_F;
    }
    // root pass: division points (Sec. V-A) or checkpoints
    int kdiv = 0, ediv = kind == kJobRoot ? flash_div(0, T, Pe) : 0x7fffffff, eprev = -1;
    const int tmid = (m + n) / 2;  // sub jobs
    // E_{t}, ..., E_{t+kSmallAhead-1} of this state, oldest first
    float er[kSmallAhead];
#pragma unroll
    for (int k = 0; k < kSmallAhead; ++k) er[k] = (own && m + k <= n) ? small_emit<KM>(a, jb, m + k, j, sB) : 0.f;
    int cur = 0;
    for (int t = m; t <= n; ++t) {
      const float e = er[0];
#pragma unroll
      for (int k = 0; k + 1 < kSmallAhead; ++k) er[k] = er[k + 1];
      er[kSmallAhead - 1] = (own && t + kSmallAhead <= n) ? small_emit<KM>(a, jb, t + kSmallAhead, j, sB) : 0.f;
      float dval;
      int g = 0;
      uint32_t mnew = 0;
      int f_mid = 0;
      if (t == m) {
        // first step of the job: pi, a stored checkpoint, or the pruned start
        // from the revealed state q_{m-1} (Sec. V-B.2)
        if (t == 0) {
          dval = own ? __fadd_rn(__ldg(a.log_pi + j), e) : -CUDART_INF_F;
        } else if (a.ckpt) {
          dval = own ? __ldg(a.snaps + jb.aux_off + (int64_t)pad * K + j) : -CUDART_INF_F;
        } else {
          const float av = own ? __ldg(a.logA + (int64_t)q_prev * K + j) : -CUDART_INF_F;
          dval = a.complete ? __fadd_rn(av, e) : __fadd_rn(__fadd_rn(s_prev, av), e);
          if (!own) dval = -CUDART_INF_F;
        }
      } else {
        const float4* dv = reinterpret_cast<const float4*>(sd[cur]);
        float bq[4];
        int gq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          bq[q] = -CUDART_INF_F;
          gq[q] = r0 + q * Q;
        }
#pragma unroll
        for (int i4 = 0; i4 < Q / 4; ++i4)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = q * Q + 4 * i4;  // local row; global r0 + i
            const float4 x = dv[(r0 + i) / 4];
            float c = __fadd_rn(x.x, A[i]);
            if (c > bq[q]) { bq[q] = c; gq[q] = r0 + i; }
            c = __fadd_rn(x.y, A[i + 1]);
            if (c > bq[q]) { bq[q] = c; gq[q] = r0 + i + 1; }
            c = __fadd_rn(x.z, A[i + 2]);
            if (c > bq[q]) { bq[q] = c; gq[q] = r0 + i + 2; }
            c = __fadd_rn(x.w, A[i + 3]);
            if (c > bq[q]) { bq[q] = c; gq[q] = r0 + i + 3; }
          }
        float bv = bq[0];
        g = gq[0];
#pragma unroll
        for (int q = 1; q < 4; ++q)
          if (bq[q] > bv) { bv = bq[q]; g = gq[q]; }
        if constexpr (TPC == 2) {
          // the pair's merge: the lower rows (h = 0) win ties; both threads
          // end with the same (maximum, row)
          const float ov = __shfl_xor_sync(0xffffffffu, bv, 1);
          const int og = __shfl_xor_sync(0xffffffffu, g, 1);
          const bool other = h == 0 ? (ov > bv) : !(bv > ov);
          if (other) { bv = ov; g = og; }
        }
        dval = own ? __fadd_rn(bv, e) : -CUDART_INF_F;
        if (lead && own && (kind == kJobVanilla || kind == kJobLeaf)) {
          const int64_t row = kind == kJobVanilla ? jb.aux_off + (int64_t)t * K
                              : a.ckpt        ? 2 * (jb.aux_off + (int64_t)Pe * K) + (int64_t)(t - m - 1) * K
                                              : (int64_t)(pad + t - m - 1) * K;
          a.psi[row + j] = (uint16_t)g;
        }
        // MidState (Alg. 2): the argmax at the step after a division point,
        // then carried along the argmax
        if (kind == kJobRoot && !a.ckpt && eprev >= 0) f_mid = (t == eprev + 1) ? 1 : 2;
        if (kind == kJobSub) f_mid = (t == tmid + 1) ? 1 : (t > tmid + 1 ? 2 : 0);
        if (f_mid) mnew = f_mid == 1 ? (uint32_t)g : smid[cur][g];
        // sub jobs keep delta_{tmid} (the previous step's delta)
        if (lead && kind == kJobSub && t == tmid + 1) ssnap[j] = sd[cur][j];
      }
      if (lead && f_mid) smid[cur ^ 1][j] = (uint16_t)mnew;
      if (kind == kJobRoot && t == ediv) {
        // division point: delta snapshot and, from the second one on, the
        // ancestor map (MidState); checkpoints keep delta only
        if (lead && own) {
          if (a.ckpt) {
            a.snaps[jb.aux_off + (int64_t)kdiv * K + j] = dval;
          } else {
            a.snaps[(int64_t)b * a.snap_stride + (int64_t)kdiv * K + j] = dval;
            if (kdiv >= 1) a.maps[(int64_t)b * a.map_stride + (int64_t)(kdiv - 1) * K + j] = (uint16_t)mnew;
          }
        }
        eprev = ediv;
        ++kdiv;
        ediv = kdiv < Pe ? flash_div(kdiv, T, Pe) : 0x7fffffff;
      }
      if (lead) sd[cur ^ 1][j] = dval;
      __syncthreads();
      cur ^= 1;
    }
    if (kind == kJobVanilla && tid < 32) {
      // termination: q_{T-1} = lowest argmax_j delta_{T-1}[j], score = delta_{T-1}[q]
      float v = sd[cur][tid];
      int qi = tid;
#pragma unroll
      for (int k = 1; k < KM / 32; ++k) {
        const float vk = sd[cur][tid + 32 * k];
        if (vk > v) { v = vk; qi = tid + 32 * k; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oq = __shfl_xor_sync(0xffffffffu, qi, o);
        if (ov > v || (ov == v && oq < qi)) { v = ov; qi = oq; }
      }
      if (tid == 0) {
        a.qlast[b] = qi;
        a.scores[b] = sd[cur][qi];
      }
    } else if (kind == kJobSub && tid == 0) {
      // Alg. 2 output: q*_{tmid} = MidState_n[q*_n]; its delta from the snapshot
      int q = smid[cur][q_n];
      q = (unsigned)q < (unsigned)K ? q : 0;
      a.paths[jb.path_off + tmid] = q;
      a.sval[jb.aux_off + tmid] = ssnap[q];
    }
  };
  if constexpr (VAN) {
    if (sB) __syncthreads();  // the staged table is complete
    if ((int)blockIdx.x < count) run_job(blockIdx.x);
  } else {
    for (;;) {
      if (tid == 0) s_k = (int)atomicAdd(a.pop, 1ull);
      __syncthreads();
      const int k = s_k;
      __syncthreads();
      if (k >= count) break;
      run_job(k);
    }
  }
}

// exact decoding: one CTA per sequence; other kinds: a persistent grid of
// the CTAs resident at once (per instance), at most one per job
// CTAs of the instance resident at once on the device (0 on an error)
template <int KM, bool VAN, int TPC>
static int small_resident(size_t sm) {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, small_fwd_kernel<KM, VAN, TPC>, KM * TPC, sm) !=
          cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * nsm;
}

template <int KM, bool VAN, int TPC>
static cudaError_t launch_small_cfg(const DenseArgs& a, int jobs, int resident, cudaStream_t st) {
  const size_t sm = small_stage_logB<KM>(a) ? (size_t)a.V * KM * sizeof(float) : 0;
  if (resident < 1) return cudaErrorInvalidConfiguration;
  const int grid = VAN ? jobs : (jobs < resident ? jobs : resident);
  small_fwd_kernel<KM, VAN, TPC><<<grid, KM * TPC, sm, st>>>(a);
  return cudaGetLastError();
}

template <int KM>
static cudaError_t launch_small_class(const DenseArgs& a, int jobs, cudaStream_t st) {
  const size_t sm = small_stage_logB<KM>(a) ? (size_t)a.V * KM * sizeof(float) : 0;
  if (a.kind == kJobVanilla) return launch_small_cfg<KM, true, 2>(a, jobs, small_resident<KM, true, 2>(sm), st);
  const int r2 = small_resident<KM, false, 2>(sm);
  if (jobs <= r2) return launch_small_cfg<KM, false, 2>(a, jobs, r2, st);
  return launch_small_cfg<KM, false, 1>(a, jobs, small_resident<KM, false, 1>(sm), st);
}

cudaError_t launch_small_forward(const DenseArgs& a, cudaStream_t st) {
  if (a.K > 128) return cudaErrorInvalidValue;
  // upper bound of the launch's jobs (task lists count on the device)
  const int jobs = (a.kind == kJobVanilla || a.kind == kJobRoot) ? a.order_count : a.max_jobs;
  if (jobs <= 0) return cudaSuccess;
  return a.K <= 64 ? launch_small_class<64>(a, jobs, st) : launch_small_class<128>(a, jobs, st);
}

}  // namespace fv
