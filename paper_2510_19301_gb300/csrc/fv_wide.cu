// fv_wide.cu -- the exact forward engine for large state spaces
// (1024 < K <= 4096, dense transitions).
//
// One persistent cooperative launch spreads every max-plus step
// (Sec. III-A, delta_t[j] = max_i (delta_{t-1}[i] + logA[i][j]) + E_t[j])
// over the whole GPU.  Up to kWS jobs (vanilla sequences, FLASH root
// passes or FLASH subtasks, Sec. V) advance in lockstep as "lanes"; lane s
// runs the launch's jobs s, s + kWS, s + 2 kWS, ... one after another.
//
// Work split of one step:
//   * column block c (kWJ = 128 target states) belongs to cluster c;
//   * CTA r of the cluster owns source rows [r RPC, (r+1) RPC): it keeps
//     delta_{t-1} of those rows (all lanes) in shared memory, the first RWR
//     rows of each warp's slice of logA resident in shared memory and
//     streams the rest from L2 (row-pair copy Ap) through a cp.async ring;
//   * every CTA finds, per (lane, target), the maximum over its rows and
//     the lowest row reaching it (value-only tropical product, chunk
//     tracking, exact re-scan of the winning chunk), and sends
//     (value, row, ancestor) to the target's owner CTA in the cluster
//     through distributed shared memory;
//   * the owner takes the lowest rank holding the maximum, adds E_t, writes
//     delta_t to a global double buffer (plus psi, ancestor maps and
//     snapshots as the job kind needs) and publishes its step count;
//   * before the next step each CTA waits (bounded) for the owners of its
//     rows and loads delta_t of its rows from L2.
// Every wait is bounded: on timeout the kernel records FV_ETIMEOUT in the
// workspace header and all CTAs leave together at the next cluster barrier.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

constexpr int kWS = kWideLanes;  // lanes
constexpr int kWNW = 8;     // warps per CTA
constexpr int kWNT = kWNW * 32;
constexpr int kWJ = 128;    // target states per cluster
constexpr int kWCH = 32;    // rows per argmax chunk
constexpr int kWNST = 4;    // cp.async ring stages per warp (4 rows each)
constexpr int kWSmemMax = 232448 - 4096;  // dynamic shared memory budget (static part kept aside)
constexpr long long kWWaitCycles = 1ll << 31;  // ~1 s at 2 GHz

struct WJob {
  int32_t b, m, n, T, Pe, q_prev, q_n, par;
  float s_prev;
  int32_t pad;
  int64_t e_off, path_off, aux_off;
};

struct WLane {
  int32_t k, state, t, term;  // state: 0 load next job, 1 running, 2 no more jobs
  int32_t kdiv, ediv, eprev, tmid;
  WJob cur, old;
};

struct __align__(16) WDesc {
  int32_t mode;    // 0 idle, 1 first step of the job, 2 max-plus step
  int32_t first;   // t == 0
  int32_t f_mid;   // 0 none, 1 MidState = psi, 2 MidState = MidState_prev[psi]
  int32_t f_snap;  // root: snapshot (+ map); sub: snapshot at t_mid
  int32_t q_prev, par, sym, pad;
  float s_prev;
  int32_t pad2;
  int64_t psi_row, snap_row, map_row;
  const float* erow;
};

__device__ __forceinline__ void wfadd2_max3(float& acc, unsigned long long d, unsigned long long a) {
  asm("{\n\t.reg .b64 c;\n\t.reg .f32 lo, hi;\n\tadd.rn.f32x2 c, %1, %2;\n\tmov.b64 {lo, hi}, c;\n\t"
      "max.f32 %0, %0, lo, hi;\n\t}"
      : "+f"(acc)
      : "l"(d), "l"(a));
}
__device__ __forceinline__ void wfadd2(unsigned long long d, unsigned long long a, float& c0, float& c1) {
  unsigned long long c;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(c) : "l"(d), "l"(a));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(c));
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__host__ __device__ inline int32_t wpe(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
__host__ __device__ inline int32_t wdiv(int32_t k, int32_t T, int32_t Pe) {
  return (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
}

bool wide_geometry(int K, int nsm, WideGeom* g) {
  if (K <= 1024) return false;
  g->NCB = (K + kWJ - 1) / kWJ;
  // clusters must fit inside GPCs: at most 16 of 8 CTAs or 32 of 4 CTAs
  // are co-resident on a 152-SM part
  if (g->NCB <= 16 && g->NCB * 8 <= nsm) g->CR = 8;
  else if (g->NCB <= 32 && g->NCB * 4 <= nsm) g->CR = 4;
  else return false;
  const int gran = g->CR * kWNW * kWCH;
  g->KR = (K + gran - 1) / gran * gran;
  g->RPC = g->KR / g->CR;
  g->RPW = g->RPC / kWNW;
  const size_t sD = sizeof(float) * (size_t)kWS * (g->RPC + g->RPC / 8);
  const size_t sMid = sizeof(uint16_t) * (size_t)kWS * g->RPC;
  const size_t ring = sizeof(float2) * (size_t)kWNW * kWNST * 2 * kWJ;
  const size_t recv = 2 * sizeof(float) * 2 * (size_t)kWS * kWJ;
  const size_t fixed = sD + sMid + ring + recv;
  if (fixed + 4096 > (size_t)kWSmemMax) return false;
  int rwr = (int)((kWSmemMax - fixed) / ((size_t)kWNW * kWJ * sizeof(float)));
  rwr &= ~3;
  if (rwr > g->RPW) rwr = g->RPW;
  if (rwr < 0) rwr = 0;
  g->RWR = rwr;
  g->smem = fixed + sizeof(float) * (size_t)kWNW * rwr * kWJ;
  g->G = g->NCB * g->CR;
  return true;
}

size_t wide_scratch_bytes(int K, int nsm) {
  // delta and MidState double buffers, sub snapshots (job parity), flags
  return align_up(2 * sizeof(float) * (size_t)kWS * K) + align_up(2 * sizeof(uint16_t) * (size_t)kWS * K) +
         align_up(2 * sizeof(float) * (size_t)kWS * K) + align_up(sizeof(uint32_t) * 8 * (size_t)(nsm + 1));
}

template <int CR>
__global__ void __launch_bounds__(kWNT, 1) wide_fwd_kernel(DenseArgs a, WideGeom g) {
  constexpr int JO = kWJ / CR;  // targets owned per CTA
  extern __shared__ __align__(16) float smem[];
  __shared__ WLane lanes[kWS];
  __shared__ WDesc wdesc[kWS];
  __shared__ int s_njobs, s_abort_local;
  __shared__ uint32_t s_abort[2][CR];

  if (a.hdr->status != 0) return;  // uniform: no CTA has started any wait

  const int K = a.K, RPC = g.RPC, RPW = g.RPW, RWR = g.RWR, RPCS = RPC + RPC / 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_ctarank();
  const int cl = blockIdx.x / CR;
  const int j0 = cl * kWJ;
  const int row0 = (int)rank * RPC;
  const int kind = a.kind;
  const int64_t SK = (int64_t)kWS * K;

  float* sD = smem;                                                        // [S][RPCS] skewed rows
  uint16_t* sMid = reinterpret_cast<uint16_t*>(sD + kWS * RPCS);           // [S][RPC]
  float2* sRing = reinterpret_cast<float2*>(sMid + kWS * RPC);             // [NW][NST][2][J]
  float* sRV = reinterpret_cast<float*>(sRing + kWNW * kWNST * 2 * kWJ);   // [2][CR][S][JO]
  uint32_t* sRI = reinterpret_cast<uint32_t*>(sRV + 2 * kWS * kWJ);        // [2][CR][S][JO]
  float2* sA = reinterpret_cast<float2*>(sRI + 2 * kWS * kWJ);             // [NW][RWR/2][J]

  // resident logA rows of every warp, from the row-pair copy
  for (int w = 0; w < kWNW; ++w) {
    const int np = RWR / 2;
    const float2* src = a.Ap + (int64_t)((row0 + w * RPW) / 2) * a.ap_stride + j0;
    float2* dst = sA + (size_t)w * np * kWJ;
    for (int x = tid; x < np * kWJ; x += kWNT) dst[x] = src[(int64_t)(x / kWJ) * a.ap_stride + (x % kWJ)];
  }
  if (tid < kWS) {
    lanes[tid].k = 0;
    lanes[tid].state = 0;
    lanes[tid].term = 0;
  }
  if (tid == 0) s_njobs = kind == kJobSub ? *a.task_count : a.order_count;
  if (tid < 2 * CR) s_abort[tid / CR][tid % CR] = 0;
  // producers of this CTA's rows: every CTA of the clusters covering them
  const int rows_hi = row0 + RPC < K ? row0 + RPC : K;
  const int c_lo = row0 / kWJ, c_hi = rows_hi > row0 ? (rows_hi - 1) / kWJ : -1;
  const int nprod = c_hi >= c_lo ? (c_hi - c_lo + 1) * CR : 0;
  cluster_sync_all();

  uint32_t tau = 0;
  for (;;) {
    const int cur = tau & 1, nxt = cur ^ 1;
    // ---- prologue: lane state machine (identical in every CTA)
    if (tid == 0) s_abort_local = 0;
    if (tid < kWS) {
      WLane& L = lanes[tid];
      L.term = 0;
      if (L.state == 1 && L.t > L.cur.n) {
        L.term = 1;
        L.old = L.cur;
        L.state = 0;
        L.k += 1;
      }
      if (L.state == 0) {
        const int gi = tid + kWS * L.k;
        if (gi < s_njobs) {
          WJob j;
          j.pad = 0;
          j.q_prev = j.q_n = 0;
          j.s_prev = 0.f;
          j.par = L.k & 1;
          if (kind != kJobSub) {
            const int b = a.order[a.order_begin + gi];
            const Job jb = a.jobs[b];
            j.b = b;
            j.m = 0;
            j.n = jb.T - 1;
            j.T = jb.T;
            j.e_off = jb.e_off;
            j.path_off = jb.path_off;
            j.aux_off = jb.aux_off;
          } else {
            const Task tk = a.tasks[gi];
            const Job jb = a.jobs[tk.b];
            j.b = tk.b;
            j.m = tk.m;
            j.n = tk.n;
            j.T = jb.T;
            j.e_off = jb.e_off;
            j.path_off = jb.path_off;
            j.aux_off = jb.aux_off;
            const int qn = a.paths[jb.path_off + tk.n];
            j.q_n = (unsigned)qn < (unsigned)K ? qn : 0;
            if (tk.m > 0) {
              const int qp = a.paths[jb.path_off + tk.m - 1];
              j.q_prev = (unsigned)qp < (unsigned)K ? qp : 0;
              j.s_prev = a.sval[jb.aux_off + tk.m - 1];
            }
          }
          j.Pe = wpe(j.T, a.P);
          L.cur = j;
          L.state = 1;
          L.t = j.m;
          L.kdiv = 0;
          L.ediv = wdiv(0, j.T, j.Pe);
          L.eprev = -1;
          L.tmid = (j.m + j.n) / 2;
        } else {
          L.state = 2;
        }
      }
      WDesc d;
      d.mode = d.first = d.f_mid = d.f_snap = d.q_prev = d.par = d.sym = d.pad = d.pad2 = 0;
      d.s_prev = 0.f;
      d.psi_row = d.snap_row = 0;
      d.map_row = -1;
      d.erow = nullptr;
      if (L.state == 1) {
        const int t = L.t;
        const WJob& jb = L.cur;
        d.mode = (t == jb.m) ? 1 : 2;
        d.first = (t == 0);
        d.q_prev = jb.q_prev;
        d.s_prev = jb.s_prev;
        d.par = jb.par;
        d.psi_row = jb.aux_off + (int64_t)t * K;
        if (a.emit == FV_EMIT_DENSE) d.erow = a.E + jb.e_off + (int64_t)t * K;
        else d.sym = __ldg(a.obs + jb.e_off + t);
        if (kind == kJobRoot) {
          const int is_div = (t == L.ediv);
          if (L.eprev >= 0) d.f_mid = (t == L.eprev + 1) ? 1 : 2;
          d.f_snap = is_div;
          d.snap_row = (int64_t)jb.b * a.snap_stride + (int64_t)L.kdiv * K;
          d.map_row = (is_div && L.kdiv >= 1) ? (int64_t)jb.b * a.map_stride + (int64_t)(L.kdiv - 1) * K : -1;
        } else if (kind == kJobSub) {
          d.f_mid = (t == L.tmid + 1) ? 1 : (t > L.tmid + 1 ? 2 : 0);
          d.f_snap = (t == L.tmid);
        }
      }
      wdesc[tid] = d;
    }
    const int live = (tid < kWS) && (lanes[tid].state != 2 || lanes[tid].term);
    if (!__syncthreads_or(live)) break;
    const int any_term = __syncthreads_or(tid < kWS && lanes[tid].term);

    // ---- owner-side prefetch of E_t (and the start terms of first steps)
    const int os = tid / JO, ol = tid % JO, oj = j0 + (int)rank * JO + ol;
    float ev = 0.f, pv = 0.f, av = 0.f;
    if (tid < kWS * JO) {
      const WDesc& d = wdesc[os];
      if (d.mode && oj < K) {
        ev = a.emit == FV_EMIT_DENSE ? __ldg(d.erow + oj) : __ldg(a.logB + (int64_t)oj * a.V + d.sym);
        if (d.mode == 1) {
          if (d.first) pv = __ldg(a.log_pi + oj);
          else av = __ldg(a.logA + (int64_t)d.q_prev * K + oj);
        }
      }
    }

    // ---- wait for the owners of this CTA's rows (all CTAs when CTA 0 must
    // read whole delta rows to finish jobs)
    if (tau > 0) {
      const bool all = (blockIdx.x == 0) && any_term;
      const int nw = all ? (int)gridDim.x : nprod;
      if (tid < nw) {
        const int p = all ? tid : (c_lo + tid / CR) * CR + tid % CR;
        const uint32_t* f = a.wide_flags + (size_t)p * 8;
        const long long t0 = clock64();
        int bad = 0, spins = 0;
        while (ld_acquire_u32(f) < tau) {
          if (++spins > 64) {
            spins = 0;
            if (*reinterpret_cast<volatile uint32_t*>(&a.hdr->status) != 0) { bad = 2; break; }
            if (clock64() - t0 > kWWaitCycles) { bad = 1; break; }
          }
        }
        __threadfence();
        if (bad == 1) set_status(a.hdr, FV_ETIMEOUT, 0x57000000u | (uint32_t)blockIdx.x);
        if (bad) s_abort_local = 1;
      }
    }
    __syncthreads();
    const int abort_local = s_abort_local;

    if (!abort_local) {
      // ---- termination of jobs that ended last step (CTA 0)
      if (blockIdx.x == 0 && any_term) {
        const int s = warp;  // kWNW == kWS
        if (lanes[s].term) {
          const WJob& jb = lanes[s].old;
          const float* dl = a.wide_D + cur * SK + (int64_t)s * K;
          if (kind == kJobVanilla) {
            float bv = -CUDART_INF_F;
            int bi = 0x7fffffff;
            for (int j = lane; j < K; j += 32) {
              const float v = dl[j];
              if (bi == 0x7fffffff || v > bv) { bv = v; bi = j; }
            }
            for (int o = 16; o > 0; o >>= 1) {
              const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
              const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
              if (oi != 0x7fffffff && (bi == 0x7fffffff || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
            }
            if (lane == 0) {
              a.qlast[jb.b] = bi;
              a.scores[jb.b] = dl[bi];
            }
          } else if (kind == kJobSub && lane == 0) {
            const int tmid = (jb.m + jb.n) / 2;
            int q = a.wide_M[cur * SK + (int64_t)s * K + jb.q_n];
            q = (unsigned)q < (unsigned)K ? q : 0;
            a.paths[jb.path_off + tmid] = q;
            a.sval[jb.aux_off + tmid] = a.wide_X[(int64_t)jb.par * SK + (int64_t)s * K + q];
          }
        }
      }
      // ---- delta_{t-1} (and MidState_{t-1}) of this CTA's rows
      for (int s = 0; s < kWS; ++s) {
        const WDesc& d = wdesc[s];
        if (d.mode != 2) continue;
        const float* src = a.wide_D + cur * SK + (int64_t)s * K;
        float* dst = sD + s * RPCS;
        for (int x = tid; x < RPC; x += kWNT) {
          const int i = row0 + x;
          dst[x + ((x >> 5) << 2)] = i < K ? src[i] : -CUDART_INF_F;
        }
        if (d.f_mid == 2) {
          const uint16_t* ms = a.wide_M + cur * SK + (int64_t)s * K;
          for (int x = tid; x < RPC; x += kWNT) {
            const int i = row0 + x;
            sMid[s * RPC + x] = i < K ? ms[i] : (uint16_t)0;
          }
        }
      }
      __syncthreads();

      // ---- main loop: value-only tropical product over this warp's RPW
      // rows; a lane covers 4 lanes x 8 targets.  Rows [0, RWR) of the
      // warp's slice come from shared memory, the rest stream through the
      // warp's cp.async ring.
      {
        const int sg = lane >> 4, jg = lane & 15;
        float acc[4][8], bst[4][8];
        int bch[4][8];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            acc[x][y] = -CUDART_INF_F;
            bst[x][y] = -CUDART_INF_F;
            bch[x][y] = 0;
          }
        const int lr0 = warp * RPW;
        const float* dlanes = sD + (sg * 4) * RPCS;
        auto quad = [&](int lr, const float2* abase) {
          const float* dbase = dlanes + lr + ((lr >> 5) << 2);
          ulonglong2 dq[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) dq[x] = *reinterpret_cast<const ulonglong2*>(dbase + x * RPCS);
          ulonglong2 aq[2][4];
#pragma unroll
          for (int pr = 0; pr < 2; ++pr)
#pragma unroll
            for (int gq = 0; gq < 4; ++gq)
              aq[pr][gq] = *reinterpret_cast<const ulonglong2*>(abase + pr * kWJ + 32 * gq);
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int gq = 0; gq < 4; ++gq) {
              wfadd2_max3(acc[x][2 * gq], dq[x].x, aq[0][gq].x);
              wfadd2_max3(acc[x][2 * gq], dq[x].y, aq[1][gq].x);
              wfadd2_max3(acc[x][2 * gq + 1], dq[x].x, aq[0][gq].y);
              wfadd2_max3(acc[x][2 * gq + 1], dq[x].y, aq[1][gq].y);
            }
          if (((lr + 4) & (kWCH - 1)) == 0) {
            const int c = lr / kWCH;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 8; ++y) {
                if (acc[x][y] > bst[x][y]) { bst[x][y] = acc[x][y]; bch[x][y] = c; }
                acc[x][y] = -CUDART_INF_F;
              }
          }
        };
        const float2* aw = sA + (size_t)warp * (RWR / 2) * kWJ + 2 * jg;
#pragma unroll 1
        for (int q = 0; q < RWR / 4; ++q) quad(lr0 + 4 * q, aw + (2 * q) * kWJ);
        float2* ring = sRing + warp * kWNST * 2 * kWJ;
        const int NIT = (RPW - RWR) / 4;
        const float2* gsrc = a.Ap + (int64_t)((row0 + lr0 + RWR) / 2) * a.ap_stride + j0;
        auto issue = [&](int it) {
          float2* dst = ring + (it % kWNST) * 2 * kWJ;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int qq = lane + 32 * u, pr = qq / (kWJ / 2), c2 = (qq % (kWJ / 2)) * 2;
            cp_async16(dst + pr * kWJ + c2, gsrc + (int64_t)(2 * it + pr) * a.ap_stride + c2);
          }
        };
#pragma unroll
        for (int k2 = 0; k2 < kWNST - 1; ++k2) {
          if (k2 < NIT) issue(k2);
          cp_async_commit();
        }
#pragma unroll 1
        for (int it = 0; it < NIT; ++it) {
          cp_async_wait<kWNST - 2>();
          __syncwarp();
          if (it + kWNST - 1 < NIT) issue(it + kWNST - 1);
          cp_async_commit();
          quad(lr0 + RWR + 4 * it, ring + (it % kWNST) * 2 * kWJ + 2 * jg);
        }
        cp_async_wait<0>();
        __syncwarp();
        // per-warp partials into the warp's own ring
        float* pvw = reinterpret_cast<float*>(ring);
        uint8_t* pcw = reinterpret_cast<uint8_t*>(pvw + kWS * kWJ);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int s = sg * 4 + x;
#pragma unroll
          for (int gq = 0; gq < 4; ++gq) {
            const int c = 2 * jg + 32 * gq;
            *reinterpret_cast<float2*>(pvw + s * kWJ + c) = make_float2(bst[x][2 * gq], bst[x][2 * gq + 1]);
            pcw[s * kWJ + c] = (uint8_t)bch[x][2 * gq];
            pcw[s * kWJ + c + 1] = (uint8_t)bch[x][2 * gq + 1];
          }
        }
      }
      __syncthreads();

      // ---- merge over warps, exact re-scan of the winning chunk, send
      // (value, row, ancestor) to the target's owner
      {
        const int jj = tid % kWJ, s0 = tid / kWJ;
        const int orank = jj / JO, ojl = jj % JO;
#pragma unroll 1
        for (int s = s0; s < kWS; s += kWNT / kWJ) {
          const WDesc& d = wdesc[s];
          if (d.mode != 2) continue;
          float bv = -CUDART_INF_F;
          int wb = 0;
#pragma unroll
          for (int w = 0; w < kWNW; ++w) {
            const float* pvw = reinterpret_cast<const float*>(sRing + w * kWNST * 2 * kWJ);
            const uint8_t* pcw = reinterpret_cast<const uint8_t*>(pvw + kWS * kWJ);
            const float v = pvw[s * kWJ + jj];
            if (w == 0 || v > bv) { bv = v; wb = pcw[s * kWJ + jj]; }
          }
          const int cb = wb * kWCH;  // first local row of the chunk
          const float* dr = sD + s * RPCS + cb + ((cb >> 5) << 2);
          const unsigned long long* ar =
              reinterpret_cast<const unsigned long long*>(a.Ap + (int64_t)((row0 + cb) / 2) * a.ap_stride + j0 + jj);
          unsigned long long avv[kWCH / 2];
#pragma unroll
          for (int k2 = 0; k2 < kWCH / 2; ++k2) avv[k2] = __ldg(ar + (int64_t)k2 * a.ap_stride);
          int arg = cb;
          float val = bv;
#pragma unroll
          for (int k2 = kWCH / 2 - 1; k2 >= 0; --k2) {
            float c0, c1;
            wfadd2(*reinterpret_cast<const unsigned long long*>(dr + 2 * k2), avv[k2], c0, c1);
            if (c1 == bv) { arg = cb + 2 * k2 + 1; val = c1; }
            if (c0 == bv) { arg = cb + 2 * k2; val = c0; }
          }
          const uint32_t m16 = d.f_mid == 2 ? (uint32_t)sMid[s * RPC + arg] : 0u;
          const uint32_t im = (uint32_t)(row0 + arg) | (m16 << 16);
          const int off = ((cur * CR + (int)rank) * kWS + s) * JO + ojl;
          if (orank == (int)rank) {
            sRV[off] = val;
            sRI[off] = im;
          } else {
            dsmem_st_f32(dsmem_addr(sRV + off, orank), val);
            dsmem_st_u32(dsmem_addr(sRI + off, orank), im);
          }
        }
      }
    }
    // ---- cluster barrier; every CTA of the cluster sees the same abort bit
    if (tid < CR) dsmem_st_u32(dsmem_addr(&s_abort[cur][rank], tid), (uint32_t)abort_local);
    cluster_arrive_release();
    cluster_wait_acquire();
    uint32_t abort_any = 0;
#pragma unroll
    for (int rr = 0; rr < CR; ++rr) abort_any |= s_abort[cur][rr];
    if (abort_any) break;

    // ---- owners: lowest rank holding the maximum, + E_t, stores
    if (tid < kWS * JO) {
      const WDesc& d = wdesc[os];
      if (d.mode && oj < K) {
        float dval;
        uint32_t mnew = 0;
        if (d.mode == 1) {
          if (d.first) dval = __fadd_rn(pv, ev);
          else dval = a.complete ? __fadd_rn(av, ev) : __fadd_rn(__fadd_rn(d.s_prev, av), ev);
        } else {
          int base = (cur * CR * kWS + os) * JO + ol;
          float bv = sRV[base];
          uint32_t bi = sRI[base];
#pragma unroll
          for (int rr = 1; rr < CR; ++rr) {
            const float v = sRV[base + rr * kWS * JO];
            if (v > bv) { bv = v; bi = sRI[base + rr * kWS * JO]; }
          }
          const uint32_t ag = bi & 0xffffu;
          dval = __fadd_rn(bv, ev);
          if (kind == kJobVanilla) a.psi[d.psi_row + oj] = (uint16_t)ag;
          if (d.f_mid) {
            mnew = d.f_mid == 1 ? ag : (bi >> 16);
            a.wide_M[nxt * SK + (int64_t)os * K + oj] = (uint16_t)mnew;
          }
        }
        if (d.f_snap) {
          if (kind == kJobRoot) {
            a.snaps[d.snap_row + oj] = dval;
            if (d.map_row >= 0) a.maps[d.map_row + oj] = (uint16_t)mnew;
          } else {
            a.wide_X[(int64_t)d.par * SK + (int64_t)os * K + oj] = dval;
          }
        }
        a.wide_D[nxt * SK + (int64_t)os * K + oj] = dval;
      }
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release_u32(a.wide_flags + (size_t)blockIdx.x * 8, tau + 1);
    }
    if (tid < kWS) {
      WLane& L = lanes[tid];
      if (L.state == 1) {
        if (kind == kJobRoot && L.t == L.ediv) {
          L.eprev = L.ediv;
          L.kdiv += 1;
          L.ediv = L.kdiv < L.cur.Pe ? wdiv(L.kdiv, L.cur.T, L.cur.Pe) : 0x7fffffff;
        }
        L.t += 1;
      }
    }
    ++tau;
  }
  cluster_sync_all();  // no CTA leaves while a peer may still write into its shared memory
}

cudaError_t launch_wide_forward(DenseArgs a, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  WideGeom g;
  if (!wide_geometry(a.K, nsm, &g)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.wide_flags, 0, sizeof(uint32_t) * 8 * (size_t)g.G, st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g.CR;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.gridDim = dim3(g.G);
  cfg.blockDim = dim3(kWNT);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e2 != cudaSuccess) return e2;
    int resident = 0;
    cudaLaunchConfig_t q = cfg;
    q.numAttrs = 1;  // occupancy query: cluster shape only
    e2 = cudaOccupancyMaxActiveClusters(&resident, kern, &q);
    if (e2 != cudaSuccess) return e2;
    if (resident < g.NCB) return cudaErrorCooperativeLaunchTooLarge;  // all CTAs must be co-resident
    return cudaLaunchKernelEx(&cfg, kern, a, g);
  };
  if (g.CR == 8) return run(wide_fwd_kernel<8>);
  return run(wide_fwd_kernel<4>);
}

}  // namespace fv
