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
// rows per argmax chunk (measured: 16 beats 32 by 1-4% and 8 at K=4096;
// the owners re-scan one chunk per output from L2)
constexpr int kWCH = 16;
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
// L2 policy: a fraction of the lines gets evict_last priority, the rest
// keep their normal priority (a streamed logA larger than L2 would otherwise
// evict itself every step).
__device__ __forceinline__ uint64_t l2_keep_policy(float frac) {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_unchanged.b64 %0, %1;" : "=l"(p) : "f"(frac));
  return p;
}
__device__ __forceinline__ void cp_async16_keep(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "l"(pol)
               : "memory");
}
// Bytes of logA the whole grid streams per step, and the share of them to
// keep in L2 (about 48 MB of a 126 MB L2 is left to the rest of the step).
float wide_l2_keep(const WideGeom& g) {
  const double streamed = (double)g.G * kWNW * (g.RPW - g.RWR) * kWJ * sizeof(float);
  if (streamed <= 0) return 1.f;
  const double f = 48.0e6 / streamed;
  return f >= 1.0 ? 1.f : (float)f;
}

__host__ __device__ inline int32_t wpe(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
__host__ __device__ inline int32_t wdiv(int32_t k, int32_t T, int32_t Pe) {
  return (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
}

template <int CR>
__global__ void wide_fwd_kernel(DenseArgs a, WideGeom g);

// Clusters of CR CTAs (one CTA per SM) that can be resident at once: a
// cluster must fit inside one GPC, so this is below nsm / CR.  Queried once
// per process; without a usable device the plain bound nsm / CR is used.
static int max_wide_clusters(int CR, int nsm) {
  static int cache[3] = {-1, -1, -1};
  const int slot = CR == 2 ? 0 : (CR == 4 ? 1 : 2);
  if (cache[slot] >= 0) return cache[slot];
  int n = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CR;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CR * nsm);
  cfg.blockDim = dim3(kWNW * 32);
  cfg.dynamicSmemBytes = kWSmemMax;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  if (CR == 2) {
    e = cudaFuncSetAttribute(wide_fwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemMax);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, wide_fwd_kernel<2>, &cfg);
  } else if (CR == 4) {
    e = cudaFuncSetAttribute(wide_fwd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemMax);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, wide_fwd_kernel<4>, &cfg);
  } else {
    e = cudaFuncSetAttribute(wide_fwd_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemMax);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, wide_fwd_kernel<8>, &cfg);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    n = nsm / CR;
  }
  cache[slot] = n;
  return n;
}

bool wide_geometry(int K, int nsm, WideGeom* g) {
  if (K <= 1024) return false;
  g->NCB = (K + kWJ - 1) / kWJ;
  // the largest cluster size whose clusters can all be co-resident
  if (g->NCB <= max_wide_clusters(8, nsm)) g->CR = 8;
  else if (g->NCB <= max_wide_clusters(4, nsm)) g->CR = 4;
  else if (g->NCB <= max_wide_clusters(2, nsm)) g->CR = 2;
  else return false;
  const int gran = g->CR * kWNW * kWCH;
  g->KR = (K + gran - 1) / gran * gran;
  g->RPC = g->KR / g->CR;
  g->RPW = g->RPC / kWNW;
  const size_t sD = sizeof(float) * (size_t)kWS * (g->RPC + g->RPC / 8);
  const size_t ring = sizeof(float2) * (size_t)kWNW * kWNST * 2 * kWJ;
  const size_t recv = 2 * sizeof(float) * 2 * (size_t)kWS * kWJ;
  const size_t fixed = sD + ring + recv;
  if (fixed + 4096 > (size_t)kWSmemMax) return false;
  int rwr = (int)((kWSmemMax - fixed) / ((size_t)kWNW * kWJ * sizeof(float)));
  rwr &= ~3;
  if (rwr > g->RPW) rwr = g->RPW;
  if (rwr < 0) rwr = 0;
  g->RWR = rwr;
  g->smem = fixed + sizeof(float) * (size_t)kWNW * rwr * kWJ;
  g->G = g->NCB * g->CR;
  g->l2_keep = wide_l2_keep(*g);
  return true;
}

size_t wide_scratch_bytes(int K, int nsm) {
  // delta and MidState double buffers, sub snapshots (job parity), flags,
  // and the column-major copy of logA read by the owners' re-scan
  const size_t lk = (size_t)kWS * wide_lane_stride(K);
  return align_up(2 * sizeof(float) * lk) + align_up(2 * sizeof(uint16_t) * lk) + align_up(2 * sizeof(float) * lk) +
         align_up(sizeof(uint32_t) * 8 * (size_t)(nsm + 1)) +
         align_up(sizeof(float) * (size_t)K * wide_lane_stride(K));
}

// 32 x 32 tiles through shared memory, so both sides are coalesced.
__global__ void wide_transpose_kernel(const float* logA, int K, int KD, float* AT) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < K && j < K) ? logA[(int64_t)i * K + j] : -CUDART_INF_F;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < K && i < KD) AT[(int64_t)j * KD + i] = tile[threadIdx.x][r];
  }
}

cudaError_t launch_wide_transpose(const float* logA, int K, float* AT, cudaStream_t st) {
  const int KD = wide_lane_stride(K);
  wide_transpose_kernel<<<dim3((K + 31) / 32, (KD + 31) / 32), dim3(32, 8), 0, st>>>(logA, K, KD, AT);
  return cudaGetLastError();
}

template <int CR>
__global__ void __launch_bounds__(kWNT, 1) wide_fwd_kernel(DenseArgs a, WideGeom g) {
  static_assert(CR == 2 || CR == 4 || CR == 8, "cluster sizes 2, 4, 8");
  constexpr int JO = kWJ / CR;  // targets owned per CTA
  constexpr int OPW = (kWS * JO + kWNT - 1) / kWNT;  // owned outputs per thread
  extern __shared__ __align__(16) float smem[];
  __shared__ WLane lanes[kWS];
  __shared__ WDesc wdesc[kWS];
  __shared__ int s_njobs, s_abort_local;
  __shared__ uint32_t s_abort[2][CR];

  // the launch must have exactly the planned shape (every index below
  // depends on it); gridDim and the cluster size are the same in every CTA
  if (gridDim.x != (unsigned)g.G || cluster_nctarank() != (unsigned)CR) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(a.hdr, FV_EUNSUPPORTED, 0x57100000u);
    return;
  }

  const int K = a.K, RPC = g.RPC, RPW = g.RPW, RWR = g.RWR, RPCS = RPC + RPC / 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_ctarank();
  const int cl = blockIdx.x / CR;
  const int j0 = cl * kWJ;
  const int row0 = (int)rank * RPC;
  const int kind = a.kind;
  const int KD = wide_lane_stride(K);  // lane stride of the global rows
  const uint64_t pol = l2_keep_policy(g.l2_keep);
  const int64_t SK = (int64_t)kWS * KD;

  float* sD = smem;                                                        // [S][RPCS] skewed rows
  float2* sRing = reinterpret_cast<float2*>(sD + kWS * RPCS);              // [NW][NST][2][J]
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
  const bool from_tasks = kind == kJobSub || kind == kJobLeaf;
  const int task0 = from_tasks && a.task_first ? *a.task_first : 0;
  if (tid == 0) s_njobs = from_tasks ? *a.task_count : a.order_count;
  if (tid < 2 * CR) s_abort[tid / CR][tid % CR] = 0;
  // producers of this CTA's rows: every CTA of the clusters covering them
  const int rows_hi = row0 + RPC < K ? row0 + RPC : K;
  const int c_lo = row0 / kWJ, c_hi = rows_hi > row0 ? (rows_hi - 1) / kWJ : -1;
  const int nprod = c_hi >= c_lo ? (c_hi - c_lo + 1) * CR : 0;
  cluster_sync_all();
  // an earlier kernel may have recorded an error: every CTA of the cluster
  // takes the same decision (the OR of what each of them read)
  if (tid < CR) dsmem_st_u32(dsmem_addr(&s_abort[1][rank], tid), a.hdr->status != 0 ? 1u : 0u);
  cluster_sync_all();
  {
    uint32_t bad = 0;
#pragma unroll
    for (int rr = 0; rr < CR; ++rr) bad |= s_abort[1][rr];
    if (bad) return;  // no peer touches this CTA's shared memory any more
  }

  // this warp's streamed logA rows (the same every step) and its ring
  float2* ring = sRing + warp * kWNST * 2 * kWJ;
  const int NIT = (RPW - RWR) / 4;
  const float2* gsrc = a.Ap + (int64_t)((row0 + warp * RPW + RWR) / 2) * a.ap_stride + j0;
  auto issue = [&](int it) {
    float2* dst = ring + (it % kWNST) * 2 * kWJ;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int qq = lane + 32 * u, pr = qq / (kWJ / 2), c2 = (qq % (kWJ / 2)) * 2;
      cp_async16_keep(dst + pr * kWJ + c2, gsrc + (int64_t)(2 * it + pr) * a.ap_stride + c2, pol);
    }
  };
  // the first kWNST-1 stages of a step, one commit group each
  auto prefetch_ring = [&]() {
#pragma unroll
    for (int k2 = 0; k2 < kWNST - 1; ++k2) {
      if (k2 < NIT) issue(k2);
      cp_async_commit();
    }
  };
  bool ring_ready = false;

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
          if (!from_tasks) {
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
            const Task tk = a.tasks[task0 + gi];
            const Job jb = a.jobs[tk.b];
            j.b = tk.b;
            j.m = tk.m;
            j.n = tk.n;
            j.T = jb.T;
            j.e_off = jb.e_off;
            j.path_off = jb.path_off;
            j.aux_off = jb.aux_off;
            j.pad = tk.pad;
            if (!a.ckpt) {
              const int qn = a.paths[jb.path_off + tk.n];
              j.q_n = (unsigned)qn < (unsigned)K ? qn : 0;
              if (tk.m > 0) {
                const int qp = a.paths[jb.path_off + tk.m - 1];
                j.q_prev = (unsigned)qp < (unsigned)K ? qp : 0;
                j.s_prev = a.sval[jb.aux_off + tk.m - 1];
              }
            }
          }
          j.Pe = a.ckpt ? ckpt_count(j.T, a.P) : wpe(j.T, a.P);
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
        d.psi_row = kind != kJobLeaf ? jb.aux_off + (int64_t)t * K
                    : a.ckpt ? 2 * (jb.aux_off + (int64_t)jb.Pe * K) + (int64_t)(t - jb.m - 1) * K
                             : (int64_t)(jb.pad + t - jb.m - 1) * K;
        if (a.emit == FV_EMIT_DENSE) d.erow = a.E + jb.e_off + (int64_t)t * K;
        else d.sym = __ldg(a.obs + jb.e_off + t);
        if (kind == kJobRoot) {
          const int is_div = (t == L.ediv);
          d.f_snap = is_div;
          if (a.ckpt) {
            // checkpoints only: delta_t at division point kdiv
            d.snap_row = jb.aux_off + (int64_t)L.kdiv * K;
          } else {
            if (L.eprev >= 0) d.f_mid = (t == L.eprev + 1) ? 1 : 2;
            d.snap_row = (int64_t)jb.b * a.snap_stride + (int64_t)L.kdiv * K;
            d.map_row = (is_div && L.kdiv >= 1) ? (int64_t)jb.b * a.map_stride + (int64_t)(L.kdiv - 1) * K : -1;
          }
        } else if (kind == kJobLeaf && a.ckpt && jb.pad >= 0) {
          // checkpoint segment: the restart reads checkpoint jb.pad
          d.snap_row = jb.aux_off + (int64_t)jb.pad * K;
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

    // ---- owner-side prefetch of E_t (and the start terms of first steps);
    // output o = tid + kWNT * u of this CTA is (lane o / JO, target o % JO)
    float ev[OPW], pv[OPW], av[OPW];
#pragma unroll
    for (int u = 0; u < OPW; ++u) {
      const int o = tid + kWNT * u, os = o / JO, oj = j0 + (int)rank * JO + o % JO;
      ev[u] = pv[u] = av[u] = 0.f;
      if (o < kWS * JO) {
        const WDesc& d = wdesc[os];
        if (d.mode && oj < K) {
          ev[u] = a.emit == FV_EMIT_DENSE ? __ldg(d.erow + oj) : __ldg(a.logB + (int64_t)oj * a.V + d.sym);
          if (d.mode == 1) {
            if (d.first) pv[u] = __ldg(a.log_pi + oj);
            else if (a.ckpt) av[u] = __ldg(a.snaps + d.snap_row + oj);  // checkpoint restart value
            else av[u] = __ldg(a.logA + (int64_t)d.q_prev * K + oj);
          }
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
          const float* dl = a.wide_D + cur * SK + (int64_t)s * KD;
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
            int q = a.wide_M[cur * SK + (int64_t)s * KD + jb.q_n];
            q = (unsigned)q < (unsigned)K ? q : 0;
            a.paths[jb.path_off + tmid] = q;
            a.sval[jb.aux_off + tmid] = a.wide_X[(int64_t)jb.par * SK + (int64_t)s * KD + q];
          }
        }
      }
      // ---- delta_{t-1} of this CTA's rows, 16-byte asynchronous copies
      // into the skewed layout (-inf beyond K)
      for (int s = 0; s < kWS; ++s) {
        if (wdesc[s].mode != 2) continue;
        const float* src = a.wide_D + cur * SK + (int64_t)s * KD + row0;
        float* dst = sD + s * RPCS;
        for (int x4 = tid * 4; x4 < RPC; x4 += kWNT * 4) {
          float* dp = dst + x4 + ((x4 >> 5) << 2);
          if (row0 + x4 + 3 < K) {
            cp_async16(dp, src + x4);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) dp[u] = row0 + x4 + u < K ? src[x4 + u] : -CUDART_INF_F;
          }
        }
      }
      cp_async_commit();
      cp_async_wait<0>();
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
        // 4 rows x (4 lanes x 8 targets); no chunk bookkeeping
        auto quad_math = [&](int lr, const float2* abase) {
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
        };
        // end of chunk c: acc is the running maximum over the rows so far,
        // so a chunk that raised it holds the first row reaching the new
        // maximum
        auto track = [&](int c) {
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) {
              if (acc[x][y] > bst[x][y]) bch[x][y] = c;
              bst[x][y] = acc[x][y];
            }
        };
        auto quad = [&](int lr, const float2* abase) {
          quad_math(lr, abase);
          if (((lr + 4) & (kWCH - 1)) == 0) track(lr / kWCH);
        };
        const float2* aw = sA + (size_t)warp * (RWR / 2) * kWJ + 2 * jg;
#pragma unroll 1
        for (int q = 0; q < RWR / 4; ++q) quad(lr0 + 4 * q, aw + (2 * q) * kWJ);
        if (!ring_ready) prefetch_ring();  // else issued during the previous step's tail
        ring_ready = false;
        auto stream_math = [&](int it) {
          cp_async_wait<kWNST - 2>();
          __syncwarp();
          if (it + kWNST - 1 < NIT) issue(it + kWNST - 1);
          cp_async_commit();
          quad_math(lr0 + RWR + 4 * it, ring + (it % kWNST) * 2 * kWJ + 2 * jg);
        };
        // streamed rows up to the first chunk boundary (the resident rows
        // end on a multiple of 4, not of kWCH), then whole chunks unrolled
        // (RPW is a multiple of kWCH, so no partial chunk is left)
        int it = 0;
#pragma unroll 1
        for (; it < NIT && ((RWR + 4 * it) & (kWCH - 1)) != 0; ++it) {
          stream_math(it);
          const int lr = lr0 + RWR + 4 * it;
          if (((lr + 4) & (kWCH - 1)) == 0) track(lr / kWCH);
        }
#pragma unroll 1
        for (; it < NIT; it += kWCH / 4) {
#pragma unroll
          for (int u = 0; u < kWCH / 4; ++u) stream_math(it + u);
          track((lr0 + RWR + 4 * it) / kWCH);
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

      // ---- merge over warps: per (lane, target) the maximum and the first
      // chunk reaching it, sent to the target's owner
      {
        const int jj = tid % kWJ, s0 = tid / kWJ;
        const int orank = jj / JO, ojl = jj % JO;
#pragma unroll
        for (int s = s0; s < kWS; s += kWNT / kWJ) {
          if (wdesc[s].mode != 2) continue;
          float bv = -CUDART_INF_F;
          uint32_t wb = 0;
#pragma unroll
          for (int w = 0; w < kWNW; ++w) {
            const float* pvw = reinterpret_cast<const float*>(sRing + w * kWNST * 2 * kWJ);
            const uint8_t* pcw = reinterpret_cast<const uint8_t*>(pvw + kWS * kWJ);
            const float v = pvw[s * kWJ + jj];
            if (w == 0 || v > bv) { bv = v; wb = pcw[s * kWJ + jj]; }
          }
          const int off = ((cur * CR + (int)rank) * kWS + s) * JO + ojl;
          if (orank == (int)rank) {
            sRV[off] = bv;
            sRI[off] = wb;
          } else {
            dsmem_st_f32(dsmem_addr(sRV + off, orank), bv);
            dsmem_st_u32(dsmem_addr(sRI + off, orank), wb);
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
    // the next step streams the same logA rows: start its first ring stages
    // now, so they load during the owner phase and the waits below
    prefetch_ring();
    ring_ready = true;

    // ---- owners: lowest rank holding the maximum, + E_t, stores
#pragma unroll
    for (int u = 0; u < OPW; ++u) {
      const int o = tid + kWNT * u, os = o / JO, ol = o % JO, oj = j0 + (int)rank * JO + ol;
      if (o >= kWS * JO) continue;
      const WDesc& d = wdesc[os];
      if (!d.mode || oj >= K) continue;
      float dval;
      uint32_t mnew = 0;
      if (d.mode == 1) {
        if (d.first) dval = __fadd_rn(pv[u], ev[u]);
        else if (a.ckpt) dval = av[u];  // delta_m exactly as the forward pass stored it
        else dval = a.complete ? __fadd_rn(av[u], ev[u]) : __fadd_rn(__fadd_rn(d.s_prev, av[u]), ev[u]);
      } else {
        // the lowest rank holding the maximum, then its first chunk reaching
        // it: re-scan those kWCH rows (descending, so the last match is the
        // lowest row); the kept value is the recomputed candidate
        const int base = (cur * CR * kWS + os) * JO + ol;
        float bv = sRV[base];
        int rb = 0;
#pragma unroll
        for (int rr = 1; rr < CR; ++rr) {
          const float v = sRV[base + rr * kWS * JO];
          if (v > bv) { bv = v; rb = rr; }
        }
        const int rowc = rb * RPC + (int)sRI[base + rb * kWS * JO] * kWCH;
        const float4* dsrc = reinterpret_cast<const float4*>(a.wide_D + cur * SK + (int64_t)os * KD + rowc);
        // the chunk's kWCH transition weights into column oj are contiguous
        // in the column-major copy: kWCH / 4 16-byte loads
        const float4* asrc = reinterpret_cast<const float4*>(a.wide_AT + (int64_t)oj * KD + rowc);
        float4 dv[kWCH / 4], av4[kWCH / 4];
#pragma unroll
        for (int k2 = 0; k2 < kWCH / 4; ++k2) dv[k2] = dsrc[k2];
#pragma unroll
        for (int k2 = 0; k2 < kWCH / 4; ++k2) av4[k2] = __ldg(asrc + k2);
        unsigned long long avv[kWCH / 2];
#pragma unroll
        for (int k2 = 0; k2 < kWCH / 4; ++k2) {
          avv[2 * k2] = ((unsigned long long)__float_as_uint(av4[k2].y) << 32) | __float_as_uint(av4[k2].x);
          avv[2 * k2 + 1] = ((unsigned long long)__float_as_uint(av4[k2].w) << 32) | __float_as_uint(av4[k2].z);
        }
        uint4 mv[kWCH / 8];
#pragma unroll
        for (int k2 = 0; k2 < kWCH / 8; ++k2) mv[k2] = make_uint4(0u, 0u, 0u, 0u);
        if (d.f_mid == 2) {
          const uint4* msrc = reinterpret_cast<const uint4*>(a.wide_M + cur * SK + (int64_t)os * KD + rowc);
#pragma unroll
          for (int k2 = 0; k2 < kWCH / 8; ++k2) mv[k2] = msrc[k2];
        }
        int arg = 0;
        uint32_t mold = 0;  // MidState_{t-1} of the winning row
        float val = bv;
#pragma unroll
        for (int k2 = kWCH / 2 - 1; k2 >= 0; --k2) {
          const float4 q4 = dv[k2 / 2];
          const float dlo = (k2 & 1) ? q4.z : q4.x, dhi = (k2 & 1) ? q4.w : q4.y;
          const unsigned long long dpair =
              ((unsigned long long)__float_as_uint(dhi) << 32) | (unsigned long long)__float_as_uint(dlo);
          const uint4 m4 = mv[k2 / 4];
          const uint32_t mw = (k2 & 3) == 0 ? m4.x : ((k2 & 3) == 1 ? m4.y : ((k2 & 3) == 2 ? m4.z : m4.w));
          float c0, c1;
          wfadd2(dpair, avv[k2], c0, c1);
          if (c1 == bv) { arg = 2 * k2 + 1; val = c1; mold = mw >> 16; }
          if (c0 == bv) { arg = 2 * k2; val = c0; mold = mw & 0xffffu; }
        }
        const uint32_t ag = (uint32_t)(rowc + arg);
        dval = __fadd_rn(val, ev[u]);
        if (kind == kJobVanilla || kind == kJobLeaf) a.psi[d.psi_row + oj] = (uint16_t)ag;
        if (d.f_mid) {
          mnew = d.f_mid == 1 ? ag : mold;
          a.wide_M[nxt * SK + (int64_t)os * KD + oj] = (uint16_t)mnew;
        }
      }
      if (d.f_snap) {
        if (kind == kJobRoot) {
          a.snaps[d.snap_row + oj] = dval;
          if (d.map_row >= 0) a.maps[d.map_row + oj] = (uint16_t)mnew;
        } else {
          a.wide_X[(int64_t)d.par * SK + (int64_t)os * KD + oj] = dval;
        }
      }
      a.wide_D[nxt * SK + (int64_t)os * KD + oj] = dval;
    }
    __syncthreads();
    if (tid == 0 && !(a.wide_withhold && blockIdx.x == 0)) {
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
  cp_async_wait<0>();   // no copy into this CTA's shared memory is left in flight
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
  if (g.CR == 4) return run(wide_fwd_kernel<4>);
  return run(wide_fwd_kernel<2>);
}

}  // namespace fv
