// fv_dense.cu -- exact max-plus Viterbi on dense transitions (Sec. III-A),
// batched over uneven-length sequences in one persistent launch.
//
// Design (GB300-first):
//  * A cluster of CL CTAs (one per SM) owns a model: CTA r keeps the column
//    slab logA[:, rJ .. rJ+J) resident in shared memory for the whole
//    launch (FP32, exact).  K <= CL*J.
//  * Each cluster runs S independent sequences ("slots") in lockstep: one
//    tick computes one time step for every slot, so every logA element read
//    from shared memory is reused S times from registers.
//  * A tick is a small tropical GEMM: out[s][j] = max_i (delta[s][i] +
//    logA[i][j]).  Warps split the i range; each lane holds a 4(s) x 8(j)
//    register tile and issues one FADD + one FMNMX per cell.  The argmax is
//    recovered exactly afterwards: the first warp whose partial maximum
//    equals the overall maximum holds the lowest maximising index, which a
//    short re-scan of that warp's rows finds (the value kept is the
//    re-computed winning candidate, so ties and signed zeros follow the
//    lowest-index rule bit for bit).
//  * delta_t (and a bank-skewed transposed copy used by the re-scan) is
//    broadcast to every CTA of the cluster through distributed shared memory;
//    one cluster barrier per tick.
//  * Slots refill from a global work counter over a longest-first order, so
//    uneven lengths keep every slot busy (continuous batching at the tick
//    level).  psi is written as uint16 rows; the backtrack is a separate
//    warp-per-sequence kernel that streams psi rows through shared memory.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

// ------------------------------------------------------------------ prep


// Single CTA: validate every sequence, lay out its aux area (exclusive scan
// in batch order) and reset the header.
__global__ void __launch_bounds__(1024) prep_kernel(PrepArgs p) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    p.hdr->status = 0;
    p.hdr->detail = 0;
    carry = 0;
  }
  for (int k = tid; k < kMaxModels; k += blockDim.x) p.hdr->pop[k] = 0ull;
  if (tid < 5) p.hdr->counters[tid] = 0ull;
  __syncthreads();
  for (int base = 0; base < p.n_seq; base += blockDim.x) {
    const int b = base + tid;
    unsigned long long need = 0;
    int32_t T = 0, m = 0;
    if (b < p.n_seq) {
      T = p.T[b];
      m = p.model_idx ? p.model_idx[b] : 0;
      if (T < 1 || m < 0 || m >= p.n_models) {
        set_status(p.hdr, FV_EINVAL, (uint32_t)b);
        T = 1;
        m = 0;
      }
      const unsigned long long K = (unsigned long long)p.mk.K[m];
      if (p.aux_kind == 1) need = ((unsigned long long)T * K + 7ull) & ~7ull;
      else if (p.aux_kind == 2) need = ((unsigned long long)T + 3ull) & ~3ull;
      else if (p.aux_kind == 3) need = ((unsigned long long)T * (unsigned long long)p.aux_mult + 3ull) & ~3ull;
    }
    // block exclusive scan of need
    unsigned long long x = need;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long v = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0ull;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      warp_sum[lane] = v;
    }
    __syncthreads();
    const unsigned long long excl = carry + (w ? warp_sum[w - 1] : 0ull) + x - need;
    if (b < p.n_seq) {
      Job j;
      j.T = T;
      j.model = m;
      j.e_off = p.e_off[b];
      j.path_off = p.path_off[b];
      j.aux_off = (int64_t)excl;
      p.jobs[b] = j;
    }
    __syncthreads();
    if (tid == blockDim.x - 1) carry = excl + need;
    __syncthreads();
  }
  if (tid == 0) {
    p.hdr->aux_need = carry;
    p.hdr->aux_cap = p.aux_cap;
    if (carry > p.aux_cap) set_status(p.hdr, FV_ENOMEM, 0);
  }
}

// order[rank(b)] = b with rank by (model asc, T desc, b asc), or
// (model asc, b asc) when nosort.  O(n^2) comparisons through shared tiles.
__global__ void __launch_bounds__(256) order_kernel(const Job* jobs, int32_t n, int32_t nosort,
                                                    int32_t* order) {
  __shared__ int32_t sT[256], sM[256];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t myT = 0, myM = 0;
  if (b < n) {
    myT = jobs[b].T;
    myM = jobs[b].model;
  }
  int32_t rank = 0;
  for (int base = 0; base < n; base += 256) {
    const int k = base + threadIdx.x;
    if (k < n) {
      sT[threadIdx.x] = jobs[k].T;
      sM[threadIdx.x] = jobs[k].model;
    }
    __syncthreads();
    const int lim = min(256, n - base);
    if (b < n) {
      for (int x = 0; x < lim; ++x) {
        const int o = base + x;
        const int32_t oM = sM[x], oT = sT[x];
        bool before;
        if (oM != myM) before = oM < myM;
        else if (!nosort && oT != myT) before = oT > myT;
        else before = o < b;
        rank += before;
      }
    }
    __syncthreads();
  }
  if (b < n) order[rank] = b;
}

// ------------------------------------------------------------ forward engine
enum SlotState : int32_t { kNeedPop = 0, kWaiting = 1, kRun = 2, kDone = 3 };

// A job as seen by a slot; rank 0 of the cluster fills it and copies it
// word by word into every CTA, so all CTAs run identical slot states.
struct PJob {
  int32_t valid, b, m, n, T, Pe, q_prev, q_n;
  float s_prev;
  int32_t pad;
  int64_t e_off, path_off, aux_off;
};
static_assert(sizeof(PJob) % 4 == 0, "PJob is copied as 32-bit words");

struct Slot {
  int32_t state, term, t;
  int32_t kdiv, ediv, eprev;  // root: next division point index / value, previous one (-1: none)
  int32_t tmid;               // sub: midpoint of the segment
  int32_t f_mid;              // this tick: 0 no MidState, 1 MidState = psi, 2 MidState = MidState_prev[psi]
  int32_t f_snap, f_map, f_k; // this tick: snapshot delta / store ancestor map / division index
  int32_t pad;
  PJob cur, pend;
};

__host__ __device__ inline int32_t flash_pe(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
// Division point e_k = floor(((k+1)T - 1) / P') of the P-way first split.
__host__ __device__ inline int32_t flash_div(int32_t k, int32_t T, int32_t Pe) {
  return (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
}

template <int J, int S, int NW, int CL>
struct DenseCfg {
  static constexpr int NT = NW * 32;
  static constexpr int LJ = J / 8;
  static constexpr int LS = 32 / LJ;
  static constexpr int OPT = S * J / NT;
  static_assert(LJ * LS == 32 && LS * 4 == S, "lane tile is 4 sequences x 8 columns");
  static_assert((S * J) % NT == 0, "epilogue outputs per thread");
  static size_t smem_bytes(int KP) {
    const int KPS = KP + KP / 32;
    return sizeof(float) * ((size_t)KP * J + 2ull * KP * S + 2ull * S * KPS + (size_t)NW * S * J +
                            (size_t)S * KP) +
           sizeof(uint16_t) * 2ull * S * KP;
  }
};

template <int J, int S, int NW, int CL>
__global__ void __launch_bounds__(NW * 32) dense_fwd_kernel(DenseArgs a) {
  using Cfg = DenseCfg<J, S, NW, CL>;
  constexpr int NT = Cfg::NT, LJ = Cfg::LJ, OPT = Cfg::OPT;
  extern __shared__ __align__(16) float smem[];
  __shared__ Slot slots[S];

  const int K = a.K, KP = a.KP, C = KP / NW, KPS = KP + KP / 32;
  float* sA = smem;                  // [KP][J]     logA column slab
  float* sD = sA + (size_t)KP * J;   // [2][KP][S]  delta, row-major in i
  float* sR = sD + 2 * KP * S;       // [2][S][KPS] delta per slot, bank-skewed
  float* sPart = sR + 2 * S * KPS;   // [NW][S][J]  per-warp partial maxima
  float* sSnap = sPart + NW * S * J; // [S][KP]     sub: delta at t_mid
  uint16_t* sMid = reinterpret_cast<uint16_t*>(sSnap + S * KP);  // [2][S][KP] MidState

  const uint32_t rank = CL > 1 ? cluster_ctarank() : 0u;
  const int j0 = (int)rank * J;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kind = a.kind;

  if (a.hdr->status != 0) return;  // an earlier kernel recorded an error: do nothing

  for (int x = tid; x < KP * J; x += NT) {
    const int i = x / J, j = j0 + x % J;
    sA[x] = (i < K && j < K) ? __ldg(a.logA + (int64_t)i * K + j) : -CUDART_INF_F;
  }
  for (int x = tid; x < 2 * KP * S + 2 * S * KPS; x += NT) sD[x] = -CUDART_INF_F;
  for (int x = tid; x < 2 * S * KP; x += NT) sMid[x] = 0;
  if (tid < S) {
    slots[tid].state = kNeedPop;
    slots[tid].term = 0;
    slots[tid].pend.valid = 0;
  }
  if (CL > 1) cluster_sync_all(); else __syncthreads();

  int cur = 0;
  for (;;) {
    // ---- prologue: slot state machine (identical in every CTA)
    if (tid < S) {
      Slot& sl = slots[tid];
      sl.term = 0;
      if (sl.state == kRun && sl.t > sl.cur.n) {
        sl.term = 1;  // sl.cur stays valid for the termination below
        sl.state = kNeedPop;
      } else if (sl.state == kWaiting) {
        if (sl.pend.valid) {
          sl.cur = sl.pend;
          sl.state = kRun;
          sl.t = sl.cur.m;
          sl.kdiv = 0;
          sl.ediv = flash_div(0, sl.cur.T, sl.cur.Pe);
          sl.eprev = -1;
          sl.tmid = (sl.cur.m + sl.cur.n) / 2;
        } else {
          sl.state = kDone;
        }
      }
      if (sl.state == kNeedPop) {
        if (rank == 0) {
          const unsigned long long k = atomicAdd(a.pop, 1ull);
          PJob pj;
          pj.valid = 0;
          pj.b = pj.m = pj.n = pj.T = pj.Pe = pj.q_prev = pj.q_n = pj.pad = 0;
          pj.s_prev = 0.f;
          pj.e_off = pj.path_off = pj.aux_off = 0;
          if (kind != kJobSub) {
            if (k < (unsigned long long)a.order_count) {
              const int b = a.order[a.order_begin + (int)k];
              const Job jb = a.jobs[b];
              pj.valid = 1;
              pj.b = b;
              pj.m = 0;
              pj.n = jb.T - 1;
              pj.T = jb.T;
              pj.Pe = flash_pe(jb.T, a.P);
              pj.e_off = jb.e_off;
              pj.path_off = jb.path_off;
              pj.aux_off = jb.aux_off;
            }
          } else if (k < (unsigned long long)*a.task_count) {
            const Task tk = a.tasks[k];
            const Job jb = a.jobs[tk.b];
            pj.valid = 1;
            pj.b = tk.b;
            pj.m = tk.m;
            pj.n = tk.n;
            pj.T = jb.T;
            pj.e_off = jb.e_off;
            pj.path_off = jb.path_off;
            pj.aux_off = jb.aux_off;
            // states revealed by earlier levels; clamped so that no value can
            // index shared memory outside the slab
            const int qn = a.paths[jb.path_off + tk.n];
            pj.q_n = (unsigned)qn < (unsigned)a.K ? qn : 0;
            if (tk.m > 0) {
              const int qp = a.paths[jb.path_off + tk.m - 1];
              pj.q_prev = (unsigned)qp < (unsigned)a.K ? qp : 0;
              pj.s_prev = a.sval[jb.aux_off + tk.m - 1];
            }
          }
          const uint32_t* src = reinterpret_cast<const uint32_t*>(&pj);
          uint32_t* dst = reinterpret_cast<uint32_t*>(&sl.pend);
          for (int w = 0; w < (int)(sizeof(PJob) / 4); ++w) {
            dst[w] = src[w];
            for (int r = 1; r < CL; ++r) dsmem_st_u32(dsmem_addr(dst + w, r), src[w]);
          }
        }
        sl.state = kWaiting;
      }
      // per-tick flags of a running job
      sl.f_mid = sl.f_snap = sl.f_map = sl.f_k = 0;
      if (sl.state == kRun) {
        const int t = sl.t;
        if (kind == kJobRoot) {
          const int is_div = (t == sl.ediv);
          if (sl.eprev >= 0) sl.f_mid = (t == sl.eprev + 1) ? 1 : 2;
          sl.f_snap = is_div;
          sl.f_map = is_div && sl.kdiv >= 1;
          sl.f_k = sl.kdiv;
        } else if (kind == kJobSub) {
          sl.f_mid = (t == sl.tmid + 1) ? 1 : (t > sl.tmid + 1 ? 2 : 0);
          sl.f_snap = (t == sl.tmid);
        }
      }
    }
    const int live = (tid < S) && (slots[tid].state != kDone || slots[tid].term);
    if (!__syncthreads_or(live)) break;

    // ---- termination of jobs that finished last tick (rank 0)
    if (rank == 0) {
      for (int s = warp; s < S; s += NW) {
        if (!slots[s].term) continue;
        const PJob& jb = slots[s].cur;
        if (kind == kJobVanilla) {
          // q_{T-1} = lowest argmax_j delta_{T-1}[j]; score = delta_{T-1}[q]
          float bv = -CUDART_INF_F;
          int bi = 0x7fffffff;
          for (int j = lane; j < K; j += 32) {
            const float v = sD[((size_t)cur * KP + j) * S + s];
            if (bi == 0x7fffffff || v > bv) { bv = v; bi = j; }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi != 0x7fffffff && (bi == 0x7fffffff || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
          }
          if (lane == 0) {
            a.qlast[jb.b] = bi;
            a.scores[jb.b] = sD[((size_t)cur * KP + bi) * S + s];
          }
        } else if (kind == kJobSub && lane == 0) {
          // Alg. 2 output: q*_{tmid} = MidState[q*_n]; its delta from the snapshot
          const int tmid = (jb.m + jb.n) / 2;
          int q = sMid[((size_t)cur * S + s) * KP + ((unsigned)jb.q_n < (unsigned)K ? jb.q_n : 0)];
          q = (unsigned)q < (unsigned)K ? q : 0;
          a.paths[jb.path_off + tmid] = q;
          a.sval[jb.aux_off + tmid] = sSnap[(size_t)s * KP + q];
        }
      }
    }

    // ---- prefetch emission scores for this thread's epilogue outputs
    float ev[OPT], pv[OPT];
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      const int o = tid + r * NT, s = o / J, j = j0 + o % J;
      ev[r] = 0.f;
      pv[r] = 0.f;
      const Slot& sl = slots[s];
      if (sl.state == kRun && j < K) {
        const int t = sl.t;
        if (a.emit == FV_EMIT_DENSE) ev[r] = __ldg(a.E + sl.cur.e_off + (int64_t)t * K + j);
        else ev[r] = __ldg(a.logB + (int64_t)j * a.V + __ldg(a.obs + sl.cur.e_off + t));
        if (t == 0) pv[r] = __ldg(a.log_pi + j);
      }
    }

    // ---- main loop: value-only tropical product over this warp's rows
    {
      const int sg = lane / LJ, jg = lane % LJ;
      float acc[4][8];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = -CUDART_INF_F;
      const float* dp = sD + (size_t)cur * KP * S + sg * 4;
      const float* ap0 = sA + 4 * jg;
      const float* ap1 = sA + 4 * LJ + 4 * jg;
      const int i0 = warp * C, i1 = i0 + C;
#pragma unroll 2
      for (int i = i0; i < i1; ++i) {
        const float4 d = *reinterpret_cast<const float4*>(dp + (size_t)i * S);
        const float4 x0 = *reinterpret_cast<const float4*>(ap0 + (size_t)i * J);
        const float4 x1 = *reinterpret_cast<const float4*>(ap1 + (size_t)i * J);
        const float dv[4] = {d.x, d.y, d.z, d.w};
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] = fmaxf(acc[x][y], __fadd_rn(dv[x], xv[y]));
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float* pp = sPart + ((size_t)warp * S + sg * 4 + x) * J;
        *reinterpret_cast<float4*>(pp + 4 * jg) = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
        *reinterpret_cast<float4*>(pp + 4 * LJ + 4 * jg) = make_float4(acc[x][4], acc[x][5], acc[x][6], acc[x][7]);
      }
    }
    __syncthreads();

    // ---- merge, exact argmax re-scan, + E, per-kind bookkeeping, broadcast
    const int nxt = cur ^ 1;
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      const int o = tid + r * NT, s = o / J, jj = o % J, j = j0 + jj;
      const Slot& sl = slots[s];
      if (sl.state != kRun || j >= K) continue;
      const PJob& jb = sl.cur;
      float dval;
      int arg = 0;
      if (sl.t == jb.m) {
        if (jb.m == 0) {
          dval = __fadd_rn(pv[r], ev[r]);
        } else {
          // pruned start (Sec. V-B.2): only transitions out of q*_{m-1}
          const float av = sA[(size_t)jb.q_prev * J + jj];
          dval = a.complete ? __fadd_rn(av, ev[r]) : __fadd_rn(__fadd_rn(jb.s_prev, av), ev[r]);
        }
      } else {
        float best = sPart[(size_t)s * J + jj];
        int wb = 0;
        for (int w = 1; w < NW; ++w) {
          const float v = sPart[((size_t)w * S + s) * J + jj];
          if (v > best) { best = v; wb = w; }
        }
        const float* dr = sR + ((size_t)cur * S + s) * KPS;
        arg = wb * C;
        float val = best;
        for (int k = C - 1; k >= 0; --k) {
          const int i = wb * C + k;
          const float c = __fadd_rn(dr[i + (i >> 5)], sA[(size_t)i * J + jj]);
          if (c == best) { arg = i; val = c; }
        }
        arg = arg < K ? arg : 0;  // only NaN inputs (unsupported) could leave it on a padded row
        if (kind == kJobVanilla) a.psi[jb.aux_off + (int64_t)sl.t * K + j] = (uint16_t)arg;
        dval = __fadd_rn(val, ev[r]);
      }
      if (sl.f_mid) {
        const uint16_t mnew = sl.f_mid == 1 ? (uint16_t)arg : sMid[((size_t)cur * S + s) * KP + arg];
        uint16_t* mp = sMid + ((size_t)nxt * S + s) * KP + j;
        *mp = mnew;
        for (int rr = 0; rr < CL; ++rr)
          if (rr != (int)rank) dsmem_st_u16(dsmem_addr(mp, rr), mnew);
        if (sl.f_map) a.maps[(int64_t)jb.b * a.map_stride + (int64_t)(sl.f_k - 1) * K + j] = mnew;
      }
      if (sl.f_snap) {
        if (kind == kJobRoot) {
          a.snaps[(int64_t)jb.b * a.snap_stride + (int64_t)sl.f_k * K + j] = dval;
        } else {
          float* sp = sSnap + (size_t)s * KP + j;
          *sp = dval;
          for (int rr = 0; rr < CL; ++rr)
            if (rr != (int)rank) dsmem_st_f32(dsmem_addr(sp, rr), dval);
        }
      }
      float* d1 = sD + ((size_t)nxt * KP + j) * S + s;
      float* d2 = sR + ((size_t)nxt * S + s) * KPS + j + (j >> 5);
      *d1 = dval;
      *d2 = dval;
      if (CL > 1) {
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) {
          if (rr == (int)rank) continue;
          dsmem_st_f32(dsmem_addr(d1, rr), dval);
          dsmem_st_f32(dsmem_addr(d2, rr), dval);
        }
      }
    }
    if (CL > 1) cluster_sync_all(); else __syncthreads();
    if (tid < S && slots[tid].state == kRun) {
      Slot& sl = slots[tid];
      if (kind == kJobRoot && sl.t == sl.ediv) {
        sl.eprev = sl.ediv;
        sl.kdiv += 1;
        sl.ediv = sl.kdiv < sl.cur.Pe ? flash_div(sl.kdiv, sl.cur.T, sl.cur.Pe) : 0x7fffffff;
      }
      sl.t += 1;
    }
    cur = nxt;
  }
  if (CL > 1) cluster_sync_all();
}

// ------------------------------------------------------------- backtrack
// One warp per sequence: stream D psi rows at a time into shared memory and
// follow q_{t-1} = psi_t[q_t] (Sec. III-A, backtracking).
__global__ void __launch_bounds__(128) backtrack_kernel(const Job* jobs, const int32_t* order,
                                                        int32_t begin, int32_t count, int32_t K,
                                                        const uint16_t* psi, const int32_t* qlast,
                                                        int32_t* paths, int32_t D, const WsHeader* hdr) {
  extern __shared__ __align__(16) uint16_t sbuf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  if (idx >= count || hdr->status != 0) return;  // no forward pass ran: nothing to follow
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  uint16_t* buf = sbuf + (size_t)warp * D * K;
  int q = qlast[b];
  q = (unsigned)q < (unsigned)K ? q : 0;
  if (lane == 0) paths[jb.path_off + jb.T - 1] = q;
  const bool vec = (K % 8) == 0;
  for (int t = jb.T - 1; t >= 1; t -= D) {
    const int nrow = min(D, t);
    // rows t, t-1, ..., t-nrow+1 are contiguous in memory: [t-nrow+1, t]
    const uint16_t* src = psi + jb.aux_off + (int64_t)(t - nrow + 1) * K;
    const int n = nrow * K;
    if (vec) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(buf);
      for (int x = lane; x < n / 8; x += 32) d4[x] = __ldcs(s4 + x);
    } else {
      for (int x = lane; x < n; x += 32) buf[x] = src[x];
    }
    __syncwarp();
    if (lane == 0) {
      for (int r = nrow - 1; r >= 0; --r) {  // row r holds psi_{t-nrow+1+r}
        const int tt = t - nrow + 1 + r;
        q = buf[r * K + ((unsigned)q < (unsigned)K ? q : 0)];
        paths[jb.path_off + tt - 1] = q;
      }
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    __syncwarp();
  }
}

// ------------------------------------------------------------ path score
// score = fl(logpi[q0] + E_0[q0]); s = fl(fl(s + logA[q_{t-1}][q_t]) + E_t[q_t])


__device__ inline float csr_weight(const ScoreArgs& a, int i, int j) {
  int lo = a.row_ptr[i], hi = a.row_ptr[i + 1] - 1;
  float best = -CUDART_INF_F;
  // rows are sorted by column; duplicates (if any) are adjacent
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = a.col[mid];
    if (c < j) lo = mid + 1;
    else if (c > j) hi = mid - 1;
    else {
      int k = mid;
      while (k > a.row_ptr[i] && a.col[k - 1] == j) --k;
      for (; k < a.row_ptr[i + 1] && a.col[k] == j; ++k) best = fmaxf(best, a.val[k]);
      break;
    }
  }
  return best;
}

__global__ void path_score_kernel(ScoreArgs a, const Job* jobs, const int32_t* order, int32_t begin,
                                  int32_t count, const int32_t* paths, float* scores, const WsHeader* hdr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count || (hdr && hdr->status != 0)) return;
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  const int32_t* q = paths + jb.path_off;
  auto emis = [&](int t, int j) -> float {
    if (a.emit == FV_EMIT_DENSE) return __ldg(a.E + jb.e_off + (int64_t)t * a.K + j);
    return __ldg(a.logB + (int64_t)j * a.V + __ldg(a.obs + jb.e_off + t));
  };
  // state ids outside [0, K) make the score -inf (a path through no state)
  int qp = q[0];
  bool bad = (unsigned)qp >= (unsigned)a.K;
  qp = bad ? 0 : qp;
  float s = __fadd_rn(__ldg(a.log_pi + qp), emis(0, qp));
  for (int t = 1; t < jb.T; ++t) {
    int qt = q[t];
    if ((unsigned)qt >= (unsigned)a.K) { bad = true; qt = 0; }
    const float w = a.trans == FV_TRANS_DENSE ? __ldg(a.logA + (int64_t)qp * a.K + qt) : csr_weight(a, qp, qt);
    s = __fadd_rn(__fadd_rn(s, w), emis(t, qt));
    qp = qt;
  }
  scores[b] = bad ? -CUDART_INF_F : s;
}

// ------------------------------------------------------------ host launchers
template <int J, int S, int NW, int CL>
static cudaError_t launch_dense_cfg(const DenseArgs& a, int max_clusters, cudaStream_t st) {
  using Cfg = DenseCfg<J, S, NW, CL>;
  auto kern = dense_fwd_kernel<J, S, NW, CL>;
  const size_t smem = Cfg::smem_bytes(a.KP);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(Cfg::NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int resident = 0;
  if (CL > 1) {
    cfg.gridDim = dim3(CL * nsm);
    e = cudaOccupancyMaxActiveClusters(&resident, kern, &cfg);
    if (e != cudaSuccess) return e;
  } else {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, smem);
    if (e != cudaSuccess) return e;
    resident = per_sm * nsm;
  }
  if (resident < 1) return cudaErrorInvalidConfiguration;
  int want = (a.max_jobs + S - 1) / S;
  if (max_clusters > 0 && want > max_clusters) want = max_clusters;
  const int nclu = want < resident ? want : resident;
  if (nclu < 1) return cudaSuccess;
  cfg.gridDim = dim3(CL * nclu);
  return cudaLaunchKernelEx(&cfg, kern, a);
}

int dense_supported_K(int K) { return K >= 1 && K <= 256; }

// Rows padded to a multiple of 4 * NW for the chosen configuration.
cudaError_t launch_dense_forward(DenseArgs a, int max_clusters, cudaStream_t st) {
  if (a.K <= 64) {
    a.KP = (a.K + 15) / 16 * 16;
    return launch_dense_cfg<64, 16, 4, 1>(a, max_clusters, st);
  }
  a.KP = (a.K + 31) / 32 * 32;
  if (a.K <= 128) return launch_dense_cfg<128, 8, 8, 1>(a, max_clusters, st);
  return launch_dense_cfg<128, 8, 8, 2>(a, max_clusters, st);
}

cudaError_t launch_prep(const PrepArgs& p, cudaStream_t st) {
  prep_kernel<<<1, 1024, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_order(const Job* jobs, int32_t n, int32_t nosort, int32_t* order, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  order_kernel<<<(n + 255) / 256, 256, 0, st>>>(jobs, n, nosort, order);
  return cudaGetLastError();
}

cudaError_t launch_backtrack(const Job* jobs, const int32_t* order, int32_t begin, int32_t count,
                             int32_t K, const uint16_t* psi, const int32_t* qlast, int32_t* paths,
                             const WsHeader* hdr, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int D = 16384 / (2 * K);
  if (D < 1) D = 1;
  if (D > 64) D = 64;
  const int warps = 4;
  const size_t smem = (size_t)warps * D * K * sizeof(uint16_t);
  cudaError_t e = cudaFuncSetAttribute(backtrack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  backtrack_kernel<<<(count + warps - 1) / warps, warps * 32, smem, st>>>(jobs, order, begin, count, K, psi,
                                                                       qlast, paths, D, hdr);
  return cudaGetLastError();
}

cudaError_t launch_path_score(const ScoreArgs& a, const Job* jobs, const int32_t* order, int32_t begin,
                              int32_t count, const int32_t* paths, float* scores, const WsHeader* hdr,
                              cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  path_score_kernel<<<(count + 127) / 128, 128, 0, st>>>(a, jobs, order, begin, count, paths, scores, hdr);
  return cudaGetLastError();
}

}  // namespace fv
