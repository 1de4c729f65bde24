// fv_dense.cu -- exact max-plus Viterbi on dense transitions (Sec. III-A),
// batched over uneven-length sequences in one persistent launch.
//
// Design (GB300-first):
//  * A cluster of CL CTAs (one per SM) owns a model: CTA r computes the
//    target columns [rJ, rJ+J).  K <= 256: its column slab of logA stays in
//    shared memory for the whole launch (FP32, exact); 256 < K <= 1024: the
//    slab streams from an L2-resident row-pair copy through a per-warp
//    cp.async ring.
//  * Each cluster runs S independent sequences ("slots") in lockstep: one
//    tick computes one time step for every slot, so every logA element read
//    from shared memory is reused S times from registers.
//  * A tick is a small tropical product: out[s][j] = max_i (delta[s][i] +
//    logA[i][j]).  Warps split the i range; each lane holds a 4(s) x 8(j) or
//    4 x 4 register tile and issues one packed add.f32x2 and one 3-input max
//    per two cells (value only).  The argmax is recovered exactly
//    afterwards: the first row chunk whose partial maximum equals the
//    overall maximum holds the lowest maximising index, which a short
//    re-scan of that chunk finds (the value kept is the re-computed winning
//    candidate, so ties and signed zeros follow the lowest-index rule bit
//    for bit).
//  * delta_t goes to every CTA of the cluster through distributed shared
//    memory: one cluster barrier per tick for two CTAs, 16-byte st.async
//    stores completing transaction bytes on the receiver's mbarrier (bounded
//    waits) for four and eight.
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
      else if (p.aux_kind == 4) need = ckpt_area(T, p.aux_mult, (int32_t)K);
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
enum SlotState : int32_t { kIdle = 0, kRun = 2, kDone = 3 };

// A job as seen by a slot; rank 0 of the cluster fills it and sends it to
// every CTA, so all CTAs run identical slot states.
struct __align__(16) PJob {
  int32_t valid, b, m, n, T, Pe, q_prev, q_n;
  float s_prev;
  int32_t pad;
  int64_t e_off, path_off, aux_off;
};
static_assert(sizeof(PJob) % 16 == 0, "PJob is sent as 16-byte pieces");

// Slot state machine, replicated in every CTA of a cluster and run by the
// thread whose index is the slot on a register copy.  The next job of a slot
// is drawn one tick before its current job ends (or when the slot is idle);
// in multi-CTA clusters a draw becomes usable two ticks later, once every CTA
// has waited for the tick in which rank 0 sent it.
struct __align__(16) Slot {
  int32_t state, term, t, kdiv;  // kdiv, ediv, eprev: root division points (next index / value, previous)
  int32_t ediv, eprev, tmid;     // tmid: sub midpoint of the segment
  int32_t drawn;                 // a job was drawn for the slot and not yet taken
  int32_t draw_tick;             // engine tick of that draw
  int32_t ndraw;                 // draws so far; draw k is kept in pend[k & 1]
  int32_t drawn_now;             // drawn in this tick's prologue
  int32_t ev;                    // first job step (t) at which the prologue must run in full
  PJob cur;
};
// What the termination of a job that ended in this tick's prologue reads.
struct __align__(16) SlotFin {
  int32_t b, m, n, q_n;
  int64_t path_off, aux_off;
};

// What every thread needs to know about a slot during one tick, written by
// the slot's owner thread in the prologue and read with vector loads.
struct __align__(16) TickDesc {
  int32_t mode;       // 0 idle, 1 first step of the job (init), 2 max-plus step
  int32_t f_mid;      // 0 none, 1 MidState = psi, 2 MidState = MidState_prev[psi]
  int32_t f_snap;     // root: this tick's delta to the global snapshot; sub: rank 0 keeps delta_{t-1}
  int32_t q_prev;     // pruned start: q*_{m-1} (0 when m == 0)
  float s_prev;       // pruned start: retained offset
  int32_t first;      // 1 when t == 0 (start from pi)
  int64_t psi_row;    // vanilla: element offset of psi_t[0]
  const float* erow;  // dense emissions: E_t row
  int64_t snap_row;   // root: element offset of the snapshot row (f_snap)
  int64_t map_row;    // root: element offset of the map row, -1 if none
  int32_t sym;        // discrete emissions: observation symbol x_t
};
static_assert(sizeof(TickDesc) == 64, "tick descriptor: 64 bytes");

// c = (d.lo + a.lo, d.hi + a.hi), two FP32 adds rounded to nearest even,
// then acc = max(acc, c.lo, c.hi) with the 3-input max.
__device__ __forceinline__ void fadd2_max3(float& acc, unsigned long long d, unsigned long long a) {
  asm("{\n\t.reg .b64 c;\n\t.reg .f32 lo, hi;\n\tadd.rn.f32x2 c, %1, %2;\n\tmov.b64 {lo, hi}, c;\n\t"
      "max.f32 %0, %0, lo, hi;\n\t}"
      : "+f"(acc)
      : "l"(d), "l"(a));
}
__device__ __forceinline__ void fadd2(unsigned long long d, unsigned long long a, float& c0, float& c1) {
  unsigned long long c;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(c) : "l"(d), "l"(a));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(c));
}


// bounded wait of the multi-CTA exchange (~1 s at 2 GHz); on expiry the
// engine records FV_ETIMEOUT and stops at the next tick
constexpr long long kClusterWaitCycles = 1ll << 31;

// TW = columns per lane (8, or 4 for the 16-warp configurations): a lane
// holds 4 slots x TW columns; a warp covers all S slots and LJ*TW columns;
// CG warps side by side cover the CTA's J columns and RG = NW/CG row groups
// split the rows.
// DEFER: the exact re-scan of a tick runs after the tick's delta has been
// sent (its latency then overlaps the exchange; streamed engines read its
// weights from L2 meanwhile) -- for jobs without
// MidState (vanilla, budget leaves, checkpoint passes); a third delta buffer
// keeps the re-scanned rows intact while the other CTAs already write the
// next tick's delta, and the MidState buffers are left out.
// MINB: CTAs per SM the configuration is sized for (2: the slab, the
// buffers and the registers of two CTAs fit one SM, so two independent
// clusters overlap one's max-plus loop with the other's merge and exchange)
template <int J, int S, int NW, int CL, int KPM, bool STREAM, int TW = 8, bool DEFER = false, int MINB = 1>
struct DenseCfg {
  static constexpr int NT = NW * 32;
  static constexpr int LS = S / 4;        // slot groups per warp
  static constexpr int LJ = 32 / LS;      // column lanes per warp
  static constexpr int WC = LJ * TW;      // columns per warp
  static constexpr int CG = J / WC;       // column groups
  static constexpr int RG = NW / CG;      // row groups
  static constexpr int OPT = S * J / NT;
  static constexpr int KP = KPM;          // rows, padded (-inf) to a fixed count
  static constexpr int C = KPM / RG;      // rows per row group
  // rows per argmax chunk: streamed engines track the first chunk reaching
  // the maximum in the loop and re-scan that chunk from L2, so smaller
  // chunks (measured: 8 rows for 4-CTA clusters, 16 for 8-CTA ones) trade
  // a little loop work for a shorter re-scan
  static constexpr int CH = STREAM ? (KPM <= 512 ? 8 : 16) : C;
  // streamed: ring stages of 4 rows per warp (4 when the third delta
  // buffer of a deferred K <= 1024 configuration takes the room of one)
  // (2 stages when two 8-warp CTAs share an SM: the other warps hide the
  // shallower ring's latency)
  static constexpr int NST = MINB >= 2 && NW >= 8 ? 2 : (KPM <= 512 ? 8 : (DEFER ? 4 : 5));
  static constexpr int KPS = KPM + KPM / 8;  // skewed delta row: i -> i + 4*(i/32)
  static constexpr int NDB = DEFER ? 3 : 2;   // delta buffers
  static constexpr int NMID = DEFER ? 0 : 2;  // MidState buffers
  static_assert(LJ * LS == 32 && LS * 4 == S && (TW == 8 || TW == 4), "lane tile is 4 sequences x TW columns");
  static_assert(J % WC == 0 && NW % CG == 0 && WC % 32 == 0, "warp tiling");
  static_assert((S * J) % NT == 0 && NT % J == 0, "epilogue: one column per thread, OPT slots");
  static_assert(C % CH == 0 && CH % 4 == 0 && (32 % CH == 0 || CH % 32 == 0), "chunks inside skew blocks");
  static_assert(!STREAM || C / CH <= 255 * 1, "chunk ids fit a byte");
  // resident: logA slab [KP/2][J] float2; streamed: per-warp ring of NST
  // stages x 2 row pairs x J float2, plus the chunk id of each partial
  static constexpr size_t a_floats = STREAM ? (size_t)NW * NST * 4 * WC : (size_t)KP * J;
  // sub-job snapshots in shared memory unless they would not fit next to
  // the rest (streamed engines and wide row-group splits keep them in the
  // workspace, one row of KP floats per slot of each cluster)
  static constexpr bool GSNAP =
      STREAM || (a_floats + (size_t)NDB * S * KPS + (size_t)RG * S * J + (size_t)S * KP) * sizeof(float) +
                        (size_t)NMID * S * KP * sizeof(uint16_t) > (size_t)(MINB >= 2 ? 100 : 220) * 1024;
  static constexpr size_t snap_floats = GSNAP ? 0 : (size_t)S * KP;
  static constexpr size_t smem_bytes =
      sizeof(float) * (a_floats + (size_t)NDB * S * KPS + (size_t)RG * S * J + snap_floats) +
      sizeof(uint16_t) * (size_t)NMID * S * KP + (STREAM ? (size_t)RG * S * J : 0);
};

template <int J, int S, int NW, int CL, int KPM, bool STREAM, int TW, bool DEFER, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) dense_fwd_kernel(DenseArgs a) {
  using Cfg = DenseCfg<J, S, NW, CL, KPM, STREAM, TW, DEFER, MINB>;
  constexpr int NDB = Cfg::NDB;
  static_assert(!DEFER || CL > 1, "deferred re-scan: multi-CTA configurations");
  constexpr int NT = Cfg::NT, LJ = Cfg::LJ, OPT = Cfg::OPT, KP = Cfg::KP, C = Cfg::C, KPS = Cfg::KPS;
  constexpr int CG = Cfg::CG, RG = Cfg::RG, WC = Cfg::WC;
  constexpr int CH = Cfg::CH, NST = Cfg::NST;
  extern __shared__ __align__(16) float smem[];
  __shared__ Slot slots[S];
  __shared__ PJob s_pend[S][2];
  __shared__ SlotFin s_fin[S];
  __shared__ TickDesc tdesc[S];
  static_assert(Cfg::smem_bytes + (sizeof(Slot) + 2 * sizeof(PJob) + sizeof(SlotFin) + sizeof(TickDesc)) * S + 64 <=
                    (MINB >= 2 ? 110 : 227) * 1024,
                "dynamic + static shared memory within what MINB CTAs per SM may use");
  // multi-CTA clusters: barrier b completes when delta_t (t & 1 == b) of
  // every CTA is in this CTA's shared memory (local warps arrive, the other
  // CTAs' 16-byte stores complete transaction bytes)
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_info[2][5];  // per tick parity: active / MidState / sub-snapshot / drawn / ended slot masks
  __shared__ int s_abort;

  const int K = a.K;
  // resident: logA column slab as row pairs sA2[i/2][jj] = (A[i][j0+jj],
  // A[i+1][j0+jj]); streamed: each warp's ring of row-pair stages, filled
  // with cp.async from the row-pair copy a.Ap in global memory
  float* sA = smem;                           // resident [KP/2][J] / streamed [NW][NST][2][J] float2
  float* sD = sA + Cfg::a_floats;             // [NDB][S][KPS] delta per slot, skewed rows
  float* sPart = sD + NDB * S * KPS;          // [RG][S][J]  per-row-group partial maxima
  float* sSnap = sPart + RG * S * J;          // resident [S][KP] sub: delta at t_mid
  uint16_t* sMid = reinterpret_cast<uint16_t*>(sSnap + Cfg::snap_floats);  // [2][S][KP] MidState
  uint8_t* sPC = reinterpret_cast<uint8_t*>(sMid + Cfg::NMID * S * KP);   // streamed [RG][S][J] chunk
  const float2* sA2 = reinterpret_cast<const float2*>(sA);
  // streamed: global snapshot rows of this cluster's slots (sub jobs)
  float* gSnap = Cfg::GSNAP ? a.snap_scratch + (size_t)(blockIdx.x / CL) * S * KP : nullptr;

  const uint32_t rank = CL > 1 ? cluster_ctarank() : 0u;
  const int j0 = (int)rank * J;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kind = a.kind;
  // epilogue mapping: this thread owns column jj for slots s0 + r * (NT / J)
  const int jj = tid % J, jcol = j0 + jj, s0 = tid / J;
  constexpr int SSTEP = NT / J;
  // delta exchange of multi-CTA clusters (measured per cluster size): two
  // CTAs use plain remote stores and a cluster barrier per tick (0); larger
  // clusters use 16-byte st.async stores that complete transaction bytes on
  // the receiver's mbarrier, so no CTA waits for its stores to be
  // acknowledged (1)
  constexpr int kExch = CL <= 2 ? 0 : 1;
  constexpr int kLag = CL == 1 ? 0 : (kExch == 0 ? 1 : 2);  // ticks from a draw until every CTA holds it

  if (a.hdr->status != 0) return;  // an earlier kernel recorded an error: do nothing

  if constexpr (!STREAM) {
    for (int x = tid; x < KP * J; x += NT) {
      const int ip = x / (2 * J), c = (x / 2) % J, i = 2 * ip + (x & 1), j = j0 + c;
      sA[x] = (i < K && j < K) ? __ldg(a.logA + (int64_t)i * K + j) : -CUDART_INF_F;
    }
  }
  for (int x = tid; x < NDB * S * KPS; x += NT) sD[x] = -CUDART_INF_F;
  for (int x = tid; x < Cfg::NMID * S * KP; x += NT) sMid[x] = 0;

  // next job for the slot: rank 0 draws an index from the shared counter and
  // reads the job (other CTAs receive it)
  auto fetch_job = [&]() -> PJob {
    PJob pj;
    pj.valid = 0;
    pj.b = pj.m = pj.n = pj.T = pj.Pe = pj.q_prev = pj.q_n = pj.pad = 0;
    pj.s_prev = 0.f;
    pj.e_off = pj.path_off = pj.aux_off = 0;
    const unsigned long long k = atomicAdd(a.pop, 1ull);
    const bool from_tasks = kind == kJobSub || kind == kJobLeaf;
    if (!from_tasks) {
      if (k < (unsigned long long)a.order_count) {
        const int b = a.order[a.order_begin + (int)k];
        const Job jb = a.jobs[b];
        pj.valid = 1;
        pj.b = b;
        pj.m = 0;
        pj.n = jb.T - 1;
        pj.T = jb.T;
        pj.Pe = a.ckpt ? ckpt_count(jb.T, a.P) : flash_pe(jb.T, a.P);
        pj.e_off = jb.e_off;
        pj.path_off = jb.path_off;
        pj.aux_off = jb.aux_off;
      }
    } else if (k < (unsigned long long)*a.task_count) {
      const Task tk = a.tasks[(a.task_first ? *a.task_first : 0) + (int64_t)k];
      const Job jb = a.jobs[tk.b];
      pj.valid = 1;
      pj.b = tk.b;
      pj.m = tk.m;
      pj.n = tk.n;
      pj.T = jb.T;
      pj.e_off = jb.e_off;
      pj.path_off = jb.path_off;
      pj.aux_off = jb.aux_off;
      pj.pad = tk.pad;
      // states revealed by earlier levels; clamped so that no value can
      // index shared memory outside the slab
      if (a.ckpt) {
        // checkpoint segment: restarts from checkpoint tk.pad (or from pi)
        pj.Pe = ckpt_count(jb.T, a.P);
      } else {
        const int qn = a.paths[jb.path_off + tk.n];
        pj.q_n = (unsigned)qn < (unsigned)a.K ? qn : 0;
        if (tk.m > 0) {
          const int qp = a.paths[jb.path_off + tk.m - 1];
          pj.q_prev = (unsigned)qp < (unsigned)a.K ? qp : 0;
          pj.s_prev = a.sval[jb.aux_off + tk.m - 1];
        }
      }
    }
    return pj;
  };
  auto draw = [&](Slot& sl, int tick) {
    const int k = sl.ndraw & 1;
    sl.ndraw += 1;
    sl.drawn = 1;
    sl.draw_tick = tick;
    sl.drawn_now = 1;
    if (rank == 0) {
      s_pend[tid][k] = fetch_job();
      if constexpr (CL > 1 && kExch == 0) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&s_pend[tid][k]);
        for (int w = 0; w < (int)(sizeof(PJob) / 4); ++w)
          for (int r = 1; r < CL; ++r) dsmem_st_u32(dsmem_addr(src + w, r), src[w]);
      }
    }
  };

  // every slot starts with one job drawn before the first tick
  if (tid < S) {
    Slot sl;
    sl.state = kIdle;
    sl.term = sl.t = sl.kdiv = sl.ediv = sl.eprev = sl.tmid = 0;
    sl.drawn = 1;
    sl.draw_tick = -kLag;
    sl.ndraw = 1;
    sl.drawn_now = 0;
    sl.ev = 0;
    sl.cur = PJob{};
    slots[tid] = sl;
    if (rank == 0) s_pend[tid][0] = fetch_job();
  }
  if (tid == 0) s_abort = 0;
  // distributed shared memory bases of the peers (byte addresses)
  uint32_t pD[CL], pMid[CL], pBar0[CL], pBar1[CL];
#pragma unroll
  for (int rr = 0; rr < CL; ++rr) {
    pD[rr] = CL > 1 ? dsmem_addr(sD, rr) : 0u;
    pMid[rr] = CL > 1 ? dsmem_addr(sMid, rr) : 0u;
    pBar0[rr] = CL > 1 ? dsmem_addr(&s_bar[0], rr) : 0u;
    pBar1[rr] = CL > 1 ? dsmem_addr(&s_bar[1], rr) : 0u;
  }
  if constexpr (CL > 1) {
    if (tid == 0) {
      mbar_init(smem_addr(&s_bar[0]), NW);
      mbar_init(smem_addr(&s_bar[1]), NW);
      fence_mbar_init_cluster();
    }
    cluster_sync_all();  // every CTA of the cluster runs: its shared memory may be written
    if (rank == 0 && tid < S) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&s_pend[tid][0]);
      for (int w = 0; w < (int)(sizeof(PJob) / 4); ++w)
        for (int r = 1; r < CL; ++r) dsmem_st_u32(dsmem_addr(src + w, r), src[w]);
    }
    cluster_sync_all();
  } else {
    __syncthreads();
  }

  int cur = 0;
  int tick = 0;
  for (;; ++tick) {
    int tick_live = 0;

    // ---- streamed: the first ring stages of this tick's logA rows
    const int sg = lane / LJ, jg = lane % LJ;
    const int cg = warp % CG, rg = warp / CG;
    float2* ring = STREAM ? reinterpret_cast<float2*>(sA) + warp * NST * 2 * WC : nullptr;
    const float2* gsrc = STREAM ? a.Ap + (int64_t)(rg * C / 2) * a.ap_stride + j0 + cg * WC : nullptr;
    constexpr int NIT = C / 4;
    auto issue = [&](int it, int slot) {
      float2* dst = ring + slot * 2 * WC;
#pragma unroll
      for (int u = 0; u < WC / 32; ++u) {
        const int q = lane + 32 * u, pr = q / (WC / 2), c2 = (q % (WC / 2)) * 2;
        cp_async16(dst + pr * WC + c2, gsrc + (int64_t)(2 * it + pr) * a.ap_stride + c2);
      }
    };
    if constexpr (STREAM) {
#pragma unroll
      for (int k = 0; k < NST - 1; ++k) {
        if (k < NIT) issue(k, k);
        cp_async_commit();
      }
    }

    // ---- multi-CTA clusters: wait until delta_{t-1} of every CTA is here
    if constexpr (CL > 1 && kExch != 0) {
      if (tick > 0) {
        const uint32_t bar = smem_addr(&s_bar[(tick - 1) & 1]);
        const uint32_t par = (uint32_t)((tick - 1) >> 1) & 1u;
        if (!mbar_try_wait_cluster(bar, par)) {
          const long long w0 = clock64();
          while (!mbar_try_wait_cluster(bar, par)) {
            if (clock64() - w0 > kClusterWaitCycles) {
              set_status(a.hdr, FV_ETIMEOUT, 3);
              s_abort = 1;
              break;
            }
          }
        }
      }
    }

    // ---- prologue: slot state machine (identical in every CTA), run by
    // the slots' owner threads in warp 0 while the other warps start this
    // tick's max-plus loop, which does not depend on it; the barrier after
    // the loop publishes the descriptors
    {
      TickDesc td;
      td.mode = 0;
      td.f_mid = td.f_snap = td.q_prev = td.first = td.sym = 0;
      td.s_prev = 0.f;
      td.psi_row = 0;
      td.erow = nullptr;
      td.snap_row = 0;
      td.map_row = -1;
      int drawn_now = 0, live = 0, term = 0;
      if (tid < S) {
        Slot sl = slots[tid];
        const bool done_before = sl.state == kDone;
        if (done_before) {
          // finished for good: its idle descriptor was stored when it ended
          if (sl.term) slots[tid].term = 0;
          sl.term = 0;
        } else if (sl.state == kRun && sl.t + 1 < sl.ev) {
          // plain step: nothing but t changes until step ev, so the
          // descriptor advances by one row
          td = tdesc[tid];
          sl.t += 1;
          sl.term = 0;
          sl.drawn_now = 0;
          td.psi_row += K;
          if (a.emit == FV_EMIT_DENSE) td.erow += K;
          else td.sym = __ldg(a.obs + sl.cur.e_off + sl.t);
          live = !s_abort;
        } else {
          // advance the job that computed its step in the previous tick
          if (sl.state == kRun) {
            if (kind == kJobRoot && sl.t == sl.ediv) {
              sl.eprev = sl.ediv;
              sl.kdiv += 1;
              sl.ediv = sl.kdiv < sl.cur.Pe ? flash_div(sl.kdiv, sl.cur.T, sl.cur.Pe) : 0x7fffffff;
            }
            sl.t += 1;
          }
          sl.term = 0;
          sl.drawn_now = 0;
          if (sl.state == kRun && sl.t > sl.cur.n) {
            // the next job may start in this prologue: keep what the
            // termination of this one reads
            sl.term = 1;
            SlotFin f;
            f.b = sl.cur.b;
            f.m = sl.cur.m;
            f.n = sl.cur.n;
            f.q_n = sl.cur.q_n;
            f.path_off = sl.cur.path_off;
            f.aux_off = sl.cur.aux_off;
            s_fin[tid] = f;
            sl.state = kIdle;
          }
          if (sl.state == kIdle && !sl.drawn) draw(sl, tick);
          if (sl.state == kIdle && sl.drawn && tick >= sl.draw_tick + kLag) {
            const PJob pj = s_pend[tid][(sl.ndraw - 1) & 1];
            sl.drawn = 0;
            if (pj.valid) {
              sl.cur = pj;
              sl.state = kRun;
              sl.t = pj.m;
              sl.kdiv = 0;
              sl.ediv = flash_div(0, pj.T, pj.Pe);
              sl.eprev = -1;
              sl.tmid = (pj.m + pj.n) / 2;
            } else {
              sl.state = kDone;
            }
          }
          // the next job is drawn one tick before this one's last step
          if (sl.state == kRun && !sl.drawn && sl.cur.n - sl.t <= 1) draw(sl, tick);
          drawn_now = sl.drawn_now;
          live = (sl.state != kDone || sl.term) && !s_abort;
          // this tick's descriptor of the slot
          if (sl.state == kRun) {
            const int t = sl.t;
            const PJob& jb = sl.cur;
            td.mode = (t == jb.m) ? 1 : 2;
            td.first = (t == 0);
            td.q_prev = jb.q_prev;
            td.s_prev = jb.s_prev;
            td.psi_row = kind != kJobLeaf ? jb.aux_off + (int64_t)t * K
                         : a.ckpt ? 2 * (jb.aux_off + (int64_t)jb.Pe * K) + (int64_t)(t - jb.m - 1) * K
                                  : (int64_t)(jb.pad + t - jb.m - 1) * K;
            if (a.emit == FV_EMIT_DENSE) td.erow = a.E + jb.e_off + (int64_t)t * K;
            else td.sym = __ldg(a.obs + jb.e_off + t);
            if (kind == kJobRoot) {
              const int is_div = (t == sl.ediv);
              td.f_snap = is_div;
              if (a.ckpt) {
                // checkpoints only: delta_t at division point kdiv
                td.snap_row = jb.aux_off + (int64_t)sl.kdiv * K;
              } else {
                if (sl.eprev >= 0) td.f_mid = (t == sl.eprev + 1) ? 1 : 2;
                td.snap_row = (int64_t)jb.b * a.snap_stride + (int64_t)sl.kdiv * K;
                td.map_row =
                    (is_div && sl.kdiv >= 1) ? (int64_t)jb.b * a.map_stride + (int64_t)(sl.kdiv - 1) * K : -1;
              }
            } else if (kind == kJobLeaf && a.ckpt && jb.pad >= 0) {
              // checkpoint segment: the restart reads checkpoint jb.pad
              td.snap_row = jb.aux_off + (int64_t)jb.pad * K;
            } else if (kind == kJobSub) {
              // delta_{tmid} is complete in shared memory at the next tick,
              // where rank 0 keeps it as the snapshot (t_mid < n)
              td.f_mid = (t == sl.tmid + 1) ? 1 : (t > sl.tmid + 1 ? 2 : 0);
              td.f_snap = (t == sl.tmid + 1);
            }
          }
          // next step at which the descriptor changes other than by one row:
          // the step after any non-steady one (first step, snapshot, map
          // reset), the draw one step before the last, the next root
          // division point and the sub snapshot step
          if (sl.state == kRun) {
            const int t = sl.t;
            int ev = sl.cur.n - 1;
            if (td.mode == 1 || td.f_snap || td.f_mid == 1) ev = min(ev, t + 1);
            if (kind == kJobRoot && sl.ediv > t) ev = min(ev, sl.ediv);
            if (kind == kJobSub && sl.tmid + 1 > t) ev = min(ev, sl.tmid + 1);
            sl.ev = ev;
          }
        }
        if (!done_before) {
          tdesc[tid] = td;
          slots[tid] = sl;
        }
        term = sl.term;
      }
      if (warp == 0) {
        const bool own = tid < S;
        const uint32_t act = __ballot_sync(0xffffffffu, own && td.mode != 0);
        const uint32_t mid = __ballot_sync(0xffffffffu, own && td.f_mid != 0);
        const uint32_t snp = __ballot_sync(0xffffffffu, own && kind == kJobSub && td.f_snap != 0);
        const uint32_t drw = __ballot_sync(0xffffffffu, own && drawn_now);
        const uint32_t trm = __ballot_sync(0xffffffffu, own && term);
        if (lane == 0) {
          s_info[tick & 1][0] = act;
          s_info[tick & 1][1] = mid;
          s_info[tick & 1][2] = snp;
          s_info[tick & 1][3] = drw;
          s_info[tick & 1][4] = trm;
        }
      }
      tick_live = live;
    }

    // ---- main loop: value-only tropical product over this warp's C rows.
    // Per 4 rows a lane loads delta[4 slots][4 rows] and logA[4 rows][8
    // columns] as row pairs and issues one add.f32x2 + one 3-input max per
    // 2 cells.
    if constexpr (STREAM) {
      // streamed: this warp's C rows (its row group) of its WC columns
      // arrive 4 rows at a time through an NST-stage cp.async ring; chunk
      // winners (first chunk of CH rows reaching the running maximum) are
      // kept per output in registers
      float acc[4][TW], bst[4][TW];
      int bch[4][TW];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < TW; ++y) {
          acc[x][y] = -CUDART_INF_F;
          bst[x][y] = -CUDART_INF_F;
          bch[x][y] = 0;
        }
      const int i0 = rg * C;
      const float* dbase0 = sD + (cur * S + sg * 4) * KPS;
#pragma unroll 1
      for (int it0 = 0; it0 < NIT; it0 += CH / 4) {
        // one chunk (CH rows) per pass, unrolled: the ring slot is a
        // compile-time index when the ring has one stage per 4-row step
#pragma unroll
        for (int u = 0; u < CH / 4; ++u) {
          const int it = it0 + u;
          cp_async_wait<NST - 2>();
          __syncwarp();
          if (it + NST - 1 < NIT) issue(it + NST - 1, NST == CH / 4 ? (u + NST - 1) % NST : (it + NST - 1) % NST);
          cp_async_commit();
          const int i = i0 + 4 * it;
          const float* dbase = dbase0 + i + ((i >> 5) << 2);
          const float2* abase = ring + (NST == CH / 4 ? u : it % NST) * 2 * WC + 2 * jg;
          ulonglong2 dq[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) dq[x] = *reinterpret_cast<const ulonglong2*>(dbase + x * KPS);
          ulonglong2 aq[2][TW / 2];
#pragma unroll
          for (int pr = 0; pr < 2; ++pr)
#pragma unroll
            for (int g = 0; g < TW / 2; ++g)
              aq[pr][g] = *reinterpret_cast<const ulonglong2*>(abase + pr * WC + 2 * LJ * g);
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int g = 0; g < TW / 2; ++g) {
              fadd2_max3(acc[x][2 * g], dq[x].x, aq[0][g].x);
              fadd2_max3(acc[x][2 * g], dq[x].y, aq[1][g].x);
              fadd2_max3(acc[x][2 * g + 1], dq[x].x, aq[0][g].y);
              fadd2_max3(acc[x][2 * g + 1], dq[x].y, aq[1][g].y);
            }
        }
        // acc is the running maximum over the rows so far: a chunk that
        // raised it holds the first row reaching the new maximum
        const int c = rg * (C / CH) + it0 / (CH / 4);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < TW; ++y) {
            if (acc[x][y] > bst[x][y]) bch[x][y] = c;
            bst[x][y] = acc[x][y];
          }
      }
      cp_async_wait<0>();
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float* pp = sPart + (rg * S + sg * 4 + x) * J + cg * WC + 2 * jg;
        uint8_t* pc = sPC + (rg * S + sg * 4 + x) * J + cg * WC + 2 * jg;
#pragma unroll
        for (int g = 0; g < TW / 2; ++g) {
          *reinterpret_cast<float2*>(pp + 2 * LJ * g) = make_float2(bst[x][2 * g], bst[x][2 * g + 1]);
          pc[2 * LJ * g] = (uint8_t)bch[x][2 * g];
          pc[2 * LJ * g + 1] = (uint8_t)bch[x][2 * g + 1];
        }
      }
    } else {
      float acc[4][TW];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < TW; ++y) acc[x][y] = -CUDART_INF_F;
      const int i0 = rg * C;
      const float* dbase = sD + (cur * S + sg * 4) * KPS + i0 + ((i0 >> 5) << 2);
      const float2* abase = sA2 + (i0 / 2) * J + cg * WC + 2 * jg;
#pragma unroll
      for (int ii = 0; ii < C; ii += 4) {
        ulonglong2 dq[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) dq[x] = *reinterpret_cast<const ulonglong2*>(dbase + x * KPS + ii);
        ulonglong2 aq[2][TW / 2];
#pragma unroll
        for (int pr = 0; pr < 2; ++pr)
#pragma unroll
          for (int g = 0; g < TW / 2; ++g)
            aq[pr][g] = *reinterpret_cast<const ulonglong2*>(abase + (ii / 2 + pr) * J + 2 * LJ * g);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int g = 0; g < TW / 2; ++g) {
            fadd2_max3(acc[x][2 * g], dq[x].x, aq[0][g].x);
            fadd2_max3(acc[x][2 * g], dq[x].y, aq[1][g].x);
            fadd2_max3(acc[x][2 * g + 1], dq[x].x, aq[0][g].y);
            fadd2_max3(acc[x][2 * g + 1], dq[x].y, aq[1][g].y);
          }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float* pp = sPart + (rg * S + sg * 4 + x) * J + cg * WC + 2 * jg;
#pragma unroll
        for (int g = 0; g < TW / 2; ++g)
          *reinterpret_cast<float2*>(pp + 2 * LJ * g) = make_float2(acc[x][2 * g], acc[x][2 * g + 1]);
      }
    }
    // every warp's partial maxima and this tick's slot descriptors are
    // published; a tick with no live slot ends the engine
    if (!__syncthreads_or(tick_live)) break;
    const uint32_t m_act = s_info[tick & 1][0], m_mid = s_info[tick & 1][1], m_snp = s_info[tick & 1][2];
    const uint32_t m_drw = s_info[tick & 1][3], m_trm = s_info[tick & 1][4];

    // ---- this thread's emission scores (column jcol, OPT slots): issued
    // now, used after the merge and re-scan, which hide their latency
    float ev[OPT], pv[OPT];
    TickDesc tdr[OPT];
#pragma unroll
    for (int r = 0; r < OPT; ++r) tdr[r] = tdesc[s0 + r * SSTEP];
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      ev[r] = 0.f;
      pv[r] = 0.f;
      if (tdr[r].mode && jcol < K) {
        ev[r] = a.emit == FV_EMIT_DENSE ? __ldg(tdr[r].erow + jcol) : __ldg(a.logB + (int64_t)jcol * a.V + tdr[r].sym);
        if (tdr[r].first) pv[r] = __ldg(a.log_pi + jcol);
      }
    }

    // ---- multi-CTA clusters: rank 0 sends the jobs drawn in this tick's
    // prologue (they complete on this tick's barrier of every other CTA)
    if constexpr (CL > 1 && kExch != 0) {
      if (rank == 0 && tid < S && ((m_drw >> tid) & 1u)) {
        const PJob& pj = s_pend[tid][(slots[tid].ndraw - 1) & 1];
        const uint4* src = reinterpret_cast<const uint4*>(&pj);
#pragma unroll
        for (int r = 1; r < CL; ++r) {
          const uint32_t dst = dsmem_addr(&pj, r);
#pragma unroll
          for (int w = 0; w < (int)(sizeof(PJob) / 16); ++w) st_async_v4(dst + 16u * w, src[w], (tick & 1) ? pBar1[r] : pBar0[r]);
        }
      }
    }

    // ---- termination of jobs that finished last tick (rank 0)
    if (rank == 0 && m_trm) {
      for (int s = warp; s < S; s += NW) {
        if (!((m_trm >> s) & 1u)) continue;
        const SlotFin& fs = s_fin[s];
        const float* dl = sD + (cur * S + s) * KPS;
        if (kind == kJobVanilla) {
          // q_{T-1} = lowest argmax_j delta_{T-1}[j]; score = delta_{T-1}[q]
          float bv = -CUDART_INF_F;
          int bi = 0x7fffffff;
          for (int j = lane; j < K; j += 32) {
            const float v = dl[j + ((j >> 5) << 2)];
            if (bi == 0x7fffffff || v > bv) { bv = v; bi = j; }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi != 0x7fffffff && (bi == 0x7fffffff || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
          }
          if (lane == 0) {
            a.qlast[fs.b] = bi;
            a.scores[fs.b] = dl[bi + ((bi >> 5) << 2)];
          }
        } else if (!DEFER && kind == kJobSub && lane == 0) {
          // Alg. 2 output: q*_{tmid} = MidState[q*_n]; its delta from the snapshot
          const int tmid = (fs.m + fs.n) / 2;
          int q = sMid[(cur * S + s) * KP + ((unsigned)fs.q_n < (unsigned)K ? fs.q_n : 0)];
          q = (unsigned)q < (unsigned)K ? q : 0;
          a.paths[fs.path_off + tmid] = q;
          a.sval[fs.aux_off + tmid] = Cfg::GSNAP ? gSnap[s * KP + q] : sSnap[s * KP + q];
        }
      }
    }

    // ---- sub jobs: rank 0 keeps delta_{tmid} (all K states) as the snapshot
    if (kind == kJobSub && rank == 0 && m_snp) {
      for (int s = 0; s < S; ++s) {
        if (!((m_snp >> s) & 1u)) continue;
        const float* dl = sD + (cur * S + s) * KPS;
        float* dst = Cfg::GSNAP ? gSnap + s * KP : sSnap + s * KP;
        for (int j = tid; j < K; j += NT) dst[j] = dl[j + ((j >> 5) << 2)];
      }
    }

    // ---- merge: per output, the first warp whose partial is the maximum
    const int nxt = cur + 1 < NDB ? cur + 1 : 0;
    float best[OPT], val[OPT];
    int wbase[OPT], arg[OPT];
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      const int s = s0 + r * SSTEP;
      const float* pp = sPart + s * J + jj;
      float bv = pp[0];
      int wb = 0;
      if constexpr (STREAM) {
        const uint8_t* pc = sPC + s * J + jj;
        wb = pc[0];
#pragma unroll
        for (int w = 1; w < RG; ++w) {
          const float v = pp[w * S * J];
          if (v > bv) { bv = v; wb = pc[w * S * J]; }
        }
      } else {
#pragma unroll
        for (int w = 1; w < RG; ++w) {
          const float v = pp[w * S * J];
          if (v > bv) { bv = v; wb = w; }
        }
      }
      best[r] = bv;
      val[r] = bv;
      wbase[r] = wb * CH;
      arg[r] = wb * CH;
    }
    // ---- exact argmax: rows of the winning chunk, descending, so the last
    // match is the lowest row; the kept value is the recomputed candidate.
    // Deferred configurations run it right away only for a zero maximum
    // (its sign is the lowest maximising row's) and otherwise after the
    // tick's delta has been sent.
    auto rescan = [&]() {
      const float* dr[OPT];
      const float2* ar[OPT];
      const int64_t astr = STREAM ? a.ap_stride : J;
#pragma unroll
      for (int r = 0; r < OPT; ++r) {
        const int s = s0 + r * SSTEP;
        dr[r] = sD + (cur * S + s) * KPS + wbase[r] + ((wbase[r] >> 5) << 2);
        ar[r] = STREAM ? a.Ap + (int64_t)(wbase[r] / 2) * a.ap_stride + jcol : sA2 + (wbase[r] / 2) * J + jj;
      }
      if constexpr (STREAM) {
        // streamed: the chunk's CH weights into column jcol are contiguous
        // in the column-major copy (L2); two outputs' loads are in flight at
        // once, then compared row by row
        const int KD = wide_lane_stride(K);
#pragma unroll
        for (int r0 = 0; r0 < OPT; r0 += 2) {
          float4 a4[2][CH / 4];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            // the copy holds K columns: padded columns (unused outputs) are not read
            const float4* src = reinterpret_cast<const float4*>(a.wide_AT + (int64_t)(jcol < K ? jcol : 0) * KD +
                                                                wbase[r0 + u]);
#pragma unroll
            for (int k = 0; k < CH / 4; ++k) a4[u][k] = __ldg(src + k);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int r = r0 + u;
#pragma unroll
            for (int k = CH / 2 - 1; k >= 0; --k) {
              const float4 q = a4[u][k / 2];
              const float lo = (k & 1) ? q.z : q.x, hi = (k & 1) ? q.w : q.y;
              const unsigned long long av =
                  ((unsigned long long)__float_as_uint(hi) << 32) | (unsigned long long)__float_as_uint(lo);
              float c0, c1;
              fadd2(*reinterpret_cast<const unsigned long long*>(dr[r] + 2 * k), av, c0, c1);
              if (c1 == best[r]) { arg[r] = wbase[r] + 2 * k + 1; val[r] = c1; }
              if (c0 == best[r]) { arg[r] = wbase[r] + 2 * k; val[r] = c0; }
            }
          }
        }
      } else {
        // four rows per step; equal nonzero floats have equal bits, so only
        // the row is tracked and a zero maximum is recomputed at that row
        // for its sign
#pragma unroll
        for (int k4 = CH / 4 - 1; k4 >= 0; --k4) {
#pragma unroll
          for (int r = 0; r < OPT; ++r) {
            const float4 d4 = *reinterpret_cast<const float4*>(dr[r] + 4 * k4);
            const unsigned long long dlo =
                ((unsigned long long)__float_as_uint(d4.y) << 32) | (unsigned long long)__float_as_uint(d4.x);
            const unsigned long long dhi =
                ((unsigned long long)__float_as_uint(d4.w) << 32) | (unsigned long long)__float_as_uint(d4.z);
            float c0, c1, c2, c3;
            fadd2(dhi, *reinterpret_cast<const unsigned long long*>(ar[r] + (2 * k4 + 1) * astr), c2, c3);
            fadd2(dlo, *reinterpret_cast<const unsigned long long*>(ar[r] + (2 * k4) * astr), c0, c1);
            if (c3 == best[r]) arg[r] = wbase[r] + 4 * k4 + 3;
            if (c2 == best[r]) arg[r] = wbase[r] + 4 * k4 + 2;
            if (c1 == best[r]) arg[r] = wbase[r] + 4 * k4 + 1;
            if (c0 == best[r]) arg[r] = wbase[r] + 4 * k4;
          }
        }
#pragma unroll
        for (int r = 0; r < OPT; ++r) {
          if (best[r] == 0.0f) {
            const int o = arg[r] - wbase[r];
            const float2 ap = ar[r][(o >> 1) * astr];
            val[r] = __fadd_rn(dr[r][o], (o & 1) ? ap.y : ap.x);
          }
        }
      }
    };
    // streamed deferred configurations: the winning chunks' weights go into
    // this warp's ring slice (idle until the next tick's first copies; each
    // lane reads back only what it staged) with cp.async right after the
    // merge, so their L2 latency overlaps + E and the exchange
    static_assert(!(STREAM && DEFER) || OPT * CH * 32 <= NST * 4 * WC, "re-scan staging fits the warp's ring");
    auto stage_issue = [&]() {
      if constexpr (STREAM && DEFER) {
        float4* stg = reinterpret_cast<float4*>(ring);
        const float* colp = a.wide_AT + (int64_t)(jcol < K ? jcol : 0) * wide_lane_stride(K);
#pragma unroll
        for (int r = 0; r < OPT; ++r)
#pragma unroll
          for (int k = 0; k < CH / 4; ++k) cp_async16(stg + (r * (CH / 4) + k) * 32 + lane, colp + wbase[r] + 4 * k);
        cp_async_commit();
      }
    };
    auto stage_finish = [&]() {
      if constexpr (STREAM && DEFER) {
        cp_async_wait<0>();
        const float4* stg = reinterpret_cast<const float4*>(ring);
#pragma unroll
        for (int r = 0; r < OPT; ++r) {
          const int s = s0 + r * SSTEP;
          const float* dr = sD + (cur * S + s) * KPS + wbase[r] + ((wbase[r] >> 5) << 2);
#pragma unroll
          for (int k = CH / 2 - 1; k >= 0; --k) {
            const float4 q = stg[(r * (CH / 4) + k / 2) * 32 + lane];
            const float lo = (k & 1) ? q.z : q.x, hi = (k & 1) ? q.w : q.y;
            const unsigned long long av =
                ((unsigned long long)__float_as_uint(hi) << 32) | (unsigned long long)__float_as_uint(lo);
            float c0, c1;
            fadd2(*reinterpret_cast<const unsigned long long*>(dr + 2 * k), av, c0, c1);
            if (c1 == best[r]) { arg[r] = wbase[r] + 2 * k + 1; val[r] = c1; }
            if (c0 == best[r]) { arg[r] = wbase[r] + 2 * k; val[r] = c0; }
          }
        }
      }
    };
    bool rescanned = false;
    if constexpr (DEFER) {
      bool zero = false;
#pragma unroll
      for (int r = 0; r < OPT; ++r) zero |= best[r] == 0.0f;
      if (zero) {
        rescan();
        rescanned = true;
      } else {
        stage_issue();
      }
    } else {
      rescan();
    }

    // ---- + E, per-kind bookkeeping, delta_t to every CTA.  Global stores
    // (psi, root maps and snapshots) are kept in registers and issued after
    // the exchange has been started.
    int st_arg[OPT], st_mid[OPT];
    float st_val[OPT];
    int64_t st_off[OPT], st_moff[OPT];
    uint32_t st_mask = 0;  // bit 2r: psi store, bit 2r+1: root snapshot (+ map)
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      const int s = s0 + r * SSTEP;
      const TickDesc& td = tdr[r];
      st_arg[r] = 0;
      st_mid[r] = 0;
      st_val[r] = 0.f;
      st_off[r] = 0;
      st_moff[r] = -1;
      if (!td.mode || jcol >= K) continue;
      float dval;
      int ag = 0;
      if (td.mode == 1) {
        if (td.first) {
          dval = __fadd_rn(pv[r], ev[r]);
        } else if (a.ckpt) {
          // checkpoint restart: delta_m exactly as the forward pass stored it
          dval = __ldg(a.snaps + td.snap_row + jcol);
        } else {
          // pruned start (Sec. V-B.2): only transitions out of q*_{m-1}
          const float av = STREAM ? __ldg(a.logA + (int64_t)td.q_prev * K + jcol)
                                  : sA[((td.q_prev >> 1) * J + jj) * 2 + (td.q_prev & 1)];
          dval = a.complete ? __fadd_rn(av, ev[r]) : __fadd_rn(__fadd_rn(td.s_prev, av), ev[r]);
        }
      } else {
        ag = arg[r] < K ? arg[r] : 0;  // only NaN inputs (unsupported) could leave it on a padded row
        if (kind == kJobVanilla || kind == kJobLeaf) {
          st_mask |= 1u << (2 * r);
          st_arg[r] = ag;
          st_off[r] = td.psi_row + jcol;
        }
        dval = __fadd_rn(val[r], ev[r]);
      }
      if (!DEFER && td.f_mid) {
        const uint16_t mnew = td.f_mid == 1 ? (uint16_t)ag : sMid[(cur * S + s) * KP + ag];
        const int mo = (nxt * S + s) * KP + jcol;
        sMid[mo] = mnew;
        st_mid[r] = mnew;
      }
      if (td.f_snap && kind == kJobRoot) {
        st_mask |= 1u << (2 * r + 1);
        st_val[r] = dval;
        st_off[r] = td.snap_row + jcol;
        st_moff[r] = td.map_row >= 0 ? td.map_row + jcol : -1;
      }
      sD[(nxt * S + s) * KPS + jcol + ((jcol >> 5) << 2)] = dval;
    }
    if constexpr (CL > 1 && kExch == 0) {
      // delta_t (and MidState) to the other CTAs with plain remote stores,
      // then the cluster barrier of this tick
      __syncwarp();
      const int wcol = j0 + (tid % J) - lane;  // first column of this warp
#pragma unroll
      for (int r0 = 0; r0 < OPT; r0 += 4) {
        const int r = r0 + lane / 8;
        const int s = s0 + r * SSTEP;
        if (r < OPT && ((m_act >> s) & 1u)) {
          const int c4 = wcol + 4 * (lane % 8);
          const int dof = (nxt * S + s) * KPS + c4 + ((c4 >> 5) << 2);
          const float4 v = *reinterpret_cast<const float4*>(sD + dof);
#pragma unroll
          for (int rr = 0; rr < CL; ++rr)
            if (rr != (int)rank) dsmem_st_v4f32(pD[rr] + 4u * dof, v.x, v.y, v.z, v.w);
        }
      }
      if (!DEFER && m_mid) {
#pragma unroll
        for (int r0 = 0; r0 < OPT; r0 += 8) {
          const int r = r0 + lane / 4;
          const int s = s0 + r * SSTEP;
          if (r < OPT && ((m_mid >> s) & 1u)) {
            const int mo = (nxt * S + s) * KP + wcol + 8 * (lane % 4);
            const float4 v = *reinterpret_cast<const float4*>(sMid + mo);
#pragma unroll
            for (int rr = 0; rr < CL; ++rr)
              if (rr != (int)rank) dsmem_st_v4f32(pMid[rr] + 2u * mo, v.x, v.y, v.z, v.w);
          }
        }
      }
      cluster_arrive_release();
    } else if constexpr (CL > 1) {
      // this warp's local writes are done: arrive on this tick's barrier
      // (warp 0 also announces the bytes the other CTAs will store here)
      __syncwarp();
      const int tb = tick & 1;
      // test hook: CTA 1 of every cluster withholds its arrivals of the
      // second tick, so the bounded waits run out (FV_TEST_WITHHOLD_STEP)
      const bool withhold = a.wide_withhold && rank == 1 && tick == 1;
      if (lane == 0 && !withhold) {
        const uint32_t bar = smem_addr(&s_bar[tb]);
        if (warp == 0) {
          const uint32_t bytes =
              (uint32_t)(CL - 1) * (uint32_t)(__popc(m_act) * J * 4 + __popc(m_mid) * J * 2) +
              (rank != 0 ? (uint32_t)__popc(m_drw) * (uint32_t)sizeof(PJob) : 0u);
          mbar_arrive_expect_tx(bar, bytes);
        } else {
          mbar_arrive(bar);
        }
      }
      const int wcol = j0 + (tid % J) - lane;  // first column of this warp
      // the warp's 32 columns of delta_t (and of MidState when set) to the
      // other CTAs, 16 bytes per store
#pragma unroll
      for (int r0 = 0; r0 < OPT; r0 += 4) {
        const int r = r0 + lane / 8;
        const int s = s0 + r * SSTEP;
        if (r < OPT && ((m_act >> s) & 1u)) {
          const int c4 = wcol + 4 * (lane % 8);
          const int dof = (nxt * S + s) * KPS + c4 + ((c4 >> 5) << 2);
          const uint4 v = *reinterpret_cast<const uint4*>(sD + dof);
#pragma unroll
          for (int rr = 0; rr < CL; ++rr)
            if (rr != (int)rank) st_async_v4(pD[rr] + 4u * dof, v, (tb ? pBar1[rr] : pBar0[rr]));
        }
      }
      if (!DEFER && m_mid) {
#pragma unroll
        for (int r0 = 0; r0 < OPT; r0 += 8) {
          const int r = r0 + lane / 4;
          const int s = s0 + r * SSTEP;
          if (r < OPT && ((m_mid >> s) & 1u)) {
            const int mo = (nxt * S + s) * KP + wcol + 8 * (lane % 4);
            const uint4 v = *reinterpret_cast<const uint4*>(sMid + mo);
#pragma unroll
            for (int rr = 0; rr < CL; ++rr)
              if (rr != (int)rank) st_async_v4(pMid[rr] + 2u * mo, v, (tb ? pBar1[rr] : pBar0[rr]));
          }
        }
      }
    } else {
      __syncthreads();
    }
    if constexpr (DEFER) {
      // the deferred re-scan (delta_t is on its way to the other CTAs);
      // staged copies are always waited for before the ring is reused
      uint32_t psi_bits = 0;
#pragma unroll
      for (int r = 0; r < OPT; ++r) psi_bits |= st_mask & (1u << (2 * r));
      if (!rescanned) {
        if constexpr (STREAM) {
          stage_finish();
        } else {
          if (psi_bits) rescan();
        }
      }
#pragma unroll
      for (int r = 0; r < OPT; ++r)
        if (st_mask & (1u << (2 * r))) st_arg[r] = arg[r] < K ? arg[r] : 0;
      if constexpr (STREAM) __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
      if (st_mask & (1u << (2 * r))) a.psi[st_off[r]] = (uint16_t)st_arg[r];
      if (st_mask & (1u << (2 * r + 1))) {
        a.snaps[st_off[r]] = st_val[r];
        if (st_moff[r] >= 0) a.maps[st_moff[r]] = (uint16_t)st_mid[r];
      }
    }
    if constexpr (CL > 1 && kExch == 0) cluster_wait_acquire();
    cur = nxt;
  }
  if constexpr (CL > 1) {
    // the last tick's stores from the other CTAs land before anyone leaves
    if (kExch != 0 && tick > 0) {
      const uint32_t bar = smem_addr(&s_bar[(tick - 1) & 1]);
      const uint32_t par = (uint32_t)((tick - 1) >> 1) & 1u;
      const long long w0 = clock64();
      while (!mbar_try_wait_cluster(bar, par))
        if (clock64() - w0 > kClusterWaitCycles) {
          set_status(a.hdr, FV_ETIMEOUT, 3);
          break;
        }
    }
    cluster_sync_all();
  }
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
template <int J, int S, int NW, int CL, int KPM, bool STREAM, int TW = 8, bool DEFER = false, int MINB = 1>
static cudaError_t launch_dense_cfg(DenseArgs a, int max_clusters, cudaStream_t st) {
  using Cfg = DenseCfg<J, S, NW, CL, KPM, STREAM, TW, DEFER, MINB>;
  auto kern = dense_fwd_kernel<J, S, NW, CL, KPM, STREAM, TW, DEFER, MINB>;
  a.KP = KPM;
  const size_t smem = Cfg::smem_bytes;
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

int device_sm_count() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;  // no device visible (sizing on a host without a GPU): GB300's count
  }
  return nsm;
}

// Jobs the engine runs at once for K's class (default configuration; for
// K <= 128, whose default is the one-CTA-per-job small-K engine, the slot
// engine's 16-warp configuration): resident clusters x slots; 0 when no
// device is visible.  It sizes the waves of budget leaves, which any engine
// runs in any order.
template <int J, int S, int NW, int CL, int KPM, bool STREAM, int TW = 8, int MINB = 1>
static int dense_cfg_slots() {
  static int cached = -1;
  if (cached >= 0) return cached;
  using Cfg = DenseCfg<J, S, NW, CL, KPM, STREAM, TW, false, MINB>;
  auto kern = dense_fwd_kernel<J, S, NW, CL, KPM, STREAM, TW, false, MINB>;
  int dev = 0, nsm = 0, resident = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return cached = 0;
  }
  if (CL > 1) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL * nsm);
    cfg.blockDim = dim3(Cfg::NT);
    cfg.dynamicSmemBytes = Cfg::smem_bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&resident, kern, &cfg) != cudaSuccess) resident = 0;
  } else {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::NT, Cfg::smem_bytes) != cudaSuccess) per_sm = 0;
    resident = per_sm * nsm;
  }
  cudaGetLastError();
  return cached = resident * S;
}

int dense_job_slots(int K) {
  if (K > 1024) return kWideLanes;
  if (K <= 64) return dense_cfg_slots<64, 16, 16, 1, 64, false, 4>();
  if (K <= 128) return dense_cfg_slots<128, 8, 16, 1, 128, false, 4>();
  if (K <= 256) return dense_cfg_slots<64, 8, 8, 4, 256, false, 4, 2>();
  if (K <= 512) return dense_cfg_slots<64, 8, 16, 8, 512, false, 4>();
  return dense_cfg_slots<128, 4, 8, 8, 1024, true, 4, 2>();
}

int dense_supported_K(int K) {
  if (K >= 1 && K <= 1024) return 1;
  WideGeom g;
  return wide_geometry(K, device_sm_count(), &g) ? 1 : 0;
}

// Streamed configurations (K > 256) read logA from a row-pair copy
// Ap[i/2][c] = (A[i][c], A[i+1][c]), rows padded to the configuration's row
// count and columns to cluster x 128, padding -inf.
void dense_stream_geometry(int K, int* KPM, int* cols) {
  if (K <= 256) { *KPM = 0; *cols = 0; return; }
  if (K > 1024) {
    WideGeom g;
    if (!wide_geometry(K, device_sm_count(), &g)) { *KPM = 0; *cols = 0; return; }
    *KPM = g.KR;
    *cols = g.NCB * 128;
    return;
  }
  if (K <= 512) { *KPM = 512; *cols = 512; return; }
  *KPM = 1024;
  *cols = 1024;
}

__global__ void ap_prep_kernel(const float* logA, int K, int KPM, int cols, float2* Ap) {
  const int64_t n = (int64_t)(KPM / 2) * cols;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int ip = (int)(x / cols), c = (int)(x % cols), i = 2 * ip;
    const float lo = (i < K && c < K) ? logA[(int64_t)i * K + c] : -CUDART_INF_F;
    const float hi = (i + 1 < K && c < K) ? logA[(int64_t)(i + 1) * K + c] : -CUDART_INF_F;
    Ap[x] = make_float2(lo, hi);
  }
}

cudaError_t launch_ap_prep(const float* logA, int K, float2* Ap, cudaStream_t st) {
  int KPM, cols;
  dense_stream_geometry(K, &KPM, &cols);
  if (!KPM) return cudaSuccess;
  ap_prep_kernel<<<1024, 256, 0, st>>>(logA, K, KPM, cols, Ap);
  return cudaGetLastError();
}

// Rows padded to a multiple of 4 * NW for the chosen configuration.
// Engine configurations per K class (variant 0 is the default).  Every
// variant computes the same values in the same order, so the choice only
// changes speed: warps per CTA and columns per lane (TW) for the resident
// classes, ring depth for the streamed ones is fixed.
int dense_k_class(int K) {
  if (K <= 64) return 0;
  if (K <= 128) return 1;
  if (K <= 256) return 2;
  if (K <= 512) return 3;
  if (K <= 1024) return 4;
  return 5;  // whole-GPU engine
}
int dense_variants(int K) {
  switch (dense_k_class(K)) {
    case 0: return 4;
    case 1: return 3;
    case 2: return 4;
    case 3: return 3;
    case 4: return 4;
    default: return 1;
  }
}

static int g_variant[6] = {0, 0, 0, 0, 0, 0};  // chosen by fv_autotune

void dense_set_variant(int K, int v) {
  const int c = dense_k_class(K);
  g_variant[c] = (v >= 0 && v < dense_variants(K)) ? v : 0;
}
int dense_get_variant(int K) { return g_variant[dense_k_class(K)]; }

cudaError_t launch_dense_forward(DenseArgs a, int max_clusters, cudaStream_t st) {
  if (a.K > 1024) return launch_wide_forward(a, st);
  const int v = a.no_tune ? 0 : g_variant[dense_k_class(a.K)];
  if (a.K <= 64) {
    if (v == 1) return launch_dense_cfg<64, 16, 8, 1, 64, false, 4>(a, max_clusters, st);
    if (v == 2) return launch_dense_cfg<64, 16, 16, 1, 64, false, 4>(a, max_clusters, st);
    if (v == 3) return launch_dense_cfg<64, 16, 4, 1, 64, false>(a, max_clusters, st);
    // default: the one-CTA-per-job small-K engine (fv_small.cu; measured
    // 3.4x faster on one K=64 sequence and 3.3x on 1024)
    return launch_small_forward(a, st);
  }
  if (a.K <= 128) {
    if (v == 1) return launch_dense_cfg<128, 8, 8, 1, 128, false>(a, max_clusters, st);
    if (v == 2) return launch_dense_cfg<128, 8, 16, 1, 128, false, 4>(a, max_clusters, st);
    // default: the small-K engine (measured 3.9x faster on one K=128
    // sequence, 1.7x on 1024)
    return launch_small_forward(a, st);
  }
  // jobs without MidState (exact decoding with psi rows, budget leaves,
  // checkpoint passes) on the 8-CTA configurations defer the re-scan past
  // the delta exchange (measured: 8% less time at K=512; with the 2-CTA
  // cluster barrier of K <= 256 it was 1-2% slower, not used)
  const bool defer = a.kind == kJobVanilla || a.kind == kJobLeaf || (a.kind == kJobRoot && a.ckpt);
  if (a.K <= 256) {
    // default: 4-CTA clusters of 64 columns, two CTAs per SM (measured 3%
    // ahead of the best 2-CTA configuration on 1024 sequences)
    if (v == 3) return launch_dense_cfg<128, 8, 16, 2, 256, false, 4>(a, max_clusters, st);
    if (v == 2) return launch_dense_cfg<128, 8, 16, 2, 256, false, 8>(a, max_clusters, st);
    if (v == 1) return launch_dense_cfg<128, 8, 8, 2, 256, false>(a, max_clusters, st);
    if (defer) return launch_dense_cfg<64, 8, 8, 4, 256, false, 4, true, 2>(a, max_clusters, st);
    return launch_dense_cfg<64, 8, 8, 4, 256, false, 4, false, 2>(a, max_clusters, st);
  }
  if (a.K <= 512) {
    // default: 8-CTA clusters of 64 columns each, so every CTA's slab of
    // logA (512 rows x 64 columns) stays in shared memory (measured: half
    // the time of the streamed 4-CTA configurations, 256 sequences);
    // variants 1 and 2 stream 128-column slabs from L2
    if (v == 2) return launch_dense_cfg<128, 8, 16, 4, 512, true, 4>(a, max_clusters, st);
    if (v == 1) return launch_dense_cfg<128, 8, 8, 4, 512, true>(a, max_clusters, st);
    if (defer) return launch_dense_cfg<64, 8, 16, 8, 512, false, 4, true>(a, max_clusters, st);
    return launch_dense_cfg<64, 8, 16, 8, 512, false, 4>(a, max_clusters, st);
  }
  if (v == 3) {
    if (defer) return launch_dense_cfg<128, 4, 4, 8, 1024, true, 4, true, 2>(a, max_clusters, st);
    return launch_dense_cfg<128, 4, 4, 8, 1024, true, 4, false, 2>(a, max_clusters, st);
  }
  if (v == 2) {
    if (defer) return launch_dense_cfg<128, 8, 8, 8, 1024, true, 8, true>(a, max_clusters, st);
    return launch_dense_cfg<128, 8, 8, 8, 1024, true>(a, max_clusters, st);
  }
  if (v == 1) {
    if (defer) return launch_dense_cfg<128, 8, 16, 8, 1024, true, 4, true>(a, max_clusters, st);
    return launch_dense_cfg<128, 8, 16, 8, 1024, true, 4>(a, max_clusters, st);
  }
  // default: 4 slots and 8 warps per CTA, a 2-stage ring, two CTAs per SM
  // (about the slot count of 8 slots on one CTA per SM; measured on 256
  // sequences: 67 ms, against 73 ms with 4 warps and a 4-stage ring and 83
  // ms for one 8-slot CTA per SM)
  if (defer) return launch_dense_cfg<128, 4, 8, 8, 1024, true, 4, true, 2>(a, max_clusters, st);
  return launch_dense_cfg<128, 4, 8, 8, 1024, true, 4, false, 2>(a, max_clusters, st);
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
