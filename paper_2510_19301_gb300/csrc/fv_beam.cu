// fv_beam.cu -- dynamic beam search (Sec. V-C) and FLASH-BS on GB300.
//
// One CTA (1024 threads; 128 or 256 for small dense steps) runs one job at
// a time (a whole sequence, or one Alg. 1 segment task) and pops the next
// job from a global counter.  Beams of at least 64 states on large CSR state
// spaces (P = 0) instead spread each sequence over a cluster of CTAs
// (beam_csr_cluster_kernel, below), and so do dense beams with
// 512 <= K <= 8192 (P = 0; beam_dense_cluster_kernel).  Dense beams with
// K <= 128 (P = 0) run small_beam_kernel, one CTA of a thread per state
// holding its transition column in registers.  A beam
// is the top-B finite candidates under (score desc, state id asc); it is
// kept sorted by state id so that the next step visits its sources in
// ascending order.  Per step:
//  * candidates: every target reachable from the beam gets its best source
//    (lowest id on equal scores).  Dense transitions: one thread per target
//    scans the beam in id order.  CSR transitions: one warp per beam entry
//    scatters 64-bit keys (order-preserving score << 32 | ~slot) with
//    atomicMax, so equal scores resolve to the lowest slot (= lowest id);
//    the winning candidate value is then recomputed exactly.  A shared
//    bitmap records the touched targets.
//  * c_j = fl(M_j + E_t[j]); exact top-B: 4-pass MSB radix select on the
//    order-preserving 32-bit key (-0 folded into +0), then the keys equal
//    to the threshold are taken lowest id first (block scan in id order).
//    K <= 256 with candidates in shared memory uses a rank select instead;
//    CSR steps list their touched candidates in shared memory when they fit.
// Beams and candidates live in shared memory when they fit (they are
// re-read several times per step), else in a per-CTA slice of the
// workspace; CSR scatter keys always live in the workspace.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <algorithm>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

constexpr int kBeamThreads = 1024;

// Order-preserving map of a float to uint32 (larger float -> larger key);
// -0 is folded into +0 so that signed zeros tie and resolve by id.
__device__ inline uint32_t ord_key(float x) {
  uint32_t u = __float_as_uint(x);
  if (u == 0x80000000u) u = 0u;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Inverse of ord_key (zero comes back as +0).
__device__ inline float ord_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ inline int block_sum(int v, int* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int s = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  __syncthreads();
  return s;
}

// Exclusive block scan of v (thread order), returns the prefix; *total.
__device__ inline int block_scan(int v, int* red, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    red[lane] = s;
  }
  __syncthreads();
  const int excl = (w ? red[w - 1] : 0) + x - v;
  *total = red[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

// csr weight of edge i -> j (max over duplicates), -inf if absent
__device__ inline float beam_csr_w(const BeamArgs& a, int i, int j) {
  int lo = a.row_ptr[i], hi = a.row_ptr[i + 1] - 1;
  const int r0 = a.row_ptr[i], r1 = a.row_ptr[i + 1];
  while (lo <= hi) {
    const int md = (lo + hi) >> 1;
    const int c = a.col[md];
    if (c < j) lo = md + 1;
    else if (c > j) hi = md - 1;
    else {
      int k = md;
      while (k > r0 && a.col[k - 1] == j) --k;
      float best = -CUDART_INF_F;
      for (; k < r1 && a.col[k] == j; ++k) best = fmaxf(best, a.val[k]);
      return best;
    }
  }
  return -CUDART_INF_F;
}

__device__ inline float beam_trans(const BeamArgs& a, int i, int j) {
  return a.trans == FV_TRANS_DENSE ? __ldg(a.logA + (int64_t)i * a.K + j) : beam_csr_w(a, i, j);
}

__device__ inline float beam_emit(const BeamArgs& a, const Job& jb, int t, int j) {
  if (a.emit == FV_EMIT_DENSE) return __ldg(a.E + jb.e_off + (int64_t)t * a.K + j);
  return __ldg(a.logB + (int64_t)j * a.V + __ldg(a.obs + jb.e_off + t));
}

// Per-CTA scratch slice.
struct BeamScratch {
  float* cval;               // [K] candidate c_j
  int32_t* cslot;            // [K] source slot in the previous beam (-1: none)
  unsigned long long* keys;  // [K] CSR scatter keys (0 = untouched)
  int32_t* id[2];            // [Bcap] beam state ids (sorted)
  float* val[2];             // [Bcap] beam scores
  int32_t* mid[2];           // [Bcap] MidState of each entry
  int32_t* src[2];           // [Bcap] source slot of each entry (previous beam)
  int32_t* snap_id;          // [Bcap] subtask: beam at t_mid
  float* snap_val;           // [Bcap]
};

// Shared-memory words of the touched bitmap, rounded to 16 bytes.
__host__ __device__ inline size_t beam_bitmap_words(int K) { return (size_t)(((K + 31) / 32 + 3) / 4 * 4); }

__device__ inline BeamScratch beam_scratch(const BeamArgs& a, uint32_t* smem) {
  BeamScratch s;
  char* base = reinterpret_cast<char*>(a.scratch) + (size_t)blockIdx.x * a.scratch_stride;
  const size_t K = (size_t)a.K, B = (size_t)a.Bcap;
  s.keys = reinterpret_cast<unsigned long long*>(base);
  base += align_up(K * 8);
  s.cval = reinterpret_cast<float*>(base);
  base += align_up(K * 4);
  s.cslot = reinterpret_cast<int32_t*>(base);
  base += align_up(K * 4);
  for (int p = 0; p < 2; ++p) {
    s.id[p] = reinterpret_cast<int32_t*>(base);
    base += align_up(B * 4);
    s.val[p] = reinterpret_cast<float*>(base);
    base += align_up(B * 4);
    s.mid[p] = reinterpret_cast<int32_t*>(base);
    base += align_up(B * 4);
    s.src[p] = reinterpret_cast<int32_t*>(base);
    base += align_up(B * 4);
  }
  s.snap_id = reinterpret_cast<int32_t*>(base);
  base += align_up(B * 4);
  s.snap_val = reinterpret_cast<float*>(base);
  // shared-memory homes (after the bitmap): beams, then candidates
  uint32_t* sp = smem + beam_bitmap_words(a.K);
  if (a.beam_smem) {
    for (int p = 0; p < 2; ++p) {
      s.id[p] = reinterpret_cast<int32_t*>(sp);
      sp += B;
      s.val[p] = reinterpret_cast<float*>(sp);
      sp += B;
      s.mid[p] = reinterpret_cast<int32_t*>(sp);
      sp += B;
      s.src[p] = reinterpret_cast<int32_t*>(sp);
      sp += B;
    }
    s.snap_id = reinterpret_cast<int32_t*>(sp);
    sp += B;
    s.snap_val = reinterpret_cast<float*>(sp);
    sp += B;
  }
  if (a.cand_smem) {
    s.cval = reinterpret_cast<float*>(sp);
    sp += K;
    s.cslot = reinterpret_cast<int32_t*>(sp);
  }
  return s;
}

size_t beam_scratch_stride(int K, int Bcap) {
  const size_t k = (size_t)K, b = (size_t)Bcap;
  return align_up(k * 8) + 2 * align_up(k * 4) + 10 * align_up(b * 4);
}

struct BeamSmem {
  uint32_t* touched;  // [ceil(K/32)]
  int* red;           // [32]
  int* hist;          // [256]
  int* misc;          // [8]
  uint32_t* lkey;     // [list_cap] ordered keys of this step's touched candidates (0: not finite)
  int32_t* lj;        // [list_cap] their state ids, ascending
  int nlist;          // entries in the list this step, -1 when the list is not in use
  int nlist_used;     // entries listed in this step (kept for clearing the keys), -1 if none
};

// Calls f(j) for every touched target j of this thread's contiguous range
// [j0, j1) of the state ids, in ascending j.
template <class F>
__device__ inline void for_touched(const BeamSmem& sm, int j0, int j1, F&& f) {
  for (int j = j0; j < j1;) {
    const int w = j >> 5, wend = min(j1, (w + 1) << 5);
    const int lo = j & 31, hi = wend - (w << 5);
    uint32_t bits = sm.touched[w] & (0xffffffffu << lo);
    if (hi < 32) bits &= (1u << hi) - 1u;
    while (bits) {
      const int jj = (w << 5) + __ffs(bits) - 1;
      bits &= bits - 1;
      f(jj);
    }
    j = wend;
  }
}

// Small state spaces (K <= kBeamRankK, candidates in shared memory): thread
// j owns candidate j, and its rank under (score desc, id asc) counts the
// finite candidates ahead of it in one broadcast loop over the K scores;
// the W first (every finite one when there are at most W) are written in id
// order after one block scan.  Same result as the radix select below.
constexpr int kBeamRankK = 256;

__device__ int select_top_b_rank(const BeamArgs& a, BeamScratch& S, BeamSmem& sm, int p, int W, int need_mid) {
  const int K = a.K, j = threadIdx.x;
  const bool mine = j < K && ((sm.touched[j >> 5] >> (j & 31)) & 1u) && isfinite(S.cval[j]);
  const float c = mine ? S.cval[j] : 0.f;
  const uint32_t key = mine ? ord_key(c) : 0u;
  const int n_fin = K <= W ? 0 : block_sum(mine ? 1 : 0, sm.red);  // every candidate fits when K <= W
  bool take = mine;
  if (n_fin > W && mine) {
    int rank = 0;
    for (int w = 0; w < ((K + 31) >> 5); ++w) {
      const uint32_t bits = sm.touched[w];
#pragma unroll 8
      for (int u = 0; u < 32; ++u) {
        const int i = (w << 5) + u;
        if (i >= K) break;
        const float ci = S.cval[i];
        const uint32_t ui = ord_key(ci);
        const bool ahead = ((bits >> u) & 1u) && isfinite(ci) && (ui > key || (ui == key && i < j));
        rank += ahead ? 1 : 0;
      }
    }
    take = rank < W;
  }
  int tot;
  const int o = block_scan(take ? 1 : 0, sm.red, &tot);
  if (take) {
    const int sl = S.cslot[j];
    S.id[p][o] = j;
    S.val[p][o] = c;
    S.src[p][o] = sl;
    if (need_mid == 1) S.mid[p][o] = S.id[p ^ 1][sl];
    else if (need_mid == 2) S.mid[p][o] = S.mid[p ^ 1][sl];
    else S.mid[p][o] = -1;
  }
  __syncthreads();
  return tot;
}

// Top-B of the candidates (finite only) -> beam buffer p, in id order, by a
// 4-pass MSB radix select on the ordered keys.  each(f) calls f(j, key) for
// this thread's candidates in ascending id (key 0: not finite), and the
// threads' candidate sets are ascending ranges in thread order, so the final
// compaction in thread order is id order.  any(f) visits the same
// candidates split among the threads in any way (the counting passes do
// not depend on order).  Returns the beam size (identical in every thread).
template <class Any, class Each>
__device__ int select_core(const BeamArgs& a, BeamScratch& S, BeamSmem& sm, int p, int W, int need_mid, Any any,
                           Each each) {
  const int tid = threadIdx.x, lane = tid & 31;
  // every candidate fits when K <= W; else count the finite ones
  bool all = a.K <= W;
  if (!all) {
    int cnt = 0;
    any([&](int, uint32_t u) { cnt += u ? 1 : 0; });
    all = block_sum(cnt, sm.red) <= W;
  }
  uint32_t thr = 0u;
  int need_eq = 0;
  if (!all) {
    uint32_t prefix = 0u, mask = 0u;
    int remaining = W;
    for (int shift = 24; shift >= 0; shift -= 8) {
      for (int k = tid; k < 256; k += blockDim.x) sm.hist[k] = 0;
      __syncthreads();
      any([&](int, uint32_t u) {
        if (u && (u & mask) == prefix) atomicAdd(&sm.hist[(u >> shift) & 0xFFu], 1);
      });
      __syncthreads();
      // the digit where the count from the top reaches `remaining`: lane l
      // holds digits 255-8l .. 248-8l, a warp scan finds the lane, the lane
      // its digit
      if (tid < 32) {
        int h[8], sum = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          h[u] = sm.hist[255 - 8 * lane - u];
          sum += h[u];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int excl = incl - sum;
        if (excl < remaining && remaining <= incl) {
          int acc = excl, d = 255 - 8 * lane - 7;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (acc + h[u] >= remaining) { d = 255 - 8 * lane - u; break; }
            acc += h[u];
          }
          sm.misc[0] = d;
          sm.misc[1] = remaining - acc;
        }
      }
      __syncthreads();
      prefix |= (uint32_t)sm.misc[0] << shift;
      mask |= 0xFFu << shift;
      remaining = sm.misc[1];
      __syncthreads();
    }
    thr = prefix;
    need_eq = remaining;  // keys == thr to take, lowest ids first
  }
  int n_gt = 0, n_eq = 0;
  each([&](int, uint32_t u) {
    if (!u) return;
    if (all || u > thr) ++n_gt;
    else if (u == thr) ++n_eq;
  });
  int tot_eq, tot;
  const int eq_before = block_scan(n_eq, sm.red, &tot_eq);
  const int take_eq = min(max(need_eq - eq_before, 0), n_eq);
  const int pos = block_scan(n_gt + take_eq, sm.red, &tot);
  int o = pos, eq_seen = 0;
  each([&](int j, uint32_t u) {
    if (!u) return;
    bool take = all || u > thr;
    if (!take && u == thr) take = (eq_seen++ < take_eq);
    if (!take) return;
    const int sl = S.cslot[j];
    S.id[p][o] = j;
    S.val[p][o] = S.cval[j];
    S.src[p][o] = sl;
    if (need_mid == 1) S.mid[p][o] = S.id[p ^ 1][sl];
    else if (need_mid == 2) S.mid[p][o] = S.mid[p ^ 1][sl];
    else S.mid[p][o] = -1;
    ++o;
  });
  __syncthreads();
  return tot;
}

__device__ int select_top_b(const BeamArgs& a, BeamScratch& S, BeamSmem& sm, int p, int W, int need_mid) {
  if (a.cand_smem && a.K <= kBeamRankK && a.K <= (int)blockDim.x) return select_top_b_rank(a, S, sm, p, W, need_mid);
  if (sm.nlist >= 0) {
    // this step's touched candidates are listed in shared memory: each
    // thread takes a contiguous piece of the (id-ordered) list
    const int n = sm.nlist, per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int e0 = min(n, (int)threadIdx.x * per), e1 = min(n, e0 + per);
    const uint32_t* lkey = sm.lkey;
    const int32_t* lj = sm.lj;
    sm.nlist = -1;
    auto list = [&](auto&& f) {
      for (int e = e0; e < e1; ++e) f(lj[e], lkey[e]);
    };
    return select_core(a, S, sm, p, W, need_mid, list, list);
  }
  const int K = a.K;
  const int per = (K + (int)blockDim.x - 1) / (int)blockDim.x;
  const int j0 = min(K, (int)threadIdx.x * per), j1 = min(K, j0 + per);
  // counting passes: ids strided over the block, so a warp reads
  // consecutive candidates; the compaction keeps the contiguous ranges
  return select_core(
      a, S, sm, p, W, need_mid,
      [&](auto&& f) {
        for (int j = threadIdx.x; j < K; j += blockDim.x) {
          if (!((sm.touched[j >> 5] >> (j & 31)) & 1u)) continue;
          const float c = S.cval[j];
          f(j, isfinite(c) ? ord_key(c) : 0u);
        }
      },
      [&](auto&& f) {
        for_touched(sm, j0, j1, [&](int j) {
          const float c = S.cval[j];
          f(j, isfinite(c) ? ord_key(c) : 0u);
        });
      });
}

// Clear the touched bitmap (and CSR keys of touched targets).
__device__ inline void clear_candidates(const BeamArgs& a, BeamScratch& S, BeamSmem& sm) {
  const int nw = (a.K + 31) >> 5;
  if (a.trans != FV_TRANS_DENSE) {
    if (sm.nlist_used > 0) {
      for (int e = threadIdx.x; e < sm.nlist_used; e += blockDim.x) S.keys[sm.lj[e]] = 0ull;
    } else {
      for (int j = threadIdx.x; j < a.K; j += blockDim.x)
        if ((sm.touched[j >> 5] >> (j & 31)) & 1u) S.keys[j] = 0ull;
    }
    __syncthreads();
  }
  for (int w = threadIdx.x; w < nw; w += blockDim.x) sm.touched[w] = 0u;
  __syncthreads();
}

// Static beam: the step's full K-entry score vector -- -inf (and no
// source) for every state no beam state leads to -- and every state marked
// as an entry, so the top-B select reads all K scores.
__device__ inline void static_full_vector(const BeamArgs& a, BeamScratch& S, BeamSmem& sm) {
  sm.nlist = -1;
  for (int j = threadIdx.x; j < a.K; j += blockDim.x)
    if (!((sm.touched[j >> 5] >> (j & 31)) & 1u)) {
      S.cval[j] = -CUDART_INF_F;
      S.cslot[j] = -1;
    }
  __syncthreads();
  for (int w = threadIdx.x; w < ((a.K + 31) >> 5); w += blockDim.x)
    sm.touched[w] = (w == (a.K >> 5)) ? ((1u << (a.K & 31)) - 1u) : 0xffffffffu;
  __syncthreads();
}

// Candidates of step t from beam buffer p (size nb) into cval/cslot/touched.
__device__ void beam_candidates(const BeamArgs& a, BeamScratch& S, BeamSmem& sm, const Job& jb, int p, int nb, int t) {
  const int K = a.K;
  sm.nlist = -1;
  sm.nlist_used = -1;
  if (a.trans == FV_TRANS_DENSE && 2 * K > (int)blockDim.x && (K & 3) == 0 && ((uintptr_t)a.logA & 15u) == 0) {
    // large K (more than one target per two threads): four adjacent targets
    // per thread (16-byte loads of logA rows); G threads per group of four
    // split the beam by slot residue and combine per target: highest value,
    // lowest slot on ties.  Measured: 22% less time per candidate step at
    // K=1024, B=256; slower for smaller K, where the scalar path below
    // already splits each target's sources over several threads
    const int K4 = K >> 2;
    int G = 1;
    while (G < 32 && 2 * G * K4 <= (int)blockDim.x) G *= 2;
    const int groups = (int)blockDim.x / G, sub = (int)threadIdx.x % G;
    for (int base = 0; base < K4; base += groups) {
      const int j4 = base + (int)threadIdx.x / G;
      float best[4];
      int sl[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        best[c] = -CUDART_INF_F;
        sl[c] = -1;
      }
      if (j4 < K4) {
        auto take = [&](int k, float4 w) {
          const float v = S.val[p][k];
          const float c0 = __fadd_rn(v, w.x), c1 = __fadd_rn(v, w.y), c2 = __fadd_rn(v, w.z), c3 = __fadd_rn(v, w.w);
          if (sl[0] < 0 || c0 > best[0]) { best[0] = c0; sl[0] = k; }
          if (sl[1] < 0 || c1 > best[1]) { best[1] = c1; sl[1] = k; }
          if (sl[2] < 0 || c2 > best[2]) { best[2] = c2; sl[2] = k; }
          if (sl[3] < 0 || c3 > best[3]) { best[3] = c3; sl[3] = k; }
        };
        // eight sources in flight per round; compared in slot order
        int k = sub;
        for (; k + 7 * G < nb; k += 8 * G) {
          float4 w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            w[u] = __ldg(reinterpret_cast<const float4*>(a.logA + (int64_t)S.id[p][k + u * G] * K) + j4);
#pragma unroll
          for (int u = 0; u < 8; ++u) take(k + u * G, w[u]);
        }
        for (; k < nb; k += G) take(k, __ldg(reinterpret_cast<const float4*>(a.logA + (int64_t)S.id[p][k] * K) + j4));
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float bv = best[c];
        int bs = sl[c];
        for (int o = 1; o < G; o <<= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o, G);
          const int os = __shfl_xor_sync(0xffffffffu, bs, o, G);
          if (os >= 0 && (bs < 0 || ov > bv || (ov == bv && os < bs))) { bv = ov; bs = os; }
        }
        const int j = 4 * j4 + c;
        if (sub == 0 && j4 < K4) {
          S.cslot[j] = bs;
          S.cval[j] = __fadd_rn(bv, beam_emit(a, jb, t, j));
          if (bs >= 0) atomicOr(&sm.touched[j >> 5], 1u << (j & 31));
        }
      }
    }
    __syncthreads();
    if (a.static_beam) static_full_vector(a, S, sm);
    return;
  }
  if (a.trans == FV_TRANS_DENSE) {
    // G threads per target (adjacent lanes) split the beam by slot
    // residue; the group keeps the highest value, the lowest slot on ties
    int G = 1;
    while (G < 32 && 2 * G * K <= (int)blockDim.x) G *= 2;
    const int groups = (int)blockDim.x / G, sub = (int)threadIdx.x % G;
    for (int base = 0; base < K; base += groups) {
      const int j = base + (int)threadIdx.x / G;
      float best = -CUDART_INF_F;
      int sl = -1;
      if (j < K) {
        // sixteen sources in flight per round; compared in slot order
        int k = sub;
        for (; k + 15 * G < nb; k += 16 * G) {
          float w[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) w[u] = __ldg(a.logA + (int64_t)S.id[p][k + u * G] * K + j);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const float c = __fadd_rn(S.val[p][k + u * G], w[u]);
            if (sl < 0 || c > best) { best = c; sl = k + u * G; }
          }
        }
        for (; k < nb; k += G) {
          const float c = __fadd_rn(S.val[p][k], __ldg(a.logA + (int64_t)S.id[p][k] * K + j));
          if (sl < 0 || c > best) { best = c; sl = k; }
        }
      }
      for (int o = 1; o < G; o <<= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o, G);
        const int os = __shfl_xor_sync(0xffffffffu, sl, o, G);
        if (os >= 0 && (sl < 0 || ov > best || (ov == best && os < sl))) { best = ov; sl = os; }
      }
      if (sub == 0 && j < K) {
        S.cslot[j] = sl;
        S.cval[j] = __fadd_rn(best, beam_emit(a, jb, t, j));
        if (sl >= 0) atomicOr(&sm.touched[j >> 5], 1u << (j & 31));
      }
    }
    __syncthreads();
    if (a.static_beam) static_full_vector(a, S, sm);
    return;
  }
  // CSR: warp per beam entry scatters keys
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int k = warp; k < nb; k += nwarp) {
    const int i = S.id[p][k];
    const float v = S.val[p][k];
    for (int e = a.row_ptr[i] + lane; e < a.row_ptr[i + 1]; e += 32) {
      const int j = a.col[e];
      const float c = __fadd_rn(v, a.val[e]);
      const unsigned long long key = ((unsigned long long)ord_key(c) << 32) | (0xFFFFFFFFull - (unsigned)k);
      atomicMax(&S.keys[j], key);
      atomicOr(&sm.touched[j >> 5], 1u << (j & 31));
    }
  }
  __syncthreads();
  const int per = (K + (int)blockDim.x - 1) / (int)blockDim.x;
  const int j0 = min(K, (int)threadIdx.x * per), j1 = min(K, j0 + per);
  // with a shared-memory list: this thread's touched targets go to
  // positions [o, o + cnt) of it, so the list is in id order
  int o = 0;
  if (a.list_cap > 0) {
    int cnt = 0;
    for_touched(sm, j0, j1, [&](int) { ++cnt; });
    int n;
    o = block_scan(cnt, sm.red, &n);
    sm.nlist = n <= a.list_cap ? n : -1;
  }
  auto cand = [&](int j) {
    const unsigned long long key = S.keys[j];
    const int sl = (int)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
    // the winning candidate is the key's value (the order map is a
    // bijection away from zero); a zero is recomputed for its sign
    float m = ord_value((uint32_t)(key >> 32));
    if (m == 0.0f) m = __fadd_rn(S.val[p][sl], beam_csr_w(a, S.id[p][sl], j));
    const float c = __fadd_rn(m, beam_emit(a, jb, t, j));
    S.cslot[j] = sl;
    S.cval[j] = c;
    return c;
  };
  sm.nlist_used = sm.nlist;
  if (sm.nlist >= 0) {
    for_touched(sm, j0, j1, [&](int j) {
      const float c = cand(j);
      sm.lkey[o] = isfinite(c) ? ord_key(c) : 0u;
      sm.lj[o] = j;
      ++o;
    });
  } else {
    // no list: ids strided over the block, so a warp touches consecutive
    // entries of the K-indexed arrays
    for (int j = threadIdx.x; j < K; j += blockDim.x)
      if ((sm.touched[j >> 5] >> (j & 31)) & 1u) cand(j);
  }
  __syncthreads();
  if (a.static_beam) static_full_vector(a, S, sm);
}

// Initial candidates at t = m: from pi (m = 0) or from the single state
// q_prev with the retained (or zero) offset (Sec. V-B.2).
__device__ void beam_init(const BeamArgs& a, BeamScratch& S, BeamSmem& sm, const Job& jb, int m, int q_prev,
                          float s_prev) {
  const int K = a.K;
  sm.nlist = -1;
  sm.nlist_used = -1;
  if (m == 0 || a.trans == FV_TRANS_DENSE) {
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      float c;
      if (m == 0) {
        c = __fadd_rn(__ldg(a.log_pi + j), beam_emit(a, jb, 0, j));
      } else {
        const float w = __ldg(a.logA + (int64_t)q_prev * K + j);
        c = a.complete ? __fadd_rn(w, beam_emit(a, jb, m, j))
                       : __fadd_rn(__fadd_rn(s_prev, w), beam_emit(a, jb, m, j));
      }
      S.cval[j] = c;
      S.cslot[j] = 0;
      atomicOr(&sm.touched[j >> 5], 1u << (j & 31));
    }
  } else {
    for (int e = a.row_ptr[q_prev] + threadIdx.x; e < a.row_ptr[q_prev + 1]; e += blockDim.x) {
      const int j = a.col[e];
      // duplicates resolve to the max weight, as csr_w does
      const float w = beam_csr_w(a, q_prev, j);
      const float c = a.complete ? __fadd_rn(w, beam_emit(a, jb, m, j))
                                 : __fadd_rn(__fadd_rn(s_prev, w), beam_emit(a, jb, m, j));
      S.cval[j] = c;
      S.cslot[j] = 0;
      atomicOr(&sm.touched[j >> 5], 1u << (j & 31));
    }
  }
  __syncthreads();
  if (a.static_beam) static_full_vector(a, S, sm);
}

// Block-wide (max value, lowest index) over per-thread candidates; idx
// 0x7fffffff marks "none".  Returns the winning index (or -1 if none or -inf).
__device__ inline int block_argmax(float v, int idx, float* rv, int* ri) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (oi != 0x7fffffff && (idx == 0x7fffffff || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { rv[w] = v; ri[w] = idx; }
  __syncthreads();
  float bv = -CUDART_INF_F;
  int bi = 0x7fffffff;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
    if (ri[k] != 0x7fffffff && (bi == 0x7fffffff || rv[k] > bv || (rv[k] == bv && ri[k] < bi))) { bv = rv[k]; bi = ri[k]; }
  }
  __syncthreads();
  return (bi == 0x7fffffff || !(bv > -CUDART_INF_F)) ? -1 : bi;
}

// Index of state q in an id-sorted beam (binary search), -1 if absent.
__device__ inline int beam_find(const int32_t* ids, int nb, int q) {
  int lo = 0, hi = nb - 1;
  while (lo <= hi) {
    const int md = (lo + hi) >> 1;
    if (ids[md] == q) return md;
    if (ids[md] < q) lo = md + 1; else hi = md - 1;
  }
  return -1;
}

__device__ inline int pe_b(int T, int P) {
  if (T <= 1) return 1;
  int p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
__device__ inline int div_b(int k, int T, int Pe) { return (int)((((int64_t)k + 1) * T - 1) / Pe); }

__global__ void __launch_bounds__(kBeamThreads, 1) beam_kernel(BeamArgs a) {
  extern __shared__ uint32_t bsm[];
  __shared__ int red[32], hist[256], misc[8], ri[32];
  __shared__ float rv[32];
  __shared__ int s_job;
  BeamSmem sm;
  sm.touched = bsm;
  sm.red = red;
  sm.hist = hist;
  sm.misc = misc;
  sm.nlist = -1;
  sm.nlist_used = -1;
  {
    // the candidate list follows the bitmap, the beams and the candidates
    uint32_t* lp = bsm + beam_bitmap_words(a.K) + (a.beam_smem ? 10 * a.Bcap : 0) + (a.cand_smem ? 2 * a.K : 0);
    sm.lkey = lp;
    sm.lj = reinterpret_cast<int32_t*>(lp + a.list_cap);
  }
  if (a.hdr->status != 0) return;
  BeamScratch S = beam_scratch(a, bsm);
  const int K = a.K, nw = (K + 31) >> 5;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) sm.touched[w] = 0u;
  if (a.trans != FV_TRANS_DENSE)
    for (int j = threadIdx.x; j < K; j += blockDim.x) S.keys[j] = 0ull;
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long k = atomicAdd(a.pop, 1ull);
      const int lim = a.kind == kJobSub ? *a.task_count : a.order_count;
      s_job = k < (unsigned long long)lim ? (int)k : -1;
    }
    __syncthreads();
    const int jk = s_job;
    __syncthreads();
    if (jk < 0) break;
    int b, m, n;
    if (a.kind == kJobSub) {
      const Task tk = a.tasks[jk];
      b = tk.b;
      m = tk.m;
      n = tk.n;
    } else {
      b = a.order[a.order_begin + jk];
      m = 0;
      n = a.jobs[b].T - 1;
    }
    const Job jb = a.jobs[b];
    const int T = jb.T;
    int q_prev = 0, q_n = 0;
    float s_prev = 0.f;
    if (a.kind == kJobSub) {
      const int qn = a.paths[jb.path_off + n];
      q_n = (unsigned)qn < (unsigned)K ? qn : 0;
      if (m > 0) {
        const int qp = a.paths[jb.path_off + m - 1];
        q_prev = (unsigned)qp < (unsigned)K ? qp : 0;
        s_prev = a.sval[jb.aux_off + m - 1];
      }
    }
    const int Pe = a.kind == kJobRoot ? pe_b(T, a.P) : 1;
    const int tmid = (m + n) / 2;
    bool done = false;
    for (int attempt = 0; attempt < 2 && !done; ++attempt) {
      // attempt 1 (subtasks only): the full state set (R9)
      int W = attempt ? K : (a.Wcap < a.Bcap ? a.Wcap : a.Bcap);
      if (W > a.Bcap) W = a.Bcap;
      // ---- t = m
      beam_init(a, S, sm, jb, m, q_prev, s_prev);
      int p = 0;
      int nb = select_top_b(a, S, sm, p, W, 0);
      clear_candidates(a, S, sm);
      int kdiv = 0, ediv = a.kind == kJobRoot ? div_b(0, T, Pe) : -1, eprev = -1, snap_n = 0;
      bool infeasible = nb == 0;
      // bookkeeping of step t (beam in buffer p, nb entries)
      auto book = [&](int t) {
        if (a.kind == kJobBeam) {
          for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            a.bp_id[jb.aux_off + (int64_t)t * a.Wcap + e] = S.id[p][e];
            a.bp_src[jb.aux_off + (int64_t)t * a.Wcap + e] = t == m ? 0 : S.src[p][e];
          }
        } else if (a.kind == kJobRoot && t == ediv) {
          const int64_t base = (int64_t)b * a.div_stride + (int64_t)kdiv * a.Wcap;
          for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            a.div_id[base + e] = S.id[p][e];
            a.div_val[base + e] = S.val[p][e];
            a.div_mid[base + e] = t == m ? -1 : S.mid[p][e];
          }
          if (threadIdx.x == 0) a.div_n[(int64_t)b * a.pe_cap + kdiv] = nb;
          eprev = ediv;
          ++kdiv;
          ediv = kdiv < Pe ? div_b(kdiv, T, Pe) : 0x7fffffff;
        } else if (a.kind == kJobSub && t == tmid) {
          for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            S.snap_id[e] = S.id[p][e];
            S.snap_val[e] = S.val[p][e];
          }
          snap_n = nb;
        }
        __syncthreads();
      };
      if (!infeasible) book(m);
      for (int t = m + 1; t <= n && !infeasible; ++t) {
        if (a.kind == kJobSub && t == n) {
          // last step: evaluate only target q_n, from every beam source (R9)
          float bv = -CUDART_INF_F;
          int bs = 0x7fffffff;
          for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const float c = __fadd_rn(S.val[p][k], beam_trans(a, S.id[p][k], q_n));
            if (bs == 0x7fffffff || c > bv) { bv = c; bs = k; }
          }
          const int sidx = block_argmax(bv, bs, rv, ri);
          if (sidx < 0) { infeasible = true; break; }
          if (threadIdx.x == 0) {
            const int q = (t == tmid + 1) ? S.id[p][sidx] : S.mid[p][sidx];
            const int x = beam_find(S.snap_id, snap_n, q);
            a.paths[jb.path_off + tmid] = (unsigned)q < (unsigned)K ? q : 0;
            a.sval[jb.aux_off + tmid] = x >= 0 ? S.snap_val[x] : -CUDART_INF_F;
          }
          __syncthreads();
          break;
        }
        // large CSR state spaces read this step's emission row at scattered
        // targets: the next step's row goes to L2 while this one is used
        if (a.trans != FV_TRANS_DENSE && a.emit == FV_EMIT_DENSE && threadIdx.x == 0 && t < n &&
            (a.K & 3) == 0 && a.K >= 4096) {
          const float* row = a.E + jb.e_off + (int64_t)(t + 1) * a.K;
          if (((uintptr_t)row & 15u) == 0) prefetch_l2_bulk(row, (uint32_t)a.K * 4u);
        }
        beam_candidates(a, S, sm, jb, p, nb, t);
        int need_mid = 0;
        if (a.kind == kJobRoot && eprev >= 0) need_mid = (t == eprev + 1) ? 1 : 2;
        if (a.kind == kJobSub) need_mid = (t == tmid + 1) ? 1 : (t > tmid + 1 ? 2 : 0);
        const int np = p ^ 1;
        nb = select_top_b(a, S, sm, np, W, need_mid);
        clear_candidates(a, S, sm);
        p = np;
        if (nb == 0) { infeasible = true; break; }
        book(t);
      }
      if (!infeasible) {
        if (a.kind == kJobBeam && threadIdx.x == 0) {
          int kb = 0;  // best final entry: highest score, lowest id
          for (int e = 1; e < nb; ++e)
            if (S.val[p][e] > S.val[p][kb]) kb = e;
          a.scores[b] = S.val[p][kb];
          a.qlast[b] = kb;
        }
        done = true;
      } else if (a.kind == kJobSub && attempt == 0 && K <= a.Bcap) {
        if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[0]), 1ull);
      } else {
        if (threadIdx.x == 0) set_status(a.hdr, FV_EINFEASIBLE, (uint32_t)b);
        done = true;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Dynamic beam on CSR transitions with one sequence spread over a cluster of
// kCB CTAs (kJobBeam, large K).  The single-CTA kernel above keeps one SM
// busy per sequence and is bound by the latency of each step's phases; here
// every phase is split kCB ways:
//  * scatter: CTA r relaxes the out-edges of its share of the beam entries
//    (64-bit atomicMax on the cluster's key array in global memory, the
//    same keys as above) and marks each target in the bitmap of the CTA
//    that owns the target's id range (distributed shared memory);
//  * candidates: CTA r lists the touched targets of its id range (ids
//    [r R, (r+1) R)) in shared memory, in id order, with c_j = M_j + E_t[j];
//  * top-B select: the MSB radix select of the single-CTA kernel with every
//    pass's 256-bin histogram summed over the cluster (each CTA reads the
//    others' histograms through distributed shared memory), so every CTA
//    takes the same threshold; keys equal to the threshold go to the lowest
//    ids first, i.e. to the lower ranks first;
//  * gather: each CTA learns how many winners the lower ranks hold and
//    writes its own at that offset, in id order -- the next beam, sorted by
//    id, in global memory, with the step's backpointers.
// Result: the same beams, paths and scores as the single-CTA kernel.
constexpr int kCB = 8;              // CTAs per sequence (portable cluster size)
constexpr int kCBThreads = 1024;

__device__ inline void dsmem_red_or(uint32_t addr, uint32_t v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ inline uint32_t dsmem_ld_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// ids per rank, its bitmap words and the shared-memory layout
__host__ __device__ inline int cb_range(int K) { return (K + kCB - 1) / kCB; }
__host__ __device__ inline size_t cb_smem_bytes(int K) {
  const size_t R = (size_t)cb_range(K), bm = ((R + 31) / 32 + 3) / 4 * 4;
  return 4 * (bm + 2 * R + 3 * 256 + 4 * kCB + 16);
}

__global__ void __launch_bounds__(kCBThreads, 1) beam_csr_cluster_kernel(BeamArgs a) {
  extern __shared__ __align__(16) uint32_t csm[];
  __shared__ int red[32];
  __shared__ int misc[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const uint32_t rank = cluster_ctarank();
  const int K = a.K, R = cb_range(K);
  const int j_lo = (int)rank * R, j_hi = min(K, j_lo + R), nloc = max(0, j_hi - j_lo);
  const int bm_words = ((R + 31) / 32 + 3) / 4 * 4;
  uint32_t* bitmap = csm;                                            // [bm_words] touched, local ids
  float* lval = reinterpret_cast<float*>(bitmap + bm_words);         // [R] listed candidate values
  int32_t* lid = reinterpret_cast<int32_t*>(lval + R);               // [R] their ids, ascending
  int* hist = reinterpret_cast<int*>(lid + R);                       // [2][256] this CTA's histograms
  int* cnt = hist + 512;                                             // [4][kCB] counts from every rank
  int* htot = cnt + 4 * kCB;                                         // [256] the cluster's histogram
  const int cl = blockIdx.x / kCB, ncl = gridDim.x / kCB;
  // the cluster's key array and beams: the scratch slice of its rank-0 CTA
  char* base = a.scratch + (size_t)(cl * kCB) * a.scratch_stride;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(base);
  base += align_up((size_t)K * 8);
  base += 2 * align_up((size_t)K * 4);  // (cval, cslot: unused here)
  int32_t* bid[2];
  float* bval[2];
  for (int q = 0; q < 2; ++q) {
    bid[q] = reinterpret_cast<int32_t*>(base);
    base += align_up((size_t)a.Bcap * 4);
    bval[q] = reinterpret_cast<float*>(base);
    base += align_up((size_t)a.Bcap * 4);
    base += 2 * align_up((size_t)a.Bcap * 4);  // (mid, src: unused here)
  }
  // every CTA of the cluster has started before shared memory is written
  // remotely; one thread of rank 0 reads the status word and tells the
  // others, so the decision to run is the same in every CTA
  __shared__ int s_go;
  cluster_sync_all();
  if (rank == 0 && tid == 0) {
    const uint32_t go = a.hdr->status == 0 ? 1u : 0u;
    for (int q = 0; q < kCB; ++q) dsmem_st_u32(dsmem_addr(&s_go, (uint32_t)q), go);
  }
  cluster_sync_all();
  if (!s_go) return;
  for (int w = tid; w < bm_words; w += blockDim.x) bitmap[w] = 0u;
  for (int j = j_lo + tid; j < j_hi; j += blockDim.x) keys[j] = 0ull;
  cluster_sync_all();

  // each thread's contiguous piece of this rank's ids / of the list
  const int per = (R + (int)blockDim.x - 1) / (int)blockDim.x;
  const int t0 = min(nloc, tid * per), t1 = min(nloc, t0 + per);

  // publish v to slot [which][rank] of every rank, then (after a cluster
  // barrier) read the kCB values
  auto publish = [&](int which, int v) {
    if (tid < kCB) dsmem_st_u32(dsmem_addr(&cnt[which * kCB + (int)rank], (uint32_t)tid), (uint32_t)v);
  };

  // top-W of the list (n entries; values lval, ids lid, ascending) over the
  // whole cluster -> beam buffer q at its global positions; returns the new
  // beam size (identical in every CTA).  Writes backpointers of step t when
  // bp_t >= 0 (source slot from the key, 0 at t = m).
  auto select_gather = [&](int n, int W, int q, int bp_t, bool from_keys, const Job& jb) -> int {
    const int e0 = min(n, tid * ((n + (int)blockDim.x - 1) / (int)blockDim.x));
    const int e1 = min(n, e0 + (n + (int)blockDim.x - 1) / (int)blockDim.x);
    int fin = 0;
    for (int e = e0; e < e1; ++e) fin += isfinite(lval[e]) ? 1 : 0;
    fin = block_sum(fin, red);
    publish(0, fin);
    cluster_sync_all();
    int total = 0;
    for (int r = 0; r < kCB; ++r) total += cnt[0 * kCB + r];
    const bool all = total <= W;
    uint32_t thr = 0u;
    int need_eq = 0;
    if (!all) {
      uint32_t prefix = 0u, mask = 0u;
      int remaining = W;
      for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        int* h = hist + (pass & 1) * 256;
        for (int k = tid; k < 256; k += blockDim.x) h[k] = 0;
        __syncthreads();
        for (int e = tid; e < n; e += blockDim.x) {
          const float c = lval[e];
          if (!isfinite(c)) continue;
          const uint32_t u = ord_key(c);
          if ((u & mask) == prefix) atomicAdd(&h[(u >> shift) & 0xFFu], 1);
        }
        for (int k = tid; k < 256; k += blockDim.x) htot[k] = 0;
        cluster_sync_all();  // every rank's histogram of this pass is complete
        // the cluster's histogram: every thread adds a few (rank, digit)
        // counts read from the other CTAs, so the remote loads overlap
        for (int x = tid; x < 256 * kCB; x += blockDim.x) {
          const int d = x & 255, r = x >> 8;
          const int v = (int)dsmem_ld_u32(dsmem_addr(&h[d], (uint32_t)r));
          if (v) atomicAdd(&htot[d], v);
        }
        __syncthreads();
        if (tid < 32) {
          int hv[8], sum = 0;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            hv[u] = htot[255 - 8 * lane - u];
            sum += hv[u];
          }
          int incl = sum;
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int excl = incl - sum;
          if (excl < remaining && remaining <= incl) {
            int acc = excl, d = 255 - 8 * lane - 7;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (acc + hv[u] >= remaining) { d = 255 - 8 * lane - u; break; }
              acc += hv[u];
            }
            misc[0] = d;
            misc[1] = remaining - acc;
          }
        }
        __syncthreads();
        prefix |= (uint32_t)misc[0] << shift;
        mask |= 0xFFu << shift;
        remaining = misc[1];
        __syncthreads();
      }
      thr = prefix;
      need_eq = remaining;
    }
    // winners of this rank: keys above the threshold, and keys equal to it
    // while the lower ranks have not taken the needed number
    int n_gt = 0, n_eq = 0;
    for (int e = e0; e < e1; ++e) {
      const float c = lval[e];
      if (!isfinite(c)) continue;
      const uint32_t u = ord_key(c);
      if (all || u > thr) ++n_gt;
      else if (u == thr) ++n_eq;
    }
    int tot_eq_loc, tot_gt_loc;
    const int eq_before_loc = block_scan(n_eq, red, &tot_eq_loc);
    block_scan(n_gt, red, &tot_gt_loc);
    publish(1, tot_gt_loc);
    publish(2, tot_eq_loc);
    cluster_sync_all();
    int eq_before = 0, win_before = 0, nb = 0;
    for (int r = 0; r < kCB; ++r) {
      const int gt_r = cnt[1 * kCB + r], eq_r = cnt[2 * kCB + r];
      const int take_r = min(max(need_eq - eq_before, 0), eq_r);
      if (r < (int)rank) win_before += gt_r + take_r;
      if (r == (int)rank) misc[2] = take_r;
      eq_before += eq_r;
      nb += gt_r + take_r;
    }
    __syncthreads();
    const int take_rank = misc[2];
    const int take_eq = min(max(take_rank - eq_before_loc, 0), n_eq);
    int tot;
    int o = win_before + block_scan(n_gt + take_eq, red, &tot);
    int eq_seen = 0;
    for (int e = e0; e < e1; ++e) {
      const float c = lval[e];
      if (!isfinite(c)) continue;
      const uint32_t u = ord_key(c);
      bool take = all || u > thr;
      if (!take && u == thr) take = (eq_seen++ < take_eq);
      if (!take) continue;
      const int j = lid[e];
      bid[q][o] = j;
      bval[q][o] = c;
      if (bp_t >= 0) {
        const int sl = from_keys ? (int)(0xFFFFFFFFull - (keys[j] & 0xFFFFFFFFull)) : 0;
        a.bp_id[jb.aux_off + (int64_t)bp_t * a.Wcap + o] = j;
        a.bp_src[jb.aux_off + (int64_t)bp_t * a.Wcap + o] = sl;
      }
      ++o;
    }
    __syncthreads();  // every thread has read its winners' keys before any is cleared
    return nb;
  };

  for (int jk = cl; jk < a.order_count; jk += ncl) {
    const int b = a.order[a.order_begin + jk];
    const Job jb = a.jobs[b];
    const int T = jb.T;
    const int W = a.Wcap < a.Bcap ? a.Wcap : a.Bcap;
    // ---- t = 0: every state of this rank's range is a candidate
    int n = 0;
    {
      int tot;
      const int o0 = block_scan(t1 - t0, red, &tot);
      for (int x = t0; x < t1; ++x) {
        const int j = j_lo + x;
        lval[o0 + x - t0] = __fadd_rn(__ldg(a.log_pi + j), beam_emit(a, jb, 0, j));
        lid[o0 + x - t0] = j;
      }
      n = tot;
      __syncthreads();
    }
    int p = 0;
    int nb = select_gather(n, W, p, 0, false, jb);
    cluster_sync_all();  // beam 0 is complete in global memory
    bool infeasible = nb == 0;
    for (int t = 1; t < T && !infeasible; ++t) {
      // the next step's emission row goes to L2 while this one is used
      if (a.emit == FV_EMIT_DENSE && tid == 0 && rank == 0 && t + 1 < T && (K & 3) == 0) {
        const float* row = a.E + jb.e_off + (int64_t)(t + 1) * K;
        if (((uintptr_t)row & 15u) == 0) prefetch_l2_bulk(row, (uint32_t)K * 4u);
      }
      // ---- scatter this rank's share of the beam entries
      const int s0 = (int)(((int64_t)nb * rank) / kCB), s1 = (int)(((int64_t)nb * (rank + 1)) / kCB);
      for (int k = s0 + warp; k < s1; k += nwarp) {
        const int i = bid[p][k];
        const float v = bval[p][k];
        for (int e = a.row_ptr[i] + lane; e < a.row_ptr[i + 1]; e += 32) {
          const int j = a.col[e];
          const float c = __fadd_rn(v, a.val[e]);
          const unsigned long long key = ((unsigned long long)ord_key(c) << 32) | (0xFFFFFFFFull - (unsigned)k);
          atomicMax(&keys[j], key);
          const int ow = j / R, jl = j - ow * R;
          dsmem_red_or(dsmem_addr(&bitmap[jl >> 5], (uint32_t)ow), 1u << (jl & 31));
        }
      }
      cluster_sync_all();  // keys and bitmaps of this step are complete
      // ---- candidates of this rank's ids, listed in id order
      {
        int c_n = 0;
        for (int x = t0; x < t1; ++x) c_n += (bitmap[x >> 5] >> (x & 31)) & 1u;
        int tot;
        int o = block_scan(c_n, red, &tot);
        for (int x = t0; x < t1; ++x) {
          if (!((bitmap[x >> 5] >> (x & 31)) & 1u)) continue;
          const int j = j_lo + x;
          const unsigned long long key = keys[j];
          const int sl = (int)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
          float m = ord_value((uint32_t)(key >> 32));
          if (m == 0.0f) m = __fadd_rn(bval[p][sl], beam_csr_w(a, bid[p][sl], j));
          lval[o] = __fadd_rn(m, beam_emit(a, jb, t, j));
          lid[o] = j;
          ++o;
        }
        n = tot;
        __syncthreads();
      }
      const int np = p ^ 1;
      nb = select_gather(n, W, np, t, true, jb);
      // ---- clear this rank's keys and bitmap
      for (int e = tid; e < n; e += blockDim.x) keys[lid[e]] = 0ull;
      for (int w = tid; w < bm_words; w += blockDim.x) bitmap[w] = 0u;
      cluster_sync_all();  // the next beam is complete; keys and bitmaps are clear
      p = np;
      if (nb == 0) infeasible = true;
    }
    if (!infeasible) {
      if (rank == 0 && tid == 0) {
        int kb = 0;  // best final entry: highest score, lowest id
        for (int e = 1; e < nb; ++e)
          if (bval[p][e] > bval[p][kb]) kb = e;
        a.scores[b] = bval[p][kb];
        a.qlast[b] = kb;
      }
    } else if (rank == 0 && tid == 0) {
      set_status(a.hdr, FV_EINFEASIBLE, (uint32_t)b);
    }
    cluster_sync_all();
  }
}

// ---------------------------------------------------------------------------
// Dynamic beam on dense transitions with one sequence spread over a cluster
// of kDC CTAs (kJobBeam, 512 <= K <= 8192).  A dense step reads B rows of
// logA (B K cells); on one SM its time is set by how fast those rows come in
// from L2.  Here CTA r owns the targets [r R, (r+1) R), R = K / kDC:
//  * candidates: its threads split (target quad, beam slot residue); every
//    thread reads 16-byte pieces of the beam sources' logA rows (a warp
//    reads whole row pieces), keeps per target the highest value, lowest
//    slot on ties, and the partials are combined through shared memory;
//    c_j = fl(M_j + E_t[j]) is then stored into the candidate vector of
//    every CTA of the cluster (distributed shared memory, double-buffered by
//    step parity);
//  * one cluster barrier: every CTA now holds all K candidates;
//  * top-B select: each CTA runs the same MSB radix select (order-preserving
//    keys, -0 folded into +0) over the K candidates and builds the next beam
//    in id order in its own shared memory, so the next step reads its
//    sources locally; each CTA writes the backpointers of its own targets.
// Same candidates, same tie rules and the same beams as the single-CTA
// kernel, hence the same paths and scores.
constexpr int kDC = 8;  // CTAs per sequence
constexpr int kDCThreads = 512;
constexpr int kDCMaxK = 8192;
constexpr int kDCKeys = kDCMaxK / kDCThreads;  // candidate keys per thread

struct DcLayout {
  int R, Q, S, G2, RS;  // targets per CTA, their quads, slot groups, lanes per target, partial row stride
  size_t words;         // dynamic shared memory (4-byte words)
};

__host__ __device__ inline DcLayout dc_layout(int K, int W) {
  DcLayout L;
  L.R = K / kDC;
  L.Q = L.R / 4;
  L.S = kDCThreads / L.Q;
  L.G2 = 1;
  while (2 * L.G2 * L.R <= kDCThreads) L.G2 *= 2;
  // padding that puts the G2 lanes of a target on distinct banks
  const int pad = 32 / L.G2 > 4 ? 32 / L.G2 : 4;
  L.RS = L.R + pad;
  // [2][K] candidates, [S][RS] partial values and slots, [3][256] histograms,
  // [R] slots of this CTA's targets, [W] beam ids, [W] beam scores
  L.words = 2 * (size_t)K + 2 * (size_t)L.S * L.RS + 768 + (size_t)L.R + 2 * (size_t)W;
  return L;
}

// Exclusive scan of two per-thread counts over the block (kDCThreads).
__device__ inline void dc_scan2(int x, int y, int* red, int* ex, int* ey, int* tx, int* ty) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int sx = x, sy = y;
  for (int o = 1; o < 32; o <<= 1) {
    const int ux = __shfl_up_sync(0xffffffffu, sx, o), uy = __shfl_up_sync(0xffffffffu, sy, o);
    if (lane >= o) { sx += ux; sy += uy; }
  }
  if (lane == 31) { red[w] = sx; red[16 + w] = sy; }
  __syncthreads();
  if (w == 0) {
    int px = lane < 16 ? red[lane] : 0, py = lane < 16 ? red[16 + lane] : 0;
    for (int o = 1; o < 16; o <<= 1) {
      const int ux = __shfl_up_sync(0xffffffffu, px, o), uy = __shfl_up_sync(0xffffffffu, py, o);
      if (lane >= o) { px += ux; py += uy; }
    }
    if (lane < 16) { red[lane] = px; red[16 + lane] = py; }
  }
  __syncthreads();
  *ex = (w ? red[w - 1] : 0) + sx - x;
  *ey = (w ? red[16 + w - 1] : 0) + sy - y;
  *tx = red[15];
  *ty = red[31];
  // (red is written again only after the caller's next block barrier)
}

__global__ void __launch_bounds__(kDCThreads, 1) beam_dense_cluster_kernel(BeamArgs a) {
  extern __shared__ __align__(16) uint32_t dsm[];
  __shared__ int red[32];
  __shared__ int s_go, s_job;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t rank = cluster_ctarank();
  const int K = a.K, W = a.Wcap < a.Bcap ? a.Wcap : a.Bcap;
  const DcLayout L = dc_layout(K, W);
  const int R = L.R, j_lo = (int)rank * R;
  float* cand = reinterpret_cast<float*>(dsm);                      // [2][K]
  float* pv = cand + 2 * K;                                          // [S][RS]
  int32_t* ps = reinterpret_cast<int32_t*>(pv + L.S * L.RS);        // [S][RS]
  int* hist = reinterpret_cast<int*>(ps + L.S * L.RS);               // [3][256]
  int32_t* lslot = hist + 768;                                       // [R]
  int32_t* bid = lslot + R;                                          // [W]
  float* bval = reinterpret_cast<float*>(bid + W);                   // [W]
  for (int k = tid; k < 768; k += blockDim.x) hist[k] = 0;
  // every CTA of the cluster has started before shared memory is written
  // remotely; one thread of rank 0 reads the status word and tells the
  // others, so the decision to run is the same in every CTA
  cluster_sync_all();
  if (rank == 0 && tid == 0) {
    const uint32_t go = a.hdr->status == 0 ? 1u : 0u;
    for (int q = 0; q < kDC; ++q) dsmem_st_u32(dsmem_addr(&s_go, (uint32_t)q), go);
  }
  cluster_sync_all();
  if (!s_go) return;

  // candidates: thread (quad qd, slot group sg)
  const int qd = tid % L.Q, sg = tid / L.Q;
  const bool cact = sg < L.S;
  const int K4 = K >> 2;
  const float4* arow = reinterpret_cast<const float4*>(a.logA) + (j_lo >> 2) + qd;
  // final combine: G2 lanes per target, NG targets per round (at most 2 rounds)
  const int G2 = L.G2, NG = kDCThreads / G2, sub = tid % G2;
  // select: keys strided over the block, compaction over contiguous id ranges
  const int per = (K + kDCThreads - 1) / kDCThreads;  // also the keys per thread
  const int c0 = min(K, tid * per), c1 = min(K, c0 + per);
  int hrot = 0;  // histogram buffer of the next radix pass

  for (;;) {
    // the next sequence (longest first) for the whole cluster: rank 0 takes
    // it from the launch's counter and tells the others
    if (rank == 0 && tid == 0) {
      const unsigned long long k = atomicAdd(a.pop, 1ull);
      const uint32_t jk = k < (unsigned long long)a.order_count ? (uint32_t)k : 0xFFFFFFFFu;
      for (int q = 0; q < kDC; ++q) dsmem_st_u32(dsmem_addr(&s_job, (uint32_t)q), jk);
    }
    cluster_sync_all();
    const int jk = s_job;
    if (jk < 0) break;  // every CTA of the cluster leaves together
    const int b = a.order[a.order_begin + jk];
    const Job jb = a.jobs[b];
    const int T = jb.T;
    int nb = 0;
    bool infeasible = false;
    for (int t = 0; t < T && !infeasible; ++t) {
      const int buf = t & 1;
      float* cv = cand + buf * K;
      // this step's emission scores of the thread's final targets
      float ev[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int x = r * NG + tid / G2;
        ev[r] = x < R ? beam_emit(a, jb, t, j_lo + x) : 0.f;
      }
      if (a.emit == FV_EMIT_DENSE && tid == 0 && t + 1 < T) {
        const float* row = a.E + jb.e_off + (int64_t)(t + 1) * K + j_lo;
        if (((uintptr_t)row & 15u) == 0) prefetch_l2_bulk(row, (uint32_t)R * 4u);
      }
      if (t == 0) {
        for (int r = 0; r < 2; ++r) {
          const int x = r * NG + tid / G2;
          if (x < R && sub == 0) {
            const float c = __fadd_rn(__ldg(a.log_pi + j_lo + x), ev[r]);
            for (int q = 0; q < kDC; ++q) dsmem_st_f32(dsmem_addr(&cv[j_lo + x], (uint32_t)q), c);
          }
        }
      } else {
        // ---- candidates of this CTA's targets from the local beam
        float best[4];
        int sl[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          best[c] = -CUDART_INF_F;
          sl[c] = -1;
        }
        if (cact) {
          auto take = [&](int k, float4 w) {
            const float v = bval[k];
            const float x0 = __fadd_rn(v, w.x), x1 = __fadd_rn(v, w.y), x2 = __fadd_rn(v, w.z),
                        x3 = __fadd_rn(v, w.w);
            if (sl[0] < 0 || x0 > best[0]) { best[0] = x0; sl[0] = k; }
            if (sl[1] < 0 || x1 > best[1]) { best[1] = x1; sl[1] = k; }
            if (sl[2] < 0 || x2 > best[2]) { best[2] = x2; sl[2] = k; }
            if (sl[3] < 0 || x3 > best[3]) { best[3] = x3; sl[3] = k; }
          };
          const int S = L.S;
          int k = sg;
          // eight sources in flight per round; compared in slot order
          for (; k + 7 * S < nb; k += 8 * S) {
            float4 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = __ldg(arow + (int64_t)bid[k + u * S] * K4);
#pragma unroll
            for (int u = 0; u < 8; ++u) take(k + u * S, w[u]);
          }
          for (; k < nb; k += S) take(k, __ldg(arow + (int64_t)bid[k] * K4));
          reinterpret_cast<float4*>(pv + sg * L.RS)[qd] = make_float4(best[0], best[1], best[2], best[3]);
          reinterpret_cast<int4*>(ps + sg * L.RS)[qd] = make_int4(sl[0], sl[1], sl[2], sl[3]);
        }
        __syncthreads();
        // ---- combine the slot groups per target, add E, send to every CTA
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (r * NG >= R) break;  // uniform
          const int x = r * NG + tid / G2;
          float bv = -CUDART_INF_F;
          int bs = -1;
          if (x < R)
            for (int s = sub; s < L.S; s += G2) {
              const float v = pv[s * L.RS + x];
              const int q = ps[s * L.RS + x];
              if (q >= 0 && (bs < 0 || v > bv || (v == bv && q < bs))) { bv = v; bs = q; }
            }
          for (int o = 1; o < G2; o <<= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int os = __shfl_xor_sync(0xffffffffu, bs, o);
            if (os >= 0 && (bs < 0 || ov > bv || (ov == bv && os < bs))) { bv = ov; bs = os; }
          }
          if (x < R) {
            const float c = __fadd_rn(bv, ev[r]);
            for (int q = sub; q < kDC; q += G2) dsmem_st_f32(dsmem_addr(&cv[j_lo + x], (uint32_t)q), c);
            if (sub == 0) lslot[x] = bs;
          }
        }
      }
      cluster_sync_all();  // every CTA holds the K candidates of step t
      // ---- top-W of the K candidates (finite only): score desc, id asc
      uint32_t ku[kDCKeys];
#pragma unroll
      for (int i = 0; i < kDCKeys; ++i) {
        if (i >= per) break;  // uniform
        const int j = tid + i * kDCThreads;
        const float c = j < K ? cv[j] : -CUDART_INF_F;
        ku[i] = isfinite(c) ? ord_key(c) : 0u;
      }
      uint32_t prefix = 0u, mask = 0u, thr_gt = 0u;
      int remaining = W, need_eq = 0;
      for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        // three histogram buffers in rotation: the one counted two passes
        // ago is cleared while this one is read, so every pass needs one
        // block barrier
        const int hb = hrot;
        hrot = hrot == 2 ? 0 : hrot + 1;
        int* h = hist + hb * 256;
#pragma unroll
        for (int i = 0; i < kDCKeys; ++i) {
          if (i >= per) break;  // uniform
          const uint32_t u = ku[i];
          const bool ok = u != 0u && (u & mask) == prefix;
          const int d = ok ? (int)((u >> shift) & 0xFFu) : -1;
          const unsigned grp = __match_any_sync(0xffffffffu, d);
          if (ok && lane == __ffs(grp) - 1) atomicAdd(&h[d], __popc(grp));
        }
        __syncthreads();
        if (tid < 256) hist[(hb == 0 ? 2 : hb - 1) * 256 + tid] = 0;
        // every warp finds the digit from the same histogram: lane l holds
        // digits 255-8l .. 248-8l
        int hv[8], sum = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          hv[u] = h[255 - 8 * lane - u];
          sum += hv[u];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (pass == 0 && total <= remaining) {
          thr_gt = 0u;  // every finite candidate fits
          need_eq = 0;
          break;
        }
        const int excl = incl - sum;
        const unsigned hit = __ballot_sync(0xffffffffu, excl < remaining && remaining <= incl);
        int acc = excl, u_hit = 7;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (acc + hv[u] >= remaining) { u_hit = u; break; }
          acc += hv[u];
        }
        const int src = __ffs(hit) - 1;
        const int dg = __shfl_sync(0xffffffffu, 255 - 8 * lane - u_hit, src);
        const int rem = __shfl_sync(0xffffffffu, remaining - acc, src);
        const int whole = __shfl_sync(0xffffffffu, hv[u_hit], src) == rem;
        prefix |= (uint32_t)dg << shift;
        mask |= 0xFFu << shift;
        remaining = rem;
        if (whole) {
          // the whole bin is needed: keys >= prefix; finite keys are
          // positive, so prefix 0 takes them all
          thr_gt = prefix ? prefix - 1u : 0u;
          need_eq = 0;
          break;
        }
        if (pass == 3) {
          thr_gt = prefix;
          need_eq = remaining;
        }
      }
      const uint32_t thr_eq = prefix;
      int n_gt = 0, n_eq = 0;
      for (int j = c0; j < c1; ++j) {
        const float c = cv[j];
        const uint32_t u = isfinite(c) ? ord_key(c) : 0u;
        if (u == 0u) continue;
        if (u > thr_gt) ++n_gt;
        else if (need_eq > 0 && u == thr_eq) ++n_eq;
      }
      int gt_before, eq_before, tot_gt, tot_eq;
      dc_scan2(n_gt, n_eq, red, &gt_before, &eq_before, &tot_gt, &tot_eq);
      const int take_eq = min(max(need_eq - eq_before, 0), n_eq);
      int o = gt_before + min(eq_before, need_eq);
      nb = tot_gt + min(tot_eq, need_eq);
      int eq_seen = 0;
      for (int j = c0; j < c1; ++j) {
        const float c = cv[j];
        const uint32_t u = isfinite(c) ? ord_key(c) : 0u;
        if (u == 0u) continue;
        bool tk = u > thr_gt;
        if (!tk && need_eq > 0 && u == thr_eq) tk = eq_seen++ < take_eq;
        if (!tk) continue;
        bid[o] = j;
        bval[o] = c;
        if (j >= j_lo && j < j_lo + R) {
          a.bp_id[jb.aux_off + (int64_t)t * a.Wcap + o] = j;
          a.bp_src[jb.aux_off + (int64_t)t * a.Wcap + o] = t == 0 ? 0 : lslot[j - j_lo];
        }
        ++o;
      }
      __syncthreads();  // the next beam is complete in this CTA
      if (nb == 0) infeasible = true;
    }
    if (!infeasible) {
      if (rank == 0 && tid == 0) {
        int kb = 0;  // best final entry: highest score, lowest id
        for (int e = 1; e < nb; ++e)
          if (bval[e] > bval[kb]) kb = e;
        a.scores[b] = bval[kb];
        a.qlast[b] = kb;
      }
    } else if (rank == 0 && tid == 0) {
      set_status(a.hdr, FV_EINFEASIBLE, (uint32_t)b);
    }
    // no CTA takes the next sequence (and overwrites s_job) while another
    // still reads this one's candidates or job index
    cluster_sync_all();
  }
}

// ---------------------------------------------------------------------------
// Dynamic beam on small dense state spaces (K <= 128, P = 0): one CTA of KM
// threads per sequence, thread j owning target j with the column logA[:, j]
// in registers, as in the small-K exact engine.  delta_{t-1} is kept for all
// K states, -inf outside the beam, so the max-plus over every row gives each
// target its best beam source: rows outside the beam only add -inf, and the
// lowest row reaching the maximum is the lowest beam slot, because the beam
// is kept in id order.  That row's slot is the number of beam states below
// it.  The top-B select ranks the finite candidates under (score desc, id
// asc) inside the CTA, and warp ballots give each winner its position in id
// order.  Same candidates, tie rules and beams as beam_kernel; a step costs
// two block barriers instead of the general kernel's dozen.
constexpr int kSBAhead = 4;               // emission scores loaded this many steps ahead
constexpr int kSBLogB = 48 * 1024;        // bytes of a discrete table staged in shared memory at most

template <int KM>
__host__ __device__ inline bool sb_stage_logB(const BeamArgs& a) {
  return a.emit != FV_EMIT_DENSE && (size_t)a.V * KM * sizeof(float) <= (size_t)kSBLogB;
}

template <int KM>
__global__ void __launch_bounds__(KM) small_beam_kernel(BeamArgs a) {
  constexpr int NWP = KM / 32;  // warps
  constexpr int Q = KM / 4;     // rows per argmax chain
  __shared__ __align__(16) float sd[2][KM];      // delta of the beam states, -inf elsewhere
  __shared__ __align__(16) uint32_t skey[KM];    // this step's ordered candidate keys (0: not finite)
  __shared__ uint32_t sbm[2][NWP];               // beam membership, one bit per state
  extern __shared__ float sbB[];                 // discrete table as [symbol][state] (when it fits)
  __shared__ int s_go;
  if ((int)blockIdx.x >= a.order_count) return;
  // an earlier kernel may have recorded an error: one thread reads the
  // status word, so that the whole CTA takes the same decision
  if (threadIdx.x == 0) s_go = a.hdr->status == 0;
  __syncthreads();
  if (!s_go) return;
  const int K = a.K, j = threadIdx.x, lane = j & 31, w = j >> 5;
  const bool own = j < K;
  const int b = a.order[a.order_begin + blockIdx.x];
  const Job jb = a.jobs[b];
  const int T = jb.T;
  const int W = a.Wcap < a.Bcap ? a.Wcap : a.Bcap;
  float A[KM];
#pragma unroll
  for (int i = 0; i < KM; ++i) A[i] = (own && i < K) ? __ldg(a.logA + (int64_t)i * K + j) : -CUDART_INF_F;
  const bool staged = sb_stage_logB<KM>(a);
  if (staged) {
    for (int x = 0; x < a.V; ++x) sbB[x * KM + j] = own ? __ldg(a.logB + (int64_t)j * a.V + x) : 0.f;
    __syncthreads();
  }
  auto emit = [&](int t) -> float {
    if (a.emit == FV_EMIT_DENSE) return __ldg(a.E + jb.e_off + (int64_t)t * K + j);
    const int x = __ldg(a.obs + jb.e_off + t);
    return staged ? sbB[x * KM + j] : __ldg(a.logB + (int64_t)j * a.V + x);
  };
  float er[kSBAhead];  // E_t .. E_{t+kSBAhead-1} of this state, oldest first
#pragma unroll
  for (int k = 0; k < kSBAhead; ++k) er[k] = (own && k < T) ? emit(k) : 0.f;
  int cur = 0;
  for (int t = 0; t < T; ++t) {
    const float e = er[0];
#pragma unroll
    for (int k = 0; k + 1 < kSBAhead; ++k) er[k] = er[k + 1];
    er[kSBAhead - 1] = (own && t + kSBAhead < T) ? emit(t + kSBAhead) : 0.f;
    float c;
    int src = 0;
    if (t == 0) {
      c = own ? __fadd_rn(__ldg(a.log_pi + j), e) : -CUDART_INF_F;
    } else {
      // candidates in ascending row order in four interleaved chains over
      // quarters of the rows; the first strictly larger one is kept, and the
      // chains merge in row order
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
          float y = __fadd_rn(x.x, A[i]);
          if (y > bq[q]) { bq[q] = y; gq[q] = i; }
          y = __fadd_rn(x.y, A[i + 1]);
          if (y > bq[q]) { bq[q] = y; gq[q] = i + 1; }
          y = __fadd_rn(x.z, A[i + 2]);
          if (y > bq[q]) { bq[q] = y; gq[q] = i + 2; }
          y = __fadd_rn(x.w, A[i + 3]);
          if (y > bq[q]) { bq[q] = y; gq[q] = i + 3; }
        }
      float bv = bq[0];
      int g = gq[0];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (bq[q] > bv) { bv = bq[q]; g = gq[q]; }
      c = own ? __fadd_rn(bv, e) : -CUDART_INF_F;
      // the source's slot: beam states with a lower id
#pragma unroll
      for (int q = 0; q < NWP; ++q) {
        const uint32_t m = sbm[cur][q];
        if (32 * q + 32 <= g) src += __popc(m);
        else if (32 * q < g) src += __popc(m & ((1u << (g - 32 * q)) - 1u));
      }
    }
    // ---- top-W of the finite candidates under (score desc, id asc)
    const uint32_t key = isfinite(c) ? ord_key(c) : 0u;
    skey[j] = key;
    const int nfin = __syncthreads_count(key != 0u);
    bool take = key != 0u;
    if (take && nfin > W) {
      int rank = 0;  // finite candidates ahead of this one (key 0 never is)
      const uint4* kv = reinterpret_cast<const uint4*>(skey);
#pragma unroll 8
      for (int i4 = 0; i4 < KM / 4; ++i4) {
        const uint4 u = kv[i4];
        const int i = 4 * i4;
        rank += (u.x > key || (u.x == key && i < j)) ? 1 : 0;
        rank += (u.y > key || (u.y == key && i + 1 < j)) ? 1 : 0;
        rank += (u.z > key || (u.z == key && i + 2 < j)) ? 1 : 0;
        rank += (u.w > key || (u.w == key && i + 3 < j)) ? 1 : 0;
      }
      take = rank < W;
    }
    sd[cur ^ 1][j] = take ? c : -CUDART_INF_F;
    const uint32_t bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) sbm[cur ^ 1][w] = bal;
    __syncthreads();  // the next beam (values and membership) is complete
    int nb = 0, pos = __popc(bal & ((1u << lane) - 1u));
#pragma unroll
    for (int q = 0; q < NWP; ++q) {
      const int cnt = __popc(sbm[cur ^ 1][q]);
      nb += cnt;
      if (q < w) pos += cnt;
    }
    if (nb == 0) {  // the beam emptied (the same in every thread)
      if (j == 0) set_status(a.hdr, FV_EINFEASIBLE, (uint32_t)b);
      return;
    }
    if (take) {
      a.bp_id[jb.aux_off + (int64_t)t * a.Wcap + pos] = j;
      a.bp_src[jb.aux_off + (int64_t)t * a.Wcap + pos] = src;
    }
    cur ^= 1;
  }
  if (j < 32) {
    // best final entry: highest score, lowest id (states outside the beam are -inf)
    float v = sd[cur][lane];
    int qi = lane;
#pragma unroll
    for (int k = 1; k < NWP; ++k) {
      const float vk = sd[cur][lane + 32 * k];
      if (vk > v) { v = vk; qi = lane + 32 * k; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oq = __shfl_xor_sync(0xffffffffu, qi, o);
      if (ov > v || (ov == v && oq < qi)) { v = ov; qi = oq; }
    }
    if (lane == 0) {
      int slot = 0;
      for (int q = 0; q < NWP; ++q) {
        const uint32_t m = sbm[cur][q];
        if (32 * q + 32 <= qi) slot += __popc(m);
        else if (32 * q < qi) slot += __popc(m & ((1u << (qi - 32 * q)) - 1u));
      }
      a.scores[b] = sd[cur][qi];
      a.qlast[b] = slot;
    }
  }
}

template <int KM>
static cudaError_t launch_small_beam_cfg(const BeamArgs& a, int jobs, cudaStream_t st) {
  const size_t sm = sb_stage_logB<KM>(a) ? (size_t)a.V * KM * sizeof(float) : 0;
  small_beam_kernel<KM><<<jobs, KM, sm, st>>>(a);
  return cudaGetLastError();
}

// Backtrack through per-step beam backpointers (one thread per sequence).
__global__ void beam_backtrack_kernel(const Job* jobs, const int32_t* order, int32_t begin, int32_t count,
                                      int32_t Wcap, const int32_t* bp_id, const int32_t* bp_src,
                                      const int32_t* qlast, int32_t* paths, const WsHeader* hdr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count || hdr->status != 0) return;
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  int slot = qlast[b];
  for (int t = jb.T - 1; t >= 0; --t) {
    const int64_t base = jb.aux_off + (int64_t)t * Wcap;
    slot = slot < 0 ? 0 : (slot >= Wcap ? Wcap - 1 : slot);
    paths[jb.path_off + t] = bp_id[base + slot];
    slot = bp_src[base + slot];
  }
}

// FLASH-BS resolve: walk the stored division-point beams (one thread per
// sequence): q_{e_{k-1}} = MidState of q_{e_k}'s entry at e_k.
__global__ void beam_resolve_kernel(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                                    int32_t Bcap /* = Wcap */, int32_t pe_cap, int64_t div_stride, const int32_t* div_id,
                                    const float* div_val, const int32_t* div_mid, const int32_t* div_n,
                                    int32_t* paths, float* sval, WsHeader* hdr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count || hdr->status != 0) return;
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  const int T = jb.T, Pe = pe_b(T, P);
  const int64_t base = (int64_t)b * div_stride;
  // best entry at T-1 = e_{Pe-1}: highest score, lowest id
  const int nlast = div_n[(int64_t)b * pe_cap + Pe - 1];
  const int32_t* ids = div_id + base + (int64_t)(Pe - 1) * Bcap;
  const float* vals = div_val + base + (int64_t)(Pe - 1) * Bcap;
  if (nlast <= 0) { set_status(hdr, FV_EINFEASIBLE, (uint32_t)b); return; }
  int kb = 0;
  for (int e = 1; e < nlast; ++e)
    if (vals[e] > vals[kb]) kb = e;
  paths[jb.path_off + T - 1] = ids[kb];
  sval[jb.aux_off + T - 1] = vals[kb];
  int entry = kb;
  for (int k = Pe - 1; k >= 1; --k) {
    const int q = div_mid[base + (int64_t)k * Bcap + entry];
    const int e = div_b(k - 1, T, Pe);
    const int n_prev = div_n[(int64_t)b * pe_cap + k - 1];
    const int x = beam_find(div_id + base + (int64_t)(k - 1) * Bcap, n_prev, q);
    if (x < 0) { set_status(hdr, FV_EINFEASIBLE, (uint32_t)b); return; }
    paths[jb.path_off + e] = q;
    sval[jb.aux_off + e] = div_val[base + (int64_t)(k - 1) * Bcap + x];
    entry = x;
  }
}

// Large CSR beams (P = 0): one cluster of kCB CTAs per sequence when the
// device can hold such a cluster; 0 when launched, 1 when not applicable.
static int launch_beam_cluster(const BeamArgs& a, int max_jobs, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (a.trans != FV_TRANS_CSR || a.kind != kJobBeam || a.static_beam || a.K < 8192) return 1;
  if (a.Wcap < 64) return 1;  // narrow beams: one CTA per sequence has less per-step latency
  const size_t smem = cb_smem_bytes(a.K);
  if (smem > (size_t)200 * 1024) return 1;
  int clusters = a.max_ctas / kCB;
  if (max_jobs < clusters) clusters = max_jobs;
  if (clusters < 1) return 1;
  if (cudaFuncSetAttribute(beam_csr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCB;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kCBThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(kCB * clusters);
  int resident = 0;
  if (cudaOccupancyMaxActiveClusters(&resident, beam_csr_cluster_kernel, &cfg) != cudaSuccess || resident < 1) {
    cudaGetLastError();
    return 1;
  }
  if (clusters > resident) cfg.gridDim = dim3(kCB * resident);
  *err = cudaLaunchKernelEx(&cfg, beam_csr_cluster_kernel, a);
  return 0;
}

// Dense beams with 512 <= K <= 8192 (P = 0): one cluster of kDC CTAs per
// sequence when that finishes the launch sooner; 0 when launched, 1 when
// not applicable.  A cluster runs a step about r times faster than one CTA
// (measured on GB300 with 64 sequences in flight: r = 2.3 at K=1024,
// B=256; 1.4-1.6 at B=16-64) but holds kDC SMs, so the launch takes the
// cluster kernel when max(T_max, sum T / clusters) < r max(T_max, sum T / SMs),
// the two makespans in units of the cluster's step time (sequences are
// taken longest first).  Without the lengths: when every sequence gets its
// own cluster.  Never under FV_SHARED_GPU: a cluster step takes about 2.5
// times the SM time of a one-CTA step, which other decodes sharing the GPU
// would pay for (measured in the serving loop: p50 519 -> 749 ms).
static int launch_beam_dense_cluster(const BeamArgs& a, int max_jobs, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (a.trans != FV_TRANS_DENSE || a.kind != kJobBeam || a.static_beam || a.per_cta) return 1;
  if (a.K < 512 || a.K > kDCMaxK || (a.K % 32) != 0 || ((uintptr_t)a.logA & 15u) != 0) return 1;
  const int W = a.Wcap < a.Bcap ? a.Wcap : a.Bcap;
  if (W < 1) return 1;
  const size_t smem = 4 * dc_layout(a.K, W).words;
  if (smem > (size_t)200 * 1024) return 1;
  int clusters = a.max_ctas / kDC;
  if (max_jobs < clusters) clusters = max_jobs;
  if (clusters < 1) return 1;
  if (cudaFuncSetAttribute(beam_dense_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kDC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kDCThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(kDC * clusters);
  int resident = 0;
  if (cudaOccupancyMaxActiveClusters(&resident, beam_dense_cluster_kernel, &cfg) != cudaSuccess || resident < 1) {
    cudaGetLastError();
    return 1;
  }
  if (a.max_T > 0 && a.sum_T > 0) {
    const double r = W >= 128 ? 2.2 : 1.4;
    const double tmax = (double)a.max_T, tsum = (double)a.sum_T;
    const double one = std::max(tmax, tsum / (double)std::max(1, a.max_ctas));
    const double clu = std::max(tmax, tsum / (double)resident);
    if (!(clu < r * one)) return 1;
  } else if (max_jobs > resident) {
    return 1;
  }
  if (clusters > resident) cfg.gridDim = dim3(kDC * resident);
  *err = cudaLaunchKernelEx(&cfg, beam_dense_cluster_kernel, a);
  return 0;
}

cudaError_t launch_beam(const BeamArgs& a, int max_jobs, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (a.trans == FV_TRANS_DENSE && a.kind == kJobBeam && !a.static_beam && a.K <= 128) {
    if (max_jobs < 1) return cudaSuccess;
    return a.K <= 64 ? launch_small_beam_cfg<64>(a, max_jobs, st) : launch_small_beam_cfg<128>(a, max_jobs, st);
  }
  {
    cudaError_t ce;
    if (launch_beam_cluster(a, max_jobs, st, &ce) == 0) return ce;
    if (launch_beam_dense_cluster(a, max_jobs, st, &ce) == 0) return ce;
  }
  BeamArgs b = a;
  size_t smem = sizeof(uint32_t) * beam_bitmap_words(a.K);
  const size_t beam_bytes = sizeof(int32_t) * 10 * (size_t)a.Bcap;
  const size_t cand_bytes = sizeof(int32_t) * 2 * (size_t)a.K;
  b.beam_smem = smem + beam_bytes <= (size_t)160 * 1024;
  if (b.beam_smem) smem += beam_bytes;
  // the static beam keeps its full score vector in the workspace
  b.cand_smem = !a.static_beam && smem + cand_bytes <= (size_t)208 * 1024;
  if (b.cand_smem) smem += cand_bytes;
  // CSR with candidates in global memory: a shared-memory list of each
  // step's touched candidates (8 bytes each) for the top-B select
  // sized for B sources of 32 out-edges each (fewer if K is smaller); a
  // step with more touched candidates uses the K-indexed arrays.  Not used
  // when it would take most of the L1 cache the CSR gathers rely on.
  b.list_cap = 0;
  if (!b.cand_smem && !a.static_beam && a.trans != FV_TRANS_DENSE) {
    size_t cap = (size_t)a.Bcap * 32;
    if (cap > (size_t)a.K) cap = (size_t)a.K;
    cap = (cap + 3) & ~(size_t)3;  // keeps the id array 16-byte aligned
    if (smem + 8 * cap <= (size_t)160 * 1024) {
      b.list_cap = (int32_t)cap;
      smem += 8 * cap;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = max_jobs < a.max_ctas ? max_jobs : a.max_ctas;
  if (grid < 1) return cudaSuccess;
  // small dense steps (beam x targets) use a smaller CTA: every step has
  // several block-wide barriers and reductions whose cost grows with the
  // thread count while the work does not
  int threads = kBeamThreads;
  if (a.trans == FV_TRANS_DENSE) {
    const long long work = (long long)(a.Bcap < a.K ? a.Bcap : a.K) * a.K;
    if (work <= 4096) threads = 128;
    else if (work <= 16384) threads = 256;
  }
  beam_kernel<<<grid, threads, smem, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_beam_backtrack(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t Wcap,
                                  const int32_t* bp_id, const int32_t* bp_src, const int32_t* qlast, int32_t* paths,
                                  const WsHeader* hdr, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  beam_backtrack_kernel<<<(count + 127) / 128, 128, 0, st>>>(jobs, order, begin, count, Wcap, bp_id, bp_src, qlast,
                                                              paths, hdr);
  return cudaGetLastError();
}

cudaError_t launch_beam_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                                int32_t Bcap, int32_t pe_cap, int64_t div_stride, const int32_t* div_id,
                                const float* div_val, const int32_t* div_mid, const int32_t* div_n, int32_t* paths,
                                float* sval, WsHeader* hdr, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  beam_resolve_kernel<<<(count + 127) / 128, 128, 0, st>>>(jobs, order, begin, count, P, Bcap, pe_cap, div_stride,
                                                            div_id, div_val, div_mid, div_n, paths, sval, hdr);
  return cudaGetLastError();
}

int beam_max_ctas() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

}  // namespace fv
