// fv_flash.cu -- FLASH Viterbi bookkeeping kernels around the forward engine:
//  * resolve: after the root pass, q*_{T-1} = lowest argmax of delta_{T-1}
//    and, walking the P'-1 ancestor maps backwards, q*_{e_k} for every
//    division point of the P-way first split (Sec. V-A.3), with the delta
//    value there (the retained offset used by the pruned start, Sec. V-B.2);
//  * task lists of Alg. 1: level 1 holds the P' segments (e_{k-1}+1, e_k)
//    of length >= 2; the children of (m, n) with t_mid = floor((m+n)/2) are
//    (m, t_mid) and (t_mid+1, n) when n-m > 2, only (m, t_mid) when n-m = 2.
//    Lists are built level by level (every parent before its children,
//    tasks of one level in any order) and written in parent order through a
//    device-wide scan, so the order is deterministic.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fv_internal.cuh"
#include "fv_launch.h"

namespace fv {

__device__ inline int32_t pe_of(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
__device__ inline int32_t div_of(int32_t k, int32_t T, int32_t Pe) {
  return (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
}

// One warp per sequence.
__global__ void __launch_bounds__(128) flash_resolve_kernel(const Job* jobs, const int32_t* order, int32_t begin,
                                                            int32_t count, int32_t K, int32_t P,
                                                            const uint16_t* maps, const float* snaps,
                                                            int64_t map_stride, int64_t snap_stride,
                                                            int32_t* paths, float* sval, float* scores,
                                                            const WsHeader* hdr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  if (idx >= count || hdr->status != 0) return;
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  const int T = jb.T, Pe = pe_of(T, P);
  const float* sn = snaps + (int64_t)b * snap_stride;
  const uint16_t* mp = maps + (int64_t)b * map_stride;
  const float* last = sn + (int64_t)(Pe - 1) * K;
  float bv = -CUDART_INF_F;
  int bi = 0x7fffffff;
  for (int j = lane; j < K; j += 32) {
    const float v = last[j];
    if (bi == 0x7fffffff || v > bv) { bv = v; bi = j; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi != 0x7fffffff && (bi == 0x7fffffff || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
  }
  if (lane != 0) return;
  int q = bi;
  const float score = last[q];
  scores[b] = score;
  paths[jb.path_off + T - 1] = q;
  sval[jb.aux_off + T - 1] = score;
  for (int k = Pe - 2; k >= 0; --k) {
    q = mp[(int64_t)k * K + q];
    q = (unsigned)q < (unsigned)K ? q : 0;
    const int e = div_of(k, T, Pe);
    paths[jb.path_off + e] = q;
    sval[jb.aux_off + e] = sn[(int64_t)k * K + q];
  }
}

// ---------------------------------------------------------------- scan
// Pass 1: each thread's item count, exclusive scan inside the block; block
// totals to bsum.  Pass 2 (one block): exclusive scan of bsum, total to
// *out_count.  Pass 3: each thread writes its items at bsum[blk] + pos.
constexpr int kScanBlock = 256;

__device__ inline int block_excl_scan(int v, int* total) {
  __shared__ int ws[kScanBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < kScanBlock / 32 ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanBlock / 32) ws[lane] = s;
  }
  __syncthreads();
  const int excl = (w ? ws[w - 1] : 0) + x - v;
  *total = ws[kScanBlock / 32 - 1];
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(1024) scan_block_sums(int32_t* bsum, int32_t nblk, int32_t* out_count) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nblk ? bsum[i] : 0;
    // block-wide inclusive scan (1024 threads)
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int s = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const int incl = (w ? ws[w - 1] : 0) + x;
    if (i < nblk) bsum[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_count = carry;
}

// Level 1: segments of the P' split of each sequence (in `order`).
__device__ inline int level1_count(const Job& jb, int P) {
  const int T = jb.T, Pe = pe_of(T, P);
  int c = 0, prev = -1;
  for (int k = 0; k < Pe; ++k) {
    const int e = div_of(k, T, Pe);
    if (e - (prev + 1) >= 1) ++c;
    prev = e;
  }
  return c;
}

__global__ void __launch_bounds__(kScanBlock) level1_pass1(const Job* jobs, const int32_t* order, int32_t begin,
                                                           int32_t count, int32_t P, int32_t* pos, int32_t* bsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = i < count ? level1_count(jobs[order[begin + i]], P) : 0;
  int total;
  const int excl = block_excl_scan(c, &total);
  if (i < count) pos[i] = excl;
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) level1_pass3(const Job* jobs, const int32_t* order, int32_t begin,
                                                           int32_t count, int32_t P, const int32_t* pos,
                                                           const int32_t* bsum, Task* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int b = order[begin + i];
  const Job jb = jobs[b];
  const int T = jb.T, Pe = pe_of(T, P);
  int w = bsum[blockIdx.x] + pos[i], prev = -1;
  for (int k = 0; k < Pe; ++k) {
    const int e = div_of(k, T, Pe);
    if (e - (prev + 1) >= 1) {
      Task t;
      t.b = b;
      t.m = prev + 1;
      t.n = e;
      t.pad = 0;
      out[w++] = t;
    }
    prev = e;
  }
}

// Children of a task list (Alg. 1).
__device__ inline int child_count(const Task& t) {
  const int d = t.n - t.m;
  return d > 2 ? 2 : (d == 2 ? 1 : 0);
}

__global__ void __launch_bounds__(kScanBlock) child_pass1(const Task* in, const int32_t* in_count, int32_t* pos,
                                                          int32_t* bsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *in_count;
  const int c = i < n ? child_count(in[i]) : 0;
  int total;
  const int excl = block_excl_scan(c, &total);
  if (i < n) pos[i] = excl;
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) child_pass3(const Task* in, const int32_t* in_count,
                                                          const int32_t* pos, const int32_t* bsum, Task* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *in_count) return;
  const Task t = in[i];
  const int c = child_count(t);
  if (!c) return;
  const int w = bsum[blockIdx.x] + pos[i];
  const int tmid = (t.m + t.n) / 2;
  Task l;
  l.b = t.b;
  l.m = t.m;
  l.n = tmid;
  l.pad = 0;
  out[w] = l;
  if (c == 2) {
    Task r;
    r.b = t.b;
    r.m = tmid + 1;
    r.n = t.n;
    r.pad = 0;
    out[w + 1] = r;
  }
}

// ---------------------------------------------------------- budget leaves
// Greedy packing in list order: a task joins the current wave while the
// wave's backpointer rows stay within budget_rows, else it opens the next
// wave.  One block: the task rows of a chunk are staged in shared memory
// and thread 0 walks them.
constexpr int kLeafChunk = 4096;

__global__ void __launch_bounds__(1024) leaf_plan_kernel(Task* tasks, const int32_t* count, int64_t budget_rows,
                                                         int32_t wave_cap, int32_t* wave_first, int32_t* wave_count,
                                                         int32_t max_waves, WsHeader* hdr) {
  __shared__ int32_t rows[kLeafChunk];
  __shared__ int32_t w_s, first_s;
  __shared__ long long used_s;
  const int n = *count;
  if (threadIdx.x == 0) {
    w_s = 0;
    first_s = 0;
    used_s = 0;
  }
  __syncthreads();
  for (int base = 0; base < n; base += kLeafChunk) {
    const int cn = n - base < kLeafChunk ? n - base : kLeafChunk;
    for (int i = threadIdx.x; i < cn; i += blockDim.x) rows[i] = tasks[base + i].n - tasks[base + i].m;
    __syncthreads();
    if (threadIdx.x == 0) {
      int w = w_s, first = first_s;
      long long used = used_s;
      for (int i = 0; i < cn; ++i) {
        const int gi = base + i, r = rows[i];
        if ((used + r > budget_rows || (wave_cap > 0 && gi - first >= wave_cap)) && gi > first) {
          if (w < max_waves) {
            wave_first[w] = first;
            wave_count[w] = gi - first;
          }
          ++w;
          first = gi;
          used = 0;
        }
        rows[i] = (int32_t)used;  // the task's row offset in its wave
        used += r;
      }
      w_s = w;
      first_s = first;
      used_s = used;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) tasks[base + i].pad = rows[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int w = w_s;
    if (n > first_s) {
      if (w < max_waves) {
        wave_first[w] = first_s;
        wave_count[w] = n - first_s;
      }
      ++w;
    }
    if (w > max_waves) set_status(hdr, FV_EUNSUPPORTED, 0x1eaf0000u | (uint32_t)w);
    for (int k = w; k < max_waves; ++k) {
      wave_first[k] = n;
      wave_count[k] = 0;
    }
  }
}

// One warp per task; lane 0 follows the chain (each step is one dependent
// 2-byte load, so the rows are not staged).
__global__ void __launch_bounds__(128) leaf_backtrack_kernel(const Task* tasks, const int32_t* wave_first,
                                                              const int32_t* wave_count, const Job* jobs,
                                                              int32_t K, const uint16_t* leaf_psi, int32_t* paths,
                                                              const WsHeader* hdr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  if (hdr->status != 0 || idx >= *wave_count || lane != 0) return;
  const Task tk = tasks[*wave_first + idx];
  const Job jb = jobs[tk.b];
  int32_t* path = paths + jb.path_off;
  int q = path[tk.n];
  q = (unsigned)q < (unsigned)K ? q : 0;
  const uint16_t* base = leaf_psi + (int64_t)tk.pad * K;
  for (int t = tk.n; t > tk.m; --t) {
    q = base[(int64_t)(t - tk.m - 1) * K + q];
    q = q < K ? q : 0;
    path[t - 1] = q;
  }
}

cudaError_t launch_leaf_plan(Task* tasks, const int32_t* count, int64_t budget_rows, int32_t wave_cap,
                             int32_t* wave_first, int32_t* wave_count, int32_t max_waves, WsHeader* hdr,
                             cudaStream_t st) {
  leaf_plan_kernel<<<1, 1024, 0, st>>>(tasks, count, budget_rows, wave_cap, wave_first, wave_count, max_waves, hdr);
  return cudaGetLastError();
}

cudaError_t launch_leaf_backtrack(const Task* tasks, const int32_t* wave_first, const int32_t* wave_count,
                                  int32_t max_count, const Job* jobs, int32_t K, const uint16_t* leaf_psi,
                                  int32_t* paths, const WsHeader* hdr, cudaStream_t st) {
  if (max_count <= 0) return cudaSuccess;
  leaf_backtrack_kernel<<<(max_count + 3) / 4, 128, 0, st>>>(tasks, wave_first, wave_count, jobs, K, leaf_psi, paths,
                                                             hdr);
  return cudaGetLastError();
}

// ------------------------------------------------- Checkpoint Viterbi
// The baseline of Sec. II-A: the forward pass (engine, kJobRoot with ckpt)
// keeps delta at C checkpoints e_k in each sequence's area; then segment k
// (steps e_{k-1}+1 .. e_k) is decoded again from checkpoint k-1 (segment 0
// from pi), latest segment first, one segment per sequence per level, and
// backtracked from the state already known at its end.

// One warp per sequence: q_{T-1} = lowest argmax of the last checkpoint
// (delta_{T-1}), its score and the path's last state.
__global__ void __launch_bounds__(128) ckpt_resolve_kernel(const Job* jobs, const int32_t* order, int32_t begin,
                                                           int32_t count, int32_t K, int32_t P, const float* area,
                                                           int32_t* paths, float* scores, const WsHeader* hdr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * (blockDim.x >> 5) + warp;
  if (idx >= count || hdr->status != 0) return;
  const int b = order[begin + idx];
  const Job jb = jobs[b];
  const float* last = area + jb.aux_off + (int64_t)(ckpt_count(jb.T, P) - 1) * K;
  float bv = -CUDART_INF_F;
  int bi = 0x7fffffff;
  for (int j = lane; j < K; j += 32) {
    const float v = last[j];
    if (bi == 0x7fffffff || v > bv) { bv = v; bi = j; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi != 0x7fffffff && (bi == 0x7fffffff || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
  }
  if (lane == 0) {
    scores[b] = last[bi];
    paths[jb.path_off + jb.T - 1] = bi;
  }
}

// Level `level` of the segment lists: for every sequence (in `order`) with
// more than `level` checkpoints, its segment C-1-level (one CTA, block scan
// so the list keeps the sequence order).  Segments without a step (segment
// 0 when e_0 = 0) are left out: their state is written by the next
// segment's backtrack.
__global__ void __launch_bounds__(1024) ckpt_tasks_kernel(const Job* jobs, const int32_t* order, int32_t begin,
                                                          int32_t count, int32_t P, int32_t level, Task* out,
                                                          int32_t* out_count) {
  __shared__ int warp_sum[32];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < count; base += blockDim.x) {
    const int i = base + tid;
    Task tk;
    int has = 0;
    if (i < count) {
      const int b = order[begin + i];
      const Job jb = jobs[b];
      const int C = ckpt_count(jb.T, P), k = C - 1 - level;
      if (k >= 0) {
        tk.b = b;
        tk.m = k == 0 ? 0 : div_of(k - 1, jb.T, C);
        tk.n = div_of(k, jb.T, C);
        tk.pad = k - 1;
        has = tk.n > tk.m;
      }
    }
    int x = has;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
      int v = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      warp_sum[lane] = v;
    }
    __syncthreads();
    const int pos = carry + (w ? warp_sum[w - 1] : 0) + x - has;
    if (has) out[pos] = tk;
    __syncthreads();
    if (tid == blockDim.x - 1) carry = pos + has;
    __syncthreads();
  }
  if (tid == 0) *out_count = carry;
}

// One thread per segment: follow q_{t-1} = psi_t[q_t] from the known
// q_n through the segment's rows (stored after the checkpoints).
__global__ void __launch_bounds__(128) ckpt_backtrack_kernel(const Task* tasks, const int32_t* count,
                                                             const Job* jobs, int32_t K, int32_t P,
                                                             const uint16_t* area16, int32_t* paths,
                                                             const WsHeader* hdr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (hdr->status != 0 || idx >= *count) return;
  const Task tk = tasks[idx];
  const Job jb = jobs[tk.b];
  int32_t* path = paths + jb.path_off;
  const uint16_t* base = area16 + 2 * (jb.aux_off + (int64_t)ckpt_count(jb.T, P) * K);
  int q = path[tk.n];
  q = (unsigned)q < (unsigned)K ? q : 0;
  for (int t = tk.n; t > tk.m; --t) {
    q = base[(int64_t)(t - tk.m - 1) * K + q];
    q = q < K ? q : 0;
    path[t - 1] = q;
  }
}

cudaError_t launch_ckpt_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t K,
                                int32_t P, const float* area, int32_t* paths, float* scores, const WsHeader* hdr,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  ckpt_resolve_kernel<<<(count + 3) / 4, 128, 0, st>>>(jobs, order, begin, count, K, P, area, paths, scores, hdr);
  return cudaGetLastError();
}

cudaError_t launch_ckpt_tasks(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                              int32_t level, Task* out, int32_t* out_count, cudaStream_t st) {
  ckpt_tasks_kernel<<<1, 1024, 0, st>>>(jobs, order, begin, count, P, level, out, out_count);
  return cudaGetLastError();
}

cudaError_t launch_ckpt_backtrack(const Task* tasks, const int32_t* count, int32_t max_count, const Job* jobs,
                                  int32_t K, int32_t P, const uint16_t* area16, int32_t* paths, const WsHeader* hdr,
                                  cudaStream_t st) {
  if (max_count <= 0) return cudaSuccess;
  ckpt_backtrack_kernel<<<(max_count + 127) / 128, 128, 0, st>>>(tasks, count, jobs, K, P, area16, paths, hdr);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FV_CHECKED
__device__ inline bool bad_score(float x) { return isnan(x) || (isinf(x) && x > 0.f); }

__global__ void check_array_kernel(const float* x, int64_t n, uint32_t what, WsHeader* hdr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (bad_score(x[i])) {
      set_status(hdr, FV_EINVAL, what);
      return;
    }
}

__global__ void check_csr_kernel(const int32_t* row_ptr, const int32_t* col, int32_t K, int64_t nnz, uint32_t what,
                                 WsHeader* hdr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[K] != nnz)) set_status(hdr, FV_EINVAL, what);
  for (int64_t i = i0; i < K; i += stride)
    if (row_ptr[i + 1] < row_ptr[i]) set_status(hdr, FV_EINVAL, what);
  for (int64_t e = i0; e < nnz; e += stride)
    if ((unsigned)col[e] >= (unsigned)K) set_status(hdr, FV_EINVAL, what);
}

// Emission rows (dense) or symbols (discrete) of every sequence of one
// model: CTA y takes sequence y, its threads stride over the T*K values.
__global__ void check_emissions_kernel(const Job* jobs, int32_t b0, int32_t model, int32_t K, const float* E,
                                       const int32_t* obs, int32_t V, WsHeader* hdr) {
  const int b = b0 + blockIdx.y;
  const Job jb = jobs[b];
  if (jb.model != model) return;
  const int64_t n = E ? (int64_t)jb.T * K : (int64_t)jb.T;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (E ? bad_score(E[jb.e_off + i]) : (unsigned)obs[jb.e_off + i] >= (unsigned)V) {
      set_status(hdr, FV_EINVAL, 0xe0000000u | (uint32_t)b);
      return;
    }
  }
}

cudaError_t launch_check_inputs(const fv_model& m, int32_t model, const Job* jobs, int32_t n_seq, const float* E,
                                const int32_t* obs, WsHeader* hdr, cudaStream_t st) {
  const uint32_t tag = 0xc0000000u | ((uint32_t)model << 8);
  check_array_kernel<<<64, 256, 0, st>>>(m.log_pi, m.K, tag | 1u, hdr);
  if (m.trans == FV_TRANS_DENSE) {
    check_array_kernel<<<1024, 256, 0, st>>>(m.logA, (int64_t)m.K * m.K, tag | 2u, hdr);
  } else {
    check_array_kernel<<<1024, 256, 0, st>>>(m.val, m.nnz, tag | 3u, hdr);
    check_csr_kernel<<<256, 256, 0, st>>>(m.row_ptr, m.col, m.K, m.nnz, tag | 4u, hdr);
  }
  if (m.emit == FV_EMIT_DISCRETE) check_array_kernel<<<256, 256, 0, st>>>(m.logB, (int64_t)m.K * m.V, tag | 5u, hdr);
  for (int b0 = 0; b0 < n_seq; b0 += 65535) {
    const int nb = n_seq - b0 < 65535 ? n_seq - b0 : 65535;
    check_emissions_kernel<<<dim3(16, nb), 256, 0, st>>>(jobs, b0, model, m.K, m.emit == FV_EMIT_DENSE ? E : nullptr,
                                                         obs, m.V, hdr);
  }
  return cudaGetLastError();
}

__global__ void reset_counter(unsigned long long* pop) { *pop = 0ull; }

cudaError_t launch_reset(unsigned long long* pop, cudaStream_t st) {
  reset_counter<<<1, 1, 0, st>>>(pop);
  return cudaGetLastError();
}

cudaError_t launch_flash_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t K,
                                 int32_t P, const uint16_t* maps, const float* snaps, int64_t map_stride,
                                 int64_t snap_stride, int32_t* paths, float* sval, float* scores,
                                 const WsHeader* hdr, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  flash_resolve_kernel<<<(count + 3) / 4, 128, 0, st>>>(jobs, order, begin, count, K, P, maps, snaps, map_stride,
                                                        snap_stride, paths, sval, scores, hdr);
  return cudaGetLastError();
}

cudaError_t launch_level1_tasks(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                                Task* out, int32_t* out_count, ScanTmp tmp, cudaStream_t st) {
  const int nblk = (count + kScanBlock - 1) / kScanBlock;
  if (nblk == 0) return cudaSuccess;
  level1_pass1<<<nblk, kScanBlock, 0, st>>>(jobs, order, begin, count, P, tmp.pos, tmp.bsum);
  scan_block_sums<<<1, 1024, 0, st>>>(tmp.bsum, nblk, out_count);
  level1_pass3<<<nblk, kScanBlock, 0, st>>>(jobs, order, begin, count, P, tmp.pos, tmp.bsum, out);
  return cudaGetLastError();
}

cudaError_t launch_child_tasks(const Task* in, const int32_t* in_count, int32_t max_in, Task* out,
                               int32_t* out_count, ScanTmp tmp, unsigned long long* pop_reset, cudaStream_t st) {
  const int nblk = (max_in + kScanBlock - 1) / kScanBlock;
  if (pop_reset) reset_counter<<<1, 1, 0, st>>>(pop_reset);
  if (nblk == 0) return cudaGetLastError();
  child_pass1<<<nblk, kScanBlock, 0, st>>>(in, in_count, tmp.pos, tmp.bsum);
  scan_block_sums<<<1, 1024, 0, st>>>(tmp.bsum, nblk, out_count);
  child_pass3<<<nblk, kScanBlock, 0, st>>>(in, in_count, tmp.pos, tmp.bsum, out);
  return cudaGetLastError();
}

}  // namespace fv
