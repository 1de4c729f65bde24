// fv_api.cu -- the extern "C" boundary of libfv: argument checks, workspace
// layout, and the launch sequence for each mode.  No device memory is
// allocated here; every scratch byte is carved out of the caller's workspace.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "fv_internal.cuh"

#include "fv_launch.h"

using namespace fv;

namespace {

// Per-model sequence ranges of the model-major order.
struct Ranges {
  std::vector<int32_t> count, begin;
};

Ranges model_ranges(const fv_batch* b, int32_t n_models) {
  Ranges r;
  r.count.assign(n_models, 0);
  r.begin.assign(n_models, 0);
  if (b->model_host) {
    for (int i = 0; i < b->n_seq; ++i) r.count[b->model_host[i]]++;
  } else {
    r.count[0] = b->n_seq;
  }
  for (int m = 1; m < n_models; ++m) r.begin[m] = r.begin[m - 1] + r.count[m - 1];
  return r;
}

int32_t pe_host(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}

// Tasks per level below a segment of length L (index 0 = the segment's own
// level), following the children rule of Alg. 1.
const std::vector<int64_t>& level_counts(int64_t L, std::unordered_map<int64_t, std::vector<int64_t>>& memo) {
  auto it = memo.find(L);
  if (it != memo.end()) return it->second;
  std::vector<int64_t> r;
  if (L >= 2) {
    r.push_back(1);
    const int64_t d = L - 1, left = d / 2 + 1, right = L - left;
    auto add = [&](int64_t len) {
      const std::vector<int64_t>& c = level_counts(len, memo);
      if (r.size() < c.size() + 1) r.resize(c.size() + 1, 0);
      for (size_t k = 0; k < c.size(); ++k) r[k + 1] += c[k];
    };
    if (d > 2) { add(left); add(right); }
    else if (d == 2) add(left);
  }
  return memo.emplace(L, std::move(r)).first->second;
}

// Largest task length and total backpointer rows (n - m) per level below a
// segment of length L: a task of length L has children of lengths
// floor((L-1)/2)+1 and L - that (only the first when L == 3).
struct LevelRows {
  std::vector<int64_t> max_len, rows;
};
const LevelRows& level_rows(int64_t L, std::unordered_map<int64_t, LevelRows>& memo) {
  auto it = memo.find(L);
  if (it != memo.end()) return it->second;
  LevelRows r;
  if (L >= 2) {
    r.max_len.push_back(L);
    r.rows.push_back(L - 1);
    const int64_t d = L - 1, left = d / 2 + 1, right = L - left;
    auto add = [&](int64_t len) {
      const LevelRows& c = level_rows(len, memo);
      if (r.rows.size() < c.rows.size() + 1) {
        r.rows.resize(c.rows.size() + 1, 0);
        r.max_len.resize(c.rows.size() + 1, 0);
      }
      for (size_t k = 0; k < c.rows.size(); ++k) {
        r.rows[k + 1] += c.rows[k];
        r.max_len[k + 1] = std::max(r.max_len[k + 1], c.max_len[k]);
      }
    };
    if (d > 2) { add(left); add(right); }
    else if (d == 2) add(left);
  }
  return memo.emplace(L, std::move(r)).first->second;
}

struct FlashPlan {
  std::vector<int32_t> levels;      // per model: number of subtask levels
  std::vector<int64_t> max_tasks;   // per model: largest level
  int64_t list_cap = 0;             // entries per task list (max over models, >= level-1 lists)
  int32_t pe_max = 1, k_max = 1;
  // budget leaves (exact FLASH with a backpointer budget): per model the
  // first level whose every task's rows fit the budget (-1: none), the
  // budget in rows, and an upper bound on the waves of that level
  std::vector<int32_t> leaf_level, leaf_waves, leaf_cap;
  std::vector<int64_t> leaf_rows, leaf_tasks;
  int32_t waves_max = 0;
  size_t leaf_bytes = 0;
};

// The sequence order of the device's order kernel (model asc, then T desc
// unless nosort, then index asc), replayed from the host lengths.
std::vector<int32_t> host_order(const fv_batch* b, bool nosort) {
  std::vector<int32_t> o(b->n_seq);
  for (int i = 0; i < b->n_seq; ++i) o[i] = i;
  auto model = [&](int i) { return b->model_host ? b->model_host[i] : 0; };
  std::sort(o.begin(), o.end(), [&](int x, int y) {
    if (model(x) != model(y)) return model(x) < model(y);
    if (!nosort && b->T_host[x] != b->T_host[y]) return b->T_host[x] > b->T_host[y];
    return x < y;
  });
  return o;
}

// Waves of the budget-leaf level exactly as the device plans them: the
// level's task list in device order (segments of each sequence in `order`,
// then children in parent order), packed greedily into waves of at most R
// backpointer rows.  Returns the wave count; *max_wave = the largest wave.
int32_t host_leaf_waves(const fv_batch* b, const std::vector<int32_t>& order, int32_t model, int32_t P,
                        int32_t level, int64_t R, int32_t cap, int64_t* max_wave) {
  std::vector<int32_t> cur, nxt;
  for (int32_t i : order) {
    if ((b->model_host ? b->model_host[i] : 0) != model) continue;
    const int32_t T = b->T_host[i], Pe = pe_host(T, P);
    int32_t prev = -1;
    for (int k = 0; k < Pe; ++k) {
      const int32_t e = (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
      if (e - prev >= 2) cur.push_back(e - prev);
      prev = e;
    }
  }
  for (int l = 0; l < level; ++l) {
    nxt.clear();
    for (int32_t L : cur) {
      const int32_t d = L - 1, left = d / 2 + 1;
      if (d > 2) { nxt.push_back(left); nxt.push_back(L - left); }
      else if (d == 2) nxt.push_back(left);
    }
    cur.swap(nxt);
  }
  int32_t waves = 0;
  int64_t used = 0, first = 0;
  *max_wave = 0;
  for (size_t i = 0; i < cur.size(); ++i) {
    const int64_t r = cur[i] - 1;
    if ((used + r > R || (cap > 0 && (int64_t)i - first >= cap)) && (int64_t)i > first) {
      *max_wave = std::max<int64_t>(*max_wave, (int64_t)i - first);
      ++waves;
      first = (int64_t)i;
      used = 0;
    }
    used += r;
  }
  if ((int64_t)cur.size() > first) {
    *max_wave = std::max<int64_t>(*max_wave, (int64_t)cur.size() - first);
    ++waves;
  }
  return waves;
}

FlashPlan plan_flash(const fv_model* models, int32_t n_models, const fv_batch* b, int32_t P,
                     uint64_t budget_bytes = 0, bool nosort = false) {
  FlashPlan fp;
  fp.levels.assign(n_models, 0);
  fp.max_tasks.assign(n_models, 0);
  fp.leaf_level.assign(n_models, -1);
  fp.leaf_waves.assign(n_models, 0);
  fp.leaf_cap.assign(n_models, 0);
  fp.leaf_rows.assign(n_models, 0);
  fp.leaf_tasks.assign(n_models, 0);
  std::vector<std::vector<int64_t>> per(n_models), maxlen(n_models), rows(n_models);
  std::unordered_map<int64_t, std::vector<int64_t>> memo;
  std::unordered_map<int64_t, LevelRows> memo_rows;
  for (int i = 0; i < b->n_seq; ++i) {
    const int m = b->model_host ? b->model_host[i] : 0;
    const int32_t T = b->T_host[i], Pe = pe_host(T, P);
    if (Pe > fp.pe_max) fp.pe_max = Pe;
    int32_t prev = -1;
    for (int k = 0; k < Pe; ++k) {
      const int32_t e = (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
      const std::vector<int64_t>& c = level_counts(e - prev, memo);
      if (per[m].size() < c.size()) per[m].resize(c.size(), 0);
      for (size_t l = 0; l < c.size(); ++l) per[m][l] += c[l];
      if (budget_bytes) {
        const LevelRows& lr = level_rows(e - prev, memo_rows);
        if (rows[m].size() < lr.rows.size()) {
          rows[m].resize(lr.rows.size(), 0);
          maxlen[m].resize(lr.rows.size(), 0);
        }
        for (size_t l = 0; l < lr.rows.size(); ++l) {
          rows[m][l] += lr.rows[l];
          maxlen[m][l] = std::max(maxlen[m][l], lr.max_len[l]);
        }
      }
      prev = e;
    }
  }
  std::vector<int32_t> order;
  for (int m = 0; m < n_models; ++m) {
    if (models[m].K > fp.k_max) fp.k_max = models[m].K;
    fp.levels[m] = (int32_t)per[m].size();
    for (int64_t c : per[m]) fp.max_tasks[m] = std::max(fp.max_tasks[m], c);
    fp.list_cap = std::max(fp.list_cap, fp.max_tasks[m]);
    if (!budget_bytes) continue;
    const int64_t R = (int64_t)(budget_bytes / (2ull * (uint64_t)models[m].K));
    for (size_t l = 0; l < rows[m].size() && R >= 1; ++l) {
      const int64_t mr = maxlen[m][l] - 1;  // rows of the level's largest task
      if (mr > R) continue;
      fp.leaf_level[m] = (int32_t)l;
      fp.leaf_rows[m] = R;
      if (order.empty()) order = host_order(b, nosort);
      int64_t mw = 0;
      fp.leaf_cap[m] = dense_job_slots(models[m].K);
      fp.leaf_waves[m] = host_leaf_waves(b, order, m, P, (int32_t)l, R, fp.leaf_cap[m], &mw);
      fp.leaf_tasks[m] = mw;
      fp.waves_max = std::max(fp.waves_max, fp.leaf_waves[m]);
      fp.leaf_bytes = std::max(fp.leaf_bytes, (size_t)R * (size_t)models[m].K * sizeof(uint16_t));
      break;
    }
  }
  fp.list_cap = std::max<int64_t>(fp.list_cap, b->n_seq);
  return fp;
}

struct Layout {
  size_t hdr, jobs, order, qlast, aux, aux2, maps, snaps, listA, listB, pos, bsum, counts, total;
  size_t leaf, waves;  // budget leaves: backpointer area, wave [first | count] arrays
  size_t bscratch, div_id, div_val, div_mid, div_n;
  size_t ap, snapx;  // streamed exact configurations (K > 256)
  size_t wide;       // whole-GPU configuration scratch (K > 1024)
  size_t at;         // column-major logA copy of the streamed configurations (256 < K <= 1024)
  uint64_t aux_elems;
  int64_t map_stride, snap_stride, list_cap;
  int32_t Wcap, Bcap, pe_cap, max_ctas;
  size_t bstride;
};

int32_t beam_wcap(const fv_model* models, int32_t n_models, int32_t B) {
  int32_t kmax = 1;
  for (int m = 0; m < n_models; ++m) kmax = std::max(kmax, models[m].K);
  return std::min(std::max(B, 1), kmax);
}

// Workspace layout of a request.  fp: task-level plan (FLASH, and BEAM
// with P >= 1).  The per-sequence aux area holds: vanilla, T*K uint16
// backpointers; flash and FLASH-BS, T floats of delta along the path; beam
// with P = 0, T*Wcap int32 state ids (a second area of the same size holds
// the source slots).
Layout layout_for(const fv_model* models, int32_t n_models, const fv_batch* b, int mode, const FlashPlan* fp,
                  int32_t B = 0, int32_t ckpt_P = 0) {
  Layout L;
  memset(&L, 0, sizeof(L));
  const int32_t n = b->n_seq;
  int32_t kmax = 1;
  for (int m = 0; m < n_models; ++m) kmax = std::max(kmax, models[m].K);
  const bool beam0 = mode == FV_BEAM && fp == nullptr;
  if (mode == FV_BEAM) L.Wcap = beam_wcap(models, n_models, B);
  L.hdr = 0;
  L.jobs = align_up(sizeof(WsHeader));
  L.order = align_up(L.jobs + sizeof(Job) * (size_t)n);
  L.qlast = align_up(L.order + sizeof(int32_t) * (size_t)n);
  L.aux = align_up(L.qlast + sizeof(int32_t) * (size_t)n);
  uint64_t aux = 0;
  for (int i = 0; i < n && b->T_host; ++i) {
    const int m = b->model_host ? b->model_host[i] : 0;
    const uint64_t T = (uint64_t)b->T_host[i], K = (uint64_t)models[m].K;
    if (mode == FV_VANILLA) aux += (T * K + 7ull) & ~7ull;
    else if (beam0) aux += (T * (uint64_t)L.Wcap + 3ull) & ~3ull;
    else if (mode == FV_CHECKPOINT) aux += ckpt_area((int32_t)T, ckpt_P, (int32_t)K);
    else aux += (T + 3ull) & ~3ull;
  }
  L.aux_elems = aux;
  size_t end = align_up(L.aux + aux * (mode == FV_VANILLA ? 2 : 4));
  if (beam0) {
    L.aux2 = end;
    end = align_up(L.aux2 + 4 * (size_t)aux);
  }
  if (mode == FV_CHECKPOINT) {
    // one segment list (a segment per sequence per level) and its count
    L.list_cap = std::max<int64_t>(n, 1);
    L.listA = end;
    L.counts = align_up(L.listA + sizeof(Task) * (size_t)L.list_cap);
    end = align_up(L.counts + 64);
  }
  if (fp) {
    L.list_cap = fp->list_cap;
    L.listA = end;
    L.listB = align_up(L.listA + sizeof(Task) * (size_t)L.list_cap);
    L.pos = align_up(L.listB + sizeof(Task) * (size_t)L.list_cap);
    L.bsum = align_up(L.pos + sizeof(int32_t) * (size_t)L.list_cap);
    L.counts = align_up(L.bsum + sizeof(int32_t) * (size_t)(L.list_cap / 256 + 2));
    end = align_up(L.counts + 64);
  }
  if (mode == FV_FLASH && fp) {
    L.map_stride = (int64_t)(fp->pe_max > 1 ? fp->pe_max - 1 : 1) * fp->k_max;
    L.snap_stride = (int64_t)fp->pe_max * fp->k_max;
    L.maps = end;
    L.snaps = align_up(L.maps + sizeof(uint16_t) * (size_t)L.map_stride * n);
    end = align_up(L.snaps + sizeof(float) * (size_t)L.snap_stride * n);
    if (fp->leaf_bytes) {
      L.leaf = end;
      L.waves = align_up(L.leaf + fp->leaf_bytes);
      end = align_up(L.waves + 2 * sizeof(int32_t) * (size_t)fp->waves_max);
    }
  }
  if (mode != FV_BEAM) {
    // row-pair copy of the largest streamed model's logA, reused per model,
    // and the streamed sub-job snapshots of every possible cluster
    size_t ap_bytes = 0;
    int32_t kpm_max = 0;
    for (int m = 0; m < n_models; ++m) {
      int kpm = 0, cols = 0;
      dense_stream_geometry(models[m].K, &kpm, &cols);
      ap_bytes = std::max(ap_bytes, (size_t)(kpm / 2) * cols * 8);
      kpm_max = std::max(kpm_max, kpm);
    }
    // resident K <= 256 configurations may keep their sub snapshots here too
    bool resident_256 = false;
    for (int m = 0; m < n_models; ++m) resident_256 |= models[m].K > 128 && models[m].K <= 256;
    if (resident_256 && !ap_bytes) {
      const int nsm = device_sm_count();
      L.snapx = end;
      end = align_up(L.snapx + sizeof(float) * (size_t)nsm * 1024);
    }
    if (ap_bytes) {
      const int nsm = device_sm_count();
      L.ap = end;
      L.snapx = align_up(L.ap + ap_bytes);
      end = align_up(L.snapx + sizeof(float) * std::max((size_t)(nsm / 4 + 1) * 8 * kpm_max, (size_t)nsm * 1024));
      if (kmax > 1024) {
        L.wide = end;
        end = align_up(L.wide + wide_scratch_bytes(kmax, nsm));
      }
      // streamed models (K <= 1024) share one column-major copy, sized for the largest
      int32_t ks = 0;
      for (int m = 0; m < n_models; ++m)
        if (models[m].K > 256 && models[m].K <= 1024) ks = std::max(ks, models[m].K);
      if (ks) {
        L.at = end;
        end = align_up(L.at + sizeof(float) * (size_t)ks * wide_lane_stride(ks));
      }
    }
  }
  if (mode == FV_BEAM) {
    L.Bcap = fp ? kmax : L.Wcap;  // FLASH-BS subtasks may be re-run with every state
    L.max_ctas = fv::beam_max_ctas();
    if (L.max_ctas < 1) L.max_ctas = 1;
    L.bstride = align_up(beam_scratch_stride(kmax, L.Bcap));
    L.bscratch = end;
    end = align_up(L.bscratch + L.bstride * (size_t)L.max_ctas);
    if (fp) {
      L.pe_cap = fp->pe_max;
      const size_t per = (size_t)L.pe_cap * L.Wcap * n;
      L.div_id = end;
      L.div_val = align_up(L.div_id + 4 * per);
      L.div_mid = align_up(L.div_val + 4 * per);
      L.div_n = align_up(L.div_mid + 4 * per);
      end = align_up(L.div_n + 4 * (size_t)L.pe_cap * n);
    }
  }
  L.total = end < 4096 ? 4096 : end;
  return L;
}

bool model_ok(const fv_model& m) {
  if (m.K < 1 || m.K > 65536 || !m.log_pi) return false;
  if (m.trans == FV_TRANS_DENSE) {
    if (!m.logA) return false;
  } else if (m.trans == FV_TRANS_CSR) {
    if (!m.row_ptr || !m.col || !m.val || m.nnz < 0) return false;
  } else {
    return false;
  }
  if (m.emit == FV_EMIT_DISCRETE) {
    if (m.V < 1 || !m.logB) return false;
  } else if (m.emit != FV_EMIT_DENSE) {
    return false;
  }
  return true;
}

fv_status check_common(const fv_model* models, int32_t n_models, const fv_batch* b) {
  if (!models || !b || n_models < 1 || n_models > kMaxModels) return FV_EINVAL;
  if (b->n_seq < 0) return FV_EINVAL;
  for (int m = 0; m < n_models; ++m)
    if (!model_ok(models[m])) return FV_EINVAL;
  if (b->n_seq == 0) return FV_OK;
  if (!b->T || !b->e_off || !b->path_off) return FV_EINVAL;
  if (n_models > 1 && (!b->model_idx || !b->model_host)) return FV_EINVAL;
  bool need_E = false, need_obs = false;
  for (int m = 0; m < n_models; ++m) {
    if (models[m].emit == FV_EMIT_DENSE) need_E = true;
    else need_obs = true;
  }
  if ((need_E && !b->E) || (need_obs && !b->obs)) return FV_EINVAL;
  if (b->T_host) {
    for (int i = 0; i < b->n_seq; ++i) {
      if (b->T_host[i] < 1) return FV_EINVAL;
      const int m = b->model_host ? b->model_host[i] : 0;
      if (m < 0 || m >= n_models) return FV_EINVAL;
    }
  }
  return FV_OK;
}

// Library-owned event pairs around the main decode kernel (timing hook).
constexpr int kMaxTimed = 256;
bool g_timing = false;
int g_timed = 0;
cudaEvent_t g_ev[2 * kMaxTimed];
bool g_ev_made = false;

void timed_begin(cudaStream_t st) {
  if (!g_timing || g_timed >= kMaxTimed) return;
  cudaEventRecord(g_ev[2 * g_timed], st);
}
void timed_end(cudaStream_t st) {
  if (!g_timing || g_timed >= kMaxTimed) return;
  cudaEventRecord(g_ev[2 * g_timed + 1], st);
  ++g_timed;
}

// Beam search (P = 0) and FLASH-BS (P >= 1) launch sequence, per model.
fv_status decode_beam(const fv_model* models, int32_t n_models, const fv_batch* batch, const fv_params* p, char* ws,
                      const Layout& L, const FlashPlan& fp, const Ranges& R, int32_t* paths_out, float* scores_out,
                      cudaStream_t st) {
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.hdr);
  Job* jobs = reinterpret_cast<Job*>(ws + L.jobs);
  int32_t* order = reinterpret_cast<int32_t*>(ws + L.order);
  int32_t* qlast = reinterpret_cast<int32_t*>(ws + L.qlast);
  const bool tasks = p->P >= 1;
  for (int m = 0; m < n_models; ++m) {
    if (!R.count[m]) continue;
    const fv_model& md = models[m];
    BeamArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.K = md.K;
    ba.trans = md.trans;
    ba.emit = md.emit;
    ba.V = md.V;
    ba.log_pi = md.log_pi;
    ba.logA = md.logA;
    ba.row_ptr = md.row_ptr;
    ba.col = md.col;
    ba.val = md.val;
    ba.logB = md.logB;
    ba.E = batch->E;
    ba.obs = batch->obs;
    ba.jobs = jobs;
    ba.order = order;
    ba.order_begin = R.begin[m];
    ba.order_count = R.count[m];
    ba.pop = &hdr->pop[m];
    ba.B = p->B;
    ba.Wcap = L.Wcap;
    ba.Bcap = L.Bcap;
    ba.P = p->P;
    ba.complete = (p->flags & FV_COMPLETE_PRUNING) ? 1 : 0;
    ba.static_beam = (p->flags & FV_STATIC_BEAM) ? 1 : 0;
    ba.per_cta = (p->flags & FV_SHARED_GPU) ? 1 : 0;
    ba.max_ctas = L.max_ctas;
    ba.scratch = ws + L.bscratch;
    ba.scratch_stride = L.bstride;
    ba.qlast = qlast;
    ba.scores = scores_out;
    ba.paths = paths_out;
    ba.hdr = hdr;
    if (batch->T_host) {
      for (int i = 0; i < batch->n_seq; ++i) {
        if ((batch->model_host ? batch->model_host[i] : 0) != m) continue;
        ba.sum_T += batch->T_host[i];
        if (batch->T_host[i] > ba.max_T) ba.max_T = batch->T_host[i];
      }
    }
    if (m > 0 && launch_reset(ba.pop, st) != cudaSuccess) return FV_ECUDA;
    if (!tasks) {
      ba.kind = kJobBeam;
      ba.bp_id = reinterpret_cast<int32_t*>(ws + L.aux);
      ba.bp_src = reinterpret_cast<int32_t*>(ws + L.aux2);
      timed_begin(st);
      if (launch_beam(ba, R.count[m], st) != cudaSuccess) return FV_ECUDA;
      timed_end(st);
      if (launch_beam_backtrack(jobs, order, R.begin[m], R.count[m], L.Wcap, ba.bp_id, ba.bp_src, qlast, paths_out,
                                hdr, st) != cudaSuccess)
        return FV_ECUDA;
      continue;
    }
    // FLASH-BS: beam root with division-point beams, resolve, task levels
    float* sval = reinterpret_cast<float*>(ws + L.aux);
    Task* lists[2] = {reinterpret_cast<Task*>(ws + L.listA), reinterpret_cast<Task*>(ws + L.listB)};
    int32_t* counts = reinterpret_cast<int32_t*>(ws + L.counts);
    ScanTmp tmp;
    tmp.pos = reinterpret_cast<int32_t*>(ws + L.pos);
    tmp.bsum = reinterpret_cast<int32_t*>(ws + L.bsum);
    ba.sval = sval;
    ba.div_id = reinterpret_cast<int32_t*>(ws + L.div_id);
    ba.div_val = reinterpret_cast<float*>(ws + L.div_val);
    ba.div_mid = reinterpret_cast<int32_t*>(ws + L.div_mid);
    ba.div_n = reinterpret_cast<int32_t*>(ws + L.div_n);
    ba.pe_cap = L.pe_cap;
    ba.div_stride = (int64_t)L.pe_cap * L.Wcap;
    ba.kind = kJobRoot;
    timed_begin(st);
    if (launch_beam(ba, R.count[m], st) != cudaSuccess) return FV_ECUDA;
    if (launch_beam_resolve(jobs, order, R.begin[m], R.count[m], p->P, L.Wcap, L.pe_cap, ba.div_stride, ba.div_id,
                            ba.div_val, ba.div_mid, ba.div_n, paths_out, sval, hdr, st) != cudaSuccess)
      return FV_ECUDA;
    if (fp.levels[m] > 0 &&
        launch_level1_tasks(jobs, order, R.begin[m], R.count[m], p->P, lists[0], &counts[0], tmp, st) != cudaSuccess)
      return FV_ECUDA;
    int c = 0;
    for (int lvl = 0; lvl < fp.levels[m]; ++lvl) {
      if (launch_reset(ba.pop, st) != cudaSuccess) return FV_ECUDA;
      ba.kind = kJobSub;
      ba.tasks = lists[c];
      ba.task_count = &counts[c];
      if (launch_beam(ba, (int)fp.max_tasks[m], st) != cudaSuccess) return FV_ECUDA;
      if (lvl + 1 < fp.levels[m] &&
          launch_child_tasks(lists[c], &counts[c], (int32_t)fp.max_tasks[m], lists[c ^ 1], &counts[c ^ 1], tmp,
                             nullptr, st) != cudaSuccess)
        return FV_ECUDA;
      c ^= 1;
    }
    timed_end(st);
    // score of the returned path: forward-order log-likelihood (R10)
    ScoreArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.K = md.K;
    sa.trans = md.trans;
    sa.emit = md.emit;
    sa.V = md.V;
    sa.log_pi = md.log_pi;
    sa.logA = md.logA;
    sa.row_ptr = md.row_ptr;
    sa.col = md.col;
    sa.val = md.val;
    sa.logB = md.logB;
    sa.E = batch->E;
    sa.obs = batch->obs;
    if (launch_path_score(sa, jobs, order, R.begin[m], R.count[m], paths_out, scores_out, hdr, st) != cudaSuccess)
      return FV_ECUDA;
  }
  return FV_OK;
}

}  // namespace

extern "C" {

const char* fv_version(void) { return "libfv 0.1 (sm_103a)"; }

const char* fv_status_str(fv_status s) {
  switch (s) {
    case FV_OK: return "ok";
    case FV_EINVAL: return "invalid argument";
    case FV_ENOMEM: return "workspace too small";
    case FV_ECUDA: return "CUDA runtime error";
    case FV_ETIMEOUT: return "device wait timed out";
    case FV_EUNSUPPORTED: return "unsupported request";
    case FV_EINFEASIBLE: return "no finite path";
  }
  return "unknown status";
}

// Exact decoding (vanilla / FLASH) of a batch with a CSR model runs the
// beam engine with every state kept (B = K): the beam then holds every
// finite state, so each step is the exact step of Sec. III-A (and FLASH-BS
// the exact FLASH).  Returns the parameters actually run.
fv_params exact_params(const fv_model* models, int32_t n_models, const fv_params* p) {
  fv_params q = *p;
  if (p->mode != FV_VANILLA && p->mode != FV_FLASH) return q;
  int32_t kmax = 0;
  bool csr = false;
  for (int m = 0; m < n_models; ++m) {
    kmax = std::max(kmax, models[m].K);
    csr = csr || models[m].trans == FV_TRANS_CSR;
  }
  if (!csr) return q;
  q.mode = FV_BEAM;
  q.B = kmax;
  q.P = p->mode == FV_FLASH ? p->P : 0;
  q.mem_budget_bytes = 0;
  return q;
}

size_t fv_workspace_size(const fv_model* models, int32_t n_models, const fv_batch* batch,
                         const fv_params* p_in) {
  if (!p_in || !batch || !batch->T_host) return 0;
  if (check_common(models, n_models, batch) != FV_OK) return 0;
  if (p_in->mode == FV_FLASH && p_in->P < 1) return 0;
  const fv_params pq = exact_params(models, n_models, p_in);
  const fv_params* p = &pq;
  if (p->mode == FV_FLASH || (p->mode == FV_BEAM && p->P >= 1)) {
    if (p->P < 1 || (p->mode == FV_BEAM && p->B < 1)) return 0;
    const FlashPlan fp = plan_flash(models, n_models, batch, p->P, p->mode == FV_FLASH ? p->mem_budget_bytes : 0,
                                    (p->flags & FV_NO_SORT) != 0);
    return layout_for(models, n_models, batch, p->mode, &fp, p->B).total;
  }
  if (p->mode == FV_BEAM && p->B < 1) return 0;
  if (p->mode != FV_VANILLA && p->mode != FV_BEAM && p->mode != FV_CHECKPOINT) return 0;
  return layout_for(models, n_models, batch, p->mode, nullptr, p->B, p->P).total;
}

fv_status fv_decode(const fv_model* models, int32_t n_models, const fv_batch* batch, const fv_params* p_in,
                    void* workspace, size_t ws_bytes, int32_t* paths_out, float* scores_out,
                    fv_stream_t stream_) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  if (!p_in) return FV_EINVAL;
  fv_status s = check_common(models, n_models, batch);
  if (s != FV_OK) return s;
  if (p_in->mode == FV_FLASH && p_in->P < 1) return FV_EINVAL;
  const fv_params pq = exact_params(models, n_models, p_in);
  const fv_params* p = &pq;
  if (!workspace || ws_bytes < 4096 || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1))) return FV_EINVAL;
  if (batch->n_seq > 0 && (!paths_out || !scores_out)) return FV_EINVAL;
  if (p->mode != FV_VANILLA && p->mode != FV_FLASH && p->mode != FV_BEAM && p->mode != FV_CHECKPOINT)
    return FV_EINVAL;
  if (p->mode == FV_FLASH && p->P < 1) return FV_EINVAL;
  if (p->mode == FV_BEAM && (p->B < 1 || p->P < 0)) return FV_EINVAL;
  if (p->mode != FV_VANILLA && !batch->T_host) return FV_EINVAL;  // task levels are planned from host lengths
  if (p->mode != FV_BEAM)
    for (int m = 0; m < n_models; ++m)
      if (models[m].trans != FV_TRANS_DENSE || !dense_supported_K(models[m].K)) return FV_EUNSUPPORTED;

  const int32_t n = batch->n_seq;
  const bool tasks = p->mode == FV_FLASH || (p->mode == FV_BEAM && p->P >= 1);
  FlashPlan fp;
  if (tasks)
    fp = plan_flash(models, n_models, batch, p->P, p->mode == FV_FLASH ? p->mem_budget_bytes : 0,
                    (p->flags & FV_NO_SORT) != 0);
  const Layout L = layout_for(models, n_models, batch, p->mode, tasks ? &fp : nullptr, p->B, p->P);
  if (batch->T_host && ws_bytes < L.total) return FV_ENOMEM;
  if (ws_bytes < L.aux) return FV_ENOMEM;
  const uint64_t cap = (ws_bytes - L.aux) / (p->mode == FV_VANILLA ? 2 : 4);
  if (n == 0) return FV_OK;

  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.hdr);
  Job* jobs = reinterpret_cast<Job*>(ws + L.jobs);
  int32_t* order = reinterpret_cast<int32_t*>(ws + L.order);
  int32_t* qlast = reinterpret_cast<int32_t*>(ws + L.qlast);
  const Ranges R = model_ranges(batch, n_models);

  PrepArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.T = batch->T;
  pa.model_idx = batch->model_idx;
  pa.e_off = batch->e_off;
  pa.path_off = batch->path_off;
  pa.n_seq = n;
  pa.n_models = n_models;
  for (int m = 0; m < n_models; ++m) pa.mk.K[m] = models[m].K;
  pa.aux_kind = p->mode == FV_VANILLA      ? 1
                : p->mode == FV_CHECKPOINT ? 4
                : (p->mode == FV_BEAM && !tasks) ? 3
                                                 : 2;
  pa.aux_mult = p->mode == FV_CHECKPOINT ? p->P : L.Wcap;
  pa.jobs = jobs;
  pa.hdr = hdr;
  pa.aux_cap = p->mode == FV_VANILLA ? cap : L.aux_elems;
  if (launch_prep(pa, st) != cudaSuccess) return FV_ECUDA;
  if (p->flags & FV_CHECKED)
    for (int m = 0; m < n_models; ++m)
      if (launch_check_inputs(models[m], m, jobs, n, batch->E, batch->obs, hdr, st) != cudaSuccess) return FV_ECUDA;
  if (launch_order(jobs, n, (p->flags & FV_NO_SORT) ? 1 : 0, order, st) != cudaSuccess) return FV_ECUDA;

  if (p->mode == FV_BEAM) return decode_beam(models, n_models, batch, p, ws, L, fp, R, paths_out, scores_out, st);

  for (int m = 0; m < n_models; ++m) {
    if (!R.count[m]) continue;
    const fv_model& md = models[m];
    DenseArgs da;
    memset(&da, 0, sizeof(da));
    da.K = md.K;
    da.logA = md.logA;
    da.log_pi = md.log_pi;
    da.emit = md.emit;
    da.V = md.V;
    da.logB = md.logB;
    da.E = batch->E;
    da.obs = batch->obs;
    da.jobs = jobs;
    da.order = order;
    da.order_begin = R.begin[m];
    da.order_count = R.count[m];
    da.max_jobs = R.count[m];
    da.pop = &hdr->pop[m];
    da.qlast = qlast;
    da.scores = scores_out;
    da.paths = paths_out;
    da.P = p->P;
    da.complete = (p->flags & FV_COMPLETE_PRUNING) ? 1 : 0;
    da.wide_withhold = (p->flags & FV_TEST_WITHHOLD_STEP) ? 1 : 0;
    da.no_tune = (p->flags & FV_NO_TUNE) ? 1 : 0;
    da.hdr = hdr;
    {
      int kpm = 0, cols = 0;
      dense_stream_geometry(md.K, &kpm, &cols);
      if (L.snapx) da.snap_scratch = reinterpret_cast<float*>(ws + L.snapx);
      if (kpm) {
        da.Ap = reinterpret_cast<const float2*>(ws + L.ap);
        da.ap_stride = cols;
        da.snap_scratch = reinterpret_cast<float*>(ws + L.snapx);
        if (launch_ap_prep(md.logA, md.K, reinterpret_cast<float2*>(ws + L.ap), st) != cudaSuccess) return FV_ECUDA;
        if (md.K <= 1024) {
          float* at = reinterpret_cast<float*>(ws + L.at);
          da.wide_AT = at;
          if (launch_wide_transpose(md.logA, md.K, at, st) != cudaSuccess) return FV_ECUDA;
        }
      }
      if (md.K > 1024) {
        // whole-GPU engine scratch: the same carving as wide_scratch_bytes
        const size_t lanes_k = (size_t)kWideLanes * wide_lane_stride(md.K);
        char* w = ws + L.wide;
        da.wide_D = reinterpret_cast<float*>(w);
        w += align_up(2 * sizeof(float) * lanes_k);
        da.wide_M = reinterpret_cast<uint16_t*>(w);
        w += align_up(2 * sizeof(uint16_t) * lanes_k);
        da.wide_X = reinterpret_cast<float*>(w);
        w += align_up(2 * sizeof(float) * lanes_k);
        da.wide_flags = reinterpret_cast<uint32_t*>(w);
        w += align_up(sizeof(uint32_t) * 8 * (size_t)(device_sm_count() + 1));
        float* at = reinterpret_cast<float*>(w);
        da.wide_AT = at;
        if (launch_wide_transpose(md.logA, md.K, at, st) != cudaSuccess) return FV_ECUDA;
      }
    }
    if (p->mode == FV_CHECKPOINT) {
      // Checkpoint Viterbi: forward pass keeping the checkpoints, last
      // state and score, then one level of segments per checkpoint,
      // latest segment first
      float* area = reinterpret_cast<float*>(ws + L.aux);
      Task* list = reinterpret_cast<Task*>(ws + L.listA);
      int32_t* count = reinterpret_cast<int32_t*>(ws + L.counts);
      int32_t levels = 0;
      for (int i = 0; i < n; ++i)
        if ((batch->model_host ? batch->model_host[i] : 0) == m)
          levels = std::max(levels, ckpt_count(batch->T_host[i], p->P));
      da.ckpt = 1;
      da.snaps = area;
      da.psi = reinterpret_cast<uint16_t*>(area);
      da.kind = kJobRoot;
      timed_begin(st);
      if (m > 0 && launch_reset(da.pop, st) != cudaSuccess) return FV_ECUDA;
      if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
      if (launch_ckpt_resolve(jobs, order, R.begin[m], R.count[m], md.K, p->P, area, paths_out, scores_out, hdr,
                              st) != cudaSuccess)
        return FV_ECUDA;
      for (int lvl = 0; lvl < levels; ++lvl) {
        if (launch_ckpt_tasks(jobs, order, R.begin[m], R.count[m], p->P, lvl, list, count, st) != cudaSuccess)
          return FV_ECUDA;
        if (launch_reset(da.pop, st) != cudaSuccess) return FV_ECUDA;
        da.kind = kJobLeaf;
        da.tasks = list;
        da.task_count = count;
        da.task_first = nullptr;
        da.max_jobs = R.count[m];
        if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
        if (launch_ckpt_backtrack(list, count, R.count[m], jobs, md.K, p->P, reinterpret_cast<uint16_t*>(area),
                                  paths_out, hdr, st) != cudaSuccess)
          return FV_ECUDA;
      }
      timed_end(st);
      continue;
    }
    if (p->mode == FV_VANILLA) {
      uint16_t* psi = reinterpret_cast<uint16_t*>(ws + L.aux);
      da.kind = kJobVanilla;
      da.psi = psi;
      timed_begin(st);
      if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
      timed_end(st);
      if (launch_backtrack(jobs, order, R.begin[m], R.count[m], md.K, psi, qlast, paths_out, hdr, st) != cudaSuccess)
        return FV_ECUDA;
      continue;
    }
    // ---- FLASH: root pass, resolve, then the task levels of Alg. 1
    float* sval = reinterpret_cast<float*>(ws + L.aux);
    uint16_t* maps = reinterpret_cast<uint16_t*>(ws + L.maps);
    float* snaps = reinterpret_cast<float*>(ws + L.snaps);
    Task* lists[2] = {reinterpret_cast<Task*>(ws + L.listA), reinterpret_cast<Task*>(ws + L.listB)};
    int32_t* counts = reinterpret_cast<int32_t*>(ws + L.counts);
    ScanTmp tmp;
    tmp.pos = reinterpret_cast<int32_t*>(ws + L.pos);
    tmp.bsum = reinterpret_cast<int32_t*>(ws + L.bsum);
    da.sval = sval;
    da.maps = maps;
    da.snaps = snaps;
    da.map_stride = L.map_stride;
    da.snap_stride = L.snap_stride;
    da.kind = kJobRoot;
    timed_begin(st);
    if (m > 0 && launch_reset(da.pop, st) != cudaSuccess) return FV_ECUDA;
    if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
    if (launch_flash_resolve(jobs, order, R.begin[m], R.count[m], md.K, p->P, maps, snaps, L.map_stride,
                             L.snap_stride, paths_out, sval, scores_out, hdr, st) != cudaSuccess)
      return FV_ECUDA;
    if (fp.levels[m] > 0 &&
        launch_level1_tasks(jobs, order, R.begin[m], R.count[m], p->P, lists[0], &counts[0], tmp, st) != cudaSuccess)
      return FV_ECUDA;
    // timing pairs: the root pass (with its resolve), then one per task
    // level, the budget-leaf waves together
    timed_end(st);
    int c = 0;
    for (int lvl = 0; lvl < fp.levels[m]; ++lvl) {
      timed_begin(st);
      if (lvl == fp.leaf_level[m]) {
        // budget leaves: every task of this level keeps its own
        // backpointer rows; waves of tasks whose rows fit the budget
        int32_t* wave_first = reinterpret_cast<int32_t*>(ws + L.waves);
        int32_t* wave_count = wave_first + fp.waves_max;
        uint16_t* leaf = reinterpret_cast<uint16_t*>(ws + L.leaf);
        if (launch_leaf_plan(lists[c], &counts[c], fp.leaf_rows[m], fp.leaf_cap[m], wave_first, wave_count,
                             fp.leaf_waves[m], hdr, st) != cudaSuccess)
          return FV_ECUDA;
        for (int w = 0; w < fp.leaf_waves[m]; ++w) {
          if (launch_reset(da.pop, st) != cudaSuccess) return FV_ECUDA;
          da.kind = kJobLeaf;
          da.tasks = lists[c];
          da.task_first = &wave_first[w];
          da.task_count = &wave_count[w];
          da.psi = leaf;
          da.max_jobs = (int32_t)fp.leaf_tasks[m];
          if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
          if (launch_leaf_backtrack(lists[c], &wave_first[w], &wave_count[w], (int32_t)fp.leaf_tasks[m], jobs, md.K,
                                    leaf, paths_out, hdr, st) != cudaSuccess)
            return FV_ECUDA;
        }
        da.task_first = nullptr;
        timed_end(st);
        break;
      }
      if (launch_reset(da.pop, st) != cudaSuccess) return FV_ECUDA;
      da.kind = kJobSub;
      da.tasks = lists[c];
      da.task_count = &counts[c];
      da.max_jobs = (int32_t)fp.max_tasks[m];
      if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
      if (lvl + 1 < fp.levels[m] &&
          launch_child_tasks(lists[c], &counts[c], (int32_t)fp.max_tasks[m], lists[c ^ 1], &counts[c ^ 1], tmp,
                             nullptr, st) != cudaSuccess)
        return FV_ECUDA;
      c ^= 1;
      timed_end(st);
    }
  }
  return FV_OK;
}

fv_status fv_path_score(const fv_model* models, int32_t n_models, const fv_batch* batch, const int32_t* paths,
                        float* scores_out, fv_stream_t stream_) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  fv_status s = check_common(models, n_models, batch);
  if (s != FV_OK) return s;
  if (batch->n_seq > 0 && (!paths || !scores_out)) return FV_EINVAL;
  for (int m = 0; m < n_models; ++m) {
    const fv_model& md = models[m];
    ScoreArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.K = md.K;
    sa.trans = md.trans;
    sa.emit = md.emit;
    sa.V = md.V;
    sa.log_pi = md.log_pi;
    sa.logA = md.logA;
    sa.row_ptr = md.row_ptr;
    sa.col = md.col;
    sa.val = md.val;
    sa.logB = md.logB;
    sa.E = batch->E;
    sa.obs = batch->obs;
    if (launch_path_score_direct(sa, m, batch->n_seq, batch->T, batch->model_idx, batch->e_off, batch->path_off,
                                 paths, scores_out, st) != cudaSuccess)
      return FV_ECUDA;
  }
  return FV_OK;
}

size_t fv_backward_workspace_size(const fv_model* models, int32_t n_models, const fv_batch* batch) {
  if (check_common(models, n_models, batch) != FV_OK) return 0;
  const size_t need = align_up(sizeof(WsHeader)) + align_up(sizeof(Job) * (size_t)batch->n_seq);
  return need < 4096 ? 4096 : need;
}

fv_status fv_backward(const fv_model* models, int32_t n_models, const fv_batch* batch, const int32_t* paths,
                      const float* grad_scores, float* dlog_pi, float* dlogA, float* dE, void* workspace,
                      size_t ws_bytes, fv_stream_t stream_) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  fv_status s = check_common(models, n_models, batch);
  if (s != FV_OK) return s;
  if (n_models != 1 || models[0].trans != FV_TRANS_DENSE || models[0].emit != FV_EMIT_DENSE)
    return FV_EUNSUPPORTED;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1))) return FV_EINVAL;
  if (batch->n_seq > 0 && (!paths || !grad_scores || !dlog_pi || !dlogA || !dE)) return FV_EINVAL;
  if (ws_bytes < fv_backward_workspace_size(models, n_models, batch)) return FV_ENOMEM;
  if (!batch->T_host) return FV_EINVAL;  // grid sizing uses the longest sequence
  const int32_t n = batch->n_seq, K = models[0].K;
  if (n == 0) return FV_OK;
  int32_t max_T = 1;
  for (int i = 0; i < n; ++i) max_T = std::max(max_T, batch->T_host[i]);
  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
  Job* jobs = reinterpret_cast<Job*>(ws + align_up(sizeof(WsHeader)));
  PrepArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.T = batch->T;
  pa.model_idx = batch->model_idx;
  pa.e_off = batch->e_off;
  pa.path_off = batch->path_off;
  pa.n_seq = n;
  pa.n_models = 1;
  pa.mk.K[0] = K;
  pa.aux_kind = 0;
  pa.jobs = jobs;
  pa.hdr = hdr;
  pa.aux_cap = 0;
  if (launch_prep(pa, st) != cudaSuccess) return FV_ECUDA;
  if (launch_backward(jobs, n, K, paths, grad_scores, dlog_pi, dlogA, dE, max_T, hdr, st) != cudaSuccess)
    return FV_ECUDA;
  return FV_OK;
}

int32_t fv_set_engine_variant(int32_t K, int32_t variant) {
  if (K < 1) return 0;
  dense_set_variant(K, variant);
  return dense_variants(K);
}

fv_status fv_autotune(const fv_model* models, int32_t n_models, const fv_batch* batch, const fv_params* p,
                      void* workspace, size_t ws_bytes, int32_t* paths_out, float* scores_out, fv_stream_t stream,
                      int32_t* chosen) {
  if (!p || !models || n_models < 1) return FV_EINVAL;
  fv_status s = check_common(models, n_models, batch);
  if (s != FV_OK) return s;
  const fv_params q = exact_params(models, n_models, p);
  std::vector<int32_t> reps;  // one K per tunable class present
  if (q.mode != FV_BEAM) {
    for (int m = 0; m < n_models; ++m) {
      const int K = models[m].K;
      if (dense_variants(K) < 2) continue;
      bool seen = false;
      for (int32_t r : reps) seen = seen || dense_k_class(r) == dense_k_class(K);
      if (!seen) reps.push_back(K);
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  fv_params run = *p;
  run.flags &= ~FV_NO_TUNE;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!reps.empty() && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) return FV_ECUDA;
  for (int32_t K : reps) {
    float best = 0.f;
    int bv = 0;
    for (int v = 0; v < dense_variants(K); ++v) {
      dense_set_variant(K, v);
      s = fv_decode(models, n_models, batch, &run, workspace, ws_bytes, paths_out, scores_out, stream);
      if (s != FV_OK) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && s == FV_OK; ++r)
        s = fv_decode(models, n_models, batch, &run, workspace, ws_bytes, paths_out, scores_out, stream);
      cudaEventRecord(e1, st);
      if (s != FV_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { s = FV_ECUDA; break; }
      s = fv_last_device_status(workspace, stream);
      if (s != FV_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (v == 0 || ms < best) { best = ms; bv = v; }
    }
    dense_set_variant(K, s == FV_OK ? bv : 0);
    if (s != FV_OK) break;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (chosen)
    for (int m = 0; m < n_models; ++m) chosen[m] = q.mode == FV_BEAM ? 0 : dense_get_variant(models[m].K);
  return s;
}

fv_status fv_timing_enable(int32_t on) {
  if (on && !g_ev_made) {
    for (int i = 0; i < 2 * kMaxTimed; ++i)
      if (cudaEventCreate(&g_ev[i]) != cudaSuccess) return FV_ECUDA;
    g_ev_made = true;
  }
  g_timing = on != 0;
  g_timed = 0;
  return FV_OK;
}

fv_status fv_timing_reset(void) {
  g_timed = 0;
  return FV_OK;
}

fv_status fv_timing_pairs(float* ms, int32_t max_pairs, int32_t* n_pairs) {
  if (!ms || !n_pairs || max_pairs < 0) return FV_EINVAL;
  const int n = g_timed < max_pairs ? g_timed : max_pairs;
  for (int i = 0; i < n; ++i) {
    if (cudaEventSynchronize(g_ev[2 * i + 1]) != cudaSuccess) return FV_ECUDA;
    if (cudaEventElapsedTime(&ms[i], g_ev[2 * i], g_ev[2 * i + 1]) != cudaSuccess) return FV_ECUDA;
  }
  *n_pairs = n;
  return FV_OK;
}

fv_status fv_timing_read(float* total_ms, int32_t* n_pairs) {
  if (!total_ms || !n_pairs) return FV_EINVAL;
  float tot = 0.f;
  for (int i = 0; i < g_timed; ++i) {
    if (cudaEventSynchronize(g_ev[2 * i + 1]) != cudaSuccess) return FV_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_ev[2 * i], g_ev[2 * i + 1]) != cudaSuccess) return FV_ECUDA;
    tot += ms;
  }
  *total_ms = tot;
  *n_pairs = g_timed;
  return FV_OK;
}

fv_status fv_last_device_status(const void* workspace, fv_stream_t stream_) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  if (!workspace) return FV_EINVAL;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FV_ECUDA;
  uint32_t v = 0;
  if (cudaMemcpy(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return FV_ECUDA;
  return static_cast<fv_status>(v);
}

}  // extern "C"
