// fv_api.cu -- the extern "C" boundary of libfv: argument checks, workspace
// layout, and the launch sequence for each mode.  No device memory is
// allocated here; every scratch byte is carved out of the caller's workspace.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "fv_internal.cuh"

#include "fv_launch.h"

using namespace fv;

namespace {

struct Layout {
  size_t hdr, jobs, order, qlast, aux, prefix;
};

Layout layout_for(int32_t n_seq) {
  Layout L;
  L.hdr = 0;
  L.jobs = align_up(sizeof(WsHeader));
  L.order = align_up(L.jobs + sizeof(Job) * (size_t)n_seq);
  L.qlast = align_up(L.order + sizeof(int32_t) * (size_t)n_seq);
  L.aux = align_up(L.qlast + sizeof(int32_t) * (size_t)n_seq);
  L.prefix = L.aux;
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

// Elements of the per-sequence aux area for a mode (must match prep_kernel).
uint64_t aux_need(const fv_model* models, const fv_batch* b, int mode) {
  uint64_t need = 0;
  for (int i = 0; i < b->n_seq; ++i) {
    const int m = b->model_host ? b->model_host[i] : 0;
    const uint64_t T = (uint64_t)b->T_host[i], K = (uint64_t)models[m].K;
    if (mode == FV_VANILLA) need += (T * K + 7ull) & ~7ull;
  }
  return need;
}

size_t aux_elem_bytes(int mode) { return mode == FV_VANILLA ? 2 : 4; }

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

size_t fv_workspace_size(const fv_model* models, int32_t n_models, const fv_batch* batch,
                         const fv_params* p) {
  if (!p || !batch || !batch->T_host) return 0;
  if (check_common(models, n_models, batch) != FV_OK) return 0;
  const Layout L = layout_for(batch->n_seq);
  size_t total = L.prefix + aux_need(models, batch, p->mode) * aux_elem_bytes(p->mode);
  total = align_up(total);
  return total < 4096 ? 4096 : total;
}

fv_status fv_decode(const fv_model* models, int32_t n_models, const fv_batch* batch, const fv_params* p,
                    void* workspace, size_t ws_bytes, int32_t* paths_out, float* scores_out,
                    fv_stream_t stream_) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream_);
  if (!p) return FV_EINVAL;
  fv_status s = check_common(models, n_models, batch);
  if (s != FV_OK) return s;
  if (!workspace || ws_bytes < 4096 || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1))) return FV_EINVAL;
  if (batch->n_seq > 0 && (!paths_out || !scores_out)) return FV_EINVAL;
  if (p->mode != FV_VANILLA && p->mode != FV_FLASH && p->mode != FV_BEAM) return FV_EINVAL;
  if (p->mode == FV_FLASH && p->P < 1) return FV_EINVAL;
  if (p->mode == FV_BEAM && (p->B < 1 || p->P < 0)) return FV_EINVAL;
  if (p->mode != FV_VANILLA) return FV_EUNSUPPORTED;
  for (int m = 0; m < n_models; ++m)
    if (models[m].trans != FV_TRANS_DENSE || !dense_supported_K(models[m].K)) return FV_EUNSUPPORTED;

  const int32_t n = batch->n_seq;
  const Layout L = layout_for(n);
  if (ws_bytes < L.prefix) return FV_ENOMEM;
  const uint64_t cap = (ws_bytes - L.prefix) / aux_elem_bytes(p->mode);
  if (batch->T_host && aux_need(models, batch, p->mode) > cap) return FV_ENOMEM;
  if (n == 0) return FV_OK;

  char* ws = static_cast<char*>(workspace);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(ws + L.hdr);
  Job* jobs = reinterpret_cast<Job*>(ws + L.jobs);
  int32_t* order = reinterpret_cast<int32_t*>(ws + L.order);
  int32_t* qlast = reinterpret_cast<int32_t*>(ws + L.qlast);
  uint16_t* psi = reinterpret_cast<uint16_t*>(ws + L.aux);

  // per-model sequence ranges of the (model-major) order
  std::vector<int32_t> count(n_models, 0), begin(n_models, 0);
  if (batch->model_host) {
    for (int i = 0; i < n; ++i) count[batch->model_host[i]]++;
  } else {
    count[0] = n;
  }
  for (int m = 1; m < n_models; ++m) begin[m] = begin[m - 1] + count[m - 1];

  PrepArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.T = batch->T;
  pa.model_idx = batch->model_idx;
  pa.e_off = batch->e_off;
  pa.path_off = batch->path_off;
  pa.n_seq = n;
  pa.n_models = n_models;
  for (int m = 0; m < n_models; ++m) pa.mk.K[m] = models[m].K;
  pa.aux_kind = 1;
  pa.jobs = jobs;
  pa.hdr = hdr;
  pa.aux_cap = cap;
  if (launch_prep(pa, st) != cudaSuccess) return FV_ECUDA;
  if (launch_order(jobs, n, (p->flags & FV_NO_SORT) ? 1 : 0, order, st) != cudaSuccess) return FV_ECUDA;

  for (int m = 0; m < n_models; ++m) {
    if (!count[m]) continue;
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
    da.order_begin = begin[m];
    da.order_count = count[m];
    da.pop = &hdr->pop[m];
    da.psi = psi;
    da.qlast = qlast;
    da.scores = scores_out;
    da.hdr = hdr;
    timed_begin(st);
    if (launch_dense_forward(da, 0, st) != cudaSuccess) return FV_ECUDA;
    timed_end(st);
    if (launch_backtrack(jobs, order, begin[m], count[m], md.K, psi, qlast, paths_out, hdr, st) != cudaSuccess)
      return FV_ECUDA;
  }
  return FV_OK;
}

fv_status fv_path_score(const fv_model* models, int32_t n_models, const fv_batch* batch, const int32_t* paths,
                        float* scores_out, fv_stream_t stream_) {
  (void)models; (void)n_models; (void)batch; (void)paths; (void)scores_out; (void)stream_;
  return FV_EUNSUPPORTED;
}

size_t fv_backward_workspace_size(const fv_model* models, int32_t n_models, const fv_batch* batch) {
  (void)models; (void)n_models; (void)batch;
  return 0;
}

fv_status fv_backward(const fv_model* models, int32_t n_models, const fv_batch* batch, const int32_t* paths,
                      const float* grad_scores, float* dlog_pi, float* dlogA, float* dE, void* workspace,
                      size_t ws_bytes, fv_stream_t stream_) {
  (void)models; (void)n_models; (void)batch; (void)paths; (void)grad_scores; (void)dlog_pi; (void)dlogA;
  (void)dE; (void)workspace; (void)ws_bytes; (void)stream_;
  return FV_EUNSUPPORTED;
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
