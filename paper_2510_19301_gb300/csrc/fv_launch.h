// fv_launch.h -- host-side launchers shared between libfv translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fv_internal.cuh"

namespace fv {

struct PrepArgs {
  const int32_t* T;
  const int32_t* model_idx;
  const int64_t* e_off;
  const int64_t* path_off;
  int32_t n_seq;
  int32_t n_models;
  ModelK mk;
  int32_t aux_kind;  // 0: none, 1: T*K uint16 backpointers, 2: T floats
  Job* jobs;
  WsHeader* hdr;
  uint64_t aux_cap;  // elements available in the aux area
};

struct DenseArgs {
  int32_t K;
  int32_t KP;  // rows padded to a multiple of 4*NW (set by the launcher)
  const float* logA;
  const float* log_pi;
  int32_t emit;
  int32_t V;
  const float* logB;
  const float* E;
  const int32_t* obs;
  const Job* jobs;
  const int32_t* order;
  int32_t order_begin;
  int32_t order_count;
  unsigned long long* pop;
  uint16_t* psi;
  int32_t* qlast;
  float* scores;
  WsHeader* hdr;
};

struct ScoreArgs {
  int32_t K, trans, emit, V;
  const float* log_pi;
  const float* logA;
  const int32_t* row_ptr;
  const int32_t* col;
  const float* val;
  const float* logB;
  const float* E;
  const int32_t* obs;
};

int dense_supported_K(int K);
cudaError_t launch_prep(const PrepArgs& p, cudaStream_t st);
cudaError_t launch_order(const Job* jobs, int32_t n, int32_t nosort, int32_t* order, cudaStream_t st);
cudaError_t launch_dense_forward(DenseArgs a, int max_clusters, cudaStream_t st);
cudaError_t launch_backtrack(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t K,
                             const uint16_t* psi, const int32_t* qlast, int32_t* paths, const WsHeader* hdr,
                             cudaStream_t st);
cudaError_t launch_path_score(const ScoreArgs& a, const Job* jobs, const int32_t* order, int32_t begin,
                              int32_t count, const int32_t* paths, float* scores, cudaStream_t st);

}  // namespace fv
