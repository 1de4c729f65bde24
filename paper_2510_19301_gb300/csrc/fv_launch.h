// fv_launch.h -- host-side launchers shared between libfv translation units.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
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
  int32_t aux_kind;  // 0: none, 1: T*K uint16 backpointers, 2: T floats, 3: T*aux_mult int32,
                     // 4: Checkpoint Viterbi area (ckpt_area with P = aux_mult)
  int32_t aux_mult;
  Job* jobs;
  WsHeader* hdr;
  uint64_t aux_cap;  // elements available in the aux area
};

// Job kinds run by the forward engine.
enum JobKind : int32_t {
  kJobVanilla = 0,  // whole sequence, psi table (Sec. III-A)
  kJobRoot = 1,     // whole sequence, P' division points (Sec. V-A.3, Alg. 2 MidState)
  kJobSub = 2,      // segment task (m, n) of Alg. 1 with the pruned start of Sec. V-B.2
  kJobBeam = 3,     // whole sequence, beam with per-step backpointers (Sec. V-C, P = 0)
  kJobLeaf = 4      // segment task (m, n) solved with its own backpointer rows psi_{m+1..n}
                    // (budget leaf); rows start at element task.pad * K of the leaf area
};

// One divide-and-conquer task (Alg. 1 tuple) of sequence b.  Checkpoint
// segments use the same tuple: (m, n) is the segment and pad the index of
// the checkpoint it restarts from (-1: it starts at t = 0 from pi).
struct Task {
  int32_t b, m, n, pad;
};

// FLASH's first split (Sec. V-A): P' = min(max(P, 2), T) parts.
__host__ __device__ inline int32_t flash_pe(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t p = P < 2 ? 2 : P;
  return p < T ? p : T;
}
// Division point e_k = floor(((k+1)T - 1) / P') of the P-way first split.
__host__ __device__ inline int32_t flash_div(int32_t k, int32_t T, int32_t Pe) {
  return (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
}

// Checkpoint Viterbi (the sqrt(T)-checkpoint baseline of Sec. II-A): the
// number C of checkpoints of a length-T sequence, ceil(sqrt(T)) unless P >= 1
// asks for P, at most T.  Checkpoint k is delta at the division point
// e_k = floor(((k+1)T - 1) / C) (e_{C-1} = T - 1); segment k covers steps
// e_{k-1}+1 .. e_k.
__host__ __device__ inline int32_t ckpt_count(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t c = P;
  if (c < 1) {
    c = (int32_t)sqrtf((float)T);
    while ((int64_t)c * c < T) ++c;
    while (c > 1 && (int64_t)(c - 1) * (c - 1) >= T) --c;
  }
  return c < T ? c : T;
}
// Backpointer rows of the longest segment (upper bound ceil(T / C)).
__host__ __device__ inline int32_t ckpt_rows(int32_t T, int32_t C) { return (T + C - 1) / C; }
// Per-sequence area of Checkpoint Viterbi, in 4-byte elements: C rows of
// K floats (the checkpoints), then ckpt_rows rows of K uint16 backpointers
// (one segment at a time), rounded to 16 bytes.
__host__ __device__ inline uint64_t ckpt_area(int32_t T, int32_t P, int32_t K) {
  const uint64_t C = (uint64_t)ckpt_count(T, P), R = (uint64_t)ckpt_rows(T, (int32_t)C);
  return (C * (uint64_t)K + (R * (uint64_t)K + 1ull) / 2ull + 3ull) & ~3ull;
}

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
  int32_t kind;               // JobKind
  const int32_t* order;       // vanilla/root: sequences in order[order_begin ..]
  int32_t order_begin;
  int32_t order_count;
  const Task* tasks;          // sub / leaf: task list and its device-side count
  const int32_t* task_count;
  const int32_t* task_first;  // sub / leaf: device-side index of the first task (null: 0)
  int32_t max_jobs;           // host upper bound of jobs (grid sizing)
  unsigned long long* pop;
  uint16_t* psi;              // vanilla: backpointer rows at job.aux_off; leaf: the leaf area
  int32_t* qlast;             // vanilla: final states
  float* scores;              // vanilla: scores
  int32_t* paths;             // flash: revealed states (paths_out)
  float* sval;                // flash: delta along the path, at job.aux_off
  uint16_t* maps;             // root: (P'-1) ancestor maps per sequence
  float* snaps;               // root: P' delta snapshots per sequence
  int64_t map_stride;         // elements per sequence
  int64_t snap_stride;
  int32_t P;
  int32_t complete;           // offset-0 (complete pruning) start for subtasks
  // Checkpoint Viterbi: kJobRoot keeps only delta at the checkpoints (no
  // MidState), in the sequence's area at job.aux_off of `snaps`; kJobLeaf
  // restarts segment tasks from those checkpoints and writes the segment's
  // backpointer rows after them (`psi` = the same area as uint16)
  int32_t ckpt;
  const float2* Ap;           // streamed configurations: row-pair copy of logA
  int64_t ap_stride;          // float2 per row pair of Ap
  float* snap_scratch;        // streamed configurations: sub snapshots [clusters][S][rows]
  // whole-GPU configuration (K > 1024): delta / MidState double buffers,
  // sub snapshots by job parity (each [2][lanes][K]) and per-CTA step flags
  float* wide_D;
  uint16_t* wide_M;
  float* wide_X;
  uint32_t* wide_flags;
  const float* wide_AT;       // column-major copy of logA, AT[j * wide_lane_stride(K) + i] = A[i][j]
                              // (streamed and whole-GPU configurations: the exact re-scan reads it)
  int32_t wide_withhold;      // test hook: CTA 0 of the whole-GPU engine never publishes its step count;
                              // CTA 1 of each 4- / 8-CTA cluster withholds its second-tick arrivals
  int32_t no_tune;            // use the default engine configuration, not the tuned one
  WsHeader* hdr;
};

// Geometry of the whole-GPU engine for one K (fv_wide.cu); it advances
// kWideLanes jobs in lockstep.
constexpr int kWideLanes = 8;
// Elements per lane in the engine's global delta / MidState / snapshot rows.
__host__ __device__ inline int wide_lane_stride(int K) { return (K + 31) / 32 * 32; }
struct WideGeom {
  int32_t CR, NCB, G, KR, RPC, RPW, RWR;  // cluster size, column blocks, CTAs, padded rows, rows per CTA / warp, resident rows per warp
  size_t smem;                            // dynamic shared memory per CTA
  float l2_keep;                          // fraction of streamed logA lines loaded with L2 evict_last priority
};

// Beam search and FLASH-BS (fv_beam.cu).
struct BeamArgs {
  int32_t K, trans, emit, V;
  const float* log_pi;
  const float* logA;
  const int32_t* row_ptr;
  const int32_t* col;
  const float* val;
  const float* logB;
  const float* E;
  const int32_t* obs;
  const Job* jobs;
  int32_t kind;               // kJobBeam, kJobRoot or kJobSub
  const int32_t* order;
  int32_t order_begin, order_count;
  const Task* tasks;
  const int32_t* task_count;
  unsigned long long* pop;
  int32_t B;                  // beam width requested
  int32_t Wcap;               // min(B, K): stride of stored beams
  int32_t Bcap;               // scratch beam capacity (K when a subtask may be re-run exactly)
  int32_t P;
  int32_t complete;
  int32_t max_ctas;
  char* scratch;              // per CTA slice of scratch_stride bytes
  size_t scratch_stride;
  int32_t* bp_id;             // beam: per sequence [T][Wcap] state ids at job.aux_off
  int32_t* bp_src;            //       and source slots
  int32_t* qlast;             // beam: slot of the best final entry
  float* scores;
  int32_t* paths;             // flash-bs: revealed states
  float* sval;                // flash-bs: beam score along the path, at job.aux_off
  int32_t* div_id;            // root: per sequence [pe_cap][Wcap] beams at the division points
  float* div_val;
  int32_t* div_mid;
  int32_t* div_n;             // root: per sequence [pe_cap] beam sizes
  int64_t div_stride;         // pe_cap * Wcap
  int32_t pe_cap;
  int32_t beam_smem;          // beams (both buffers + subtask snapshot) live in shared memory
  int32_t cand_smem;          // candidate values / sources live in shared memory
  int32_t list_cap;           // CSR with candidates in global memory: entries of the shared-memory
                              // list of a step's touched candidates (ordered key, state id); 0 = none
  // static beam (the SIEVE-BS style comparator of Sec. II-B / V-C.1): every
  // step writes the full K-entry score vector (-inf where no beam state
  // leads) to the workspace and selects the top B from all K entries
  int32_t static_beam;
  // lengths of the launch's sequences, from the host copy (0: not given);
  // used only to choose between one CTA and one cluster per sequence
  int64_t sum_T;
  int32_t max_T;
  int32_t per_cta;            // one CTA per sequence (FV_SHARED_GPU)
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
// Engine configuration variants of a K class and the tuned choice.
int dense_k_class(int K);
int dense_job_slots(int K);
int dense_variants(int K);
void dense_set_variant(int K, int v);
int dense_get_variant(int K);
int device_sm_count();
bool wide_geometry(int K, int nsm, WideGeom* g);
size_t wide_scratch_bytes(int K, int nsm);
cudaError_t launch_wide_forward(DenseArgs a, cudaStream_t st);
// small state spaces (K <= 128), every job kind: a CTA of K-class threads per
// job, a thread per state (fv_small.cu)
cudaError_t launch_small_forward(const DenseArgs& a, cudaStream_t st);
// AT[j * KD + i] = logA[i * K + j] (rows K..KD-1 are -inf), KD = wide_lane_stride(K).
cudaError_t launch_wide_transpose(const float* logA, int K, float* AT, cudaStream_t st);
void dense_stream_geometry(int K, int* KPM, int* cols);
cudaError_t launch_ap_prep(const float* logA, int K, float2* Ap, cudaStream_t st);
cudaError_t launch_prep(const PrepArgs& p, cudaStream_t st);
cudaError_t launch_order(const Job* jobs, int32_t n, int32_t nosort, int32_t* order, cudaStream_t st);
cudaError_t launch_dense_forward(DenseArgs a, int max_clusters, cudaStream_t st);
cudaError_t launch_backtrack(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t K,
                             const uint16_t* psi, const int32_t* qlast, int32_t* paths, const WsHeader* hdr,
                             cudaStream_t st);
cudaError_t launch_flash_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count,
                                 int32_t K, int32_t P, const uint16_t* maps, const float* snaps,
                                 int64_t map_stride, int64_t snap_stride, int32_t* paths, float* sval,
                                 float* scores, const WsHeader* hdr, cudaStream_t st);
// Level-1 tasks of Alg. 1 (the P' segments of every sequence) and the
// children of a task list, written in parent order through a device scan.
struct ScanTmp {
  int32_t* pos;     // [max_items]
  int32_t* bsum;    // [ceil(max_items / 256)]
};
cudaError_t launch_level1_tasks(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                                Task* out, int32_t* out_count, ScanTmp tmp, cudaStream_t st);
cudaError_t launch_child_tasks(const Task* in, const int32_t* in_count, int32_t max_in, Task* out,
                               int32_t* out_count, ScanTmp tmp, unsigned long long* pop_reset, cudaStream_t st);
cudaError_t launch_reset(unsigned long long* pop, cudaStream_t st);
// Checkpoint Viterbi (fv_flash.cu): q_{T-1} and the score from the last
// checkpoint; the segment list of one level; the segment backtrack.
cudaError_t launch_ckpt_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t K,
                                int32_t P, const float* area, int32_t* paths, float* scores, const WsHeader* hdr,
                                cudaStream_t st);
cudaError_t launch_ckpt_tasks(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                              int32_t level, Task* out, int32_t* out_count, cudaStream_t st);
cudaError_t launch_ckpt_backtrack(const Task* tasks, const int32_t* count, int32_t max_count, const Job* jobs,
                                  int32_t K, int32_t P, const uint16_t* area16, int32_t* paths, const WsHeader* hdr,
                                  cudaStream_t st);
// FV_CHECKED: scan one model's arrays, and the emission scores (dense) or
// symbols (discrete) of the sequences decoded with it, for values the
// decoder does not accept; records FV_EINVAL in the header.
cudaError_t launch_check_inputs(const fv_model& m, int32_t model, const Job* jobs, int32_t n_seq, const float* E,
                                const int32_t* obs, WsHeader* hdr, cudaStream_t st);
// Budget leaves: greedy packing of a task list into waves whose backpointer
// rows (n - m per task) fit budget_rows and that hold at most wave_cap tasks
// (0: no cap; the engine's concurrent job slots, so a wave runs in one
// round); writes each task's row offset into
// Task::pad and the waves' [first, count) into wave_first / wave_count
// (max_waves entries, unused ones empty).
cudaError_t launch_leaf_plan(Task* tasks, const int32_t* count, int64_t budget_rows, int32_t wave_cap,
                             int32_t* wave_first, int32_t* wave_count, int32_t max_waves, WsHeader* hdr,
                             cudaStream_t st);
// q_{t-1} = psi_t[q_t] from the known q_n down to t = m + 1 for every task of
// one wave (max_count bounds the wave's size).
cudaError_t launch_leaf_backtrack(const Task* tasks, const int32_t* wave_first, const int32_t* wave_count,
                                  int32_t max_count, const Job* jobs, int32_t K, const uint16_t* leaf_psi,
                                  int32_t* paths, const WsHeader* hdr, cudaStream_t st);
size_t beam_scratch_stride(int K, int Bcap);
int beam_max_ctas();
cudaError_t launch_beam(const BeamArgs& a, int max_jobs, cudaStream_t st);
cudaError_t launch_beam_backtrack(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t Wcap,
                                  const int32_t* bp_id, const int32_t* bp_src, const int32_t* qlast, int32_t* paths,
                                  const WsHeader* hdr, cudaStream_t st);
cudaError_t launch_beam_resolve(const Job* jobs, const int32_t* order, int32_t begin, int32_t count, int32_t P,
                                int32_t Wcap, int32_t pe_cap, int64_t div_stride, const int32_t* div_id,
                                const float* div_val, const int32_t* div_mid, const int32_t* div_n, int32_t* paths,
                                float* sval, WsHeader* hdr, cudaStream_t st);
cudaError_t launch_backward(const Job* jobs, int32_t n_seq, int32_t K, const int32_t* paths, const float* g,
                            float* dlog_pi, float* dlogA, float* dE, int32_t max_T, const WsHeader* hdr,
                            cudaStream_t st);
cudaError_t launch_path_score_direct(const ScoreArgs& a, int32_t model, int32_t n_seq, const int32_t* T,
                                     const int32_t* model_idx, const int64_t* e_off, const int64_t* path_off,
                                     const int32_t* paths, float* scores, cudaStream_t st);
cudaError_t launch_path_score(const ScoreArgs& a, const Job* jobs, const int32_t* order, int32_t begin,
                              int32_t count, const int32_t* paths, float* scores, const WsHeader* hdr,
                              cudaStream_t st);

}  // namespace fv
