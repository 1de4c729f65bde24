/*
 * fv.h -- C ABI of libfv, a GB300 (sm_103a) implementation of the decoding
 * hot path of FLASH Viterbi (Deng et al., arXiv 2510.19301).
 *
 * Operations (paper references are to that article):
 *   - exact Viterbi decoding, Sec. III-A: delta_t(j) = max_i[delta_{t-1}(i)
 *     A_ij] B_j(x_t) with argmax backpointers psi_t(j), evaluated in the log
 *     domain (Sec. III-A, last paragraph);
 *   - FLASH Viterbi, Sec. V-A/V-B: Alg. 1 (non-recursive divide and conquer
 *     with the P-way first split of Sec. V-A.3) running Alg. 2 (subtask
 *     decoding with MidState) under the pruned initialisation of Sec. V-B.2;
 *   - dynamic beam search and FLASH-BS, Sec. V-C;
 *   - a path-count backward (not in the paper).
 *
 * Numerics: every score is IEEE binary32, round-to-nearest-even, in this
 * order: delta_0[j] = logpi[j] + E_0[j];
 *   delta_t[j] = (max_i (delta_{t-1}[i] + logA[i][j])) + E_t[j],
 * every argmax takes the LOWEST index, and the value kept is the winning
 * candidate itself.  FLASH uses the retained offset of Def. 3,
 *   delta_m[j] = ((delta_{m-1}[q_{m-1}] + logA[q_{m-1}][j]) + E_m[j]),
 * so its paths and scores are bit-identical to the exact decoder.
 *
 * Memory: all array pointers are DEVICE pointers owned by the caller unless
 * the field name ends in _host.  The library never allocates device memory:
 * every scratch byte lives in the caller's workspace (size from
 * fv_workspace_size).  No pointer is retained after a call returns.  Work is
 * enqueued on the given stream; calls return before the GPU finishes.
 *
 * Errors: argument errors are returned at once and nothing is enqueued.
 * Errors found on the device (bad lengths or model indices, a workspace too
 * small for the lengths actually present, a wait that ran out, an
 * infeasible beam) are recorded in a status word inside the workspace; read
 * it with fv_last_device_status after the stream is synchronised.  Nothing
 * traps, aborts or prints.
 */
#ifndef FV_H
#define FV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fv_stream_t; /* same handle as cudaStream_t */

typedef enum {
  FV_OK = 0,
  FV_EINVAL = 1,        /* bad argument                                   */
  FV_ENOMEM = 2,        /* workspace too small                             */
  FV_ECUDA = 3,         /* a CUDA runtime call failed                      */
  FV_ETIMEOUT = 4,      /* a bounded device wait ran out                   */
  FV_EUNSUPPORTED = 5,  /* valid request the library does not implement    */
  FV_EINFEASIBLE = 6    /* no finite path (beam emptied / unreachable q_n) */
} fv_status;

typedef enum {
  FV_VANILLA = 0,   /* full T x K uint16 backpointer table + backtrack (Sec. III-A) */
  FV_FLASH = 1,     /* non-recursive D&C with MidState (Alg. 1, Alg. 2)            */
  FV_BEAM = 2,      /* dynamic beam (Sec. V-C); P >= 1 makes it FLASH-BS          */
  FV_CHECKPOINT = 3 /* Checkpoint Viterbi, the baseline of Sec. II-A (see below)  */
} fv_mode;

typedef enum { FV_TRANS_DENSE = 0, FV_TRANS_CSR = 1 } fv_trans_kind;
typedef enum { FV_EMIT_DENSE = 0, FV_EMIT_DISCRETE = 1 } fv_emit_kind;

/* fv_params.flags */
#define FV_COMPLETE_PRUNING 0x1u /* offset-0 re-initialisation of Sec. V-B.2     */
#define FV_NO_SORT 0x2u          /* keep batch order (skip longest-first order)  */
/* Check the inputs on the device before decoding: NaN or +inf in logpi,
 * logA / CSR weights, logB or the batch's emission scores, or a malformed
 * CSR graph (row_ptr not non-decreasing from 0 to nnz, a column outside
 * [0, K)), records FV_EINVAL in the status word and nothing is decoded.
 * Without this flag such inputs are undefined (-inf is always allowed). */
#define FV_CHECKED 0x4u
/* Run the default engine configuration instead of the one chosen by
 * fv_autotune / fv_set_engine_variant. */
#define FV_NO_TUNE 0x8u
/* FV_BEAM: run the static beam the paper contrasts with its dynamic one
 * (Sec. II-B; Sec. V-C.1), as in SIEVE-BS: every step first writes the
 * score of all K states (-inf where no beam state leads) to the workspace,
 * then keeps the top B of those K entries.  Same beams, paths and scores as
 * the dynamic beam (the top-B rule is the same); only the work per step and
 * the per-step candidate storage differ (K entries instead of the states
 * the beam reaches).  A comparator for benchmarks. */
#define FV_STATIC_BEAM 0x10u
/* The call shares the GPU with other decodes running at the same time (a
 * serving loop): take the kernel configuration with the least SM time per
 * step rather than the one that finishes this call soonest on an idle GPU.
 * Today this keeps dense beams (P = 0) on one CTA per sequence, which takes
 * about a third of the SM time per step of one 8-CTA cluster per sequence.
 * Results are the same either way. */
#define FV_SHARED_GPU 0x20u
/* Test hook for failure detection: the first CTA of the whole-GPU engine
 * (dense K > 1024) never publishes its step count, and CTA 1 of every 4- or
 * 8-CTA cluster of the streamed engine (256 < K <= 1024) withholds its
 * arrivals on the delta exchange of the second tick, so the bounded waits on
 * them run out (about one second each); the call then reports FV_ETIMEOUT in
 * the status word and the CUDA context stays usable.  No other effect. */
#define FV_TEST_WITHHOLD_STEP 0x80000000u

/* One HMM, lambda = (pi, A, B) of Sec. III. K <= 65536 (backpointers are
 * uint16).  Dense transitions: logA[i*K + j] = log A_ij, row = source state.
 * CSR transitions: out-edges of state i are col[row_ptr[i] .. row_ptr[i+1]),
 * with log-weights val[...]; a missing edge is log 0 = -inf.  Dense
 * emissions: the batch supplies E_t[j] = log B_j(x_t) directly.  Discrete
 * emissions: logB[j*V + v] = log B_{j,v} and the batch supplies symbols. */
typedef struct {
  int32_t K;
  const float* log_pi;     /* [K]                                   */
  int32_t trans;           /* fv_trans_kind                         */
  const float* logA;       /* dense [K*K]                           */
  const int32_t* row_ptr;  /* CSR [K+1]                             */
  const int32_t* col;      /* CSR [nnz]                             */
  const float* val;        /* CSR [nnz]                             */
  int64_t nnz;
  int32_t emit;            /* fv_emit_kind                          */
  int32_t V;               /* discrete: number of symbols           */
  const float* logB;       /* discrete: [K*V]                       */
} fv_model;

/* A batch of sequences, each decoded under one model.  Sequence b has
 * T[b] >= 1 steps.  Dense emissions: its row t is E[e_off[b] + t*K ..
 * + K) (K of its model).  Discrete: its symbol t is obs[e_off[b] + t].
 * Its path goes to paths_out[path_off[b] .. + T[b]).  The _host arrays are
 * host copies used for planning; T_host is required by fv_workspace_size
 * and, when given to fv_decode, lets it check the workspace at once.
 * model_host (or model_idx) may be NULL: every sequence uses model 0. */
typedef struct {
  int32_t n_seq;
  const int32_t* T_host;      /* HOST [n_seq]                    */
  const int32_t* model_host;  /* HOST [n_seq] or NULL            */
  const int32_t* T;           /* [n_seq]                         */
  const int32_t* model_idx;   /* [n_seq] or NULL                 */
  const int64_t* e_off;       /* [n_seq] elements                */
  const float* E;             /* dense emission scores           */
  const int32_t* obs;         /* discrete symbols                */
  const int64_t* path_off;    /* [n_seq] elements of paths_out   */
} fv_batch;

/* mode and its knobs: P = parallelism degree of the first split (Sec.
 * V-A.3; P < 2 means the binary root of Alg. 2), B = beam width (Sec. V-C;
 * B >= K keeps every finite state).
 *
 * mem_budget_bytes (FV_FLASH only): bytes of per-segment backpointer
 * tables the decoder may hold at once.  The first task level of Alg. 1
 * whose every task (m, n) fits -- (n - m) rows of K uint16 -- is solved
 * directly instead of being split further: the pruned start of Sec. V-B.2,
 * the recursion of Sec. III-A keeping psi_{m+1..n}, and the backtrack from
 * the known q*_n.  Those tasks run in waves whose tables fit the budget;
 * results are unchanged.  0 = pure divide and conquer.  The workspace grows
 * by at most the budget plus a small wave table.
 *
 * FV_CHECKPOINT (Checkpoint Viterbi, the comparison baseline of Sec. II-A):
 * one forward pass keeps delta only at C checkpoints, C = ceil(sqrt(T))
 * when P < 1, else min(P, T); checkpoint k is delta at e_k = floor(((k+1)T
 * - 1)/C).  Then the segments between checkpoints are decoded again from
 * the stored delta, latest first, each with its own backpointer rows, and
 * backtracked from the state already known at the segment's end.  Paths
 * and scores equal FV_VANILLA's bit for bit; per sequence the decoder
 * holds C rows of K floats and one segment of at most ceil(T/C) rows of K
 * uint16 (O(K sqrt T) instead of O(K T)), and decoding costs about two
 * forward passes plus one engine launch per checkpoint level.  Dense
 * transitions only (FV_EUNSUPPORTED for CSR), K <= 4096.
 *
 * Supported: FV_VANILLA and FV_FLASH on dense transitions need
 * K <= 4096 (FV_EUNSUPPORTED otherwise); K > 1024 runs one cooperative
 * launch over the whole GPU whose device waits are bounded (FV_ETIMEOUT in
 * the status word if one runs out).  FV_BEAM takes dense or CSR
 * transitions with K <= 65536.  A batch with a CSR model is decoded
 * exactly by the beam of Sec. V-C with every state kept (B = K; FLASH
 * becomes FLASH-BS with the same P), which gives the same paths and scores
 * as the exact recursion; mem_budget_bytes does not apply there, and a
 * sequence with no finite path is reported as FV_EINFEASIBLE. */
typedef struct {
  int32_t mode;               /* fv_mode                         */
  int32_t P;
  int32_t B;
  uint64_t mem_budget_bytes;
  uint32_t flags;
} fv_params;

/* Bytes of device workspace fv_decode needs for this request (>= 4096).
 * Returns 0 on invalid arguments. */
size_t fv_workspace_size(const fv_model* models, int32_t n_models,
                         const fv_batch* batch, const fv_params* params);

/* Decode every sequence of the batch.  Writes paths_out (int32 state ids)
 * and scores_out[b] (the path's log-likelihood, forward order).  The
 * workspace must be 256-byte aligned and at least fv_workspace_size bytes;
 * its contents on entry do not matter.  Asynchronous on `stream`. */
fv_status fv_decode(const fv_model* models, int32_t n_models, const fv_batch* batch,
                    const fv_params* params, void* workspace, size_t ws_bytes,
                    int32_t* paths_out, float* scores_out, fv_stream_t stream);

/* Gradient of L = sum_b grad_scores[b] * score_b with every path held
 * fixed (the Viterbi score is piecewise linear in the inputs):
 *   dlog_pi[j]    = sum_b g_b [q_{b,0} = j]
 *   dlogA[i*K+j]  = sum_b g_b #{t >= 1: q_{b,t-1} = i, q_{b,t} = j}
 *   dE[e_off[b] + t*K + j] = g_b [q_{b,t} = j]   (0 elsewhere)
 * Sums run over b in ascending order, each term the FP32 product g_b*count,
 * starting from +0, so the result is deterministic.  Dense transitions and
 * dense emissions only; one model (n_models == 1).  dE uses E's layout and
 * every element of it covered by the batch is written. */
fv_status fv_backward(const fv_model* models, int32_t n_models, const fv_batch* batch,
                      const int32_t* paths, const float* grad_scores,
                      float* dlog_pi, float* dlogA, float* dE,
                      void* workspace, size_t ws_bytes, fv_stream_t stream);

/* Bytes of workspace fv_backward needs. */
size_t fv_backward_workspace_size(const fv_model* models, int32_t n_models,
                                  const fv_batch* batch);

/* Status recorded on the device by the last call that used `workspace`
 * (synchronises `stream`). */
fv_status fv_last_device_status(const void* workspace, fv_stream_t stream);

/* Static description of a status code. */
const char* fv_status_str(fv_status s);

/* Recompute score_b = log-likelihood of paths (forward order of Sec.
 * III-A) for every sequence.  Dense or CSR transitions (a missing edge
 * gives -inf). */
fv_status fv_path_score(const fv_model* models, int32_t n_models, const fv_batch* batch,
                        const int32_t* paths, float* scores_out, fv_stream_t stream);

/* Optional timing of the main decode kernels, for roofline reports.  While
 * enabled, every fv_decode records CUDA event pairs (library-owned, at most
 * 256 pairs) around its main decode kernel launches on the call's stream.
 * fv_timing_read synchronises on the recorded pairs and returns the total
 * elapsed milliseconds and the number of pairs since the last reset. */
fv_status fv_timing_enable(int32_t on);
fv_status fv_timing_reset(void);
fv_status fv_timing_read(float* total_ms, int32_t* n_pairs);
/* The recorded pairs one by one (milliseconds each, in recording order, at
 * most max_pairs; *n_pairs = how many were written).  A FLASH decode records
 * one pair for its root pass (with the resolve) and one per task level of
 * Alg. 1 (the budget-leaf waves of the leaf level together); the other
 * modes one pair per decode.  Synchronises on the recorded pairs. */
fv_status fv_timing_pairs(float* ms, int32_t max_pairs, int32_t* n_pairs);

/* Autotuning of the exact forward engine (not in the paper).  Dense exact
 * decoding has, per class of K (<= 64, <= 128, <= 256, <= 512, <= 1024),
 * several engine configurations -- the one-CTA-per-job small-K engine
 * (K <= 128), cluster sizes, CTAs per SM, warps per CTA and columns per
 * lane -- that compute the same values in the same order and differ only
 * in speed.  fv_autotune
 * decodes the given request once per candidate of every class present
 * (one warm-up and two timed calls each, CUDA events on `stream`), keeps
 * the fastest per class for every later fv_decode in this process, and
 * writes the chosen variant of each model's class to chosen[m] (may be
 * NULL).  Same arguments and outputs as fv_decode; it synchronises the
 * stream, so it is not capturable.  Requests without tunable classes
 * return FV_OK at once with chosen[] = 0.  Device errors are returned. */
fv_status fv_autotune(const fv_model* models, int32_t n_models, const fv_batch* batch,
                      const fv_params* params, void* workspace, size_t ws_bytes,
                      int32_t* paths_out, float* scores_out, fv_stream_t stream,
                      int32_t* chosen);

/* Set the engine variant of K's class directly (0 = default); returns the
 * number of variants of that class.  For tuning studies and tests. */
int32_t fv_set_engine_variant(int32_t K, int32_t variant);

/* Bytes of the static device scratch behind fv_decode_noalloc. */
#define FV_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* Exact decoding (mode FV_VANILLA, dense transitions) without any device
 * allocation, for callers that may not allocate device memory at decode
 * time: code held to a memory budget fixed at start-up, plug-ins whose host
 * owns the device allocator, or latency-critical paths where an allocation
 * could block.  The paper has no counterpart to this entry point.
 *
 * Same inputs, outputs and results as fv_decode with mode FV_VANILLA, but
 * the scratch lives in a file-scope device array of
 * FV_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library holds
 * until the process exits.  batch->T_host is required; a request whose
 * workspace (fv_workspace_size for FV_VANILLA) exceeds that size is rejected
 * with FV_ENOMEM before anything is enqueued.  No cudaMalloc, cudaFree or
 * other allocating routine is called.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture.  Every call shares the one array, so calls that overlap
 * on the GPU (two streams, two threads) race and corrupt each other's
 * results: serialise them.  The address is cached per device ordinal, so
 * the entry point works in the device's primary context (the one the CUDA
 * runtime uses) and must not be called after cudaDeviceReset in the same
 * process.  Models with CSR transitions are refused with FV_EUNSUPPORTED.
 * Device-side errors (bad lengths on the device, a wait that ran out) are
 * recorded in the shared scratch like fv_decode's; read them with
 * fv_decode_noalloc_status. */
fv_status fv_decode_noalloc(const fv_model* models, int32_t n_models, const fv_batch* batch,
                            int32_t* paths_out, float* scores_out, fv_stream_t stream);

/* Status recorded on the device by the last fv_decode_noalloc call on the
 * current device (synchronises `stream`, then copies the status word out of
 * the static scratch; allocates nothing).  FV_OK before any call. */
fv_status fv_decode_noalloc_status(fv_stream_t stream);

/* Measured ceiling of the max-plus cell (not in the paper): runs the
 * exact decoder's inner instruction pair -- one packed add.rn.f32x2 of two
 * candidates delta[i] + logA[i][j] and one 3-input max.f32 into the running
 * maximum, the cell of the tropical product of Sec. III-A -- on every SM
 * (one CTA of 512 threads per SM; per thread and round, two source pairs
 * read from shared memory, as the engines read delta, against 16 weight
 * pairs in registers: 32 pairs, 64 cells, `iters` rounds), after one short
 * warm-up launch.  Two forms of the adds are timed (one packed
 * add.rn.f32x2, or two scalar add.rn.f32) and the faster is reported.
 * Writes cells per second (CUDA events on `stream`), cells per clock per SM
 * (clock64 of the first CTA; may be NULL) and the SM count (may be NULL).
 * Synchronises `stream`; not capturable.  Allocates no device memory. */
fv_status fv_maxplus_peak(int32_t iters, double* cells_per_s, double* cells_per_clk_sm,
                          int32_t* sm_count, fv_stream_t stream);

/* Library version string. */
const char* fv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FV_H */
