/*
 * fv_oracle.c -- plain, slow, single-threaded CPU oracle for FLASH Viterbi
 * (Deng et al., "FLASH Viterbi: Fast and Adaptive Viterbi Decoding for
 * Modern Data Systems", arXiv 2510.19301).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded by the test-suite, by the smoke check and by the CPU-baseline leg of
 * the benchmark.  The GPU library never links, loads or calls it, and it
 * shares no source with the GPU library.
 *
 * Arithmetic: IEEE-754 binary32, round-to-nearest-even, no contraction
 * (compiled with -O2 -ffp-contract=off -fno-fast-math).  The paper does not
 * fix a float width; the GPU path computes in FP32 and must match this file to
 * 0 ulp, so this file computes in FP32 in the fixed order stated below.
 *
 * Readings of points the paper leaves open:
 *  R1  Emission scores are added outside the max:
 *        delta_t[j] = fl( max_i fl(delta_{t-1}[i] + logA[i][j]) + E_t[j] ).
 *  R2  Every argmax takes the lowest index; the value kept is the winning
 *      candidate itself (so +0/-0 ties keep the lower index's sign).
 *  R3  P-way root split points e_k = floor(((k+1)T-1)/P'),
 *      P' = min(max(P,2),T) (P=1 runs the binary root of Alg. 2).
 *  R4  Pruned re-initialisation keeps the retained offset s_{m-1}
 *      (Def. 3): delta_m[j] = fl(fl(s_{m-1} + logA[q_{m-1}][j]) + E_m[j]).
 *      The complete-pruning form of Sec. V-B.2 (offset 0) is a flag.
 *  R5  Alg. 1 terminates when every task has been processed; each task
 *      reveals one new state so there are T-P' tasks after the root.
 *  R6  Beams are the top-B finite candidates under (score desc, id asc).
 *  R7  FLASH-BS subtasks evaluate target q_n in their last step directly;
 *      if it is unreachable the subtask is re-run with the full state set.
 *  R8  MidState updates read the previous step's MidState (double buffer).
 *
 * Status codes match the library: 0 ok, 1 invalid argument, 2 no memory,
 * 6 infeasible (a beam became empty / no finite path).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EINFEASIBLE 6

typedef struct {
  int32_t K;
  const float* log_pi;     /* [K]   log pi_j                                 */
  int32_t csr;             /* 0: dense logA, 1: CSR out-edges              */
  const float* logA;       /* dense [K*K], logA[i*K+j] = log A_ij          */
  const int32_t* row_ptr;  /* CSR [K+1]                                     */
  const int32_t* col;      /* CSR [nnz], target state of each edge          */
  const float* val;        /* CSR [nnz], log-weight of each edge            */
} orc_model;

/* ------------------------------------------------------------------------ */
/* Transition lookup for a single (i, j): logA[i][j], or -inf when the CSR  */
/* graph has no edge i->j.  Used only by initialisation and path scoring.   */
static float trans(const orc_model* m, int32_t i, int32_t j) {
  if (!m->csr) return m->logA[(int64_t)i * m->K + j];
  float best = -INFINITY;
  for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e)
    if (m->col[e] == j && m->val[e] > best) best = m->val[e];
  return best;
}

/* ------------------------------------------------------------------------ */
/* One exact Viterbi step (Sec. III-A, recursion for delta_t and psi_t, in  */
/* log form as in Alg. 2): for every target j, scan sources i ascending,    */
/* c = fl(dprev[i] + logA[i][j]); keep the first strict maximum (R2); then  */
/* dnext[j] = fl(best + Et[j]) (R1) and psi[j] = its source.                */
/* The dense loop visits i in the outer loop and j in the inner loop; each  */
/* target still sees its candidates in ascending i, one at a time.          */
static void exact_step(const orc_model* m, const float* dprev, const float* Et,
                       float* best, float* dnext, int32_t* psi) {
  const int32_t K = m->K;
  if (!m->csr) {
    for (int32_t i = 0; i < K; ++i) {
      const float* Ai = m->logA + (int64_t)i * K;
      for (int32_t j = 0; j < K; ++j) {
        float c = dprev[i] + Ai[j];
        if (i == 0 || c > best[j]) { best[j] = c; psi[j] = i; }
      }
    }
  } else {
    /* Missing edges are -inf candidates; a -inf candidate never beats the
       initial -inf, so psi stays 0 exactly as in the dense rule. */
    for (int32_t j = 0; j < K; ++j) { best[j] = -INFINITY; psi[j] = 0; }
    for (int32_t i = 0; i < K; ++i)
      for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e) {
        int32_t j = m->col[e];
        float c = dprev[i] + m->val[e];
        if (c > best[j]) { best[j] = c; psi[j] = i; }
      }
  }
  for (int32_t j = 0; j < K; ++j) dnext[j] = best[j] + Et[j];
}

/* Lowest index of the maximum of v[0..K) (termination, Sec. III-A).       */
static int32_t argmax_lowest(const float* v, int32_t K) {
  int32_t q = 0;
  for (int32_t j = 1; j < K; ++j) if (v[j] > v[q]) q = j;
  return q;
}

/* ======================================================================== */
/* Vanilla Viterbi with a full backpointer table (Sec. III-A).             */
int orc_viterbi(const orc_model* m, int32_t T, const float* E,
                int32_t* path, float* score) {
  if (!m || T < 1 || m->K < 1) return ORC_EINVAL;
  const int32_t K = m->K;
  float* d0 = malloc(sizeof(float) * K);
  float* d1 = malloc(sizeof(float) * K);
  float* best = malloc(sizeof(float) * K);
  int32_t* psi = malloc(sizeof(int32_t) * (size_t)T * K);
  if (!d0 || !d1 || !best || !psi) { free(d0); free(d1); free(best); free(psi); return ORC_ENOMEM; }
  for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + E[j];       /* t = 0 */
  for (int32_t t = 1; t < T; ++t) {
    exact_step(m, d0, E + (int64_t)t * K, best, d1, psi + (int64_t)t * K);
    float* tmp = d0; d0 = d1; d1 = tmp;
  }
  int32_t q = argmax_lowest(d0, K);
  *score = d0[q];
  path[T - 1] = q;
  for (int32_t t = T - 1; t >= 1; --t) { q = psi[(int64_t)t * K + q]; path[t - 1] = q; }
  free(d0); free(d1); free(best); free(psi);
  return ORC_OK;
}

/* ======================================================================== */
/* Path score (log-likelihood of a given path) in the forward order:       */
/* s = fl(logpi[q0] + E0[q0]); s = fl(fl(s + logA[q_{t-1}][q_t]) + E_t[q_t]) */
float orc_path_score(const orc_model* m, int32_t T, const float* E, const int32_t* path) {
  const int32_t K = m->K;
  float s = m->log_pi[path[0]] + E[path[0]];
  for (int32_t t = 1; t < T; ++t) {
    s = s + trans(m, path[t - 1], path[t]);
    s = s + E[(int64_t)t * K + path[t]];
  }
  return s;
}

/* ======================================================================== */
/* FLASH Viterbi: Alg. 1 (non-recursive divide and conquer with the P-way   */
/* first split of Sec. V-A.3) driving Alg. 2 (subtask decoding) with the    */
/* pruned initialisation of Sec. V-B.2 (R4).                                */

typedef struct {           /* a queued subtask (m, n) and what it inherits  */
  int32_t m, n;
  int32_t q_prev;          /* q*_{m-1} (unused when m == 0)                 */
  float s_prev;            /* delta_{m-1}[q*_{m-1}], the retained offset    */
} orc_task;

/* Root task (Alg. 1, first Decoding call): the full recursion over        */
/* [0, T-1] with one MidState array per division point e_k (k < P'-1),     */
/* started at e_k+1 from PreState and then chained (Alg. 2, MidState       */
/* rules; R8).  Reveals q* and delta at every division point.              */
static int flash_root(const orc_model* m, int32_t T, const float* E, int32_t Pe,
                      const int32_t* e, int32_t* path, float* sval, float* score) {
  const int32_t K = m->K;
  const int32_t nd = Pe - 1;                 /* division points before T-1  */
  float* d0 = malloc(sizeof(float) * K);
  float* d1 = malloc(sizeof(float) * K);
  float* best = malloc(sizeof(float) * K);
  int32_t* pre = malloc(sizeof(int32_t) * K);
  int32_t* mid = malloc(sizeof(int32_t) * (size_t)(nd > 0 ? nd : 1) * K);
  int32_t* mid_new = malloc(sizeof(int32_t) * K);
  float* snap = malloc(sizeof(float) * (size_t)Pe * K);
  if (!d0 || !d1 || !best || !pre || !mid || !mid_new || !snap) {
    free(d0); free(d1); free(best); free(pre); free(mid); free(mid_new); free(snap);
    return ORC_ENOMEM;
  }
  for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + E[j];
  for (int32_t k = 0; k < Pe; ++k)
    if (e[k] == 0) memcpy(snap + (int64_t)k * K, d0, sizeof(float) * K);
  for (int32_t t = 1; t < T; ++t) {
    exact_step(m, d0, E + (int64_t)t * K, best, d1, pre);
    float* tmp = d0; d0 = d1; d1 = tmp;
    for (int32_t k = 0; k < nd; ++k) {
      int32_t* mk = mid + (int64_t)k * K;
      if (t == e[k] + 1) {
        for (int32_t j = 0; j < K; ++j) mk[j] = pre[j];
      } else if (t > e[k] + 1) {
        for (int32_t j = 0; j < K; ++j) mid_new[j] = mk[pre[j]];
        memcpy(mk, mid_new, sizeof(int32_t) * K);
      }
    }
    for (int32_t k = 0; k < Pe; ++k)
      if (e[k] == t) memcpy(snap + (int64_t)k * K, d0, sizeof(float) * K);
  }
  int32_t qT = argmax_lowest(d0, K);
  *score = d0[qT];
  path[T - 1] = qT;
  sval[T - 1] = d0[qT];
  for (int32_t k = 0; k < nd; ++k) {
    int32_t q = mid[(int64_t)k * K + qT];
    path[e[k]] = q;
    sval[e[k]] = snap[(int64_t)k * K + q];
  }
  free(d0); free(d1); free(best); free(pre); free(mid); free(mid_new); free(snap);
  return ORC_OK;
}

/* Subtask decoding (Alg. 2) of segment (m, n) whose end state q*_n is     */
/* known.  Initialisation: m == 0 uses pi (Alg. 2, base case); otherwise   */
/* only transitions out of q*_{m-1} are kept (Sec. V-B.2) with the         */
/* retained offset (R4) or offset 0 (complete pruning).  Outputs           */
/* q*_{tmid} = MidState[q*_n] and delta_{tmid}[q*_{tmid}].                 */
static int flash_subtask(const orc_model* m, const float* E, const orc_task* tk,
                         int32_t q_n, int complete, int32_t* q_mid, float* s_mid) {
  const int32_t K = m->K;
  const int32_t tmid = (tk->m + tk->n) / 2;
  float* d0 = malloc(sizeof(float) * K);
  float* d1 = malloc(sizeof(float) * K);
  float* best = malloc(sizeof(float) * K);
  float* snap = malloc(sizeof(float) * K);
  int32_t* pre = malloc(sizeof(int32_t) * K);
  int32_t* mid = malloc(sizeof(int32_t) * K);
  int32_t* mid_new = malloc(sizeof(int32_t) * K);
  if (!d0 || !d1 || !best || !snap || !pre || !mid || !mid_new) {
    free(d0); free(d1); free(best); free(snap); free(pre); free(mid); free(mid_new);
    return ORC_ENOMEM;
  }
  const float* Em = E + (int64_t)tk->m * K;
  if (tk->m == 0) {
    for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + Em[j];
  } else {
    for (int32_t j = 0; j < K; ++j) {
      float a = trans(m, tk->q_prev, j);
      d0[j] = complete ? (a + Em[j]) : ((tk->s_prev + a) + Em[j]);
    }
  }
  if (tmid == tk->m) memcpy(snap, d0, sizeof(float) * K);
  for (int32_t t = tk->m + 1; t <= tk->n; ++t) {
    exact_step(m, d0, E + (int64_t)t * K, best, d1, pre);
    float* tmp = d0; d0 = d1; d1 = tmp;
    if (t == tmid) memcpy(snap, d0, sizeof(float) * K);
    if (t == tmid + 1) {
      for (int32_t j = 0; j < K; ++j) mid[j] = pre[j];
    } else if (t > tmid + 1) {
      for (int32_t j = 0; j < K; ++j) mid_new[j] = mid[pre[j]];
      memcpy(mid, mid_new, sizeof(int32_t) * K);
    }
  }
  *q_mid = mid[q_n];
  *s_mid = snap[*q_mid];
  free(d0); free(d1); free(best); free(snap); free(pre); free(mid); free(mid_new);
  return ORC_OK;
}

/* P' and the division points e_k (R3).                                    */
static int32_t split_points(int32_t T, int32_t P, int32_t* e) {
  int32_t Pe = (T == 1) ? 1 : (P < 2 ? 2 : P);
  if (Pe > T) Pe = T;
  for (int32_t k = 0; k < Pe; ++k) e[k] = (int32_t)((((int64_t)k + 1) * T - 1) / Pe);
  return Pe;
}

int32_t orc_split_points(int32_t T, int32_t P, int32_t* e) { return split_points(T, P, e); }

/* Budget leaf (the memory-bounded end of Alg. 1's recursion): a segment  */
/* (m, n) whose backpointer rows psi_{m+1..n} fit the budget is decoded    */
/* directly -- the same pruned start as a subtask (R4), the recursion of   */
/* Sec. III-A with psi kept for the segment, then the backtrack from the   */
/* known q*_n writes q*_{n-1} .. q*_m.                                      */
static int flash_leaf(const orc_model* m, const float* E, const orc_task* tk, int32_t q_n, int complete,
                      int32_t* path) {
  const int32_t K = m->K, rows = tk->n - tk->m;
  float* d0 = malloc(sizeof(float) * K);
  float* d1 = malloc(sizeof(float) * K);
  float* best = malloc(sizeof(float) * K);
  int32_t* psi = malloc(sizeof(int32_t) * (size_t)(rows > 0 ? rows : 1) * K);
  if (!d0 || !d1 || !best || !psi) { free(d0); free(d1); free(best); free(psi); return ORC_ENOMEM; }
  const float* Em = E + (int64_t)tk->m * K;
  if (tk->m == 0) {
    for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + Em[j];
  } else {
    for (int32_t j = 0; j < K; ++j) {
      float a = trans(m, tk->q_prev, j);
      d0[j] = complete ? (a + Em[j]) : ((tk->s_prev + a) + Em[j]);
    }
  }
  for (int32_t t = tk->m + 1; t <= tk->n; ++t) {
    exact_step(m, d0, E + (int64_t)t * K, best, d1, psi + (int64_t)(t - tk->m - 1) * K);
    float* tmp = d0; d0 = d1; d1 = tmp;
  }
  int32_t q = q_n;
  for (int32_t t = tk->n; t > tk->m; --t) {
    q = psi[(int64_t)(t - tk->m - 1) * K + q];
    path[t - 1] = q;
  }
  free(d0); free(d1); free(best); free(psi);
  return ORC_OK;
}

/* FLASH Viterbi with a backpointer budget of budget_rows rows of K      */
/* entries: a dequeued task with n - m <= budget_rows is a leaf (above);    */
/* budget_rows = 0 is the pure divide-and-conquer of Alg. 1.  task_log     */
/* (optional, 3*T ints) receives (m, n, tmid) of every subtask in           */
/* processing order; *n_tasks their count, *n_leaves the leaves solved.     */
int orc_flash_budget(const orc_model* m, int32_t T, const float* E, int32_t P, int32_t complete,
                     int64_t budget_rows, int32_t* path, float* score, int32_t* task_log, int32_t* n_tasks,
                     int32_t* n_leaves) {
  if (!m || T < 1 || m->K < 1 || P < 1 || budget_rows < 0) return ORC_EINVAL;
  int32_t* e = malloc(sizeof(int32_t) * T);
  float* sval = malloc(sizeof(float) * T);
  orc_task* queue = malloc(sizeof(orc_task) * (size_t)T);
  if (!e || !sval || !queue) { free(e); free(sval); free(queue); return ORC_ENOMEM; }
  int32_t Pe = split_points(T, P, e);
  int rc = flash_root(m, T, E, Pe, e, path, sval, score);
  int32_t head = 0, tail = 0, count = 0;
  /* InitialEnqueue: the P' segments (e_{k-1}+1, e_k); a segment of one     */
  /* step is already revealed by the root and needs no task.               */
  for (int32_t k = 0; rc == ORC_OK && k < Pe; ++k) {
    int32_t mm = (k == 0) ? 0 : e[k - 1] + 1, nn = e[k];
    if (nn - mm >= 1) {
      queue[tail].m = mm; queue[tail].n = nn;
      queue[tail].q_prev = mm > 0 ? path[mm - 1] : 0;
      queue[tail].s_prev = mm > 0 ? sval[mm - 1] : 0.0f;
      ++tail;
    }
  }
  /* Task loop of Alg. 1 (serial FIFO order).                               */
  int32_t leaves = 0;
  while (rc == ORC_OK && head < tail) {
    orc_task tk = queue[head++];
    if ((int64_t)(tk.n - tk.m) <= budget_rows) {
      rc = flash_leaf(m, E, &tk, path[tk.n], complete, path);
      ++leaves;
      continue;
    }
    int32_t tmid = (tk.m + tk.n) / 2;
    int32_t qm; float sm;
    rc = flash_subtask(m, E, &tk, path[tk.n], complete, &qm, &sm);
    if (rc != ORC_OK) break;
    path[tmid] = qm; sval[tmid] = sm;
    if (task_log) { task_log[3 * count] = tk.m; task_log[3 * count + 1] = tk.n; task_log[3 * count + 2] = tmid; }
    ++count;
    if (tk.n - tk.m > 2) {
      queue[tail].m = tk.m; queue[tail].n = tmid; queue[tail].q_prev = tk.q_prev; queue[tail].s_prev = tk.s_prev; ++tail;
      queue[tail].m = tmid + 1; queue[tail].n = tk.n; queue[tail].q_prev = qm; queue[tail].s_prev = sm; ++tail;
    } else if (tk.n - tk.m == 2) {
      queue[tail].m = tk.m; queue[tail].n = tmid; queue[tail].q_prev = tk.q_prev; queue[tail].s_prev = tk.s_prev; ++tail;
    }
  }
  if (n_tasks) *n_tasks = count;
  if (n_leaves) *n_leaves = leaves;
  free(e); free(sval); free(queue);
  return rc;
}

/* FLASH Viterbi without a budget (Alg. 1 + Alg. 2 throughout).            */
int orc_flash(const orc_model* m, int32_t T, const float* E, int32_t P, int32_t complete,
              int32_t* path, float* score, int32_t* task_log, int32_t* n_tasks) {
  return orc_flash_budget(m, T, E, P, complete, 0, path, score, task_log, n_tasks, NULL);
}

/* ======================================================================== */
/* Checkpoint Viterbi (the baseline of Sec. II-A, after Tarnas et al.):     */
/* one forward pass keeps delta only at P' evenly spaced checkpoints        */
/* (P' = ceil(sqrt(T)) by default, as the paper describes it), then the    */
/* segments between checkpoints are decoded again from the last one,       */
/* latest segment first, each with its own backpointer rows, and           */
/* backtracked from the state already known at its end.  Checkpoints are   */
/* the division points e_k of R3 (e_{P'-1} = T-1); segment k covers steps   */
/* e_{k-1}+1 .. e_k and restarts from the stored delta_{e_{k-1}} (segment  */
/* 0 from pi at t = 0).  The restarts are exact, so every backpointer      */
/* equals the full table's.  Memory: P' rows of K floats plus one segment  */
/* of at most ceil(T/P') rows.  *max_rows receives the largest segment.    */
int32_t orc_checkpoint_count(int32_t T, int32_t P) {
  if (T <= 1) return 1;
  int32_t c = P;
  if (c < 1) {
    c = (int32_t)ceil(sqrt((double)T));
    while ((int64_t)c * c < T) ++c;           /* exact integer ceiling */
    while (c > 1 && (int64_t)(c - 1) * (c - 1) >= T) --c;
  }
  return c < T ? c : T;
}

int orc_checkpoint(const orc_model* m, int32_t T, const float* E, int32_t P, int32_t* path, float* score,
                   int32_t* n_ckpt, int32_t* max_rows) {
  if (!m || T < 1 || m->K < 1) return ORC_EINVAL;
  const int32_t K = m->K, C = orc_checkpoint_count(T, P);
  int32_t* e = malloc(sizeof(int32_t) * (size_t)C);
  float* ck = malloc(sizeof(float) * (size_t)C * K);
  float* d0 = malloc(sizeof(float) * K);
  float* d1 = malloc(sizeof(float) * K);
  float* best = malloc(sizeof(float) * K);
  int32_t* junk = malloc(sizeof(int32_t) * K);
  const int32_t seg_cap = (T + C - 1) / C + 1;
  int32_t* psi = malloc(sizeof(int32_t) * (size_t)seg_cap * K);
  if (!e || !ck || !d0 || !d1 || !best || !junk || !psi) {
    free(e); free(ck); free(d0); free(d1); free(best); free(junk); free(psi);
    return ORC_ENOMEM;
  }
  for (int32_t k = 0; k < C; ++k) e[k] = (int32_t)((((int64_t)k + 1) * T - 1) / C);
  /* forward pass: delta kept only at the checkpoints */
  int32_t kc = 0;
  for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + E[j];
  if (e[0] == 0) { memcpy(ck, d0, sizeof(float) * K); kc = 1; }
  for (int32_t t = 1; t < T; ++t) {
    exact_step(m, d0, E + (int64_t)t * K, best, d1, junk);
    float* tmp = d0; d0 = d1; d1 = tmp;
    if (kc < C && t == e[kc]) { memcpy(ck + (int64_t)kc * K, d0, sizeof(float) * K); ++kc; }
  }
  const float* last = ck + (int64_t)(C - 1) * K;
  int32_t q = argmax_lowest(last, K);
  *score = last[q];
  path[T - 1] = q;
  /* segments, latest first */
  int32_t rows_max = 0;
  for (int32_t k = C - 1; k >= 0; --k) {
    const int32_t mm = (k == 0) ? 0 : e[k - 1], nn = e[k], rows = nn - mm;
    if (rows > rows_max) rows_max = rows;
    if (rows < 1) continue;
    if (k == 0) {
      for (int32_t j = 0; j < K; ++j) d0[j] = m->log_pi[j] + E[j];
    } else {
      memcpy(d0, ck + (int64_t)(k - 1) * K, sizeof(float) * K);
    }
    for (int32_t t = mm + 1; t <= nn; ++t) {
      exact_step(m, d0, E + (int64_t)t * K, best, d1, psi + (int64_t)(t - mm - 1) * K);
      float* tmp = d0; d0 = d1; d1 = tmp;
    }
    q = path[nn];
    for (int32_t t = nn; t > mm; --t) {
      q = psi[(int64_t)(t - mm - 1) * K + q];
      path[t - 1] = q;
    }
  }
  if (n_ckpt) *n_ckpt = C;
  if (max_rows) *max_rows = rows_max;
  free(e); free(ck); free(d0); free(d1); free(best); free(junk); free(psi);
  return ORC_OK;
}

/* ======================================================================== */
/* Dynamic beam search (Sec. V-C).  A beam is a set of (state, score)      */
/* entries: the top-B finite candidates under (score desc, id asc) (R6).   */

typedef struct { int32_t id; float v; int32_t src; int32_t mid; } orc_cand;

static int cand_order(const void* a, const void* b) {  /* score desc, id asc */
  const orc_cand* x = a; const orc_cand* y = b;
  if (x->v > y->v) return -1;
  if (x->v < y->v) return 1;
  return (x->id > y->id) - (x->id < y->id);
}
static int id_order(const void* a, const void* b) {
  const orc_cand* x = a; const orc_cand* y = b;
  return (x->id > y->id) - (x->id < y->id);
}

/* Keep the top-B finite entries of c[0..n), then re-sort them by id so the */
/* next step visits its sources in ascending order.  Returns the size.     */
static int32_t select_top_b(orc_cand* c, int32_t n, int32_t B) {
  int32_t f = 0;
  for (int32_t k = 0; k < n; ++k) if (isfinite(c[k].v)) c[f++] = c[k];
  qsort(c, (size_t)f, sizeof(orc_cand), cand_order);
  if (f > B) f = B;
  qsort(c, (size_t)f, sizeof(orc_cand), id_order);
  return f;
}

/* One beam step: for every target reachable from the beam (all K targets  */
/* for dense logA, successors for CSR) the best source in ascending id     */
/* order (first strict maximum), then fl(best + E_t[j]).  `mid_of_src`     */
/* maps a source entry index to the value carried forward in `mid`.        */
/* Writes the unselected candidate list into out (size returned).          */
static int32_t beam_candidates(const orc_model* m, const orc_cand* beam, int32_t nb,
                               const float* Et, float* best, int32_t* arg, int32_t* slot,
                               uint8_t* touched, orc_cand* out) {
  const int32_t K = m->K;
  int32_t n = 0;
  for (int32_t j = 0; j < K; ++j) { best[j] = -INFINITY; arg[j] = -1; touched[j] = 0; }
  for (int32_t k = 0; k < nb; ++k) {
    int32_t i = beam[k].id;
    if (!m->csr) {
      const float* Ai = m->logA + (int64_t)i * K;
      for (int32_t j = 0; j < K; ++j) {
        float c = beam[k].v + Ai[j];
        touched[j] = 1;
        if (arg[j] < 0 || c > best[j]) { best[j] = c; arg[j] = i; slot[j] = k; }
      }
    } else {
      for (int32_t e = m->row_ptr[i]; e < m->row_ptr[i + 1]; ++e) {
        int32_t j = m->col[e];
        float c = beam[k].v + m->val[e];
        touched[j] = 1;
        if (arg[j] < 0 || c > best[j]) { best[j] = c; arg[j] = i; slot[j] = k; }
      }
    }
  }
  for (int32_t j = 0; j < K; ++j)
    if (touched[j]) {
      out[n].id = j; out[n].v = best[j] + Et[j]; out[n].src = arg[j]; out[n].mid = slot[j];
      ++n;
    }
  return n;
}

typedef struct {
  float* best; int32_t* arg; int32_t* slot; uint8_t* touched; orc_cand* cand;
} beam_scratch;

static int scratch_alloc(beam_scratch* s, int32_t K) {
  s->best = malloc(sizeof(float) * K); s->arg = malloc(sizeof(int32_t) * K);
  s->slot = malloc(sizeof(int32_t) * K); s->touched = malloc((size_t)K);
  s->cand = malloc(sizeof(orc_cand) * (size_t)K);
  return (s->best && s->arg && s->slot && s->touched && s->cand) ? ORC_OK : ORC_ENOMEM;
}
static void scratch_free(beam_scratch* s) {
  free(s->best); free(s->arg); free(s->slot); free(s->touched); free(s->cand);
}

/* Beam with per-step beam backpointers (P = 0): stores, per step, the     */
/* beam's states and their sources (O(T*B) memory) and backtracks from the */
/* best final entry.  Returns ORC_EINFEASIBLE if a beam becomes empty.      */
int orc_beam(const orc_model* m, int32_t T, const float* E, int32_t B,
             int32_t* path, float* score) {
  if (!m || T < 1 || m->K < 1 || B < 1) return ORC_EINVAL;
  const int32_t K = m->K;
  const int32_t W = B < K ? B : K;
  beam_scratch s;
  int32_t* ids = malloc(sizeof(int32_t) * (size_t)T * W);
  int32_t* src = malloc(sizeof(int32_t) * (size_t)T * W);
  int32_t* cnt = malloc(sizeof(int32_t) * (size_t)T);
  orc_cand* beam = malloc(sizeof(orc_cand) * (size_t)W);
  int rc = scratch_alloc(&s, K);
  if (rc != ORC_OK || !ids || !src || !cnt || !beam) {
    scratch_free(&s); free(ids); free(src); free(cnt); free(beam); return ORC_ENOMEM;
  }
  for (int32_t j = 0; j < K; ++j) { s.cand[j].id = j; s.cand[j].v = m->log_pi[j] + E[j]; s.cand[j].src = 0; s.cand[j].mid = 0; }
  int32_t nb = select_top_b(s.cand, K, W);
  for (int32_t t = 0; rc == ORC_OK; ) {
    if (nb == 0) { rc = ORC_EINFEASIBLE; break; }
    memcpy(beam, s.cand, sizeof(orc_cand) * (size_t)nb);
    cnt[t] = nb;
    for (int32_t k = 0; k < nb; ++k) { ids[(int64_t)t * W + k] = beam[k].id; src[(int64_t)t * W + k] = beam[k].src; }
    if (++t == T) break;
    int32_t n = beam_candidates(m, beam, nb, E + (int64_t)t * K, s.best, s.arg, s.slot, s.touched, s.cand);
    nb = select_top_b(s.cand, n, W);
  }
  if (rc == ORC_OK) {
    int32_t kb = 0;                          /* best entry: score desc, id asc */
    for (int32_t k = 1; k < nb; ++k)
      if (beam[k].v > beam[kb].v) kb = k;
    *score = beam[kb].v;
    int32_t q = beam[kb].id, sq = beam[kb].src;
    path[T - 1] = q;
    for (int32_t t = T - 1; t >= 1; --t) {
      q = sq; path[t - 1] = q;
      int32_t k = 0;
      while (ids[(int64_t)(t - 1) * W + k] != q) ++k;
      sq = src[(int64_t)(t - 1) * W + k];
    }
  } else {
    for (int32_t t = 0; t < T; ++t) path[t] = 0;
    *score = -INFINITY;
  }
  scratch_free(&s); free(ids); free(src); free(cnt); free(beam);
  return rc;
}

/* Static beam (the SIEVE-BS style beam the paper contrasts with its own,  */
/* Sec. II-B and Sec. V-C.1): every step first computes the score of all K */
/* states -- the best transition from the previous beam, -inf where none   */
/* leads -- and only then keeps the top B of the whole K-entry vector       */
/* (score desc, id asc; -inf never kept).  Beam backpointers per step as   */
/* in orc_beam; the final state is the best entry.                         */
typedef struct { float v; int32_t id; } orc_entry;
static int entry_order(const void* a, const void* b) {  /* score desc, id asc */
  const orc_entry* x = a; const orc_entry* y = b;
  if (x->v > y->v) return -1;
  if (x->v < y->v) return 1;
  return (x->id > y->id) - (x->id < y->id);
}
static int entry_id_order(const void* a, const void* b) {
  const orc_entry* x = a; const orc_entry* y = b;
  return (x->id > y->id) - (x->id < y->id);
}

int orc_beam_static(const orc_model* m, int32_t T, const float* E, int32_t B, int32_t* path, float* score) {
  if (!m || T < 1 || m->K < 1 || B < 1) return ORC_EINVAL;
  const int32_t K = m->K, W = B < K ? B : K;
  float* full = malloc(sizeof(float) * K);      /* scores of all K states, this step */
  int32_t* from = malloc(sizeof(int32_t) * K);  /* their source state (-1: none)     */
  orc_entry* idx = malloc(sizeof(orc_entry) * K);
  float* bval = malloc(sizeof(float) * W);      /* current beam, id order            */
  int32_t* bid = malloc(sizeof(int32_t) * W);
  int32_t* ids = malloc(sizeof(int32_t) * (size_t)T * W);
  int32_t* src = malloc(sizeof(int32_t) * (size_t)T * W);
  int32_t* cnt = malloc(sizeof(int32_t) * (size_t)T);
  if (!full || !from || !idx || !bval || !bid || !ids || !src || !cnt) {
    free(full); free(from); free(idx); free(bval); free(bid); free(ids); free(src); free(cnt);
    return ORC_ENOMEM;
  }
  int rc = ORC_OK;
  int32_t nb = 0;
  for (int32_t t = 0; t < T; ++t) {
    const float* Et = E + (int64_t)t * K;
    for (int32_t j = 0; j < K; ++j) { full[j] = -INFINITY; from[j] = -1; }
    if (t == 0) {
      for (int32_t j = 0; j < K; ++j) full[j] = m->log_pi[j] + Et[j];
    } else {
      /* each state's best transition from the beam: sources visited in */
      /* ascending id, so a target keeps its first strict maximum         */
      for (int32_t k = 0; k < nb; ++k) {
        const int32_t i = bid[k];
        const int32_t e0 = m->csr ? m->row_ptr[i] : 0, e1 = m->csr ? m->row_ptr[i + 1] : K;
        for (int32_t e = e0; e < e1; ++e) {
          const int32_t j = m->csr ? m->col[e] : e;
          const float c = bval[k] + (m->csr ? m->val[e] : m->logA[(int64_t)i * K + j]);
          if (from[j] < 0 || c > full[j]) { full[j] = c; from[j] = i; }
        }
      }
      for (int32_t j = 0; j < K; ++j) {
        if (from[j] >= 0 && full[j] > -INFINITY) full[j] = full[j] + Et[j];
        else { full[j] = -INFINITY; from[j] = -1; }
      }
    }
    for (int32_t j = 0; j < K; ++j) { idx[j].v = full[j]; idx[j].id = j; }
    qsort(idx, (size_t)K, sizeof(orc_entry), entry_order);
    int32_t n = 0;
    while (n < W && n < K && idx[n].v > -INFINITY) ++n;
    qsort(idx, (size_t)n, sizeof(orc_entry), entry_id_order);
    if (n == 0) { rc = ORC_EINFEASIBLE; break; }
    for (int32_t k = 0; k < n; ++k) {
      const int32_t j = idx[k].id;
      bid[k] = j;
      bval[k] = full[j];
      ids[(int64_t)t * W + k] = j;
      src[(int64_t)t * W + k] = from[j];
    }
    nb = n;
    cnt[t] = n;
  }
  if (rc == ORC_OK) {
    int32_t kb = 0;
    for (int32_t k = 1; k < nb; ++k) if (bval[k] > bval[kb]) kb = k;
    *score = bval[kb];
    int32_t q = bid[kb];
    path[T - 1] = q;
    for (int32_t t = T - 1; t >= 1; --t) {
      int32_t k = 0;
      while (ids[(int64_t)t * W + k] != q) ++k;
      q = src[(int64_t)t * W + k];
      path[t - 1] = q;
    }
  } else {
    for (int32_t t = 0; t < T; ++t) path[t] = 0;
    *score = -INFINITY;
  }
  free(full); free(from); free(idx); free(bval); free(bid); free(ids); free(src); free(cnt);
  return rc;
}

/* Index of state `id` in an id-sorted beam (binary search); -1 if absent. */
static int32_t beam_find(const orc_cand* beam, int32_t nb, int32_t id) {
  int32_t lo = 0, hi = nb - 1;
  while (lo <= hi) {
    int32_t md = (lo + hi) / 2;
    if (beam[md].id == id) return md;
    if (beam[md].id < id) lo = md + 1; else hi = md - 1;
  }
  return -1;
}

/* FLASH-BS root: beam search over [0, T-1] where every beam entry carries */
/* one MidState per division point (Sec. V-C.2: State, OptProb, MidState). */
static int flash_bs_root(const orc_model* m, int32_t T, const float* E, int32_t W,
                         int32_t Pe, const int32_t* e, int32_t* path, float* sval) {
  const int32_t K = m->K, nd = Pe - 1;
  beam_scratch s;
  orc_cand* beam = malloc(sizeof(orc_cand) * (size_t)W);
  int32_t* mids = malloc(sizeof(int32_t) * (size_t)W * (nd > 0 ? nd : 1));
  int32_t* mids_new = malloc(sizeof(int32_t) * (size_t)W * (nd > 0 ? nd : 1));
  orc_cand* snap = malloc(sizeof(orc_cand) * (size_t)W * Pe);
  int32_t* snap_n = malloc(sizeof(int32_t) * (size_t)Pe);
  int rc = scratch_alloc(&s, K);
  if (rc != ORC_OK || !beam || !mids || !mids_new || !snap || !snap_n) {
    scratch_free(&s); free(beam); free(mids); free(mids_new); free(snap); free(snap_n); return ORC_ENOMEM;
  }
  for (int32_t j = 0; j < K; ++j) { s.cand[j].id = j; s.cand[j].v = m->log_pi[j] + E[j]; s.cand[j].src = 0; s.cand[j].mid = 0; }
  int32_t nb = select_top_b(s.cand, K, W);
  for (int32_t t = 0; ; ) {
    if (nb == 0) { rc = ORC_EINFEASIBLE; break; }
    /* MidState of the new entries from their source entries (R8).          */
    for (int32_t k = 0; k < nd; ++k)
      for (int32_t x = 0; x < nb; ++x) {
        int32_t v;
        if (t == e[k] + 1) v = s.cand[x].src;
        else if (t > e[k] + 1) v = mids[(int64_t)s.cand[x].mid * nd + k];
        else v = -1;
        mids_new[(int64_t)x * nd + k] = v;
      }
    memcpy(mids, mids_new, sizeof(int32_t) * (size_t)nb * (nd > 0 ? nd : 0));
    memcpy(beam, s.cand, sizeof(orc_cand) * (size_t)nb);
    for (int32_t k = 0; k < Pe; ++k)
      if (e[k] == t) { memcpy(snap + (int64_t)k * W, beam, sizeof(orc_cand) * (size_t)nb); snap_n[k] = nb; }
    if (++t == T) break;
    int32_t n = beam_candidates(m, beam, nb, E + (int64_t)t * K, s.best, s.arg, s.slot, s.touched, s.cand);
    nb = select_top_b(s.cand, n, W);
  }
  if (rc == ORC_OK) {
    int32_t kb = 0;
    for (int32_t k = 1; k < nb; ++k) if (beam[k].v > beam[kb].v) kb = k;
    path[T - 1] = beam[kb].id;
    sval[T - 1] = beam[kb].v;
    for (int32_t k = 0; k < nd; ++k) {
      int32_t q = mids[(int64_t)kb * nd + k];
      path[e[k]] = q;
      int32_t x = beam_find(snap + (int64_t)k * W, snap_n[k], q);
      sval[e[k]] = snap[(int64_t)k * W + x].v;
    }
  }
  scratch_free(&s); free(beam); free(mids); free(mids_new); free(snap); free(snap_n);
  return rc;
}

/* FLASH-BS subtask (m, n): beam search from the pruned start, MidState per */
/* entry from tmid+1 on; in step n only target q*_n is evaluated (R7).     */
/* Returns ORC_EINFEASIBLE when q*_n cannot be reached from the beam.       */
static int flash_bs_subtask(const orc_model* m, const float* E, const orc_task* tk,
                            int32_t q_n, int32_t W, int complete,
                            int32_t* q_mid, float* s_mid) {
  const int32_t K = m->K, tmid = (tk->m + tk->n) / 2;
  beam_scratch s;
  orc_cand* beam = malloc(sizeof(orc_cand) * (size_t)W);
  orc_cand* snap = malloc(sizeof(orc_cand) * (size_t)W);
  int32_t* mid = malloc(sizeof(int32_t) * (size_t)W);
  int32_t* mid_new = malloc(sizeof(int32_t) * (size_t)W);
  int rc = scratch_alloc(&s, K);
  if (rc != ORC_OK || !beam || !snap || !mid || !mid_new) {
    scratch_free(&s); free(beam); free(snap); free(mid); free(mid_new); return ORC_ENOMEM;
  }
  const float* Em = E + (int64_t)tk->m * K;
  for (int32_t j = 0; j < K; ++j) {
    s.cand[j].id = j; s.cand[j].src = 0; s.cand[j].mid = 0;
    if (tk->m == 0) s.cand[j].v = m->log_pi[j] + Em[j];
    else {
      float a = trans(m, tk->q_prev, j);
      s.cand[j].v = complete ? (a + Em[j]) : ((tk->s_prev + a) + Em[j]);
    }
  }
  int32_t nb = select_top_b(s.cand, K, W), nsnap = 0;
  for (int32_t t = tk->m; ; ) {
    if (nb == 0) { rc = ORC_EINFEASIBLE; break; }
    for (int32_t x = 0; x < nb; ++x)
      mid_new[x] = (t == tmid + 1) ? s.cand[x].src : (t > tmid + 1 ? mid[s.cand[x].mid] : -1);
    memcpy(mid, mid_new, sizeof(int32_t) * (size_t)nb);
    memcpy(beam, s.cand, sizeof(orc_cand) * (size_t)nb);
    if (t == tmid) { memcpy(snap, beam, sizeof(orc_cand) * (size_t)nb); nsnap = nb; }
    ++t;
    if (t == tk->n) {
      /* Last step: evaluate target q_n from every beam source.             */
      float best = -INFINITY; int32_t arg = -1, slot = -1;
      for (int32_t k = 0; k < nb; ++k) {
        float c = beam[k].v + trans(m, beam[k].id, q_n);
        if (arg < 0 || c > best) { best = c; arg = beam[k].id; slot = k; }
      }
      if (!(best > -INFINITY)) { rc = ORC_EINFEASIBLE; break; }
      int32_t q = (t == tmid + 1) ? arg : mid[slot];
      *q_mid = q;
      *s_mid = snap[beam_find(snap, nsnap, q)].v;
      break;
    }
    int32_t n = beam_candidates(m, beam, nb, E + (int64_t)t * K, s.best, s.arg, s.slot, s.touched, s.cand);
    nb = select_top_b(s.cand, n, W);
  }
  scratch_free(&s); free(beam); free(snap); free(mid); free(mid_new);
  return rc;
}

/* FLASH-BS Viterbi (Sec. V-C): Alg. 1 over beam subtasks.  *n_reruns      */
/* counts subtasks that had to be re-run with the full state set (R7).     */
int orc_flash_bs(const orc_model* m, int32_t T, const float* E, int32_t P, int32_t B,
                 int32_t complete, int32_t* path, float* score, int32_t* n_reruns) {
  if (!m || T < 1 || m->K < 1 || P < 1 || B < 1) return ORC_EINVAL;
  const int32_t K = m->K, W = B < K ? B : K;
  int32_t* e = malloc(sizeof(int32_t) * T);
  float* sval = malloc(sizeof(float) * T);
  orc_task* queue = malloc(sizeof(orc_task) * (size_t)T);
  if (!e || !sval || !queue) { free(e); free(sval); free(queue); return ORC_ENOMEM; }
  int32_t Pe = split_points(T, P, e), reruns = 0;
  int rc = flash_bs_root(m, T, E, W, Pe, e, path, sval);
  int32_t head = 0, tail = 0;
  for (int32_t k = 0; rc == ORC_OK && k < Pe; ++k) {
    int32_t mm = (k == 0) ? 0 : e[k - 1] + 1, nn = e[k];
    if (nn - mm >= 1) {
      queue[tail].m = mm; queue[tail].n = nn;
      queue[tail].q_prev = mm > 0 ? path[mm - 1] : 0;
      queue[tail].s_prev = mm > 0 ? sval[mm - 1] : 0.0f;
      ++tail;
    }
  }
  while (rc == ORC_OK && head < tail) {
    orc_task tk = queue[head++];
    int32_t tmid = (tk.m + tk.n) / 2, qm; float sm;
    rc = flash_bs_subtask(m, E, &tk, path[tk.n], W, complete, &qm, &sm);
    if (rc == ORC_EINFEASIBLE) {
      ++reruns;
      rc = flash_bs_subtask(m, E, &tk, path[tk.n], K, complete, &qm, &sm);
    }
    if (rc != ORC_OK) break;
    path[tmid] = qm; sval[tmid] = sm;
    if (tk.n - tk.m > 2) {
      queue[tail].m = tk.m; queue[tail].n = tmid; queue[tail].q_prev = tk.q_prev; queue[tail].s_prev = tk.s_prev; ++tail;
      queue[tail].m = tmid + 1; queue[tail].n = tk.n; queue[tail].q_prev = qm; queue[tail].s_prev = sm; ++tail;
    } else if (tk.n - tk.m == 2) {
      queue[tail].m = tk.m; queue[tail].n = tmid; queue[tail].q_prev = tk.q_prev; queue[tail].s_prev = tk.s_prev; ++tail;
    }
  }
  if (rc == ORC_OK) *score = orc_path_score(m, T, E, path);
  else { for (int32_t t = 0; t < T; ++t) path[t] = 0; *score = -INFINITY; }
  if (n_reruns) *n_reruns = reruns;
  free(e); free(sval); free(queue);
  return rc;
}

/* ======================================================================== */
/* Gradient of sum_b g_b * score_b along fixed paths (structured-perceptron */
/* backward; not in the paper).  For every model parameter the terms are    */
/* added in ascending sequence order, each term fl(g_b * count), starting   */
/* from +0; entries no path touches stay +0.                                */
/*   dlog_pi[j]  += g_b * [q_{b,0} = j]                                     */
/*   dlogA[i][j] += g_b * #{t : q_{b,t-1} = i, q_{b,t} = j}                  */
/*   dE[b][t][q_{b,t}] = g_b   (every other entry of dE is +0)              */
/* E and dE use the packed layout: sequence b starts at e_off[b] floats.    */
int orc_grad(int32_t K, int32_t n_seq, const int32_t* T, const int64_t* e_off,
             const int64_t* path_off, const int32_t* paths, const float* g,
             float* dlog_pi, float* dlogA, float* dE) {
  if (K < 1 || n_seq < 0) return ORC_EINVAL;
  int32_t* cnt = calloc((size_t)K * K, sizeof(int32_t));
  if (!cnt) return ORC_ENOMEM;
  for (int32_t j = 0; j < K; ++j) dlog_pi[j] = 0.0f;
  for (int64_t x = 0; x < (int64_t)K * K; ++x) dlogA[x] = 0.0f;
  for (int32_t b = 0; b < n_seq; ++b) {
    const int32_t* q = paths + path_off[b];
    float* dEb = dE + e_off[b];
    for (int64_t x = 0; x < (int64_t)T[b] * K; ++x) dEb[x] = 0.0f;
    for (int32_t t = 0; t < T[b]; ++t) dEb[(int64_t)t * K + q[t]] = g[b];
    dlog_pi[q[0]] = dlog_pi[q[0]] + g[b] * 1.0f;
    for (int32_t t = 1; t < T[b]; ++t) cnt[(int64_t)q[t - 1] * K + q[t]] += 1;
    for (int32_t t = 1; t < T[b]; ++t) {
      int64_t x = (int64_t)q[t - 1] * K + q[t];
      if (cnt[x] != 0) {
        dlogA[x] = dlogA[x] + g[b] * (float)cnt[x];
        cnt[x] = 0;
      }
    }
  }
  free(cnt);
  return ORC_OK;
}
