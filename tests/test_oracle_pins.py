"""Pins for the CPU oracle: each test checks the oracle against something
other than itself -- brute force over all K^T paths, closed forms, the
paper's worked T=16 schedule, its theorems as invariants, and float64 finite
differences -- so that a dropped term, a wrong index or a wrong tie rule in
the oracle fails here."""
import itertools
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Independent helpers (no oracle code): brute force and float64 Viterbi.

def brute_scores(log_pi, logA, E):
    """Forward-order FP32 score of every one of the K^T paths.
    Returns (paths [K^T, T], scores [K^T])."""
    T, K = E.shape
    paths = np.array(list(itertools.product(range(K), repeat=T)), dtype=np.int64)
    s = (log_pi[paths[:, 0]] + E[0, paths[:, 0]]).astype(np.float32)
    for t in range(1, T):
        s = (s + logA[paths[:, t - 1], paths[:, t]]).astype(np.float32)
        s = (s + E[t, paths[:, t]]).astype(np.float32)
    return paths, s


def lex_min_reversed(paths):
    """Path whose reversed sequence (q_{T-1}, ..., q_0) is smallest."""
    rev = paths[:, ::-1]
    order = np.lexsort(tuple(rev[:, k] for k in range(rev.shape[1] - 1, -1, -1)))
    return paths[order[0]]


def viterbi_f64(log_pi, logA, E):
    d = log_pi.astype(np.float64) + E[0].astype(np.float64)
    A = logA.astype(np.float64)
    for t in range(1, E.shape[0]):
        d = (d[:, None] + A).max(axis=0) + E[t].astype(np.float64)
    return d.max()


def bits(x):
    return np.float32(x).view(np.int32)


# --------------------------------------------------------------------------
# Vanilla Viterbi (Sec. III-A).

@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("T", [1, 2, 3, 5, 8])
def test_vanilla_matches_brute_force_score(oracle, K, T):
    if K ** T > 70000:
        pytest.skip("too many paths")
    for seed in range(3):
        log_pi, logA, E = W.random_small(K, T, seed=100 * K + 10 * T + seed)
        hmm = oracle.HMM(log_pi, logA)
        path, score = oracle.viterbi(hmm, E)
        paths, s = brute_scores(log_pi, logA, E)
        assert bits(score) == bits(s.max())
        # returned path attains the maximum; recomputed score equals it
        match = np.all(paths == path[None, :], axis=1)
        assert bits(s[match][0]) == bits(score)
        assert bits(oracle.path_score(hmm, E, path)) == bits(score)


@pytest.mark.parametrize("K,T", [(2, 8), (3, 6), (4, 5), (4, 8)])
def test_vanilla_tie_rule_integer_inputs(oracle, K, T):
    """Integer inputs are exact in FP32 and full of ties: the lowest-index
    rule returns the optimal path whose reversed sequence is smallest."""
    for seed in range(6):
        log_pi, logA, E = W.random_small(K, T, seed=seed, integer=True, lo=-2, hi=2)
        hmm = oracle.HMM(log_pi, logA)
        path, score = oracle.viterbi(hmm, E)
        paths, s = brute_scores(log_pi, logA, E)
        best = paths[s == s.max()]
        assert score == s.max()
        assert np.array_equal(path, lex_min_reversed(best))


def test_vanilla_with_neg_inf_transitions_matches_brute_force(oracle):
    for seed in range(10):
        log_pi, logA, E = W.random_small(4, 6, seed=seed, neg_inf_frac=0.5)
        hmm = oracle.HMM(log_pi, logA)
        path, score = oracle.viterbi(hmm, E)
        paths, s = brute_scores(log_pi, logA, E)
        assert bits(score) == bits(s.max())


def test_closed_form_identical_rows(oracle):
    """A[i,j] = a_j: q_t = argmax_j(a_j + E_t[j]) for t >= 1 and
    q_0 = argmax(logpi + E_0) (integer data, exact)."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        K, T = int(rng.integers(2, 12)), int(rng.integers(1, 30))
        a = rng.integers(-5, 6, K).astype(np.float32)
        logA = np.tile(a, (K, 1))
        log_pi = rng.integers(-5, 6, K).astype(np.float32)
        E = rng.integers(-5, 6, (T, K)).astype(np.float32)
        path, _ = oracle.viterbi(oracle.HMM(log_pi, logA), E)
        want = [int(np.argmax(log_pi + E[0]))] + [int(np.argmax(a + E[t])) for t in range(1, T)]
        assert path.tolist() == want


def test_closed_form_diagonal(oracle):
    """Off-diagonal -inf: the path is constant at
    argmax_j(logpi_j + (T-1) A_jj + sum_t E_t[j])."""
    rng = np.random.default_rng(8)
    for _ in range(10):
        K, T = int(rng.integers(1, 10)), int(rng.integers(1, 40))
        diag = rng.integers(-4, 5, K).astype(np.float32)
        logA = np.full((K, K), -np.inf, np.float32)
        logA[np.arange(K), np.arange(K)] = diag
        log_pi = rng.integers(-4, 5, K).astype(np.float32)
        E = rng.integers(-4, 5, (T, K)).astype(np.float32)
        path, score = oracle.viterbi(oracle.HMM(log_pi, logA), E)
        tot = log_pi.astype(np.int64) + (T - 1) * diag.astype(np.int64) + E.astype(np.int64).sum(0)
        j = int(np.argmax(tot))
        assert path.tolist() == [j] * T
        assert score == tot[j]


def test_single_step_and_single_state(oracle):
    log_pi = np.array([0.5, 2.0, 2.0, -1.0], np.float32)
    E = np.array([[1.0, 0.0, 0.0, 9.0]], np.float32)
    path, score = oracle.viterbi(oracle.HMM(log_pi, np.zeros((4, 4), np.float32)), E)
    assert path.tolist() == [3] and score == np.float32(8.0)
    # K = 1: the only path, score = sum in forward order
    E1 = np.array([[0.25], [0.5], [-1.0]], np.float32)
    path, score = oracle.viterbi(oracle.HMM(np.array([1.0], np.float32), np.array([[-0.5]], np.float32)), E1)
    assert path.tolist() == [0, 0, 0] and score == np.float32(((1.0 + 0.25) - 0.5 + 0.5) - 0.5 - 1.0)


def test_all_neg_inf_gives_zero_path(oracle):
    K, T = 3, 4
    log_pi = np.full(K, -np.inf, np.float32)
    path, score = oracle.viterbi(oracle.HMM(log_pi, np.zeros((K, K), np.float32)),
                                 np.zeros((T, K), np.float32))
    assert path.tolist() == [0] * T and score == -np.inf


def test_csr_equals_dense_with_neg_inf(oracle):
    rng = np.random.default_rng(11)
    for _ in range(10):
        K, T = int(rng.integers(2, 20)), int(rng.integers(1, 30))
        row_ptr, col, val = W.random_csr(K, min(K, 3), rng)
        logA = np.full((K, K), -np.inf, np.float32)
        for i in range(K):
            logA[i, col[row_ptr[i]:row_ptr[i + 1]]] = val[row_ptr[i]:row_ptr[i + 1]]
        log_pi = rng.standard_normal(K).astype(np.float32)
        E = rng.standard_normal((T, K)).astype(np.float32)
        pd, sd = oracle.viterbi(oracle.HMM(log_pi, logA), E)
        pc, sc = oracle.viterbi(oracle.HMM(log_pi, None, row_ptr, col, val), E)
        assert np.array_equal(pd, pc) and bits(sd) == bits(sc)


def test_discrete_emissions_gather(oracle):
    c = W.config1(T=50)
    E = oracle.expand_discrete(c["logB"], c["obs"])
    assert E.shape == (50, 64)
    assert E[7, 5] == c["logB"][5, c["obs"][7]]


# --------------------------------------------------------------------------
# FLASH (Alg. 1, Alg. 2, Sec. V-A.3, Sec. V-B.2; Theorems 1-3).

def _golden_schedules():
    out, cur = {}, None
    for line in open(os.path.join(GOLDEN, "schedule_T16.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "P":
            cur = int(line[1]); out[cur] = {"root": None, "tasks": []}
        elif line[0] == "root":
            out[cur]["root"] = [int(x) for x in line[1:]]
        else:
            out[cur]["tasks"].append(tuple(int(x) for x in line[1:]))
    return out


@pytest.mark.parametrize("P", [1, 4])
def test_flash_schedule_T16_matches_paper(oracle, P):
    g = _golden_schedules()[P]
    assert oracle.split_points(16, P) == g["root"]
    log_pi, logA, E = W.random_small(3, 16, seed=5)
    _, _, tasks = oracle.flash(oracle.HMM(log_pi, logA), E, P)
    assert [tuple(x) for x in tasks.tolist()] == g["tasks"]


def _levels(T, P, tasks, oracle):
    """Level of every task: root segments are level 1; a task's level is one
    more than that of the smallest earlier task containing it."""
    lv = []
    for k, (m, n, _) in enumerate(tasks):
        parents = [(tasks[p][1] - tasks[p][0], lv[p]) for p in range(k)
                   if tasks[p][0] <= m and n <= tasks[p][1] and (tasks[p][0], tasks[p][1]) != (m, n)]
        lv.append(1 if not parents else min(parents)[1] + 1)
    return lv


def test_flash_cycle_model_sec_VA4(oracle):
    """Sec. V-A.4: sequential binary D&C takes log T cycles (4 at T=16);
    P=4 takes 1 + (log T - log P)/P = 1.5 cycles.  A cycle is the full
    decoding time of the length-T sequence; a level of tasks costs its total
    segment length divided by the P threads."""
    log_pi, logA, E = W.random_small(2, 16, seed=1)
    for P, want in ((1, 4.0), (4, 1.5)):
        _, _, tasks = oracle.flash(oracle.HMM(log_pi, logA), E, P)
        tasks = [tuple(t) for t in tasks.tolist()]
        lv = _levels(16, P, tasks, oracle)
        threads = 1 if P == 1 else P
        cyc = 1.0
        for L in sorted(set(lv)):
            work = sum(n - m + 1 for (m, n, _), l in zip(tasks, lv) if l == L)
            cyc += work / (threads * 16)
        assert cyc == pytest.approx(want)


def test_flash_segment_of_three_enqueues_one_child(oracle):
    """Sec. V-A.3: when a segment has length 3 the right child shares its
    parent's midpoint, so only the left child is enqueued."""
    log_pi, logA, E = W.random_small(2, 12, seed=2)
    _, _, tasks = oracle.flash(oracle.HMM(log_pi, logA), E, 4)
    assert oracle.split_points(12, 4) == [2, 5, 8, 11]
    assert [tuple(t) for t in tasks.tolist()] == [
        (0, 2, 1), (3, 5, 4), (6, 8, 7), (9, 11, 10), (0, 1, 0), (3, 4, 3), (6, 7, 6), (9, 10, 9)]


@pytest.mark.parametrize("T", [1, 2, 3, 5, 7, 13, 16, 31, 64, 97])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 7, 16, 200])
def test_flash_equals_vanilla_and_reveals_each_t_once(oracle, T, P):
    """Theorem 2 with the retained offset: bit-identical to vanilla.
    TotalTask = T - P' + 1 (Alg. 1) and every t is revealed exactly once."""
    K = 5
    log_pi, logA, E = W.random_small(K, T, seed=T * 1000 + P)
    hmm = oracle.HMM(log_pi, logA)
    pv, sv = oracle.viterbi(hmm, E)
    pf, sf, tasks = oracle.flash(hmm, E, P)
    assert np.array_equal(pv, pf)
    assert bits(sv) == bits(sf)
    root = oracle.split_points(T, P)
    Pe = len(root)
    assert Pe == (1 if T == 1 else min(max(P, 2), T))
    assert len(tasks) + 1 == T - Pe + 1
    revealed = root + [int(t) for t in tasks[:, 2]] if len(tasks) else list(root)
    assert sorted(revealed) == list(range(T))


def test_flash_equals_vanilla_random_sizes(oracle):
    rng = np.random.default_rng(3)
    for _ in range(60):
        K, T, P = int(rng.integers(1, 40)), int(rng.integers(1, 300)), int(rng.integers(1, 70))
        log_pi, logA = W.random_model(K, rng)
        E = W.gaussian_emissions(T, K, rng)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        pf, sf, _ = oracle.flash(hmm, E, P)
        assert np.array_equal(pv, pf) and bits(sv) == bits(sf)


def test_flash_integer_ties_and_neg_inf(oracle):
    for seed in range(40):
        log_pi, logA, E = W.random_small(4, 23, seed=seed, integer=True, lo=-1, hi=1,
                                         neg_inf_frac=0.3 if seed % 2 else 0.0)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        for P in (1, 3, 8):
            pf, sf, _ = oracle.flash(hmm, E, P)
            assert np.array_equal(pv, pf) and bits(sv) == bits(sf)


def test_flash_complete_pruning_theorem3(oracle):
    """Complete pruning (offset 0) gives the same path in exact arithmetic
    (integer data); with generic floats the path may differ only by a
    near-tie, so its float64 score equals the optimum to rounding."""
    for seed in range(20):
        log_pi, logA, E = W.random_small(4, 19, seed=seed, integer=True, lo=-3, hi=3)
        hmm = oracle.HMM(log_pi, logA)
        pv, _ = oracle.viterbi(hmm, E)
        pc, _, _ = oracle.flash(hmm, E, 3, complete=True)
        assert np.array_equal(pv, pc)
    rng = np.random.default_rng(4)
    for _ in range(10):
        log_pi, logA = W.random_model(16, rng)
        E = W.gaussian_emissions(200, 16, rng)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        pc, _, _ = oracle.flash(hmm, E, 4, complete=True)
        f64 = lambda p: float(log_pi[p[0]]) + sum(float(logA[p[t - 1], p[t]]) for t in range(1, len(p))) + float(E[np.arange(len(p)), p].astype(np.float64).sum())
        assert abs(f64(pc) - f64(pv)) <= 1e-3


@pytest.mark.parametrize("K,T", [(2, 8), (3, 6), (4, 5), (4, 8)])
@pytest.mark.parametrize("budget", [1, 2, 3, 100])
def test_flash_budget_leaves_match_brute_force(oracle, K, T, budget):
    """Leaves (segment backpointers + backtrack from the known q_n) keep
    the exact optimum: the path's score is the brute-force maximum and the
    path is the vanilla one (lowest-index rule)."""
    for seed in range(4):
        log_pi, logA, E = W.random_small(K, T, seed=seed + 31 * K + T)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        _, scores = brute_scores(log_pi, logA, E)
        for P in (1, 2, 3):
            pb, sb, _, _ = oracle.flash_budget(hmm, E, P, budget)
            idx = int(np.ravel_multi_index(tuple(int(q) for q in pb), (K,) * T))
            assert scores[idx] == scores.max()
            assert np.array_equal(pb, pv) and bits(sb) == bits(sv)


@pytest.mark.parametrize("T,P", [(16, 4), (31, 3), (97, 7), (200, 16)])
def test_flash_budget_task_accounting(oracle, T, P):
    """Budget 0 is the pure divide-and-conquer (T - P' subtasks, no leaf).
    A budget as large as any segment turns every first-level segment of
    length >= 2 into a leaf and leaves no subtask.  In between, every
    revealed state is still revealed exactly once (subtasks reveal one
    midpoint each, a leaf of n - m rows reveals n - m states)."""
    K = 4
    log_pi, logA, E = W.random_small(K, T, seed=T + P)
    hmm = oracle.HMM(log_pi, logA)
    root = oracle.split_points(T, P)
    Pe = len(root)
    segs = [(0 if k == 0 else root[k - 1] + 1, root[k]) for k in range(Pe)]
    segs = [(m, n) for m, n in segs if n - m >= 1]
    _, _, n0, l0 = oracle.flash_budget(hmm, E, P, 0)
    assert (n0, l0) == (T - Pe, 0)
    _, _, n1, l1 = oracle.flash_budget(hmm, E, P, T)
    assert (n1, l1) == (0, len(segs))
    pv, sv = oracle.viterbi(hmm, E)
    for budget in (1, 2, 3, 5, 9):
        pb, sb, nt, nl = oracle.flash_budget(hmm, E, P, budget)
        assert np.array_equal(pb, pv) and bits(sb) == bits(sv)
        assert nt + nl >= len(segs) and nt <= T - Pe


def test_flash_budget_integer_ties_neg_inf_and_complete(oracle):
    for seed in range(30):
        log_pi, logA, E = W.random_small(4, 29, seed=seed + 500, integer=True, lo=-1, hi=1,
                                         neg_inf_frac=0.3 if seed % 2 else 0.0)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        for P, budget in ((1, 1), (3, 2), (4, 4), (8, 40)):
            pb, sb, _, _ = oracle.flash_budget(hmm, E, P, budget)
            assert np.array_equal(pv, pb) and bits(sv) == bits(sb)
        # complete pruning with integer data: exact arithmetic, same path
        pc, _, _, _ = oracle.flash_budget(hmm, E, 3, 2, complete=True)
        if not np.isinf(sv):
            assert np.array_equal(pv, pc)


# --------------------------------------------------------------------------
# Beam and FLASH-BS (Sec. V-C).

def greedy_from(v, q, logA, E, t0, t1):
    """Textbook greedy decoding (what a beam of width 1 is), carrying the
    running FP32 score v from state q at t0-1 through t0..t1 in forward
    order.  Returns (states, scores)."""
    states, scores = [], []
    for t in range(t0, t1 + 1):
        c = ((np.float32(v) + logA[q]).astype(np.float32) + E[t]).astype(np.float32)
        q = int(np.argmax(c))
        v = c[q]
        states.append(q)
        scores.append(v)
    return states, scores


def greedy_path(log_pi, logA, E):
    c = (log_pi + E[0]).astype(np.float32)
    q = int(np.argmax(c))
    st, sc = greedy_from(c[q], q, logA, E, 1, E.shape[0] - 1)
    return [q] + st, [c[q]] + sc


def test_beam_width_one_is_greedy(oracle):
    rng = np.random.default_rng(12)
    for _ in range(20):
        K, T = int(rng.integers(2, 30)), int(rng.integers(1, 60))
        log_pi, logA = W.random_model(K, rng)
        E = W.gaussian_emissions(T, K, rng)
        path, score, rc = oracle.beam(oracle.HMM(log_pi, logA), E, 1)
        assert rc == 0
        assert path.tolist() == greedy_path(log_pi, logA, E)[0]


def test_beam_full_width_equals_vanilla(oracle):
    rng = np.random.default_rng(13)
    for _ in range(20):
        K, T = int(rng.integers(1, 30)), int(rng.integers(1, 80))
        log_pi, logA = W.random_model(K, rng)
        E = W.gaussian_emissions(T, K, rng)
        hmm = oracle.HMM(log_pi, logA)
        pv, sv = oracle.viterbi(hmm, E)
        for B in (K, K + 3):
            pb, sb, rc = oracle.beam(hmm, E, B)
            assert rc == 0 and np.array_equal(pv, pb) and bits(sv) == bits(sb)
            for P in (1, 2, 5):
                pf, sf, reruns, rc = oracle.flash_bs(hmm, E, P, B)
                assert rc == 0 and reruns == 0
                assert np.array_equal(pv, pf) and bits(sv) == bits(sf)


def test_beam_full_width_csr_equals_exact_csr(oracle):
    rng = np.random.default_rng(14)
    for _ in range(10):
        K, T = int(rng.integers(4, 40)), int(rng.integers(1, 60))
        row_ptr, col, val = W.random_csr(K, 3, rng)
        log_pi = rng.standard_normal(K).astype(np.float32)
        E = rng.standard_normal((T, K)).astype(np.float32)
        hmm = oracle.HMM(log_pi, None, row_ptr, col, val)
        pv, sv = oracle.viterbi(hmm, E)
        if not np.isfinite(sv):
            continue
        pb, sb, rc = oracle.beam(hmm, E, K)
        assert rc == 0 and np.array_equal(pv, pb) and bits(sv) == bits(sb)


def test_beam_scores_are_path_scores_and_bounded(oracle):
    rng = np.random.default_rng(15)
    for _ in range(20):
        K, T = int(rng.integers(8, 64)), int(rng.integers(2, 200))
        log_pi, logA = W.random_model(K, rng)
        E = W.gaussian_emissions(T, K, rng)
        hmm = oracle.HMM(log_pi, logA)
        _, sv = oracle.viterbi(hmm, E)
        for B in (1, 2, 5):
            pb, sb, _ = oracle.beam(hmm, E, B)
            assert bits(oracle.path_score(hmm, E, pb)) == bits(sb)
            assert sb <= sv
            pf, sf, _, _ = oracle.flash_bs(hmm, E, 3, B)
            assert bits(oracle.path_score(hmm, E, pf)) == bits(sf)
            assert sf <= sv


def flash_bs_width_one(log_pi, logA, E, P, split_points):
    """FLASH-BS with B = 1 written from its definition: the root is greedy
    decoding of the whole sequence; every subtask (m,n) runs greedy decoding
    from (q_{m-1}, s_{m-1}) (from pi when m = 0) and reveals the greedy
    state and score at t_mid (Alg. 1 schedule)."""
    T = E.shape[0]
    g, gs = greedy_path(log_pi, logA, E)
    path, sval = [None] * T, [None] * T
    e = split_points
    for t in e:
        path[t], sval[t] = g[t], gs[t]
    queue = []
    for k, n in enumerate(e):
        m = 0 if k == 0 else e[k - 1] + 1
        if n - m >= 1:
            queue.append((m, n))
    while queue:
        m, n = queue.pop(0)
        tm = (m + n) // 2
        if m == 0:
            st, sc = greedy_path(log_pi, logA, E[: tm + 1])
        else:
            st, sc = greedy_from(sval[m - 1], path[m - 1], logA, E, m, tm)
            st, sc = [None] * m + st, [None] * m + sc
        path[tm], sval[tm] = st[tm], sc[tm]
        if n - m > 2:
            queue += [(m, tm), (tm + 1, n)]
        elif n - m == 2:
            queue.append((m, tm))
    return path


def test_flash_bs_width_one_reduces_to_greedy_segments(oracle):
    rng = np.random.default_rng(16)
    for _ in range(20):
        K, T, P = int(rng.integers(2, 20)), int(rng.integers(1, 50)), int(rng.integers(1, 6))
        log_pi, logA = W.random_model(K, rng)
        E = W.gaussian_emissions(T, K, rng)
        pf, _, _, rc = oracle.flash_bs(oracle.HMM(log_pi, logA), E, P, 1)
        assert rc == 0
        assert pf.tolist() == flash_bs_width_one(log_pi, logA, E, P, oracle.split_points(T, P))


# --------------------------------------------------------------------------
# Gradient (path counts).

def test_grad_sums_and_counts(oracle):
    rng = np.random.default_rng(21)
    K = 6
    T = np.array([1, 5, 9, 2], np.int32)
    paths = rng.integers(0, K, int(T.sum())).astype(np.int32)
    dpi, dA, dE = oracle.grad(K, T, paths, np.ones(4, np.float32))
    assert dpi.sum() == 4 and dA.sum() == (T - 1).sum() and dE.sum() == T.sum()
    off = 0
    cnt = np.zeros((K, K))
    for b, Tb in enumerate(T):
        q = paths[off:off + Tb]
        for t in range(1, Tb):
            cnt[q[t - 1], q[t]] += 1
        off += Tb
    assert np.array_equal(dA, cnt.astype(np.float32))


def test_grad_matches_float64_finite_differences(oracle):
    """Generic position: the optimal path is locally constant, so the
    derivative of the float64 max-score is the path count."""
    rng = np.random.default_rng(22)
    K, n = 5, 3
    T = np.array([7, 4, 10], np.int32)
    logA = rng.standard_normal((K, K)).astype(np.float32)
    log_pi = rng.standard_normal(K).astype(np.float32)
    Es = [rng.standard_normal((t, K)).astype(np.float32) for t in T]
    g = rng.standard_normal(n).astype(np.float32)
    hmm = oracle.HMM(log_pi, logA)
    paths = np.concatenate([oracle.viterbi(hmm, E)[0] for E in Es])
    dpi, dA, dE = oracle.grad(K, T, paths, g)

    def L(lp, A, Es_):
        return sum(float(g[b]) * viterbi_f64(lp, A, Es_[b]) for b in range(n))

    h = 1e-6
    A64 = logA.astype(np.float64)
    for i in range(K):
        for j in range(K):
            Ap, Am = A64.copy(), A64.copy()
            Ap[i, j] += h; Am[i, j] -= h
            fd = (L(log_pi, Ap, Es) - L(log_pi, Am, Es)) / (2 * h)
            assert abs(fd - dA[i, j]) < 1e-5
    lp64 = log_pi.astype(np.float64)
    for j in range(K):
        pp, pm = lp64.copy(), lp64.copy()
        pp[j] += h; pm[j] -= h
        assert abs((L(pp, A64, Es) - L(pm, A64, Es)) / (2 * h) - dpi[j]) < 1e-5
    # one emission entry per sequence
    off = 0
    for b in range(n):
        t, j = int(T[b] // 2), int(rng.integers(0, K))
        Ep = [E.astype(np.float64) for E in Es]; Em = [E.astype(np.float64) for E in Es]
        Ep[b][t, j] += h; Em[b][t, j] -= h
        fd = (L(lp64, A64, Ep) - L(lp64, A64, Em)) / (2 * h)
        assert abs(fd - dE[off + t * K + j]) < 1e-5
        off += int(T[b]) * K


# --------------------------------------------------------------------------
# Checkpoint Viterbi (the sqrt(T)-checkpoint baseline of Sec. II-A).

@pytest.mark.parametrize("K,T", [(2, 8), (3, 6), (4, 5), (4, 8), (1, 7), (3, 1)])
def test_checkpoint_matches_brute_force(oracle, K, T):
    """Score = the brute-force maximum bit for bit; on integer data the
    path is the optimal one whose reversed sequence is smallest (the same
    tie rule as the full table)."""
    for seed in range(4):
        for integer in (False, True):
            log_pi, logA, E = W.random_small(K, T, seed=31 * seed + K, integer=integer, lo=-2, hi=2)
            hmm = oracle.HMM(log_pi, logA)
            paths, s = brute_scores(log_pi, logA, E)
            for P in (0, 1, 2, 3, T):
                path, score, _, _ = oracle.checkpoint(hmm, E, P)
                assert bits(score) == bits(s.max())
                match = np.all(paths == path[None, :], axis=1)
                assert bits(s[match][0]) == bits(score)
                if integer:
                    assert np.array_equal(path, lex_min_reversed(paths[s == s.max()]))


def test_checkpoint_equals_full_table_and_memory_bound(oracle):
    """Restarting each segment from the exact stored delta reproduces every
    backpointer of the full table, so the path and score are the full
    table's for any checkpoint count (prime T, T below P, ties, -inf).
    Memory: ceil(sqrt(T)) checkpoints by default and segments of at most
    ceil(T/P') backpointer rows."""
    import math
    rng = np.random.default_rng(11)
    for T in (1, 2, 3, 5, 16, 17, 31, 64, 97, 100, 257):
        for trial in range(2):
            K = int(rng.integers(1, 7))
            log_pi, logA, E = W.random_small(K, T, seed=int(rng.integers(1 << 30)), integer=bool(trial),
                                             lo=-3, hi=3, neg_inf_frac=0.2)
            hmm = oracle.HMM(log_pi, logA)
            pv, sv = oracle.viterbi(hmm, E)
            for P in (0, 1, 2, 3, 7, T, T + 5):
                path, score, nc, rows = oracle.checkpoint(hmm, E, P)
                assert np.array_equal(path, pv), (T, P)
                assert bits(score) == bits(sv)
                want = (1 if T == 1 else min(T, math.isqrt(T - 1) + 1)) if P <= 0 else min(P, T)
                assert nc == want == oracle.checkpoint_count(T, P)
                assert rows <= -(-T // nc)
