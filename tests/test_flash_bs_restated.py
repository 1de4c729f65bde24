"""Pin of the oracle's FLASH-BS for beam widths 1 < B < K.

FLASH-BS (Sec. V-C) runs Alg. 1's queue of subtasks with the dynamic beam of
Sec. V-C.2 as the step: every beam entry carries its State, its OptProb and,
per division point, the MidState of its best path (Sec. V-C.2, the three
components of a heap entry).  The functions below restate the method in
plain Python, keyed by STATE ID everywhere (dicts state -> value), so a
mix-up between a beam slot and a state id -- invisible when B = 1 (one slot)
or B = K (slot == id) -- makes the oracle disagree with them.

Readings (the same the oracle documents): the beam is the top-B finite
candidates under (score desc, id asc); a target's best source is the lowest
id among equal candidates; division points e_k = floor(((k+1)T - 1)/P') with
P' = min(max(P, 2), T); a subtask (m, n) restarts from q*_{m-1} with the
retained offset of Def. 3 (offset 0 under complete pruning); its last step
evaluates only the known end state q*_n from every beam source, and when no
source reaches q*_n the subtask is run again with every state kept (a rerun);
the returned score is the path's forward-order log-likelihood.

No code is shared with ``oracle/``: this file imports it only to compare.
"""
from collections import deque

import numpy as np
import pytest

import oracle

f32 = np.float32
NEG = f32(-np.inf)


class Restated:
    """One HMM: dense log-transitions (absent edges -inf) or CSR out-edges."""

    def __init__(self, lp, A=None, succ=None):
        self.lp = [f32(x) for x in lp]
        self.K = len(self.lp)
        self.A = A
        self.succ = succ  # CSR: succ[i] = [(j, w), ...]

    def out_edges(self, i):
        if self.A is not None:
            return [(j, f32(self.A[i][j])) for j in range(self.K)]
        return self.succ[i]

    def a(self, i, j):
        """log A_ij, -inf when the CSR graph has no edge i -> j."""
        if self.A is not None:
            return f32(self.A[i][j])
        best = NEG
        for jj, w in self.succ[i]:
            if jj == j and w > best:
                best = w
        return best


def split_points(T, P):
    Pe = 1 if T == 1 else min(max(P, 2), T)
    return [((k + 1) * T - 1) // Pe for k in range(Pe)]


def top_b(cand, B):
    """Ids of the B best finite candidates (score desc, id asc), in id order."""
    finite = [j for j, v in cand.items() if np.isfinite(v)]
    finite.sort(key=lambda j: (-float(cand[j]), j))
    return sorted(finite[:B])


def expand(hmm, beam, Et):
    """One dynamic-beam step: only transitions out of the beam's states are
    evaluated; every target reached gets its best source and the score
    fl(fl(OptProb[i] + log A_ij) + E_t[j])."""
    best, src = {}, {}
    for i in sorted(beam):
        for j, w in hmm.out_edges(i):
            c = f32(beam[i] + w)
            if j not in best or c > best[j]:
                best[j], src[j] = c, i
    return {j: f32(best[j] + Et[j]) for j in best}, src


def root(hmm, E, B, e):
    """Beam over [0, T-1]; per entry one MidState per division point before
    T-1.  Returns {t: (q*_t, delta at t)} for T-1 and every division point,
    or None when the beam empties."""
    T = len(E)
    nd = len(e) - 1
    c0 = {j: f32(hmm.lp[j] + E[0][j]) for j in range(hmm.K)}
    beam = {j: c0[j] for j in top_b(c0, B)}
    mid = {j: [None] * nd for j in beam}
    snaps = {}
    for t in range(T):
        if t > 0:
            cand, src = expand(hmm, beam, E[t])
            keep = top_b(cand, B)
            new_mid = {}
            for j in keep:
                row = []
                for k in range(nd):
                    if t == e[k] + 1:
                        row.append(src[j])
                    elif t > e[k] + 1:
                        row.append(mid[src[j]][k])
                    else:
                        row.append(None)
                new_mid[j] = row
            beam, mid = {j: cand[j] for j in keep}, new_mid
        if not beam:
            return None
        for k, ek in enumerate(e):
            if ek == t:
                snaps[k] = dict(beam)
    qT = min(beam, key=lambda j: (-float(beam[j]), j))
    known = {T - 1: (qT, beam[qT])}
    for k in range(nd):
        q = mid[qT][k]
        known[e[k]] = (q, snaps[k][q])
    return known


def subtask(hmm, E, m, n, q_prev, s_prev, q_n, B, complete):
    """Subtask (m, n) with known end state q*_n: pruned start, beam steps,
    MidState from t_mid + 1, and a last step that scores q*_n alone.
    Returns (q*_{t_mid}, delta at t_mid) or None if q*_n is unreachable."""
    tmid = (m + n) // 2
    if m == 0:
        c = {j: f32(hmm.lp[j] + E[0][j]) for j in range(hmm.K)}
    elif complete:
        c = {j: f32(hmm.a(q_prev, j) + E[m][j]) for j in range(hmm.K)}
    else:
        c = {j: f32(f32(s_prev + hmm.a(q_prev, j)) + E[m][j]) for j in range(hmm.K)}
    beam = {j: c[j] for j in top_b(c, B)}
    mid, snap, t = {}, None, m
    while True:
        if not beam:
            return None
        if t == tmid:
            snap = dict(beam)
        t += 1
        if t == n:
            best, arg = None, None
            for i in sorted(beam):
                x = f32(beam[i] + hmm.a(i, q_n))
                if best is None or x > best:
                    best, arg = x, i
            if not best > NEG:
                return None
            q = arg if t == tmid + 1 else mid[arg]
            return q, snap[q]
        cand, src = expand(hmm, beam, E[t])
        keep = top_b(cand, B)
        if t == tmid + 1:
            mid = {j: src[j] for j in keep}
        elif t > tmid + 1:
            mid = {j: mid[src[j]] for j in keep}
        beam = {j: cand[j] for j in keep}


def path_score(hmm, E, path):
    s = f32(hmm.lp[path[0]] + E[0][path[0]])
    for t in range(1, len(path)):
        s = f32(f32(s + hmm.a(path[t - 1], path[t])) + E[t][path[t]])
    return s


def flash_bs_restated(hmm, E, P, B, complete=False):
    """-> (path, score, reruns), or None when no finite path is found."""
    T = len(E)
    e = split_points(T, P)
    known = root(hmm, E, B, e)
    if known is None:
        return None
    fifo = deque()
    for k in range(len(e)):
        m, n = (0 if k == 0 else e[k - 1] + 1), e[k]
        if n - m >= 1:
            fifo.append((m, n))
    reruns = 0
    while fifo:
        m, n = fifo.popleft()
        q_prev, s_prev = known[m - 1] if m > 0 else (None, None)
        r = subtask(hmm, E, m, n, q_prev, s_prev, known[n][0], B, complete)
        if r is None:
            reruns += 1
            r = subtask(hmm, E, m, n, q_prev, s_prev, known[n][0], hmm.K, complete)
            if r is None:
                return None
        tmid = (m + n) // 2
        known[tmid] = r
        if n - m > 2:
            fifo.append((m, tmid))
            fifo.append((tmid + 1, n))
        elif n - m == 2:
            fifo.append((m, tmid))
    path = [known[t][0] for t in range(T)]
    return np.array(path, np.int32), path_score(hmm, E, path), reruns


# --------------------------------------------------------------------------
# Case generators: dense with -inf entries, integer ties, CSR.

def dense_case(rng, K, T, p_absent, integer):
    if integer:
        lp = rng.integers(-2, 3, K).astype(np.float32)
        A = rng.integers(-2, 3, (K, K)).astype(np.float32)
        E = rng.integers(-2, 3, (T, K)).astype(np.float32)
    else:
        lp = rng.standard_normal(K).astype(np.float32)
        A = rng.standard_normal((K, K)).astype(np.float32)
        E = rng.standard_normal((T, K)).astype(np.float32)
    A[rng.random((K, K)) < p_absent] = -np.inf
    return oracle.HMM(lp, A), Restated(lp, A=A), E


def csr_case(rng, K, T, max_deg):
    lp = rng.standard_normal(K).astype(np.float32)
    E = rng.standard_normal((T, K)).astype(np.float32)
    row_ptr, col, val, succ = [0], [], [], []
    for _ in range(K):
        js = sorted(int(j) for j in rng.choice(K, size=int(rng.integers(1, max_deg + 1)), replace=False))
        ws = rng.standard_normal(len(js)).astype(np.float32)
        col += js
        val += [float(w) for w in ws]
        succ.append([(j, f32(w)) for j, w in zip(js, ws)])
        row_ptr.append(len(col))
    hmm = oracle.HMM(lp, row_ptr=np.array(row_ptr, np.int32), col=np.array(col, np.int32),
                     val=np.array(val, np.float32))
    return hmm, Restated(lp, succ=succ), E


def draw_case(rng):
    """Small cases (K 3..7, T 1..13) of every kind, plus longer sparse ones
    (K 8..20, T 15..40, 2-4 out-edges, B 2..3) in which a subtask's beam often
    loses the route to q*_n, so the rerun is exercised."""
    kind = int(rng.integers(0, 5))     # 3 and 4: longer sparse cases
    if kind < 3:
        K, T = int(rng.integers(3, 8)), int(rng.integers(1, 14))
        B = int(rng.integers(2, K))          # 1 < B < K
    else:
        K, T = int(rng.integers(8, 21)), int(rng.integers(15, 41))
        B = int(rng.integers(2, 4))
    P = int(rng.integers(1, 9))
    if kind == 0:
        h, r, E = dense_case(rng, K, T, float(rng.choice([0.0, 0.3, 0.6])), integer=False)
    elif kind == 1:
        h, r, E = dense_case(rng, K, T, float(rng.choice([0.0, 0.4])), integer=True)
    elif kind == 2:
        h, r, E = csr_case(rng, K, T, max_deg=int(rng.integers(1, K)))
    else:
        h, r, E = csr_case(rng, K, T, max_deg=int(rng.integers(2, 5)))
    return h, r, E, P, B, bool(rng.integers(0, 4) == 0)


def bits(x):
    return np.float32(x).view(np.int32)


def check(h, r, E, P, B, complete):
    ref = flash_bs_restated(r, E, P, B, complete)
    p, s, reruns, rc = oracle.flash_bs(h, E, P, B, complete)
    if ref is None:
        assert rc == 6
        return None
    assert rc == 0
    assert np.array_equal(p, ref[0]), (p, ref[0])
    assert bits(s) == bits(ref[1])
    assert reruns == ref[2]
    return ref[2]


# --------------------------------------------------------------------------

def test_restatement_reduces_to_vanilla_at_full_width(oracle):
    """Sanity of the restatement itself: with B = K it is exact Viterbi
    (pinned against brute force elsewhere), so it must equal vanilla."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        K, T = int(rng.integers(2, 6)), int(rng.integers(1, 10))
        h, r, E = dense_case(rng, K, T, 0.0, integer=False)
        pv, sv = oracle.viterbi(h, E)
        path, score, reruns = flash_bs_restated(r, E, int(rng.integers(1, 6)), K)
        assert np.array_equal(path, pv) and bits(score) == bits(sv) and reruns == 0


def test_restatement_flash_bs_seeded_sweep(oracle):
    """800 seeded cases, 1 < B < K: dense (with -inf), integer ties and CSR,
    P in 1..8, retained and complete pruning.  Path, score bits and the
    rerun count must match; some cases must exercise the rerun."""
    rng = np.random.default_rng(20251019)
    n_rerun_cases = n_feasible = 0
    for _ in range(800):
        got = check(*draw_case(rng))
        if got is not None:
            n_feasible += 1
            n_rerun_cases += got > 0
    assert n_feasible >= 600
    assert n_rerun_cases >= 10


try:
    from hypothesis import given, settings, strategies as st
except ImportError:  # the seeded sweep above still runs
    given = None

if given is not None:
    @settings(max_examples=300, deadline=None)
    @given(st.integers(0, 2 ** 32 - 1))
    def test_restatement_flash_bs_hypothesis(oracle, seed):
        check(*draw_case(np.random.default_rng(seed)))
