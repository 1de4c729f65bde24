"""Property-based checks of the oracle (hypothesis, CPU): for random small
models the exact decoder reaches the brute-force optimum, and every
exact variant of the paper's method (FLASH for any P, with or without a
backpointer budget; the beam with every state kept) returns the same path
and score bit for bit; the returned score is the path's own
forward-order log-likelihood."""
import itertools

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402


def model_strategy(max_k=4, max_t=6, integer=False):
    @st.composite
    def draw(d):
        K = d(st.integers(1, max_k))
        T = d(st.integers(1, max_t))
        seed = d(st.integers(0, 2 ** 31 - 1))
        rng = np.random.default_rng(seed)
        if integer:
            lp = rng.integers(-2, 3, K).astype(np.float32)
            A = rng.integers(-2, 3, (K, K)).astype(np.float32)
            E = rng.integers(-2, 3, (T, K)).astype(np.float32)
        else:
            lp = rng.standard_normal(K).astype(np.float32)
            A = rng.standard_normal((K, K)).astype(np.float32)
            E = rng.standard_normal((T, K)).astype(np.float32)
        if d(st.booleans()):
            A[rng.random((K, K)) < 0.3] = -np.inf
        return lp, A, E
    return draw()


def brute_best(lp, A, E):
    T, K = E.shape
    best = -np.inf
    for q in itertools.product(range(K), repeat=T):
        s = np.float32(lp[q[0]] + E[0, q[0]])
        for t in range(1, T):
            s = np.float32(np.float32(s + A[q[t - 1], q[t]]) + E[t, q[t]])
        best = max(best, float(s))
    return best


def bits(x):
    return np.float32(x).view(np.int32)


@settings(max_examples=150, deadline=None)
@given(model_strategy(), st.integers(1, 8), st.integers(0, 6))
def test_exact_variants_agree(case, P, budget):
    lp, A, E = case
    hmm = oracle.HMM(lp, A)
    pv, sv = oracle.viterbi(hmm, E)
    assert float(sv) == brute_best(lp, A, E)
    pf, sf, _ = oracle.flash(hmm, E, P)
    pb, sb, _, _ = oracle.flash_budget(hmm, E, P, budget)
    assert np.array_equal(pv, pf) and bits(sv) == bits(sf)
    assert np.array_equal(pv, pb) and bits(sv) == bits(sb)
    if np.isfinite(sv):
        assert bits(oracle.path_score(hmm, E, pv)) == bits(sv)
        pw, sw, rc = oracle.beam(hmm, E, lp.shape[0])
        assert rc == 0 and np.array_equal(pv, pw) and bits(sv) == bits(sw)


@settings(max_examples=100, deadline=None)
@given(model_strategy(max_k=5, max_t=9, integer=True), st.integers(1, 9))
def test_integer_ties_flash_equals_vanilla(case, P):
    lp, A, E = case
    hmm = oracle.HMM(lp, A)
    pv, sv = oracle.viterbi(hmm, E)
    pf, sf, _ = oracle.flash(hmm, E, P)
    assert np.array_equal(pv, pf) and bits(sv) == bits(sf)


def beam_restated(lp, A, E, B):
    """The dynamic beam of Sec. V-C written out in Python: each step keeps
    the top-B finite candidates under (score desc, state id asc); a target's
    candidate comes from its best beam source (lowest id on equal scores),
    and the final state is the best entry (highest score, lowest id)."""
    T, K = E.shape
    f32 = np.float32
    c0 = [f32(lp[j] + E[0, j]) for j in range(K)]

    def top(c):
        fin = [j for j in range(K) if np.isfinite(c[j])]
        fin.sort(key=lambda j: (-float(c[j]), j))
        return sorted(fin[:B])

    beam = top(c0)
    vals = {j: c0[j] for j in beam}
    back = []
    for t in range(1, T):
        if not beam:
            return None
        c, src = [f32(-np.inf)] * K, [None] * K
        for j in range(K):
            best, arg = None, None
            for i in beam:  # ascending id
                x = f32(vals[i] + A[i, j])
                if best is None or x > best:
                    best, arg = x, i
            c[j] = f32(best + E[t, j])
            src[j] = arg
        beam = top(c)
        vals = {j: c[j] for j in beam}
        back.append({j: src[j] for j in beam})
    if not beam:
        return None
    q = min(beam, key=lambda j: (-float(vals[j]), j))
    score = vals[q]
    path = [q]
    for bp in reversed(back):
        q = bp[q]
        path.append(q)
    return np.array(path[::-1], np.int32), score


@settings(max_examples=150, deadline=None)
@given(model_strategy(max_k=6, max_t=7), st.integers(1, 6))
def test_beam_matches_restatement(case, B):
    lp, A, E = case
    K = lp.shape[0]
    B = min(B, K)
    hmm = oracle.HMM(lp, A)
    ref = beam_restated(lp, A, E, B)
    p, s, rc = oracle.beam(hmm, E, B)
    if ref is None:
        assert rc == 6
        return
    assert rc == 0 and np.array_equal(p, ref[0]) and bits(s) == bits(ref[1])


@settings(max_examples=100, deadline=None)
@given(model_strategy(max_k=5, max_t=9), st.integers(1, 9))
def test_full_width_flash_bs_equals_vanilla(case, P):
    lp, A, E = case
    hmm = oracle.HMM(lp, A)
    pv, sv = oracle.viterbi(hmm, E)
    if not np.isfinite(sv):
        return
    pf, sf, _, rc = oracle.flash_bs(hmm, E, P, lp.shape[0])
    assert rc == 0 and np.array_equal(pv, pf) and bits(sv) == bits(sf)


@st.composite
def csr_case(d, max_k=6, max_t=7):
    K = d(st.integers(1, max_k))
    T = d(st.integers(1, max_t))
    rng = np.random.default_rng(d(st.integers(0, 2 ** 31 - 1)))
    lp = rng.standard_normal(K).astype(np.float32)
    E = rng.standard_normal((T, K)).astype(np.float32)
    row_ptr, col, val = [0], [], []
    dense = np.full((K, K), -np.inf, np.float32)
    for i in range(K):
        succ = sorted(rng.choice(K, size=int(rng.integers(1, K + 1)), replace=False))
        w = rng.standard_normal(len(succ)).astype(np.float32)
        col += [int(j) for j in succ]
        val += [float(x) for x in w]
        dense[i, succ] = w
        row_ptr.append(len(col))
    return lp, E, np.array(row_ptr, np.int32), np.array(col, np.int32), np.array(val, np.float32), dense


@settings(max_examples=100, deadline=None)
@given(csr_case(), st.integers(1, 6))
def test_csr_beam_matches_restatement_on_dense_equivalent(case, B):
    lp, E, rp, col, val, dense = case
    K = lp.shape[0]
    B = min(B, K)
    csr = oracle.HMM(lp, row_ptr=rp, col=col, val=val)
    pv, sv = oracle.viterbi(csr, E)
    pd, sd = oracle.viterbi(oracle.HMM(lp, dense), E)
    assert np.array_equal(pv, pd) and bits(sv) == bits(sd)
    ref = beam_restated(lp, dense, E, B)
    p, s, rc = oracle.beam(csr, E, B)
    if ref is None:
        assert rc == 6
        return
    assert rc == 0 and np.array_equal(p, ref[0]) and bits(s) == bits(ref[1])


@settings(max_examples=150, deadline=None)
@given(model_strategy(max_k=6, max_t=7), st.integers(1, 7))
def test_static_beam_matches_restatement_and_dynamic(case, B):
    """The static beam (all K scores of a step, then the top B) against the
    Python restatement of the beam (which sorts every candidate) and the
    oracle's dynamic beam: same paths and score bits, same infeasibility.
    With B >= K it is exact decoding."""
    lp, A, E = case
    K = lp.shape[0]
    hmm = oracle.HMM(lp, A)
    Bc = min(B, K)
    ref = beam_restated(lp, A, E, Bc)
    p, s, rc = oracle.beam_static(hmm, E, B)
    pd, sd, rcd = oracle.beam(hmm, E, B)
    assert rc == rcd
    if ref is None:
        assert rc == 6
        return
    assert rc == 0 and np.array_equal(p, ref[0]) and bits(s) == bits(ref[1])
    assert np.array_equal(p, pd) and bits(s) == bits(sd)
    if B >= K:
        pv, sv = oracle.viterbi(hmm, E)
        assert np.array_equal(p, pv) and bits(s) == bits(sv)


@settings(max_examples=80, deadline=None)
@given(csr_case(), st.integers(1, 6))
def test_static_beam_csr_matches_restatement(case, B):
    lp, E, rp, col, val, dense = case
    K = lp.shape[0]
    csr = oracle.HMM(lp, row_ptr=rp, col=col, val=val)
    ref = beam_restated(lp, dense, E, min(B, K))
    p, s, rc = oracle.beam_static(csr, E, B)
    if ref is None:
        assert rc == 6
        return
    assert rc == 0 and np.array_equal(p, ref[0]) and bits(s) == bits(ref[1])
