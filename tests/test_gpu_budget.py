"""FLASH with a backpointer budget (budget leaves): the first task level
whose tasks' backpointer rows fit the budget is solved directly, in waves,
with segment backpointers and a backtrack from the known q_n.  Paths and
scores must equal the oracle's (which equal vanilla Viterbi bit for bit)
for every budget, P and engine (resident, streamed and whole-GPU)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    import paper_2510_19301_gb300 as fv
    fv._lib.load(build_if_missing=True)
    return fv


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


def run(fv, K, lengths, Ps, budgets_rows, seed, ties=False):
    rng = np.random.default_rng(seed)
    if ties:
        log_pi = rng.integers(-1, 2, K).astype(np.float32)
        logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
        logA[rng.random((K, K)) < 0.3] = -np.inf
        E_list = [rng.integers(-1, 2, (int(t), K)).astype(np.float32) for t in lengths]
    else:
        log_pi, logA = W.random_model(K, rng)
        E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    for P in Ps:
        for rows in budgets_rows:
            budget = int(rows) * K * 2
            paths, scores = fv.decode([m], b, mode="flash", P=P, mem_budget=budget)
            paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
            off = 0
            for i, (p, s) in enumerate(ref):
                T = lengths[i]
                assert np.array_equal(paths[off:off + T], p), f"K={K} P={P} budget rows={rows} seq {i} T={T}"
                assert bits(scores[i]) == bits(s), f"K={K} P={P} budget rows={rows} seq {i}"
                off += T


def test_budget_resident_engine(fv):
    rng = np.random.default_rng(1)
    lengths = [1, 2, 3, 4, 17] + list(rng.integers(1, 400, 15))
    total = int(np.sum(lengths))
    run(fv, 256, lengths, (1, 4, 16), (1, 2, 7, 64, total // 16, 10 ** 6), seed=2)


def test_budget_streamed_engine(fv):
    rng = np.random.default_rng(3)
    lengths = [1, 2, 5] + list(rng.integers(1, 200, 9))
    run(fv, 512, lengths, (2, 8), (1, 9, 100), seed=4)


def test_budget_whole_gpu_engine(fv):
    rng = np.random.default_rng(5)
    lengths = [1, 2, 3] + list(rng.integers(1, 40, 8))
    run(fv, 2048, lengths, (1, 4), (1, 3, 1000), seed=6)


def test_budget_integer_ties(fv):
    rng = np.random.default_rng(7)
    lengths = list(rng.integers(1, 120, 12))
    run(fv, 64, lengths, (3,), (1, 4, 33), seed=8, ties=True)
