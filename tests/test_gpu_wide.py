"""Whole-GPU configuration of the exact decoder (1024 < K <= 4096): every
max-plus step is spread over all clusters of one cooperative launch, up to 8
jobs advancing in lockstep.  Paths and scores must match the oracle exactly
for vanilla and FLASH (root pass, resolve and every task level), including
launches with more jobs than lanes, ties and -inf transitions."""
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


def check(fv, log_pi, logA, E_list, modes):
    lengths = [e.shape[0] for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    res = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    for mode, kw in modes:
        paths, scores = fv.decode([m], b, mode=mode, **kw)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (p, s) in enumerate(res):
            T = lengths[i]
            assert np.array_equal(paths[off:off + T], p), f"{mode} {kw} seq {i} T={T}"
            assert bits(scores[i]) == bits(s), f"{mode} {kw} seq {i}: {scores[i]} vs {s}"
            off += T


@pytest.mark.parametrize("K,tmax,n", [(1025, 90, 11), (2048, 50, 10), (3000, 30, 9), (4096, 22, 10)])
def test_wide_vanilla_and_flash(fv, K, tmax, n):
    rng = np.random.default_rng(K + 1)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3] + list(rng.integers(1, tmax, n - 3))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    check(fv, log_pi, logA, E_list, [("vanilla", {}), ("flash", {"P": 1}), ("flash", {"P": 4})])


def test_wide_ties_and_neg_inf(fv):
    rng = np.random.default_rng(9)
    K = 2100
    log_pi = rng.integers(-1, 2, K).astype(np.float32)
    logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
    logA[rng.random((K, K)) < 0.4] = -np.inf
    E_list = [rng.integers(-1, 2, (int(t), K)).astype(np.float32) for t in rng.integers(1, 40, 9)]
    check(fv, log_pi, logA, E_list, [("vanilla", {}), ("flash", {"P": 2})])


def test_wide_unreachable_states(fv):
    """Rows of -inf (states nobody can leave) and a start restricted to a few
    states: many targets see only -inf candidates."""
    rng = np.random.default_rng(10)
    K = 1500
    log_pi = np.full(K, -np.inf, np.float32)
    log_pi[rng.choice(K, 5, replace=False)] = 0.0
    logA = rng.standard_normal((K, K)).astype(np.float32)
    logA[rng.random(K) < 0.5, :] = -np.inf
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in (1, 7, 30)]
    check(fv, log_pi, logA, E_list, [("vanilla", {}), ("flash", {"P": 3})])
