"""Streamed-logA configurations of the exact decoder (256 < K <= 1024): the
row-pair copy of logA is read through a cp.async ring and the argmax chunks
are re-scanned from it.  Paths and scores must match the oracle exactly,
for vanilla and FLASH."""
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


@pytest.mark.parametrize("K", [257, 300, 512, 513, 777, 1024])
def test_large_k_vanilla_and_flash(fv, K):
    rng = np.random.default_rng(K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 40] + list(rng.integers(1, 160, 10))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    res = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    for mode, kw in (("vanilla", {}), ("flash", {"P": 4})):
        paths, scores = fv.decode([m], b, mode=mode, **kw)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (p, s) in enumerate(res):
            T = lengths[i]
            assert np.array_equal(paths[off:off + T], p), f"{mode} seq {i} T={T}"
            assert bits(scores[i]) == bits(s), f"{mode} seq {i}"
            off += T


def test_large_k_ties_and_neg_inf(fv):
    rng = np.random.default_rng(5)
    K = 600
    log_pi = rng.integers(-1, 2, K).astype(np.float32)
    logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
    logA[rng.random((K, K)) < 0.4] = -np.inf
    E_list = [rng.integers(-1, 2, (int(t), K)).astype(np.float32) for t in rng.integers(1, 60, 8)]
    lengths = [e.shape[0] for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    for mode in ("vanilla", "flash"):
        paths, scores = fv.decode([m], b, mode=mode, P=2)
        paths = paths.cpu().numpy()
        off = 0
        for i, e in enumerate(E_list):
            p, s = oracle.viterbi(hmm, e)
            assert np.array_equal(paths[off:off + len(e)], p)
            assert bits(scores.cpu().numpy()[i]) == bits(s)
            off += len(e)
