"""GPU parity of FLASH Viterbi (root pass with P-way division maps, resolve,
level-by-level subtasks with the retained-offset pruned start) against the
oracle's Alg. 1 / Alg. 2: identical paths and 0-ulp scores.  At full size
the FLASH result must also equal the GPU exact decoder on every sequence."""
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


def check_flash(fv, log_pi, logA, E_list, P, complete=False):
    K = log_pi.shape[0]
    lengths = [e.shape[0] for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    flags = fv._lib.FV_COMPLETE_PRUNING if complete else 0
    paths, scores = fv.decode([m], b, mode="flash", P=P, flags=flags)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    res = oracle.map_sequences(lambda e: oracle.flash(hmm, e, P, complete=complete), E_list)
    off = 0
    for i, (p, s, _) in enumerate(res):
        T = lengths[i]
        assert np.array_equal(paths[off:off + T], p), f"seq {i} T={T} P={P}"
        if not complete:
            assert bits(scores[i]) == bits(s), f"seq {i} score"
        off += T


@pytest.mark.parametrize("P", [1, 2, 3, 4, 7, 16, 64, 5000])
@pytest.mark.parametrize("K", [5, 64, 200])
def test_flash_random(fv, K, P):
    rng = np.random.default_rng(K * 131 + P)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 4, 5, 13, 16, 31, 97, 128, 257] + list(rng.integers(1, 500, 12))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    check_flash(fv, log_pi, logA, E_list, P)


@pytest.mark.parametrize("K", [3, 40, 129])
def test_flash_ties_and_neg_inf(fv, K):
    rng = np.random.default_rng(7 + K)
    for frac in (0.0, 0.5):
        log_pi = rng.integers(-1, 2, K).astype(np.float32)
        logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
        logA[rng.random((K, K)) < frac] = -np.inf
        E_list = [rng.integers(-1, 2, (int(t), K)).astype(np.float32) for t in rng.integers(1, 90, 16)]
        for P in (1, 4):
            check_flash(fv, log_pi, logA, E_list, P)


def test_flash_complete_pruning_matches_oracle(fv):
    rng = np.random.default_rng(11)
    K = 48
    log_pi, logA = W.random_model(K, rng)
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in rng.integers(2, 300, 20)]
    check_flash(fv, log_pi, logA, E_list, 4, complete=True)


def test_flash_discrete_emissions(fv):
    c = W.config1()
    m = fv.Model(c["log_pi"], c["logA"], logB=c["logB"])
    b = fv.Batch([c["T"]], obs=c["obs"], models=[m])
    E = oracle.expand_discrete(c["logB"], c["obs"])
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    for P in (1, 16):
        paths, scores = fv.decode([m], b, mode="flash", P=P)
        p, s, _ = oracle.flash(hmm, E, P)
        assert np.array_equal(paths.cpu().numpy(), p)
        assert bits(scores.cpu().numpy()[0]) == bits(s)


def test_flash_multiple_models(fv):
    rng = np.random.default_rng(5)
    Ks = [64, 200, 17]
    models_np = [W.random_model(K, rng) for K in Ks]
    mi = rng.integers(0, 3, 24)
    lengths = rng.integers(1, 200, 24)
    E_list = [W.gaussian_emissions(int(t), Ks[m], rng) for t, m in zip(lengths, mi)]
    models = [fv.Model(lp, A) for lp, A in models_np]
    E = torch.from_numpy(np.concatenate([e.reshape(-1) for e in E_list])).cuda()
    b = fv.Batch(lengths, E=E, model_index=mi, models=models)
    paths, scores = fv.decode(models, b, mode="flash", P=8)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    off = 0
    for i in range(24):
        p, s = oracle.viterbi(oracle.HMM(*models_np[mi[i]]), E_list[i])
        assert np.array_equal(paths[off:off + lengths[i]], p)
        assert bits(scores[i]) == bits(s)
        off += lengths[i]


@pytest.mark.parametrize("P", [4, 16, 64])
def test_flash_config2_full_size_equals_vanilla(fv, P):
    """Benchmark workload: FLASH == the GPU exact decoder on all 1024
    sequences, and == the oracle on a sample."""
    K = 256
    log_pi, logA = W.config2_model()
    lengths = W.config2_lengths()
    E = W.gaussian_emissions_packed_device(int(lengths.sum()), K, seed=2)
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E.view(-1), models=[m])
    pv, sv = [x.clone() for x in fv.decode([m], b, mode="vanilla")]
    pf, sf = fv.decode([m], b, mode="flash", P=P)
    assert torch.equal(pv, pf)
    assert torch.equal(sv.view(torch.int32), sf.view(torch.int32))
    rng = np.random.default_rng(P)
    pick = [int(np.argmax(lengths))] + list(rng.choice(len(lengths), 5, replace=False))
    e_off, p_off = W.packed_offsets(lengths, K)
    hmm = oracle.HMM(log_pi, logA)
    jobs = [E.view(-1)[e_off[i]:e_off[i] + lengths[i] * K].view(-1, K).cpu().numpy() for i in pick]
    res = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), jobs)
    P_ = pf.cpu().numpy()
    for i, (p, s) in zip(pick, res):
        assert np.array_equal(P_[p_off[i]:p_off[i] + lengths[i]], p)
