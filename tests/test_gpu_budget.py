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


def test_budget_discrete_emissions(fv):
    """Leaves on symbol emissions (config-1 shape: K=64, V=32)."""
    K, V = 64, 32
    rng = np.random.default_rng(11)
    log_pi, logA = W.random_model(K, rng)
    logB = W._log_dirichlet(rng, 0.5, (K, V)).astype(np.float32)
    lengths = [1, 2, 7, 150, 333, 1000]
    obs_list = [W.sample_hmm_sequence(log_pi, logA, logB, t, rng) for t in lengths]
    m = fv.Model(log_pi, logA, logB=logB)
    b = fv.Batch(lengths, obs=np.concatenate(obs_list), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    E_list = [oracle.expand_discrete(logB, o) for o in obs_list]
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    for P, rows in ((4, 16), (16, 3), (2, 10 ** 5)):
        paths, scores = fv.decode([m], b, mode="flash", P=P, mem_budget=rows * K * 2)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (p, s) in enumerate(ref):
            assert np.array_equal(paths[off:off + lengths[i]], p), f"P={P} rows={rows} seq {i}"
            assert bits(scores[i]) == bits(s)
            off += lengths[i]


@pytest.mark.parametrize("flags", [0, 2])
def test_budget_two_models_and_batch_order(fv, flags):
    """Two models (K=64 and K=256) in one batch: the leaf waves of each model
    are planned from the model-major task order (longest first, or batch
    order with FV_NO_SORT)."""
    rng = np.random.default_rng(12 + flags)
    models, hmms = [], []
    for K in (64, 256):
        log_pi, logA = W.random_model(K, rng)
        models.append(fv.Model(log_pi, logA))
        hmms.append(oracle.HMM(log_pi, logA))
    midx = rng.integers(0, 2, 14).astype(np.int32)
    lengths = [int(t) for t in rng.integers(1, 300, 14)]
    Ks = [64, 256]
    E_list = [W.gaussian_emissions(t, Ks[mi], rng) for t, mi in zip(lengths, midx)]
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate([e.ravel() for e in E_list])).cuda(),
                 model_index=midx, models=models)
    ref = [oracle.viterbi(hmms[mi], e) for e, mi in zip(E_list, midx)]
    for P, rows in ((4, 12), (8, 40)):
        paths, scores = fv.decode(models, b, mode="flash", P=P, mem_budget=rows * 256 * 2, flags=flags)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (p, s) in enumerate(ref):
            assert np.array_equal(paths[off:off + lengths[i]], p), f"P={P} seq {i}"
            assert bits(scores[i]) == bits(s)
            off += lengths[i]


def test_budget_complete_pruning_exact_data(fv):
    """Complete pruning (offset-0 starts) on integer data, where no rounding
    happens: leaves and subtasks give the vanilla path."""
    rng = np.random.default_rng(13)
    K = 48
    log_pi = rng.integers(-3, 4, K).astype(np.float32)
    logA = rng.integers(-3, 4, (K, K)).astype(np.float32)
    lengths = [int(t) for t in rng.integers(2, 90, 10)]
    E_list = [rng.integers(-3, 4, (t, K)).astype(np.float32) for t in lengths]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    for P, rows in ((3, 4), (5, 20)):
        paths, _ = fv.decode([m], b, mode="flash", P=P, mem_budget=rows * K * 2,
                             flags=fv._lib.FV_COMPLETE_PRUNING)
        paths = paths.cpu().numpy()
        off = 0
        for i, e in enumerate(E_list):
            pb, _, _, _ = oracle.flash_budget(hmm, e, P, rows, complete=True)
            assert np.array_equal(paths[off:off + lengths[i]], pb), f"P={P} seq {i}"
            off += lengths[i]
