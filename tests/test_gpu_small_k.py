"""The small-K engine (K <= 128, one CTA of 64 or 128 threads per job, the
default at K <= 128) against the oracle: paths identical, scores equal to
0 ulp, on the cases that exercise the argmax rule (integer ties, -inf
transitions and all--inf steps, signed zeros), discrete emissions, several
models in one batch, a batch of many sequences, and every job kind: FLASH
root passes and subtasks (retained offset and complete pruning), budget
leaves and both Checkpoint Viterbi passes."""
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


@pytest.fixture
def small(fv):
    """Selects the default configuration (exact jobs on the small-K kernel)
    for every K <= 64 decode of the test."""
    fv.set_engine_variant(64, 0)
    try:
        yield fv
    finally:
        fv.set_engine_variant(64, 0)


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


def check(fv, log_pi, logA, E_list):
    K = log_pi.shape[0]
    lengths = [e.shape[0] for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    paths, scores = fv.decode([m], b)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    res = oracle.map_sequences(lambda e: oracle.viterbi(oracle.HMM(log_pi, logA), e), E_list)
    off = 0
    for i, (p, s) in enumerate(res):
        T = lengths[i]
        assert np.array_equal(paths[off:off + T], p), f"K={K} seq {i} (T={T})"
        assert bits(scores[i]) == bits(s), f"K={K} seq {i} score {scores[i]!r} vs {s!r}"
        off += T


@pytest.mark.parametrize("K", [1, 2, 3, 7, 16, 31, 32, 33, 48, 63, 64])
def test_random_models(small, K):
    rng = np.random.default_rng(700 + K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 5, 17, 64, 97, 1, 250] + [int(t) for t in rng.integers(1, 300, 30)]
    check(small, log_pi, logA, [W.gaussian_emissions(t, K, rng) for t in lengths])


@pytest.mark.parametrize("K", [4, 37, 64])
def test_integer_ties_and_neg_inf(small, K):
    rng = np.random.default_rng(800 + K)
    for frac in (0.0, 0.6, 0.97):
        log_pi = rng.integers(-2, 3, K).astype(np.float32)
        logA = rng.integers(-2, 3, (K, K)).astype(np.float32)
        logA[rng.random((K, K)) < frac] = -np.inf
        E_list = [rng.integers(-2, 3, (int(t), K)).astype(np.float32) for t in rng.integers(1, 80, 25)]
        check(small, log_pi, logA, E_list)


def test_signed_zero_ties(small):
    K = 8
    log_pi = np.zeros(K, np.float32)
    logA = np.zeros((K, K), np.float32)
    logA[::2] = -0.0
    E_list = [np.where(np.arange(K) % 3 == 0, -0.0, 0.0).astype(np.float32)[None].repeat(t, 0)
              for t in (1, 2, 5, 9)]
    check(small, log_pi, logA, E_list)


def test_discrete_emissions_config1(small):
    c = W.config1()
    m = small.Model(c["log_pi"], c["logA"], logB=c["logB"])
    b = small.Batch([c["T"]], obs=c["obs"], models=[m])
    paths, scores = small.decode([m], b)
    p, s = oracle.viterbi(oracle.HMM(c["log_pi"], c["logA"]), oracle.expand_discrete(c["logB"], c["obs"]))
    assert np.array_equal(paths.cpu().numpy(), p)
    assert bits(scores.cpu().numpy()[0]) == bits(s)


def test_models_of_both_engines_in_one_batch(small):
    """K=17 and K=64 run on the small-K kernel, K=200 on the slot engine."""
    rng = np.random.default_rng(15)
    Ks = [64, 200, 17]
    models_np = [W.random_model(K, rng) for K in Ks]
    mi = rng.integers(0, 3, 30)
    lengths = rng.integers(1, 150, 30)
    E_list = [W.gaussian_emissions(int(t), Ks[m], rng) for t, m in zip(lengths, mi)]
    models = [small.Model(lp, A) for lp, A in models_np]
    E = torch.from_numpy(np.concatenate([e.reshape(-1) for e in E_list])).cuda()
    b = small.Batch(lengths, E=E, model_index=mi, models=models)
    paths, scores = small.decode(models, b)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    off = 0
    for i in range(30):
        p, s = oracle.viterbi(oracle.HMM(*models_np[mi[i]]), E_list[i])
        assert np.array_equal(paths[off:off + lengths[i]], p)
        assert bits(scores[i]) == bits(s)
        off += lengths[i]


def test_many_sequences(small):
    """2000 sequences: more CTAs than the GPU holds at once."""
    rng = np.random.default_rng(16)
    K = 64
    log_pi, logA = W.random_model(K, rng)
    lengths = [int(t) for t in rng.integers(1, 120, 2000)]
    check(small, log_pi, logA, [W.gaussian_emissions(t, K, rng) for t in lengths])


@pytest.fixture
def small128(fv):
    """The default K <= 128 configuration: exact jobs on the small-K kernel
    (a 128-thread CTA per sequence)."""
    fv.set_engine_variant(128, 0)
    try:
        yield fv
    finally:
        fv.set_engine_variant(128, 0)


@pytest.mark.parametrize("K", [65, 97, 127, 128])
def test_random_models_up_to_128(small128, K):
    rng = np.random.default_rng(900 + K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 17, 130, 1] + [int(t) for t in rng.integers(1, 300, 25)]
    check(small128, log_pi, logA, [W.gaussian_emissions(t, K, rng) for t in lengths])


def test_integer_ties_and_neg_inf_up_to_128(small128):
    rng = np.random.default_rng(1000)
    K = 100
    for frac in (0.0, 0.6, 0.97):
        log_pi = rng.integers(-2, 3, K).astype(np.float32)
        logA = rng.integers(-2, 3, (K, K)).astype(np.float32)
        logA[rng.random((K, K)) < frac] = -np.inf
        E_list = [rng.integers(-2, 3, (int(t), K)).astype(np.float32) for t in rng.integers(1, 80, 25)]
        check(small128, log_pi, logA, E_list)


def test_many_sequences_up_to_128(small128):
    rng = np.random.default_rng(17)
    K = 128
    log_pi, logA = W.random_model(K, rng)
    lengths = [int(t) for t in rng.integers(1, 120, 1500)]
    check(small128, log_pi, logA, [W.gaussian_emissions(t, K, rng) for t in lengths])


def decode_modes_check(fv, log_pi, logA, E_list, mode, **kw):
    """One decode in `mode` against the oracle's restatement of it."""
    lengths = [e.shape[0] for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    complete = bool(kw.pop("complete", False))
    flags = fv._lib.FV_COMPLETE_PRUNING if complete else 0
    paths, scores = fv.decode([m], b, mode=mode, flags=flags, **kw)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    P = kw.get("P", 1)
    if mode == "checkpoint":
        ref = oracle.map_sequences(lambda e: oracle.checkpoint(hmm, e, P)[:2], E_list)
    elif kw.get("mem_budget"):
        rows = kw["mem_budget"] // (2 * log_pi.shape[0])
        ref = oracle.map_sequences(lambda e: oracle.flash_budget(hmm, e, P, rows, complete=complete)[:2], E_list)
    else:
        ref = oracle.map_sequences(lambda e: oracle.flash(hmm, e, P, complete=complete)[:2], E_list)
    off = 0
    for i, (p, s) in enumerate(ref):
        T = lengths[i]
        assert np.array_equal(paths[off:off + T], p), f"{mode} {kw} seq {i} (T={T})"
        if not complete:
            assert bits(scores[i]) == bits(s), f"{mode} {kw} seq {i} score"
        off += T


@pytest.mark.parametrize("K", [5, 37, 64, 100, 128])
@pytest.mark.parametrize("case", ["flash4", "flash16", "flash_complete", "budget", "checkpoint"])
def test_flash_budget_checkpoint_kinds(fv, K, case):
    """FLASH root passes and subtasks, budget leaves and both Checkpoint
    Viterbi passes on the small-K engine (the K <= 128 default)."""
    fv.set_engine_variant(K, 0)
    rng = np.random.default_rng(1100 + K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 9, 40, 130, 257] + [int(t) for t in rng.integers(1, 300, 12)]
    E_list = [W.gaussian_emissions(t, K, rng) for t in lengths]
    kw = {"flash4": dict(mode="flash", P=4), "flash16": dict(mode="flash", P=16),
          "flash_complete": dict(mode="flash", P=4, complete=True),
          "budget": dict(mode="flash", P=4, mem_budget=24 * K * 2),
          "checkpoint": dict(mode="checkpoint", P=0)}[case]
    mode = kw.pop("mode")
    decode_modes_check(fv, log_pi, logA, E_list, mode, **kw)


def test_integer_ties_flash_and_budget(fv):
    rng = np.random.default_rng(1200)
    K = 40
    fv.set_engine_variant(K, 0)
    log_pi = rng.integers(-2, 3, K).astype(np.float32)
    logA = rng.integers(-2, 3, (K, K)).astype(np.float32)
    logA[rng.random((K, K)) < 0.6] = -np.inf
    E_list = [rng.integers(-2, 3, (int(t), K)).astype(np.float32) for t in rng.integers(1, 120, 20)]
    decode_modes_check(fv, log_pi, logA, E_list, "flash", P=8)
    decode_modes_check(fv, log_pi, logA, E_list, "flash", P=8, mem_budget=16 * K * 2)
    decode_modes_check(fv, log_pi, logA, E_list, "checkpoint", P=0)
