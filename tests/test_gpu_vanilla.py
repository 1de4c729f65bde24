"""GPU parity of the exact decoder (full backpointer table) against the CPU
oracle: paths must be identical and scores equal to 0 ulp (the GPU performs
the same FP32 additions as the oracle, in the same order, plus exact
maxima)."""
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


def run_and_check(fv, log_pi, logA, E_list, mode="vanilla", **kw):
    K = log_pi.shape[0]
    lengths = [e.shape[0] for e in E_list]
    E = np.concatenate(E_list) if E_list else np.zeros((0, K), np.float32)
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(E).cuda(), models=[m])
    paths, scores = fv.decode([m], b, mode=mode, **kw)
    paths = paths.cpu().numpy()
    scores = scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    res = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    off = 0
    for i, (p, s) in enumerate(res):
        T = lengths[i]
        assert np.array_equal(paths[off:off + T], p), f"seq {i} (T={T}) path differs"
        assert bits(scores[i]) == bits(s), f"seq {i} score {scores[i]!r} vs {s!r}"
        off += T
    return paths, scores


@pytest.mark.parametrize("K", [1, 2, 3, 7, 16, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256])
def test_random_models_many_lengths(fv, K):
    rng = np.random.default_rng(K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 3, 5, 17, 64, 97, 1, 250] + list(rng.integers(1, 300, 40))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    run_and_check(fv, log_pi, logA, E_list)


@pytest.mark.parametrize("K", [4, 37, 160])
def test_integer_ties_and_neg_inf(fv, K):
    """Small-integer data (many exact ties) and -inf transitions exercise the
    lowest-index rule and the all--inf argmax."""
    rng = np.random.default_rng(100 + K)
    for frac in (0.0, 0.6):
        log_pi = rng.integers(-2, 3, K).astype(np.float32)
        logA = rng.integers(-2, 3, (K, K)).astype(np.float32)
        logA[rng.random((K, K)) < frac] = -np.inf
        E_list = [rng.integers(-2, 3, (int(t), K)).astype(np.float32) for t in rng.integers(1, 80, 25)]
        run_and_check(fv, log_pi, logA, E_list)


def test_signed_zero_ties(fv):
    """+0 and -0 candidates tie; the lower index wins and keeps its sign."""
    K = 8
    log_pi = np.zeros(K, np.float32)
    logA = np.zeros((K, K), np.float32)
    logA[::2] = -0.0
    E_list = [np.where(np.arange(K) % 3 == 0, -0.0, 0.0).astype(np.float32)[None].repeat(t, 0)
              for t in (1, 2, 5, 9)]
    run_and_check(fv, log_pi, logA, E_list)


def test_discrete_emissions_config1(fv):
    c = W.config1()
    m = fv.Model(c["log_pi"], c["logA"], logB=c["logB"])
    b = fv.Batch([c["T"]], obs=c["obs"], models=[m])
    paths, scores = fv.decode([m], b)
    E = oracle.expand_discrete(c["logB"], c["obs"])
    p, s = oracle.viterbi(oracle.HMM(c["log_pi"], c["logA"]), E)
    assert np.array_equal(paths.cpu().numpy(), p)
    assert bits(scores.cpu().numpy()[0]) == bits(s)


def test_multiple_models_in_one_batch(fv):
    rng = np.random.default_rng(5)
    Ks = [64, 200, 17]
    models_np = [W.random_model(K, rng) for K in Ks]
    mi = rng.integers(0, 3, 30)
    lengths = rng.integers(1, 150, 30)
    E_list = [W.gaussian_emissions(int(t), Ks[m], rng) for t, m in zip(lengths, mi)]
    models = [fv.Model(lp, A) for lp, A in models_np]
    E = torch.from_numpy(np.concatenate([e.reshape(-1) for e in E_list])).cuda()
    b = fv.Batch(lengths, E=E, model_index=mi, models=models)
    paths, scores = fv.decode(models, b)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    off = 0
    for i in range(30):
        p, s = oracle.viterbi(oracle.HMM(*models_np[mi[i]]), E_list[i])
        assert np.array_equal(paths[off:off + lengths[i]], p)
        assert bits(scores[i]) == bits(s)
        off += lengths[i]


def test_deterministic_and_order_independent(fv):
    rng = np.random.default_rng(9)
    K = 256
    log_pi, logA = W.random_model(K, rng)
    lengths = rng.integers(1, 400, 64)
    E = torch.from_numpy(W.gaussian_emissions(int(lengths.sum()), K, rng)).cuda()
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E, models=[m])
    p1, s1 = [x.clone() for x in fv.decode([m], b)]
    p2, s2 = [x.clone() for x in fv.decode([m], b, flags=fv._lib.FV_NO_SORT)]
    assert torch.equal(p1, p2) and torch.equal(s1.view(torch.int32), s2.view(torch.int32))


def test_workspace_too_small_is_reported(fv):
    rng = np.random.default_rng(1)
    K = 32
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    E = torch.from_numpy(W.gaussian_emissions(500, K, rng)).cuda()
    b = fv.Batch([500], E=E, models=[m])
    d = fv.Decoder([m], b)
    small = torch.empty(8192, dtype=torch.uint8, device="cuda")
    d2 = fv.Decoder([m], b, workspace=small)
    with pytest.raises(fv.FVError) as ei:
        d2.launch()
    assert ei.value.status == fv._lib.FV_ENOMEM
    # without host lengths the check happens on the device
    b._no_host = True
    bs = b.struct()
    bs.T_host = None
    import ctypes
    rc = d.lib.fv_decode(d._arr, 1, ctypes.byref(bs), ctypes.byref(d._ps), ctypes.c_void_p(small.data_ptr()),
                         small.numel(), ctypes.c_void_p(d.paths.data_ptr()), ctypes.c_void_p(d.scores.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fv._lib.FV_OK
    assert d.lib.fv_last_device_status(ctypes.c_void_p(small.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == fv._lib.FV_ENOMEM


def test_config2_full_size_sampled(fv):
    """The benchmark workload (1024 sequences, K=256, T ~ U[500,4000]) in
    every engine configuration of its K class (the benchmark times the one
    the autotuner picks); a sample of sequences (the longest, the shortest,
    and random ones) is checked against the oracle."""
    K = 256
    log_pi, logA = W.config2_model()
    lengths = W.config2_lengths()
    e_total = int(lengths.sum())
    E = W.gaussian_emissions_packed_device(e_total, K, seed=2)
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E.view(-1), models=[m])
    rng = np.random.default_rng(0)
    pick = sorted(set([int(np.argmax(lengths)), int(np.argmin(lengths))] + list(rng.choice(len(lengths), 14, replace=False))))
    e_off, p_off = W.packed_offsets(lengths, K)
    hmm = oracle.HMM(log_pi, logA)
    jobs = [E.view(-1)[e_off[i]:e_off[i] + lengths[i] * K].view(-1, K).cpu().numpy() for i in pick]
    res = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), jobs)
    nv = fv.set_engine_variant(K, 0)
    try:
        for v in range(nv):
            fv.set_engine_variant(K, v)
            paths, scores = fv.decode([m], b)
            P = paths.cpu().numpy()
            S = scores.cpu().numpy()
            for i, (p, s) in zip(pick, res):
                assert np.array_equal(P[p_off[i]:p_off[i] + lengths[i]], p), f"variant {v} seq {i}"
                assert bits(S[i]) == bits(s), f"variant {v} seq {i}"
    finally:
        fv.set_engine_variant(K, 0)
