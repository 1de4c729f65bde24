"""Engine variants and the autotuner: every configuration of a K class
computes the same values in the same order, so each one must match the
oracle bit for bit, and decoding after fv_autotune must equal decoding
with the default configuration (FV_NO_TUNE)."""
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


@pytest.mark.parametrize("K", [37, 64, 100, 128, 200, 256, 300, 512, 777, 1024])
def test_every_variant_matches_oracle(fv, K):
    rng = np.random.default_rng(K + 900)
    log_pi, logA = W.random_model(K, rng)
    lengths = [1, 2, 7, 33] + [int(t) for t in rng.integers(1, 300, 10)]
    E_list = [W.gaussian_emissions(t, K, rng) for t in lengths]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    nv = fv.set_engine_variant(K, 0)
    assert nv >= 2
    try:
        for v in range(nv):
            fv.set_engine_variant(K, v)
            # vanilla and budget leaves take the deferred re-scan where a
            # configuration has it; FLASH root and sub jobs do not
            for mode, kw in (("vanilla", {}), ("flash", {"P": 4}), ("flash", {"P": 4, "mem_budget": 40 * K * 2})):
                paths, scores = fv.decode([m], b, mode=mode, **kw)
                paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
                off = 0
                for i, (p, s) in enumerate(ref):
                    T = lengths[i]
                    assert np.array_equal(paths[off:off + T], p), f"K={K} variant {v} {mode} seq {i}"
                    assert bits(scores[i]) == bits(s)
                    off += T
    finally:
        fv.set_engine_variant(K, 0)


def test_autotune_keeps_results(fv):
    rng = np.random.default_rng(5)
    models, Ks = [], (64, 256)
    for K in Ks:
        lp, A = W.random_model(K, rng)
        models.append(fv.Model(lp, A))
    midx = np.array([0, 1] * 20, np.int32)
    lengths = [int(t) for t in rng.integers(50, 800, 40)]
    E = np.concatenate([W.gaussian_emissions(t, Ks[mi], rng).ravel() for t, mi in zip(lengths, midx)])
    b = fv.Batch(lengths, E=torch.from_numpy(E).cuda(), model_index=midx, models=models)
    ref_p, ref_s = [x.clone() for x in fv.decode(models, b, flags=fv._lib.FV_NO_TUNE)]
    try:
        chosen = fv.autotune(models, b)
        assert len(chosen) == 2 and all(0 <= c < fv.set_engine_variant(K, c) for c, K in zip(chosen, Ks))
        for c, K in zip(chosen, Ks):
            fv.set_engine_variant(K, c)
        p, s = fv.decode(models, b)
        assert torch.equal(p, ref_p) and torch.equal(s.view(torch.int32), ref_s.view(torch.int32))
    finally:
        for K in Ks:
            fv.set_engine_variant(K, 0)
