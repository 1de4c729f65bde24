"""GPU parity on the paper's Erdos-Renyi workload family (Sec. VI):
transition graphs with edge probability p (absent edges -inf), discrete
emissions over 50 symbols, observation sequences sampled from the HMM.
Every mode is compared with the oracle bit for bit: vanilla, FLASH (pure
divide and conquer and with a memory budget), the dynamic beam and
FLASH-BS (narrow beams follow the oracle's canonical top-B)."""
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


def er_batch(K, p, lengths, seed):
    """One ER model and several observation sequences sampled from it."""
    c = W.erdos_renyi_case(K, 1, p, seed=seed)
    rng = np.random.default_rng(seed + 101)
    obs = [W.sample_hmm_sequence(c["log_pi"], c["logA"], c["logB"], int(T), rng) for T in lengths]
    return c, obs


def decode_er(fv, c, obs, **kw):
    m = fv.Model(c["log_pi"], c["logA"], logB=c["logB"])
    b = fv.Batch([len(o) for o in obs], obs=np.concatenate(obs), models=[m])
    paths, scores = fv.decode([m], b, **kw)
    return paths.cpu().numpy(), scores.cpu().numpy()


def check(paths, scores, obs, ref):
    off = 0
    for i, o in enumerate(obs):
        T = len(o)
        p, s = ref[i][0], ref[i][1]
        assert np.array_equal(paths[off:off + T], p), f"sequence {i}"
        assert bits(scores[i]) == bits(s), f"sequence {i}"
        off += T


@pytest.mark.parametrize("K", [32, 200, 512])
@pytest.mark.parametrize("p", [0.05, 0.253, 1.0])
def test_er_exact_modes(fv, K, p):
    lengths = [1, 2, 64, 511]
    c, obs = er_batch(K, p, lengths, seed=K + int(p * 1000))
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    Es = [oracle.expand_discrete(c["logB"], o) for o in obs]
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), Es)
    check(*decode_er(fv, c, obs, mode="vanilla"), obs, ref)
    for P in (4, 16):
        check(*decode_er(fv, c, obs, mode="flash", P=P), obs, ref)
    # memory budget of 1/16 of the full backpointer table
    table = sum(lengths) * K * 2
    check(*decode_er(fv, c, obs, mode="flash", P=16, mem_budget=table // 16), obs, ref)


@pytest.mark.parametrize("K,B", [(64, 16), (200, 32), (512, 128)])
def test_er_beam_modes(fv, K, B):
    lengths = [1, 33, 300]
    c, obs = er_batch(K, 0.253, lengths, seed=7 * K + B)
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    Es = [oracle.expand_discrete(c["logB"], o) for o in obs]
    ref = oracle.map_sequences(lambda e: oracle.beam(hmm, e, B), Es)
    check(*decode_er(fv, c, obs, mode="beam", B=B, P=0), obs, ref)
    ref = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, 4, B), Es)
    check(*decode_er(fv, c, obs, mode="beam", B=B, P=4), obs, ref)


def test_er_large_state_space(fv):
    """K = 2048 runs in the whole-GPU engine."""
    c, obs = er_batch(2048, 0.253, [40], seed=3)
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    Es = [oracle.expand_discrete(c["logB"], o) for o in obs]
    ref = [oracle.viterbi(hmm, Es[0])]
    check(*decode_er(fv, c, obs, mode="vanilla"), obs, ref)
    check(*decode_er(fv, c, obs, mode="flash", P=4), obs, ref)
