"""Checkpoint Viterbi (FV_CHECKPOINT, the sqrt(T)-checkpoint baseline of
Sec. II-A) on the GPU against the oracle's Checkpoint Viterbi and its exact
decoder: paths equal and scores equal to 0 ulp, for every engine (resident
K <= 256, streamed K <= 1024, whole-GPU K > 1024), default (ceil(sqrt T))
and explicit checkpoint counts, T = 1 and T below the count, discrete
emissions, and its O(K sqrt T) workspace."""
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


def run(fv, K, lengths, P, seed, integer=False):
    rng = np.random.default_rng(seed)
    log_pi, logA = W.random_model(K, rng)
    if integer:
        logA = rng.integers(-2, 3, (K, K)).astype(np.float32)
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    if integer:
        E_list = [np.round(e).astype(np.float32) for e in E_list]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    d = fv.Decoder([m], b, mode="checkpoint", P=P)
    paths, scores = d(check=True)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    ref = oracle.map_sequences(lambda e: oracle.checkpoint(hmm, e, P), E_list)
    van = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    off = 0
    for i, (r, v) in enumerate(zip(ref, van)):
        T = lengths[i]
        assert np.array_equal(r[0], v[0]) and bits(r[1]) == bits(v[1])
        assert np.array_equal(paths[off:off + T], r[0]), f"K={K} P={P} seq {i} T={T}"
        assert bits(scores[i]) == bits(r[1]), f"K={K} P={P} seq {i}"
        off += T
    return d


@pytest.mark.parametrize("K", [1, 5, 64, 100, 128, 256, 300, 512, 1024])
@pytest.mark.parametrize("P", [0, 1, 3, 1000])
def test_checkpoint_matches_oracle(fv, K, P):
    lengths = [1, 2, 3, 17, 64, 65, 257, 600]
    run(fv, K, lengths, P, seed=K * 10 + P)


@pytest.mark.parametrize("K", [1100, 2048])
def test_checkpoint_whole_gpu_engine(fv, K):
    run(fv, K, [1, 5, 40, 130, 300, 9, 77, 200, 31, 64], 0, seed=K)
    run(fv, K, [50, 120], 7, seed=K + 1)


def test_checkpoint_integer_ties(fv):
    run(fv, 37, [1, 4, 50, 200, 333], 0, seed=5, integer=True)
    run(fv, 256, [100, 999], 5, seed=6, integer=True)


def test_checkpoint_discrete_emissions(fv):
    w = W.config1()
    m = fv.Model(w["log_pi"], w["logA"], logB=w["logB"])
    b = fv.Batch([w["T"]], obs=w["obs"], models=[m])
    pv, sv = [x.clone() for x in fv.decode([m], b, mode="vanilla")]
    pc, sc = fv.decode([m], b, mode="checkpoint", P=0)
    assert torch.equal(pv, pc) and torch.equal(sv.view(torch.int32), sc.view(torch.int32))
    hmm = oracle.HMM(w["log_pi"], w["logA"])
    p, s, nc, _ = oracle.checkpoint(hmm, oracle.expand_discrete(w["logB"], w["obs"]), 0)
    assert nc == 32 and np.array_equal(pc.cpu().numpy()[:w["T"]], p) and bits(sc[0].item()) == bits(s)


def test_checkpoint_memory_is_k_sqrt_t(fv):
    """For long sequences the workspace holds the checkpoints and one
    segment of backpointers, far below the full table."""
    K = 256
    lengths = [4000] * 16
    m = fv.Model(*W.random_model(K, np.random.default_rng(1)))
    b = fv.Batch(lengths, E=torch.zeros(sum(lengths) * K, device="cuda"), models=[m])
    full = fv.workspace_size([m], b, mode="vanilla")
    ck = fv.workspace_size([m], b, mode="checkpoint", P=0)
    per_seq = 64 * K * 4 + 63 * K * 2  # ceil(sqrt 4000) checkpoints + one segment of ceil(4000/64) rows
    assert ck < full / 10
    assert ck <= 16 * (per_seq + 16) + (full - 16 * 4000 * K * 2) + 16 * 64 + 4096


def test_checkpoint_config2_sampled(fv):
    """The benchmark batch (1024 sequences, K = 256, T in [500, 4000]):
    bit-identical to the exact decoder on the GPU, and a sample of
    sequences against the oracle's Checkpoint Viterbi."""
    K = 256
    log_pi, logA = W.config2_model()
    lengths = W.config2_lengths()
    E = W.gaussian_emissions_packed_device(int(lengths.sum()), K, seed=2)
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E.view(-1), models=[m])
    pv, sv = [x.clone() for x in fv.decode([m], b, mode="vanilla")]
    d = fv.Decoder([m], b, mode="checkpoint", P=0)
    pc, sc = d(check=True)
    assert torch.equal(pv, pc) and torch.equal(sv.view(torch.int32), sc.view(torch.int32))
    e_off, p_off = W.packed_offsets(lengths, K)
    hmm = oracle.HMM(log_pi, logA)
    pick = [int(np.argmax(lengths)), int(np.argmin(lengths)), 3, 500]
    jobs = [E.view(-1)[e_off[i]:e_off[i] + lengths[i] * K].view(-1, K).cpu().numpy() for i in pick]
    res = oracle.map_sequences(lambda e: oracle.checkpoint(hmm, e, 0), jobs)
    P_ = pc.cpu().numpy()
    for i, r in zip(pick, res):
        assert np.array_equal(P_[p_off[i]:p_off[i] + lengths[i]], r[0])
        assert bits(sc[i].item()) == bits(r[1])
