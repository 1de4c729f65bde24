"""The large dense configuration: K = 4096 states with Dirichlet(0.1)
transition rows, batch 8.  Parity with the oracle on a T-prefix of all 8
sequences (vanilla, FLASH, FLASH with a 1/16 backpointer budget); at the
full length T = 100 000 the properties that hold at any size: every exact
mode returns the same paths and scores, and each score is the oracle's
forward-order log-likelihood of the returned path."""
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


@pytest.fixture(scope="module")
def model():
    return W.config3_dense_model()


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


def test_config3_prefix_parity(fv, model):
    log_pi, logA = model
    K, n, T = 4096, 8, 24
    E = W.gaussian_emissions_packed_device(n * T, K, seed=3, device="cuda")
    m = fv.Model(log_pi, logA)
    b = fv.Batch([T] * n, E=E.view(-1), models=[m])
    E_list = list(E.view(n, T, K).cpu().numpy())
    hmm = oracle.HMM(log_pi, logA)
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    table = n * T * K * 2
    for kw in ({"mode": "vanilla"}, {"mode": "flash", "P": 16}, {"mode": "flash", "P": 16, "mem_budget": table // 16}):
        paths, scores = fv.decode([m], b, **kw)
        paths, scores = paths.cpu().numpy().reshape(n, T), scores.cpu().numpy()
        for i, (p, s) in enumerate(ref):
            assert np.array_equal(paths[i], p), f"{kw} seq {i}"
            assert bits(scores[i]) == bits(s), f"{kw} seq {i}"


def test_config3_full_length_properties(fv, model):
    log_pi, logA = model
    K, n, T = 4096, 8, 100000
    E = W.gaussian_emissions_packed_device(n * T, K, seed=3, device="cuda", chunk_rows=1 << 16)
    m = fv.Model(log_pi, logA)
    b = fv.Batch([T] * n, E=E.view(-1), models=[m])
    pv, sv = [x.clone() for x in fv.decode([m], b, mode="vanilla")]
    pb, sb = fv.decode([m], b, mode="flash", P=16, mem_budget=n * T * K * 2 // 16)
    assert torch.equal(pv, pb)
    assert torch.equal(sv.view(torch.int32), sb.view(torch.int32))
    hmm = oracle.HMM(log_pi, logA)
    paths = pv.cpu().numpy().reshape(n, T)
    Ev = E.view(n, T, K)
    for i in range(n):
        s = oracle.path_score(hmm, Ev[i].cpu().numpy(), paths[i])
        assert bits(s) == bits(sv[i].item()), f"seq {i}"
