"""Exact decoding (vanilla and FLASH) on CSR transitions: the library runs
the beam with every state kept (B = K), which the oracle pins show is the
exact recursion.  Paths and scores must equal the oracle's exact CSR
Viterbi bit for bit."""
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


@pytest.mark.parametrize("K,deg,tmax", [(50, 6, 150), (200, 12, 120), (1000, 4, 60)])
def test_csr_exact_modes(fv, K, deg, tmax):
    rng = np.random.default_rng(K * 3 + deg)
    rp, col, val = W.random_csr(K, deg, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    m = fv.Model(log_pi, row_ptr=rp, col=col, val=val)
    lengths = [1, 2, 3] + [int(t) for t in rng.integers(1, tmax, 7)]
    E_list = [W.gaussian_emissions(t, K, rng) for t in lengths]
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, None, rp, col, val)
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), E_list)
    for mode, kw in (("vanilla", {}), ("flash", {"P": 1}), ("flash", {"P": 4})):
        paths, scores = fv.decode([m], b, mode=mode, **kw)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (p, s) in enumerate(ref):
            T = lengths[i]
            assert np.array_equal(paths[off:off + T], p), f"{mode} {kw} seq {i} T={T}"
            assert bits(scores[i]) == bits(s), f"{mode} {kw} seq {i}"
            off += T
