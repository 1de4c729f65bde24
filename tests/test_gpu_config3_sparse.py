"""The large sparse configuration: K = 65536 states, 32 distinct uniform
successors per state (CSR), Dirichlet(1) edge weights, batch 8.  Dynamic
beam search (Sec. V-C) with B in {128, 512, 2048} and FLASH-BS must match
the oracle exactly on a T-prefix of all 8 sequences."""
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
def case(fv):
    log_pi, rp, col, val = W.config3_sparse_model()
    K, n, T = 65536, 8, 60
    E = W.gaussian_emissions_packed_device(n * T, K, seed=4, device="cuda")
    m = fv.Model(log_pi, row_ptr=rp, col=col, val=val)
    b = fv.Batch([T] * n, E=E.view(-1), models=[m])
    hmm = oracle.HMM(log_pi, None, rp, col, val)
    return m, b, hmm, list(E.view(n, T, K).cpu().numpy()), n, T


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


@pytest.mark.parametrize("B,P", [(128, 0), (512, 0), (2048, 0), (512, 4)])
def test_config3_sparse_beam_prefix(fv, case, B, P):
    m, b, hmm, E_list, n, T = case
    paths, scores = fv.decode([m], b, mode="beam", B=B, P=P)
    paths, scores = paths.cpu().numpy().reshape(n, T), scores.cpu().numpy()
    if P == 0:
        ref = oracle.map_sequences(lambda e: oracle.beam(hmm, e, B), E_list)
    else:
        ref = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, P, B), E_list)
    for i, r in enumerate(ref):
        assert r[-1] == 0
        assert np.array_equal(paths[i], r[0]), f"B={B} P={P} seq {i}"
        assert bits(scores[i]) == bits(r[1]), f"B={B} P={P} seq {i}"
