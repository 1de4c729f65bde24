"""The static beam (FV_STATIC_BEAM: every step writes all K scores, then
keeps the top B of them) on the GPU against the oracle's static beam and,
for FLASH-BS, its beam-subtask decoding: identical paths and 0-ulp scores
for dense and CSR transitions; and identical to the dynamic beam."""
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


def check(fv, m, hmm, E_list, B, P):
    lengths = [e.shape[0] for e in E_list]
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    ds = fv.Decoder([m], b, mode="beam", B=B, P=P, flags=fv._lib.FV_STATIC_BEAM)
    ps, ss = [x.clone() for x in ds(check=True)]
    pd, sd = fv.decode([m], b, mode="beam", B=B, P=P)
    assert torch.equal(ps, pd) and torch.equal(ss.view(torch.int32), sd.view(torch.int32))
    if P == 0:
        ref = oracle.map_sequences(lambda e: oracle.beam_static(hmm, e, B), E_list)
    else:
        ref = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, P, B), E_list)
    ps, ss = ps.cpu().numpy(), ss.cpu().numpy()
    off = 0
    for i, r in enumerate(ref):
        T = lengths[i]
        assert r[-1] == 0
        assert np.array_equal(ps[off:off + T], r[0]), f"seq {i} B={B} P={P}"
        assert bits(ss[i]) == bits(r[1]), f"seq {i} B={B} P={P}"
        off += T


@pytest.mark.parametrize("K,B", [(7, 3), (64, 16), (300, 64), (1024, 256)])
@pytest.mark.parametrize("P", [0, 4])
def test_static_beam_dense(fv, K, B, P):
    rng = np.random.default_rng(K + B + P)
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    hmm = oracle.HMM(log_pi, logA)
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in [1, 2, 30, 200, 451]]
    check(fv, m, hmm, E_list, B, P)


@pytest.mark.parametrize("K,deg,B", [(400, 4, 2), (4096, 32, 128), (65536, 32, 512)])
@pytest.mark.parametrize("P", [0, 4])
def test_static_beam_csr(fv, K, deg, B, P):
    rng = np.random.default_rng(K + B + P + 1)
    rp, col, val = W.random_csr(K, deg, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    m = fv.Model(log_pi, row_ptr=rp, col=col, val=val)
    hmm = oracle.HMM(log_pi, None, rp, col, val)
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in [1, 3, 40, 120]]
    check(fv, m, hmm, E_list, B, P)
