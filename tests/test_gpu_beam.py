"""GPU parity of dynamic beam search (Sec. V-C) and FLASH-BS against the
oracle: identical paths and 0-ulp scores, dense and CSR transitions; beams
at least as wide as the state set reproduce exact decoding."""
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


def make_model(fv, log_pi, logA=None, csr=None):
    if csr is None:
        return fv.Model(log_pi, logA), oracle.HMM(log_pi, logA)
    rp, col, val = csr
    return fv.Model(log_pi, row_ptr=rp, col=col, val=val), oracle.HMM(log_pi, None, rp, col, val)


def run_beam(fv, m, hmm, E_list, B, P):
    lengths = [e.shape[0] for e in E_list]
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    paths, scores = fv.decode([m], b, mode="beam", P=P, B=B)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    if P == 0:
        res = oracle.map_sequences(lambda e: oracle.beam(hmm, e, B), E_list)
    else:
        res = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, P, B), E_list)
    off = 0
    for i, r in enumerate(res):
        p, s = r[0], r[1]
        T = lengths[i]
        assert r[-1] == 0, "oracle found the case infeasible"
        assert np.array_equal(paths[off:off + T], p), f"seq {i} T={T} B={B} P={P}"
        assert bits(scores[i]) == bits(s), f"seq {i} score {scores[i]} vs {s}"
        off += T


@pytest.mark.parametrize("P", [0, 1, 4])
@pytest.mark.parametrize("K,B", [(7, 1), (7, 3), (33, 5), (64, 16), (130, 40), (300, 64), (64, 64), (20, 100)])
def test_dense_beam(fv, K, B, P):
    rng = np.random.default_rng(K * 7 + B + 100 * P)
    log_pi, logA = W.random_model(K, rng)
    m, hmm = make_model(fv, log_pi, logA)
    lengths = [1, 2, 3, 9, 40] + list(rng.integers(1, 150, 8))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    run_beam(fv, m, hmm, E_list, B, P)


@pytest.mark.parametrize("P", [0, 2, 8])
@pytest.mark.parametrize("K,deg,B", [(50, 6, 4), (200, 12, 16), (1000, 32, 128)])
def test_csr_beam(fv, K, deg, B, P):
    rng = np.random.default_rng(K + deg + B + P)
    rp, col, val = W.random_csr(K, deg, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    m, hmm = make_model(fv, log_pi, csr=(rp, col, val))
    lengths = [1, 2, 5] + list(rng.integers(2, 120, 6))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    run_beam(fv, m, hmm, E_list, B, P)


def test_beam_integer_ties(fv):
    rng = np.random.default_rng(3)
    K = 24
    log_pi = rng.integers(-1, 2, K).astype(np.float32)
    logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
    m, hmm = make_model(fv, log_pi, logA)
    E_list = [rng.integers(-1, 2, (int(t), K)).astype(np.float32) for t in rng.integers(1, 60, 10)]
    for B in (1, 5, 24):
        for P in (0, 3):
            run_beam(fv, m, hmm, E_list, B, P)


@pytest.mark.parametrize("P", [0, 4])
def test_full_width_beam_is_exact(fv, P):
    rng = np.random.default_rng(17)
    K = 128
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    lengths = rng.integers(1, 300, 20)
    E = torch.from_numpy(W.gaussian_emissions(int(lengths.sum()), K, rng)).cuda()
    b = fv.Batch(lengths, E=E, models=[m])
    pv, sv = [x.clone() for x in fv.decode([m], b, mode="vanilla")]
    pb, sb = fv.decode([m], b, mode="beam", P=P, B=K)
    assert torch.equal(pv, pb)
    assert torch.equal(sv.view(torch.int32), sb.view(torch.int32))


def test_csr_subtask_rerun_matches_oracle(fv):
    """Sparse graphs where the subtask beam misses q_n: both sides re-run the
    subtask with every state (R9) and agree."""
    rng = np.random.default_rng(23)
    K, deg = 400, 4
    rp, col, val = W.random_csr(K, deg, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    m, hmm = make_model(fv, log_pi, csr=(rp, col, val))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in (60, 80, 100)]
    reruns = [oracle.flash_bs(hmm, e, 4, 2)[2] for e in E_list]
    assert sum(reruns) > 0, "case does not exercise the re-run"
    run_beam(fv, m, hmm, E_list, 2, 4)


@pytest.mark.parametrize("K,deg", [(8192, 4), (10001, 32)])
@pytest.mark.parametrize("B", [1, 64, 256, 1000, 4000])
def test_csr_beam_large_k_cluster_engine(fv, K, deg, B):
    """Large CSR state spaces (K >= 8192, P = 0) run one sequence per
    cluster of CTAs when the beam holds at least 64 states (id ranges
    split over the CTAs, cluster-wide top-B), narrower beams one CTA:
    same results as the oracle, including ranges of unequal size (K not a
    multiple of the cluster size) and ties between ranks (integer weights
    and emissions)."""
    rng = np.random.default_rng(K + B)
    rp, col, val = W.random_csr(K, deg, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    lengths = [1, 2, 50, 300]
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    m, hmm = make_model(fv, log_pi, csr=(rp, col, val))
    run_beam(fv, m, hmm, E_list, B, 0)
    # integer data: many equal candidates, resolved by the lowest id
    val_i = np.round(val * 2).astype(np.float32)
    lp_i = np.round(log_pi).astype(np.float32)
    E_i = [np.round(e).astype(np.float32) for e in E_list]
    m2, hmm2 = make_model(fv, lp_i, csr=(rp, col, val_i))
    run_beam(fv, m2, hmm2, E_i, B, 0)
