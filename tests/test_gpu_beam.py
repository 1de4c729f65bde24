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


def _masked_model(K, rng, frac):
    """Dense model with a fraction of the transitions absent (-inf); every
    state keeps its self-transition."""
    log_pi, logA = W.random_model(K, rng)
    drop = rng.random((K, K)) < frac
    np.fill_diagonal(drop, False)
    logA = np.where(drop, -np.inf, logA).astype(np.float32)
    return log_pi, logA


@pytest.mark.parametrize("K,B", [(512, 1), (512, 64), (544, 200), (768, 7), (1024, 256), (1024, 1024),
                                 (2048, 100), (4096, 300), (8192, 64)])
def test_dense_beam_cluster_engine(fv, K, B):
    """Dense beams with 512 <= K <= 8192 (P = 0) run one sequence per
    cluster of CTAs (targets split over the CTAs, every CTA selecting the
    top B of all K candidates): same paths and scores as the oracle, with
    absent transitions, with integer data (equal candidates and signed
    zeros, resolved by the lowest id), and with more sequences than the
    GPU holds clusters."""
    rng = np.random.default_rng(K * 3 + B)
    log_pi, logA = _masked_model(K, rng, 0.3)
    m, hmm = make_model(fv, log_pi, logA)
    lengths = [1, 2, 3, 40, 120] if K <= 2048 else [1, 2, 17, 30]
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    run_beam(fv, m, hmm, E_list, B, 0)
    # integer data: many equal candidates; np.round gives -0 for small negatives
    lp_i = np.round(log_pi).astype(np.float32)
    A_i = np.round(logA * 2).astype(np.float32)
    E_i = [np.round(e).astype(np.float32) for e in E_list]
    m2, hmm2 = make_model(fv, lp_i, A_i)
    run_beam(fv, m2, hmm2, E_i, B, 0)


def test_dense_beam_cluster_engine_many_sequences(fv):
    """More sequences than resident clusters: each cluster decodes several
    sequences in turn (one long sequence among short ones, so that the
    launch takes the cluster kernel)."""
    rng = np.random.default_rng(77)
    K = 512
    log_pi, logA = W.random_model(K, rng)
    m, hmm = make_model(fv, log_pi, logA)
    lengths = [200] + list(rng.integers(1, 60, 44))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    run_beam(fv, m, hmm, E_list, 32, 0)


def test_dense_beam_cluster_engine_discrete(fv):
    """Symbol emissions (logB rows selected by the observations) on the
    cluster engine."""
    rng = np.random.default_rng(78)
    K, V = 1024, 40
    log_pi, logA = W.random_model(K, rng)
    logB = np.log(rng.dirichlet(np.full(V, 0.5), K)).astype(np.float32)
    m = fv.Model(log_pi, logA, logB=logB)
    lengths = [1, 5, 90, 200]
    obs = [rng.integers(0, V, t).astype(np.int32) for t in lengths]
    b = fv.Batch(lengths, obs=torch.from_numpy(np.concatenate(obs)).cuda(), models=[m])
    paths, scores = fv.decode([m], b, mode="beam", P=0, B=128)
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    off = 0
    for i, (t, o) in enumerate(zip(lengths, obs)):
        p, s, st = oracle.beam(hmm, oracle.expand_discrete(logB, o), 128)
        assert st == 0
        assert np.array_equal(paths[off:off + t], p), f"seq {i}"
        assert bits(scores[i]) == bits(s)
        off += t


def test_dense_beam_cluster_engine_infeasible(fv):
    """A beam that empties (every candidate -inf) is reported as
    FV_EINFEASIBLE, as the oracle finds it, and the next call decodes."""
    rng = np.random.default_rng(79)
    K = 512
    log_pi, logA = W.random_model(K, rng)
    # state 0 is the only possible start and leads nowhere
    log_pi = np.full(K, -np.inf, np.float32)
    log_pi[0] = 0.0
    logA[0, :] = -np.inf
    m, hmm = make_model(fv, log_pi, logA)
    E = W.gaussian_emissions(10, K, rng)
    assert oracle.beam(hmm, E, 16)[2] == 6
    b = fv.Batch([10], E=torch.from_numpy(E).cuda(), models=[m])
    with pytest.raises(fv._lib.FVError) as ei:
        fv.decode([m], b, mode="beam", P=0, B=16)
    assert ei.value.status == fv._lib.FV_EINFEASIBLE
    log_pi2, logA2 = W.random_model(K, rng)
    m2, hmm2 = make_model(fv, log_pi2, logA2)
    run_beam(fv, m2, hmm2, [W.gaussian_emissions(30, K, rng)], 16, 0)


def test_dense_beam_many_short_sequences_one_cta_each(fv):
    """Many sequences of equal length finish sooner with one CTA each than
    with one cluster each (the launch picks by the two makespans): the
    single-CTA kernel's four-targets-per-thread path at K >= 512, P = 0,
    against the oracle."""
    rng = np.random.default_rng(80)
    K = 512
    log_pi, logA = _masked_model(K, rng, 0.2)
    m, hmm = make_model(fv, log_pi, logA)
    E_list = [W.gaussian_emissions(30, K, rng) for _ in range(160)]
    run_beam(fv, m, hmm, E_list, 64, 0)


def test_shared_gpu_flag_keeps_results(fv):
    """FV_SHARED_GPU (one CTA per sequence for dense beams, as a serving loop
    asks) decodes a lone K=1024 sequence exactly like the cluster kernel the
    launch takes without it, and both equal the oracle."""
    rng = np.random.default_rng(81)
    K, B = 1024, 256
    log_pi, logA = W.random_model(K, rng)
    m, hmm = make_model(fv, log_pi, logA)
    E = W.gaussian_emissions(150, K, rng)
    b = fv.Batch([150], E=torch.from_numpy(E).cuda(), models=[m])
    pc, sc = [x.clone() for x in fv.decode([m], b, mode="beam", P=0, B=B)]
    ps, ss = fv.decode([m], b, mode="beam", P=0, B=B, flags=fv._lib.FV_SHARED_GPU)
    assert torch.equal(pc, ps)
    assert torch.equal(sc.view(torch.int32), ss.view(torch.int32))
    p, s, st = oracle.beam(hmm, E, B)
    assert st == 0 and np.array_equal(ps.cpu().numpy(), p) and bits(ss.cpu().numpy()[0]) == bits(s)


@pytest.mark.parametrize("K", [1, 5, 33, 64, 65, 100, 128])
def test_small_k_beam_engine(fv, K):
    """Dense beams with K <= 128 (P = 0) run one CTA per sequence with a
    thread per state (delta -inf outside the beam, full max-plus, rank
    select): same paths and scores as the oracle for narrow and full-width
    beams, with absent transitions, integer data (equal candidates, signed
    zeros) and many sequences."""
    rng = np.random.default_rng(300 + K)
    log_pi, logA = _masked_model(K, rng, 0.3)
    m, hmm = make_model(fv, log_pi, logA)
    lengths = [1, 2, 3, 40, 300] + list(rng.integers(1, 80, 40))
    E_list = [W.gaussian_emissions(int(t), K, rng) for t in lengths]
    lp_i = np.round(log_pi).astype(np.float32)
    A_i = np.round(logA * 2).astype(np.float32)
    E_i = [np.round(e).astype(np.float32) for e in E_list]
    m2, hmm2 = make_model(fv, lp_i, A_i)
    for B in sorted({1, 3, 16, max(1, K - 1), K, K + 5}):
        run_beam(fv, m, hmm, E_list, B, 0)
        run_beam(fv, m2, hmm2, E_i, B, 0)


@pytest.mark.parametrize("K,V", [(64, 32), (128, 200)])
def test_small_k_beam_engine_discrete(fv, K, V):
    """Symbol emissions on the small-K beam engine: the table staged in
    shared memory (64 x 32) and read from global memory (128 x 200)."""
    rng = np.random.default_rng(K + V)
    log_pi, logA = W.random_model(K, rng)
    logB = np.log(rng.dirichlet(np.full(V, 0.5), K)).astype(np.float32)
    m = fv.Model(log_pi, logA, logB=logB)
    lengths = [1, 7, 300, 1000]
    obs = [rng.integers(0, V, t).astype(np.int32) for t in lengths]
    b = fv.Batch(lengths, obs=torch.from_numpy(np.concatenate(obs)).cuda(), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    for B in (1, 16, K):
        paths, scores = fv.decode([m], b, mode="beam", P=0, B=B)
        paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
        off = 0
        for i, (t, o) in enumerate(zip(lengths, obs)):
            p, s, st = oracle.beam(hmm, oracle.expand_discrete(logB, o), B)
            assert st == 0
            assert np.array_equal(paths[off:off + t], p), f"seq {i} B={B}"
            assert bits(scores[i]) == bits(s)
            off += t


def test_small_k_beam_engine_infeasible(fv):
    """An emptied beam on the small-K engine is FV_EINFEASIBLE, as in the
    oracle."""
    rng = np.random.default_rng(82)
    K = 64
    log_pi, logA = W.random_model(K, rng)
    log_pi = np.full(K, -np.inf, np.float32)
    log_pi[3] = 0.0
    logA[3, :] = -np.inf
    m, hmm = make_model(fv, log_pi, logA)
    E = W.gaussian_emissions(10, K, rng)
    assert oracle.beam(hmm, E, 4)[2] == 6
    b = fv.Batch([10], E=torch.from_numpy(E).cuda(), models=[m])
    with pytest.raises(fv._lib.FVError) as ei:
        fv.decode([m], b, mode="beam", P=0, B=4)
    assert ei.value.status == fv._lib.FV_EINFEASIBLE
