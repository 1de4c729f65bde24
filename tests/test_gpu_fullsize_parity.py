"""Oracle parity on the long paths of the large configurations, element by
element (paths equal, scores equal to 0 ulp):

* dense K = 4096 (Dirichlet 0.1 rows), all 8 sequences at T = 2000: vanilla,
  FLASH P = 16 (several task levels) and FLASH P = 16 under a backpointer
  budget of 1/16 of the full table (budget leaves in more than one wave),
  each against the oracle's exact decoder (FLASH is bit-identical to it);
* dense K = 4096 with 12 sequences, more than the whole-GPU engine's 8
  lanes, so lanes run several jobs one after another;
* sparse K = 65536 (32 successors per state), all 8 sequences at the
  benchmarked T = 2000: dynamic beam and FLASH-BS (P = 4) at B = 128, 512
  and 2048;
* the dense beam at the serving shapes: K = 64, 256, 1024 with B = 256,
  P = 0 and P = 4, lengths from 100 to 3000 (K = 1024 takes the
  four-targets-per-thread candidate step of the beam kernel).

The oracle runs on the host cores, one sequence per thread."""
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


def check_against(paths, scores, lengths, ref, what):
    off = 0
    for i, r in enumerate(ref):
        T = lengths[i]
        assert r[-1] == 0 if len(r) > 2 else True, f"{what}: oracle status {r[-1]} on seq {i}"
        assert np.array_equal(paths[off:off + T], r[0]), f"{what}: path of seq {i}"
        assert bits(scores[i]) == bits(r[1]), f"{what}: score of seq {i} ({scores[i]} vs {r[1]})"
        off += T


@pytest.mark.parametrize("n,T", [(8, 2000), (12, 600)])
def test_config3_dense_long_prefix(fv, n, T):
    log_pi, logA = W.config3_dense_model()
    K = 4096
    E = W.gaussian_emissions_packed_device(n * T, K, seed=3 + n, device="cuda")
    m = fv.Model(log_pi, logA)
    b = fv.Batch([T] * n, E=E.view(-1), models=[m])
    hmm = oracle.HMM(log_pi, logA)
    ref = oracle.map_sequences(lambda e: oracle.viterbi(hmm, e), list(E.view(n, T, K).cpu().numpy()))
    table = n * T * K * 2
    runs = [{"mode": "vanilla"}, {"mode": "flash", "P": 16}, {"mode": "flash", "P": 16, "mem_budget": table // 16}]
    for kw in runs:
        d = fv.Decoder([m], b, **kw)
        paths, scores = d(check=True)
        check_against(paths.cpu().numpy(), scores.cpu().numpy(), [T] * n, ref, f"K=4096 n={n} T={T} {kw}")


@pytest.fixture(scope="module")
def sparse_case(fv):
    log_pi, rp, col, val = W.config3_sparse_model()
    K, n, T = 65536, 8, 2000
    E = W.gaussian_emissions_packed_device(n * T, K, seed=4, device="cuda", chunk_rows=1 << 13)
    m = fv.Model(log_pi, row_ptr=rp, col=col, val=val)
    b = fv.Batch([T] * n, E=E.view(-1), models=[m])
    hmm = oracle.HMM(log_pi, None, rp, col, val)
    return m, b, hmm, list(E.view(n, T, K).cpu().numpy()), n, T


@pytest.mark.parametrize("B", [128, 512, 2048])
@pytest.mark.parametrize("P", [0, 4])
def test_config3_sparse_benchmarked_prefix(fv, sparse_case, B, P):
    m, b, hmm, E_list, n, T = sparse_case
    d = fv.Decoder([m], b, mode="beam", B=B, P=P)
    paths, scores = d(check=True)
    if P == 0:
        ref = oracle.map_sequences(lambda e: oracle.beam(hmm, e, B), E_list)
    else:
        ref = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, P, B), E_list)
    check_against(paths.cpu().numpy(), scores.cpu().numpy(), [T] * n, ref, f"sparse B={B} P={P}")


@pytest.mark.parametrize("K", [64, 256, 1024])
@pytest.mark.parametrize("P", [0, 4])
def test_dense_beam_serving_shapes(fv, K, P):
    rng = np.random.default_rng(1000 + K + P)
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    hmm = oracle.HMM(log_pi, logA)
    lengths = [100, 257, 700, 1500, 3000]
    E_list = [W.gaussian_emissions(t, K, rng) for t in lengths]
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    B = 256
    d = fv.Decoder([m], b, mode="beam", B=B, P=P)
    paths, scores = d(check=True)
    if P == 0:
        ref = oracle.map_sequences(lambda e: oracle.beam(hmm, e, B), E_list)
    else:
        ref = oracle.map_sequences(lambda e: oracle.flash_bs(hmm, e, P, B), E_list)
    check_against(paths.cpu().numpy(), scores.cpu().numpy(), lengths, ref, f"dense beam K={K} B={B} P={P}")
    # one request at a time, as the server issues them, gives the same result
    for i in (0, 4):
        bi = fv.Batch([lengths[i]], E=torch.from_numpy(E_list[i]).cuda(), models=[m])
        pi_, si_ = fv.decode([m], bi, mode="beam", B=B, P=P)
        check_against(pi_.cpu().numpy(), si_.cpu().numpy(), [lengths[i]], [ref[i]], f"lone K={K} P={P} seq {i}")
