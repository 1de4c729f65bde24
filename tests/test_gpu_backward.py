"""GPU backward (path-count gradient) against the oracle's gradient (bit
for bit, ascending-sequence summation), against float32 finite differences
of the GPU decoder in generic position, and through torch.autograd on the
CRF-style workload (K=128 tags, linear emission layer)."""
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


@pytest.mark.parametrize("K", [1, 5, 128, 200])
def test_backward_matches_oracle_gradient(fv, K):
    rng = np.random.default_rng(K)
    log_pi, logA = W.random_model(K, rng)
    lengths = np.array([1, 2, 7] + list(rng.integers(1, 400, 30)), np.int32)
    E = torch.from_numpy(W.gaussian_emissions(int(lengths.sum()), K, rng)).cuda()
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E, models=[m])
    for g in (np.ones(len(lengths), np.float32), rng.standard_normal(len(lengths)).astype(np.float32)):
        for paths in (fv.decode([m], b)[0].clone(),
                      torch.from_numpy(rng.integers(0, K, int(lengths.sum())).astype(np.int32)).cuda()):
            dpi, dA, dE = fv.backward(m, b, paths, torch.from_numpy(g).cuda())
            opi, oA, oE = oracle.grad(K, lengths, paths.cpu().numpy(), g)
            assert np.array_equal(bits(dpi.cpu().numpy()), bits(opi))
            assert np.array_equal(bits(dA.cpu().numpy()), bits(oA))
            assert np.array_equal(bits(dE.cpu().numpy().reshape(-1)), bits(oE))


def test_backward_finite_differences(fv):
    """Generic position: the decoded path is locally constant, so
    (score(A + h e_ij) - score(A - h e_ij)) / 2h equals the path count."""
    rng = np.random.default_rng(9)
    K, T = 16, 60
    log_pi, logA = W.random_model(K, rng)
    E = W.gaussian_emissions(T, K, rng)
    Ed = torch.from_numpy(E).cuda()

    def score(lp, A):
        m = fv.Model(lp, A)
        return float(fv.decode([m], fv.Batch([T], E=Ed, models=[m]))[1][0].item())

    m = fv.Model(log_pi, logA)
    b = fv.Batch([T], E=Ed, models=[m])
    paths = fv.decode([m], b)[0].clone()
    dpi, dA, _ = fv.backward(m, b, paths, torch.ones(1, device="cuda"))
    dA = dA.cpu().numpy()
    h = 1e-2
    for (i, j) in [(int(paths[t - 1]), int(paths[t])) for t in (5, 20, 40)] + [(0, 1), (3, 7)]:
        Ap, Am = logA.copy(), logA.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (score(log_pi, Ap) - score(log_pi, Am)) / (2 * h)
        assert abs(fd - dA[i, j]) < 0.05, (i, j, fd, dA[i, j])


def test_autograd_crf_step_config4_subset(fv):
    """Differentiable decoding step: E = X W^T + b from 256-dim features,
    scores through ViterbiScore (FLASH forward), gradients to W, b, logA and
    logpi; checked against the oracle's gradient on the decoded paths."""
    c = W.config4(n_seq=64)
    K = c["K"]
    lengths = c["T"]
    torch.backends.cuda.matmul.allow_tf32 = False
    X = torch.from_numpy(c["X"]).cuda()
    Wt = torch.from_numpy(c["W"]).cuda().requires_grad_(True)
    bt = torch.from_numpy(c["b"]).cuda().requires_grad_(True)
    logA = torch.from_numpy(c["logA"]).cuda().requires_grad_(True)
    log_pi = torch.from_numpy(c["log_pi"]).cuda().requires_grad_(True)
    E = X @ Wt.T + bt
    g = torch.from_numpy(np.random.default_rng(1).standard_normal(len(lengths)).astype(np.float32)).cuda()
    scores = fv.ViterbiScore.apply(log_pi, logA, E, lengths, "flash", 16)
    (scores * g).sum().backward()
    # oracle on the same inputs
    En = E.detach().cpu().numpy()
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    off = np.concatenate([[0], np.cumsum(lengths)])
    res = oracle.map_sequences(lambda i: oracle.viterbi(hmm, En[off[i]:off[i + 1]]), range(len(lengths)))
    paths = np.concatenate([r[0] for r in res])
    assert np.array_equal(bits(scores.detach().cpu().numpy()), bits(np.array([r[1] for r in res])))
    opi, oA, oE = oracle.grad(K, lengths, paths, g.cpu().numpy())
    assert np.array_equal(bits(logA.grad.cpu().numpy()), bits(oA))
    assert np.array_equal(bits(log_pi.grad.cpu().numpy()), bits(opi))
    # dE flows into the linear layer: db = sum_rows dE
    assert torch.allclose(bt.grad.cpu(), torch.from_numpy(oE.reshape(-1, K).sum(0)), atol=1e-4)


def test_path_score_recompute_equals_returned_score(fv):
    """fv_path_score (forward-order log-likelihood) of the decoded path is
    the returned score, bit for bit, for every mode; and matches the
    oracle's path score on arbitrary paths (dense and CSR)."""
    rng = np.random.default_rng(4)
    K = 96
    log_pi, logA = W.random_model(K, rng)
    lengths = rng.integers(1, 300, 25)
    E = torch.from_numpy(W.gaussian_emissions(int(lengths.sum()), K, rng)).cuda()
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=E, models=[m])
    for mode, kw in (("vanilla", {}), ("flash", {"P": 8}), ("beam", {"B": 10, "P": 0}), ("beam", {"B": 10, "P": 4})):
        paths, scores = [x.clone() for x in fv.decode([m], b, mode=mode, **kw)]
        rec = fv.path_score([m], b, paths)
        assert torch.equal(rec[:b.n].view(torch.int32), scores[:b.n].view(torch.int32)), mode
    rp, col, val = W.random_csr(K, 8, rng)
    mc = fv.Model(log_pi, row_ptr=rp, col=col, val=val)
    hc = oracle.HMM(log_pi, None, rp, col, val)
    bc = fv.Batch(lengths, E=E, models=[mc])
    rand = rng.integers(0, K, int(lengths.sum())).astype(np.int32)
    rec = fv.path_score([mc], bc, torch.from_numpy(rand).cuda()).cpu().numpy()
    En = E.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(lengths)])
    for i in range(len(lengths)):
        want = oracle.path_score(hc, En[off[i]:off[i + 1]], rand[off[i]:off[i + 1]])
        assert bits(rec[i]) == bits(want)
