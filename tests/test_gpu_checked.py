"""FV_CHECKED: NaN or +inf in any score array, a malformed CSR graph or an
out-of-range symbol is found on the device before decoding and reported
as FV_EINVAL in the status word; -inf is accepted, and clean inputs decode
exactly as without the flag."""
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


def status_of(fv, models, b, **kw):
    d = fv.Decoder(models, b, flags=fv._lib.FV_CHECKED, **kw)
    d.launch()
    torch.cuda.synchronize()
    return d


def dense_case(K=64, lengths=(5, 40, 17), seed=0):
    rng = np.random.default_rng(seed)
    log_pi, logA = W.random_model(K, rng)
    E = np.concatenate([W.gaussian_emissions(t, K, rng) for t in lengths])
    return log_pi, logA, E, list(lengths)


@pytest.mark.parametrize("mode", ["vanilla", "flash", "beam"])
def test_checked_rejects_nan_and_pos_inf(fv, mode):
    L = fv._lib
    kw = {"vanilla": {}, "flash": {"P": 4}, "beam": {"B": 8, "P": 0}}[mode]
    for where in ("logA", "log_pi", "E_nan", "E_inf"):
        log_pi, logA, E, lengths = dense_case()
        if where == "logA":
            logA[3, 7] = np.nan
        elif where == "log_pi":
            log_pi[5] = np.inf
        elif where == "E_nan":
            E[50, 2] = np.nan
        else:
            E[-1, 0] = np.inf
        m = fv.Model(log_pi, logA)
        b = fv.Batch(lengths, E=torch.from_numpy(E).cuda(), models=[m])
        d = status_of(fv, [m], b, mode=mode, **kw)
        assert d.device_status() == L.FV_EINVAL, (mode, where)


def test_checked_accepts_neg_inf_and_matches_unchecked(fv):
    log_pi, logA, E, lengths = dense_case(seed=1)
    logA[np.random.default_rng(2).random(logA.shape) < 0.3] = -np.inf
    E[10, :5] = -np.inf
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(E).cuda(), models=[m])
    d = status_of(fv, [m], b)
    assert d.device_status() == 0
    p0, s0 = fv.decode([m], b)
    assert torch.equal(d.paths, p0) and torch.equal(d.scores.view(torch.int32), s0.view(torch.int32))
    hmm = oracle.HMM(log_pi, logA)
    off = 0
    for i, t in enumerate(lengths):
        p, s = oracle.viterbi(hmm, E[off:off + t])
        assert np.array_equal(d.paths.cpu().numpy()[off:off + t], p)
        off += t


def test_checked_rejects_malformed_csr_and_symbols(fv):
    L = fv._lib
    rng = np.random.default_rng(3)
    K = 100
    rp, col, val = W.random_csr(K, 5, rng)
    log_pi = W._log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    lengths = [7, 9]
    E = torch.from_numpy(np.concatenate([W.gaussian_emissions(t, K, rng) for t in lengths])).cuda()
    bad_col = col.copy()
    bad_col[17] = K + 3
    m = fv.Model(log_pi, row_ptr=rp, col=bad_col, val=val)
    b = fv.Batch(lengths, E=E, models=[m])
    assert status_of(fv, [m], b, mode="beam", B=16, P=0).device_status() == L.FV_EINVAL
    bad_rp = rp.copy()
    bad_rp[40], bad_rp[41] = bad_rp[41], bad_rp[40]
    m = fv.Model(log_pi, row_ptr=bad_rp, col=col, val=val)
    b = fv.Batch(lengths, E=E, models=[m])
    assert status_of(fv, [m], b, mode="beam", B=16, P=0).device_status() == L.FV_EINVAL
    # discrete emissions: a symbol outside [0, V)
    Kd, V = 16, 8
    lp, A = W.random_model(Kd, rng)
    logB = W._log_dirichlet(rng, 0.5, (Kd, V)).astype(np.float32)
    obs = rng.integers(0, V, 30).astype(np.int32)
    obs[12] = V
    md = fv.Model(lp, A, logB=logB)
    bd = fv.Batch([30], obs=obs, models=[md])
    assert status_of(fv, [md], bd).device_status() == L.FV_EINVAL
