"""The paper's Erdos-Renyi workload family (Sec. VI): generator structure,
and the oracle's exact decoders agreeing on these -inf-heavy transition
matrices (FLASH and the full-width beam reproduce vanilla bit for bit,
Sec. V-B.3 and V-C; the returned score is the forward-order score of the
returned path, Sec. III-A)."""
import numpy as np
import pytest

import oracle
import workloads as W


def bits(a):
    return np.asarray(a, np.float32).view(np.int32)


@pytest.mark.parametrize("K,p", [(64, 0.05), (256, 0.253), (512, 0.253), (128, 1.0)])
def test_er_generator_structure(K, p):
    c = W.erdos_renyi_case(K, 50, p, seed=11)
    A = c["logA"]
    finite = np.isfinite(A)
    # every state keeps an out-edge; density is p plus the forced edge
    assert finite.any(axis=1).all()
    expect = p + (1.0 - p) / K
    assert abs(finite.mean() - expect) < 4.0 * np.sqrt(expect * (1 - expect) / A.size) + 1e-9
    # rows are distributions over the present edges
    rows = np.exp(A.astype(np.float64)).sum(axis=1)
    assert np.allclose(rows, 1.0, atol=1e-5)
    assert np.allclose(np.exp(c["log_pi"].astype(np.float64)).sum(), 1.0, atol=1e-5)
    assert np.allclose(np.exp(c["logB"].astype(np.float64)).sum(axis=1), 1.0, atol=1e-5)
    assert c["obs"].dtype == np.int32 and c["obs"].min() >= 0 and c["obs"].max() < c["V"]
    # seeded
    d = W.erdos_renyi_case(K, 50, p, seed=11)
    assert np.array_equal(bits(A), bits(d["logA"])) and np.array_equal(c["obs"], d["obs"])


def test_er_sweep_ranges_match_the_paper():
    assert W.ER_DEFAULT == dict(K=512, T=512, p=0.253, V=50)
    ps = W.ER_P_SWEEP
    assert ps[0] == 0.05 and ps[-1] == 1.0
    assert all(abs(b / a - 1.5) < 1e-12 for a, b in zip(ps[:-2], ps[1:-1]))
    assert any(abs(x - 0.253) < 1e-3 for x in ps)
    assert W.ER_SIZE_SWEEP[0] == 32 and W.ER_SIZE_SWEEP[-1] == 2048
    assert W.ER_BEAM_SWEEP[0] == 1024 and W.ER_BEAM_SWEEP[-1] == 32


@pytest.mark.parametrize("p", [0.05, 0.253, 1.0])
def test_er_oracle_exact_variants_agree(p):
    K, T = 24, 41
    c = W.erdos_renyi_case(K, T, p, seed=5)
    hmm = oracle.HMM(c["log_pi"], c["logA"])
    E = oracle.expand_discrete(c["logB"], c["obs"])
    pv, sv = oracle.viterbi(hmm, E)
    assert np.isfinite(sv)
    assert bits(oracle.path_score(hmm, E, pv)) == bits(sv)
    for P in (1, 4, 16, T):
        pf, sf, _ = oracle.flash(hmm, E, P)
        assert np.array_equal(pf, pv) and bits(sf) == bits(sv)
    pb, sb, st = oracle.beam(hmm, E, K)
    assert st == 0 and np.array_equal(pb, pv) and bits(sb) == bits(sv)
    pfs, sfs, _, st = oracle.flash_bs(hmm, E, 4, K)
    assert st == 0 and np.array_equal(pfs, pv) and bits(sfs) == bits(sv)
