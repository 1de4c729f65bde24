"""Serving loop on the GPU: requests of mixed K and T, exact and beam,
arrive over time, are packed per class into shared launches and overlap on
the device; every result must equal the result of decoding that request
alone (bit for bit), a sample of served requests of each mode must equal
the oracle, and latency percentiles are reported."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bits(x):
    return np.float32(x).view(np.int32)


@pytest.mark.parametrize("shared", [True, False])
def test_results_in_the_mix_equal_results_alone(shared):
    import paper_2510_19301_gb300 as fv
    from paper_2510_19301_gb300.serve import GpuBackend, Server, poisson_requests
    fv._lib.load(build_if_missing=True)
    reqs = poisson_requests(rate=2000.0, seconds=0.04, seed=11, Ks=(64, 256, 1024), tmin=20, tmax=600)
    assert len(reqs) > 30
    be = GpuBackend(n_streams=16, keep_results=True, shared_models=shared)
    # engine configurations tuned on a short launch per K class (results do
    # not depend on them: the alone-decodes below use the same library)
    tuned = be.tune((64, 256, 1024), T=200, n=4)
    assert set(tuned) == {64, 256, 1024}
    assert all(0 <= v < fv.set_engine_variant(K, v) for K, v in tuned.items())
    srv = Server(be, mem_budget_bytes=4 << 30, max_inflight=16)
    rep = srv.run(reqs)
    assert rep["failed"] == 0 and rep["requests"] == len(reqs)
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    assert rep["launches"] < len(reqs), "no launch carried more than one request"
    overlapped = sum(1 for r in srv.done
                     if r.admitted < max((o.finished for o in srv.done if o.rid < r.rid), default=-1.0))
    assert overlapped > 0, "no request ran while another was on the GPU"
    # alone: same seeded inputs, one request at a time on the default stream
    checked = {"exact": 0, "beam": 0}
    for r in srv.done:
        log_pi, logA, E = be.make_inputs(r)
        m = fv.Model(log_pi, logA)
        b = fv.Batch([r.T], E=E.view(-1), models=[m])
        mode = {"exact": "vanilla", "beam": "beam"}[r.mode]
        p, s = fv.decode([m], b, mode=mode, B=r.B if r.mode == "beam" else 0, P=0 if r.mode == "beam" else 1)
        pm, sm = r.result
        assert np.array_equal(p[:r.T].cpu().numpy(), pm), r
        assert bits(s[0].item()) == bits(sm)
        # the oracle on a few requests of each mode
        if checked[r.mode] < 3 and r.T <= 300:
            hmm = oracle.HMM(log_pi.cpu().numpy(), logA.cpu().numpy())
            e = E.cpu().numpy()
            ref = oracle.viterbi(hmm, e) if r.mode == "exact" else oracle.beam(hmm, e, r.B)
            assert np.array_equal(ref[0], pm) and bits(ref[1]) == bits(sm), r
            checked[r.mode] += 1
    assert checked["exact"] >= 1 and checked["beam"] >= 1
