"""Failure detection without a GPU fault: with the test hook
FV_TEST_WITHHOLD_STEP one CTA of the whole-GPU engine never publishes its
step count, and one CTA of every 4- or 8-CTA cluster of the streamed engine
withholds its arrivals on the delta exchange of the second tick, so the
bounded waits that depend on them run out (about a second).  The call must
report FV_ETIMEOUT through the workspace status word, leave the CUDA context
usable, and the next ordinary call must decode exactly."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("K,variant", [(1100, 0), (300, 0), (300, 1), (1000, 0), (1000, 2), (1000, 3), (200, 0)])
def test_withheld_step_times_out_and_context_survives(K, variant):
    """K=300: variant 0 is the resident 8-CTA cluster configuration of the
    K <= 512 class, variant 1 the streamed 4-CTA one; K=1000 variants 0
    and 3 and K=200 variant 0 run two CTAs per SM, K=1000 variant 2 one
    8-warp CTA; all exchange delta through mbarriers."""
    import paper_2510_19301_gb300 as fv
    from paper_2510_19301_gb300 import _lib as L
    fv._lib.load(build_if_missing=True)
    fv.set_engine_variant(K, variant)
    try:
        _withhold_case(fv, L, K)
    finally:
        fv.set_engine_variant(K, 0)


def _withhold_case(fv, L, K):
    rng = np.random.default_rng(77 + K)
    log_pi, logA = W.random_model(K, rng)
    lengths = [5, 9, 3]
    E_list = [W.gaussian_emissions(t, K, rng) for t in lengths]
    m = fv.Model(log_pi, logA)
    b = fv.Batch(lengths, E=torch.from_numpy(np.concatenate(E_list)).cuda(), models=[m])
    dec = fv.Decoder([m], b, mode="vanilla", flags=L.FV_TEST_WITHHOLD_STEP)
    dec.launch()
    torch.cuda.synchronize()
    assert dec.device_status() == L.FV_ETIMEOUT
    # the context is intact: an ordinary decode right after is exact
    paths, scores = fv.decode([m], b, mode="vanilla")
    paths, scores = paths.cpu().numpy(), scores.cpu().numpy()
    hmm = oracle.HMM(log_pi, logA)
    off = 0
    for i, e in enumerate(E_list):
        p, s = oracle.viterbi(hmm, e)
        assert np.array_equal(paths[off:off + lengths[i]], p)
        assert np.float32(scores[i]).view(np.int32) == np.float32(s).view(np.int32)
        off += lengths[i]
