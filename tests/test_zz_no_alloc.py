"""fv_decode_noalloc: exact decoding for callers that may not allocate device
memory at decode time (fixed start-up budgets, plug-ins whose host owns the
allocator, latency-critical paths).  Its scratch is a static device array
shared by every call, so this test checks two calls in a row against
fv_decode on the same inputs, bit for bit, and that an oversize request is
refused.  Kept in a file of its own that is collected last."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call_noalloc(fv, models, batch, n_paths):
    lib = fv._lib.load(build_if_missing=True)
    arr = fv._models_array(models)
    bs = batch.struct()
    paths = torch.full((max(n_paths, 1),), -1, dtype=torch.int32, device="cuda")
    scores = torch.full((max(batch.n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    rc = lib.fv_decode_noalloc(arr, len(models), ctypes.byref(bs), ctypes.c_void_p(paths.data_ptr()),
                               ctypes.c_void_p(scores.data_ptr()), ctypes.c_void_p(st.cuda_stream))
    torch.cuda.synchronize()
    return rc, paths, scores


def test_noalloc_matches_decode_on_two_calls_in_a_row():
    import paper_2510_19301_gb300 as fv
    fv._lib.load(build_if_missing=True)
    rng = np.random.default_rng(77)
    for K, lengths in ((64, [1000]), (256, list(rng.integers(1, 600, 24)))):
        log_pi, logA = W.random_model(K, rng)
        E = torch.from_numpy(W.gaussian_emissions(int(np.sum(lengths)), K, rng)).cuda()
        m = fv.Model(log_pi, logA)
        b = fv.Batch(lengths, E=E, models=[m])
        want_p, want_s = [x.clone() for x in fv.decode([m], b)]
        for _ in range(2):
            rc, p, s = _call_noalloc(fv, [m], b, b.path_len)
            assert rc == fv._lib.FV_OK
            assert torch.equal(p[:b.path_len], want_p[:b.path_len])
            assert torch.equal(s[:b.n].view(torch.int32), want_s[:b.n].view(torch.int32))


def test_noalloc_rejects_oversize_request():
    import paper_2510_19301_gb300 as fv
    K = 256
    rng = np.random.default_rng(3)
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    lengths = [40000]  # 40000 * 256 * 2 bytes of backpointers > 16 MiB
    E = torch.zeros((lengths[0], K), dtype=torch.float32, device="cuda")
    b = fv.Batch(lengths, E=E, models=[m])
    rc, _, _ = _call_noalloc(fv, [m], b, b.path_len)
    assert rc == fv._lib.FV_ENOMEM
