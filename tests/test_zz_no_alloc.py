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
    # K=64 / 256: resident engines; K=512 / 1024: streamed cluster engines,
    # whose row-pair copy of logA is carved out of the static scratch too.
    for K, lengths in ((64, [1000]), (256, list(rng.integers(1, 600, 24))),
                       (512, [2000, 700, 33]), (1024, [1500, 400])):
        log_pi, logA = W.random_model(K, rng)
        E = torch.from_numpy(W.gaussian_emissions(int(np.sum(lengths)), K, rng)).cuda()
        m = fv.Model(log_pi, logA)
        b = fv.Batch(lengths, E=E, models=[m])
        want_p, want_s = [x.clone() for x in fv.decode([m], b)]
        for _ in range(2):
            rc, p, s = _call_noalloc(fv, [m], b, b.path_len)
            assert rc == fv._lib.FV_OK
            assert fv._lib.load().fv_decode_noalloc_status(
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == fv._lib.FV_OK
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


def test_noalloc_refuses_whole_gpu_engine_sizes():
    """K=2048 needs the whole-GPU engine's buffers and a column-major copy
    of logA, more than the static scratch holds: refused before any work."""
    import paper_2510_19301_gb300 as fv
    K = 2048
    rng = np.random.default_rng(5)
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    E = torch.zeros((100, K), dtype=torch.float32, device="cuda")
    b = fv.Batch([100], E=E, models=[m])
    rc, p, _ = _call_noalloc(fv, [m], b, b.path_len)
    assert rc == fv._lib.FV_ENOMEM
    assert int(p.min()) == -1 and int(p.max()) == -1  # nothing was written


def test_noalloc_reports_device_side_errors():
    """A device length array with an invalid entry (T = 0) while the host
    lengths are valid: the prep kernel records FV_EINVAL in the static
    scratch and no decode kernel runs.  fv_decode_noalloc returns FV_OK
    (the error is found on the device), fv_decode_noalloc_status reports it,
    and the next valid call clears it and decodes exactly."""
    import paper_2510_19301_gb300 as fv
    lib = fv._lib.load(build_if_missing=True)
    K = 64
    rng = np.random.default_rng(9)
    log_pi, logA = W.random_model(K, rng)
    m = fv.Model(log_pi, logA)
    lengths = [300, 200]
    E = torch.from_numpy(W.gaussian_emissions(sum(lengths), K, rng)).cuda()
    b = fv.Batch(lengths, E=E, models=[m])
    want_p, want_s = [x.clone() for x in fv.decode([m], b)]
    bad = b.T.clone()
    bad[1] = 0
    arr = fv._models_array([m])
    bs = b.struct()
    bs.T = ctypes.c_void_p(bad.data_ptr())
    paths = torch.full((b.path_len,), -1, dtype=torch.int32, device="cuda")
    scores = torch.zeros((b.n,), dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.fv_decode_noalloc(arr, 1, ctypes.byref(bs), ctypes.c_void_p(paths.data_ptr()),
                               ctypes.c_void_p(scores.data_ptr()), st)
    assert rc == fv._lib.FV_OK
    assert lib.fv_decode_noalloc_status(st) == fv._lib.FV_EINVAL
    rc, p, s = _call_noalloc(fv, [m], b, b.path_len)
    assert rc == fv._lib.FV_OK
    assert lib.fv_decode_noalloc_status(st) == fv._lib.FV_OK
    assert torch.equal(p[:b.path_len], want_p[:b.path_len])
    assert torch.equal(s[:b.n].view(torch.int32), want_s[:b.n].view(torch.int32))
