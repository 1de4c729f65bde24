"""C-ABI boundary checks that need no GPU: the library builds, loads and
exports every function include/fv.h declares; argument errors come back at
once without touching the device; workspace sizes follow the documented
layout."""
import ctypes

import numpy as np
import pytest

from paper_2510_19301_gb300 import _lib as L
from paper_2510_19301_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_exports_every_declared_function(lib):
    names = L.declared_functions()
    assert "fv_decode" in names and "fv_backward" in names and "fv_workspace_size" in names
    for n in names:
        assert hasattr(lib, n), f"libfv.so does not export {n}"


def test_header_constants_match_binding():
    """Every flag, status and enum value include/fv.h defines has the same
    value in the Python binding."""
    import re
    src = open(L.HEADER).read()
    defines = dict(re.findall(r"#define\s+(FV_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", src))
    assert "FV_SHARED_GPU" in defines and "FV_STATIC_BEAM" in defines
    for name, v in defines.items():
        assert getattr(L, name) == int(v, 0), name
    for name, v in re.findall(r"\b(FV_[A-Z0-9_]+)\s*=\s*(\d+)", src):
        assert getattr(L, name) == int(v), name


def test_status_strings(lib):
    for s in range(7):
        assert lib.fv_status_str(s)
    assert b"sm_103a" in lib.fv_version()


FAKE = ctypes.c_void_p(0x10000)  # never dereferenced by the calls below


def _model(K=8, dense=True):
    m = L.fv_model()
    m.K = K
    m.log_pi = FAKE
    m.trans = L.FV_TRANS_DENSE if dense else L.FV_TRANS_CSR
    m.logA = FAKE if dense else None
    if not dense:
        m.row_ptr = m.col = m.val = FAKE
        m.nnz = 4 * K
    m.emit = L.FV_EMIT_DENSE
    return m


def _batch(T):
    T = np.ascontiguousarray(np.asarray(T, np.int32))
    b = L.fv_batch()
    b.n_seq = len(T)
    b.T_host = T.ctypes.data_as(ctypes.c_void_p)
    b.T = b.e_off = b.path_off = b.E = FAKE
    return b, T


def _params(mode=L.FV_VANILLA, P=1, B=0):
    p = L.fv_params()
    p.mode, p.P, p.B = mode, P, B
    return p


def test_workspace_size_vanilla_layout(lib):
    m = (L.fv_model * 1)(_model(K=10))
    b, T = _batch([3, 1, 17])
    sz = lib.fv_workspace_size(m, 1, ctypes.byref(b), ctypes.byref(_params()))
    aux = sum(((t * 10 + 7) // 8) * 8 for t in T) * 2
    assert sz >= aux and sz % 256 == 0
    b2, _ = _batch([3, 1, 18])
    assert lib.fv_workspace_size(m, 1, ctypes.byref(b2), ctypes.byref(_params())) >= sz


def test_argument_errors_return_at_once(lib):
    m = (L.fv_model * 1)(_model())
    b, T = _batch([4, 5])
    p = _params()
    ws = ctypes.c_void_p(0x100000)
    # null models / batch / params
    assert lib.fv_decode(None, 1, ctypes.byref(b), ctypes.byref(p), ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL
    assert lib.fv_decode(m, 1, None, ctypes.byref(p), ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL
    assert lib.fv_decode(m, 1, ctypes.byref(b), None, ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL
    # T < 1
    bad, _ = _batch([4, 0])
    assert lib.fv_decode(m, 1, ctypes.byref(bad), ctypes.byref(p), ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL
    assert lib.fv_workspace_size(m, 1, ctypes.byref(bad), ctypes.byref(p)) == 0
    # unaligned workspace
    assert lib.fv_decode(m, 1, ctypes.byref(b), ctypes.byref(p), ctypes.c_void_p(0x100010), 1 << 20,
                         FAKE, FAKE, None) == L.FV_EINVAL
    # workspace too small for the declared lengths (checked on the host)
    long_b, _ = _batch([4000, 5000])
    assert lib.fv_decode(m, 1, ctypes.byref(long_b), ctypes.byref(p), ws, 8192, FAKE, FAKE, None) == L.FV_ENOMEM
    # K out of range
    big = (L.fv_model * 1)(_model(K=70000))
    assert lib.fv_decode(big, 1, ctypes.byref(b), ctypes.byref(p), ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL
    # bad mode and knobs
    assert lib.fv_decode(m, 1, ctypes.byref(b), ctypes.byref(_params(mode=7)), ws, 1 << 20, FAKE, FAKE,
                         None) == L.FV_EINVAL
    assert lib.fv_decode(m, 1, ctypes.byref(b), ctypes.byref(_params(mode=L.FV_FLASH, P=0)), ws, 1 << 20,
                         FAKE, FAKE, None) == L.FV_EINVAL
    assert lib.fv_decode(m, 1, ctypes.byref(b), ctypes.byref(_params(mode=L.FV_BEAM, B=0)), ws, 1 << 20,
                         FAKE, FAKE, None) == L.FV_EINVAL
    # several models need per-sequence model indices
    m2 = (L.fv_model * 2)(_model(), _model())
    assert lib.fv_decode(m2, 2, ctypes.byref(b), ctypes.byref(p), ws, 1 << 20, FAKE, FAKE, None) == L.FV_EINVAL


def test_noalloc_argument_refusals(lib):
    """fv_decode_noalloc refuses, before any CUDA call: missing host lengths,
    CSR models, and requests larger than its static scratch."""
    m = (L.fv_model * 1)(_model())
    b, T = _batch([4, 5])
    b.T_host = None
    assert lib.fv_decode_noalloc(m, 1, ctypes.byref(b), FAKE, FAKE, None) == L.FV_EINVAL
    b, T = _batch([4, 5])
    csr = (L.fv_model * 1)(_model(dense=False))
    assert lib.fv_decode_noalloc(csr, 1, ctypes.byref(b), FAKE, FAKE, None) == L.FV_EUNSUPPORTED
    big, Tb = _batch([40000])
    m256 = (L.fv_model * 1)(_model(K=256))
    assert lib.fv_decode_noalloc(m256, 1, ctypes.byref(big), FAKE, FAKE, None) == L.FV_ENOMEM


def test_empty_batch_is_ok_without_device_work(lib):
    m = (L.fv_model * 1)(_model())
    b, _ = _batch([])
    p = _params()
    assert lib.fv_decode(m, 1, ctypes.byref(b), ctypes.byref(p), ctypes.c_void_p(0x100000), 1 << 20,
                         None, None, None) == L.FV_OK


def test_flash_budget_workspace_accounting():
    """The budget adds at most the budget itself (plus the wave table) to the
    FLASH workspace, and none at all when it is below one backpointer row."""
    import ctypes
    from paper_2510_19301_gb300 import _lib as L
    lib = L.load()
    K = 256
    lengths = np.array([1000, 2000, 3000, 500], np.int32)
    m = L.fv_model()
    m.K = K
    m.trans = L.FV_TRANS_DENSE
    m.emit = L.FV_EMIT_DENSE
    m.log_pi = ctypes.c_void_p(256)
    m.logA = ctypes.c_void_p(256)
    b = L.fv_batch()
    b.n_seq = len(lengths)
    b.T_host = lengths.ctypes.data_as(ctypes.c_void_p)
    for f in ("T", "e_off", "E", "path_off"):
        setattr(b, f, ctypes.c_void_p(256))

    def ws(budget):
        p = L.fv_params()
        p.mode = L.FV_FLASH
        p.P = 16
        p.mem_budget_bytes = budget
        return lib.fv_workspace_size(ctypes.byref(m), 1, ctypes.byref(b), ctypes.byref(p))

    base = ws(0)
    assert base > 0
    assert ws(2 * K - 1) == base
    table = int(lengths.sum()) * K * 2
    for budget in (table // 16, table // 64, 10 * 2 * K):
        extra = ws(budget) - base
        assert 0 < extra <= budget + 4096, (budget, extra)
