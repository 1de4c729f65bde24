"""GB300-native FLASH Viterbi (arXiv 2510.19301): Python binding over libfv.

Everything here marshals arguments for the C ABI in ``include/fv.h``; every
step of the decoding path runs in libfv's sm_103a kernels.  PyTorch provides
device memory and streams only.  There is no CPU fallback: if libfv.so is
missing, the calls raise.

    m = Model(log_pi, logA)                        # device tensors
    b = Batch(lengths, E=E_packed)                 # E: [sum T, K] float32
    paths, scores = decode([m], b, mode="flash", P=16)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from ._lib import FVError

__all__ = ["Model", "Batch", "Decoder", "decode", "path_score", "workspace_size", "backward",
           "ViterbiScore", "FVError", "MODES", "autotune", "set_engine_variant"]

MODES = {"vanilla": L.FV_VANILLA, "flash": L.FV_FLASH, "beam": L.FV_BEAM, "checkpoint": L.FV_CHECKPOINT}


def _f32(x, device):
    return torch.as_tensor(x, dtype=torch.float32, device=device).contiguous()


def _i32(x, device):
    return torch.as_tensor(x, dtype=torch.int32, device=device).contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Model:
    """One HMM lambda = (pi, A, B) held on the device.

    Dense transitions: ``logA`` [K, K] (row = source).  CSR transitions:
    ``row_ptr`` [K+1], ``col`` [nnz], ``val`` [nnz] (out-edges, sorted
    columns).  Discrete emissions: ``logB`` [K, V]; otherwise the batch
    supplies emission scores directly."""

    def __init__(self, log_pi, logA=None, *, row_ptr=None, col=None, val=None, logB=None,
                 device="cuda"):
        self.log_pi = _f32(log_pi, device)
        self.K = int(self.log_pi.shape[0])
        self.logA = None if logA is None else _f32(logA, device).reshape(self.K, self.K)
        self.row_ptr = None if row_ptr is None else _i32(row_ptr, device)
        self.col = None if col is None else _i32(col, device)
        self.val = None if val is None else _f32(val, device)
        self.logB = None if logB is None else _f32(logB, device)
        if self.logA is None and self.row_ptr is None:
            raise ValueError("need logA (dense) or row_ptr/col/val (CSR)")

    @property
    def csr(self):
        return self.logA is None

    def struct(self):
        m = L.fv_model()
        m.K = self.K
        m.log_pi = _ptr(self.log_pi)
        m.trans = L.FV_TRANS_CSR if self.csr else L.FV_TRANS_DENSE
        m.logA = _ptr(self.logA)
        m.row_ptr, m.col, m.val = _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val)
        m.nnz = 0 if self.col is None else int(self.col.numel())
        m.emit = L.FV_EMIT_DISCRETE if self.logB is not None else L.FV_EMIT_DENSE
        m.V = 0 if self.logB is None else int(self.logB.shape[1])
        m.logB = _ptr(self.logB)
        return m


class Batch:
    """Sequences of uneven length, packed.

    ``lengths``: T_b per sequence.  Dense emissions ``E``: float32 tensor
    whose sequence b starts at element ``e_off[b]`` (default: packed rows
    [sum T_b, K_b]).  Discrete: ``obs`` int32 symbols, packed.  Paths are
    returned packed in the same order (``path_off``)."""

    def __init__(self, lengths, *, E=None, obs=None, model_index=None, models=None,
                 e_off=None, path_off=None, device="cuda"):
        self.T_host = np.ascontiguousarray(np.asarray(lengths, dtype=np.int32).reshape(-1))
        self.n = int(self.T_host.shape[0])
        self.model_host = None if model_index is None else np.ascontiguousarray(
            np.asarray(model_index, dtype=np.int32).reshape(-1))
        Ks = None
        if models is not None:
            Ks = np.array([m.K for m in models], np.int64)
        T64 = self.T_host.astype(np.int64)
        if path_off is None:
            path_off = np.zeros(self.n, np.int64)
            if self.n:
                path_off[1:] = np.cumsum(T64)[:-1]
        if e_off is None:
            if obs is not None:
                e_off = path_off.copy()
            else:
                if Ks is None:
                    if E is None or E.dim() != 2:
                        raise ValueError("pass models= or a 2-D packed E to derive offsets")
                    kk = np.full(self.n, int(E.shape[1]), np.int64)
                else:
                    mi = self.model_host if self.model_host is not None else np.zeros(self.n, np.int64)
                    kk = Ks[mi]
                e_off = np.zeros(self.n, np.int64)
                if self.n:
                    e_off[1:] = np.cumsum(T64 * kk)[:-1]
        self.e_off_host = np.asarray(e_off, np.int64)
        self.path_off_host = np.asarray(path_off, np.int64)
        self.total_steps = int(T64.sum())
        self.path_len = int((self.path_off_host + T64).max()) if self.n else 0
        self.T = _i32(self.T_host, device)
        self.model_idx = None if self.model_host is None else _i32(self.model_host, device)
        self.e_off = torch.as_tensor(self.e_off_host, dtype=torch.int64, device=device)
        self.path_off = torch.as_tensor(self.path_off_host, dtype=torch.int64, device=device)
        self.E = None if E is None else E.contiguous()
        if self.E is not None and self.E.dtype != torch.float32:
            raise TypeError("E must be float32")
        self.obs = None if obs is None else _i32(obs, device)
        self.device = device

    def struct(self):
        b = L.fv_batch()
        b.n_seq = self.n
        b.T_host = self.T_host.ctypes.data_as(ctypes.c_void_p)
        b.model_host = None if self.model_host is None else self.model_host.ctypes.data_as(ctypes.c_void_p)
        b.T = _ptr(self.T)
        b.model_idx = _ptr(self.model_idx)
        b.e_off = _ptr(self.e_off)
        b.E = _ptr(self.E)
        b.obs = _ptr(self.obs)
        b.path_off = _ptr(self.path_off)
        return b


def _params(mode, P, B, mem_budget, flags):
    p = L.fv_params()
    p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    p.P, p.B = int(P), int(B)
    p.mem_budget_bytes = int(mem_budget)
    p.flags = int(flags)
    return p


def _models_array(models):
    arr = (L.fv_model * len(models))()
    for i, m in enumerate(models):
        arr[i] = m.struct()
    return arr


def workspace_size(models, batch, mode="vanilla", P=1, B=0, mem_budget=0, flags=0):
    lib = L.load()
    arr = _models_array(models)
    bs = batch.struct()
    ps = _params(mode, P, B, mem_budget, flags)
    return int(lib.fv_workspace_size(arr, len(models), ctypes.byref(bs), ctypes.byref(ps)))


class Decoder:
    """A prepared decode call: structs, workspace and outputs are built once
    so that repeated launches cost one C call each (used by the benchmark)."""

    def __init__(self, models, batch, mode="vanilla", P=1, B=0, mem_budget=0, flags=0,
                 workspace=None, paths=None, scores=None):
        self.lib = L.load()
        self.models = list(models)
        self.batch = batch
        self._arr = _models_array(self.models)
        self._bs = batch.struct()
        self._ps = _params(mode, P, B, mem_budget, flags)
        self.ws_bytes = int(self.lib.fv_workspace_size(self._arr, len(self.models), ctypes.byref(self._bs),
                                                       ctypes.byref(self._ps)))
        if self.ws_bytes == 0:
            raise FVError(L.FV_EINVAL, "fv_workspace_size")
        dev = batch.device
        self.workspace = workspace if workspace is not None else torch.empty(
            self.ws_bytes, dtype=torch.uint8, device=dev)
        if self.workspace.data_ptr() % 256:
            raise ValueError("workspace must be 256-byte aligned")
        self.paths = paths if paths is not None else torch.empty(max(batch.path_len, 1), dtype=torch.int32,
                                                                  device=dev)
        self.scores = scores if scores is not None else torch.empty(max(batch.n, 1), dtype=torch.float32,
                                                                     device=dev)

    def launch(self, stream=None):
        st = stream if stream is not None else torch.cuda.current_stream()
        rc = self.lib.fv_decode(self._arr, len(self.models), ctypes.byref(self._bs), ctypes.byref(self._ps),
                                _ptr(self.workspace), self.workspace.numel(), _ptr(self.paths),
                                _ptr(self.scores), ctypes.c_void_p(st.cuda_stream))
        if rc != L.FV_OK:
            raise FVError(rc, "fv_decode")

    def device_status(self, stream=None):
        st = stream if stream is not None else torch.cuda.current_stream()
        return int(self.lib.fv_last_device_status(_ptr(self.workspace), ctypes.c_void_p(st.cuda_stream)))

    def __call__(self, stream=None, check=True):
        self.launch(stream)
        if check:
            s = self.device_status(stream)
            if s != L.FV_OK:
                raise FVError(s, "fv_decode (device)")
        return self.paths, self.scores


def autotune(models, batch, mode="vanilla", P=1, B=0, mem_budget=0, flags=0, stream=None):
    """Time every engine configuration of the K classes in this request and
    keep the fastest for later decodes in this process (fv_autotune).
    Returns the chosen variant per model."""
    if isinstance(models, Model):
        models = [models]
    d = Decoder(models, batch, mode=mode, P=P, B=B, mem_budget=mem_budget, flags=flags)
    st = stream if stream is not None else torch.cuda.current_stream()
    chosen = (ctypes.c_int32 * len(d.models))()
    rc = d.lib.fv_autotune(d._arr, len(d.models), ctypes.byref(d._bs), ctypes.byref(d._ps), _ptr(d.workspace),
                           d.workspace.numel(), _ptr(d.paths), _ptr(d.scores), ctypes.c_void_p(st.cuda_stream),
                           chosen)
    if rc != L.FV_OK:
        raise FVError(rc, "fv_autotune")
    return list(chosen)


def set_engine_variant(K, variant):
    """Force the engine variant of K's class (0 = default); returns the
    number of variants of that class."""
    return int(L.load().fv_set_engine_variant(int(K), int(variant)))


def decode(models, batch, mode="vanilla", P=1, B=0, mem_budget=0, flags=0, stream=None, check=True):
    """Decode every sequence; returns (paths int32 [packed], scores float32 [n])."""
    if isinstance(models, Model):
        models = [models]
    d = Decoder(models, batch, mode, P, B, mem_budget, flags)
    return d(stream, check)


def backward(model, batch, paths, grad_scores, stream=None):
    """Gradient of sum_b g_b * score_b with the paths held fixed:
    (dlog_pi [K], dlogA [K, K], dE like batch.E).  Deterministic (terms
    added in ascending sequence order)."""
    lib = L.load()
    arr = _models_array([model])
    bs = batch.struct()
    dev = batch.device
    g = _f32(grad_scores, dev)
    dpi = torch.empty(model.K, dtype=torch.float32, device=dev)
    dA = torch.empty((model.K, model.K), dtype=torch.float32, device=dev)
    dE = torch.zeros_like(batch.E)
    wsz = int(lib.fv_backward_workspace_size(arr, 1, ctypes.byref(bs)))
    if wsz == 0:
        raise FVError(L.FV_EINVAL, "fv_backward_workspace_size")
    ws = torch.empty(wsz, dtype=torch.uint8, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.fv_backward(arr, 1, ctypes.byref(bs), _ptr(paths), _ptr(g), _ptr(dpi), _ptr(dA), _ptr(dE),
                         _ptr(ws), ws.numel(), ctypes.c_void_p(st.cuda_stream))
    if rc != L.FV_OK:
        raise FVError(rc, "fv_backward")
    s_ = int(lib.fv_last_device_status(_ptr(ws), ctypes.c_void_p(st.cuda_stream)))
    if s_ != L.FV_OK:
        raise FVError(s_, "fv_backward (device)")
    return dpi, dA, dE


class ViterbiScore(torch.autograd.Function):
    """scores = ViterbiScore.apply(log_pi, logA, E, lengths[, mode, P]).

    Forward decodes every sequence (FLASH by default, so only the paths are
    kept: O(P K) working memory per sequence instead of the T x K table) and
    returns the Viterbi scores; backward scatters the path counts
    (structured-perceptron / CRF-style training)."""

    @staticmethod
    def forward(ctx, log_pi, logA, E, lengths, mode="flash", P=16):
        m = Model(log_pi.detach(), logA.detach(), device=E.device)
        b = Batch(lengths, E=E.detach().reshape(-1), models=[m], device=E.device)
        paths, scores = decode([m], b, mode=mode, P=P)
        ctx.save_for_backward(paths)
        ctx.model, ctx.batch, ctx.E_shape = m, b, E.shape
        return scores[: b.n].clone()

    @staticmethod
    def backward(ctx, grad_scores):
        (paths,) = ctx.saved_tensors
        dpi, dA, dE = backward(ctx.model, ctx.batch, paths, grad_scores.contiguous())
        return dpi, dA, dE.reshape(ctx.E_shape), None, None, None


def path_score(models, batch, paths, stream=None):
    """Log-likelihood of given paths in the forward order (Sec. III-A)."""
    if isinstance(models, Model):
        models = [models]
    lib = L.load()
    arr = _models_array(models)
    bs = batch.struct()
    out = torch.empty(max(batch.n, 1), dtype=torch.float32, device=batch.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.fv_path_score(arr, len(models), ctypes.byref(bs), _ptr(paths), _ptr(out),
                           ctypes.c_void_p(st.cuda_stream))
    if rc != L.FV_OK:
        raise FVError(rc, "fv_path_score")
    return out


def maxplus_peak(iters=20000, stream=None):
    """Measured max-plus ceiling of this GPU (fv_maxplus_peak): returns
    (cells per second, cells per clock per SM, SM count)."""
    lib = L.load()
    cps = ctypes.c_double(0.0)
    cpc = ctypes.c_double(0.0)
    sms = ctypes.c_int32(0)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.fv_maxplus_peak(int(iters), ctypes.byref(cps), ctypes.byref(cpc), ctypes.byref(sms),
                             ctypes.c_void_p(st.cuda_stream))
    if rc != L.FV_OK:
        raise FVError(rc, "fv_maxplus_peak")
    return cps.value, cpc.value, sms.value
