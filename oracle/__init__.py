"""CPU oracle for FLASH Viterbi (arXiv 2510.19301) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded C (``fv_oracle.c``) behind ctypes.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the GPU library never does, and the two
share no code.  Every function follows a passage of the paper:

* ``viterbi``      -- Sec. III-A recursion for delta/psi, termination and
                      backtrack (full backpointer table).
* ``flash``        -- Alg. 1 (non-recursive divide and conquer, P-way first
                      split of Sec. V-A.3) over Alg. 2 (subtask decoding) with
                      the pruned initialisation of Sec. V-B.2.
* ``beam``         -- dynamic beam search of Sec. V-C with per-step beam
                      backpointers (P = 0).
* ``flash_bs``     -- FLASH-BS (Sec. V-C on top of Alg. 1/Alg. 2).
* ``beam_static``  -- the static beam the paper contrasts with its dynamic
                      one (Sec. II-B, Sec. V-C.1): all K scores of a step,
                      then the top B of them.
* ``checkpoint``   -- Checkpoint Viterbi, the sqrt(T)-checkpoint baseline of
                      Sec. II-A (forward pass keeping delta at checkpoints,
                      then segments re-decoded latest first).
* ``path_score``   -- log-likelihood of a path in forward order.
* ``grad``         -- path-count gradient (not in the paper).

All arithmetic is FP32 in a fixed order; the readings of points the paper
leaves open are listed at the top of ``fv_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (atomic rename, safe under xdist)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Model(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("log_pi", ctypes.c_void_p),
        ("csr", ctypes.c_int32),
        ("logA", ctypes.c_void_p),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("val", ctypes.c_void_p),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        lib.orc_viterbi.argtypes = [P, i32, P, P, P]
        lib.orc_flash.argtypes = [P, i32, P, i32, i32, P, P, P, P]
        lib.orc_flash_budget.argtypes = [P, i32, P, i32, i32, ctypes.c_int64, P, P, P, P, P]
        lib.orc_flash_budget.restype = ctypes.c_int
        lib.orc_beam.argtypes = [P, i32, P, i32, P, P]
        lib.orc_flash_bs.argtypes = [P, i32, P, i32, i32, i32, P, P, P]
        lib.orc_path_score.argtypes = [P, i32, P, P]
        lib.orc_path_score.restype = ctypes.c_float
        lib.orc_grad.argtypes = [i32, i32, P, P, P, P, P, P, P, P]
        lib.orc_beam_static.argtypes = [P, i32, P, i32, P, P]
        lib.orc_beam_static.restype = ctypes.c_int
        lib.orc_checkpoint.argtypes = [P, i32, P, i32, P, P, P, P]
        lib.orc_checkpoint.restype = ctypes.c_int
        lib.orc_checkpoint_count.argtypes = [i32, i32]
        lib.orc_checkpoint_count.restype = i32
        lib.orc_split_points.argtypes = [i32, i32, P]
        lib.orc_split_points.restype = i32
        for f in (lib.orc_viterbi, lib.orc_flash, lib.orc_beam, lib.orc_flash_bs, lib.orc_grad):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class HMM:
    """Host copy of one model: dense ``logA`` [K,K] (row = source) or CSR
    out-edges (``row_ptr``, ``col``, ``val``)."""

    def __init__(self, log_pi, logA=None, row_ptr=None, col=None, val=None):
        self.log_pi = _f32(log_pi)
        self.K = int(self.log_pi.shape[0])
        self.csr = logA is None
        self.logA = None if self.csr else _f32(logA).reshape(self.K, self.K)
        self.row_ptr = None if not self.csr else _i32(row_ptr)
        self.col = None if not self.csr else _i32(col)
        self.val = None if not self.csr else _f32(val)
        self._s = _Model(self.K, _ptr(self.log_pi), int(self.csr), _ptr(self.logA),
                         _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val))

    @property
    def ref(self):
        return ctypes.byref(self._s)


def _E(E, K):
    E = _f32(E)
    assert E.ndim == 2 and E.shape[1] == K, "E must be [T, K]"
    return E


def expand_discrete(logB, obs):
    """E_t[j] = log B_{j, x_t} (a gather; Sec. III, discrete emissions)."""
    logB = _f32(logB)
    return np.ascontiguousarray(logB[:, np.asarray(obs, dtype=np.int64)].T)


def viterbi(hmm: HMM, E):
    """Exact Viterbi with a full backpointer table -> (path int32[T], score)."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    rc = _load().orc_viterbi(hmm.ref, T, _ptr(E), _ptr(path), _ptr(score))
    if rc:
        raise RuntimeError(f"orc_viterbi failed: {rc}")
    return path, score[0]


def flash(hmm: HMM, E, P: int, complete: bool = False):
    """FLASH Viterbi -> (path, score, tasks[n,3] of (m, n, t_mid) in order)."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    log = np.zeros(3 * T, np.int32)
    n = np.zeros(1, np.int32)
    rc = _load().orc_flash(hmm.ref, T, _ptr(E), int(P), int(complete), _ptr(path),
                           _ptr(score), _ptr(log), _ptr(n))
    if rc:
        raise RuntimeError(f"orc_flash failed: {rc}")
    return path, score[0], log[: 3 * n[0]].reshape(-1, 3)


def flash_budget(hmm: HMM, E, P: int, budget_rows: int, complete: bool = False):
    """FLASH Viterbi whose tasks with n - m <= budget_rows are solved as
    leaves (segment backpointers + backtrack) -> (path, score, n_tasks,
    n_leaves)."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    n = np.zeros(1, np.int32)
    nl = np.zeros(1, np.int32)
    rc = _load().orc_flash_budget(hmm.ref, T, _ptr(E), int(P), int(complete), ctypes.c_int64(int(budget_rows)),
                                  _ptr(path), _ptr(score), None, _ptr(n), _ptr(nl))
    if rc:
        raise RuntimeError(f"orc_flash_budget failed: {rc}")
    return path, score[0], int(n[0]), int(nl[0])


def beam(hmm: HMM, E, B: int):
    """Dynamic beam (P = 0) -> (path, score, status) ; status 6 = empty beam."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    rc = _load().orc_beam(hmm.ref, T, _ptr(E), int(B), _ptr(path), _ptr(score))
    if rc not in (0, 6):
        raise RuntimeError(f"orc_beam failed: {rc}")
    return path, score[0], rc


def beam_static(hmm: HMM, E, B: int):
    """Static beam (full K-entry score vector per step, then top B) ->
    (path, score, status); status 6 = empty beam."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    rc = _load().orc_beam_static(hmm.ref, T, _ptr(E), int(B), _ptr(path), _ptr(score))
    if rc not in (0, 6):
        raise RuntimeError(f"orc_beam_static failed: {rc}")
    return path, score[0], rc


def flash_bs(hmm: HMM, E, P: int, B: int, complete: bool = False):
    """FLASH-BS -> (path, score, reruns, status)."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    reruns = np.zeros(1, np.int32)
    rc = _load().orc_flash_bs(hmm.ref, T, _ptr(E), int(P), int(B), int(complete),
                              _ptr(path), _ptr(score), _ptr(reruns))
    if rc not in (0, 6):
        raise RuntimeError(f"orc_flash_bs failed: {rc}")
    return path, score[0], int(reruns[0]), rc


def checkpoint(hmm: HMM, E, P: int = 0):
    """Checkpoint Viterbi with P checkpoints (P <= 0: ceil(sqrt(T))) ->
    (path, score, n_checkpoints, largest segment in rows)."""
    E = _E(E, hmm.K)
    T = E.shape[0]
    path = np.zeros(T, np.int32)
    score = np.zeros(1, np.float32)
    nc = np.zeros(1, np.int32)
    mr = np.zeros(1, np.int32)
    rc = _load().orc_checkpoint(hmm.ref, T, _ptr(E), int(P), _ptr(path), _ptr(score), _ptr(nc), _ptr(mr))
    if rc:
        raise RuntimeError(f"orc_checkpoint failed: {rc}")
    return path, score[0], int(nc[0]), int(mr[0])


def checkpoint_count(T: int, P: int = 0) -> int:
    return int(_load().orc_checkpoint_count(int(T), int(P)))


def path_score(hmm: HMM, E, path):
    E = _E(E, hmm.K)
    path = _i32(path)
    return np.float32(_load().orc_path_score(hmm.ref, E.shape[0], _ptr(E), _ptr(path)))


def split_points(T: int, P: int):
    e = np.zeros(max(T, 1), np.int32)
    n = _load().orc_split_points(int(T), int(P), _ptr(e))
    return [int(x) for x in e[:n]]


def grad(K: int, T, paths_packed, g):
    """Path-count gradient for sequences sharing one model.

    ``T`` int32[n], ``paths_packed`` int32[sum T], ``g`` float32[n] ->
    (dlog_pi[K], dlogA[K,K], dE packed [sum T*K])."""
    T = _i32(T)
    n = T.shape[0]
    path_off = np.zeros(n, np.int64)
    e_off = np.zeros(n, np.int64)
    if n:
        path_off[1:] = np.cumsum(T.astype(np.int64))[:-1]
        e_off[1:] = np.cumsum(T.astype(np.int64) * K)[:-1]
    paths_packed = _i32(paths_packed)
    g = _f32(g)
    dpi = np.zeros(K, np.float32)
    dA = np.zeros(K * K, np.float32)
    dE = np.zeros(int(T.astype(np.int64).sum()) * K, np.float32)
    rc = _load().orc_grad(K, n, _ptr(T), _ptr(e_off), _ptr(path_off), _ptr(paths_packed),
                          _ptr(g), _ptr(dpi), _ptr(dA), _ptr(dE))
    if rc:
        raise RuntimeError(f"orc_grad failed: {rc}")
    return dpi, dA.reshape(K, K), dE


def map_sequences(fn, jobs, threads: int | None = None):
    """Run ``fn(job)`` over jobs on a thread pool.  ctypes drops the GIL during
    each foreign call, so the oracle runs on ``threads`` cores at once."""
    threads = threads or os.cpu_count() or 1
    if threads == 1:
        return [fn(j) for j in jobs]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, jobs))
