"""Seeded synthetic inputs shaped like the FLASH Viterbi workloads.

This module only draws inputs (Dirichlet rows, log-softmaxed Gaussian
emission scores, sampled observation sequences, random CSR graphs, Poisson
arrivals).  It holds none of the decoding arithmetic, so the GPU tests, the
benchmark and the CPU oracle tests can all draw from it.

Recipe (all FP32 after drawing in float64; logs taken in float64):

* ``config1``: K=64 HMM, logpi and rows of A ~ log Dirichlet(1), emission
  rows ~ Dirichlet(0.5) over V=32 symbols, one sequence of T=1000 sampled
  from the HMM itself.
* ``config2``: K=256, rows of A ~ log Dirichlet(1) (one A shared by the
  batch), 1024 sequences with T ~ U{500..4000}, E_t = log_softmax(N(0,1)^K).
* ``config3_dense``: K=4096, rows of A ~ log Dirichlet(0.1), 8 x T=100000.
* ``config3_sparse``: K=65536, 32 distinct uniform successors per state
  (sorted), edge weights log Dirichlet(1) per row, 8 x T=100000.
* ``config4``: K=128 tags, 512 sequences with T ~ U{20..512}, transition and
  start scores N(0, 0.5^2), E = X W^T + b from 256-dim N(0,1) features.
* ``config5``: Poisson arrivals at 2000/s for 60 s; per request K in
  {64,256,1024}, T = floor(exp(U(ln 100, ln 20000))), Dirichlet(1) model,
  log-softmax emissions, half exact and half beam (B=256).

The erdos_renyi helpers follow the paper's own synthetic family (edge
probability p, missing edges are -inf, discrete emissions over 50 symbols;
``ER_*`` hold its default point and sweep ranges).
"""
from __future__ import annotations

import math

import numpy as np


def _log_dirichlet(rng, alpha, shape):
    p = rng.dirichlet(np.full(shape[-1], alpha, dtype=np.float64), size=shape[:-1])
    with np.errstate(divide="ignore"):
        return np.log(p)


def log_softmax_rows(x64):
    m = x64.max(axis=-1, keepdims=True)
    z = x64 - m
    return z - np.log(np.exp(z).sum(axis=-1, keepdims=True))


def random_model(K, rng, alpha=1.0, dtype=np.float32):
    """(log_pi [K], logA [K,K]) with Dirichlet(alpha) rows, logged."""
    log_pi = _log_dirichlet(rng, alpha, (K,)).astype(dtype)
    logA = _log_dirichlet(rng, alpha, (K, K)).astype(dtype)
    return log_pi, logA


def gaussian_emissions(T, K, rng):
    """E [T,K] = log_softmax(N(0,1)^K) per step, FP32."""
    return log_softmax_rows(rng.standard_normal((T, K))).astype(np.float32)


def random_small(K, T, seed, integer=False, lo=-8, hi=8, neg_inf_frac=0.0):
    """Tiny case for pins: i.i.d. values, optionally small integers (exact in
    FP32, many ties) and optionally some -inf transitions."""
    rng = np.random.default_rng(seed)
    if integer:
        log_pi = rng.integers(lo, hi + 1, K).astype(np.float32)
        logA = rng.integers(lo, hi + 1, (K, K)).astype(np.float32)
        E = rng.integers(lo, hi + 1, (T, K)).astype(np.float32)
    else:
        log_pi = rng.standard_normal(K).astype(np.float32)
        logA = rng.standard_normal((K, K)).astype(np.float32)
        E = rng.standard_normal((T, K)).astype(np.float32)
    if neg_inf_frac > 0:
        logA[rng.random((K, K)) < neg_inf_frac] = -np.inf
    return log_pi, logA, E


def sample_hmm_sequence(log_pi, logA, logB, T, rng):
    """Sample q_0 ~ pi, q_t ~ A[q_{t-1}], x_t ~ B[q_t]; returns obs int32[T]."""
    pi = np.exp(log_pi.astype(np.float64)); pi /= pi.sum()
    A = np.exp(logA.astype(np.float64)); A /= A.sum(axis=1, keepdims=True)
    Bm = np.exp(logB.astype(np.float64)); Bm /= Bm.sum(axis=1, keepdims=True)
    K, V = Bm.shape
    obs = np.empty(T, np.int32)
    q = rng.choice(K, p=pi)
    for t in range(T):
        if t:
            q = rng.choice(K, p=A[q])
        obs[t] = rng.choice(V, p=Bm[q])
    return obs


def config1(seed=1, K=64, V=32, T=1000):
    rng = np.random.default_rng(seed)
    log_pi, logA = random_model(K, rng, 1.0)
    logB = _log_dirichlet(rng, 0.5, (K, V)).astype(np.float32)
    obs = sample_hmm_sequence(log_pi, logA, logB, T, rng)
    return dict(K=K, V=V, T=T, log_pi=log_pi, logA=logA, logB=logB, obs=obs)


def uneven_lengths(n, lo, hi, rng):
    return rng.integers(lo, hi + 1, n).astype(np.int32)


def config2_model(seed=2, K=256):
    rng = np.random.default_rng(seed)
    log_pi, logA = random_model(K, rng, 1.0)
    return log_pi, logA


def config2_lengths(seed=2, n_seq=1024, lo=500, hi=4000):
    rng = np.random.default_rng(seed + 1000)
    return uneven_lengths(n_seq, lo, hi, rng)


def packed_offsets(T, K):
    """Start offsets (in elements) of each sequence in a packed [sum T, K]
    emission buffer and a packed [sum T] path buffer."""
    T = np.asarray(T, dtype=np.int64)
    e_off = np.zeros(len(T), np.int64)
    p_off = np.zeros(len(T), np.int64)
    if len(T):
        e_off[1:] = np.cumsum(T * K)[:-1]
        p_off[1:] = np.cumsum(T)[:-1]
    return e_off, p_off


def gaussian_emissions_packed_host(T, K, seed):
    """Packed emission rows for a batch, drawn on the host (small batches)."""
    rng = np.random.default_rng(seed)
    total = int(np.sum(np.asarray(T, np.int64)))
    return log_softmax_rows(rng.standard_normal((total, K))).astype(np.float32)


def gaussian_emissions_packed_device(total_rows, K, seed, device="cuda", chunk_rows=1 << 20):
    """Packed emission rows drawn on the device (large batches): FP32 normal
    draws from a seeded Philox generator, log-softmax in float64, cast."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((total_rows, K), dtype=torch.float32, device=device)
    for r0 in range(0, total_rows, chunk_rows):
        r1 = min(total_rows, r0 + chunk_rows)
        x = torch.randn((r1 - r0, K), generator=g, device=device, dtype=torch.float32)
        out[r0:r1] = torch.log_softmax(x.double(), dim=-1).float()
    return out


def config3_dense_model(seed=3, K=4096):
    rng = np.random.default_rng(seed)
    log_pi = _log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    logA = _log_dirichlet(rng, 0.1, (K, K)).astype(np.float32)
    return log_pi, logA


def random_csr(K, deg, rng, alpha=1.0):
    """Each state gets `deg` distinct uniform successors (sorted) with edge
    weights log Dirichlet(alpha) over its row."""
    col = np.empty((K, deg), np.int32)
    for i in range(K):
        col[i] = np.sort(rng.choice(K, size=deg, replace=False))
    val = _log_dirichlet(rng, alpha, (K, deg)).astype(np.float32)
    row_ptr = (np.arange(K + 1, dtype=np.int64) * deg).astype(np.int32)
    return row_ptr, col.reshape(-1), val.reshape(-1)


def config3_sparse_model(seed=4, K=65536, deg=32):
    rng = np.random.default_rng(seed)
    log_pi = _log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    row_ptr, col, val = random_csr(K, deg, rng, 1.0)
    return log_pi, row_ptr, col, val


def config4(seed=5, n_seq=512, K=128, D=256, lo=20, hi=512):
    """Transition/start scores and a random linear emission layer."""
    rng = np.random.default_rng(seed)
    logA = (0.5 * rng.standard_normal((K, K))).astype(np.float32)
    log_pi = (0.5 * rng.standard_normal(K)).astype(np.float32)
    T = uneven_lengths(n_seq, lo, hi, rng)
    W = (rng.standard_normal((K, D)) / 16.0).astype(np.float32)
    bias = (rng.standard_normal(K) / 16.0).astype(np.float32)
    X = rng.standard_normal((int(T.sum()), D)).astype(np.float32)
    return dict(K=K, D=D, T=T, log_pi=log_pi, logA=logA, W=W, b=bias, X=X)


def config5_requests(seed=6, rate=2000.0, seconds=60.0, Ks=(64, 256, 1024),
                     tmin=100, tmax=20000, beam_B=256):
    """Arrival schedule: list of dicts (arrival time, K, T, mode, seeds)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    rid = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        K = int(rng.choice(Ks))
        T = int(math.floor(math.exp(rng.uniform(math.log(tmin), math.log(tmax)))))
        beam = bool(rng.random() < 0.5)
        out.append(dict(rid=rid, t=t, K=K, T=T, mode="beam" if beam else "exact",
                        B=beam_B if beam else 0, seed=int(rng.integers(1 << 31))))
        rid += 1
    return out


def erdos_renyi_model(K, p, seed):
    """Paper's synthetic family: edge i->j present with probability p,
    weights log Dirichlet(1) over present edges, absent edges -inf."""
    rng = np.random.default_rng(seed)
    mask = rng.random((K, K)) < p
    mask[np.arange(K), rng.integers(0, K, K)] = True
    w = rng.gamma(1.0, size=(K, K)) * mask
    w /= w.sum(axis=1, keepdims=True)
    with np.errstate(divide="ignore"):
        logA = np.log(w).astype(np.float32)
    log_pi = _log_dirichlet(rng, 1.0, (K,)).astype(np.float32)
    return log_pi, logA


# The paper's default point and sweeps of its synthetic family (Sec. VI):
# |O| = 50 symbols, p = 0.253, K = T = 512; p from 0.05 to 1 in steps of
# x1.5, K and T from 32 to 2048, beam width from 1024 down to 32.
ER_DEFAULT = dict(K=512, T=512, p=0.253, V=50)
ER_P_SWEEP = tuple(min(1.0, 0.05 * 1.5 ** k) for k in range(9))  # 0.05 ... 1.0
ER_SIZE_SWEEP = (32, 64, 128, 256, 512, 1024, 2048)
ER_BEAM_SWEEP = (1024, 512, 256, 128, 64, 32)


def erdos_renyi_case(K, T, p, V=50, seed=0):
    """One HMM of the paper's Erdos-Renyi family and one observation
    sequence sampled from it: transitions as in erdos_renyi_model (every
    state keeps at least one out-edge), emission rows Dirichlet(1) over V
    symbols, start log Dirichlet(1)."""
    log_pi, logA = erdos_renyi_model(K, p, seed)
    rng = np.random.default_rng(seed + 7)
    logB = _log_dirichlet(rng, 1.0, (K, V)).astype(np.float32)
    obs = sample_hmm_sequence(log_pi, logA, logB, T, rng)
    return dict(K=K, T=T, p=p, V=V, log_pi=log_pi, logA=logA, logB=logB, obs=obs)
