"""CPU checks of the two algorithmic claims the GPU beam kernels rest on,
written here in plain Python (no code shared with the kernels):

* top-B by a 4-pass MSB radix select on order-preserving keys, with the
  early exit when a pass's whole digit bin is needed (every key with that
  prefix is taken), equals the definition: the B finite candidates first
  under (score desc, state id asc), -0 tied with +0 (Sec. V-C; the cluster
  beam kernels);
* a beam step computed as a full max-plus over every state, with delta set
  to -inf outside the beam and the lowest maximising row kept, gives the
  same beams, backpointer slots, paths and scores as the oracle's dynamic
  beam (Sec. V-C; the small-K beam kernel)."""
import numpy as np

import oracle
import workloads as W


def ord_key(x):
    u = int(np.float32(x).view(np.uint32))
    if u == 0x80000000:
        u = 0
    return (~u) & 0xFFFFFFFF if (u & 0x80000000) else (u | 0x80000000)


def radix_top(vals, Wd):
    """Ids taken by the radix select, in id order."""
    ku = [ord_key(v) if np.isfinite(v) else 0 for v in vals]
    prefix = mask = thr_gt = 0
    remaining, need_eq = Wd, 0
    for p in range(4):
        shift = 24 - 8 * p
        h = [0] * 256
        for u in ku:
            if u and (u & mask) == prefix:
                h[(u >> shift) & 255] += 1
        if p == 0 and sum(h) <= remaining:
            thr_gt, need_eq = 0, 0
            break
        acc = 0
        for d in range(255, -1, -1):
            if acc + h[d] >= remaining:
                break
            acc += h[d]
        rem = remaining - acc
        prefix |= d << shift
        mask |= 0xFF << shift
        remaining = rem
        if h[d] == rem:  # the whole bin: keys >= prefix
            thr_gt, need_eq = (prefix - 1 if prefix else 0), 0
            break
        if p == 3:
            thr_gt, need_eq = prefix, remaining
    out, eq = [], 0
    for j, u in enumerate(ku):
        if not u:
            continue
        if u > thr_gt:
            out.append(j)
        elif need_eq and u == prefix and eq < need_eq:
            out.append(j)
            eq += 1
    return out


def sorted_top(vals, Wd):
    fin = sorted(((-ord_key(v), j) for j, v in enumerate(vals) if np.isfinite(v)))
    return sorted(j for _, j in fin[:Wd])


def test_radix_select_equals_definition():
    rng = np.random.default_rng(0)
    pool = np.array([-np.inf, 0.0, -0.0, 1.0, -1.0, -3.4e38, 3.4e38, 2.5], np.float32)
    for trial in range(600):
        K = int(rng.integers(1, 200))
        kind = trial % 4
        if kind == 0:
            v = rng.normal(size=K).astype(np.float32)
        elif kind == 1:
            v = np.round(rng.normal(size=K)).astype(np.float32)
        elif kind == 2:
            v = rng.choice(pool, K)
        else:
            v = (rng.normal(size=K) * 1e-3 - 5).astype(np.float32)
        Wd = int(rng.integers(1, K + 2))
        assert radix_top(v, Wd) == sorted_top(v, Wd), (trial, K, Wd)


def fadd(a, b):
    return np.float32(np.float32(a) + np.float32(b))


def masked_full_beam(log_pi, logA, E, B):
    """Beam decode with each step a full max-plus over delta masked to -inf
    outside the beam -> (path, score) or None if the beam empties."""
    K, T = logA.shape[0], E.shape[0]
    Wd = min(B, K)
    bp_id = np.zeros((T, Wd), np.int64)
    bp_src = np.zeros((T, Wd), np.int64)
    sd = np.full(K, -np.inf, np.float32)
    inbeam = np.zeros(K, bool)
    for t in range(T):
        c = np.full(K, -np.inf, np.float32)
        g = np.zeros(K, np.int64)
        for j in range(K):
            if t == 0:
                c[j] = fadd(log_pi[j], E[0, j])
                continue
            bv, gg = np.float32(-np.inf), 0
            for i in range(K):  # ascending rows, first strictly larger kept
                x = fadd(sd[i], logA[i, j])
                if x > bv:
                    bv, gg = x, i
            c[j] = fadd(bv, E[t, j])
            g[j] = gg
        take = np.zeros(K, bool)
        fin = [j for j in range(K) if np.isfinite(c[j])]
        for j in sorted_top(c, Wd):
            take[j] = True
        assert set(np.nonzero(take)[0]) <= set(fin)
        if not take.any():
            return None
        pos = np.cumsum(take) - take
        for j in np.nonzero(take)[0]:
            bp_id[t, pos[j]] = j
            bp_src[t, pos[j]] = 0 if t == 0 else int(inbeam[:g[j]].sum())
        sd = np.where(take, c, np.float32(-np.inf)).astype(np.float32)
        inbeam = take
    best = None
    for j in np.nonzero(inbeam)[0]:
        if best is None or sd[j] > sd[best]:
            best = j
    slot = int(inbeam[:best].sum())
    path = np.zeros(T, np.int64)
    path[T - 1] = bp_id[T - 1, slot]
    for t in range(T - 1, 0, -1):
        slot = bp_src[t, slot]
        path[t - 1] = bp_id[t - 1, slot]
    return path, sd[best]


def test_masked_full_max_plus_beam_equals_oracle():
    rng = np.random.default_rng(1)
    checked = infeasible = 0
    for trial in range(120):
        K = int(rng.integers(1, 16))
        B = int(rng.integers(1, K + 3))
        T = int(rng.integers(1, 10))
        if trial % 3 == 0:
            log_pi = rng.integers(-1, 2, K).astype(np.float32)
            logA = rng.integers(-1, 2, (K, K)).astype(np.float32)
            E = rng.integers(-1, 2, (T, K)).astype(np.float32)
            E[rng.random((T, K)) < 0.1] = -0.0
        else:
            log_pi, logA = W.random_model(K, rng)
            E = W.gaussian_emissions(T, K, rng)
            if trial % 3 == 1:
                logA[rng.random((K, K)) < 0.3] = -np.inf
        p, s, st = oracle.beam(oracle.HMM(log_pi, logA), E, B)
        r = masked_full_beam(log_pi, logA, E, B)
        if st != 0:
            assert r is None
            infeasible += 1
            continue
        assert r is not None
        assert np.array_equal(r[0], p), (trial, K, B, T)
        assert np.float32(r[1]).view(np.int32) == np.float32(s).view(np.int32)
        checked += 1
    assert checked > 100
