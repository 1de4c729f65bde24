"""Continuous-batching decode server (not in the paper).

Requests (an HMM, emission scores, a mode) arrive over time.  The server
keeps a FIFO of waiting requests and a set of in-flight ones.  Each loop
iteration it

  1. reaps finished requests (event polling; latency = completion - arrival),
  2. admits waiting requests in arrival order while the device-memory budget
     (decoder workspace + inputs + outputs of every in-flight request) and
     the stream slots allow,
  3. launches every admitted request's decode on its own stream, so requests
     that arrive while others are on the GPU overlap with them.

Device state (delta/backpointers in the workspace) stays on the device for
the whole life of a request.  The decode itself is one ``fv_decode`` call
per request; nothing is computed on the host.

The backend is pluggable: ``GpuBackend`` runs libfv; tests drive the
admission and failure logic with a host-only fake.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    K: int
    T: int
    mode: str = "exact"          # "exact" (vanilla), "flash" or "beam"
    B: int = 256
    P: int = 0
    seed: int = 0
    arrival: float = 0.0         # seconds since the start of the run
    # filled by the server
    admitted: float = math.nan
    finished: float = math.nan
    status: int = -1
    nbytes: int = 0
    result: object = None

    @property
    def latency(self):
        return self.finished - self.arrival


class Server:
    def __init__(self, backend, mem_budget_bytes: int = 40 << 30, max_inflight: int = 64,
                 clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.budget = int(mem_budget_bytes)
        self.max_inflight = int(max_inflight)
        self.clock = clock
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list[tuple[Request, object]] = []
        self.done: list[Request] = []
        self.failed: list[Request] = []
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.not_served = 0
        self.t0 = None

    def now(self):
        return self.clock() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def step(self):
        # 1. reap
        still = []
        for req, handle in self.inflight:
            st = self.backend.poll(handle)
            if st is None:
                still.append((req, handle))
                continue
            req.finished = self.now()
            req.status = st
            req.result = self.backend.result(handle)
            self.backend.release(handle)
            self.bytes_in_use -= req.nbytes
            (self.done if st == 0 else self.failed).append(req)
        self.inflight = still
        # 2./3. admit in arrival order while memory and slots allow
        while self.waiting and len(self.inflight) < self.max_inflight:
            req = self.waiting[0]
            need = self.backend.bytes_needed(req)
            if need > self.budget:  # can never fit: reject instead of blocking the queue
                self.waiting.popleft()
                req.status = -2
                req.finished = self.now()
                self.failed.append(req)
                continue
            if self.bytes_in_use + need > self.budget:
                break
            self.waiting.popleft()
            try:
                handle = self.backend.launch(req)
            except Exception:  # launch failure is reported, not retried
                req.status = -3
                req.finished = self.now()
                self.failed.append(req)
                continue
            req.admitted = self.now()
            req.nbytes = need
            self.bytes_in_use += need
            self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
            self.inflight.append((req, handle))

    def run(self, requests, realtime: bool = True, idle_sleep: float = 0.0, max_wall: float = math.inf):
        """Replay requests at their arrival times (host clock) until all are
        finished.  With realtime=False every request is available at once.
        After max_wall seconds no more requests are admitted; those still
        waiting are reported as not served."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self.t0 = self.clock()
        i = 0
        while i < len(reqs) or self.waiting or self.inflight:
            if self.now() > max_wall:
                self.not_served = len(self.waiting) + (len(reqs) - i)
                self.waiting.clear()
                i = len(reqs)
                while self.inflight:
                    self.step()
                break
            now = self.now()
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                self.submit(reqs[i])
                i += 1
            self.step()
            if idle_sleep:
                time.sleep(idle_sleep)
        return self.report()

    def report(self):
        lat = np.array([r.latency for r in self.done]) if self.done else np.zeros(0)
        wall = max([r.finished for r in self.done + self.failed], default=0.0)
        cells = sum(self.backend.cells(r) for r in self.done)
        steps = sum(r.T * r.K for r in self.done)
        return {
            "requests": len(self.done), "failed": len(self.failed), "not_served": self.not_served,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
            "throughput_req_s": len(self.done) / wall if wall else None,
            "state_steps_per_s": steps / wall if wall else None,
            "cells_per_s": cells / wall if wall else None,
            "wall_s": wall, "peak_bytes": self.peak_bytes, "budget_bytes": self.budget,
        }


class GpuBackend:
    """libfv backend: one stream per in-flight request from a pool; model and
    emission scores are drawn on that stream (seeded by the request) before
    the decode, so the host never touches them."""

    def __init__(self, n_streams: int = 32, device: str = "cuda", keep_results: bool = False):
        import torch

        from . import Batch, Decoder, Model
        self.torch = torch
        self.Batch, self.Decoder, self.Model = Batch, Decoder, Model
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.free = list(range(n_streams))
        self.keep = keep_results

    # -- inputs -----------------------------------------------------------
    def make_inputs(self, req: Request):
        """Dirichlet(1) model and log_softmax(N(0,1)) emissions, seeded."""
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(req.seed))
        K = req.K
        gam = torch._standard_gamma(torch.ones((K + 1, K), device=self.device, dtype=torch.float64), generator=g)
        probs = gam / gam.sum(dim=1, keepdim=True)
        log_pi = probs[K].log().float()
        logA = probs[:K].log().float()
        x = torch.randn((req.T, K), generator=g, device=self.device, dtype=torch.float32)
        E = torch.log_softmax(x.double(), dim=-1).float()
        return log_pi, logA, E

    def _decoder(self, req, log_pi, logA, E):
        m = self.Model(log_pi, logA, device=self.device)
        b = self.Batch([req.T], E=E.view(-1), models=[m], device=self.device)
        mode = {"exact": "vanilla", "flash": "flash", "beam": "beam"}[req.mode]
        return self.Decoder([m], b, mode=mode, P=req.P if req.mode != "exact" else 1,
                            B=req.B if req.mode == "beam" else 0)

    def tune(self, Ks=(64, 256, 1024), T=2000):
        """Engine configuration of each K class picked by the autotuner on one
        representative request (a single sequence of T steps): requests here
        are single sequences, not the full batches the defaults were chosen
        for.  Results do not depend on the choice.  Returns {K: variant}."""
        from . import autotune
        chosen = {}
        for K in Ks:
            req = Request(rid=-1, K=int(K), T=int(T), seed=12345 + int(K))
            log_pi, logA, E = self.make_inputs(req)
            m = self.Model(log_pi, logA, device=self.device)
            b = self.Batch([req.T], E=E.view(-1), models=[m], device=self.device)
            chosen[int(K)] = int(autotune([m], b, mode="vanilla")[0])
        return chosen

    def bytes_needed(self, req: Request):
        K, T = req.K, req.T
        inputs = 4 * (K * K + K + T * K)
        outputs = 4 * (T + 1)
        if req.mode == "exact":
            ws = 2 * T * K
        elif req.mode == "beam":
            ws = 8 * T * min(req.B, K) + 4 * 4 * K
        else:
            ws = 4 * T + 8 * 4 * K * max(2, req.P)
        return inputs + outputs + ws + (1 << 16)

    def cells(self, req: Request):
        if req.mode == "beam":
            return (req.T - 1) * min(req.B, req.K) * req.K
        return (req.T - 1) * req.K * req.K

    def launch(self, req: Request):
        torch = self.torch
        if not self.free:
            raise RuntimeError("no free stream")
        si = self.free.pop()
        st = self.streams[si]
        with torch.cuda.stream(st):
            log_pi, logA, E = self.make_inputs(req)
            dec = self._decoder(req, log_pi, logA, E)
            dec.launch(st)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"si": si, "dec": dec, "ev": ev, "inputs": (log_pi, logA, E)}

    def poll(self, h):
        if not h["ev"].query():
            return None
        return h["dec"].device_status(self.streams[h["si"]])

    def result(self, h):
        if not self.keep:
            return None
        d = h["dec"]
        T = d.batch.path_len
        return d.paths[:T].cpu().numpy(), float(d.scores[0].item())

    def release(self, h):
        self.free.append(h["si"])
        h.clear()


def poisson_requests(rate, seconds, seed=6, Ks=(64, 256, 1024), tmin=100, tmax=20000, beam_B=256,
                     beam_frac=0.5, exact_mode="exact"):
    """The serving workload: Poisson arrivals, K uniform in Ks, T log-uniform
    in [tmin, tmax], a seeded coin for exact vs beam."""
    rng = np.random.default_rng(seed)
    t, rid, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        K = int(rng.choice(Ks))
        T = int(math.floor(math.exp(rng.uniform(math.log(tmin), math.log(tmax)))))
        beam = bool(rng.random() < beam_frac)
        out.append(Request(rid=rid, K=K, T=T, mode="beam" if beam else exact_mode, B=beam_B if beam else 0,
                           P=0, seed=int(rng.integers(1 << 31)), arrival=t))
        rid += 1
    return out
