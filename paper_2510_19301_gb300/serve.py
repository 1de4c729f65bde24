"""Continuous-batching decode server (not in the paper).

Requests (an observation sequence to decode with an HMM of one of the
served state-space sizes, a mode) arrive over time.  The server keeps a FIFO
of waiting requests and a set of in-flight launches.  Each loop iteration it

  1. reaps finished launches (event polling; a request's latency is the
     completion of its launch minus its arrival),
  2. admits waiting requests in arrival order while the device-memory budget
     (workspace + inputs + outputs of everything in flight) and the launch
     slots allow,
  3. packs the admitted requests of one class -- same K, same mode and beam
     parameters -- into ONE ``fv_decode`` batch and launches it on a free
     stream.  Inside the launch the persistent engine refills its sequence
     slots at tick granularity, so the requests of a batch share clusters
     and logA tiles; launches of different classes and of later arrivals
     run concurrently on other streams and SMs.

Device state (delta / backpointers in the workspace) stays on the device for
the whole life of a launch; nothing is computed on the host.

Models: by default the server holds one model per K class (Dirichlet(1)
transitions and initial distribution, drawn once from a fixed seed) and
every request brings its own emission scores, drawn on the device from the
request's seed; requests of one class can then share engine slots.  With
``shared_models=False`` every request also brings its own model; a batch
then carries one model per request (at most 64 per launch, the engine's
model table) and the engine decodes them model by model.

The backend is pluggable: ``GpuBackend`` runs libfv; tests drive the
admission, batching and failure logic with host-only fakes.  A backend
without ``launch_batch`` is driven one request per launch.
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

    @property
    def klass(self):
        """Requests of one class can share one launch."""
        return (self.K, self.mode, self.B if self.mode == "beam" else 0, self.P if self.mode != "exact" else 0)


class Server:
    def __init__(self, backend, mem_budget_bytes: int = 40 << 30, max_inflight: int = 64,
                 clock: Callable[[], float] = time.perf_counter, max_batch: int = 1024):
        self.backend = backend
        self.budget = int(mem_budget_bytes)
        self.max_inflight = int(max_inflight)   # launches in flight
        self.max_batch = int(max_batch)         # requests per launch
        self.clock = clock
        self.batched = hasattr(backend, "launch_batch")
        self.waiting: collections.deque[Request] = collections.deque()
        self.inflight: list[tuple[list[Request], object]] = []
        self.done: list[Request] = []
        self.failed: list[Request] = []
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.not_served = 0
        self.launches = 0
        self.t0 = None

    def now(self):
        return self.clock() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _reap(self):
        still = []
        for reqs, handle in self.inflight:
            st = self.backend.poll(handle)
            if st is None:
                still.append((reqs, handle))
                continue
            t = self.now()
            sts = st if isinstance(st, (list, tuple)) else [st] * len(reqs)
            for i, req in enumerate(reqs):
                req.finished = t
                req.status = int(sts[i])
                req.result = self.backend.result(handle, i) if self.batched else self.backend.result(handle)
                self.bytes_in_use -= req.nbytes
                (self.done if req.status == 0 else self.failed).append(req)
            self.backend.release(handle)
        self.inflight = still

    def _fail(self, req, status):
        req.status = status
        req.finished = self.now()
        self.failed.append(req)

    def step(self):
        self._reap()
        # admit in arrival order while memory allows; group by class
        groups: dict[tuple, list[Request]] = {}
        order: list[tuple] = []
        n_launch = len(self.inflight)
        while self.waiting:
            req = self.waiting[0]
            need = self.backend.bytes_needed(req)
            if need > self.budget:  # can never fit: reject instead of blocking the queue
                self.waiting.popleft()
                self._fail(req, -2)
                continue
            if self.bytes_in_use + need > self.budget:
                break
            key = req.klass if self.batched else ("req", req.rid)
            if key not in groups:
                if n_launch >= self.max_inflight:
                    break
                groups[key] = []
                order.append(key)
                n_launch += 1
            elif len(groups[key]) >= self.max_batch:
                break
            self.waiting.popleft()
            req.nbytes = need
            self.bytes_in_use += need
            groups[key].append(req)
        self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
        for key in order:
            reqs = groups[key]
            try:
                handle = self.backend.launch_batch(reqs) if self.batched else self.backend.launch(reqs[0])
            except Exception:  # launch failure is reported, not retried
                for req in reqs:
                    self.bytes_in_use -= req.nbytes
                    self._fail(req, -3)
                continue
            t = self.now()
            for req in reqs:
                req.admitted = t
            self.launches += 1
            self.inflight.append((reqs, handle))

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
                    self._reap()
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
            "launches": self.launches,
            "requests_per_launch": len(self.done + self.failed) / self.launches if self.launches else None,
        }


class GpuBackend:
    """libfv backend: one stream per in-flight launch from a pool.  A launch
    decodes a batch of requests of one class with one ``fv_decode`` call;
    each request's emission scores are drawn on that stream from its seed
    (and, without shared models, its model too), so the host never touches
    them."""

    MAX_MODELS = 64  # the engine's model table per launch

    def __init__(self, n_streams: int = 32, device: str = "cuda", keep_results: bool = False,
                 shared_models: bool = True, model_seed: int = 6):
        import torch

        from . import Batch, Decoder, Model
        from ._lib import FV_SHARED_GPU
        self.torch = torch
        self.Batch, self.Decoder, self.Model = Batch, Decoder, Model
        self.FV_SHARED_GPU = FV_SHARED_GPU
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.free = list(range(n_streams))
        self.keep = keep_results
        self.shared = shared_models
        self.model_seed = int(model_seed)
        self._models = {}

    # -- inputs -----------------------------------------------------------
    def _dirichlet_model(self, K, seed):
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(seed))
        gam = torch._standard_gamma(torch.ones((K + 1, K), device=self.device, dtype=torch.float64), generator=g)
        probs = gam / gam.sum(dim=1, keepdim=True)
        return probs[K].log().float(), probs[:K].log().float()

    def model_for(self, K):
        """The served model of class K (shared models): Dirichlet(1) rows and
        initial distribution from a fixed seed, drawn once."""
        if K not in self._models:
            self._models[K] = self._dirichlet_model(K, self.model_seed * 100003 + K)
        return self._models[K]

    def emissions(self, req: Request, out=None):
        """log_softmax(N(0,1)) emission scores of the request, from its seed
        (after its model's draws when it brings its own model)."""
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(req.seed))
        if not self.shared:
            torch._standard_gamma(torch.ones((req.K + 1, req.K), device=self.device, dtype=torch.float64),
                                  generator=g)
        x = torch.randn((req.T, req.K), generator=g, device=self.device, dtype=torch.float32)
        E = torch.log_softmax(x.double(), dim=-1).float()
        if out is not None:
            out.copy_(E.view(-1))
            return out
        return E

    def make_inputs(self, req: Request):
        """(log_pi, logA, E) of a request, exactly as a launch draws them."""
        if self.shared:
            log_pi, logA = self.model_for(req.K)
        else:
            log_pi, logA = self._dirichlet_model(req.K, req.seed)
        return log_pi, logA, self.emissions(req)

    @staticmethod
    def _mode(req):
        return {"exact": "vanilla", "flash": "flash", "beam": "beam"}[req.mode]

    def tune(self, Ks=(64, 256, 1024), T=2000, n=16):
        """Engine configuration of each K class picked by the autotuner on a
        representative launch (n requests of T steps).  Results do not depend
        on the choice.  Returns {K: variant}."""
        from . import autotune
        chosen = {}
        for K in Ks:
            reqs = [Request(rid=-1 - i, K=int(K), T=int(T), seed=12345 + int(K) + i) for i in range(n)]
            dec, _, _ = self._batch_decoder(reqs)
            chosen[int(K)] = int(autotune(dec.models, dec.batch, mode="vanilla")[0])
        return chosen

    def bytes_needed(self, req: Request):
        K, T = req.K, req.T
        inputs = 4 * (T * K) + (0 if self.shared else 4 * (K * K + K))
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

    def _batch_decoder(self, reqs):
        """Inputs and a prepared decoder for one class of requests."""
        torch = self.torch
        r0 = reqs[0]
        K = r0.K
        lengths = [r.T for r in reqs]
        E = torch.empty(sum(lengths) * K, dtype=torch.float32, device=self.device)
        off = 0
        for r in reqs:
            self.emissions(r, out=E[off:off + r.T * K])
            off += r.T * K
        if self.shared:
            log_pi, logA = self.model_for(K)
            models = [self.Model(log_pi, logA, device=self.device)]
            mi = None
        else:
            models = [self.Model(*self._dirichlet_model(K, r.seed), device=self.device) for r in reqs]
            mi = list(range(len(reqs)))
        b = self.Batch(lengths, E=E, models=models, model_index=mi, device=self.device)
        # launches overlap on the device: kernels with the least SM time per step
        dec = self.Decoder(models, b, mode=self._mode(r0), P=r0.P if r0.mode != "exact" else 1,
                           B=r0.B if r0.mode == "beam" else 0, flags=self.FV_SHARED_GPU)
        return dec, E, models

    def launch_batch(self, reqs):
        torch = self.torch
        if not self.free:
            raise RuntimeError("no free stream")
        if not self.shared and len(reqs) > self.MAX_MODELS:
            raise ValueError("a launch carries at most 64 models")
        si = self.free.pop()
        st = self.streams[si]
        try:
            with torch.cuda.stream(st):
                dec, E, models = self._batch_decoder(reqs)
                dec.launch(st)
                ev = torch.cuda.Event()
                ev.record(st)
        except Exception:
            self.free.append(si)
            raise
        return {"si": si, "dec": dec, "ev": ev, "inputs": (E, models), "n": len(reqs)}

    def launch(self, req: Request):
        return self.launch_batch([req])

    def poll(self, h):
        if not h["ev"].query():
            return None
        return h["dec"].device_status(self.streams[h["si"]])

    def result(self, h, i=0):
        if not self.keep:
            return None
        d = h["dec"]
        off = int(d.batch.path_off_host[i])
        T = int(d.batch.T_host[i])
        return d.paths[off:off + T].cpu().numpy(), float(d.scores[i].item())

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
