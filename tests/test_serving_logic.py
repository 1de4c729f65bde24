"""Host-side logic of the continuous-batching server, driven by a fake
backend (no GPU): FIFO admission under the memory budget, rejection of
requests that can never fit, launch failures reported without stopping the
loop, and the latency statistics."""
import pytest

from paper_2510_19301_gb300.serve import Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


class FakeBackend:
    def __init__(self, work_ticks=3, fail_rids=()):
        self.work = work_ticks
        self.fail = set(fail_rids)
        self.launched = []

    def bytes_needed(self, r):
        return r.K  # toy size

    def cells(self, r):
        return r.T * r.K * r.K

    def launch(self, r):
        if r.rid in self.fail:
            raise RuntimeError("injected launch failure")
        self.launched.append(r.rid)
        return {"left": self.work}

    def poll(self, h):
        h["left"] -= 1
        return 0 if h["left"] <= 0 else None

    def result(self, h):
        return None

    def release(self, h):
        pass


def reqs(sizes):
    return [Request(rid=i, K=k, T=10, arrival=0.0005 * i) for i, k in enumerate(sizes)]


def test_budget_is_never_exceeded_and_order_is_fifo():
    be = FakeBackend()
    srv = Server(be, mem_budget_bytes=100, max_inflight=8, clock=FakeClock())
    rep = srv.run(reqs([40, 40, 40, 30, 10, 60, 5]), realtime=False)
    assert rep["requests"] == 7 and rep["failed"] == 0
    assert srv.peak_bytes <= 100
    assert be.launched == sorted(be.launched)
    assert srv.bytes_in_use == 0


def test_too_large_request_is_rejected_not_blocking():
    be = FakeBackend()
    srv = Server(be, mem_budget_bytes=50, clock=FakeClock())
    rep = srv.run(reqs([10, 500, 10]), realtime=False)
    assert rep["requests"] == 2 and rep["failed"] == 1
    assert [r.status for r in srv.failed] == [-2]


def test_launch_failure_is_reported_and_loop_continues():
    be = FakeBackend(fail_rids={1})
    srv = Server(be, mem_budget_bytes=1000, clock=FakeClock())
    rep = srv.run(reqs([10, 10, 10, 10]), realtime=False)
    assert rep["requests"] == 3 and rep["failed"] == 1
    assert srv.failed[0].rid == 1 and srv.failed[0].status == -3


def test_inflight_limit_and_latency_stats():
    be = FakeBackend(work_ticks=5)
    srv = Server(be, mem_budget_bytes=10**9, max_inflight=2, clock=FakeClock())
    rep = srv.run(reqs([1] * 10), realtime=False)
    assert rep["requests"] == 10
    lat = sorted(r.latency for r in srv.done)
    assert rep["p50_ms"] == pytest.approx(1e3 * (lat[4] + lat[5]) / 2)
    assert all(r.admitted >= r.arrival for r in srv.done)


class FakeBatchBackend(FakeBackend):
    """Backend that takes one launch per class of requests."""

    def __init__(self, work_ticks=3, fail_rids=()):
        super().__init__(work_ticks, fail_rids)
        self.batches = []

    def launch_batch(self, rs):
        if any(r.rid in self.fail for r in rs):
            raise RuntimeError("injected launch failure")
        self.batches.append([r.rid for r in rs])
        return {"left": self.work, "n": len(rs)}

    def result(self, h, i=0):
        return None


def test_batched_launches_group_one_class_and_keep_fifo():
    be = FakeBatchBackend(work_ticks=4)
    rs = [Request(rid=i, K=(64 if i % 3 else 256), T=10, mode=("beam" if i % 2 else "exact"), arrival=0.0)
          for i in range(12)]
    srv = Server(be, mem_budget_bytes=10**9, max_inflight=16, clock=FakeClock())
    rep = srv.run(rs, realtime=False)
    assert rep["requests"] == 12 and rep["failed"] == 0
    # every launch holds requests of one class, in arrival order
    for b in be.batches:
        assert len({rs[i].klass for i in b}) == 1 and b == sorted(b)
    assert len(be.batches) == len({r.klass for r in rs})
    assert rep["launches"] == len(be.batches) and rep["requests_per_launch"] == 12 / len(be.batches)
    # a request finishes with its launch
    for b in be.batches:
        assert len({srv.done[[r.rid for r in srv.done].index(i)].finished for i in b}) == 1


def test_batched_budget_and_failures():
    be = FakeBatchBackend(fail_rids={5})
    rs = [Request(rid=i, K=30 + (i % 2), T=10, arrival=0.001 * i) for i in range(10)]
    srv = Server(be, mem_budget_bytes=100, max_inflight=8, clock=FakeClock(), max_batch=2)
    rep = srv.run(rs, realtime=False)
    assert srv.peak_bytes <= 100 and srv.bytes_in_use == 0
    assert all(len(b) <= 2 for b in be.batches)
    failed = sorted(r.rid for r in srv.failed)
    assert 5 in failed and rep["requests"] + rep["failed"] == 10
    assert all(r.status == -3 for r in srv.failed)
