"""Host logic of the continuous-batching server (no GPU): admission against the
HBM budget, routing of large and small requests, at most `lanes` launches in
flight, completion and draining; a launch the library refuses (an injected
error) fails its own requests only, and waits time out on the host.  The library handle, CUDA streams and events
are replaced by fakes that record the calls; a fake event completes when the
test says so."""
import contextlib

import pytest
import torch

from paper_2008_04447_gb300 import serve


class FakeHandle:
    log = []

    def tuxv(self, A, Omega, b, p, k, prec=None, stream=None):
        FakeHandle.log.append(("tuxv", tuple(A.shape), k))
        m, n = A.shape
        return (torch.zeros(m, k), torch.zeros(k, k), torch.zeros(n, k), None, torch.zeros(1, dtype=torch.int32))

    def tuxv_batched(self, problems, prec=None, stream=None, outputs=None):
        FakeHandle.log.append(("batched", [tuple(t[0].shape) for t in problems]))
        return outputs, torch.zeros(len(problems), dtype=torch.int32)


class FakeEvent:
    live = []

    def __init__(self):
        self.done = False
        FakeEvent.live.append(self)

    def record(self, stream=None):
        pass

    def query(self):
        return self.done


class FakeStream:
    cuda_stream = 0

    def __init__(self, device=None):
        pass


@pytest.fixture
def fakes(monkeypatch):
    FakeHandle.log = []
    FakeEvent.live = []
    monkeypatch.setattr(serve, "Handle", FakeHandle)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    return FakeHandle.log


def req(m, n, k=8, b=8, p=4):
    return torch.zeros(m, n), torch.zeros(b + p, m), b, p, k


def finish_all():
    for e in FakeEvent.live:
        e.done = True


def test_oversized_request_is_rejected(fakes):
    srv = serve.Server(budget_bytes=1e6, lanes=2, device="cpu")
    with pytest.raises(MemoryError):
        srv.submit(*req(2000, 1000))
    assert srv.rejected == 1


def test_admission_never_exceeds_the_budget(fakes):
    one = serve.footprint_bytes(300, 200, 8, 8, 4)
    srv = serve.Server(budget_bytes=2.5 * one, lanes=4, device="cpu")
    rs = [srv.submit(*req(300, 200)) for _ in range(5)]
    srv.pump()
    assert srv.used <= srv.budget
    assert sum(r.admitted > 0 for r in rs) == 2          # only two fit
    finish_all()
    srv.pump()                                            # reap frees memory, admits the next ones
    assert srv.used <= srv.budget
    assert sum(r.admitted > 0 for r in rs) == 4
    for _ in range(4):
        finish_all()
        srv.pump()
    assert srv.idle() and len(srv.completed) == 5 and srv.used == 0


def test_large_requests_go_alone_to_the_single_problem_path(fakes):
    srv = serve.Server(budget_bytes=1e12, lanes=3, large_mn=100 * 100, device="cpu")
    small = [srv.submit(*req(64 + 8 * i, 48)) for i in range(4)]
    big = srv.submit(*req(300, 200, k=16))
    srv.pump()
    kinds = [c[0] for c in fakes]
    assert kinds.count("tuxv") == 1 and kinds.count("batched") == 1
    batched = next(c for c in fakes if c[0] == "batched")[1]
    assert len(batched) == 4
    assert batched == sorted(batched, key=lambda s: -(s[0] * s[1]))   # largest first
    assert ("tuxv", (300, 200), 16) in fakes
    finish_all()
    srv.pump()
    for r in small + [big]:
        assert r.wait(1) is not None


def test_at_most_lanes_launches_in_flight(fakes):
    srv = serve.Server(budget_bytes=1e12, lanes=2, large_mn=10, device="cpu")   # every request is large
    rs = [srv.submit(*req(50, 40)) for _ in range(5)]
    srv.pump()
    assert len(fakes) == 2 and sum(s is not None for s in srv.busy) == 2
    srv.pump()
    assert len(fakes) == 2                                # nothing frees, nothing starts
    FakeEvent.live[0].done = True
    srv.pump()
    assert len(fakes) == 3                                # one lane freed, one launch
    for _ in range(5):
        finish_all()
        srv.pump()
    srv.drain(timeout=1.0)
    assert all(r.done >= r.started >= r.admitted >= r.arrival for r in rs)
    st = srv.stats()
    assert st["completed"] == 5


def test_tile_policy_reaches_every_lane(fakes):
    srv = serve.Server(budget_bytes=1e9, lanes=3, device="cpu", tiles=(64, 16))
    assert all(h.batch_tiles == (64, 16) for h, _ in srv.lanes)
    srv = serve.Server(budget_bytes=1e9, lanes=2, device="cpu")
    assert all(not hasattr(h, "batch_tiles") for h, _ in srv.lanes)


class FailingHandle(FakeHandle):
    """Refuses any batch holding a problem with 77 rows (an injected library error)."""

    def tuxv_batched(self, problems, prec=None, stream=None, outputs=None):
        if any(t[0].shape[0] == 77 for t in problems):
            FakeHandle.log.append(("refused", len(problems)))
            raise RuntimeError("rq_tuxv_batched failed with status -1001")
        return super().tuxv_batched(problems, prec, stream, outputs)


def test_a_failed_launch_fails_its_requests_and_serving_goes_on(fakes, monkeypatch):
    monkeypatch.setattr(serve, "Handle", FailingHandle)
    srv = serve.Server(budget_bytes=1e12, lanes=1, device="cpu")
    bad = [srv.submit(*req(77, 40)), srv.submit(*req(60, 40))]       # batched together, refused together
    srv.pump()
    assert all(r.error is not None for r in bad) and srv.used == 0 and srv.busy == [None]
    for r in bad:
        with pytest.raises(RuntimeError, match="request failed"):
            r.wait(0)
    good = srv.submit(*req(64, 48))
    srv.pump()
    finish_all()
    srv.pump()
    assert good.wait(0) is not None and good.error is None
    st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 1 and srv.used == 0


def test_waits_time_out_on_the_host(fakes):
    srv = serve.Server(budget_bytes=1e12, lanes=1, device="cpu")
    r = srv.submit(*req(64, 48))
    srv.pump()                                    # launched; its event never completes
    with pytest.raises(TimeoutError):
        r.wait(0.01)
    with pytest.raises(TimeoutError):
        srv.drain(timeout=0.05)
    finish_all()
    srv.drain(timeout=1.0)
    assert r.wait(0) is not None


def test_an_allocation_failure_at_admission_fails_that_request(fakes, monkeypatch):
    srv = serve.Server(budget_bytes=1e12, lanes=1, device="cpu")
    real = torch.empty

    def empty(shape, **kw):
        if shape[1] == 99:
            raise RuntimeError("CUDA out of memory")
        return real(shape, **kw)
    monkeypatch.setattr(torch, "empty", empty)
    bad = srv.submit(*req(99, 40))
    good = srv.submit(*req(64, 40))
    srv.pump()
    with pytest.raises(RuntimeError, match="request failed"):
        bad.wait(0)
    finish_all()
    srv.pump()
    assert good.wait(0) is not None and srv.used == 0 and srv.stats()["failed"] == 1


def test_fp64_requests_all_go_to_the_single_problem_path(fakes):
    """The batched kernel is FP32-only: in FP64 every request is launched alone
    through rq_tuxv, and its footprint counts 8-byte elements."""
    from paper_2008_04447_gb300 import RQ_FP64
    srv = serve.Server(budget_bytes=1e9, lanes=3, device="cpu", prec=RQ_FP64)
    rs = [srv.submit(*req(100, 80)) for _ in range(4)]
    assert all(r.large for r in rs)
    assert rs[0].nbytes == serve.footprint_bytes(100, 80, 8, 8, 4, elem=8)
    srv.pump()
    assert [e[0] for e in fakes] == ["tuxv", "tuxv", "tuxv"]
    finish_all()
    srv.pump()
    finish_all()
    srv.pump()
    assert len(srv.completed) == 4 and srv.used == 0
    assert all(e[0] == "tuxv" for e in fakes)
