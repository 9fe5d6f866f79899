"""Continuous-batching server for truncated low-rank approximation (TUXV) requests.

Requests (A, Omega, b, p, k) arrive at any time.  The server admits them
against an HBM byte budget (inputs, outputs and their share of the scratch),
packs every admitted small request into the next batched launch
(``rq_tuxv_batched``: one persistent kernel over uneven problems) and sends
large ones to the whole-GPU ``rq_tuxv``.  In FP64 (``prec=RQ_FP64``, the plain
FP64 path, which the batched kernel does not provide) every request goes to
``rq_tuxv``.  Up to ``lanes`` launches are on the
GPU at once, each on its own CUDA stream with its own library handle, so
requests that arrive while others run start as soon as a lane and memory free
up, and their work overlaps on the device.  A request's result does not
depend on what it was batched with (each problem is computed by one CTA).  A
launch the library refuses fails the requests of that launch (``wait`` raises)
and frees their memory; the server goes on with the others.

Only argument marshalling and scheduling live here; all arithmetic runs in the
CUDA library.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

from . import RQ_FP32, RQ_FP64, Handle

__all__ = ["Request", "Server", "footprint_bytes"]


def footprint_bytes(m, n, k, b, p, elem=4):
    """HBM bytes a request holds while admitted: A, Omega, U, X, V, and scratch."""
    l = b + p
    io = elem * (m * n + l * m + m * k + k * k + n * k)
    scratch = elem * (l * n + 2 * k * n + 3 * m * k + m * b + 2 * n * k + max(m, n) * (k + b)) + 64 * 1024
    return io + scratch


@dataclass
class Request:
    A: object
    Omega: object
    b: int
    p: int
    k: int
    arrival: float = 0.0
    admitted: float = 0.0
    started: float = 0.0
    done: float = 0.0
    out: tuple = None
    info: object = None
    nbytes: int = 0
    large: bool = False
    error: object = None             # the exception that failed the request's launch, if any
    _ev: threading.Event = field(default_factory=threading.Event)

    @property
    def shape(self):
        return tuple(self.A.shape)

    def wait(self, timeout=None):
        if not self._ev.wait(timeout):
            raise TimeoutError("request not finished")
        if self.error is not None:
            raise RuntimeError("request failed") from self.error
        return self.out

    @property
    def latency(self):
        return self.done - self.arrival


class Server:
    """Admission + continuous batching over ``lanes`` concurrent GPU launches."""

    def __init__(self, budget_bytes=120e9, lanes=3, max_batch=4096, large_mn=2048 * 1024, prec=RQ_FP32,
                 device=None, tiles=None):
        """prec: RQ_FP32 (default: FP32 storage, FP32 sketch, 3xTF32 tensor-core
        products, FP64 Householder scalars and norms), RQ_MIXED (the sketch from
        bfloat16-rounded inputs) or RQ_FP64 (every request through rq_tuxv).
        tiles: the batched kernel's tile policy (skinny_m, skinny_n) for every
        lane, e.g. from Handle.tune_batched on a representative batch; None
        keeps the library's default."""
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.large_mn = large_mn
        self.prec = prec
        self.lanes = [(Handle(), torch.cuda.Stream(device=self.device)) for _ in range(lanes)]
        if tiles is not None:
            for h, _ in self.lanes:
                h.batch_tiles = tuple(tiles)
        self.busy = [None] * lanes       # (requests, event) per lane
        self.pending = []                # submitted, not admitted
        self.ready = []                  # admitted, not launched
        self.used = 0
        self.completed = []
        self.failed = []
        self.rejected = 0
        self.lock = threading.Lock()
        self._stop = False
        self._thread = None

    # -- client side -------------------------------------------------------
    def submit(self, A, Omega, b, p, k):
        m, n = A.shape
        r = Request(A, Omega, b, p, k, arrival=time.perf_counter())
        r.nbytes = footprint_bytes(m, n, k, b, p, elem=8 if self.prec == RQ_FP64 else 4)
        r.large = m * n > self.large_mn or self.prec == RQ_FP64
        if r.nbytes > self.budget:
            self.rejected += 1
            raise MemoryError("request larger than the server's HBM budget")
        with self.lock:
            self.pending.append(r)
        return r

    # -- server side -------------------------------------------------------
    def _admit(self, now):
        while self.pending and self.used + self.pending[0].nbytes <= self.budget:
            r = self.pending.pop(0)
            self.used += r.nbytes
            r.admitted = now
            m, n = r.A.shape
            torch = self.torch
            if not r.large:              # a large request gets its outputs from rq_tuxv at launch
                try:
                    r.out = (torch.empty((r.k, m), dtype=r.A.dtype, device=self.device).t(),
                             torch.empty((r.k, r.k), dtype=r.A.dtype, device=self.device).t(),
                             torch.empty((r.k, n), dtype=r.A.dtype, device=self.device).t())
                except RuntimeError as exc:  # the device ran out of memory below the budget
                    self._fail([r], exc, now)
                    continue
            self.ready.append(r)

    def _reap(self, now):
        for i, slot in enumerate(self.busy):
            if slot is not None and slot[1].query():
                for r in slot[0]:
                    r.done = now
                    self.used -= r.nbytes
                    self.completed.append(r)
                    r._ev.set()
                self.busy[i] = None

    def _launch(self, now):
        torch = self.torch
        for i, slot in enumerate(self.busy):
            if slot is not None or not self.ready:
                continue
            h, st = self.lanes[i]
            if self.ready[0].large:
                batch = [self.ready.pop(0)]
            else:
                batch = [r for r in self.ready if not r.large][: self.max_batch]
                ids = {id(r) for r in batch}
                self.ready = [r for r in self.ready if id(r) not in ids]
                batch.sort(key=lambda r: -(r.A.shape[0] * r.A.shape[1] * r.k))
            for r in batch:
                r.started = now
            try:
                with torch.cuda.stream(st):
                    if batch[0].large:
                        r = batch[0]
                        U2, X2, V2, _, info = h.tuxv(r.A, r.Omega, r.b, r.p, r.k, prec=self.prec, stream=st)
                        r.out = (U2, X2, V2)
                        r.info = info
                    else:
                        outs, info = h.tuxv_batched([(r.A, r.Omega, r.b, r.p, r.k) for r in batch],
                                                    prec=self.prec, stream=st, outputs=[r.out for r in batch])
                        for j, r in enumerate(batch):
                            r.info = info[j:j + 1]
                    ev = torch.cuda.Event()
                    ev.record(st)
            except Exception as exc:  # the library refused the launch: fail these requests, keep serving
                self._fail(batch, exc, now)
                continue
            self.busy[i] = (batch, ev)

    def _fail(self, batch, exc, now):
        for r in batch:
            r.error = exc
            r.done = now
            self.used -= r.nbytes
            self.failed.append(r)
            r._ev.set()

    def pump(self):
        """One scheduling pass: retire finished launches, admit, launch."""
        now = time.perf_counter()
        with self.lock:
            self._reap(now)
            self._admit(now)
            self._launch(now)

    def idle(self):
        with self.lock:
            return not self.pending and not self.ready and all(s is None for s in self.busy)

    def start(self, poll_s=5e-5):
        def loop():
            while not self._stop:
                self.pump()
                time.sleep(poll_s)
        self._stop = False
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop = True
        if self._thread is not None:
            self._thread.join()
        self._thread = None

    def drain(self, timeout=60.0):
        t0 = time.perf_counter()
        while not self.idle():
            if self._thread is None:
                self.pump()
            time.sleep(1e-4)
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain")

    def stats(self):
        import numpy as np
        lat = np.array([r.latency for r in self.completed]) if self.completed else np.zeros(1)
        if len(self.completed) > 1:
            span = max(r.done for r in self.completed) - min(r.arrival for r in self.completed)
        else:
            span = float("nan")
        return {"completed": len(self.completed), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "req_per_s": len(self.completed) / span,
                "rejected": self.rejected, "failed": len(self.failed)}
