"""Continuous-batching request loop for extremum-graph requests.

Requests (one scalar field each) arrive at any time.  Each engine owns one
library handle (its own device workspace) and one CUDA stream; an idle engine
takes, in arrival order, every queued request that fits its batch limits and
the free device-memory budget, uploads the fields, runs them as ONE batched
submission (eg_batch_submit: one launch per pipeline step for the whole batch)
and returns each result.  With two or more engines, requests that arrive
while a batch is on the GPU are admitted into the next batch as soon as an
engine and memory are free, and the batches overlap on the device.

Admission: a request reserves an estimate of the device memory it needs
(field, labels, library workspace, graph) from a budget set at start-up (a
fraction of the free HBM, or an explicit cap).  Requests wait while the budget
is short; a request larger than the whole budget is refused with
EG_ERR_BUSY.  Results are copied to host memory, so a request's device state
lives only from admission to completion.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field as dc_field
from typing import Callable, List, Optional

import numpy as np

EG_ERR_BUSY = 7


class DeviceResult:
    """A served result kept in device memory (the library's buffers) until
    release(): counts and device pointers of the graph (eg_get_graph_device),
    and to_host() for a host copy when the client wants one."""

    def __init__(self, engine, rid, graph_c):
        self.engine, self.rid, self.graph = engine, rid, graph_c
        self._lock = threading.Lock()
        self.released = False

    def to_host(self, labels: bool = False):
        with self._lock:
            if self.released:
                raise RuntimeError("result already released")
            return self.engine.handle.get_graph(self.rid, labels=labels)

    def release(self):
        with self._lock:
            if not self.released:
                self.engine.handle.release(self.rid)
                self.released = True


@dataclass
class Request:
    values: np.ndarray                 # float32 field, numpy shape = reversed(extents)
    pinned: object = None              # the same values in a page-locked torch tensor, if given so
    rid: int = 0
    arrival: float = 0.0               # time.perf_counter() when submitted
    admitted: float = 0.0
    done: float = 0.0
    result: object = None              # engine-specific (eg.Graph for the GPU engine)
    status: int = 0
    batch: int = -1                    # batch sequence number it ran in
    engine: int = -1
    event: threading.Event = dc_field(default_factory=threading.Event)
    nbytes: int = 0                    # device bytes reserved for it while admitted

    @property
    def n(self) -> int:
        return int(self.values.size)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def request_bytes(n_vertices: int, d: int) -> int:
    """Device bytes reserved for one request: field + labels (4+4 B/vertex),
    classification records (16 B/vertex), per-brick state, graph outputs."""
    return 26 * int(n_vertices) + (1 << 16)


class GpuEngine:
    """Runs batches through the CUDA library on one stream with its own handle.

    results="host": every request's graph is copied to numpy arrays and its
    device state freed.  results="device": the graph stays in device memory
    (a DeviceResult) until the client releases it."""

    def __init__(self, device: int = 0, minimum: bool = False, results: str = "host"):
        import torch
        from . import eg
        if results not in ("host", "device"):
            raise ValueError("results must be 'host' or 'device'")
        self.torch = torch
        self.eg = eg
        self.device = device
        self.results = results
        # every batch of a request stream has its own layout, so capturing a
        # CUDA graph per batch would never be repaid by a replay: launch directly
        self.handle = eg.Handle(device, minimum=minimum, config=eg.EGConfig(flags=eg.EG_FLAG_NO_GRAPH))
        self.stream = torch.cuda.Stream(device=device)
        # one page-locked staging buffer and one device buffer per engine,
        # grown on demand and reused: a batch's fields travel in ONE copy
        self._pinned = None
        self._dev = None
        self._staged = None  # event: the last upload has left the staging buffer

    def _upload(self, reqs: List[Request]):
        """Device views of the batch's fields: fields that arrived in
        page-locked memory are copied straight from it (one asynchronous copy
        each); otherwise the batch is staged into the engine's page-locked
        buffer and travels in one copy."""
        torch = self.torch
        sizes = [r.n for r in reqs]
        if all(r.pinned is not None for r in reqs):
            padded = [(n + 3) & ~3 for n in sizes]  # 16-byte aligned fields
            total = sum(padded)
            if self._dev is None or self._dev.numel() < total:
                self._dev = torch.empty(max(total, 1 << 20), dtype=torch.float32, device=self.device)
            # one call for all the batch's copies (views of one buffer)
            slots = self._dev[:total].split(padded)
            dst = [sl[:n] for sl, n in zip(slots, sizes)]
            src = [r.pinned.view(-1) for r in reqs]
            foreach = getattr(torch, "_foreach_copy_", None)
            if foreach is not None:
                foreach(dst, src, non_blocking=True)
            else:
                for a, b in zip(dst, src):
                    a.copy_(b, non_blocking=True)
            return dst
        offs = np.concatenate([[0], np.cumsum([(n + 3) & ~3 for n in sizes])])  # 16-byte aligned fields
        total = int(offs[-1])
        if self._pinned is None or self._pinned.numel() < total:
            if self._staged is not None:
                self._staged.synchronize()
            cap = max(total, 1 << 20)
            self._pinned = torch.empty(cap, dtype=torch.float32, pin_memory=True)
            self._dev = torch.empty(cap, dtype=torch.float32, device=self.device)
        elif self._staged is not None:
            self._staged.synchronize()  # the previous batch's copy has read the buffer
        host = self._pinned.numpy()
        for r, o in zip(reqs, offs[:-1]):
            host[int(o):int(o) + r.n] = r.values.reshape(-1)
        self._dev[:total].copy_(self._pinned[:total], non_blocking=True)
        self._staged = torch.cuda.Event()
        self._staged.record(self.stream)
        return [self._dev[int(o):int(o) + r.n].view(r.values.shape) for r, o in zip(reqs, offs[:-1])]

    def run(self, reqs: List[Request]) -> None:
        torch = self.torch
        with torch.cuda.stream(self.stream):
            ts = self._upload(reqs)
            ids = self.handle.batch_submit_ptrs([t.data_ptr() for t in ts],
                                                [tuple(reversed(r.values.shape)) for r in reqs], self.stream)
            keep = set()
            try:
                if self.results == "host":
                    for r, rid in zip(reqs, ids):
                        r.result = self.handle.get_graph(rid, labels=False)
                else:
                    for r, rid, g in zip(reqs, ids, self.handle.get_graphs_device(ids)):
                        r.result = DeviceResult(self, rid, g)
                        keep.add(rid)
            finally:
                for rid in ids:
                    if rid not in keep:
                        self.handle.release(rid)
        del ts

    def close(self):
        self.handle.close()


class Server:
    """Continuous batching over one or more engines with device-memory admission.

    The engines' threads run Python between their library calls, so a
    collection of the interpreter's cyclic garbage collector stalls them all;
    in a process holding many objects that pause sets the latency tail.
    Callers that serve under latency targets should collect once and call
    gc.freeze() before the stream starts (the benchmark does)."""

    def __init__(self, engines: list, budget_bytes: int, max_batch: int = 128,
                 max_batch_vertices: int = 1 << 28,
                 bytes_fn: Callable[[int, int], int] = request_bytes,
                 on_done: Optional[Callable[[Request], None]] = None):
        self.engines = engines
        self.on_done = on_done  # called by the worker for every finished request
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.max_batch_vertices = max_batch_vertices
        self.bytes_fn = bytes_fn
        self.queue: collections.deque = collections.deque()
        self.cv = threading.Condition()
        self.in_use = 0
        self.stop_flag = False
        self.next_rid = 0
        self.batches = 0
        self.completed: List[Request] = []
        self.deferred_waits = 0
        self.max_in_flight_batches = 0
        self.in_flight_batches = 0
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(len(engines))]
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------- client
    def submit(self, values) -> Request:
        """values: a float32 numpy array, or a contiguous float32 torch CPU
        tensor in page-locked memory (copied to the device without staging)."""
        if hasattr(values, "is_pinned"):
            if str(values.dtype) != "torch.float32" or not values.is_contiguous() or values.is_cuda:
                raise ValueError("a tensor request must be a contiguous float32 CPU tensor")
            r = Request(values=values.numpy(), pinned=values if values.is_pinned() else None)
        else:
            r = Request(values=np.ascontiguousarray(values, dtype=np.float32))
        with self.cv:
            r.rid = self.next_rid
            self.next_rid += 1
            r.arrival = time.perf_counter()
            r.nbytes = self.bytes_fn(r.n, r.values.ndim)
            if r.nbytes > self.budget:
                r.status = EG_ERR_BUSY
                r.done = r.arrival
                r.event.set()
                self.completed.append(r)
                return r
            self.queue.append(r)
            self.cv.notify_all()
        return r

    def close(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()

    def drain(self, timeout: float = 600.0) -> bool:
        end = time.perf_counter() + timeout
        with self.cv:
            while self.queue or self.in_flight_batches:
                left = end - time.perf_counter()
                if left <= 0:
                    return False
                self.cv.wait(left)
        return True

    # ------------------------------------------------------------- worker
    def _take(self) -> List[Request]:
        """Under the lock: admit queued requests, in order, while they fit."""
        batch, verts, need = [], 0, 0
        for r in self.queue:  # (not modified while iterated; popped below)
            b = r.nbytes
            if len(batch) >= self.max_batch or (batch and verts + r.n > self.max_batch_vertices):
                break
            if self.in_use + need + b > self.budget:
                self.deferred_waits += 1
                break  # keep arrival order: later requests wait behind this one
            batch.append(r)
            verts += r.n
            need += b
        for r in batch:
            self.queue.popleft()
        self.in_use += need
        self.peak_in_use = max(getattr(self, "peak_in_use", 0), self.in_use)
        return batch

    def _worker(self, ei: int):
        eng = self.engines[ei]
        while True:
            with self.cv:
                batch = []
                while True:
                    if self.queue:
                        batch = self._take()
                        if batch:
                            break
                    elif self.stop_flag:
                        return
                    self.cv.wait(0.05)
                seq = self.batches
                self.batches += 1
                self.in_flight_batches += 1
                self.max_in_flight_batches = max(self.max_in_flight_batches, self.in_flight_batches)
            t_adm = time.perf_counter()
            status = 0
            try:
                eng.run(batch)
            except Exception as e:  # a failed batch reports its status per request
                status = getattr(e, "status", -1)
            t_done = time.perf_counter()
            if self.on_done is not None:
                for r in batch:
                    r.status = status
                    self.on_done(r)
            with self.cv:
                for r in batch:
                    r.admitted, r.done, r.batch, r.engine = t_adm, t_done, seq, ei
                    r.status = status
                    self.completed.append(r)
                    r.event.set()
                self.in_use -= sum(r.nbytes for r in batch)
                self.in_flight_batches -= 1
                self.cv.notify_all()

    # ------------------------------------------------------------- metrics
    def stats(self) -> dict:
        ok = [r for r in self.completed if r.status == 0]
        if not ok:
            return {"requests": 0}
        lat = np.array([r.latency for r in ok])
        t0 = min(r.arrival for r in ok)
        t1 = max(r.done for r in ok)
        nv = sum(r.n for r in ok)
        return {"requests": len(ok), "refused": sum(r.status == EG_ERR_BUSY for r in self.completed),
                "failed": sum(r.status not in (0, EG_ERR_BUSY) for r in self.completed),
                "vertices": nv, "makespan_s": t1 - t0, "throughput_mvps": nv / (t1 - t0) / 1e6,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "batches": self.batches, "max_in_flight_batches": self.max_in_flight_batches,
                "deferred_waits": self.deferred_waits}


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival offsets (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def replay(server: Server, fields: List[np.ndarray], offsets: np.ndarray) -> List[Request]:
    """Submit fields[i] at start + offsets[i] (client side of a benchmark)."""
    reqs = []
    t0 = time.perf_counter()
    for f, off in zip(fields, offsets):
        now = time.perf_counter() - t0
        if off > now:
            time.sleep(off - now)
        reqs.append(server.submit(f))
    return reqs
