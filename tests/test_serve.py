"""Serving loop: scheduling and admission on CPU (fake engine), and on the GPU
the guarantee that a request's result is the same alone and in the mix."""
import threading
import time

import numpy as np
import pytest

from paper_2303_02724_gb300 import fields as F
from paper_2303_02724_gb300 import serve


class FakeEngine:
    """Stands in for the GPU: records batches, 'computes' a checksum."""

    def __init__(self, delay=0.01):
        self.delay = delay
        self.batches = []
        self.lock = threading.Lock()

    def run(self, reqs):
        with self.lock:
            self.batches.append([r.rid for r in reqs])
        time.sleep(self.delay)
        for r in reqs:
            r.result = float(np.sum(r.values, dtype=np.float64))


def test_continuous_batching_fifo_and_budget():
    eng = [FakeEngine(0.02), FakeEngine(0.02)]
    per = serve.request_bytes(1000, 2)
    srv = serve.Server(eng, budget_bytes=5 * per, max_batch=4)
    rng = np.random.default_rng(0)
    vals = [rng.standard_normal((10, 100)).astype(np.float32) for _ in range(40)]
    reqs = []
    for v in vals:
        reqs.append(srv.submit(v))
        time.sleep(0.001)
    assert srv.drain(30)
    srv.close()
    st = srv.stats()
    assert st["requests"] == 40 and st["refused"] == 0 and st["failed"] == 0
    for r, v in zip(reqs, vals):
        assert r.event.is_set() and r.result == float(np.sum(v, dtype=np.float64))
    # batch limits and the memory budget were respected
    all_batches = eng[0].batches + eng[1].batches
    assert all(len(b) <= 4 for b in all_batches)
    assert srv.peak_in_use <= 5 * per
    # arrival order is kept inside every batch, and requests arriving while
    # others ran were batched together (continuous batching)
    assert all(b == sorted(b) for b in all_batches)
    assert any(len(b) > 1 for b in all_batches)
    # two engines had batches in flight at the same time
    assert st["max_in_flight_batches"] == 2


def test_tensor_requests_and_completion_callback():
    """Requests may arrive as float32 CPU tensors (page-locked ones are marked
    for a copy without staging); every finished request is handed to the
    on_done callback once, before its waiter is released."""
    torch = pytest.importorskip("torch")
    seen = []
    eng = [FakeEngine(0.005)]
    srv = serve.Server(eng, budget_bytes=1 << 30, max_batch=4, on_done=lambda r: seen.append(r.rid))
    t = torch.arange(1000, dtype=torch.float32).reshape(10, 100)
    r = srv.submit(t)
    assert r.pinned is None and r.values.shape == (10, 100) and r.n == 1000
    with pytest.raises(ValueError):
        srv.submit(t.to(torch.int32))
    with pytest.raises(ValueError):
        srv.submit(t.t())
    assert srv.drain(10)
    srv.close()
    assert r.result == float(np.sum(t.numpy(), dtype=np.float64))
    assert seen == [r.rid]


def test_admission_defers_and_refuses():
    eng = [FakeEngine(0.05)]
    per = serve.request_bytes(1000, 2)
    srv = serve.Server(eng, budget_bytes=int(1.5 * per), max_batch=8)
    a = srv.submit(np.zeros((10, 100), np.float32))
    b = srv.submit(np.zeros((10, 100), np.float32))   # must wait for a (budget)
    big = srv.submit(np.zeros((100, 100), np.float32))  # can never fit: refused
    assert big.event.is_set() and big.status == serve.EG_ERR_BUSY
    assert srv.drain(10)
    srv.close()
    assert a.status == 0 and b.status == 0
    assert b.admitted >= a.done  # b only started after a released its memory
    assert srv.stats()["deferred_waits"] >= 1


def test_poisson_arrivals_rate():
    off = serve.poisson_arrivals(1000.0, 20000, 4)
    assert np.all(np.diff(off) > 0)
    assert abs(off[-1] / 20000 - 1e-3) < 5e-5


@pytest.mark.gpu
@pytest.mark.parametrize("results", ["host", "device"])
def test_served_results_equal_alone(results):
    torch = pytest.importorskip("torch")
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available()
    _build.build()
    reqs = [(e, s, g) for (e, s, g) in F.serve_requests(4, 24, n_lo=1e3, n_hi=2e5)]
    vals = [F.serve_field(e, s, g).values for (e, s, g) in reqs]
    alone = []
    with eg.Handle(0) as h:
        for v in vals:
            alone.append(h.graph_of(torch.from_numpy(v).cuda(), labels=False))
    engines = [serve.GpuEngine(0, results=results), serve.GpuEngine(0, results=results)]
    srv = serve.Server(engines, budget_bytes=1 << 34, max_batch=8)
    out = serve.replay(srv, vals, serve.poisson_arrivals(2000.0, len(vals), 1))
    assert srv.drain(120)
    srv.close()
    st = srv.stats()
    assert st["requests"] == len(vals) and st["failed"] == 0
    for r, g in zip(out, alone):
        assert r.status == 0
        got = r.result if results == "host" else r.result.to_host()
        if results == "device":
            assert r.result.graph.n_saddles == g.saddles.size
            r.result.release()
        for k in ["maxima", "saddles", "sad_b0", "row_ptr", "col"]:
            assert np.array_equal(getattr(got, k), getattr(g, k)), k
        assert np.array_equal(got.max_val.view(np.uint32), g.max_val.view(np.uint32))
    for e in engines:
        e.close()
    assert st["batches"] < len(vals)  # requests shared batches
