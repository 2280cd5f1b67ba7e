"""Persistence-directed cancellation (Sec. 3.5) on the GPU (eg_get_cancelled,
data-parallel rounds) against the oracle's serial queue (oracle.cancel),
element by element: the keep flag of every saddle and the survivor of every
maximum, for 1D-5D fields, both graphs, thresholds from "nothing" to
"everything", ties, multi-brick and batched results."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg_mod():
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    eg.load()
    return eg


def _taus(og):
    """Thresholds spanning the costs of the oracle graph: below all, a few
    quantiles of the initial simple-saddle costs, and infinity."""
    if og.saddles.size == 0:
        return [-1.0, 0.0, np.inf]
    spread = float(np.float32(og.max_val.max()) - np.float32(og.max_val.min()))
    qs = [float(np.float32(spread * q)) for q in (1e-3, 0.02, 0.1, 0.3)]
    return [-1.0, 0.0] + qs + [np.inf]


def _check(eg_mod, h, f, minimum):
    og = oracle.compute(f.values, minimum=minimum)
    t = torch.from_numpy(f.values).cuda()
    rid = h.compute(t)
    try:
        for tau in _taus(og):
            want = oracle.cancel_graph(og, tau, minimum=minimum)
            alive, surv, n, rounds = h.get_cancelled(rid, tau)
            assert np.array_equal(alive, want.alive), (f.name, tau)
            assert np.array_equal(surv, want.survivor), (f.name, tau)
            assert n == want.n_cancelled
            assert rounds >= 1
    finally:
        h.release(rid)


CASES = {
    "1d": lambda: F.white_noise((3000,), 1),
    "2d_cfg": lambda: F.config_2d_256(side=120),
    "2d_ties": lambda: F.integer_ties((60, 50), 2, 4),
    "3d_grf": lambda: F.grf((40, 36, 32), 2),
    "3d_gauss": lambda: F.config_3d_256(side=80),
    "3d_ties": lambda: F.integer_ties((21, 19, 17), 3, 3),
    "4d_white": lambda: F.white_noise((9, 8, 7, 6), 4),
    "5d_white": lambda: F.white_noise((5, 5, 4, 4, 3), 5),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("minimum", [False, True])
def test_cancel_matches_oracle(eg_mod, case, minimum):
    f = CASES[case]()
    with eg_mod.Handle(0, minimum=minimum) as h:
        _check(eg_mod, h, f, minimum)


@pytest.mark.parametrize("minimum", [False, True])
def test_cancel_many_saddles(eg_mod, minimum):
    """More saddles than the one-CTA tail takes at once (~70 K): the first
    rounds run over all CTAs, the rest in the tail."""
    f = F.grf((96, 96, 96), 2)
    og = oracle.compute(f.values, minimum=minimum)
    assert og.saddles.size > 40000
    t = torch.from_numpy(f.values).cuda()
    with eg_mod.Handle(0, minimum=minimum) as h:
        rid = h.compute(t)
        try:
            spread = float(np.float32(og.max_val.max()) - np.float32(og.max_val.min()))
            for tau in [float(np.float32(spread * 0.02)), float(np.float32(spread * 0.2)), np.inf]:
                want = oracle.cancel_graph(og, tau, minimum=minimum)
                alive, surv, n, rounds = h.get_cancelled(rid, tau)
                assert np.array_equal(alive, want.alive), tau
                assert np.array_equal(surv, want.survivor), tau
        finally:
            h.release(rid)


def test_cancel_on_batched_results(eg_mod):
    fs = [F.white_noise(e, zlib.crc32(repr(e).encode()) % 1000) for e in [(70, 40), (13, 12, 11), (30,), (6, 5, 4, 3)]]
    ts = [torch.from_numpy(f.values).cuda() for f in fs]
    with eg_mod.Handle(0) as h:
        ids = h.batch_submit(ts)
        try:
            for f, rid in zip(fs, ids):
                og = oracle.compute(f.values)
                for tau in [0.05, np.inf]:
                    want = oracle.cancel_graph(og, tau)
                    alive, surv, _, _ = h.get_cancelled(rid, tau)
                    assert np.array_equal(alive, want.alive) and np.array_equal(surv, want.survivor)
        finally:
            for rid in ids:
                h.release(rid)


def test_cancel_rejects_bad_arguments(eg_mod):
    import ctypes
    f = F.white_noise((20, 20), 3)
    with eg_mod.Handle(0) as h:
        rid = h.compute(torch.from_numpy(f.values).cuda())
        lib = eg_mod.load()
        a = np.empty(4096, np.uint8)
        s = np.empty(4096, np.uint32)
        st = lib.eg_get_cancelled(h._h, ctypes.c_uint64(rid), ctypes.c_float(float("nan")),
                                  ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(s.ctypes.data), None, None)
        assert st == eg_mod.EG_ERR_ARG
        st = lib.eg_get_cancelled(h._h, ctypes.c_uint64(rid), ctypes.c_float(1.0), None, None, None, None)
        assert st == eg_mod.EG_ERR_ARG
        st = lib.eg_get_cancelled(h._h, ctypes.c_uint64(rid + 99), ctypes.c_float(1.0),
                                  ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(s.ctypes.data), None, None)
        assert st == eg_mod.EG_ERR_ARG
        h.release(rid)
        # a result of another element type
        u = F.quantise(F.grf((16, 16, 8), 2), "uint8")
        rid = h.compute(eg_mod.device_array(u.values), dtype=u.values.dtype)
        st = lib.eg_get_cancelled(h._h, ctypes.c_uint64(rid), ctypes.c_float(1.0),
                                  ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(s.ctypes.data), None, None)
        assert st == eg_mod.EG_ERR_ARG
        h.release(rid)
