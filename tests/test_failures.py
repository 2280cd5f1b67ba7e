"""Failure detection without faulting the GPU: host-side fault injection and
bounded device waits that report a status."""
import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    from paper_2303_02724_gb300 import _build, eg as eg_mod
    assert torch.cuda.is_available()
    _build.build()
    return eg_mod


def test_bad_arguments_are_status_codes(eg):
    import ctypes
    lib = eg.load()
    with eg.Handle(0) as h:
        rid = ctypes.c_uint64()
        ext = (ctypes.c_int64 * 4)(4, 4, 0, 0)
        t = torch.zeros(16, device="cuda")
        # d out of range, zero extent, NULL field
        assert lib.eg_compute(h._h, ctypes.c_void_p(t.data_ptr()), 6, ext, None, ctypes.byref(rid)) == eg.EG_ERR_ARG
        assert lib.eg_compute(h._h, ctypes.c_void_p(t.data_ptr()), 0, ext, None, ctypes.byref(rid)) == eg.EG_ERR_ARG
        assert lib.eg_compute(h._h, ctypes.c_void_p(t.data_ptr()), 3, ext, None, ctypes.byref(rid)) == eg.EG_ERR_ARG
        assert lib.eg_compute(h._h, None, 2, ext, None, ctypes.byref(rid)) == eg.EG_ERR_ARG
        assert lib.eg_release(h._h, 123456) == eg.EG_ERR_ARG
        big = (ctypes.c_int64 * 4)(1 << 16, 1 << 16, 2, 0)  # more than 2^32 - 1 vertices
        assert lib.eg_compute(h._h, ctypes.c_void_p(t.data_ptr()), 3, big, None, ctypes.byref(rid)) == eg.EG_ERR_ARG


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_injected_allocation_failure_then_recovery(eg, k):
    f = F.grf((40, 36, 32), 2)
    t = torch.from_numpy(f.values).cuda()
    with eg.Handle(0) as h:
        h.debug_fail_alloc(k)
        with pytest.raises(eg.EGError) as ei:
            h.graph_of(t)
        assert ei.value.status == eg.EG_ERR_OOM
        # no leak of half-built results; the next call succeeds and is exact
        g = h.graph_of(t)
        o = oracle.compute(f.values)
        assert np.array_equal(g.labels, o.label) and np.array_equal(g.col, o.col)


def test_bounded_device_wait_reports_timeout(eg):
    with eg.Handle(0) as h:
        assert h.debug_wait_timeout() == eg.EG_ERR_TIMEOUT
        # the context is still usable
        f = F.white_noise((30, 20, 10), 3)
        g = h.graph_of(torch.from_numpy(f.values).cuda())
        assert np.array_equal(g.labels, oracle.compute(f.values).label)
