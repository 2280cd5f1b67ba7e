"""The allocation-free entry point (eg_labels_static) against the oracle.

Some callers cannot let the library allocate device memory (another allocator
owns it, a hard memory budget, or a loop where cudaMalloc/cudaFree would
synchronise the device); eg_labels_static serves them from a fixed scratch
array compiled into the library.  Its labels must equal, exactly, the oracle's
labels of the same field (Algorithm 2's end points for every vertex), on
consecutive calls that share that scratch array, up to the largest accepted
size, and the calls must leave the device's free memory unchanged.  This file
is collected last so that a failure here leaves every other test already run."""
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


def _static_labels(eg_mod, t, minimum):
    out = torch.full(tuple(t.shape), -1, dtype=torch.int32, device=t.device)
    st = eg_mod.labels_static(t, out, minimum=minimum)
    torch.cuda.synchronize()
    assert st == eg_mod.EG_OK, eg_mod.status_str(st)
    return out.cpu().numpy().view(np.uint32).reshape(-1)


@pytest.mark.parametrize("minimum", [False, True])
def test_static_labels_equal_oracle(eg_mod, minimum):
    cases = [F.grf((40, 36, 32), 2), F.config_2d_256(side=300), F.white_noise((9, 8, 7, 6), 3),
             F.integer_ties((64, 48, 21), 5, 3), F.white_noise((1000,), 4)]
    for f in cases:
        want = oracle.compute(f.values, minimum=minimum).label
        t = torch.from_numpy(f.values).cuda()
        # two calls in a row on the same scratch array, each checked
        for _ in range(2):
            got = _static_labels(eg_mod, t, minimum)
            assert np.array_equal(got, want)


def test_static_largest_field_and_no_allocation(eg_mod):
    m = eg_mod.STATIC_MAX_VERTICES
    f = F.white_noise((1024, 1024), 8)
    assert f.values.size == m
    want = oracle.compute(f.values).label
    t = torch.from_numpy(f.values).cuda()
    got = _static_labels(eg_mod, t, False)  # first call: the library's device code is loaded
    assert np.array_equal(got, want)
    out = torch.full((1024, 1024), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert eg_mod.labels_static(t, out) == eg_mod.EG_OK
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, "eg_labels_static changed the device's free memory"
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(-1), want)


def test_static_rejects_oversized_field(eg_mod):
    n = eg_mod.STATIC_MAX_VERTICES + 1
    t = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert eg_mod.labels_static(t, out) == eg_mod.EG_ERR_ARG
