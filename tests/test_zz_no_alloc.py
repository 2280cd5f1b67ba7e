"""The allocation-free entry point (eg_labels_static) against eg_compute.

Some callers cannot let the library allocate device memory; eg_labels_static
serves them from a fixed scratch array compiled into the library.  Its labels
must equal, exactly, the labels of the regular entry point on the same field,
on consecutive calls that share that scratch array.  This file is collected
last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

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


def _reference_labels(eg_mod, t, minimum=False):
    with eg_mod.Handle(0, minimum=minimum) as h:
        return h.graph_of(t).labels


@pytest.mark.parametrize("minimum", [False, True])
def test_static_labels_equal_regular_entry_point(eg_mod, minimum):
    cases = [F.grf((40, 36, 32), 2), F.config_2d_256(side=300), F.white_noise((9, 8, 7, 6), 3),
             F.integer_ties((64, 48, 21), 5, 3)]
    for f in cases:
        t = torch.from_numpy(f.values).cuda()
        want = _reference_labels(eg_mod, t, minimum)
        # two calls in a row on the same scratch array, each checked
        for _ in range(2):
            out = torch.full(f.values.shape, -1, dtype=torch.int32, device="cuda")
            st = eg_mod.labels_static(t, out, minimum=minimum)
            torch.cuda.synchronize()
            assert st == eg_mod.EG_OK, eg_mod.status_str(st)
            got = out.cpu().numpy().view(np.uint32).reshape(-1)
            assert np.array_equal(got, want)


def test_static_rejects_oversized_field(eg_mod):
    n = eg_mod.STATIC_MAX_VERTICES + 1
    t = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert eg_mod.labels_static(t, out) == eg_mod.EG_ERR_ARG
    # the largest accepted size still works
    m = eg_mod.STATIC_MAX_VERTICES
    t2 = torch.from_numpy(F.white_noise((1024, 1024), 8).values).cuda()
    assert t2.numel() == m
    out2 = torch.zeros(m, dtype=torch.int32, device="cuda")
    assert eg_mod.labels_static(t2, out2.view(1024, 1024)) == eg_mod.EG_OK
