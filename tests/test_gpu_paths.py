"""Arc geometry (EG_FLAG_PATHS) on the GPU vs the oracle's gradient paths,
element by element; every call goes through the C ABI."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hp():
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    h = eg.Handle(0, paths=True)
    yield h
    h.close()


@pytest.fixture(scope="module")
def hp_min():
    from paper_2303_02724_gb300 import _build, eg
    _build.build()
    h = eg.Handle(0, minimum=True, paths=True)
    yield h
    h.close()


def gpu_paths(h, values):
    rid = h.compute(torch.from_numpy(np.ascontiguousarray(values)).cuda())
    try:
        g = h.get_graph(rid)
        ptr, vtx = h.get_paths(rid)
    finally:
        h.release(rid)
    return g, ptr, vtx


def check(h, values, minimum=False):
    g, ptr, vtx = gpu_paths(h, values)
    o = oracle.compute(values, minimum=minimum, paths=True)
    assert np.array_equal(g.labels, o.label), "labels"
    assert np.array_equal(g.saddles, o.saddles) and np.array_equal(g.col, o.col), "graph"
    assert ptr.size == o.n_paths + 1
    assert np.array_equal(ptr, o.path_ptr), "path_ptr"
    assert np.array_equal(vtx, o.path_vtx), "path_vtx"


SHAPES = [(7,), (33,), (5, 3), (17, 9), (64, 48), (4, 4, 4), (9, 7, 5), (40, 36, 32), (3, 3, 3, 3),
          (6, 5, 4, 3), (12, 1500), (3, 3, 3, 3, 3), (6, 5, 4, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind", ["normal", "ties"])
def test_paths_match_oracle(hp, shape, kind):
    seed = zlib.crc32(repr((shape, kind, "paths")).encode()) % 1000
    f = F.white_noise(shape, seed) if kind == "normal" else F.integer_ties(shape, seed, 3)
    check(hp, f.values)


@pytest.mark.parametrize("shape", [(33,), (17, 9), (20, 18, 16), (5, 4, 3, 3)], ids=lambda s: "x".join(map(str, s)))
def test_paths_minimum_graph(hp_min, shape):
    check(hp_min, F.white_noise(shape, 11).values, minimum=True)


def test_paths_long_gradient_paths(hp):
    # smooth field: paths of tens of steps across many bricks
    check(hp, F.config_3d_256(side=48).values)
    check(hp, F.config_2d_256(side=200).values)


def test_paths_config_3d_256_full(hp):
    check(hp, F.config_3d_256().values)


def test_paths_only_where_asked():
    from paper_2303_02724_gb300 import _build, eg
    _build.build()
    h = eg.Handle(0)
    try:
        flds = [F.white_noise((20, 18, 16), s).values for s in (1, 2, 3)]
        ts = [torch.from_numpy(v).cuda() for v in flds]
        ids = h.batch_submit(ts, flags=[eg.EG_FLAG_PATHS, 0, eg.EG_FLAG_PATHS])
        for v, rid, want in zip(flds, ids, (True, False, True)):
            g = h.get_graph(rid)
            o = oracle.compute(v, paths=True)
            assert np.array_equal(g.labels, o.label)
            if want:
                ptr, vtx = h.get_paths(rid)
                assert np.array_equal(ptr, o.path_ptr) and np.array_equal(vtx, o.path_vtx)
            else:
                with pytest.raises(eg.EGError) as ei:
                    h.get_paths(rid)
                assert ei.value.status == eg.EG_ERR_ARG
            h.release(rid)
    finally:
        h.close()
