"""Arc bundling on the GPU (eg_get_bundled) vs the oracle's bundling."""
import itertools
import zlib

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handles():
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    hs = {False: eg.Handle(0), True: eg.Handle(0, minimum=True)}
    yield hs
    for h in hs.values():
        h.close()


def gpu_bundle(h, values):
    rid = h.compute(torch.from_numpy(np.ascontiguousarray(values)).cuda())
    try:
        g = h.get_graph(rid, labels=False)
        keep = h.get_bundled(rid)
    finally:
        h.release(rid)
    return g, keep


def bundle_vectorised(saddles, sad_val, row_ptr, col, minimum=False):
    """The same rule with array operations (for fields too large for the
    oracle's loops): best saddle per pair of maxima by a lexicographic sort."""
    u = np.diff(row_ptr.astype(np.int64))
    pi, pa, pb = [], [], []
    for k in range(2, int(u.max(initial=0)) + 1):
        rows = np.nonzero(u == k)[0]
        if rows.size == 0:
            continue
        ends = col[row_ptr[rows][:, None].astype(np.int64) + np.arange(k)[None, :]]
        for x, y in itertools.combinations(range(k), 2):
            pi.append(rows)
            pa.append(ends[:, x])
            pb.append(ends[:, y])
    keep = (u < 2).astype(np.uint8)
    if not pi:
        return keep
    pi, pa, pb = np.concatenate(pi), np.concatenate(pa).astype(np.uint64), np.concatenate(pb).astype(np.uint64)
    v = sad_val[pi].astype(np.float64)
    s = saddles[pi].astype(np.int64)
    if minimum:
        v, s = -v, -s
    order = np.lexsort((s, v, pb, pa))  # by pair, then value, then index
    pa, pb, pi = pa[order], pb[order], pi[order]
    last = np.ones(pi.size, bool)
    last[:-1] = (pa[1:] != pa[:-1]) | (pb[1:] != pb[:-1])
    keep[pi[last]] = 1
    return keep


@pytest.mark.parametrize("shape", [(12, 10), (64, 48), (6, 5, 4), (20, 18, 16), (3, 3, 3, 3), (8, 7, 6, 5),
                                   (4, 4, 3, 3, 3)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind", ["normal", "ties"])
@pytest.mark.parametrize("minimum", [False, True])
def test_bundling_matches_oracle(handles, shape, kind, minimum):
    seed = zlib.crc32(repr((shape, kind, "gpu-bundle")).encode()) % 1000
    f = (F.white_noise(shape, seed) if kind == "normal" else F.integer_ties(shape, seed, 3)).values
    g, keep = gpu_bundle(handles[minimum], f)
    o = oracle.compute(f, minimum=minimum)
    assert np.array_equal(g.saddles, o.saddles)
    want = oracle.bundle(o, minimum=minimum)
    assert np.array_equal(keep, want)
    assert np.array_equal(want, bundle_vectorised(o.saddles, o.sad_val, o.row_ptr, o.col, minimum))


def test_bundling_large_field(handles):
    f = F.config_3d_512(side=160).values
    g, keep = gpu_bundle(handles[False], f)
    want = bundle_vectorised(g.saddles, g.sad_val, g.row_ptr, g.col)
    assert np.array_equal(keep, want)
    assert 0 < int(keep.sum()) < g.saddles.size


def test_bundling_no_saddles(handles):
    g, keep = gpu_bundle(handles[False], np.arange(30, dtype=np.float32).reshape(5, 6))
    assert g.saddles.size == 0 and keep.size == 0
