"""Parity at the full sizes of the synthetic configurations.

* 2D 256x256 and 3D 256^3: the whole result against the oracle.
* 3D 512^3 GRF (134M vertices, too large for the sequential oracle in a test):
  the oracle runs on random interior sub-boxes.  Classification is local (a
  vertex and its 1-ring), and the index order inside a sub-box is the global
  order restricted to it, so for every vertex at least one layer inside a
  sub-box the oracle's beta0+, maximum/saddle status and gradient pointer are
  the global ones.  They pin the GPU result through:
    - maxima and saddles (with beta0+) inside the box equal the oracle's;
    - label(v) == label(asc(v)) for every inner vertex (the GPU labels follow
      the oracle's gradient);
    - for every inner saddle, its arcs are exactly {label(rep(C))} over the
      oracle's upper-link representatives;
  plus global invariants over all 134M labels (every label is a maximum).
"""
import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    h = eg.Handle(0)
    yield h
    h.close()


def _same(gg, og):
    assert np.array_equal(gg.maxima, og.maxima)
    assert np.array_equal(gg.saddles, og.saddles)
    assert np.array_equal(gg.sad_b0, og.sad_b0)
    assert np.array_equal(gg.row_ptr, og.row_ptr)
    assert np.array_equal(gg.col, og.col)
    assert np.array_equal(gg.labels, og.label)
    assert np.array_equal(gg.max_val.view(np.uint32), og.max_val.view(np.uint32))
    assert np.array_equal(gg.sad_val.view(np.uint32), og.sad_val.view(np.uint32))


def test_config_3d_256_full(handle):
    f = F.config_3d_256()
    g = handle.graph_of(torch.from_numpy(f.values).cuda())
    _same(g, oracle.compute(f.values))


def _check_box(g, vals, z0, y0, x0, b, is_max_gpu, sad_index):
    n2, n1, n0 = vals.shape
    sub = np.ascontiguousarray(vals[z0:z0 + b, y0:y0 + b, x0:x0 + b])
    o = oracle.compute(sub)
    lz, ly, lx = np.meshgrid(np.arange(b), np.arange(b), np.arange(b), indexing="ij")
    inner = ((lz > 0) & (lz < b - 1) & (ly > 0) & (ly < b - 1) & (lx > 0) & (lx < b - 1)).reshape(-1)
    loc = np.arange(b ** 3)[inner]

    def to_global(li):
        li = np.asarray(li, np.int64)
        x, y, z = li % b, (li // b) % b, li // (b * b)
        return ((z + z0) * n1 + (y + y0)) * n0 + (x + x0)

    gv = to_global(loc)
    # classification of inner vertices
    assert np.array_equal(o.beta0p[loc] == 0, is_max_gpu[gv])
    o_sad = set(to_global(o.saddles[np.isin(o.saddles, loc)]).tolist())
    g_sad_here = set(gv[sad_index[gv] >= 0].tolist())
    assert o_sad == g_sad_here
    # labels follow the oracle's gradient
    asc_g = to_global(o.asc[loc])
    assert np.array_equal(g.labels[gv], g.labels[asc_g])
    # arcs of inner saddles: the ends are the labels of the oracle's upper-link
    # representatives (the representatives depend on the saddle's link only)
    inner_sad = np.flatnonzero(np.isin(o.saddles, loc))
    for i_o in inner_sad[:300]:
        s_g = int(to_global([o.saddles[i_o]])[0])
        i = sad_index[s_g]
        assert g.sad_b0[i] == o.sad_b0[i_o]
        row = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        want = np.unique(g.labels[to_global(o.saddle_reps(i_o))])
        assert np.array_equal(row, want.astype(np.uint32))


def test_config_3d_512_sampled(handle):
    f = F.config_3d_512()
    vals = f.values
    g = handle.graph_of(torch.from_numpy(vals).cuda())
    N = vals.size
    is_max = np.zeros(N, bool)
    is_max[g.maxima] = True
    # global invariants
    assert np.all(is_max[g.labels])
    assert np.array_equal(g.labels[g.maxima], g.maxima)
    assert len(g.row_ptr) == len(g.saddles) + 1 and g.row_ptr[-1] == len(g.col)
    assert np.all(is_max[g.col])
    assert np.all(np.diff(g.saddles.astype(np.int64)) > 0) and np.all(np.diff(g.maxima.astype(np.int64)) > 0)
    assert np.array_equal(g.max_val.view(np.uint32), vals.reshape(-1)[g.maxima].view(np.uint32))
    assert np.array_equal(g.sad_val.view(np.uint32), vals.reshape(-1)[g.saddles].view(np.uint32))
    sad_index = np.full(N, -1, np.int64)
    sad_index[g.saddles] = np.arange(len(g.saddles))
    rng = np.random.default_rng(99)
    b = 28
    boxes = [(0, 0, 0), (512 - b, 512 - b, 512 - b)]
    boxes += [tuple(int(t) for t in rng.integers(0, 512 - b, size=3)) for _ in range(6)]
    for (z0, y0, x0) in boxes:
        _check_box(g, vals, z0, y0, x0, b, is_max, sad_index)
