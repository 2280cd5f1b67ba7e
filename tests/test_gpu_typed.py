"""Element types other than float32 (Sec. 5: 8- to 64-bit integers, float64):
GPU path vs the CPU oracle, bit-exact (labels, nodes, arcs; value copies
compared as bytes), through the C ABI (eg_compute_typed, eg_batch_submit with
EG_FLAG_DTYPE, eg_get_bundled, eg_get_paths)."""
import ctypes
import zlib

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TYPES = [t for t in F.ELEMENT_TYPES if t != "float32"]


@pytest.fixture(scope="module")
def handles():
    from paper_2303_02724_gb300 import _build, eg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    hs = {False: eg.Handle(0), True: eg.Handle(0, minimum=True)}
    yield hs
    for h in hs.values():
        h.close()


def typed_graph(h, values, labels=True):
    from paper_2303_02724_gb300 import eg
    t = eg.device_array(values)
    rid = h.compute(t, dtype=values.dtype)
    try:
        return h.get_graph(rid, labels=labels)
    finally:
        h.release(rid)


def assert_same(gg, og, labels=True):
    assert np.array_equal(gg.maxima, og.maxima), "maxima"
    assert np.array_equal(gg.saddles, og.saddles), "saddles"
    assert np.array_equal(gg.sad_b0, og.sad_b0), "beta0+"
    assert np.array_equal(gg.row_ptr, og.row_ptr), "row_ptr"
    assert np.array_equal(gg.col, og.col), "col"
    assert gg.n_paths == og.n_paths
    assert gg.max_val.dtype == og.max_val.dtype and gg.sad_val.dtype == og.sad_val.dtype
    assert gg.max_val.tobytes() == og.max_val.tobytes(), "max_val"
    assert gg.sad_val.tobytes() == og.sad_val.tobytes(), "sad_val"
    if labels:
        assert np.array_equal(gg.labels, og.label), "labels"


EDGE_SHAPES = [(9,), (8, 8), (17, 9), (4, 4, 4), (9, 7, 5), (3, 3, 3, 3), (5, 4, 3, 2), (1, 1, 1, 7),
               (3, 3, 3, 3, 3)]


@pytest.mark.parametrize("dtype", TYPES)
@pytest.mark.parametrize("shape", EDGE_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("minimum", [False, True])
def test_edge_values(handles, dtype, shape, minimum):
    """Each type's boundary values (extremes, both sides of the sign bit,
    neighbours float32 cannot separate), heavy ties."""
    seed = zlib.crc32(repr((shape, dtype, "gpu")).encode()) % 10000
    f = F.typed_ties(shape, seed, dtype).values
    og = oracle.compute(f, extents=shape, minimum=minimum, dtype=f.dtype)
    assert_same(typed_graph(handles[minimum], f), og)


@pytest.mark.parametrize("dtype", TYPES)
@pytest.mark.parametrize("case", ["grf3d", "gauss2d", "rows2d_wide", "white4d", "plateaus3d"])
def test_quantised_fields(handles, dtype, case):
    """Structured fields in every type, several bricks and a ragged tail:
    3D and 2D fields (plane-marching classifier for the narrow types), 2D rows
    longer than 1024 and 4D (flat classifier), and coarse plateaus (32 levels)
    where the index tie-break decides most comparisons."""
    base, levels = {
        "grf3d": (lambda: F.grf((48, 40, 36), 2), None),
        "gauss2d": (lambda: F.config_2d_256(side=150), None),
        "rows2d_wide": (lambda: F.white_noise((1100, 7), 5), None),
        "white4d": (lambda: F.white_noise((9, 8, 7, 6), 6), None),
        "plateaus3d": (lambda: F.config_3d_256(side=33), 32),
    }[case]
    fld = base()
    f = F.quantise(fld, dtype, levels=levels if np.dtype(dtype).kind in "iu" else None).values
    og = oracle.compute(f, extents=fld.extents, dtype=f.dtype)
    assert_same(typed_graph(handles[False], f), og)


@pytest.mark.parametrize("dtype", ["float64", "int32", "uint16"])
def test_minimum_graph_quantised(handles, dtype):
    fld = F.grf((40, 36, 30), 9)
    f = F.quantise(fld, dtype).values
    og = oracle.compute(f, extents=fld.extents, minimum=True, dtype=f.dtype)
    assert_same(typed_graph(handles[True], f), og)


def test_float64_image_of_float32_field(handles):
    """Every float32 is a float64 and the order is kept, so the float64 image
    of a float32 field has the same graph (values widened)."""
    fld = F.config_3d_256(side=40)
    g32 = handles[False].graph_of(torch.from_numpy(fld.values).cuda())
    g64 = typed_graph(handles[False], fld.values.astype(np.float64))
    for k in ["labels", "maxima", "saddles", "sad_b0", "row_ptr", "col"]:
        assert np.array_equal(getattr(g32, k), getattr(g64, k)), k
    assert np.array_equal(g32.max_val.astype(np.float64), g64.max_val)


def test_batch_mixed_types(handles):
    """One submission holding every type (and float32), replayed from its
    captured graphs on a second submission with new values."""
    from paper_2303_02724_gb300 import eg
    h = handles[False]
    shapes = [(40, 33), (20, 18, 9), (7, 6, 5, 4), (1100, 3), (30, 30)]
    for rep in range(2):
        vals, dts = [], []
        for i, dt in enumerate(F.ELEMENT_TYPES):
            shape = shapes[i % len(shapes)]
            fld = F.grf(shape, 100 * rep + i) if len(shape) == 3 else F.white_noise(shape, 100 * rep + i)
            vals.append(F.quantise(fld, dt, levels=50 if np.dtype(dt).kind in "iu" else None).values)
            dts.append(np.dtype(dt))
        ts = [eg.device_array(v) for v in vals]
        ids = h.batch_submit(ts, dtypes=dts)
        for rid, v, dt in zip(ids, vals, dts):
            gg = h.get_graph(rid)
            h.release(rid)
            og = oracle.compute(v, dtype=dt)
            assert_same(gg, og)


@pytest.mark.parametrize("dtype", ["uint64", "int64", "float64", "int8", "uint32"])
@pytest.mark.parametrize("minimum", [False, True])
def test_bundling(handles, dtype, minimum):
    from paper_2303_02724_gb300 import eg
    for seed, shape in [(1, (12, 11, 10)), (2, (30, 25)), (3, (6, 5, 4, 4))]:
        f = F.typed_ties(shape, seed, dtype).values
        h = handles[minimum]
        rid = h.compute(eg.device_array(f), dtype=f.dtype)
        try:
            gg = h.get_graph(rid, labels=False)
            keep = h.get_bundled(rid)
        finally:
            h.release(rid)
        og = oracle.compute(f, extents=shape, minimum=minimum, dtype=f.dtype)
        assert_same(gg, og, labels=False)
        assert np.array_equal(keep, oracle.bundle(og, minimum=minimum))


def test_paths(handles):
    from paper_2303_02724_gb300 import eg
    h = eg.Handle(0, paths=True)
    try:
        for dt, shape in [("uint8", (20, 17, 9)), ("int64", (13, 12, 11)), ("float64", (5, 5, 4, 3))]:
            f = F.quantise(F.grf(shape, 4) if len(shape) == 3 else F.white_noise(shape, 4), dt, levels=40
                           if np.dtype(dt).kind in "iu" else None).values
            rid = h.compute(eg.device_array(f), dtype=f.dtype)
            ptr, vtx = h.get_paths(rid)
            h.release(rid)
            og = oracle.compute(f, extents=shape, paths=True, dtype=f.dtype)
            assert np.array_equal(ptr, og.path_ptr) and np.array_equal(vtx, og.path_vtx)
    finally:
        h.close()


def test_errors(handles):
    from paper_2303_02724_gb300 import eg
    h = handles[False]
    f = np.zeros((8, 8), np.float64)
    f[3, 4] = np.nan
    with pytest.raises(eg.EGError) as ei:
        typed_graph(h, f)
    assert ei.value.status == eg.EG_ERR_NAN
    # unknown type code, misaligned field
    lib = eg.load()
    t = torch.zeros(65, dtype=torch.int64, device="cuda")
    ext = (ctypes.c_int64 * 1)(64)
    rid = ctypes.c_uint64()
    st = lib.eg_compute_typed(h._h, ctypes.c_void_p(t.data_ptr()), 10, 1, ext, None, ctypes.byref(rid))
    assert st == eg.EG_ERR_ARG
    st = lib.eg_compute_typed(h._h, ctypes.c_void_p(t.data_ptr() + 4), eg.DTYPES[np.dtype(np.int64)], 1, ext,
                              None, ctypes.byref(rid))
    assert st == eg.EG_ERR_ARG
    assert lib.eg_dtype_size(9) == 8 and lib.eg_dtype_size(3) == 1 and lib.eg_dtype_size(10) == 0
    # the context is still usable
    g = typed_graph(h, np.arange(12, dtype=np.int16).reshape(3, 4))
    assert g.maxima.tolist() == [11]
