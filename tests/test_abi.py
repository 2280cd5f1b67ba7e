"""The C-ABI library builds, loads and exports every symbol include/eg.h declares.

No compute call is made (this runs without a GPU)."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2303_02724_gb300 import _build, eg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "eg.h")).read()
    return sorted(set(re.findall(r"EG_API\s+[^;]*?\b(eg_\w+)\s*\(", src, re.S)))


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for name in ["eg_create", "eg_destroy", "eg_compute", "eg_batch_submit", "eg_get_graph",
                 "eg_release", "eg_status_str"]:
        assert name in syms


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(eg_\w+)\b", out))
    missing = [s for s in _declared_symbols() if s not in exported]
    assert not missing, missing
    # nothing else leaks out of the library under the eg_ prefix
    assert exported <= set(_declared_symbols())


def test_binding_covers_header():
    assert set(eg.SIGNATURES) == set(_declared_symbols())


def test_loads_and_host_only_calls(lib_path):
    lib = eg.load(lib_path)
    assert eg.status_str(eg.EG_ERR_NAN) == "field contains NaN"
    assert eg.status_str(0) == "ok"
    # workspace estimate is pure host arithmetic
    assert eg.workspace_bytes((256, 256)) > 256 * 256 * 4
    assert eg.workspace_bytes((0, 4)) == 0
    assert eg.workspace_bytes((1 << 16, 1 << 16, 2)) == 0  # more than 2^32 - 1 vertices
    assert lib.eg_launch_count(None) == 0
    assert lib.eg_release(None, 1) == eg.EG_ERR_ARG
    assert lib.eg_destroy(None) == eg.EG_OK


def test_graph_buffers_views():
    from paper_2303_02724_gb300 import eg
    b = eg.GraphBuffers(5, 7, 11, 13)
    assert b.fits(5, 7, 11, 13) and not b.fits(6, 7, 11, 13) and not b.fits(5, 7, 12)
    g = b.views(2, 3, 4)
    assert (g.maxima.size, g.saddles.size, g.row_ptr.size, g.col.size, g.labels) == (2, 3, 4, 4, None)
    assert g.row_ptr.dtype == np.uint64 and g.sad_b0.dtype == np.uint8
    assert np.shares_memory(g.col, b.arrays["col"])
    assert b.views(0, 0, 0, 13).labels.size == 13
    with pytest.raises(ValueError):
        b.views(6, 0, 0)
    # value copies take the field's element type; buffers of another type do not fit
    b64 = eg.GraphBuffers(5, 7, 11, dtype=np.uint64)
    g64 = b64.views(2, 3, 4, dtype=np.uint64)
    assert g64.max_val.dtype == np.uint64 and g64.sad_val.dtype == np.uint64
    assert g64.maxima.dtype == np.uint32 and g64.col.dtype == np.uint32
    assert not b64.fits(2, 3, 4) and not b.fits(2, 3, 4, dtype=np.int8)
    with pytest.raises(ValueError):
        b64.views(2, 3, 4)


def test_element_type_codes():
    """The binding's element-type codes follow eg_dtype, and the library
    reports each type's size (no GPU needed)."""
    from paper_2303_02724_gb300 import eg
    lib = eg.load()
    for dt, code in eg.DTYPES.items():
        assert lib.eg_dtype_size(code) == dt.itemsize
        assert eg.dtype_flag(dt) == code << 16
    assert lib.eg_dtype_size(-1) == 0 and lib.eg_dtype_size(len(eg.DTYPES)) == 0
    hdr = open(os.path.join(ROOT, "include", "eg.h")).read()
    names = {"float32": "F32", "float64": "F64", "int8": "I8", "uint8": "U8", "int16": "I16", "uint16": "U16",
             "int32": "I32", "uint32": "U32", "int64": "I64", "uint64": "U64"}
    for dt, code in eg.DTYPES.items():
        assert re.search(rf"EG_DTYPE_{names[dt.name]}\s*=\s*{code}\b", hdr), dt


def test_kernel_fingerprint_ignores_comments_only():
    """The profiles' traffic figures are tied to a kernel's code: comments
    and layout do not change the fingerprint, code and string literals do."""
    a = "int a = 1; // one\n/* block\n comment */ float f(float x) { return x * 2.f; }\n"
    b = "int a = 1;\n\n   float f(float x)  {  return x * 2.f; }   // changed comment\n"
    c = "int a = 2; float f(float x) { return x * 2.f; }\n"
    d = 'const char *s = "// kept"; int a = 1;\n'
    e = 'const char *s = "// kept!"; int a = 1;\n'
    fp = lambda t: _build.code_fingerprint_of([("k.cu", t)])
    assert fp(a) == fp(b)
    assert fp(a) != fp(c)
    assert fp(d) != fp(e)
    assert _build._code_text(d) == 'const char *s = "// kept"; int a = 1;'


def test_bench_byte_accounting():
    """The roofline's algorithmic bytes: the field in its element type, the
    labels, the records and the graph (counts of a hand-made result)."""
    import bench
    c = dict(n_vertices=1000, n_maxima=10, n_saddles=20, n_paths=45, n_arcs=40)
    kb = bench.kernel_bytes(c)
    assert kb["classify"] == 4 * 1000 + 4 * 1000 + 12 * 30
    assert kb["resolve"] == 8 * 1000
    assert kb["emit"] == 12 * 30 + 4 * 45 + 8 * 10 + 9 * 20 + 8 * 21 + 4 * 40
    assert bench.path_bytes(c) == 8 * 1000 + 8 * 10 + 9 * 20 + 8 * 21 + 4 * 40
    # a uint8 field: 1 byte per value read and per value copy
    kb8 = bench.kernel_bytes(c, es=1)
    assert kb8["classify"] == 1000 + 4 * 1000 + 12 * 30
    assert bench.path_bytes(c, es=1) == 1000 + 4 * 1000 + 5 * 10 + 6 * 20 + 8 * 21 + 4 * 40


def _bench(args, env_extra=None):
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          timeout=300, cwd=ROOT, env=env)


def test_bench_reference_arm_line():
    """The reference arm times the oracle on the host cores and prints one
    JSON line with the contract's keys (no GPU needed)."""
    import json
    r = _bench(["--impl", "reference", "--workload", "gauss2d256", "--steps", "1", "--warmup", "0",
                "--ref-sample-vertices", "65536"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "Mvertices/s" and line["higher_is_better"] is True
    assert line["warmup"] >= 3 and line["steps"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Mvertices/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "65536 vertices" in line["config"]["sample"]


def test_bench_reference_sample_is_bounded():
    """The reference arm keeps the cpu_baseline leg's sample for a usual run
    and shrinks it when many steps would take the oracle more than a few
    minutes in all."""
    import bench
    four_m = 4 * 1024 * 1024
    assert bench.ref_sample_cap(20, 5, four_m) == four_m
    big = bench.ref_sample_cap(200, 3, four_m)
    assert big < four_m and big * 203 <= bench.REF_BUDGET_VERTICES
    assert bench.ref_sample_cap(10 ** 7, 3, four_m) == 65536


def test_bench_reference_arm_other_ranks_are_silent():
    """Under a multi-rank launch only rank 0 runs the reference arm; the
    other ranks exit 0 without work or output."""
    r = _bench(["--impl", "reference", "--workload", "gauss2d256", "--steps", "1", "--warmup", "0",
                "--ref-sample-vertices", "65536"], {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_labels_static_checks_arguments_before_any_launch():
    """eg_labels_static's binding rejects a labels buffer of another size, a
    non-float32 field, a float labels buffer and strided views before it
    touches the library (CPU tensors here: no device is involved)."""
    torch = pytest.importorskip("torch")
    f = torch.zeros((4, 5), dtype=torch.float32)
    with pytest.raises(ValueError, match="elements"):
        eg.labels_static(f, torch.zeros(19, dtype=torch.int32))
    with pytest.raises(ValueError, match="float32"):
        eg.labels_static(f.to(torch.int32), torch.zeros(20, dtype=torch.int32))
    with pytest.raises(ValueError, match="integer"):
        eg.labels_static(f, torch.zeros(20, dtype=torch.float32))
    with pytest.raises(ValueError, match="contiguous"):
        eg.labels_static(torch.zeros((5, 4), dtype=torch.float32).t(), torch.zeros((4, 5), dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        eg.labels_static(f, torch.zeros((4, 5), dtype=torch.int32))


def test_checked_build_compiles_with_the_same_symbols():
    """The bounds-checked variant (EG_CHECKED) builds and exports exactly the
    declared symbols (no GPU needed)."""
    path = _build.build(checked=True)
    assert path.endswith("libeg_checked.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    assert set(re.findall(r"\b(eg_\w+)\b", out)) == set(_declared_symbols())
