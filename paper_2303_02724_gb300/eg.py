"""Python binding of the C ABI in include/eg.h (argument marshalling only).

Every step of the computation runs in the CUDA library; this module only
converts torch tensors / numpy arrays to pointers and sizes and back.  There
is no CPU fallback: if libeg.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# EG_CHECKED_LIBRARY=1 selects the bounds-checked build (libeg_checked.so,
# built by _build.build(checked=True)) for test runs
LIB_PATH = os.path.join(_HERE, "libeg_checked.so" if os.environ.get("EG_CHECKED_LIBRARY") == "1" else "libeg.so")
MAX_DIM = 5

EG_OK, EG_ERR_ARG, EG_ERR_NAN, EG_ERR_OOM, EG_ERR_CUDA = 0, 1, 2, 3, 4
EG_ERR_NOT_CONVERGED, EG_ERR_TIMEOUT, EG_ERR_BUSY, EG_ERR_INTERNAL = 5, 6, 7, 8
EG_FLAG_MINIMUM_GRAPH = 0x1
EG_FLAG_NO_LABELS = 0x2
EG_FLAG_NO_GRAPH = 0x4
EG_FLAG_PATHS = 0x8
EG_FLAG_NO_FUSED = 0x10

# element types (eg_dtype): numpy dtype <-> code; EG_FLAG_DTYPE(t) = t << 16
DTYPES = {np.dtype(np.float32): 0, np.dtype(np.float64): 1, np.dtype(np.int8): 2, np.dtype(np.uint8): 3,
          np.dtype(np.int16): 4, np.dtype(np.uint16): 5, np.dtype(np.int32): 6, np.dtype(np.uint32): 7,
          np.dtype(np.int64): 8, np.dtype(np.uint64): 9}
DTYPE_OF_CODE = {v: k for k, v in DTYPES.items()}


def dtype_flag(dtype) -> int:
    """eg_field_desc.flags bits naming a field's element type."""
    return DTYPES[np.dtype(dtype)] << 16


class EGError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})" if what else status_str(status))


class EGConfig(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("classify_rows", ctypes.c_int32),
                ("classify_planes", ctypes.c_int32), ("resolve_walks", ctypes.c_int32),
                ("persistent_ctas", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k in ["flags", "classify_rows", "classify_planes",
                                               "resolve_walks", "persistent_ctas"]}


class EGFieldDesc(ctypes.Structure):
    _fields_ = [("field", ctypes.c_void_p), ("d", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("extents", ctypes.c_int64 * MAX_DIM)]


# the same layout as a numpy record, for filling many descriptors at once
_DESC_DTYPE = np.dtype([("field", np.uint64), ("d", np.int32), ("flags", np.int32),
                        ("extents", np.int64, (MAX_DIM,))])
assert _DESC_DTYPE.itemsize == ctypes.sizeof(EGFieldDesc)


class EGGraphC(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("dtype", ctypes.c_int32), ("extents", ctypes.c_int64 * MAX_DIM),
                ("n_vertices", ctypes.c_int64), ("n_maxima", ctypes.c_int64),
                ("n_saddles", ctypes.c_int64), ("n_paths", ctypes.c_int64),
                ("n_arcs", ctypes.c_int64),
                ("maxima", ctypes.c_void_p), ("max_val", ctypes.c_void_p),
                ("saddles", ctypes.c_void_p), ("sad_beta0", ctypes.c_void_p),
                ("sad_val", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("labels", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); every symbol declared in include/eg.h
_P = ctypes.c_void_p
SIGNATURES = {
    "eg_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(EGConfig)]),
    "eg_destroy": (ctypes.c_int, [_P]),
    "eg_compute": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "eg_compute_host": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "eg_compute_typed": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "eg_dtype_size": (ctypes.c_size_t, [ctypes.c_int]),
    "eg_batch_submit": (ctypes.c_int, [_P, ctypes.POINTER(EGFieldDesc), ctypes.c_int, _P,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "eg_get_graph": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(EGGraphC)]),
    "eg_get_graph_device": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(EGGraphC)]),
    "eg_get_graphs_device": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
                                            ctypes.POINTER(EGGraphC), ctypes.POINTER(ctypes.c_int32)]),
    "eg_get_paths": (ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "eg_get_bundled": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "eg_get_cancelled": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_float, _P, _P,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "eg_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "eg_workspace_bytes": (ctypes.c_uint64, [ctypes.c_int, _P]),
    "eg_mem_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64)]),
    "eg_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "eg_step_times": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]),
    "eg_launch_count": (ctypes.c_uint64, [_P]),
    "eg_debug_fail_alloc": (ctypes.c_int, [_P, ctypes.c_int]),
    "eg_debug_wait_timeout": (ctypes.c_int, [_P, _P]),
    "eg_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "eg_labels_static": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_uint32, _P, _P]),
    "eg_autotune": (ctypes.c_int, [_P, ctypes.POINTER(EGFieldDesc), ctypes.c_int, _P, ctypes.POINTER(EGConfig)]),
}

STATIC_MAX_VERTICES = 1 << 20


def load(path: str = LIB_PATH):
    """Load libeg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the library has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_str(s: int) -> str:
    try:
        return load().eg_status_str(int(s)).decode()
    except Exception:  # library missing: still give a readable message
        return f"status {s}"


def _check(s: int, what: str):
    if s != EG_OK:
        raise EGError(s, what)


def _extents_of(shape) -> tuple:
    return tuple(int(x) for x in reversed(tuple(shape)))


@dataclass
class Graph:
    """Extremum graph copied to host memory."""
    d: int
    extents: tuple
    n_vertices: int
    n_paths: int
    maxima: np.ndarray
    max_val: np.ndarray
    saddles: np.ndarray
    sad_b0: np.ndarray
    sad_val: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    labels: Optional[np.ndarray]

    def arcs(self):
        out = set()
        for i, s in enumerate(self.saddles.tolist()):
            for m in self.col[self.row_ptr[i]:self.row_ptr[i + 1]].tolist():
                out.add((s, m))
        return out


class GraphBuffers:
    """Host arrays a result is copied into, sized for up to M maxima, S
    saddles, A arcs and N labels.  pinned=True allocates page-locked memory
    (through torch), so the device-to-host copies run at link speed; the same
    buffers can be reused for every result that fits (the Graph returned by
    get_graph then views them, so it is only valid until the next reuse)."""

    _FIELDS = (("maxima", np.uint32, "M"), ("max_val", None, "M"), ("saddles", np.uint32, "S"),
               ("sad_b0", np.uint8, "S"), ("sad_val", None, "S"), ("row_ptr", np.uint64, "S1"),
               ("col", np.uint32, "A"), ("labels", np.uint32, "N"))

    def __init__(self, M: int, S: int, A: int, N: int = 0, pinned: bool = False, dtype=np.float32):
        self.cap = {"M": int(M), "S": int(S), "S1": int(S) + 1, "A": int(A), "N": int(N)}
        self.dtype = np.dtype(dtype)  # element type of the value copies
        self.arrays = {}
        for name, dt, k in self._FIELDS:
            dt = self.dtype if dt is None else dt
            n = self.cap[k]
            if pinned and n:
                import torch
                buf = torch.empty(n * np.dtype(dt).itemsize, dtype=torch.uint8, pin_memory=True).numpy()
                self.arrays[name] = buf.view(dt)
            else:
                self.arrays[name] = np.empty(n, dt)

    def fits(self, M: int, S: int, A: int, N: int = 0, dtype=np.float32) -> bool:
        c = self.cap
        return (M <= c["M"] and S <= c["S"] and A <= c["A"] and N <= c["N"]
                and np.dtype(dtype) == self.dtype)

    def views(self, M: int, S: int, A: int, N: int = 0, dtype=np.float32) -> Graph:
        if not self.fits(M, S, A, N, dtype):
            raise ValueError("result larger than the buffers")
        a = self.arrays
        return Graph(d=0, extents=(), n_vertices=0, n_paths=0, maxima=a["maxima"][:M], max_val=a["max_val"][:M],
                     saddles=a["saddles"][:S], sad_b0=a["sad_b0"][:S], sad_val=a["sad_val"][:S],
                     row_ptr=a["row_ptr"][:S + 1], col=a["col"][:A], labels=a["labels"][:N] if N else None)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Handle:
    """One library handle on one CUDA device."""

    def __init__(self, device: int = 0, minimum: bool = False, config: Optional[EGConfig] = None,
                 paths: bool = False):
        lib = load()
        cfg = config if config is not None else EGConfig()
        if minimum:
            cfg.flags |= EG_FLAG_MINIMUM_GRAPH
        if paths:
            cfg.flags |= EG_FLAG_PATHS
        h = ctypes.c_void_p()
        _check(lib.eg_create(ctypes.byref(h), int(device), ctypes.byref(cfg)), "eg_create")
        self._h = h
        self._lib = lib
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._lib.eg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- submit
    def compute(self, field, stream=None, dtype=None) -> int:
        """field: contiguous CUDA tensor; axis 0 of the grid is its LAST dim.
        dtype None: float32 (eg_compute).  Otherwise a numpy element type (see
        DTYPES): the tensor holds the elements as raw bytes of that size (any
        torch dtype of the same item size, e.g. from device_array) and the call
        is eg_compute_typed."""
        if not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA tensor")
        ext = _extents_of(field.shape)
        e = (ctypes.c_int64 * max(1, len(ext)))(*ext)
        rid = ctypes.c_uint64()
        if dtype is None:
            if field.dtype.itemsize != 4:
                raise ValueError("field must be a float32 CUDA tensor (or pass dtype)")
            _check(self._lib.eg_compute(self._h, ctypes.c_void_p(field.data_ptr()), len(ext), e,
                                        ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(rid)),
                   "eg_compute")
        else:
            dt = np.dtype(dtype)
            if dt not in DTYPES or field.element_size() != dt.itemsize:
                raise ValueError(f"element type {dt} does not match the tensor")
            _check(self._lib.eg_compute_typed(self._h, ctypes.c_void_p(field.data_ptr()), DTYPES[dt], len(ext),
                                              e, ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(rid)),
                   "eg_compute_typed")
        return rid.value

    def compute_host(self, field: np.ndarray, stream=None) -> int:
        """field: float32 numpy array in host memory (copied inside the call)."""
        a = np.ascontiguousarray(field, dtype=np.float32)
        ext = _extents_of(a.shape)
        e = (ctypes.c_int64 * max(1, len(ext)))(*ext)
        rid = ctypes.c_uint64()
        _check(self._lib.eg_compute_host(self._h, ctypes.c_void_p(a.ctypes.data), len(ext), e,
                                         ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(rid)),
               "eg_compute_host")
        return rid.value

    def batch_submit(self, fields: Sequence, stream=None, flags: Sequence[int] = (),
                     dtypes: Sequence = ()) -> list:
        """dtypes[i] (numpy element type, default float32) names the element
        type of fields[i] (a CUDA tensor of that item size)."""
        n = len(fields)
        descs = self._descs(fields, flags, dtypes)
        ids = (ctypes.c_uint64 * max(1, n))()
        _check(self._lib.eg_batch_submit(self._h, descs, n, ctypes.c_void_p(_stream_ptr(stream)), ids),
               "eg_batch_submit")
        return [ids[i] for i in range(n)]

    def batch_submit_ptrs(self, ptrs: Sequence[int], extents: Sequence[tuple], stream=None) -> list:
        """eg_batch_submit for float32 fields given as device addresses and
        their extents (axis 0 first), without tensor objects per field."""
        n = len(ptrs)
        # the descriptor array filled column by column (EGFieldDesc's layout)
        arr = np.zeros(max(1, n), dtype=_DESC_DTYPE)
        arr["field"][:n] = ptrs
        for i, ext in enumerate(extents):
            arr["d"][i] = len(ext)
            arr["extents"][i, :len(ext)] = ext
        descs = ctypes.cast(arr.ctypes.data, ctypes.POINTER(EGFieldDesc))
        ids = (ctypes.c_uint64 * max(1, n))()
        _check(self._lib.eg_batch_submit(self._h, descs, n, ctypes.c_void_p(_stream_ptr(stream)), ids),
               "eg_batch_submit")
        return list(ids[:n])

    def autotune(self, fields: Sequence, stream=None) -> dict:
        """Pick the fastest knob values on these fields; returns them."""
        descs = self._descs(fields)
        best = EGConfig()
        _check(self._lib.eg_autotune(self._h, descs, len(fields), ctypes.c_void_p(_stream_ptr(stream)),
                                     ctypes.byref(best)), "eg_autotune")
        return best.as_dict()

    def _descs(self, fields, flags=(), dtypes=()):
        n = len(fields)
        descs = (EGFieldDesc * max(1, n))()
        for i, f in enumerate(fields):
            dt = np.dtype(dtypes[i]) if i < len(dtypes) and dtypes[i] is not None else np.dtype(np.float32)
            if not f.is_cuda or dt not in DTYPES or f.element_size() != dt.itemsize or not f.is_contiguous():
                raise ValueError("fields must be contiguous CUDA tensors of their element types")
            ext = _extents_of(f.shape)
            descs[i].field = f.data_ptr()
            descs[i].d = len(ext)
            descs[i].flags = (int(flags[i]) if i < len(flags) else 0) | (DTYPES[dt] << 16)
            for k, x in enumerate(ext):
                descs[i].extents[k] = x
        return descs

    # --------------------------------------------------------------- results
    def counts(self, rid: int) -> dict:
        g = EGGraphC()
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        return dict(n_vertices=g.n_vertices, n_maxima=g.n_maxima, n_saddles=g.n_saddles,
                    n_paths=g.n_paths, n_arcs=g.n_arcs)

    def get_graph(self, rid: int, labels: bool = True, buffers: "GraphBuffers" = None) -> Graph:
        """Copy a result to host memory.  With `buffers` (see GraphBuffers, e.g.
        pinned and reused across calls) the arrays of the returned Graph are
        views into them; otherwise fresh numpy arrays."""
        g = EGGraphC()
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        M, S, A, N = g.n_maxima, g.n_saddles, g.n_arcs, g.n_vertices
        vdt = DTYPE_OF_CODE[g.dtype]
        if buffers is None:
            buffers = GraphBuffers(M, S, A, N if labels else 0, dtype=vdt)
        out = buffers.views(M, S, A, N if labels else 0, dtype=vdt)
        out.d, out.extents, out.n_vertices, out.n_paths = g.d, tuple(g.extents[:g.d]), N, g.n_paths
        if not labels:
            out.labels = None
        g.maxima = out.maxima.ctypes.data
        g.max_val = out.max_val.ctypes.data
        g.saddles = out.saddles.ctypes.data
        g.sad_beta0 = out.sad_b0.ctypes.data
        g.sad_val = out.sad_val.ctypes.data
        g.row_ptr = out.row_ptr.ctypes.data
        g.col = out.col.ctypes.data
        g.labels = out.labels.ctypes.data if labels else None
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        return out

    def get_bundled(self, rid: int) -> np.ndarray:
        """Arc bundling of a finished result: uint8 per saddle, 1 = kept."""
        g = EGGraphC()
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        keep = np.empty(max(1, g.n_saddles), np.uint8)
        _check(self._lib.eg_get_bundled(self._h, ctypes.c_uint64(rid), ctypes.c_void_p(keep.ctypes.data)),
               "eg_get_bundled")
        return keep[:g.n_saddles]

    def get_cancelled(self, rid: int, tau: float):
        """Persistence-directed cancellation of a finished float32 result with
        threshold tau: (alive uint8[S], survivor uint32[M], n_cancelled,
        rounds)."""
        g = EGGraphC()
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        alive = np.empty(max(1, g.n_saddles), np.uint8)
        surv = np.empty(max(1, g.n_maxima), np.uint32)
        n = ctypes.c_int64()
        rounds = ctypes.c_int32()
        _check(self._lib.eg_get_cancelled(self._h, ctypes.c_uint64(rid), ctypes.c_float(tau),
                                          ctypes.c_void_p(alive.ctypes.data), ctypes.c_void_p(surv.ctypes.data),
                                          ctypes.byref(n), ctypes.byref(rounds)), "eg_get_cancelled")
        return alive[:g.n_saddles], surv[:g.n_maxima], int(n.value), int(rounds.value)

    def path_count(self, rid: int) -> int:
        """Number of path vertices of a result computed with EG_FLAG_PATHS."""
        nv = ctypes.c_uint64()
        _check(self._lib.eg_get_paths(self._h, ctypes.c_uint64(rid), None, None, ctypes.byref(nv)), "eg_get_paths")
        return int(nv.value)

    def get_paths(self, rid: int):
        """Arc geometry of a result computed with EG_FLAG_PATHS: (path_ptr
        uint64[n_paths + 1], path_vtx uint32[...]); path p is
        path_vtx[path_ptr[p]:path_ptr[p + 1]] = saddle, representative, ...,
        maximum."""
        nv = ctypes.c_uint64()
        _check(self._lib.eg_get_paths(self._h, ctypes.c_uint64(rid), None, None, ctypes.byref(nv)), "eg_get_paths")
        g = EGGraphC()
        _check(self._lib.eg_get_graph(self._h, ctypes.c_uint64(rid), ctypes.byref(g)), "eg_get_graph")
        ptr = np.empty(g.n_paths + 1, np.uint64)
        vtx = np.empty(max(1, nv.value), np.uint32)[:nv.value]
        _check(self._lib.eg_get_paths(self._h, ctypes.c_uint64(rid), ctypes.c_void_p(ptr.ctypes.data),
                                      ctypes.c_void_p(vtx.ctypes.data), ctypes.byref(nv)), "eg_get_paths")
        return ptr, vtx

    def get_graph_device(self, rid: int) -> EGGraphC:
        g = EGGraphC()
        _check(self._lib.eg_get_graph_device(self._h, ctypes.c_uint64(rid), ctypes.byref(g)),
               "eg_get_graph_device")
        return g

    def get_graphs_device(self, rids: Sequence[int]) -> list:
        """get_graph_device for many results in one library call."""
        n = len(rids)
        ids = (ctypes.c_uint64 * max(1, n))(*rids)
        gs = (EGGraphC * max(1, n))()
        _check(self._lib.eg_get_graphs_device(self._h, ids, n, gs, None), "eg_get_graphs_device")
        return [gs[i] for i in range(n)]

    def release(self, rid: int):
        _check(self._lib.eg_release(self._h, ctypes.c_uint64(rid)), "eg_release")

    def mem_info(self):
        fr, to, he = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.eg_mem_info(self._h, ctypes.byref(fr), ctypes.byref(to), ctypes.byref(he)),
               "eg_mem_info")
        return fr.value, to.value, he.value

    def set_timing(self, enable: bool = True):
        _check(self._lib.eg_set_timing(self._h, int(bool(enable))), "eg_set_timing")

    def step_times(self, rid: int):
        """(classify, resolve, emit, total) device milliseconds of a computation."""
        ms = (ctypes.c_float * 4)()
        _check(self._lib.eg_step_times(self._h, ctypes.c_uint64(rid), ms), "eg_step_times")
        return tuple(float(x) for x in ms)

    def launch_count(self) -> int:
        return int(self._lib.eg_launch_count(self._h))

    def debug_fail_alloc(self, k: int):
        _check(self._lib.eg_debug_fail_alloc(self._h, int(k)), "eg_debug_fail_alloc")

    def debug_wait_timeout(self, stream=None) -> int:
        """Status of a device wait that is made to run out (EG_ERR_TIMEOUT)."""
        return int(self._lib.eg_debug_wait_timeout(self._h, ctypes.c_void_p(_stream_ptr(stream))))

    # ------------------------------------------------------------- one shot
    def graph_of(self, field, labels: bool = True, stream=None, dtype=None) -> Graph:
        """compute + get_graph + release (dtype as for compute)."""
        rid = self.compute(field, stream, dtype=dtype)
        try:
            return self.get_graph(rid, labels)
        finally:
            self.release(rid)


def labels_static(field, labels, minimum: bool = False, stream=None):
    """Allocation-free labels (eg_labels_static): field and labels are CUDA
    tensors (float32 / int32-sized, same shape); returns the status code."""
    import torch
    # every check runs before the library is touched: a labels buffer smaller
    # than the field would be written past its end by the kernels
    if field.dtype != torch.float32:
        raise ValueError("field must be a float32 tensor")
    if labels.dtype.itemsize != 4 or labels.dtype.is_floating_point:
        raise ValueError("labels must be a 4-byte integer tensor")
    if labels.numel() != field.numel():
        raise ValueError(f"labels hold {labels.numel()} elements, the field {field.numel()}")
    if not field.is_contiguous() or not labels.is_contiguous():
        raise ValueError("field and labels must be contiguous")
    if not field.is_cuda or not labels.is_cuda:
        raise ValueError("field and labels must be CUDA tensors")
    cur = torch.cuda.current_device()
    if field.device.index != cur or labels.device.index != cur:
        raise ValueError(f"field and labels must be on the current device (cuda:{cur})")
    lib = load()
    ext = _extents_of(field.shape)
    e = (ctypes.c_int64 * max(1, len(ext)))(*ext)
    return int(lib.eg_labels_static(ctypes.c_void_p(field.data_ptr()), len(ext), e,
                                    EG_FLAG_MINIMUM_GRAPH if minimum else 0,
                                    ctypes.c_void_p(labels.data_ptr()),
                                    ctypes.c_void_p(_stream_ptr(stream))))


def workspace_bytes(extents) -> int:
    e = (ctypes.c_int64 * max(1, len(extents)))(*extents)
    return int(load().eg_workspace_bytes(len(extents), e))


def device_array(a: np.ndarray, device: int = 0):
    """Copy a numpy array of any element type in DTYPES to a CUDA tensor with
    the same bytes and shape (unsigned types travel as the signed torch type
    of the same size); pass its numpy dtype to Handle.compute / batch_submit."""
    import torch
    a = np.ascontiguousarray(a)
    view = {1: np.int8, 2: np.int16, 4: np.int32, 8: np.int64}
    if a.dtype.kind == "u" and a.dtype != np.uint8:
        a = a.view(view[a.dtype.itemsize])
    return torch.from_numpy(a).to(f"cuda:{device}")
