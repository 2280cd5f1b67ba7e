"""Sequential CPU oracle for the extremum graph (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or calls it, and the two share no code: the
oracle is plain C in ``eg_oracle.c`` built with the host compiler.

Every function of the C file follows the paper's definitions one vertex at a
time (Sec. 3.2 Algorithm 1, Sec. 3.3 and Table 1, Sec. 3.4 Algorithm 2, Sec. 2
for the arcs); see its header for the list.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eg_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "eg_cancel.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libeg_oracle.so")
_lock = threading.Lock()
_lib = None

EO_OK, EO_ERR_ARG, EO_ERR_NAN, EO_ERR_OOM = 0, 1, 2, 3

# element types of the C oracle (Sec. 5: 8- to 64-bit integers, 32/64-bit floats)
DTYPES = {np.dtype(np.float32): 0, np.dtype(np.float64): 1, np.dtype(np.int8): 2,
          np.dtype(np.uint8): 3, np.dtype(np.int16): 4, np.dtype(np.uint16): 5,
          np.dtype(np.int32): 6, np.dtype(np.uint32): 7, np.dtype(np.int64): 8,
          np.dtype(np.uint64): 9}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math: IEEE comparisons only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(p) for p in _SRCS)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.eo_compute.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_void_p)]
        lib.eo_compute.restype = ctypes.c_int
        lib.eo_compute_typed.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]
        lib.eo_compute_typed.restype = ctypes.c_int
        lib.eo_counts.argtypes = [P, P]
        lib.eo_counts.restype = None
        lib.eo_copy.argtypes = [P] * 12
        lib.eo_copy.restype = None
        lib.eo_free.argtypes = [P]
        lib.eo_free.restype = None
        lib.eo_path_vertices.argtypes = [P]
        lib.eo_path_vertices.restype = ctypes.c_uint64
        lib.eo_paths.argtypes = [P, P, P]
        lib.eo_paths.restype = None
        lib.eo_neighbour_offsets.argtypes = [ctypes.c_int, P]
        lib.eo_neighbour_offsets.restype = ctypes.c_int
        lib.eo_grid_adjacent.argtypes = [ctypes.c_int, P, P]
        lib.eo_grid_adjacent.restype = ctypes.c_int
        lib.ec_cancel.argtypes = [ctypes.c_int64, P, P, ctypes.c_int64, P, P, P, P, ctypes.c_int,
                                  ctypes.c_float, P, P, P]
        lib.ec_cancel.restype = ctypes.c_int
        _lib = lib
        return lib


@dataclass
class OracleGraph:
    """Extremum graph plus the per-vertex arrays it is built from."""
    asc: np.ndarray      # uint32[N]   gradient pointer (itself at a maximum)
    label: np.ndarray    # uint32[N]   maximum reached
    beta0p: np.ndarray   # uint8[N]    upper-link components
    maxima: np.ndarray   # uint32[M]   ascending
    max_val: np.ndarray  # [M] values at the maxima, in the field's element type
    saddles: np.ndarray  # uint32[S]   ascending
    sad_b0: np.ndarray   # uint8[S]
    sad_val: np.ndarray  # [S] values at the saddles, in the field's element type
    row_ptr: np.ndarray  # uint64[S+1]
    col: np.ndarray      # uint32[A]
    n_paths: int         # sum of beta0+ over saddles
    reps: np.ndarray = None  # uint32[P] UpperLinkRep per saddle (ascending ids, saddles in order)
    path_ptr: np.ndarray = None  # uint64[P+1] offsets of the arc geometry (paths=True)
    path_vtx: np.ndarray = None  # uint32[...] s, rep, gradient(rep), ..., maximum per path

    def path(self, p):
        """Vertices of path number p (saddle, representative, ..., maximum)."""
        return self.path_vtx[self.path_ptr[p]:self.path_ptr[p + 1]]

    def saddle_reps(self, i):
        """Upper-link representatives of saddle number i."""
        off = int(self.sad_b0[:i].sum())
        return self.reps[off:off + int(self.sad_b0[i])]

    def arcs(self):
        """Set of (saddle, maximum) pairs."""
        out = set()
        for i, s in enumerate(self.saddles.tolist()):
            for m in self.col[self.row_ptr[i]:self.row_ptr[i + 1]].tolist():
                out.add((s, m))
        return out


def compute(field: np.ndarray, extents=None, naive: bool = False,
            minimum: bool = False, paths: bool = False, dtype=None) -> OracleGraph:
    """Extremum graph of ``field``.

    ``extents`` lists the grid size per axis with axis 0 fastest; by default it
    is the numpy shape reversed, so a C-ordered array ``a[z, y, x]`` has
    ``x`` as axis 0.  ``minimum`` selects the minimum graph (reversed order).
    ``paths`` adds the arc geometry (Algorithm 2's gradient paths).
    ``dtype``: the element type the values are compared in (one of DTYPES);
    None means float32 (the field is converted to it).
    """
    lib = _load()
    dt = np.dtype(np.float32 if dtype is None else dtype)
    if dt not in DTYPES:
        raise OracleError(f"unsupported element type {dt}")
    f = np.ascontiguousarray(field, dtype=dt).reshape(-1)
    if extents is None:
        extents = tuple(reversed(np.asarray(field).shape))
    ext = np.ascontiguousarray(extents, dtype=np.int64)
    d = int(ext.size)
    h = ctypes.c_void_p()
    st = lib.eo_compute_typed(f.ctypes.data, DTYPES[dt], d, ext.ctypes.data, int(naive),
                              int(minimum), ctypes.byref(h))
    if st != EO_OK:
        raise OracleError({EO_ERR_ARG: "bad argument", EO_ERR_NAN: "NaN in field",
                           EO_ERR_OOM: "out of memory"}.get(st, str(st)))
    try:
        c = np.zeros(5, dtype=np.int64)
        lib.eo_counts(h, c.ctypes.data)
        n, nm, ns, npaths, na = (int(x) for x in c)
        g = OracleGraph(
            asc=np.empty(n, np.uint32), label=np.empty(n, np.uint32),
            beta0p=np.empty(n, np.uint8), maxima=np.empty(nm, np.uint32),
            max_val=np.empty(nm, dt), saddles=np.empty(ns, np.uint32),
            sad_b0=np.empty(ns, np.uint8), sad_val=np.empty(ns, dt),
            row_ptr=np.empty(ns + 1, np.uint64), col=np.empty(na, np.uint32),
            n_paths=npaths, reps=np.empty(npaths, np.uint32))
        lib.eo_copy(h, g.asc.ctypes.data, g.label.ctypes.data, g.beta0p.ctypes.data,
                    g.maxima.ctypes.data, g.max_val.ctypes.data, g.saddles.ctypes.data,
                    g.sad_b0.ctypes.data, g.sad_val.ctypes.data, g.row_ptr.ctypes.data,
                    g.col.ctypes.data, g.reps.ctypes.data)
        if paths:
            nv = int(lib.eo_path_vertices(h))
            g.path_ptr = np.empty(npaths + 1, np.uint64)
            g.path_vtx = np.empty(nv, np.uint32)
            lib.eo_paths(h, g.path_ptr.ctypes.data, g.path_vtx.ctypes.data)
        return g
    finally:
        lib.eo_free(h)


def bundle(g: OracleGraph, minimum: bool = False) -> np.ndarray:
    """Arc bundling (Sec. 3.5): when several saddles connect the same two
    maxima, only the highest of them (value, then index; lowest for the
    minimum graph) stands for that pair.  A saddle is kept when it stands for
    at least one pair of its arc ends; a saddle whose arcs all end at one
    maximum connects no pair and is kept.  Returns uint8[S], 1 = kept.
    Plain loops: for small fields only."""
    vals = g.sad_val.tolist()  # Python int / float: exact for every element type

    def higher(i):
        v, s = vals[i], int(g.saddles[i])
        return (-v, -s) if minimum else (v, s)

    best = {}
    ends = [g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist() for i in range(g.saddles.size)]
    for i, e in enumerate(ends):
        for a in range(len(e)):
            for b in range(a + 1, len(e)):
                pair = (e[a], e[b])
                if pair not in best or higher(i) > higher(best[pair]):
                    best[pair] = i
    keep = np.zeros(g.saddles.size, np.uint8)
    for i, e in enumerate(ends):
        pairs = [(e[a], e[b]) for a in range(len(e)) for b in range(a + 1, len(e))]
        keep[i] = 1 if not pairs or any(best[p] == i for p in pairs) else 0
    return keep


@dataclass
class Cancellation:
    """Persistence-directed cancellation of an extremum graph (Sec. 3.5)."""
    alive: np.ndarray     # uint8[S]  1 = the saddle is still in the graph
    survivor: np.ndarray  # uint32[M] vertex id of the maximum each maximum was merged into
    n_cancelled: int

    def simplified_arcs(self, g) -> set:
        """(saddle, maximum) pairs of the simplified graph: the kept saddles
        with the survivors of their arc ends."""
        surv = dict(zip(g.maxima.tolist(), self.survivor.tolist()))
        out = set()
        for i, s in enumerate(g.saddles.tolist()):
            if self.alive[i]:
                for m in g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist():
                    out.add((s, surv[m]))
        return out


def cancel(maxima, max_val, saddles, sad_val, row_ptr, col, tau: float,
           minimum: bool = False) -> Cancellation:
    """Persistence-directed cancellation (Sec. 3.5) of an extremum graph
    given as arrays (maxima and saddles ascending, float32 values, the CSR of
    arc ends as maximum vertex ids) with persistence threshold tau (float32).
    The steps and the readings of the open cases are listed in eg_cancel.c."""
    lib = _load()
    mx = np.ascontiguousarray(maxima, np.uint32)
    mv = np.ascontiguousarray(max_val, np.float32)
    sd = np.ascontiguousarray(saddles, np.uint32)
    sv = np.ascontiguousarray(sad_val, np.float32)
    rp = np.ascontiguousarray(row_ptr, np.uint64)
    cl = np.ascontiguousarray(col, np.uint32)
    alive = np.empty(sd.size, np.uint8)
    surv = np.empty(mx.size, np.uint32)
    n = ctypes.c_int64(0)
    st = lib.ec_cancel(mx.size, mx.ctypes.data, mv.ctypes.data, sd.size, sd.ctypes.data, sv.ctypes.data,
                       rp.ctypes.data, cl.ctypes.data, int(minimum), ctypes.c_float(tau), alive.ctypes.data,
                       surv.ctypes.data, ctypes.byref(n))
    if st != EO_OK:
        raise OracleError({EO_ERR_ARG: "bad argument", EO_ERR_OOM: "out of memory"}.get(st, str(st)))
    return Cancellation(alive, surv, int(n.value))


def cancel_graph(g: OracleGraph, tau: float, minimum: bool = False) -> Cancellation:
    """cancel() on an oracle result (float32 fields)."""
    return cancel(g.maxima, g.max_val, g.saddles, g.sad_val, g.row_ptr, g.col, tau, minimum)


def neighbour_offsets(d: int) -> np.ndarray:
    """Offsets kept by Algorithm 1 against the origin, shape (2(2^d-1), d)."""
    lib = _load()
    out = np.zeros((2 * (2 ** d - 1), d), dtype=np.int64)
    n = lib.eo_neighbour_offsets(d, out.ctypes.data)
    if n < 0:
        raise OracleError("bad dimension")
    return out[:n]


def grid_adjacent(p, q) -> bool:
    """Algorithm 1 on two coordinate vectors."""
    lib = _load()
    a = np.ascontiguousarray(p, dtype=np.int64)
    b = np.ascontiguousarray(q, dtype=np.int64)
    return bool(lib.eo_grid_adjacent(int(a.size), a.ctypes.data, b.ctypes.data))
