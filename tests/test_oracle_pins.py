"""Pins of the CPU oracle against facts that do not come from the oracle itself.

  * golden closed forms derived by hand (tests/golden/*.txt, each cites the
    definitions it follows);
  * brute force on tiny grids (tests/brute.py: all-pairs Algorithm 1, BFS
    components, sort-based order, naive walks);
  * the neighbour count 2(2^d - 1) stated in Sec. 3.2;
  * the Euler-characteristic identity for a PL function on a disk (2D), which
    ties the beta0+ counts of all vertices to a global invariant;
  * symmetries of the Freudenthal neighbourhood (axis permutation, reflection)
    and invariance under f -> 2f;
  * densities of maxima in iid noise, 1 / (2^(d+1) - 1) in the interior.
"""
import glob
import zlib
import os

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F
from tests.brute import alg1_adjacent, brute_graph, sos_rank

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- golden ----

def _read_golden(path):
    meta, sec = {}, {}
    for line in open(path):
        line = line.rstrip("\n")
        if not line.strip():
            continue
        if line.startswith("#"):
            if ":" in line:
                k, v = line[1:].split(":", 1)
                meta[k.strip()] = v.strip()
            continue
        k, v = line.split(":", 1)
        sec[k.strip()] = v.strip()
    return meta, sec


def _golden_field(meta, sec):
    ext = tuple(int(x) for x in meta["extents"].split())
    if "field" in sec:
        vals = np.array([float(x) for x in sec["field"].split()], np.float32)
    else:
        g = np.array([float(x) for x in sec["gx"].split()], np.float64)
        h = np.array([float(x) for x in sec["hy"].split()], np.float64)
        vals = (h[:, None] + g[None, :]).astype(np.float32).reshape(-1)
    return ext, vals


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))),
                         ids=lambda p: os.path.basename(p))
def test_golden(path):
    meta, sec = _read_golden(path)
    ext, vals = _golden_field(meta, sec)
    g = oracle.compute(vals, extents=ext, minimum=bool(int(meta.get("minimum", "0"))), paths=True)
    ints = lambda s: [int(x) for x in s.split()] if s else []
    assert g.maxima.tolist() == ints(sec["maxima"])
    assert g.saddles.tolist() == ints(sec.get("saddles", ""))
    assert g.sad_b0.tolist() == ints(sec.get("beta0", ""))
    arcs = {tuple(int(y) for y in a.split(",")) for a in sec.get("arcs", "").split()}
    assert g.arcs() == arcs
    if "labels" in sec:
        assert g.label.tolist() == ints(sec["labels"])
    if "labels_rule" in sec:  # 2d_separable: x<=3 -> 29, x>=4 -> 33
        x = np.arange(vals.size) % ext[0]
        assert np.array_equal(g.label, np.where(x <= 3, 29, 33).astype(np.uint32))
    assert np.array_equal(g.max_val, vals[g.maxima])
    assert np.array_equal(g.sad_val, vals[g.saddles])
    if "paths" in sec:
        want = [[int(y) for y in a.split(",")] for a in sec["paths"].split()]
        assert [g.path(p).tolist() for p in range(g.n_paths)] == want


# ----------------------------------------------------------- Algorithm 1 ----

@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_neighbour_count(d):
    off = oracle.neighbour_offsets(d)
    assert len(off) == 2 * (2 ** d - 1)                   # Sec. 3.2
    assert len({tuple(o) for o in off}) == len(off)
    assert {tuple(-o) for o in off} == {tuple(o) for o in off}  # symmetric


def test_neighbours_2d_3d_match_figure():
    # Fig. 2 (c,f): 6 neighbours in 2D, 14 in 3D; the 2D set is the hexagon
    got2 = {tuple(o) for o in oracle.neighbour_offsets(2)}
    assert got2 == {(1, 0), (0, 1), (1, 1), (-1, 0), (0, -1), (-1, -1)}
    got3 = {tuple(o) for o in oracle.neighbour_offsets(3)}
    assert len(got3) == 14 and (1, 1, 1) in got3 and (1, -1, 0) not in got3


def test_alg1_cases():
    assert not oracle.grid_adjacent((0, 0), (0, 0))
    assert oracle.grid_adjacent((1, 1), (0, 0))
    assert oracle.grid_adjacent((0, 0), (1, 1))
    assert not oracle.grid_adjacent((1, 0), (0, 1))
    assert not oracle.grid_adjacent((2, 0), (0, 0))
    assert oracle.grid_adjacent((3, 4, 5, 6), (3, 5, 6, 6))
    for p, q in [((0, 0, 0), (1, 0, 1)), ((2, 2), (1, 2)), ((0, 1), (1, 0))]:
        assert oracle.grid_adjacent(p, q) == alg1_adjacent(p, q)


# ------------------------------------------------------------ brute force ---

SHAPES = [(8, 8), (4, 4, 4), (3, 3, 3, 3), (10,), (5, 3), (1, 7), (2, 1, 3), (3, 2, 2, 2),
          (2, 2), (1,), (2,), (1, 1, 1), (5, 4, 3), (6, 1), (2, 2, 2, 2, 2), (3, 3, 2, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind", ["normal", "ties"])
@pytest.mark.parametrize("minimum", [False, True])
def test_brute_force(shape, kind, minimum):
    n = int(np.prod(shape))
    seed = zlib.crc32(repr((shape, kind)).encode()) % 1000
    f = (F.white_noise(shape, seed) if kind == "normal" else F.integer_ties(shape, seed, 3)).values
    g = oracle.compute(f, extents=shape, minimum=minimum, paths=True)
    b = brute_graph(f, shape, minimum=minimum)
    assert g.asc.tolist() == b["asc"].tolist()
    assert g.label.tolist() == b["label"].tolist()
    assert g.beta0p.tolist() == b["beta"].tolist()
    assert g.maxima.tolist() == b["maxima"]
    assert g.saddles.tolist() == b["saddles"]
    assert g.arcs() == b["arcs"]
    assert g.n_paths == sum(len(b["reps"][s]) for s in b["saddles"])
    for i, s_ in enumerate(b["saddles"]):
        assert g.saddle_reps(i).tolist() == sorted(int(x) for x in b["reps"][s_])
    assert [g.path(p).tolist() for p in range(g.n_paths)] == b["paths"]
    assert n == g.label.size


def test_naive_equals_memo():
    for f in [F.config_2d_256(side=96).values, F.white_noise((17, 13, 11), 7).values,
              F.integer_ties((9, 8, 7, 3), 3, 2).values]:
        a = oracle.compute(f)
        b = oracle.compute(f, naive=True)
        assert np.array_equal(a.label, b.label)
        assert np.array_equal(a.col, b.col)


# ------------------------------------------------------------- invariants ---

def _higher(f, v, w):
    return (f[w] > f[v]) | ((f[w] == f[v]) & (w > v))


@pytest.mark.parametrize("case", ["2d", "3d", "4d", "ties3d"])
def test_invariants(case):
    f = {"2d": lambda: F.config_2d_256(side=80),
         "3d": lambda: F.config_3d_256(side=24),
         "4d": lambda: F.white_noise((7, 6, 5, 6), 11),
         "ties3d": lambda: F.integer_ties((12, 10, 9), 5, 3)}[case]()
    vals = f.values.reshape(-1)
    g = oracle.compute(f.values)
    n = vals.size
    v = np.arange(n, dtype=np.uint32)
    is_max = np.zeros(n, bool)
    is_max[g.maxima] = True
    # maxima are exactly the fixed points of the gradient (empty upper link)
    assert np.array_equal(is_max, g.asc == v)
    assert np.array_equal(is_max, g.beta0p == 0)
    # the gradient strictly climbs
    nm = ~is_max
    assert np.all(_higher(vals, v[nm], g.asc[nm]))
    # every label is a maximum, maxima label themselves
    assert np.all(is_max[g.label])
    assert np.array_equal(g.label[g.maxima], g.maxima)
    assert len(g.maxima) >= 1
    # CSR rows sorted, unique, maxima only; label(s) is among the arcs of s
    for i, s in enumerate(g.saddles):
        row = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0)
        assert np.all(is_max[row])
        assert g.label[s] in row
        assert 1 <= len(row) <= g.sad_b0[i]
    assert g.n_paths == int(g.sad_b0.sum())
    assert np.array_equal(g.sad_b0, g.beta0p[g.saddles])


def test_scale_invariance():
    f = F.config_3d_256(side=20).values
    a = oracle.compute(f)
    b = oracle.compute(f * np.float32(2.0))
    assert np.array_equal(a.label, b.label) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.saddles, b.saddles)


def _remap_graph(g, mapping):
    """Graph with every vertex id v replaced by mapping[v] (sets, no order)."""
    M = set(mapping[g.maxima].tolist())
    S = set(mapping[g.saddles].tolist())
    A = {(int(mapping[s]), int(mapping[m])) for s, m in g.arcs()}
    return M, S, A


@pytest.mark.parametrize("shape", [(9, 7), (6, 5, 4), (4, 3, 5, 3)])
def test_axis_permutation_and_reflection(shape):
    f = F.white_noise(shape, 21).values
    assert len(np.unique(f)) == f.size  # tie-free: SoS plays no part
    g = oracle.compute(f)
    ids = np.arange(f.size).reshape(f.shape)
    d = len(shape)
    # reflection of every axis: v -> N-1-v
    fr = f[(slice(None, None, -1),) * d].copy()
    gr = oracle.compute(fr)
    mapping = ids[(slice(None, None, -1),) * d].reshape(-1)  # new id -> old id
    inv = np.empty_like(mapping)
    inv[mapping] = np.arange(f.size)
    assert _remap_graph(g, inv) == (set(gr.maxima.tolist()), set(gr.saddles.tolist()), gr.arcs())
    # cyclic permutation of axes
    perm = tuple(range(1, d)) + (0,)
    fp = np.ascontiguousarray(np.transpose(f, perm))
    gp = oracle.compute(fp)
    mapping = np.transpose(ids, perm).reshape(-1)
    inv = np.empty_like(mapping)
    inv[mapping] = np.arange(f.size)
    assert _remap_graph(g, inv) == (set(gp.maxima.tolist()), set(gp.saddles.tolist()), gp.arcs())
    assert np.array_equal(inv[g.label], gp.label[inv])


@pytest.mark.parametrize("shape", [(9, 7), (6, 5, 4), (4, 3, 3, 3), (3, 3, 3, 2, 3)])
@pytest.mark.parametrize("kind", ["white", "ties", "zeros_infs"])
def test_minimum_graph_is_maximum_graph_of_negated_reflection(shape, kind):
    """The minimum graph reverses the order (value, then index).  Negating
    the field reverses the values, and reflecting every axis (v -> N-1-v)
    reverses the index order while mapping the neighbourhood onto itself, so
    the minimum graph of f is the maximum graph of -f on the reflected grid
    with every id v read as N-1-v: with ties, signed zeros and infinities
    too."""
    rng = np.random.default_rng(sum(shape) * 7 + len(kind))
    if kind == "white":
        f = F.white_noise(shape, 31).values
    elif kind == "ties":
        f = F.integer_ties(shape, 32, 3).values
    else:
        pool = np.array([-np.inf, -1.0, -0.0, 0.0, 1.0, np.inf], np.float32)
        f = pool[rng.integers(0, len(pool), size=shape)]
    d = len(shape)
    N = f.size
    h = np.ascontiguousarray(-f[(slice(None, None, -1),) * d])
    gmin = oracle.compute(f, minimum=True)
    gh = oracle.compute(h)
    back = lambda a: (N - 1 - np.asarray(a, np.int64)).astype(np.uint32)
    assert np.array_equal(np.sort(back(gh.maxima)), gmin.maxima)
    assert np.array_equal(np.sort(back(gh.saddles)), gmin.saddles)
    assert np.array_equal(back(gh.label)[::-1], gmin.label)
    assert np.array_equal(back(gh.asc)[::-1], gmin.asc)
    assert np.array_equal(gh.beta0p[::-1], gmin.beta0p)
    assert {(int(N - 1 - s), int(N - 1 - m)) for s, m in gh.arcs()} == gmin.arcs()
    b0h = dict(zip(back(gh.saddles).tolist(), gh.sad_b0.tolist()))
    assert [b0h[s] for s in gmin.saddles.tolist()] == gmin.sad_b0.tolist()


def _interior_minima_2d(f):
    ny, nx = f.shape
    c = f[1:-1, 1:-1]
    cnt = np.ones_like(c, dtype=bool)
    for dy, dx in [(0, 1), (1, 0), (1, 1), (0, -1), (-1, 0), (-1, -1)]:
        nb = f[1 + dy:ny - 1 + dy, 1 + dx:nx - 1 + dx]
        cnt &= nb > c
    return int(cnt.sum())


@pytest.mark.parametrize("which", ["cfg2d", "white", "ties"])
def test_euler_characteristic_2d(which):
    """Sum over vertices of 1 - chi(upper link) = chi(disk) = 1.

    In 2D a proper part of a link is a union of beta0+ paths (chi = beta0+),
    and only an interior minimum has the whole link cycle above it (chi = 0)."""
    f = {"cfg2d": lambda: F.config_2d_256(side=120).values,
         "white": lambda: F.white_noise((37, 29), 3).values,
         "ties": lambda: F.integer_ties((31, 23), 4, 5).values}[which]()
    if which == "ties":
        # make the interior-minimum count below use the same perturbed order
        rank = np.argsort(np.lexsort((np.arange(f.size), f.reshape(-1))))
        f = rank.reshape(f.shape).astype(np.float32)
    g = oracle.compute(f)
    total = int(np.sum(1 - g.beta0p.astype(np.int64))) + _interior_minima_2d(f)
    assert total == 1


@pytest.mark.parametrize("d,shape", [(2, (300, 300)), (3, (48, 48, 48)), (4, (16, 16, 16, 16))])
def test_maxima_density_iid(d, shape):
    f = F.white_noise(shape, 100 + d).values
    g = oracle.compute(f)
    x = np.unravel_index(g.maxima.astype(np.int64), f.shape)
    interior = np.ones(len(g.maxima), bool)
    for k in range(d):
        interior &= (x[k] > 0) & (x[k] < f.shape[k] - 1)
    n_int = int(np.prod([s - 2 for s in shape]))
    p = 1.0 / (2 ** (d + 1) - 1)
    got = interior.sum()
    sigma = np.sqrt(n_int * p * (1 - p))
    assert abs(got - n_int * p) < 5 * sigma


def test_single_gaussian_one_maximum():
    for ext in [(33, 29), (17, 19, 15)]:
        f = F.gaussian_sum(ext, 9, 1, (5.0, 5.0), (1.0, 1.0), True, None).values
        g = oracle.compute(f)
        assert len(g.maxima) == 1
        assert np.all(g.label == g.maxima[0])


@pytest.mark.parametrize("shape", [(5, 4, 3), (3, 3, 3, 2)])
def test_constant_field_higher_d(shape):
    n = int(np.prod(shape))
    g = oracle.compute(np.zeros(shape[::-1], np.float32))
    assert g.maxima.tolist() == [n - 1] and len(g.saddles) == 0
    assert np.all(g.label == n - 1)


def test_signed_zero_and_inf():
    # -0 == +0 ties by index; infinities are ordinary ordered values
    f = np.array([0.0, -0.0, np.inf, -np.inf, 1.0], np.float32)
    g = oracle.compute(f)
    b = brute_graph(f, (5,))
    assert g.maxima.tolist() == b["maxima"] == [2, 4]
    assert g.label.tolist() == b["label"].tolist()


def test_errors():
    with pytest.raises(oracle.OracleError):
        oracle.compute(np.array([0.0, np.nan], np.float32))
    with pytest.raises(oracle.OracleError):
        oracle.compute(np.zeros(4, np.float32), extents=(0, 4))
    with pytest.raises(oracle.OracleError):
        oracle.compute(np.zeros(4, np.float32), extents=(1,) * 7)


# ------------------------------------------------------------ arc bundling ---

@pytest.mark.parametrize("shape", [(8, 8), (12, 10), (6, 5, 4), (4, 4, 3), (3, 3, 3, 3), (5, 4, 3, 3)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("kind", ["normal", "ties"])
@pytest.mark.parametrize("minimum", [False, True])
def test_bundling_brute_force(shape, kind, minimum):
    """Sec. 3.5 restated on the brute-force graph: for every pair of maxima
    joined by some saddle, the rank-highest saddle joining it is kept (so the
    pair stays connected), and every kept saddle with two or more arc ends is
    that highest saddle for at least one of its pairs."""
    seed = zlib.crc32(repr((shape, kind, "bundle")).encode()) % 1000
    f = (F.white_noise(shape, seed) if kind == "normal" else F.integer_ties(shape, seed, 3)).values
    g = oracle.compute(f, extents=shape, minimum=minimum)
    keep = oracle.bundle(g, minimum=minimum)
    b = brute_graph(f, shape, minimum=minimum)
    rank = sos_rank(np.asarray(f, np.float32).reshape(-1).astype(np.float64), minimum)
    ends = {s: sorted({m for (t, m) in b["arcs"] if t == s}) for s in b["saddles"]}
    kept = {int(s) for s, k in zip(g.saddles.tolist(), keep.tolist()) if k}
    pairs = {}
    for s, e in ends.items():
        for x in range(len(e)):
            for y in range(x + 1, len(e)):
                pairs.setdefault((e[x], e[y]), []).append(s)
    for pr, ss in pairs.items():
        top = max(ss, key=lambda s: rank[s])
        assert top in kept, (pr, ss)
    for s in kept:
        e = ends[s]
        if len(e) >= 2:
            assert any(max(pairs[(e[x], e[y])], key=lambda t: rank[t]) == s
                       for x in range(len(e)) for y in range(x + 1, len(e)))
    for s, e in ends.items():
        if len(e) < 2:
            assert s in kept
    assert len(kept) <= len(ends)


def test_bundling_keeps_single_pair_saddle_structure():
    # 1D: every pair of adjacent maxima has exactly one saddle between them
    f = np.array([0, 5, 1, 4, 2, 8, 3], np.float32)
    g = oracle.compute(f)
    assert oracle.bundle(g).tolist() == [1, 1]


# ---------------------------------------------------------- element types ---
# Sec. 5: the library takes 8- to 64-bit integers and 32/64-bit floats.  The
# order is still (value, then index); values are compared in their own type.

TYPED_SHAPES = [(8, 8), (4, 4, 4), (3, 3, 3, 3), (9,), (5, 3, 2)]


@pytest.mark.parametrize("dtype", F.ELEMENT_TYPES)
@pytest.mark.parametrize("shape", TYPED_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("minimum", [False, True])
def test_typed_brute_force(dtype, shape, minimum):
    """Boundary values of each type (extremes, both sides of the sign bit,
    neighbours float32 cannot separate) against the brute force, whose
    sort-based order compares the values in their own type."""
    seed = zlib.crc32(repr((shape, dtype)).encode()) % 1000
    f = F.typed_ties(shape, seed, dtype).values
    g = oracle.compute(f, extents=shape, minimum=minimum, dtype=f.dtype)
    b = brute_graph(f, shape, minimum=minimum, dtype=f.dtype)
    assert g.asc.tolist() == b["asc"].tolist()
    assert g.label.tolist() == b["label"].tolist()
    assert g.beta0p.tolist() == b["beta"].tolist()
    assert g.maxima.tolist() == b["maxima"]
    assert g.saddles.tolist() == b["saddles"]
    assert g.arcs() == b["arcs"]
    for i, s_ in enumerate(b["saddles"]):
        assert g.saddle_reps(i).tolist() == sorted(int(x) for x in b["reps"][s_])
    flat = f.reshape(-1)
    assert g.max_val.dtype == f.dtype and g.sad_val.dtype == f.dtype
    assert g.max_val.tobytes() == flat[g.maxima].tobytes()
    assert g.sad_val.tobytes() == flat[g.saddles].tobytes()


@pytest.mark.parametrize("dtype", ["uint64", "int64", "uint32", "int32", "float64"])
def test_typed_differs_from_float32(dtype):
    """Values that float32 merges (2^24 and 2^24+1, 2^53 and 2^53+1, 1 and
    1+2^-30) must stay ordered: a 1D field whose float32 image is constant
    still has its maximum at the largest value, not at the last index."""
    hi = {"uint64": 2 ** 53 + 1, "int64": 2 ** 53 + 1, "uint32": 2 ** 24 + 1,
          "int32": 2 ** 24 + 1, "float64": 1.0 + 2.0 ** -30}[dtype]
    lo = {"float64": 1.0}.get(dtype, hi - 1)
    f = np.array([lo, hi, lo], dtype=dtype)
    assert np.unique(f.astype(np.float32)).size == 1
    g = oracle.compute(f, dtype=f.dtype)
    assert g.maxima.tolist() == [1]
    assert g.label.tolist() == [1] * 3
    g32 = oracle.compute(f.astype(np.float32))
    assert g32.maxima.tolist() == [2]


@pytest.mark.parametrize("dtype", ["int8", "uint8", "int16", "uint16"])
def test_typed_narrow_equals_float32(dtype):
    """Integers of at most 16 bits are exact in float32 with their order and
    ties kept, so the graph of the typed field equals that of its float32
    image (the float32 path is pinned independently above)."""
    for shape, seed in [((12, 10), 1), ((6, 5, 4), 2), ((4, 3, 3, 3), 3)]:
        f = F.quantise(F.white_noise(shape, seed), dtype, levels=6).values
        g = oracle.compute(f, extents=shape, dtype=f.dtype)
        g32 = oracle.compute(f.astype(np.float32), extents=shape)
        assert np.array_equal(g.label, g32.label)
        assert np.array_equal(g.maxima, g32.maxima) and np.array_equal(g.saddles, g32.saddles)
        assert np.array_equal(g.row_ptr, g32.row_ptr) and np.array_equal(g.col, g32.col)
        assert np.array_equal(g.max_val.astype(np.float32), g32.max_val)


def test_typed_nan_and_bad_type():
    with pytest.raises(oracle.OracleError):
        oracle.compute(np.array([0.0, np.nan], np.float64), dtype=np.float64)
    with pytest.raises(oracle.OracleError):
        oracle.compute(np.zeros(4, np.float16), dtype=np.float16)
    g = oracle.compute(np.array([-np.inf, 0.0, -0.0, np.inf, 1.0]), dtype=np.float64)
    assert g.maxima.tolist() == [3]


def test_typed_bundling_uses_exact_values():
    """Arc bundling ranks saddles by their values in the field's own type."""
    for dtype in ["uint64", "int64", "float64", "int8"]:
        for seed in range(3):
            shape = (7, 6, 5)
            f = F.typed_ties(shape, seed, dtype).values
            g = oracle.compute(f, extents=shape, dtype=f.dtype)
            keep = oracle.bundle(g)
            b = brute_graph(f, shape, dtype=f.dtype)
            rank = sos_rank(f.reshape(-1))
            pairs = {}
            for s in b["saddles"]:
                e = sorted({m for (t, m) in b["arcs"] if t == s})
                for x in range(len(e)):
                    for y in range(x + 1, len(e)):
                        pairs.setdefault((e[x], e[y]), []).append(s)
            kept = {int(s) for s, k in zip(g.saddles.tolist(), keep.tolist()) if k}
            for ss in pairs.values():
                assert max(ss, key=lambda s: rank[s]) in kept


# ------------------------------------------------------------------- 5D ----

def link_independent_set(d):
    """Pairwise non-adjacent neighbour offsets of the origin: every positive
    offset whose axis pattern has a elements and every negative one with b
    elements, a + b > d (so a positive and a negative pattern always share
    an axis: not adjacent; two patterns of one size are incomparable: not
    adjacent), sizes chosen to maximise the count.  The largest such sets
    have 3, 6, 10 and 20 members in 2D..5D."""
    from itertools import combinations
    from math import comb
    a, b = max(((a, b) for a in range(1, d + 1) for b in range(1, d + 1) if a + b > d),
               key=lambda ab: comb(d, ab[0]) + comb(d, ab[1]))
    out = []
    for size, sign in [(a, 1), (b, -1)]:
        for axes in combinations(range(d), size):
            out.append(tuple(sign if i in axes else 0 for i in range(d)))
    return out


def many_component_field(d):
    """3^d grid: the centre low, the offsets of link_independent_set high,
    every other vertex lower still, so the centre's upper link is that
    independent set: one component per member."""
    ind = set(link_independent_set(d))
    f = np.full((3,) * d, -20.0, np.float32)
    for o in oracle.neighbour_offsets(d):
        idx = tuple(1 + int(x) for x in reversed(o))  # numpy axes are reversed
        f[idx] = 10.0 if tuple(int(x) for x in o) in ind else -10.0
    f[(1,) * d] = 0.0
    return f


def test_independent_sets_are_largest():
    """The constructed sets are independent under Algorithm 1, and (where
    networkx is available) no larger independent set exists."""
    for d in [2, 3, 4, 5]:
        ind = link_independent_set(d)
        assert all(not alg1_adjacent(p, q) for p in ind for q in ind)
    nx = pytest.importorskip("networkx")
    for d in [2, 3, 4, 5]:
        off = [tuple(int(x) for x in o) for o in oracle.neighbour_offsets(d)]
        comp = nx.Graph()
        comp.add_nodes_from(range(len(off)))
        comp.add_edges_from((i, j) for i in range(len(off)) for j in range(i + 1, len(off))
                            if not alg1_adjacent(off[i], off[j]))
        assert max(len(c) for c in nx.find_cliques(comp)) == len(link_independent_set(d))


@pytest.mark.parametrize("d,count", [(2, 3), (3, 6), (4, 10), (5, 20)])
def test_most_components(d, count):
    """The independence number of the link graph bounds beta0+ (3, 6, 10 and
    20 in 2D..5D); a field whose centre's upper link is a largest
    independent set reaches it, and the brute force agrees."""
    f = many_component_field(d)
    ext = (3,) * d
    centre = sum(3 ** i for i in range(d))
    g = oracle.compute(f, extents=ext)
    assert len(link_independent_set(d)) == count
    assert int(g.beta0p[centre]) == count
    b = brute_graph(f, ext)
    assert int(b["beta"][centre]) == count
    assert g.label.tolist() == b["label"].tolist()
    assert g.arcs() == b["arcs"]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_link_edges_by_axis_patterns(d):
    """The link structure the GPU classifiers build on (link components as
    closures over axis patterns): two neighbour offsets of a vertex are
    adjacent under Algorithm 1 iff they have the same sign and comparable
    axis patterns (one a subset of the other), or opposite signs and disjoint
    patterns."""
    off = [tuple(int(x) for x in o) for o in oracle.neighbour_offsets(d)]
    for a in off:
        for b in off:
            if a == b:
                continue
            pa = {i for i, x in enumerate(a) if x}
            pb = {i for i, x in enumerate(b) if x}
            same = (sum(a) > 0) == (sum(b) > 0)
            rule = (pa <= pb or pb <= pa) if same else not (pa & pb)
            assert alg1_adjacent(a, b) == rule, (a, b)
