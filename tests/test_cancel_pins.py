"""Pins of the oracle's persistence-directed cancellation (Sec. 3.5) to things
other than itself:

  * hand-derived cases (tests/golden/cancel/*.txt, each with its derivation);
  * brute force: the process the paper's steps describe, written without a
    queue -- at every step scan all saddles, cancel the one of lowest current
    (cost, id) if it is within the threshold -- on random small graphs, with
    ties and multi-saddles;
  * the elder rule: on graphs whose saddles all join two maxima and whose
    costs are distinct, cancelling in order of persistence must pair every
    maximum with the saddle at which, sweeping down from the top, its
    component first meets a component with a higher maximum (a merge tree
    built independently with a union-find);
  * invariants on extremum graphs of fields: threshold -> infinity leaves the
    global maximum alone, a negative threshold cancels nothing, scaling the
    field and the threshold by 2 changes nothing, the minimum graph of -f is
    the maximum graph of f, and every kept saddle is above the threshold or
    joins one maximum.
"""
import glob
import os
import random

import numpy as np
import pytest

import oracle
from paper_2303_02724_gb300 import fields as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cancel")


def _read(path):
    meta, cases = {}, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        k = k.strip()
        if k == "case":
            tau, alive, surv = [x.strip() for x in v.split("|")]
            cases.append((float(tau), [int(x) for x in alive.split()[1:]], [int(x) for x in surv.split()[1:]]))
        else:
            meta[k] = v.strip()
    mx = [tuple(x.split(":")) for x in meta["maxima"].split()]
    sd = [tuple(x.split(":")) for x in meta["saddles"].split()]
    maxima = np.array([int(a) for a, _ in mx], np.uint32)
    max_val = np.array([float(b) for _, b in mx], np.float32)
    saddles = np.array([int(a) for a, _, _ in sd], np.uint32)
    sad_val = np.array([float(b) for _, b, _ in sd], np.float32)
    ends = [sorted(int(e) for e in c.split(",")) for _, _, c in sd]
    row_ptr = np.concatenate([[0], np.cumsum([len(e) for e in ends])]).astype(np.uint64)
    col = np.array([e for es in ends for e in es], np.uint32)
    return (maxima, max_val, saddles, sad_val, row_ptr, col), cases


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))),
                         ids=lambda p: os.path.basename(p))
def test_golden_cancellation(path):
    g, cases = _read(path)
    assert cases
    for tau, alive, surv in cases:
        c = oracle.cancel(*g, tau)
        assert c.alive.tolist() == alive, (tau, c.alive)
        assert c.survivor.tolist() == surv, (tau, c.survivor)
        assert c.n_cancelled == len(alive) - sum(alive)
        # without equal values, the minimum graph of the negated values is the
        # same process (with ties the vertex-id tie-break does not flip)
        if len(set(g[1].tolist()) | set(g[3].tolist())) == len(g[1]) + len(g[3]):
            m = oracle.cancel(g[0], -g[1], g[2], -g[3], g[4], g[5], tau, minimum=True)
            assert m.alive.tolist() == alive and m.survivor.tolist() == surv


# ---------------------------------------------------------- brute force ----

def _cost(mv_of, sv, roots, minimum):
    """(second highest, highest) root under (value, id) and the float32 cost."""
    key = (lambda r: (-mv_of[r], -r)) if minimum else (lambda r: (mv_of[r], r))
    order = sorted(roots, key=key, reverse=True)
    fm, fs = np.float32(mv_of[order[1]]), np.float32(sv)
    c = np.float32(0.0) if fm == fs else (fs - fm if minimum else fm - fs)
    return np.float32(c), order[0]


def brute_cancel(maxima, max_val, saddles, sad_val, row_ptr, col, tau, minimum=False):
    mv_of = {int(m): np.float32(v) for m, v in zip(maxima, max_val)}
    root = {int(m): int(m) for m in maxima}

    def find(m):
        while root[m] != m:
            m = root[m]
        return m

    alive = [1] * len(saddles)
    tau = np.float32(tau)
    while True:
        best = None
        for i in range(len(saddles)):
            if not alive[i]:
                continue
            rs = {find(int(e)) for e in col[row_ptr[i]:row_ptr[i + 1]]}
            if len(rs) < 2:
                continue
            c, h = _cost(mv_of, sad_val[i], rs, minimum)
            if c > tau:
                continue
            k = (float(c), int(saddles[i]))
            if best is None or k < best[0]:
                best = (k, i, rs, h)
        if best is None:
            break
        _, i, rs, h = best
        alive[i] = 0
        for r in rs:
            if r != h:
                root[r] = h
    return np.array(alive, np.uint8), np.array([find(int(m)) for m in maxima], np.uint32)


def random_graph(rng, nm, ns, max_deg, ints=False, simple=False):
    ids = sorted(rng.sample(range(4 * (nm + ns) + 8), nm + ns))
    rng.shuffle(ids)
    mids, sids = sorted(ids[:nm]), sorted(ids[nm:])
    if ints:
        mval = {m: float(rng.randint(5, 9)) for m in mids}
    else:
        mval = {m: rng.uniform(1.0, 10.0) for m in mids}
    rows, svals = [], []
    for _ in sids:
        k = 2 if simple else rng.randint(1, min(max_deg, nm))
        ends = sorted(rng.sample(mids, k))
        lo = min(mval[e] for e in ends)
        # a saddle is lower than every maximum it reaches
        svals.append(float(rng.randint(0, int(lo))) if ints else rng.uniform(0.0, lo))
        rows.append(ends)
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.uint64)
    return (np.array(mids, np.uint32), np.array([mval[m] for m in mids], np.float32), np.array(sids, np.uint32),
            np.array(svals, np.float32), row_ptr, np.array([e for r in rows for e in r], np.uint32))


@pytest.mark.parametrize("seed", range(60))
def test_against_brute_force(seed):
    rng = random.Random(seed)
    nm, ns = rng.randint(2, 14), rng.randint(1, 24)
    g = random_graph(rng, nm, ns, 4, ints=seed % 3 == 0)
    taus = [-1.0, 0.0, np.inf, float(np.float32(rng.uniform(0, 6))), float(np.float32(rng.uniform(0, 2)))]
    for tau in taus:
        for minimum in (False, True):
            if minimum:
                gg = (g[0], -g[1], g[2], -g[3], g[4], g[5])
            else:
                gg = g
            want_alive, want_surv = brute_cancel(*gg, tau, minimum=minimum)
            c = oracle.cancel(*gg, tau, minimum=minimum)
            assert np.array_equal(c.alive, want_alive), (seed, tau, minimum)
            assert np.array_equal(c.survivor, want_surv), (seed, tau, minimum)


# ------------------------------------------------------------ elder rule ----

def elder_pairs(maxima, max_val, saddles, sad_val, row_ptr, col):
    """Merge tree by a union-find over saddles in decreasing (value, id):
    {saddle: (dying maximum, persistence)} for every saddle that joins two
    components; the younger (lower) maximum dies."""
    mv = {int(m): float(v) for m, v in zip(maxima, max_val)}
    parent = {int(m): int(m) for m in maxima}
    top = {int(m): int(m) for m in maxima}

    def find(m):
        while parent[m] != m:
            m = parent[m]
        return m

    order = sorted(range(len(saddles)), key=lambda i: (float(sad_val[i]), int(saddles[i])), reverse=True)
    pairs = {}
    for i in order:
        a, b = (int(x) for x in col[row_ptr[i]:row_ptr[i + 1]])
        ra, rb = find(a), find(b)
        if ra == rb:
            continue
        ta, tb = top[ra], top[rb]
        hi, lo = (ta, tb) if (mv[ta], ta) > (mv[tb], tb) else (tb, ta)
        pairs[int(saddles[i])] = (lo, float(np.float32(mv[lo]) - np.float32(sad_val[i])))
        parent[ra if top[ra] == lo else rb] = ra if top[ra] == hi else rb
        top[find(a)] = hi
    return pairs


@pytest.mark.parametrize("seed", range(40))
def test_simple_saddles_follow_the_elder_rule(seed):
    rng = random.Random(1000 + seed)
    while True:
        g = random_graph(rng, rng.randint(2, 16), rng.randint(1, 30), 2, simple=True)
        pairs = elder_pairs(*g)
        pers = [p for _, p in pairs.values()]
        if len(set(pers)) == len(pers):  # distinct costs: no tie-break involved
            break
    for tau in [np.inf, float(np.float32(np.median(pers))) if pers else 0.0, 0.0]:
        c = oracle.cancel(*g, tau)
        want = {s for s, (_, p) in pairs.items() if p <= np.float32(tau)}
        got = {int(s) for s, a in zip(g[2], c.alive) if not a}
        assert got == want, (seed, tau)
        dead = {m for s, (m, p) in pairs.items() if p <= np.float32(tau)}
        assert {int(m) for m, r in zip(g[0], c.survivor) if r != m} == dead


# ------------------------------------------------ invariants on fields ----

def _field_graph(f, minimum=False):
    return oracle.compute(f.values, minimum=minimum)


def _check_kept(g, c, tau, minimum=False):
    """Every kept saddle is above the threshold or joins one maximum."""
    surv = dict(zip(g.maxima.tolist(), c.survivor.tolist()))
    mv = dict(zip(g.maxima.tolist(), g.max_val.tolist()))
    for i in np.flatnonzero(c.alive):
        rs = {surv[int(m)] for m in g.col[g.row_ptr[i]:g.row_ptr[i + 1]]}
        if len(rs) >= 2:
            cost, _ = _cost(mv, g.sad_val[i], rs, minimum)
            assert cost > np.float32(tau)
    # survivors are survivors of themselves
    for m, r in surv.items():
        assert surv[r] == r


@pytest.mark.parametrize("case", ["grf", "gauss2d", "ties", "white4d"])
def test_field_invariants(case):
    f = {"grf": lambda: F.grf((24, 20, 18), 2), "gauss2d": lambda: F.config_2d_256(side=80),
         "ties": lambda: F.integer_ties((30, 28), 3, 5), "white4d": lambda: F.white_noise((6, 5, 5, 4), 7)}[case]()
    g = _field_graph(f)
    # infinity: the extremum graph of a connected grid collapses to the global maximum
    c = oracle.cancel_graph(g, np.inf)
    gmax = int(g.maxima[np.lexsort((g.maxima, g.max_val))[-1]])
    assert set(c.survivor.tolist()) == {gmax}
    # each cancellation merges at least one maximum (a multi-saddle several)
    assert 1 <= c.n_cancelled <= g.maxima.size - 1 or g.maxima.size == 1
    _check_kept(g, c, np.inf)
    assert oracle.cancel_graph(g, -1.0).n_cancelled == 0
    vals = np.sort(g.max_val)
    for tau in [0.0, float(np.float32((vals[-1] - vals[0]) / 7)), float(np.float32((vals[-1] - vals[0]) / 2))]:
        c = oracle.cancel_graph(g, tau)
        _check_kept(g, c, tau)
        # scaling the field and the threshold by 2 is exact in float32
        g2 = _field_graph(F.Field(f.values * np.float32(2), f.extents))
        c2 = oracle.cancel_graph(g2, np.float32(2) * np.float32(tau))
        assert np.array_equal(c.alive, c2.alive) and np.array_equal(c.survivor, c2.survivor)
        # the minimum graph of -f is the maximum graph of f (tie-free fields:
        # the vertex-id tie-break does not flip with the values)
        if np.unique(f.values).size < f.values.size:
            continue
        gm = _field_graph(F.Field(-f.values, f.extents), minimum=True)
        cm = oracle.cancel_graph(gm, tau, minimum=True)
        assert np.array_equal(c.alive, cm.alive) and np.array_equal(c.survivor, cm.survivor)


# ------------------------------------------- the device's round schedule ----

def rounds_model(maxima, max_val, saddles, sad_val, row_ptr, col, tau, minimum=False):
    """The schedule the device runs (data-parallel rounds), written out in
    Python on the graph arrays: in every round each waiting saddle computes its
    current maxima, cost and lb (lowest maximum minus the saddle); a saddle is
    cancelled when its (cost, id) is below the (lb, id) of every other waiting
    saddle that reaches one of its dying maxima, or when it is the globally
    cheapest; merges follow chains.  Must reproduce the serial queue."""
    mv = {int(m): np.float32(v) for m, v in zip(maxima, max_val)}
    root = {int(m): int(m) for m in maxima}
    state = [0] * len(saddles)  # 0 waiting, 1 cancelled, 2 never
    tau32 = np.float32(tau)
    order = (lambda r: (-mv[r], -r)) if minimum else (lambda r: (mv[r], r))
    rounds = 0
    while True:
        rounds += 1
        info = {}
        for i in range(len(saddles)):
            if state[i]:
                continue
            rs = sorted({root[int(e)] for e in col[row_ptr[i]:row_ptr[i + 1]]}, key=order, reverse=True)
            if len(rs) < 2:
                state[i] = 2
                continue
            fs = np.float32(sad_val[i])

            def cost_to(m):
                fm = mv[m]
                return np.float32(0) if fm == fs else (fs - fm if minimum else fm - fs)
            c, lb = cost_to(rs[1]), cost_to(rs[-1])
            if lb > tau32:
                state[i] = 2
                continue
            info[i] = (rs, (float(c), int(saddles[i])), (float(lb), int(saddles[i])))
        cand = [k[1] for k in info.values() if k[1][0] <= tau32]
        if not cand:
            return np.array([0 if s == 1 else 1 for s in state], np.uint8), \
                np.array([root[int(m)] for m in maxima], np.uint32), rounds
        gmin = min(cand)
        reach = {}
        for i, (rs, _, lk) in info.items():
            for r in rs:
                reach.setdefault(r, []).append((lk, i))
        merge = {}
        for i, (rs, ck, _) in info.items():
            if ck[0] > tau32:
                continue
            safe = ck == gmin or all(lk > ck for r in rs[1:] for lk, j in reach[r] if j != i)
            if safe:
                state[i] = 1
                for r in rs[1:]:
                    assert r not in merge  # dying maxima of one round are disjoint
                    merge[r] = rs[0]
        for m in root:
            r = root[m]
            while r in merge:
                r = merge[r]
            root[m] = r


@pytest.mark.parametrize("seed", range(80))
def test_round_schedule_matches_serial_queue(seed):
    rng = random.Random(5000 + seed)
    nm, ns = rng.randint(2, 30), rng.randint(1, 60)
    g = random_graph(rng, nm, ns, 5, ints=seed % 4 == 0, simple=seed % 5 == 1)
    for tau in [0.0, float(np.float32(rng.uniform(0, 3))), float(np.float32(rng.uniform(0, 8))), np.inf]:
        for minimum in (False, True):
            gg = (g[0], -g[1], g[2], -g[3], g[4], g[5]) if minimum else g
            c = oracle.cancel(*gg, tau, minimum=minimum)
            alive, surv, _ = rounds_model(*gg, tau, minimum=minimum)
            assert np.array_equal(alive, c.alive), (seed, tau, minimum)
            assert np.array_equal(surv, c.survivor), (seed, tau, minimum)


def test_round_schedule_on_a_field_graph_takes_few_rounds():
    """On the extremum graph of a random field the rounds stay far below the
    number of cancellations (the schedule is parallel, not serial)."""
    g = oracle.compute(F.grf((24, 20, 18), 2).values)
    c = oracle.cancel_graph(g, np.inf)
    alive, surv, rounds = rounds_model(g.maxima, g.max_val, g.saddles, g.sad_val, g.row_ptr, g.col, np.inf)
    assert np.array_equal(alive, c.alive) and np.array_equal(surv, c.survivor)
    assert rounds < c.n_cancelled / 4, (rounds, c.n_cancelled)
