"""Pins of the oracle's Bloom join (Section 2.1; the BloomJoin baseline of
Section 4): a one-hop transfer in one direction.  Each edge's filter holds
the keys of its building table's selected rows (the smaller table, or t0
of a one-way edge) and is probed once by the other end.

Pinned by a hand-worked chain where the transfer removes more than the
Bloom join, by the definitional semi-join on tiny random graphs (exact
sets), by the reduction to the forward pass of a transfer on a star (every
builder a source), and by the containments the paper implies: the transfer
(exact) never keeps a row the one-hop schedule drops, Bloom survivors
contain the exact ones, and the join result is unchanged."""
import dataclasses

import numpy as np
import pytest

import workloads as W

ONE_WAY = 1


def _rows(bm, n):
    return W.rows_from_bitmap(bm, n).tolist()


def _chain():
    """R(B) - S(B, C) - T(C), 3 < 4 < 5 rows, so the edges point R -> S -> T.
    R keeps row 0 (B = 1).  One hop: S keeps its rows with B = 1 (0 and 3);
    T is probed with S's SELECTED keys C = 10, 20, 30, 40 and keeps rows 0..3
    (not 50).  A transfer carries R's predicate on to T: S's survivors have
    C = 10, 40, so T keeps rows 0 and 3, and the backward pass changes
    nothing further."""
    R = W.Table("R", 3, [np.array([1, 2, 3], np.int32)], ["B"], W.bitmap_from_rows(3, [0]))
    S = W.Table("S", 4, [np.array([1, 2, 3, 1], np.int32), np.array([10, 20, 30, 40], np.int32)],
                ["B", "C"], None)
    T = W.Table("T", 5, [np.array([10, 20, 30, 40, 50], np.int32)], ["C"], None)
    return W.Workload("chain", [R, S, T], [W.Edge(0, (0,), 1, (0,)), W.Edge(1, (1,), 2, (0,))],
                      bits_per_key=64)


@pytest.mark.parametrize("exact", [True, False])
def test_chain_one_hop_stops_after_one_edge(oracle_lib, exact):
    w = _chain()
    oh = oracle_lib.one_hop(w, exact=exact)
    assert _rows(oh["surv"][0], 3) == [0]
    assert _rows(oh["surv"][1], 4) == [0, 3]
    t_rows = _rows(oh["surv"][2], 5)
    if exact:
        assert t_rows == [0, 1, 2, 3]
    else:  # no false negatives; at 64 bits per key the key 50 is rejected too
        assert set(t_rows) >= {0, 1, 2, 3}
    pt = oracle_lib.transfer(w, exact=exact)
    assert _rows(pt["surv"][1][2], 5) == [0, 3]
    assert _rows(pt["surv"][1][1], 4) == [0, 3]
    assert oh["count"] == [1, 2, len(t_rows)]


def test_chain_filters_hold_the_selected_keys(oracle_lib):
    """S -> T's filter is built from S's 4 selected rows (c = 4, not S's 2
    transfer survivors) and equals a filter built from those keys alone."""
    w = _chain()
    oh = oracle_lib.one_hop(w)
    nb = oracle_lib.nblocks_for(4, 5, 64, 256)
    assert oh["nblocks"][1] == nb
    hs = [oracle_lib.hash1(x) for x in (10, 20, 30, 40)]
    assert np.array_equal(oh["filters"][1], oracle_lib.filter_build(hs, nb, 256, 4))
    assert oh["nblocks"][0] == oracle_lib.nblocks_for(1, 4, 64, 256)
    assert np.array_equal(oh["filters"][0], oracle_lib.filter_build([oracle_lib.hash1(1)],
                                                                    oh["nblocks"][0], 256, 4))


def _builder(w, i):
    e = w.edges[i]
    if e.flags & ONE_WAY:
        return e.t0
    import oracle
    return oracle.orient([t.n_rows for t in w.tables], w.edges)["src"][i]


def _side(e, v):
    return e.c0 if e.t0 == v else e.c1


def _key(t, cols, r):
    return tuple(int(t.cols[c][r]) for c in cols)


def _selected(t):
    if t.sel is None:
        return list(range(t.n_rows))
    return _rows(t.sel, t.n_rows)


def _semi_join_one_hop(w):
    """The definition: a selected row of v survives iff, for every edge whose
    filter v probes, its key equals the key of some selected row of the
    edge's builder."""
    keys = []
    for i, e in enumerate(w.edges):
        b = _builder(w, i)
        keys.append({_key(w.tables[b], _side(e, b), r) for r in _selected(w.tables[b])})
    out = []
    for v, t in enumerate(w.tables):
        keep = []
        for r in _selected(t):
            ok = True
            for i, e in enumerate(w.edges):
                if v not in (e.t0, e.t1) or _builder(w, i) == v:
                    continue
                ok = ok and _key(t, _side(e, v), r) in keys[i]
            if ok:
                keep.append(r)
        out.append(keep)
    return out


def _tiny(n, acyclic, one_way_prob=0.0, base=7000):
    rng = np.random.default_rng(base)
    out = []
    for s in range(n):
        w = W.random_tiny(base + s + (0 if acyclic else 500), 2 + s % 5, max_rows=14, domain=5,
                          acyclic=acyclic, composite_prob=0.25)
        edges = [dataclasses.replace(e, flags=ONE_WAY if rng.random() < one_way_prob else 0) for e in w.edges]
        out.append(dataclasses.replace(w, edges=edges))
    return out


@pytest.mark.parametrize("one_way_prob", [0.0, 0.4])
def test_exact_one_hop_is_the_one_hop_semi_join(oracle_lib, one_way_prob):
    for w in _tiny(30, True, one_way_prob) + _tiny(30, False, one_way_prob):
        oh = oracle_lib.one_hop(w, exact=True)
        want = _semi_join_one_hop(w)
        for v, t in enumerate(w.tables):
            assert _rows(oh["surv"][v], t.n_rows) == want[v], (w.name, v)
            assert oh["count"][v] == len(want[v])


@pytest.mark.parametrize("one_way_prob", [0.0, 0.4])
def test_transfer_keeps_no_row_one_hop_drops(oracle_lib, one_way_prob):
    """Exact sets: a transfer's filters hold subsets of the selected keys the
    one-hop filters hold, and its backward pass only removes more."""
    for w in _tiny(30, True, one_way_prob) + _tiny(30, False, one_way_prob):
        oh = oracle_lib.one_hop(w, exact=True)
        pt = oracle_lib.transfer(w, exact=True)
        for v, t in enumerate(w.tables):
            assert set(_rows(pt["surv"][1][v], t.n_rows)) <= set(_rows(oh["surv"][v], t.n_rows))


@pytest.mark.parametrize("bpk", [2, 10])
def test_bloom_one_hop_contains_exact_and_keeps_join_result(oracle_lib, bpk):
    for w in _tiny(25, True) + _tiny(25, False):
        w.bits_per_key = bpk
        ex = oracle_lib.one_hop(w, exact=True)
        bl = oracle_lib.one_hop(w)
        for v, t in enumerate(w.tables):
            assert set(_rows(ex["surv"][v], t.n_rows)) <= set(_rows(bl["surv"][v], t.n_rows))
            assert set(_rows(bl["surv"][v], t.n_rows)) <= set(_selected(t))
        before = oracle_lib.brute_force(w)["n_results"]
        for v, t in enumerate(w.tables):
            t.sel = bl["surv"][v].copy()
        assert oracle_lib.brute_force(w)["n_results"] == before


def _small_star(seed=11):
    """Fact F (4000 rows, no predicate) with three dimensions of 50..400
    rows that carry predicates: every dimension is a source of the transfer
    graph."""
    rng = np.random.default_rng(seed)
    dims, edges, fcols = [], [], []
    for i, m in enumerate((50, 120, 400)):
        d = W.Table(f"D{i}", m, [np.arange(m, dtype=np.int64) * 7 + i], ["id"],
                    W.bitmap_from_bools(rng.random(m) < 0.3))
        dims.append(d)
        fcols.append((rng.integers(0, m, 4000) * 7 + i).astype(np.int64))
        edges.append(W.Edge(i + 1, (0,), 0, (i,)))
    F = W.Table("F", 4000, fcols, [f"fk{i}" for i in range(3)], None)
    return W.Workload("star_small", [F] + dims, edges, bits_per_key=8)


def test_star_one_hop_is_the_forward_pass(oracle_lib):
    """On a star whose dimensions are all smaller than the fact table, every
    builder is a source of the transfer graph: the forward pass builds the
    same filters from the same selected rows, so the fact table's one-hop
    survivors are its forward survivors, bit for bit (Section 2.1's remark
    that a star lets every dimension's predicate reach the fact table)."""
    w = _small_star()
    oh = oracle_lib.one_hop(w)
    pt = oracle_lib.transfer(w)
    assert np.array_equal(oh["surv"][0], pt["surv"][0][0])
    for i in range(len(w.edges)):
        assert oh["nblocks"][i] == pt["nblocks"][0][i]
        assert np.array_equal(oh["filters"][i], pt["filters"][0][i])
    for v in range(1, w.n_tables):  # nothing reaches a dimension in one hop
        assert np.array_equal(oh["surv"][v], w.tables[v].sel)


def test_one_way_edge_builds_on_t0_even_when_larger(oracle_lib):
    """L (6 rows) LEFT JOIN R (4 rows): the transfer graph points R -> L, but a
    one-way edge builds on t0 = L, so R is filtered by L's selected keys and
    L is never filtered by R."""
    L = W.Table("L", 6, [np.array([0, 1, 2, 3, 4, 5], np.int32)], ["k"], W.bitmap_from_rows(6, [1, 2]))
    R = W.Table("R", 4, [np.array([1, 2, 7, 1], np.int32)], ["k"], W.bitmap_from_rows(4, [0, 2, 3]))
    w = W.Workload("lj", [L, R], [W.Edge(0, (0,), 1, (0,), ONE_WAY)])
    oh = oracle_lib.one_hop(w, exact=True)
    assert _rows(oh["surv"][0], 6) == [1, 2]
    assert _rows(oh["surv"][1], 4) == [0, 3]
