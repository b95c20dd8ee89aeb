"""One-direction edges (Section 3.4, outer joins): the edge of t0 LEFT JOIN
t1 transfers filters only from t0 to t1, so in exactly one pass, and t1
never removes a row of t0."""
import dataclasses

import numpy as np
import pytest

import workloads as W

ONE_WAY = 1


def _two(keys0, sel0, keys1, sel1=None, one_way=True):
    L = W.Table("L", len(keys0), [np.asarray(keys0, np.int32)], ["k"],
                None if sel0 is None else W.bitmap_from_rows(len(keys0), sel0))
    R = W.Table("R", len(keys1), [np.asarray(keys1, np.int32)], ["k"],
                None if sel1 is None else W.bitmap_from_rows(len(keys1), sel1))
    return W.Workload("lj", [L, R], [W.Edge(0, (0,), 1, (0,), ONE_WAY if one_way else 0)])


def _rows(res, p, v, n):
    return W.rows_from_bitmap(res["surv"][p][v], n).tolist()


def test_left_join_forward_when_left_is_smaller(oracle_lib):
    """L (4 rows, keeps rows 0, 1: keys 0, 1) LEFT JOIN R (6 rows, keys
    0 1 2 3 0 5).  L is smaller, so the edge points L -> R and transfers in
    the forward pass: R keeps rows 0, 1, 4.  In the backward pass it would
    point R -> L, which is blocked: L keeps both its rows (an inner join
    would keep them too here, but never fewer), and no filter is built."""
    w = _two([0, 1, 2, 3], [0, 1], [0, 1, 2, 3, 0, 5])
    ex = oracle_lib.transfer(w, exact=True)
    assert _rows(ex, 1, 0, 4) == [0, 1]
    assert _rows(ex, 1, 1, 6) == [0, 1, 4]
    bl = oracle_lib.transfer(w)  # a Bloom filter may also pass rows 2, 3 or 5
    assert _rows(bl, 1, 0, 4) == [0, 1]
    assert set(_rows(bl, 1, 1, 6)) >= {0, 1, 4}
    res = oracle_lib.transfer(w)
    assert res["nblocks"][0][0] >= 1 and res["nblocks"][1][0] == 0


def test_left_join_backward_when_left_is_larger(oracle_lib):
    """L (5 rows, keeps rows 0, 1: keys 0, 1) LEFT JOIN R (3 rows, keys
    0 9 1).  R is smaller, so the forward pass would send R -> L: blocked,
    L keeps rows 0, 1 and no filter is built.  The backward pass sends
    L -> R: R keeps rows 0 and 2."""
    w = _two([0, 1, 2, 3, 4], [0, 1], [0, 9, 1])
    ex = oracle_lib.transfer(w, exact=True)
    assert _rows(ex, 0, 0, 5) == [0, 1] and _rows(ex, 1, 0, 5) == [0, 1]
    assert _rows(ex, 0, 1, 3) == [0, 1, 2] and _rows(ex, 1, 1, 3) == [0, 2]
    bl = oracle_lib.transfer(w)
    assert bl["nblocks"][0][0] == 0 and bl["nblocks"][1][0] >= 1


def test_left_join_semantics_brute_force(oracle_lib):
    """Exact sets, two tables: the preserved side keeps every selected row,
    the other side keeps the selected rows that match one of them -- the
    rows that take part in L LEFT JOIN R."""
    rng = np.random.default_rng(3)
    for _ in range(40):
        n0, n1 = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        k0 = rng.integers(-3, 6, n0)
        k1 = rng.integers(-3, 6, n1)
        s0 = sorted(rng.choice(n0, size=int(rng.integers(0, n0 + 1)), replace=False).tolist())
        s1 = sorted(rng.choice(n1, size=int(rng.integers(0, n1 + 1)), replace=False).tolist())
        res = oracle_lib.transfer(_two(k0, s0, k1, s1), exact=True)
        left_keys = {int(k0[r]) for r in s0}
        assert _rows(res, 1, 0, n0) == s0
        assert _rows(res, 1, 1, n1) == [r for r in s1 if int(k1[r]) in left_keys]


@pytest.mark.parametrize("exact", [True, False])
def test_preserved_side_is_as_without_the_edge(oracle_lib, exact):
    """In a tree, cutting a one-way edge t0 -> t1 leaves t0's component
    unchanged: nothing crosses from t1's side to t0's.  So every table on
    t0's side ends with exactly the rows (and builds exactly the filters) it
    has when the edge is removed -- in Bloom mode too."""
    for seed in range(30):
        w = W.random_tiny(900 + seed, 4 + seed % 4, max_rows=60, acyclic=True, composite_prob=0.2)
        i = seed % len(w.edges)
        cut = w.edges[i]
        w1 = dataclasses.replace(w, edges=[dataclasses.replace(e, flags=ONE_WAY) if j == i else e
                                           for j, e in enumerate(w.edges)])
        w0 = dataclasses.replace(w, edges=[e for j, e in enumerate(w.edges) if j != i])
        # t0's component without the edge
        comp, stack = {cut.t0}, [cut.t0]
        while stack:
            v = stack.pop()
            for e in w0.edges:
                for a, b in ((e.t0, e.t1), (e.t1, e.t0)):
                    if a == v and b not in comp:
                        comp.add(b)
                        stack.append(b)
        r1, r0 = oracle_lib.transfer(w1, exact=exact), oracle_lib.transfer(w0, exact=exact)
        for v in comp:
            for p in range(2):
                assert np.array_equal(r1["surv"][p][v], r0["surv"][p][v]), (seed, v, p)
        # an inner join on the edge keeps a subset of the rows, on every table
        ri = oracle_lib.transfer(w, exact=exact)
        for v in range(w.n_tables):
            assert (ri["surv"][1][v] & r1["surv"][1][v] == ri["surv"][1][v]).all(), (seed, v)


def test_unknown_flags_rejected(oracle_lib):
    w = _two([0, 1], [0], [0, 1], one_way=False)
    w = dataclasses.replace(w, edges=[dataclasses.replace(w.edges[0], flags=2)])
    with pytest.raises(ValueError):
        oracle_lib.transfer(w)
