"""Pins of the oracle's transfer schedule against what the paper fixes:
the Fig. 2 and Fig. 3 worked examples, the size-ordered transfer graph,
the semi-join (exact-set) reading of a transfer checked by brute-force
join, Bloom survivors containing the exact ones, and an unchanged join
result."""
import numpy as np
import pytest

import workloads as W
from _fixtures import golden_workload, rows1


def _bitmap_rows(words, n):
    return set(W.rows_from_bitmap(words, n).tolist())


@pytest.mark.parametrize("exact", [True, False])
def test_fig2_filter_transformation(oracle_lib, exact):
    w, g, tid = golden_workload("fig2_filter_transformation.json", bits_per_key=64)
    res = oracle_lib.transfer(w, exact=exact)
    for name, rows in g["expect_forward_survivors"].items():
        v = tid[name]
        assert rows1(res["surv"][0][v], w.tables[v].n_rows) == rows
    if exact:
        ps, bs = res["sectors"][0][tid["R"]]
        assert (ps, bs) == (g["expect_forward_sectors_R"]["probe"], g["expect_forward_sectors_R"]["build"])
    else:
        # the outgoing filter holds exactly the keys of rows 3 and 5: each probes true,
        # and a filter built from those keys alone is bit-identical
        e = g["expect_outgoing_keys"]["edge"]
        keys = g["expect_outgoing_keys"]["keys"]
        nb = res["nblocks"][0][e]
        assert nb == oracle_lib.nblocks_for(2, 6, 64, 256)
        hs = [oracle_lib.hash1(x) for x in keys]
        assert np.array_equal(res["filters"][0][e], oracle_lib.filter_build(hs, nb, 256, 4))


@pytest.mark.parametrize("exact", [True, False])
def test_fig3_forward_then_backward(oracle_lib, exact):
    w, g, tid = golden_workload("fig3_forward_backward.json", bits_per_key=64)
    res = oracle_lib.transfer(w, exact=exact)
    for p, key in ((0, "expect_forward_survivors"), (1, "expect_backward_survivors")):
        for name, rows in g[key].items():
            v = tid[name]
            assert rows1(res["surv"][p][v], w.tables[v].n_rows) == rows, (p, name)


def test_transfer_graph_points_small_to_big_with_id_ties(oracle_lib):
    n_rows = [50, 10, 50, 7, 1000]
    edges = [W.Edge(0, (0,), 1, (0,)), W.Edge(0, (1,), 2, (0,)), W.Edge(3, (0,), 4, (0,)),
             W.Edge(4, (1,), 2, (1,)), W.Edge(2, (2,), 1, (1,))]
    o = oracle_lib.orient(n_rows, edges)
    assert list(zip(o["src"], o["dst"])) == [(1, 0), (0, 2), (3, 4), (2, 4), (1, 2)]
    assert o["order"] == [3, 1, 0, 2, 4]
    pos = {v: i for i, v in enumerate(o["order"])}
    assert all(pos[s] < pos[d] for s, d in zip(o["src"], o["dst"]))  # a topological order


def _in_tree(w):
    """True when every table has at most one outgoing edge in the size-ordered DAG."""
    import oracle
    o = oracle.orient([t.n_rows for t in w.tables], w.edges)
    outdeg = np.bincount(o["src"], minlength=w.n_tables) if w.edges else np.zeros(w.n_tables)
    return bool((outdeg <= 1).all())


def _tiny_cases(acyclic, n=40):
    out = []
    for s in range(n):
        nt = 2 + s % 5
        w = W.random_tiny(1000 + s + (0 if acyclic else 5000), nt, max_rows=14, domain=5,
                          acyclic=acyclic, composite_prob=0.25)
        out.append(w)
    return out


def test_exact_mode_equals_full_reduction_on_in_trees(oracle_lib):
    checked = 0
    for w in _tiny_cases(True, 80):
        if not _in_tree(w):
            continue
        ex = oracle_lib.transfer(w, exact=True)
        bf = oracle_lib.brute_force(w)
        for v, t in enumerate(w.tables):
            assert _bitmap_rows(ex["surv"][1][v], t.n_rows) == set(bf["participating"][v]), (w.name, v)
        checked += 1
    assert checked >= 20


def test_exact_mode_contains_full_reduction_on_any_graph(oracle_lib):
    for w in _tiny_cases(True, 30) + _tiny_cases(False, 30):
        ex = oracle_lib.transfer(w, exact=True)
        bf = oracle_lib.brute_force(w)
        for v, t in enumerate(w.tables):
            assert set(bf["participating"][v]) <= _bitmap_rows(ex["surv"][1][v], t.n_rows)
            # semi-joins only ever remove rows: backward survivors within forward survivors
            assert _bitmap_rows(ex["surv"][1][v], t.n_rows) <= _bitmap_rows(ex["surv"][0][v], t.n_rows)


def test_exact_mode_is_a_fixpoint_on_in_trees(oracle_lib):
    for w in _tiny_cases(True, 40):
        if not _in_tree(w):
            continue
        ex = oracle_lib.transfer(w, exact=True)
        for v, t in enumerate(w.tables):
            t.sel = ex["surv"][1][v].copy()
        again = oracle_lib.transfer(w, exact=True)
        for v in range(w.n_tables):
            assert np.array_equal(again["surv"][1][v], ex["surv"][1][v])


@pytest.mark.parametrize("bpk", [2, 10])
def test_bloom_survivors_contain_exact_and_keep_join_result(oracle_lib, bpk):
    for w in _tiny_cases(True, 30) + _tiny_cases(False, 30):
        w.bits_per_key = bpk
        ex = oracle_lib.transfer(w, exact=True)
        bl = oracle_lib.transfer(w, exact=False)
        for p in range(2):
            for v, t in enumerate(w.tables):
                assert _bitmap_rows(ex["surv"][p][v], t.n_rows) <= _bitmap_rows(bl["surv"][p][v], t.n_rows)
        before = oracle_lib.brute_force(w)["n_results"]
        for v, t in enumerate(w.tables):
            t.sel = bl["surv"][1][v].copy()
        assert oracle_lib.brute_force(w)["n_results"] == before


def test_every_survivor_key_probes_true_in_its_outgoing_filter(oracle_lib):
    w = W.chain3(scale=0.2)
    res = oracle_lib.transfer(w)
    o = oracle_lib.orient([t.n_rows for t in w.tables], w.edges)
    for p in range(2):
        for i, e in enumerate(w.edges):
            b = o["src"][i] if p == 0 else o["dst"][i]
            cols = e.c0 if e.t0 == b else e.c1
            col = w.tables[b].cols[cols[0]]
            rows = W.rows_from_bitmap(res["surv"][p][b], w.tables[b].n_rows)
            hs = [oracle_lib.hash1(int(col[r])) for r in rows]
            assert oracle_lib.filter_probe(res["filters"][p][i], res["nblocks"][p][i], 256, 4, hs).all()


def test_lip_probe_order_sectors(oracle_lib):
    """Two incoming filters into V (64 int32 rows = 8 sectors per column).

    Sender P keeps 1 of its 8 rows (pass rate 1/8) and sender Q keeps all 4
    (rate 1), so P's filter is probed first, over all 8 sectors of V.k_p;
    it leaves the rows whose key is P's one surviving key: rows 0..7 only
    (sector 0), so Q's column is read in 1 sector.  Exact sets, so no false
    positives blur the count.
    """
    P = W.Table("P", 8, [np.arange(8, dtype=np.int32)], ["k"], W.bitmap_from_rows(8, [0]))
    Q = W.Table("Q", 4, [np.arange(4, dtype=np.int32)], ["k"], None)
    kp = np.repeat(np.arange(8, dtype=np.int32), 8)        # rows 0..7 carry key 0
    kq = (np.arange(64) % 4).astype(np.int32)
    V = W.Table("V", 64, [kp, kq], ["k_p", "k_q"], None)
    w = W.Workload("lip", [P, Q, V], [W.Edge(0, (0,), 2, (0,)), W.Edge(1, (0,), 2, (1,))])
    res = oracle_lib.transfer(w, exact=True)
    assert res["sectors"][0][2] == (8 + 1, 0)
    assert W.rows_from_bitmap(res["surv"][0][2], 64).tolist() == list(range(8))


def test_probe_order_is_builder_level_first(oracle_lib):
    """A less selective filter from a lower DAG level is probed first.

    Ranks: B0 (4 rows) < A (8) < B1 (16) < V (64); edges A->V, B0->B1, B1->V,
    so in the forward pass A and B0 are on level 0, B1 on level 1, V on 2.
    A keeps rows 0..3 (keys 0..3, rate 4/8); B0 keeps key 0, so B1 keeps its
    rows 0, 4, 8, 12 (rate 4/16).  LIP alone would probe B1's filter first;
    the builder level puts A's first.  V.k_a = row // 8 passes A for rows
    0..31, read over all 8 sectors of V.k_a (int32: 8 rows per sector); then
    V.k_b = row % 16 is probed on rows 0..31 only: 4 sectors.  Total 12
    (LIP alone would read 8 + 8 = 16).  Survivors: rows 0..31 with
    row % 4 == 0.  Exact sets, so no false positives blur the count.
    """
    B0 = W.Table("B0", 4, [np.arange(4, dtype=np.int32)], ["k"], W.bitmap_from_rows(4, [0]))
    A = W.Table("A", 8, [np.arange(8, dtype=np.int32)], ["k"], W.bitmap_from_rows(8, [0, 1, 2, 3]))
    i16 = np.arange(16, dtype=np.int32)
    B1 = W.Table("B1", 16, [i16 % 4, i16], ["b0", "bv"], None)
    i64 = np.arange(64, dtype=np.int32)
    V = W.Table("V", 64, [i64 // 8, i64 % 16], ["k_a", "k_b"], None)
    w = W.Workload("levels", [B0, A, B1, V],
                   [W.Edge(1, (0,), 3, (0,)), W.Edge(0, (0,), 2, (0,)), W.Edge(2, (1,), 3, (1,))])
    res = oracle_lib.transfer(w, exact=True)
    assert res["count"][0][2] == 4
    assert res["sectors"][0][3] == (8 + 4, 0)
    assert W.rows_from_bitmap(res["surv"][0][3], 64).tolist() == list(range(0, 32, 4))


def test_chain3_exact_magnitudes(oracle_lib):
    """Expected sizes of the 3-table chain (10k/100k/10k, 10% and 20% kept):
    S keeps ~100k*0.1*0.2 = 2000 rows; R keeps ~1000*(1-e^-2) ~ 865 and T
    ~2000*(1-e^-1) ~ 1264 (Poisson occupancy)."""
    w = W.chain3()
    ex = oracle_lib.transfer(w, exact=True)
    c = ex["count"][1]
    assert 1800 < c[1] < 2200
    assert 800 < c[0] < 930
    assert 1180 < c[2] < 1350
    bl = oracle_lib.transfer(w)
    assert all(bl["count"][1][v] >= c[v] for v in range(3))


def _levels_workload():
    B0 = W.Table("B0", 4, [np.arange(4, dtype=np.int32)], ["k"], W.bitmap_from_rows(4, [0]))
    A = W.Table("A", 8, [np.arange(8, dtype=np.int32)], ["k"], W.bitmap_from_rows(8, [0, 1, 2, 3]))
    i16 = np.arange(16, dtype=np.int32)
    B1 = W.Table("B1", 16, [i16 % 4, i16], ["b0", "bv"], None)
    i64 = np.arange(64, dtype=np.int32)
    V = W.Table("V", 64, [i64 // 8, i64 % 16], ["k_a", "k_b"], None)
    return W.Workload("levels", [B0, A, B1, V],
                      [W.Edge(1, (0,), 3, (0,)), W.Edge(0, (0,), 2, (0,)), W.Edge(2, (1,), 3, (1,))])


@pytest.mark.parametrize("order,sectors", [(0, 8 + 4), (1, 8 + 8), (2, 8 + 4)])
def test_probe_order_modes_levels_example(oracle_lib, order, sectors):
    """The example above under each probe order.  LIP alone (order 1) probes
    B1's filter (rate 4/16) before A's (4/8): B1 passes V's rows with
    row % 16 in {0, 4, 8, 12}, two in every 8-row sector, so both columns are
    read in all 8 sectors.  Edge-id order (2) probes edge 0 (A's) first, as
    the level order does.  The survivors never change."""
    res = oracle_lib.transfer(_levels_workload(), exact=True, probe_order=order)
    assert res["sectors"][0][3] == (sectors, 0)
    assert W.rows_from_bitmap(res["surv"][0][3], 64).tolist() == list(range(0, 32, 4))


@pytest.mark.parametrize("order,sectors", [(0, 8 + 1), (1, 8 + 1), (2, 8 + 8)])
def test_probe_order_modes_edge_id_example(oracle_lib, order, sectors):
    """The LIP example with Q's edge listed first.  Both builders are on
    level 0; LIP (orders 0 and 1) still probes P's filter (rate 1/8) first:
    8 + 1 sectors.  Edge-id order probes Q's filter (rate 1) first, which
    keeps every row (8 sectors of V.k_q), then P's over all 8 sectors of V.k_p."""
    P = W.Table("P", 8, [np.arange(8, dtype=np.int32)], ["k"], W.bitmap_from_rows(8, [0]))
    Q = W.Table("Q", 4, [np.arange(4, dtype=np.int32)], ["k"], None)
    kp = np.repeat(np.arange(8, dtype=np.int32), 8)
    kq = (np.arange(64) % 4).astype(np.int32)
    V = W.Table("V", 64, [kp, kq], ["k_p", "k_q"], None)
    w = W.Workload("lip_rev", [P, Q, V], [W.Edge(1, (0,), 2, (1,)), W.Edge(0, (0,), 2, (0,))])
    res = oracle_lib.transfer(w, exact=True, probe_order=order)
    assert res["sectors"][0][2] == (sectors, 0)
    assert W.rows_from_bitmap(res["surv"][0][2], 64).tolist() == list(range(8))


def test_probe_order_never_changes_results(oracle_lib):
    for i in range(12):
        w = W.random_tiny(500 + i, 3 + i % 4, max_rows=200, acyclic=(i % 3 != 0), composite_prob=0.3)
        base = oracle_lib.transfer(w)
        for order in (1, 2):
            got = oracle_lib.transfer(w, probe_order=order)
            assert got["count"] == base["count"]
            assert got["nblocks"] == base["nblocks"]
            for p in range(2):
                for a, b in zip(got["surv"][p], base["surv"][p]):
                    assert np.array_equal(a, b)
                for a, b in zip(got["filters"][p], base["filters"][p]):
                    assert np.array_equal(a, b)
