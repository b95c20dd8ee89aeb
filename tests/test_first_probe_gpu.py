"""The first-probe pass against the oracle.

A forward-pass visit of a table with no selection bitmap, incoming edges
and at least 2^20 rows runs its first probe (in probe order) as a separate
streaming kernel and its other probes in the scan kernel.  Results, filter
words and the sector accounting must equal the oracle's bit for bit, and
equal the same transfer with the pass switched off, across the kernel's
paths: int64 keys (prefetched), int32 keys, a composite first key, the
first filter in shared memory or probed from L2, k fixed or read at run
time, ragged and whole last tiles, and the 2^20-row threshold.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

MIN_ROWS = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2307_15255_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _col_sectors(n, dtype):
    """32-byte sectors of rows 0..n-1 of a column: 8 rows per sector for int32, 4 for int64."""
    per = 8 if dtype == np.int32 else 4
    return -(-n // per)


def _run(w, oracle_lib, **kw):
    from _gpu import assert_same, run_gpu
    got = run_gpu(w, **kw)
    assert_same(got, oracle_lib.transfer(w), w)
    return got


def _first_edge_cols(w, v, got):
    """Key columns of the incoming edges of table v's forward visit."""
    order = sorted(range(w.n_tables), key=lambda t: (w.tables[t].n_rows, t))
    rank = {t: i for i, t in enumerate(order)}
    cols = []
    for e in w.edges:
        if e.t0 == v and rank[e.t1] < rank[v]:
            cols.append(e.c0)
        elif e.t1 == v and rank[e.t0] < rank[v]:
            cols.append(e.c1)
    return cols


def _check_first(w, got, v, expect):
    flag, sectors = got["first"][0][v]
    assert flag == (1 if expect else 0), (v, flag)
    if not expect:
        assert sectors == 0
        return
    # the pass read every sector of one incoming edge's key column(s)
    t = w.tables[v]
    options = {sum(_col_sectors(t.n_rows, t.cols[c].dtype.type) for c in cs) for cs in _first_edge_cols(w, v, got)}
    assert sectors in options, (sectors, options)
    # never in the backward pass
    assert got["first"][1][v] == (0, 0)


@pytest.mark.parametrize("kw", [
    dict(int64=True, composite=True, zipf=1.1, bits_per_key=16),  # int64, prefetched, smem filter
    dict(int64=False, bits_per_key=10),                             # int32 keys
    dict(int64=True, bits_per_key=10, k=7, block_bits=512),         # k read at run time, 512-bit blocks
])
def test_snowflake_fact_first_probe(oracle_lib, kw):
    w = W.snowflake(scale=0.25, **kw)  # fact 1.5M rows: 96 rows in its last tile
    assert w.tables[0].n_rows >= MIN_ROWS and w.tables[0].n_rows % 256 != 0
    got = _run(w, oracle_lib)
    _check_first(w, got, 0, True)
    for v in range(1, w.n_tables):  # smaller tables, or tables with a selection
        _check_first(w, got, v, False)


def test_composite_key_probed_first(oracle_lib):
    # both builders are sources (level 0); the composite-key one keeps 1% of
    # its rows, the other 50%, so the composite key is the first probe
    rng = np.random.default_rng(21)
    n = MIN_ROWS + 333
    nm, nd = 20_000, 3000
    m1 = rng.permutation(nm).astype(np.int64) * 5 + 1
    m2 = rng.integers(-4, 4, nm).astype(np.int64)
    d = rng.permutation(nd).astype(np.int64) - 1500
    M = W.Table("M", nm, [m1, m2], ["k1", "k2"], W.bitmap_from_bools(rng.random(nm) < 0.01))
    D = W.Table("D", nd, [d], ["id"], W.bitmap_from_bools(rng.random(nd) < 0.5))
    rm, rd = rng.integers(0, nm, n), rng.integers(0, nd, n)
    F = W.Table("F", n, [m1[rm], m2[rm], d[rd]], ["fk_m1", "fk_m2", "fk_d"], None)
    w = W.Workload("composite_first", [F, M, D], [W.Edge(0, (0, 1), 1, (0, 1)), W.Edge(0, (2,), 2, (0,))],
                   16, 4, 256, 0)
    got = _run(w, oracle_lib)
    _check_first(w, got, 0, True)
    assert got["first"][0][0][1] == 2 * _col_sectors(n, np.int64)


@pytest.mark.parametrize("smem", [0, 64 * 1024, 220 * 1024])
def test_filter_budgets(oracle_lib, smem):
    # 0: the first filter is read through L1/L2; larger budgets than the
    # first-probe kernel's own 46 KB cap are clamped to it
    w = W.snowflake(scale=0.25, int64=True, bits_per_key=16, sel=(0.1, 0.6, 0.3))
    got = _run(w, oracle_lib, launch=(256, smem, 0))
    _check_first(w, got, 0, True)


def test_large_first_filter_does_not_fit_shared_memory(oracle_lib):
    # the first filter (D2 keeps 60%: 30k keys at 16 bits/key, 60 KB) exceeds the 40 KB budget
    w = W.snowflake(scale=0.25, int64=True, bits_per_key=16, sel=(0.9, 0.6, 0.95))
    got = _run(w, oracle_lib)
    _check_first(w, got, 0, True)


def test_first_probe_off_gives_identical_results(oracle_lib):
    from _gpu import run_gpu
    w = W.snowflake(scale=0.25, int64=True, composite=True, zipf=1.1, bits_per_key=16)
    on = _run(w, oracle_lib, first_probe=True)
    off = _run(w, oracle_lib, first_probe=False)
    assert off["first"][0][0] == (0, 0)
    assert on["first"][0][0][0] == 1
    for p in range(2):
        for v in range(w.n_tables):
            assert np.array_equal(on["surv"][p][v], off["surv"][p][v])
            assert on["sectors"][p][v] == off["sectors"][p][v]
    # graph replays with the pass toggled in between
    from _gpu import collect, session_for
    s = session_for(w, graph=True)
    try:
        import paper_2307_15255_b300.pt as P
        for flag in (True, False, True):
            P.pt_set_first_probe(s.ctx, flag)
            s.run()
            c = collect(s, w)
            assert c["first"][0][0][0] == int(flag)
            for v in range(w.n_tables):
                assert np.array_equal(c["surv"][1][v], on["surv"][1][v])
    finally:
        s.close()


@pytest.mark.parametrize("kw", [
    dict(int64=True, composite=True, zipf=1.1, bits_per_key=16),
    dict(int64=False, bits_per_key=10, k=7, block_bits=512),
])
def test_early_scan_gives_identical_results(oracle_lib, kw):
    # the fact table's in-edges come from D2 and D3 (level 0) and M (level 2):
    # the first-probe pass takes one level-0 filter, the early scan the other,
    # and the visit's scan M's; the same survivors, filters and sectors as one
    # scan after M's build
    import paper_2307_15255_b300.pt as P
    from _gpu import assert_same, collect, folded, session_for
    w = W.snowflake(scale=0.25, **kw)
    want = oracle_lib.transfer(w)
    with session_for(w, graph=True) as s:
        P.pt_set_kernel_timing(s.ctx, True)
        for flag in (True, False, True):
            P.pt_set_early_scan(s.ctx, flag)
            s.run()
            got = collect(s, w)
            assert_same(got, want, w)
            kt = P.pt_get_kernel_times(s.ctx)
            assert kt["scan_launches"] == 2 * w.n_tables - len(folded(s, w)) + int(flag)
    # no early scan in the other probe orders (their order may interleave levels)
    with session_for(w, probe_order=1) as s:
        P.pt_set_early_scan(s.ctx, True)
        P.pt_set_kernel_timing(s.ctx, True)
        s.run()
        assert_same(collect(s, w), oracle_lib.transfer(w, probe_order=1), w)
        assert P.pt_get_kernel_times(s.ctx)["scan_launches"] == 2 * w.n_tables - len(folded(s, w))


def _two_tables(n_fact, seed, dtype=np.int64):
    """A fact table of n_fact rows whose one key joins a 5000-row dim with a 3% selection."""
    rng = np.random.default_rng(seed)
    nd = 5000
    d = rng.permutation(nd).astype(dtype) * 7 - 11000
    f = d[rng.integers(0, nd, n_fact)]
    D = W.Table("D", nd, [d], ["id"], W.bitmap_from_bools(rng.random(nd) < 0.03))
    F = W.Table("F", n_fact, [f], ["fk"], None)
    return W.Workload("two", [F, D], [W.Edge(0, (0,), 1, (0,))], 16, 4, 256, 0)


@pytest.mark.parametrize("n_fact,expect", [(MIN_ROWS - 1, False), (MIN_ROWS, True), (MIN_ROWS + 1, True),
                                           (MIN_ROWS + 255, True), (3 * MIN_ROWS + 31, True)])
def test_threshold_and_tails(oracle_lib, n_fact, expect):
    w = _two_tables(n_fact, 11 + n_fact % 97)
    got = _run(w, oracle_lib)
    _check_first(w, got, 0, expect)


def test_int32_tail_and_negative_keys(oracle_lib):
    w = _two_tables(MIN_ROWS + 77, 5, dtype=np.int32)
    got = _run(w, oracle_lib)
    _check_first(w, got, 0, True)


def test_kernel_times_split_probe_phase():
    import paper_2307_15255_b300.pt as P
    from _gpu import folded, session_for
    w = W.snowflake(scale=0.25, int64=True, bits_per_key=16)
    s = session_for(w, graph=True)
    try:
        P.pt_set_kernel_timing(s.ctx, True)
        for _ in range(3):
            s.run()
        kt = P.pt_get_kernel_times(s.ctx)
        assert kt["first_launches"] == 1  # the fact table's forward visit only
        # one per visit (no early scan by default), but for the fact table's backward
        # visit, which a transfer run folds into its forward scan and its insert
        assert kt["scan_launches"] == 2 * w.n_tables - len(folded(s, w)) == 2 * w.n_tables - 1
        assert kt["first_ms"] > 0 and kt["scan_ms"] > 0 and kt["build_ms"] > 0
        tot = P.pt_get_kernel_time(s.ctx)
        assert tot["scan_launches"] == kt["first_launches"] + kt["scan_launches"]
        assert abs(tot["scan_ms"] - (kt["first_ms"] + kt["scan_ms"])) < 1e-6
    finally:
        s.close()
