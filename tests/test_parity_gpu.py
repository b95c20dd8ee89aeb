"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU
oracle: survivor bitmaps and counts of every table after each pass, the
words and size of every filter built in each pass, and the key-sector
accounting of every visit."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2307_15255_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _check(w, oracle_lib, **kw):
    from _gpu import assert_same, run_gpu
    got = run_gpu(w, **kw)
    want = oracle_lib.transfer(w)
    assert_same(got, want, w)
    return got


def test_chain3_full_size(oracle_lib):
    _check(W.chain3(), oracle_lib)


@pytest.mark.parametrize("bpk,k,B", [(10, 4, 256), (8, 4, 256), (16, 4, 512), (10, 7, 512), (3, 1, 256),
                                     (64, 16, 256)])
def test_snowflake_small_filter_params(oracle_lib, bpk, k, B):
    _check(W.snowflake(scale=0.02, bits_per_key=bpk, k=k, block_bits=B), oracle_lib)


def test_snowflake_int64_composite_zipf_small(oracle_lib):
    _check(W.snowflake(scale=0.02, int64=True, composite=True, zipf=1.1, bits_per_key=16), oracle_lib)


def test_cyclic_small(oracle_lib):
    _check(W.cyclic5(scale=0.005), oracle_lib)


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("make", [
    # fact table of 1.2M rows: its first probe runs as a pass of its own
    lambda: W.snowflake(scale=0.2, int64=True, composite=True, zipf=1.1, bits_per_key=16),
    lambda: W.cyclic5(scale=0.06),
], ids=["snowflake_x0.2", "cyclic5_x0.06"])
def test_probe_orders(oracle_lib, order, make):
    # level-then-LIP, LIP, and edge-id order: the same survivors and filters,
    # and each order's own sector counts
    from _gpu import assert_same, run_gpu
    w = make()
    got = run_gpu(w, probe_order=order)
    assert_same(got, oracle_lib.transfer(w, probe_order=order), w)


def _one_way(w, idx):
    import dataclasses
    return dataclasses.replace(w, edges=[dataclasses.replace(e, flags=1) if i in idx else e
                                         for i, e in enumerate(w.edges)])


@pytest.mark.parametrize("make", [
    lambda: _one_way(W.chain3(), {0}),
    lambda: _one_way(W.chain3(), {0, 1}),
    # fact table of 1.2M rows (first-probe pass); one edge one-way each way round
    lambda: _one_way(W.snowflake(scale=0.2, int64=True, composite=True, zipf=1.1, bits_per_key=16), {1, 4}),
    lambda: _one_way(W.cyclic5(scale=0.02), {0, 3}),
], ids=["chain3_e0", "chain3_both", "snowflake_x0.2", "cyclic5"])
def test_one_way_edges(oracle_lib, make):
    # left-outer-join edges (Section 3.4): each active in one pass only
    _check(make(), oracle_lib)


def test_one_way_edges_random_tiny(oracle_lib):
    from _gpu import assert_same, run_gpu
    rng = np.random.default_rng(17)
    for i in range(16):
        w = W.random_tiny(1300 + i, 3 + i % 5, max_rows=200, acyclic=(i % 2 == 0), composite_prob=0.3)
        w = _one_way(w, {j for j in range(len(w.edges)) if rng.random() < 0.5})
        assert_same(run_gpu(w), oracle_lib.transfer(w), w)


def test_seeded_hash(oracle_lib):
    w = W.chain3(scale=0.3)
    w.seed = 0xDEADBEEF12345678
    _check(w, oracle_lib)


@pytest.mark.parametrize("launch", [(128, 0, 0), (256, 16 * 1024, 0), (64, 0, 2), (256, 180 * 1024, 1),
                                    (256, 4 * 1024, 3)])
def test_launch_shapes_give_identical_results(oracle_lib, launch):
    # smem budget 0 forces every probe through L1/L2; small budgets split filters between the two
    _check(W.snowflake(scale=0.03, bits_per_key=16), oracle_lib, launch=launch)


@pytest.mark.parametrize("cluster,smem", [(1, 8 * 1024), (2, 8 * 1024), (4, 8 * 1024), (4, 2 * 1024),
                                          (4, 96 * 1024)])
def test_cluster_spread_filters(oracle_lib, cluster, smem):
    # small shared-memory budgets push the filters into the cluster-spread (or global) path
    _check(W.snowflake(scale=0.03, int64=True, composite=True, bits_per_key=16), oracle_lib,
           launch=(256, smem, 0), cluster=cluster)


def test_random_tiny_graphs(oracle_lib):
    for s in range(60):
        w = W.random_tiny(7000 + s, 2 + s % 5, max_rows=200, domain=40, acyclic=(s % 3 != 0),
                          composite_prob=0.3)
        _check(w, oracle_lib)


def test_edge_cases_sizes(oracle_lib):
    rng = np.random.default_rng(1)
    for n_small, n_big in [(0, 5), (1, 1), (31, 33), (32, 64), (1, 1000), (0, 0), (33, 4097)]:
        a = rng.integers(0, 50, n_small).astype(np.int32)
        b = rng.integers(0, 50, n_big).astype(np.int64)
        c = rng.integers(0, 50, n_big + 3).astype(np.int32)
        A = W.Table("A", n_small, [a], ["k"], W.bitmap_from_bools(rng.random(n_small) < 0.5))
        Bt = W.Table("B", n_big, [b, b.copy()], ["k", "j"], None)
        Ct = W.Table("C", n_big + 3, [c], ["j"], W.bitmap_from_bools(rng.random(n_big + 3) < 0.7))
        lone = W.Table("L", 7, [np.arange(7, dtype=np.int32)], ["x"], None)  # no edges at all
        w = W.Workload("edge", [A, Bt, Ct, lone], [W.Edge(0, (0,), 1, (0,)), W.Edge(1, (1,), 2, (0,))])
        _check(w, oracle_lib)


def test_empty_and_full_selections(oracle_lib):
    w = W.chain3(scale=0.1)
    w.tables[0].sel = np.zeros_like(w.tables[0].sel)
    _check(w, oracle_lib)
    w = W.chain3(scale=0.1)
    w.tables[2].sel = W.bitmap_from_bools(np.ones(w.tables[2].n_rows, bool))
    _check(w, oracle_lib)


def test_mixed_dense_and_sparse_input_runs(oracle_lib):
    # the fact table's selection alternates all-ones runs (dense sub-rounds of
    # the scan) with sparse stretches, so queued rows and dense rows meet in
    # the same stages; survivors and sector counts must still equal the oracle's
    rng = np.random.default_rng(77)
    n = 400_000 + 13
    dims = []
    for nd, frac in ((3000, 0.2), (50_000, 0.5), (700, 0.9)):
        d = rng.permutation(nd).astype(np.int64) * 3 + 5
        dims.append(W.Table(f"D{nd}", nd, [d], ["id"], W.bitmap_from_bools(rng.random(nd) < frac)))
    cols = [d.cols[0][rng.integers(0, d.n_rows, n)] for d in dims]
    keep = np.zeros(n, bool)
    for start in range(0, n, 9000):
        if (start // 9000) % 2 == 0:
            keep[start:start + 5000] = True                       # runs of whole words
        else:
            keep[start:start + 9000] = rng.random(min(9000, n - start)) < 0.05
    F = W.Table("F", n, cols, ["a", "b", "c"], W.bitmap_from_bools(keep))
    w = W.Workload("mixed", [F] + dims, [W.Edge(0, (i,), i + 1, (0,)) for i in range(3)], 16, 4, 256, 0)
    _check(w, oracle_lib)


def test_graph_mode_host_columns_and_repeat(oracle_lib):
    from _gpu import assert_same, collect, session_for
    w = W.snowflake(scale=0.02, int64=True, composite=True, bits_per_key=10)
    want = oracle_lib.transfer(w)
    import paper_2307_15255_b300.pt as P
    for kw in ({"graph": True}, {"host": True, "pin": True}, {"host": True}):
        s = session_for(w, **kw)
        try:
            for i in range(3):  # replays and reruns give the same bits, on 3 streams or 1
                P.pt_set_streams(s.ctx, 1 if i == 1 else 3)
                s.run()
                assert_same(collect(s, w), want, w)
        finally:
            s.close()


def test_update_table_then_rerun(oracle_lib):
    from _gpu import assert_same, collect, device_tables, session_for
    w = W.chain3(scale=0.2)
    s = session_for(w, graph=True)
    try:
        s.run()
        w2 = W.chain3(scale=0.2, seed=99)
        tabs = device_tables(w2)
        for v, (n, cols, sel) in enumerate(tabs):
            s.update(v, cols, sel)
        s.run()
        assert_same(collect(s, w2), oracle_lib.transfer(w2), w2)
    finally:
        s.close()


def test_state_errors():
    import paper_2307_15255_b300.pt as P
    ctx = P.pt_create()
    try:
        x = torch.arange(10, dtype=torch.int32, device="cuda")
        P.pt_register_table(ctx, 10, [(x.data_ptr(), P.PT_I32, P.PT_MEM_DEVICE)])
        with pytest.raises(P.PtError) as ei:
            P.pt_run_forward(ctx)
        assert ei.value.status == P.PT_ERR_STATE
        P.pt_set_join_graph(ctx, [])
        P.pt_plan(ctx, 1)
        with pytest.raises(P.PtError) as ei:
            P.pt_run_backward(ctx)
        assert ei.value.status == P.PT_ERR_STATE
        with pytest.raises(P.PtError) as ei:
            P.pt_get_survivors(ctx, 0, None)
        assert ei.value.status == P.PT_ERR_STATE
        with pytest.raises(P.PtError) as ei:
            P.pt_get_pass_survivors(ctx, 0, 3, None)
        assert ei.value.status == P.PT_ERR_INVALID
        P.pt_run_forward(ctx)
        assert P.pt_get_survivors(ctx, 0, None) == 10
    finally:
        P.pt_destroy(ctx)


def test_misaligned_device_column_is_rejected():
    import paper_2307_15255_b300.pt as P
    ctx = P.pt_create()
    try:
        x = torch.arange(16, dtype=torch.int32, device="cuda")
        with pytest.raises(P.PtError) as ei:
            P.pt_register_table(ctx, 10, [(x.data_ptr() + 4, P.PT_I32, P.PT_MEM_DEVICE)])
        assert ei.value.status == P.PT_ERR_INVALID
    finally:
        P.pt_destroy(ctx)


@pytest.mark.slow
@pytest.mark.parametrize("cfg", ["snowflake", "snowflake_x10_b8", "snowflake_x10_b16", "cyclic5"])
def test_full_size_configs(oracle_lib, cfg):
    """The full workloads, in the launch shape the benchmark uses, bit for bit."""
    if cfg == "snowflake":
        w = W.snowflake()
    elif cfg.startswith("snowflake_x10"):
        bpk = 8 if cfg.endswith("b8") else 16
        w = W.snowflake(scale=10, int64=True, composite=True, zipf=1.1, bits_per_key=bpk)
    else:
        w = W.cyclic5()
    _check(w, oracle_lib)


def test_kernel_timing_direct_and_graph():
    """Scan kernels are bracketed by CUDA events in both launch modes."""
    import paper_2307_15255_b300.pt as P
    from _gpu import folded, session_for
    w = W.snowflake(scale=0.02)
    s = session_for(w)
    try:
        P.pt_set_kernel_timing(s.ctx, True)
        s.run()
        kt = P.pt_get_kernel_time(s.ctx)
        skip = folded(s, w)
        assert skip  # the fact table's backward visit
        assert kt["scan_launches"] == 2 * w.n_tables - len(skip) and kt["scan_ms"] > 0
        P.pt_set_graph_mode(s.ctx, True)
        P.pt_set_kernel_timing(s.ctx, True)
        n0 = P.pt_get_launch_count(s.ctx)
        for _ in range(3):
            s.run()
        kt = P.pt_get_kernel_time(s.ctx)  # the last replay
        assert kt["scan_launches"] == 2 * w.n_tables - len(skip) and kt["scan_ms"] > 0
        assert P.pt_get_launch_count(s.ctx) - n0 == 3 * (P.pt_get_launch_count(s.ctx) - n0) // 3 > 0
        # the same events one launch at a time: one scan per (pass, table), times adding up
        lt = P.pt_get_launch_times(s.ctx)
        scans = [(x["pass"], x["table"]) for x in lt if x["kind"] == "scan"]
        assert sorted(scans) == sorted((p, v) for p in range(2) for v in range(w.n_tables)
                                       if not (p == 1 and v in skip))
        assert abs(sum(x["ms"] for x in lt if x["kind"] == "scan") - kt["scan_ms"]) < 1e-3
        assert all(x["ms"] > 0 and x["start_ms"] >= 0 for x in lt)
    finally:
        s.close()


def test_autotuner_keeps_results_exact(oracle_lib, tmp_path):
    from _gpu import assert_same, collect, session_for
    from paper_2307_15255_b300 import autotune
    w = W.snowflake(scale=0.02, bits_per_key=16)
    s = session_for(w)
    try:
        cache = str(tmp_path / "tune.json")
        r = autotune.tune(s, candidates=[(256, 40 * 1024, 0), (128, 0, 0)], runs=2, cache_path=cache)
        assert not r["cached"] and len(r["trials"]) == 2
        r2 = autotune.tune(s, cache_path=cache)
        assert r2["cached"] and tuple(r2["launch"]) == tuple(r["launch"])
        s.run()
        assert_same(collect(s, w), oracle_lib.transfer(w), w)
    finally:
        s.close()


def test_injected_allocation_failure_reports_oom(monkeypatch):
    import paper_2307_15255_b300.pt as P
    ctx = P.pt_create()
    try:
        x = torch.arange(64, dtype=torch.int32, device="cuda")
        P.pt_register_table(ctx, 64, [(x.data_ptr(), P.PT_I32, P.PT_MEM_DEVICE)])
        P.pt_register_table(ctx, 64, [(x.data_ptr(), P.PT_I32, P.PT_MEM_DEVICE)])
        P.pt_set_join_graph(ctx, [(0, (0,), 1, (0,))])
        monkeypatch.setenv("PT_INJECT_OOM", "1")
        with pytest.raises(P.PtError) as ei:
            P.pt_plan(ctx, 2)
        assert ei.value.status == P.PT_ERR_OOM
        monkeypatch.delenv("PT_INJECT_OOM")
        P.pt_plan(ctx, 2)  # the context is still usable
        P.pt_run_transfer(ctx)
        assert P.pt_get_survivors(ctx, 1, None) == 64
    finally:
        P.pt_destroy(ctx)


def test_server_arena_too_large_reports_oom():
    import paper_2307_15255_b300.pt as P
    with pytest.raises(P.PtError) as ei:
        P.pt_server_create(arena_bytes=1 << 52)
    assert ei.value.status == P.PT_ERR_OOM


def test_filter_tuner_choice_is_exact(oracle_lib):
    # the tuner times whole transfers under each (bits per key, block bits, k);
    # the configuration it returns gives the oracle's results for that configuration
    import dataclasses

    from _gpu import assert_same, device_tables, edges_of, run_gpu
    from paper_2307_15255_b300 import autotune
    w = W.snowflake(scale=0.05, int64=True, composite=True, zipf=1.1, bits_per_key=16)
    r = autotune.tune_filter(device_tables(w), edges_of(w), w.seed, candidates=[(16, 256, 4), (8, 512, 4), (12, 256, 3)],
                             runs=2)
    assert len(r["trials"]) == 3 and all(t["ms"] > 0 for t in r["trials"])
    assert r["ms"] == min(t["ms"] for t in r["trials"])
    wt = dataclasses.replace(w, bits_per_key=r["bits_per_key"], block_bits=r["block_bits"], k=r["k"])
    assert_same(run_gpu(wt), oracle_lib.transfer(wt), wt)
    # and every trial's survivor total is the oracle's for its configuration
    for t in r["trials"]:
        wc = dataclasses.replace(w, bits_per_key=t["bits_per_key"], block_bits=t["block_bits"], k=t["k"])
        assert t["survivors"] == sum(oracle_lib.transfer(wc)["count"][1])


@pytest.mark.parametrize("make", [
    W.chain3,
    lambda: W.snowflake(scale=0.05, int64=True, composite=True, zipf=1.1, bits_per_key=16),
], ids=["chain3", "snowflake_x0.05"])
def test_join_count_on_survivors(oracle_lib, make):
    # the join phase on the reduced tables equals the oracle's count on the
    # unreduced selections (the snowflake is cyclic: rejected)
    from _gpu import session_for
    w = make()
    with session_for(w) as s:
        s.run()
        try:
            want = oracle_lib.join_count(w)
        except ValueError:
            from paper_2307_15255_b300 import pt as P
            with pytest.raises(P.PtError) as ei:
                s.join_count()
            assert ei.value.status == P.PT_ERR_UNSUPPORTED
            return
        assert s.join_count() == want


def test_join_count_random_trees(oracle_lib):
    from _gpu import session_for
    for seed in range(12):
        w = W.random_tiny(2200 + seed, 2 + seed % 5, max_rows=300, domain=8, acyclic=True, composite_prob=0.3)
        with session_for(w) as s:
            s.run()
            assert s.join_count() == oracle_lib.join_count(w), seed


def test_join_count_star_forest_and_one_way(oracle_lib):
    import dataclasses

    from _gpu import session_for
    from paper_2307_15255_b300 import pt as P
    # a star with a selective predicate on each dimension, plus a disconnected
    # pair of tables: a forest, whose count is the product of its trees'
    w = W.star(scale=0.003, bits_per_key=12)
    rng = np.random.default_rng(9)
    tabs = [w.tables[0]] + [dataclasses.replace(t, sel=W.bitmap_from_rows(t.n_rows, rng.choice(
        t.n_rows, size=max(1, t.n_rows // 5), replace=False))) for t in w.tables[1:]]
    extra = W.random_tiny(31, 2, max_rows=50, domain=5)
    k = len(tabs)
    w2 = W.Workload("forest", tabs + extra.tables,
                    w.edges + [dataclasses.replace(e, t0=e.t0 + k, t1=e.t1 + k) for e in extra.edges])
    with session_for(w2) as s:
        s.run()
        assert s.join_count() == oracle_lib.join_count(w2)
    w3 = dataclasses.replace(w2, edges=[dataclasses.replace(w2.edges[0], flags=1)] + w2.edges[1:])
    with session_for(w3) as s:
        s.run()
        with pytest.raises(P.PtError) as ei:
            s.join_count()
        assert ei.value.status == P.PT_ERR_UNSUPPORTED


@pytest.mark.parametrize("bpk,k,B", [(16, 4, 256), (10, 7, 512), (12, 3, 256)])
def test_many_rows_into_a_tiny_filter(oracle_lib, bpk, k, B):
    # 300k fact rows whose foreign key takes one of 12 values: the fact table's
    # backward filter for the 12-row dimension has one or two blocks and is
    # built from every surviving fact row (the insert builds a filter that
    # small in each CTA's shared memory first, then ORs it into the filter)
    rng = np.random.default_rng(21 + k)
    nd, nf = 12, 300_000
    d = np.arange(nd, dtype=np.int64) * 3 + 1
    D = W.Table("D", nd, [d], ["id"], W.bitmap_from_rows(nd, [0, 2, 3, 5, 7, 11]))
    F = W.Table("F", nf, [d[rng.integers(0, nd, nf)]], ["fk"], None)
    w = W.Workload("tiny", [F, D], [W.Edge(0, (0,), 1, (0,))], bpk, k, B, 0)
    _check(w, oracle_lib)


@pytest.mark.parametrize("bpk,k,B", [(16, 4, 256), (12, 3, 256), (10, 7, 512)])
def test_more_building_rows_than_probe_rows_skewed(oracle_lib, bpk, k, B):
    # 400k fact rows with Zipf(1.1) foreign keys into a 20k-row dimension: the
    # fact table's backward build has 20 times more rows than the dimension,
    # so the insert reads each key's words and skips atomics that would set
    # nothing new (the filter is far larger than the shared-memory copies)
    rng = np.random.default_rng(31 + k)
    nd, nf = 20_000, 400_000
    d = rng.permutation(nd).astype(np.int64) * 5 - 7
    D = W.Table("D", nd, [d], ["id"], W.bitmap_from_bools(rng.random(nd) < 0.6))
    F = W.Table("F", nf, [d[W.fk_rows(rng, nd, nf, 1.1)]], ["fk"], None)
    w = W.Workload("skew", [F, D], [W.Edge(0, (0,), 1, (0,))], bpk, k, B, 0)
    _check(w, oracle_lib)


@pytest.mark.parametrize("graph", [False, True])
def test_transfer_and_separate_passes_alternate(oracle_lib, graph):
    # a transfer run folds the fact table's pass-through backward visit (its
    # forward scan zeroes that visit's filters of the previous run, its insert
    # counts the build sectors); separate forward and backward runs launch the
    # pass-through kernel instead.  Any sequence gives the same survivors,
    # filters and sectors.
    from _gpu import assert_same, collect, folded, session_for
    w = W.snowflake(scale=0.05, bits_per_key=12)
    want = oracle_lib.transfer(w)
    with session_for(w, graph=graph) as s:
        for mode in ("transfer", "split", "transfer", "backward twice", "transfer", "transfer"):
            if mode == "transfer":
                s.run()
            else:
                s.forward()
                s.backward()
                if mode == "backward twice":
                    s.backward()
            assert_same(collect(s, w), want, w)
        assert folded(s, w)


@pytest.mark.parametrize("streams", [1, 2, 3])
def test_random_graphs_with_one_way_edges_on_few_streams(oracle_lib, streams):
    # a transfer run chains each backward visit onto its own forward visit and
    # its backward builders only; one-way edges build in one pass, so some
    # visits have builders in one pass and not the other
    import dataclasses
    from _gpu import assert_same, collect, session_for
    from paper_2307_15255_b300 import pt as P
    rng = np.random.default_rng(77 + streams)
    for seed in range(10):
        w = W.random_tiny(5200 + 10 * streams + seed, 3 + seed % 4, max_rows=3000, domain=40,
                          acyclic=seed % 2 == 0, composite_prob=0.25)
        w = dataclasses.replace(w, edges=[dataclasses.replace(e, flags=int(rng.random() < 0.3)) for e in w.edges])
        want = oracle_lib.transfer(w)
        with session_for(w, graph=seed % 2 == 1) as s:
            P.pt_set_streams(s.ctx, streams)
            for _ in range(2):
                s.run()
            assert_same(collect(s, w), want, w)


@pytest.mark.parametrize("pdl,streams,graph", [(False, 3, False), (False, 1, True), (True, 1, False), (True, 3, True),
                                               (True, 2, True), (True, 2, False)])
def test_dependent_launches_and_streams(oracle_lib, pdl, streams, graph):
    # programmatic dependent launches on or off, every visit on one stream or
    # spread over two or three (visits whose planned streams fold onto one then
    # share it: the waits between them are left to stream order), direct
    # launches or a captured graph: the same results
    from _gpu import assert_same, collect, session_for
    from paper_2307_15255_b300 import pt as P
    w = W.snowflake(scale=0.25, int64=True, composite=True, zipf=1.1, bits_per_key=16)
    want = oracle_lib.transfer(w)
    with session_for(w, graph=graph) as s:
        P.pt_set_dependent_launch(s.ctx, pdl)
        P.pt_set_streams(s.ctx, streams)
        for _ in range(2):
            s.run()
        assert_same(collect(s, w), want, w)
