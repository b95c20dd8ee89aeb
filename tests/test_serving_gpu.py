"""Served queries give the transfer's exact results: every query of a mix,
run in batches, one at a time, or while memory admission holds queries
back, has the same final survivor bitmaps as the oracle (and therefore as
a planned context, which the parity tests pin to the oracle)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def star():
    from paper_2307_15255_b300 import build
    build.build()
    w = W.star(scale=0.002, bits_per_key=16)
    qs = W.serving_queries(w, 24, rate_qps=0, seed=7, sel_lo=0.01, sel_hi=0.5)
    return w, qs


def query_workload(w, q):
    tables = []
    for j, t in enumerate(q.inst_table):
        base = w.tables[t]
        tables.append(W.Table(f"i{j}", base.n_rows, base.cols, base.col_names, q.sel[j]))
    return W.Workload("q", tables, q.edges, w.bits_per_key, w.k, w.block_bits, w.seed)


def run_server(w, qs, max_batch, max_inflight, arena, device_sel=False):
    import paper_2307_15255_b300.pt as P
    srv = P.pt_server_create(w.bits_per_key, w.k, w.block_bits, w.seed, arena, max_batch, max_inflight)
    keep = []
    try:
        for t in w.tables:
            cols = [torch.from_numpy(c).cuda() for c in t.cols]
            keep += cols
            P.pt_server_register_table(srv, t.n_rows, [(c.data_ptr(), P.PT_I64, P.PT_MEM_DEVICE) for c in cols])
        P.pt_server_start(srv)
        tickets = []
        for q in qs:
            if device_sel:
                sels = [None if s is None else torch.from_numpy(np.ascontiguousarray(s).view(np.int32)).cuda()
                        for s in q.sel]
                ptrs = [None if s is None else s.data_ptr() for s in sels]
                mem = P.PT_MEM_DEVICE
            else:
                sels = [None if s is None else np.ascontiguousarray(s, dtype=np.uint32) for s in q.sel]
                ptrs = [None if s is None else s.ctypes.data for s in sels]
                mem = P.PT_MEM_HOST
            keep += [s for s in sels if s is not None]
            tickets.append(P.pt_server_submit(srv, q.inst_table, ptrs, [(e.t0, e.c0, e.t1, e.c1) for e in q.edges],
                                              mem))
        out = []
        for q, t in zip(qs, tickets):
            assert P.pt_server_wait(srv, t) == P.PT_OK
            res = []
            for j, tb in enumerate(q.inst_table):
                n = w.tables[tb].n_rows
                bm = np.zeros(max((n + 31) // 32, 1), np.uint32)
                c = P.pt_server_survivors(srv, t, j, bm.ctypes.data)
                res.append((bm[: (n + 31) // 32], c))
            P.pt_server_release(srv, t)
            out.append(res)
        stats = P.pt_server_stats(srv)
        assert stats["completed"] == len(qs)
        return out
    finally:
        P.pt_server_destroy(srv)


@pytest.mark.parametrize("max_batch,max_inflight,arena,device_sel", [(8, 2, 1 << 30, False), (1, 1, 1 << 30, False),
                                                                    (4, 2, 60 << 20, False), (16, 3, 1 << 30, True)])
def test_served_results_equal_oracle(star, oracle_lib, max_batch, max_inflight, arena, device_sel):
    w, qs = star
    got = run_server(w, qs, max_batch, max_inflight, arena, device_sel)
    for q, res in zip(qs, got):
        want = oracle_lib.transfer(query_workload(w, q))
        for j, (bm, c) in enumerate(res):
            assert np.array_equal(bm, want["surv"][1][j]), (q.inst_table, j)
            assert c == want["count"][1][j]


def test_server_rejects_bad_queries(star):
    import paper_2307_15255_b300.pt as P
    w, qs = star
    srv = P.pt_server_create(w.bits_per_key, w.k, w.block_bits, w.seed, 1 << 26, 2, 1)
    try:
        x = torch.arange(64, dtype=torch.int64, device="cuda")
        P.pt_server_register_table(srv, 64, [(x.data_ptr(), P.PT_I64, P.PT_MEM_DEVICE)])
        with pytest.raises(P.PtError) as ei:
            P.pt_server_submit(srv, [0, 0], [None, None], [(0, (0,), 1, (0,))])
        assert ei.value.status == P.PT_ERR_STATE  # not started
        P.pt_server_start(srv)
        with pytest.raises(P.PtError) as ei:
            P.pt_server_submit(srv, [0, 3], [None, None], [(0, (0,), 1, (0,))])
        assert ei.value.status == P.PT_ERR_INVALID
        with pytest.raises(P.PtError) as ei:
            P.pt_server_submit(srv, [0] * 7, [None] * 7, [])
        assert ei.value.status == P.PT_ERR_INVALID
        t = P.pt_server_submit(srv, [0, 0], [None, None], [(0, (0,), 1, (0,))])
        assert P.pt_server_wait(srv, t) == P.PT_OK
        assert P.pt_server_survivors(srv, t, 1, None) == 64
        P.pt_server_release(srv, t)
        with pytest.raises(P.PtError):
            P.pt_server_poll(srv, t)
    finally:
        P.pt_server_destroy(srv)


@pytest.mark.slow
def test_served_full_size_star_samples(oracle_lib):
    """The serving workload at full size (fact 100M rows): a few queries of a
    batch, checked against the oracle bit for bit."""
    w = W.star(scale=1.0, bits_per_key=16)
    pool = W.selection_pool(w, size=8)
    qs = W.serving_queries(w, 6, rate_qps=0, pool=pool)
    got = run_server(w, qs, 8, 2, 48 << 30, device_sel=True)
    for q, res in list(zip(qs, got))[:3]:
        want = oracle_lib.transfer(query_workload(w, q))
        for j, (bm, c) in enumerate(res):
            assert np.array_equal(bm, want["surv"][1][j]), (q.inst_table, j)
            assert c == want["count"][1][j]


def test_cyclic_graph_through_batched_launches(oracle_lib):
    # the cyclic 5-table graph (a triangle plus two pendant tables), several
    # queries with their own selections in one batch: every visit of a DAG
    # level of every query runs in the same scan, size/clear and insert launches
    from paper_2307_15255_b300 import build
    build.build()
    w = W.cyclic5(scale=0.05)
    rng = np.random.default_rng(5)
    qs = []
    for i in range(3):
        sel = [t.sel for t in w.tables]
        if i > 0:  # other 5% selections on T2 and E
            for v in (2, 4):
                n = w.tables[v].n_rows
                sel[v] = W.bitmap_from_rows(n, rng.choice(n, size=n // 20, replace=False))
        qs.append(W.Query(list(range(w.n_tables)), sel, list(w.edges)))
    got = run_server(w, qs, 8, 2, 1 << 30)
    for q, res in zip(qs, got):
        want = oracle_lib.transfer(query_workload(w, q))
        for j, (bm, c) in enumerate(res):
            assert np.array_equal(bm, want["surv"][1][j]), j
            assert c == want["count"][1][j]
