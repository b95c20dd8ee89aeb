"""The allocation-free entry point pt_visit_static against the planned path.

pt_visit_static serves callers that cannot allocate device memory
(engines that own all device memory through their own pool, services that
must not hit out-of-memory mid query, paths where an allocation's implicit
device synchronization is not acceptable).  It runs one visit with caller-owned inputs and outputs and keeps
its scratch in a fixed device array.  Here it redoes single visits of a
transfer that a planned context ran, from the same incoming filters, and
must reproduce that context's survivor bitmap, survivor count, outgoing
filter words and filter size bit for bit -- on several calls in a row,
since every call reuses the same scratch.

This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ran():
    from paper_2307_15255_b300 import build
    build.build()
    from _gpu import device_tables, edges_of
    from paper_2307_15255_b300.session import TransferSession
    w = W.snowflake(scale=0.05, int64=True, composite=True, bits_per_key=10)
    tables = device_tables(w)
    s = TransferSession(tables, edges_of(w), w.bits_per_key, w.k, w.block_bits, w.seed)
    s.run()
    torch.cuda.synchronize()
    yield w, tables, s
    s.close()


def _code(t):
    import paper_2307_15255_b300.pt as P
    return P.PT_I32 if t.dtype == torch.int32 else P.PT_I64


def _visit(w, tables, s, v, pass_=0):
    """Run table v's visit of pass 0 through pt_visit_static; return its outputs."""
    import paper_2307_15255_b300.pt as P
    o = P.pt_plan_graph([t.n_rows for t in w.tables], edges_of_tuples(w))
    probes, builds, keep = [], [], []
    n = w.tables[v].n_rows
    cols = tables[v][1]
    for e, edge in enumerate(w.edges):
        side = edge.c0 if edge.t0 == v else edge.c1
        key = [(cols[c].data_ptr(), _code(cols[c])) for c in side]
        if o["dst"][e] == v:  # incoming in the forward pass: probe the filter the planned run built
            f = s.filter(pass_, e)
            nb = torch.tensor([f.numel() * 32 // w.block_bits], dtype=torch.int64, device="cuda")
            keep += [f, nb]
            probes.append((key, f.data_ptr(), nb.data_ptr()))
        elif o["src"][e] == v:  # outgoing: build into a caller-owned buffer
            other = edge.t1 if edge.t0 == v else edge.t0
            m = min(n, w.tables[other].n_rows)
            cap = max(1, -(-m * w.bits_per_key // w.block_bits))
            buf = torch.full((cap * w.block_bits // 32,), -1, dtype=torch.int32, device="cuda")
            nbo = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            keep += [buf, nbo]
            builds.append((key, buf.data_ptr(), cap, w.tables[other].n_rows, nbo.data_ptr(), e, buf, nbo))
    sel = tables[v][2]
    out_bits = torch.full((max((n + 31) // 32, 1),), -1, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    P.pt_visit_static(n, None if sel is None else sel.data_ptr(), probes,
                      [b[:5] for b in builds], out_bits.data_ptr(), count.data_ptr(),
                      w.bits_per_key, w.k, w.block_bits, w.seed, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    res = {"bits": out_bits[: (n + 31) // 32].cpu().numpy().view(np.uint32), "count": int(count.item()),
           "filters": {}}
    for (_, _, _, _, _, e, buf, nbo) in builds:
        nb = int(nbo.item())
        res["filters"][e] = (nb, buf[: nb * w.block_bits // 32].cpu().numpy().view(np.uint32))
    return res


def edges_of_tuples(w):
    return [(e.t0, e.c0, e.t1, e.c1) for e in w.edges]


def _planned(s, w, v, pass_=0):
    bm, c = s.survivors(v, pass_)
    return bm.cpu().numpy().view(np.uint32), c


def test_static_visits_match_planned_context(ran):
    w, tables, s = ran
    M, F = 1, 0
    # M: one incoming filter, one outgoing composite-key filter; F: three incoming filters;
    # then M again, so the second M call runs on scratch the F call left behind
    for v in (M, F, M):
        got = _visit(w, tables, s, v)
        bits, cnt = _planned(s, w, v)
        assert np.array_equal(got["bits"], bits), v
        assert got["count"] == cnt, v
        for e, (nb, words) in got["filters"].items():
            want = s.filter(0, e).cpu().numpy().view(np.uint32)
            assert nb == len(want) * 32 // w.block_bits, e
            assert np.array_equal(words, want), e


@pytest.mark.parametrize("n_dims", [5, 8])
def test_static_visit_with_many_incoming_filters(n_dims):
    # five and eight incoming filters need more queue space per warp, so the
    # entry point runs fewer warps per CTA to stay within its shared memory;
    # the survivors must not change, on two calls in a row
    from _gpu import device_tables, edges_of
    from paper_2307_15255_b300.session import TransferSession
    rng = np.random.default_rng(40 + n_dims)
    nv = 200_003
    dims, cols, edges = [], [], []
    for j in range(n_dims):
        nd = 500 + 300 * j
        d = rng.permutation(nd).astype(np.int64) * 3 - 7
        dims.append(W.Table(f"D{j}", nd, [d], ["id"], W.bitmap_from_bools(rng.random(nd) < 0.8)))
        cols.append(d[rng.integers(0, nd, nv)])
        edges.append(W.Edge(0, (j,), j + 1, (0,)))
    V = W.Table("V", nv, cols, [f"k{j}" for j in range(n_dims)], None)
    w = W.Workload("many_filters", [V] + dims, edges, 16, 4, 256, 0)
    tables = device_tables(w)
    s = TransferSession(tables, edges_of(w), w.bits_per_key, w.k, w.block_bits, w.seed)
    try:
        s.run()
        torch.cuda.synchronize()
        bits, cnt = _planned(s, w, 0)
        assert cnt > 0
        for _ in range(2):
            got = _visit(w, tables, s, 0)
            assert np.array_equal(got["bits"], bits)
            assert got["count"] == cnt
    finally:
        s.close()


def test_static_visit_rejects_too_many_rows():
    import paper_2307_15255_b300.pt as P
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PtError) as ei:
        P.pt_visit_static(P.PT_STATIC_MAX_ROWS + 1, None, [], [], x.data_ptr(), None)
    assert ei.value.status == P.PT_ERR_INVALID
    assert "limit" in str(ei.value)
