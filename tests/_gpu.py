"""Run a workloads.Workload through the CUDA library (via the C ABI) and
collect the same outputs the oracle produces."""
import numpy as np
import torch

from paper_2307_15255_b300.session import TransferSession


def device_tables(w, host=False, pin=False):
    tables = []
    for t in w.tables:
        cols = []
        for c in t.cols:
            x = torch.from_numpy(np.ascontiguousarray(c))
            cols.append(x.pin_memory() if (host and pin) else (x if host else x.cuda()))
        sel = None
        if t.sel is not None:
            s = torch.from_numpy(np.ascontiguousarray(t.sel).view(np.int32))
            sel = s.pin_memory() if (host and pin) else (s if host else s.cuda())
        tables.append((t.n_rows, cols, sel))
    return tables


def edges_of(w):
    return [(e.t0, tuple(e.c0), e.t1, tuple(e.c1), e.flags) for e in w.edges]


def session_for(w, launch=None, graph=False, host=False, pin=False, cluster=None, first_probe=None,
                probe_order=None, schedule=0):
    return TransferSession(device_tables(w, host, pin), edges_of(w), w.bits_per_key, w.k, w.block_bits,
                           w.seed, launch=launch, graph=graph, cluster=cluster, first_probe=first_probe,
                           probe_order=probe_order, schedule=schedule)


def collect(s, w):
    nt, ne = w.n_tables, len(w.edges)
    out = {"surv": [[None] * nt for _ in range(2)], "count": [[0] * nt for _ in range(2)],
           "filters": [[None] * ne for _ in range(2)], "nblocks": [[0] * ne for _ in range(2)],
           "sectors": [[None] * nt for _ in range(2)]}
    for p in range(2):
        for v in range(nt):
            bm, c = s.survivors(v, p)
            out["surv"][p][v] = bm.cpu().numpy().view(np.uint32)
            out["count"][p][v] = c
            st = s.stats(p, v)
            out["sectors"][p][v] = (st["probe_sectors"], st["build_sectors"])
            out.setdefault("first", [[None] * nt for _ in range(2)])[p][v] = (st["first_probe"],
                                                                              st["first_probe_sectors"])
        for e in range(ne):
            f = s.filter(p, e).cpu().numpy().view(np.uint32)
            out["filters"][p][e] = f
            out["nblocks"][p][e] = len(f) * 32 // w.block_bits
    return out


def folded(s, w):
    """Tables whose backward visit passes its forward survivors through (no
    incoming filter, some outgoing): inside a transfer run no scan-kind kernel
    launches for them (the forward scan and the backward insert do its work)."""
    out = set()
    for v in range(w.n_tables):
        st = s.stats(1, v)
        if st is not None and st["n_in"] == 0 and st["n_out"] > 0:
            out.add(v)
    return out


def run_gpu(w, **kw):
    s = session_for(w, **kw)
    try:
        s.run()
        return collect(s, w)
    finally:
        s.close()


def assert_same(got, want, w, sectors=True):
    for p in range(2):
        for v in range(w.n_tables):
            n = w.tables[v].n_rows
            g, o = got["surv"][p][v][: (n + 31) // 32], want["surv"][p][v]
            assert np.array_equal(g, o), f"pass {p} table {v}: survivor bitmaps differ"
            assert got["count"][p][v] == want["count"][p][v], (p, v)
            if sectors:
                assert tuple(got["sectors"][p][v]) == tuple(want["sectors"][p][v]), (p, v)
        for e in range(len(w.edges)):
            assert got["nblocks"][p][e] == want["nblocks"][p][e], (p, e)
            assert np.array_equal(got["filters"][p][e], want["filters"][p][e]), f"pass {p} edge {e}: filters differ"


def collect_one_hop(s, w):
    """A one-hop session's results in the oracle's one_hop() shape: pass 1's
    survivors, pass 0's filters, and pass 0's survivors of the builders."""
    out = {"surv": [], "count": [], "filters": [], "nblocks": [], "built": {}}
    for v in range(w.n_tables):
        bm, c = s.survivors(v)
        out["surv"].append(bm.cpu().numpy().view(np.uint32))
        out["count"].append(c)
        if s.stats(0, v) is not None:
            bm0, c0 = s.survivors(v, 0)
            out["built"][v] = (bm0.cpu().numpy().view(np.uint32), c0)
    for e in range(len(w.edges)):
        f = s.filter(0, e).cpu().numpy().view(np.uint32)
        out["filters"].append(f)
        out["nblocks"].append(len(f) * 32 // w.block_bits)
    return out


def assert_same_one_hop(got, want, w):
    for v in range(w.n_tables):
        n = w.tables[v].n_rows
        assert np.array_equal(got["surv"][v][: (n + 31) // 32], want["surv"][v]), f"table {v}: survivors differ"
        assert got["count"][v] == want["count"][v], v
    for e in range(len(w.edges)):
        assert got["nblocks"][e] == want["nblocks"][e], e
        assert np.array_equal(got["filters"][e], want["filters"][e]), f"edge {e}: filters differ"
    # a builder's pass-0 survivors are its selection
    for v, (bm, c) in got["built"].items():
        t = w.tables[v]
        nw = (t.n_rows + 31) // 32
        sel = t.sel if t.sel is not None else _all_rows(t.n_rows)
        assert np.array_equal(bm[:nw], sel[:nw]), v
        assert c == int(sum(bin(int(x)).count("1") for x in sel[:nw]))


def _all_rows(n):
    words = np.full((n + 31) // 32, 0xFFFFFFFF, np.uint32)
    if n % 32:
        words[-1] = (1 << (n % 32)) - 1
    return words
