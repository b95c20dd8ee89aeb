"""Helpers shared by the tests: load the hand-made golden workloads."""
import json
import os

import numpy as np

from workloads import Edge, Table, Workload, bitmap_from_rows

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_json(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def golden_workload(name, bits_per_key=10, k=4, block_bits=256, dtype=np.int32):
    """Workload from a fixture; returns (workload, fixture dict, table name -> id)."""
    g = load_json(name)
    tid = {t["name"]: i for i, t in enumerate(g["tables"])}
    tables = []
    colidx = []
    for t in g["tables"]:
        names = list(t["cols"].keys())
        cols = [np.asarray(t["cols"][c], dtype=dtype) for c in names]
        n = len(cols[0])
        sel = None if t["sel"] is None else bitmap_from_rows(n, np.asarray(t["sel"]) - 1)
        tables.append(Table(t["name"], n, cols, names, sel))
        colidx.append({c: j for j, c in enumerate(names)})
    edges = []
    for e in g["edges"]:
        a, b = tid[e["t0"]], tid[e["t1"]]
        edges.append(Edge(a, tuple(colidx[a][c] for c in e["c0"]), b,
                          tuple(colidx[b][c] for c in e["c1"])))
    return Workload(name, tables, edges, bits_per_key, k, block_bits, 0), g, tid


def rows1(words, n):
    """1-based row numbers of the set bits of a bitmap."""
    from workloads import rows_from_bitmap
    return [int(r) + 1 for r in rows_from_bitmap(words, n)]
