"""CPU oracle for predicate transfer -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product (the CUDA library and
its binding) never loads it, and this package imports nothing from the
product: the two are independent implementations of the same definitions
(hash, filter layout, size rule, schedule; see ``pt_oracle.c``).

* :func:`transfer` runs ``pt_oracle.c`` -- plain single-threaded loops --
  over a :class:`workloads.Workload`, in Bloom mode or in exact-set mode
  (the semi-join program of the paper's Section 3.2 "Filter Type").
* :func:`brute_force` enumerates the full join of the selected rows of a
  tiny workload (Section 2.2: the rows that take part in the join result
  are what the Yannakakis semi-join phase keeps).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False) -> str:
    """Compile pt_oracle.c into liboracle.so next to it (gcc, -O2), and the
    same source with OpenMP into liboracle_omp.so (multi-core timing only)."""
    for lib_path, extra in ((_LIB, ["-Wno-unknown-pragmas"]), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-std=c11", "-Wall", *extra, "-shared", "-fPIC", "-o", lib_path + ".tmp", _SRC]
            subprocess.check_call(cmd)
            os.replace(lib_path + ".tmp", lib_path)
    return _LIB


class _Table(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_cols", C.c_int32), ("cols", C.POINTER(C.c_void_p)),
                ("dtypes", C.POINTER(C.c_int32)), ("sel", C.c_void_p)]


class _Edge(C.Structure):
    _fields_ = [("t0", C.c_int32), ("ncols", C.c_int32), ("c0", C.c_int32 * 2), ("t1", C.c_int32),
                ("c1", C.c_int32 * 2), ("flags", C.c_uint32)]


class _Cfg(C.Structure):
    _fields_ = [("bits_per_key", C.c_int32), ("k", C.c_int32), ("block_bits", C.c_int32),
                ("probe_order", C.c_int32), ("seed", C.c_uint64)]


_lib = None
_lib_omp = None


def _declare(L):
    L.o_hash1.restype = C.c_uint64
    L.o_hash1.argtypes = [C.c_uint64, C.c_uint64]
    L.o_hash2.restype = C.c_uint64
    L.o_hash2.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.o_key.restype = C.c_uint64
    L.o_key.argtypes = [C.c_void_p, C.c_int32, C.c_int64]
    L.o_nblocks.restype = C.c_int64
    L.o_nblocks.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32]
    L.o_block_of.restype = C.c_int64
    L.o_block_of.argtypes = [C.c_uint64, C.c_int64]
    L.o_bits_of.restype = None
    L.o_bits_of.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    L.o_filter_insert.restype = None
    L.o_filter_insert.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_uint64]
    L.o_filter_probe.restype = C.c_int
    L.o_filter_probe.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_uint64]
    L.o_orient.restype = C.c_int
    L.o_orient.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p]
    L.o_transfer.restype = C.c_int
    L.o_transfer.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                             C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p]
    L.o_one_hop.restype = C.c_int
    L.o_one_hop.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                            C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.o_set_threads.restype = C.c_int
    L.o_set_threads.argtypes = [C.c_int32]
    L.o_join_count.restype = C.c_int
    L.o_join_count.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def lib():
    """The plain (single-threaded) oracle."""
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def lib_threads(threads: int):
    """The OpenMP build of the same source, set to ``threads`` threads.
    Returns the library and the thread count it will use."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _declare(C.CDLL(_LIB_OMP))
    used = int(_lib_omp.o_set_threads(int(threads)))
    return _lib_omp, used


# ---- single-function views -------------------------------------------------

def hash1(x: int, seed: int = 0) -> int:
    return int(lib().o_hash1(x & (2**64 - 1), seed))


def hash2(a: int, b: int, seed: int = 0) -> int:
    return int(lib().o_hash2(a & (2**64 - 1), b & (2**64 - 1), seed))


def nblocks_for(c: int, n_probe: int, bits_per_key: int, block_bits: int) -> int:
    return int(lib().o_nblocks(c, n_probe, bits_per_key, block_bits))


def block_of(h: int, nblocks: int) -> int:
    return int(lib().o_block_of(h, nblocks))


def bits_of(h: int, block_bits: int, k: int) -> List[int]:
    out = (C.c_int32 * k)()
    lib().o_bits_of(h, block_bits, k, out)
    return list(out)


def filter_build(hashes, nblocks: int, block_bits: int, k: int) -> np.ndarray:
    words = np.zeros(nblocks * block_bits // 32, np.uint32)
    L = lib()
    for h in hashes:
        L.o_filter_insert(words.ctypes.data, nblocks, block_bits, k, int(h))
    return words


def filter_probe(words: np.ndarray, nblocks: int, block_bits: int, k: int, hashes) -> np.ndarray:
    L = lib()
    return np.array([L.o_filter_probe(words.ctypes.data, nblocks, block_bits, k, int(h))
                     for h in hashes], dtype=bool)


def orient(n_rows: List[int], edges) -> Dict[str, list]:
    nt, ne = len(n_rows), len(edges)
    nr = np.asarray(n_rows, np.int64)
    ea = (_Edge * max(ne, 1))()
    for i, e in enumerate(edges):
        _fill_edge(ea[i], e)
    src = np.zeros(max(ne, 1), np.int32)
    dst = np.zeros(max(ne, 1), np.int32)
    order = np.zeros(max(nt, 1), np.int32)
    lib().o_orient(nt, nr.ctypes.data, ne, C.addressof(ea), src.ctypes.data, dst.ctypes.data,
                   order.ctypes.data)
    return {"src": src[:ne].tolist(), "dst": dst[:ne].tolist(), "order": order[:nt].tolist()}


def _fill_edge(dst: _Edge, e) -> None:
    dst.t0 = e.t0
    dst.t1 = e.t1
    dst.ncols = len(e.c0)
    for j in range(len(e.c0)):
        dst.c0[j] = e.c0[j]
        dst.c1[j] = e.c1[j]
    dst.flags = e.flags


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.int32:
        return 0
    if a.dtype == np.int64:
        return 1
    raise TypeError(f"key columns must be int32 or int64, got {a.dtype}")


def max_filter_words(n0: int, n1: int, bits_per_key: int, block_bits: int) -> int:
    """Words of the largest filter an edge between tables of n0 and n1 rows can get."""
    return nblocks_for(min(n0, n1), max(n0, n1), bits_per_key, block_bits) * block_bits // 32


# ---- the whole transfer ----------------------------------------------------

def _tables(w, keep):
    ta = (_Table * w.n_tables)()
    for i, t in enumerate(w.tables):
        cols = [np.ascontiguousarray(c) for c in t.cols]
        keep.extend(cols)
        ptrs = (C.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        dts = (C.c_int32 * len(cols))(*[_dtype_code(c) for c in cols])
        keep.extend([ptrs, dts])
        ta[i].n_rows = t.n_rows
        ta[i].n_cols = len(cols)
        ta[i].cols = C.cast(ptrs, C.POINTER(C.c_void_p))
        ta[i].dtypes = C.cast(dts, C.POINTER(C.c_int32))
        if t.sel is not None:
            s = np.ascontiguousarray(t.sel, dtype=np.uint32)
            keep.append(s)
            ta[i].sel = s.ctypes.data
        else:
            ta[i].sel = None
    return ta


def join_count(w, rows: Optional[List[Optional[np.ndarray]]] = None) -> int:
    """Size of the join (Section 3.3) of the rows set in ``rows[v]`` (uint32
    bitmaps; None: the tables' selections) over an acyclic join graph of
    inner equi-joins, counted by sorting and summing per key (no tuple is
    built).  Raises ValueError for a cyclic graph or a one-way edge."""
    L = lib()
    keep = []
    ta = _tables(w, keep)
    ea = (_Edge * max(len(w.edges), 1))()
    for i, e in enumerate(w.edges):
        _fill_edge(ea[i], e)
    if rows is None:
        rows = [t.sel for t in w.tables]
    arrs = [None if r is None else np.ascontiguousarray(r, dtype=np.uint32) for r in rows]
    keep.extend(a for a in arrs if a is not None)
    ptrs = (C.c_void_p * w.n_tables)(*[None if a is None else a.ctypes.data for a in arrs])
    out = C.c_uint64()
    rc = L.o_join_count(w.n_tables, C.addressof(ta), len(w.edges), C.addressof(ea), C.addressof(ptrs),
                        C.byref(out))
    if rc != 0:
        raise ValueError("join count needs an acyclic graph of inner joins" if rc == -2 else "invalid workload")
    return int(out.value)


def transfer(w, exact: bool = False, seed: Optional[int] = None, threads: int = 1,
             probe_order: int = 0) -> Dict[str, list]:
    """Forward + backward predicate transfer over workload ``w``.

    Returns ``surv[p][v]`` (uint32 bitmaps), ``count[p][v]``,
    ``filters[p][e]`` (uint32 words, Bloom mode), ``nblocks[p][e]`` and
    ``sectors[p][v] = (probe_sectors, build_sectors)``; ``p`` is 0 for the
    forward pass and 1 for the backward pass.  ``threads`` > 1 runs the
    OpenMP build of the same source (identical results; timing only).
    ``probe_order`` 0/1/2: builder level then LIP, LIP, or edge id (only
    the sector counts depend on it).
    """
    L = lib() if threads <= 1 else lib_threads(threads)[0]
    nt, ne = w.n_tables, len(w.edges)
    keep = []  # keep ctypes buffers alive during the call
    ta = (_Table * nt)()
    for i, t in enumerate(w.tables):
        cols = [np.ascontiguousarray(c) for c in t.cols]
        keep.extend(cols)
        ptrs = (C.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        dts = (C.c_int32 * len(cols))(*[_dtype_code(c) for c in cols])
        keep.extend([ptrs, dts])
        ta[i].n_rows = t.n_rows
        ta[i].n_cols = len(cols)
        ta[i].cols = C.cast(ptrs, C.POINTER(C.c_void_p))
        ta[i].dtypes = C.cast(dts, C.POINTER(C.c_int32))
        if t.sel is not None:
            s = np.ascontiguousarray(t.sel, dtype=np.uint32)
            keep.append(s)
            ta[i].sel = s.ctypes.data
        else:
            ta[i].sel = None
    ea = (_Edge * max(ne, 1))()
    for i, e in enumerate(w.edges):
        _fill_edge(ea[i], e)
    cfg = _Cfg(w.bits_per_key, w.k, w.block_bits, probe_order, w.seed if seed is None else seed)
    surv = [[np.zeros((t.n_rows + 31) // 32, np.uint32) for t in w.tables] for _ in range(2)]
    surv_ptrs = (C.c_void_p * (2 * nt))(*[s.ctypes.data for p in surv for s in p])
    count = np.zeros(2 * nt, np.int64)
    filt = []
    for _p in range(2):
        row = []
        for e in w.edges:
            n0, n1 = w.tables[e.t0].n_rows, w.tables[e.t1].n_rows
            row.append(np.zeros(1 if exact else max_filter_words(n0, n1, w.bits_per_key,
                                                                   w.block_bits), np.uint32))
        filt.append(row)
    filt_ptrs = (C.c_void_p * max(2 * ne, 1))(*[f.ctypes.data for p in filt for f in p])
    nblocks = np.zeros(max(2 * ne, 1), np.int64)
    sectors = np.zeros(2 * nt * 2, np.int64)
    rc = L.o_transfer(nt, C.addressof(ta), ne, C.addressof(ea), C.addressof(cfg), int(exact),
                      C.addressof(surv_ptrs), count.ctypes.data, C.addressof(filt_ptrs),
                      nblocks.ctypes.data, sectors.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the workload")
    wpb = w.block_bits // 32
    out_f = [[filt[p][e][: nblocks[p * ne + e] * wpb].copy() for e in range(ne)] for p in range(2)]
    return {
        "surv": surv,
        "count": [[int(count[p * nt + v]) for v in range(nt)] for p in range(2)],
        "filters": out_f,
        "nblocks": [[int(nblocks[p * ne + e]) for e in range(ne)] for p in range(2)],
        "sectors": [[(int(sectors[(p * nt + v) * 2]), int(sectors[(p * nt + v) * 2 + 1]))
                     for v in range(nt)] for p in range(2)],
    }


def one_hop(w, exact: bool = False, seed: Optional[int] = None, threads: int = 1) -> Dict[str, list]:
    """The Bloom join (Section 2.1): every edge's filter is built from its
    building table's selected rows (the smaller table, or t0 of a one-way
    edge) and probed once by the other end.

    Returns ``surv[v]`` (uint32 bitmaps), ``count[v]``, ``filters[e]``
    (uint32 words, Bloom mode) and ``nblocks[e]``.
    """
    L = lib() if threads <= 1 else lib_threads(threads)[0]
    nt, ne = w.n_tables, len(w.edges)
    keep = []
    ta = _tables(w, keep)
    ea = (_Edge * max(ne, 1))()
    for i, e in enumerate(w.edges):
        _fill_edge(ea[i], e)
    cfg = _Cfg(w.bits_per_key, w.k, w.block_bits, 0, w.seed if seed is None else seed)
    surv = [np.zeros((t.n_rows + 31) // 32, np.uint32) for t in w.tables]
    surv_ptrs = (C.c_void_p * max(nt, 1))(*[s.ctypes.data for s in surv])
    count = np.zeros(max(nt, 1), np.int64)
    filt = [np.zeros(1 if exact else max_filter_words(w.tables[e.t0].n_rows, w.tables[e.t1].n_rows,
                                                       w.bits_per_key, w.block_bits), np.uint32)
            for e in w.edges]
    filt_ptrs = (C.c_void_p * max(ne, 1))(*[f.ctypes.data for f in filt])
    nblocks = np.zeros(max(ne, 1), np.int64)
    rc = L.o_one_hop(nt, C.addressof(ta), ne, C.addressof(ea), C.addressof(cfg), int(exact),
                     C.addressof(surv_ptrs), count.ctypes.data, C.addressof(filt_ptrs), nblocks.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the workload")
    wpb = w.block_bits // 32
    return {
        "surv": surv,
        "count": [int(count[v]) for v in range(nt)],
        "filters": [filt[e][: nblocks[e] * wpb].copy() for e in range(ne)],
        "nblocks": [int(nblocks[e]) for e in range(ne)],
    }


def alg_bytes(w, res: Dict[str, list], sel_read: bool = True) -> Dict[str, int]:
    """Bytes the transfer must move through HBM, summed over both passes.

    Per visit: the input bitmap (the selection in the forward pass, when
    there is one; the forward survivors in the backward pass) and the
    survivor bitmap, 4 bytes each per 32 rows; 32 bytes per key-column
    sector read by the probes and builds; 8 bytes per survivor for the
    compacted row ids (written, then read) when the visit builds filters;
    and the outgoing filters' words, written once.
    """
    o = orient([t.n_rows for t in w.tables], w.edges)
    src, dst = o["src"], o["dst"]
    total = {"bitmap": 0, "keys": 0, "ids": 0, "filters": 0}
    for p in range(2):
        for v, t in enumerate(w.tables):
            nw = (t.n_rows + 31) // 32
            has_in = (t.sel is not None) if p == 0 else True
            total["bitmap"] += 4 * nw * (2 if has_in and sel_read else 1)
            ps, bs = res["sectors"][p][v]
            total["keys"] += 32 * (ps + bs)
            outs = [i for i in range(len(w.edges)) if (src[i] if p == 0 else dst[i]) == v]
            if outs:
                total["ids"] += 8 * res["count"][p][v]
            for i in outs:
                total["filters"] += res["nblocks"][p][i] * w.block_bits // 8
    total["total"] = sum(total.values())
    return total


# ---- brute force (tiny inputs only) ----------------------------------------

def brute_force(w, limit: int = 5_000_000) -> Dict[str, object]:
    """Enumerate the join of the selected rows of every table of ``w``.

    A join result picks one selected row per table such that every edge's
    key columns are equal (composite keys compare both columns; int32 and
    int64 values compare as integers).  Returns the number of results and,
    per table, the rows that take part in at least one result -- the full
    reduction that the Yannakakis semi-join phase reaches on acyclic
    queries (Section 2.2).
    """
    nt = w.n_tables
    rows = []
    for t in w.tables:
        if t.sel is None:
            rows.append(list(range(t.n_rows)))
        else:
            rows.append([r for r in range(t.n_rows) if (int(t.sel[r >> 5]) >> (r & 31)) & 1])
    vals = [[[int(x) for x in c] for c in t.cols] for t in w.tables]

    # visit tables so that each one after the first joins an earlier one where possible
    order = [0]
    while len(order) < nt:
        nxt = None
        for e in w.edges:
            for a, b in ((e.t0, e.t1), (e.t1, e.t0)):
                if a in order and b not in order and nxt is None:
                    nxt = b
        if nxt is None:
            nxt = min(set(range(nt)) - set(order))
        order.append(nxt)
    pos = {v: i for i, v in enumerate(order)}
    checks: List[list] = [[] for _ in range(nt)]
    for e in w.edges:
        a, b = (e.t0, e.t1) if pos[e.t0] < pos[e.t1] else (e.t1, e.t0)
        ca, cb = (e.c0, e.c1) if a == e.t0 else (e.c1, e.c0)
        checks[pos[b]].append((a, ca, cb))

    part = [set() for _ in range(nt)]
    assign = [-1] * nt
    n_results = 0

    def rec(i: int) -> None:
        nonlocal n_results
        if n_results > limit:
            raise RuntimeError("brute-force join too large")
        if i == nt:
            n_results += 1
            for v in range(nt):
                part[v].add(assign[v])
            return
        v = order[i]
        for r in rows[v]:
            ok = True
            for (a, ca, cb) in checks[i]:
                ra = assign[a]
                for x, y in zip(ca, cb):
                    if vals[a][x][ra] != vals[v][y][r]:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                assign[v] = r
                rec(i + 1)
        assign[v] = -1

    sys.setrecursionlimit(max(1000, 10 * nt))
    rec(0)
    return {"n_results": n_results, "participating": [sorted(s) for s in part]}
