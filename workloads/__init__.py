"""Seeded synthetic join workloads for predicate transfer.

This module only makes inputs: key columns, local-predicate selection
bitmaps and the join graph (which key columns each equi-join edge
connects).  It holds none of the transfer's arithmetic (no hashing, no
filter layout, no schedule), so both the CPU oracle and the CUDA path can
be fed from it without sharing any of the method's code.

Layouts produced here
---------------------
* a key column is a 1-D ``numpy`` array of ``int32`` or ``int64``;
* a selection bitmap is ``uint32[ceil(n/32)]``: row ``r`` is bit ``r & 31``
  of word ``r >> 5`` (least significant bit = lower row id); tail bits
  beyond ``n`` are zero;
* an edge joins ``tables[t0].cols[c0[i]] == tables[t1].cols[c1[i]]`` for
  every ``i`` (one column, or two for a composite key).

The workload shapes stand in for the paper's TPC-H experiments (Section 4;
TPC-H itself is not used): a 3-table chain like the Fig. 3 example, a
6-table snowflake whose sizes mirror the tables of TPC-H Q5 at scale
factors 1 and 10 (Tables 1-2), a cyclic 5-table graph and a resident star
for serving.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20230728


@dataclasses.dataclass
class Table:
    name: str
    n_rows: int
    cols: List[np.ndarray]
    col_names: List[str]
    sel: Optional[np.ndarray] = None  # uint32 bitmap or None (all rows)

    def col(self, name: str) -> int:
        return self.col_names.index(name)


@dataclasses.dataclass
class Edge:
    t0: int
    c0: Tuple[int, ...]
    t1: int
    c1: Tuple[int, ...]
    flags: int = 0


@dataclasses.dataclass
class Workload:
    name: str
    tables: List[Table]
    edges: List[Edge]
    bits_per_key: int = 10
    k: int = 4
    block_bits: int = 256
    seed: int = 0

    @property
    def n_tables(self) -> int:
        return len(self.tables)

    def nbytes(self) -> int:
        b = 0
        for t in self.tables:
            b += sum(c.nbytes for c in t.cols)
            if t.sel is not None:
                b += t.sel.nbytes
        return b


# --------------------------------------------------------------------------
# bitmap helpers (input layout only)
# --------------------------------------------------------------------------

def n_words(n: int) -> int:
    return (n + 31) // 32


def bitmap_from_rows(n: int, rows: np.ndarray) -> np.ndarray:
    bits = np.zeros(n_words(n) * 32, dtype=bool)
    bits[np.asarray(rows, dtype=np.int64)] = True
    return np.packbits(bits, bitorder="little").view("<u4").astype(np.uint32)


def bitmap_from_bools(bits: np.ndarray) -> np.ndarray:
    n = len(bits)
    pad = np.zeros(n_words(n) * 32, dtype=bool)
    pad[:n] = bits
    return np.packbits(pad, bitorder="little").view("<u4").astype(np.uint32)


def rows_from_bitmap(words: np.ndarray, n: int) -> np.ndarray:
    bits = np.unpackbits(np.ascontiguousarray(words, dtype="<u4").view(np.uint8),
                         bitorder="little")[:n]
    return np.nonzero(bits)[0]


def bools_from_bitmap(words: np.ndarray, n: int) -> np.ndarray:
    bits = np.unpackbits(np.ascontiguousarray(words, dtype="<u4").view(np.uint8),
                         bitorder="little")
    return bits[:n].astype(bool)


def popcount_bitmap(words: np.ndarray) -> int:
    return int(np.unpackbits(np.ascontiguousarray(words, dtype="<u4").view(np.uint8)).sum())


# --------------------------------------------------------------------------
# key generators
# --------------------------------------------------------------------------

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _odd_u64(rng: np.random.Generator) -> np.uint64:
    return np.uint64(int(rng.integers(0, 2**62, dtype=np.uint64)) * 2 + 1)


def _scramble64(rng: np.random.Generator, x: np.ndarray) -> np.ndarray:
    """Injective u64 map x -> x*a + c (mod 2^64), a odd: distinct in, distinct out.

    An affine map drawn from the generator; it spreads small integer ids
    over the whole 64-bit range so that int64 keys use their high bits.
    """
    a = _odd_u64(rng)
    c = np.uint64(int(rng.integers(0, 2**63, dtype=np.uint64)))
    with np.errstate(over="ignore"):
        return (x.astype(np.uint64) * a + c).view(np.int64)


def pk_column(rng: np.random.Generator, n: int, int64: bool) -> np.ndarray:
    """Distinct primary keys in random row order."""
    perm = rng.permutation(n)
    if not int64:
        return perm.astype(np.int32)
    return _scramble64(rng, perm.astype(np.uint64))


def bounded_power_law_ranks(rng: np.random.Generator, m: int, n: int, s: float,
                            chunk: int = 8_000_000) -> np.ndarray:
    """n ranks in [0, m) with P(rank ~ r) proportional to (r+1)^-s.

    Continuous inverse-CDF sampling of the bounded power law on [1, m+1),
    floored: a Zipf(s)-shaped draw without an m-entry table.
    """
    out = np.empty(n, dtype=np.int64)
    a = 1.0 - s
    hi = float(m + 1) ** a
    for lo in range(0, n, chunk):
        u = rng.random(min(chunk, n - lo))
        x = ((hi - 1.0) * u + 1.0) ** (1.0 / a)
        r = np.floor(x).astype(np.int64) - 1
        np.clip(r, 0, m - 1, out=r)
        out[lo:lo + len(r)] = r
    return out


def fk_rows(rng: np.random.Generator, m: int, n: int, zipf: Optional[float]) -> np.ndarray:
    """Target row (in [0, m)) of each of n foreign keys."""
    if zipf is None:
        return rng.integers(0, m, n, dtype=np.int64)
    ranks = bounded_power_law_ranks(rng, m, n, zipf)
    perm = rng.permutation(m)
    return perm[ranks]


def selection(rng: np.random.Generator, n: int, frac: float) -> np.ndarray:
    """Exact-count uniform random subset of floor(frac*n) rows, as a bitmap."""
    k = int(math.floor(frac * n))
    rows = rng.choice(n, size=k, replace=False) if k > 0 else np.zeros(0, np.int64)
    return bitmap_from_rows(n, rows)


def _scaled(n: int, scale: float, minimum: int = 1) -> int:
    return max(minimum, int(round(n * scale)))


# --------------------------------------------------------------------------
# the five workload shapes
# --------------------------------------------------------------------------

def chain3(scale: float = 1.0, seed: int = BASE_SEED + 0, bits_per_key: int = 10,
           k: int = 4, block_bits: int = 256) -> Workload:
    """R(a) - S(a, b) - T(b): R 10k, S 100k, T 10k rows, int32 keys.

    S.a / S.b are uniform over the R / T keys; local predicates keep 10% of
    R and 20% of T (exact-count uniform subsets).
    """
    rng = _rng(seed)
    nr, ns, nt = _scaled(10_000, scale), _scaled(100_000, scale), _scaled(10_000, scale)
    ra = pk_column(rng, nr, False)
    tb = pk_column(rng, nt, False)
    sa = ra[fk_rows(rng, nr, ns, None)]
    sb = tb[fk_rows(rng, nt, ns, None)]
    R = Table("R", nr, [ra], ["a"], selection(rng, nr, 0.10))
    S = Table("S", ns, [sa, sb], ["a", "b"], None)
    T = Table("T", nt, [tb], ["b"], selection(rng, nt, 0.20))
    edges = [Edge(0, (0,), 1, (0,)), Edge(1, (1,), 2, (0,))]
    return Workload("chain3", [R, S, T], edges, bits_per_key, k, block_bits, 0)


def snowflake(scale: float = 1.0, int64: bool = False, composite: bool = False,
              zipf: Optional[float] = None, seed: int = BASE_SEED + 1,
              bits_per_key: int = 10, k: int = 4, block_bits: int = 256,
              sel: Sequence[float] = (0.10, 0.01, 0.30)) -> Workload:
    """Six-table snowflake shaped like TPC-H Q5's tables.

    fact F (6M x scale) -> mid M (1.5M), dim2 D2 (200k), dim3 D3 (10k);
    M -> dim1 D1 (150k); D1 and D3 -> a 25-row table N (N stays 25 rows at
    every scale, as a nation table does).  Predicates keep sel[0] of D1,
    sel[1] of D2 and sel[2] of D3.  ``composite`` makes the F->M key two
    columns: M's key is (s(i >> 3), i & 7) for a scrambled s.  ``zipf``
    skews all three fact foreign keys by a bounded power law.
    """
    rng = _rng(seed)
    nF = _scaled(6_000_000, scale)
    nM = _scaled(1_500_000, scale)
    nD2 = _scaled(200_000, scale)
    nD3 = _scaled(10_000, scale)
    nD1 = _scaled(150_000, scale)
    nN = 25
    dt = np.int64 if int64 else np.int32

    n_id = pk_column(rng, nN, int64)
    d3_id = pk_column(rng, nD3, int64)
    d1_id = pk_column(rng, nD1, int64)
    d2_id = pk_column(rng, nD2, int64)
    d3_fk = n_id[fk_rows(rng, nN, nD3, None)]
    d1_fk = n_id[fk_rows(rng, nN, nD1, None)]
    if composite:
        i = rng.permutation(nM).astype(np.uint64)
        m_k1 = _scramble64(rng, i >> np.uint64(3))
        m_k2 = (i & np.uint64(7)).astype(np.int64)
        m_cols = [m_k1, m_k2]
        m_names = ["k1", "k2"]
    else:
        m_cols = [pk_column(rng, nM, int64)]
        m_names = ["id"]
    m_fk = d1_id[fk_rows(rng, nD1, nM, None)]
    t = fk_rows(rng, nM, nF, zipf)
    f_m = [c[t] for c in m_cols]
    del t
    f_d2 = d2_id[fk_rows(rng, nD2, nF, zipf)]
    f_d3 = d3_id[fk_rows(rng, nD3, nF, zipf)]

    F = Table("F", nF, f_m + [f_d2, f_d3],
              (["fk_m1", "fk_m2"] if composite else ["fk_m"]) + ["fk_d2", "fk_d3"])
    M = Table("M", nM, m_cols + [m_fk], m_names + ["fk_d1"])
    D2 = Table("D2", nD2, [d2_id], ["id"], selection(rng, nD2, sel[1]))
    D3 = Table("D3", nD3, [d3_id, d3_fk], ["id", "fk_n"], selection(rng, nD3, sel[2]))
    D1 = Table("D1", nD1, [d1_id, d1_fk], ["id", "fk_n"], selection(rng, nD1, sel[0]))
    N = Table("N", nN, [n_id], ["id"], None)
    for tb in (F, M, D2, D3, D1, N):
        tb.cols = [np.ascontiguousarray(c, dtype=dt) for c in tb.cols]
    nk = 2 if composite else 1
    edges = [
        Edge(0, tuple(range(nk)), 1, tuple(range(nk))),  # F.fk_m  = M.id
        Edge(0, (nk,), 2, (0,)),                           # F.fk_d2 = D2.id
        Edge(0, (nk + 1,), 3, (0,)),                       # F.fk_d3 = D3.id
        Edge(1, (nk,), 4, (0,)),                           # M.fk_d1 = D1.id
        Edge(4, (1,), 5, (0,)),                            # D1.fk_n = N.id
        Edge(3, (1,), 5, (0,)),                            # D3.fk_n = N.id
    ]
    name = "snowflake" if scale <= 1.0 else f"snowflake_x{scale:g}"
    return Workload(name, [F, M, D2, D3, D1, N], edges, bits_per_key, k, block_bits, 0)


def cyclic5(scale: float = 1.0, seed: int = BASE_SEED + 3, bits_per_key: int = 10,
            k: int = 4, block_bits: int = 256) -> Workload:
    """Triangle T0-T1-T2 plus pendants D-T1 and E-T0; int64 keys.

    T0 20M, T1 5M, T2 5M, D 1M, E 100k rows (x scale).  Each edge has one
    column on either side, uniform over [0, min(n_u, n_v)) and scrambled by
    one injective map per edge.  Predicates keep 5% of T2 and of E.
    """
    rng = _rng(seed)
    n = [_scaled(20_000_000, scale), _scaled(5_000_000, scale), _scaled(5_000_000, scale),
         _scaled(1_000_000, scale), _scaled(100_000, scale)]
    pairs = [(0, 1), (0, 2), (1, 2), (1, 3), (0, 4)]
    cols: List[List[np.ndarray]] = [[] for _ in n]
    names: List[List[str]] = [[] for _ in n]
    edges = []
    tn = ["T0", "T1", "T2", "D", "E"]
    for (u, v) in pairs:
        dom = min(n[u], n[v])
        a = _odd_u64(rng)
        c = np.uint64(int(rng.integers(0, 2**63, dtype=np.uint64)))
        with np.errstate(over="ignore"):
            ku = (rng.integers(0, dom, n[u]).astype(np.uint64) * a + c).view(np.int64)
            kv = (rng.integers(0, dom, n[v]).astype(np.uint64) * a + c).view(np.int64)
        edges.append(Edge(u, (len(cols[u]),), v, (len(cols[v]),)))
        cols[u].append(ku)
        names[u].append("k_" + tn[v])
        cols[v].append(kv)
        names[v].append("k_" + tn[u])
    tables = [Table(tn[i], n[i], cols[i], names[i], None) for i in range(5)]
    tables[2].sel = selection(rng, n[2], 0.05)
    tables[4].sel = selection(rng, n[4], 0.05)
    return Workload("cyclic5", tables, edges, bits_per_key, k, block_bits, 0)


def star(scale: float = 1.0, seed: int = BASE_SEED + 4, bits_per_key: int = 10,
         k: int = 4, block_bits: int = 256) -> Workload:
    """Resident star for serving: F 100M rows with four int64 foreign keys
    to D0 25M, D1 2M, D2 1M, D3 100k (x scale); no predicates (queries
    bring their own)."""
    rng = _rng(seed)
    nd = [_scaled(25_000_000, scale), _scaled(2_000_000, scale), _scaled(1_000_000, scale),
          _scaled(100_000, scale)]
    nF = _scaled(100_000_000, scale)
    dims = [pk_column(rng, m, True) for m in nd]
    fks = [d[fk_rows(rng, len(d), nF, None)] for d in dims]
    F = Table("F", nF, fks, [f"fk_d{i}" for i in range(4)], None)
    tables = [F] + [Table(f"D{i}", nd[i], [dims[i]], ["id"], None) for i in range(4)]
    edges = [Edge(0, (i,), i + 1, (0,)) for i in range(4)]
    return Workload("star", tables, edges, bits_per_key, k, block_bits, 0)


@dataclasses.dataclass
class Query:
    """One served query: table instances over the resident star and edges
    between instances.  ``inst_table[j]`` is the resident table of instance
    j; ``sel[j]`` its own selection bitmap (None = all rows)."""
    inst_table: List[int]
    sel: List[Optional[np.ndarray]]
    edges: List[Edge]
    arrival_s: float = 0.0


def selection_pool(w: Workload, size: int = 32, seed: int = BASE_SEED + 41, sel_lo: float = 0.001,
                   sel_hi: float = 0.5) -> List[List[np.ndarray]]:
    """Per dimension table of a star, `size` exact-count uniform selections
    with log-uniform selectivities in [sel_lo, sel_hi].

    Each is a random window of one seeded permutation of the table's rows,
    so a pool costs one permutation per table instead of one per query.
    """
    rng = _rng(seed)
    pools: List[List[np.ndarray]] = [[]]
    for t in w.tables[1:]:
        n = t.n_rows
        perm = rng.permutation(n)
        pool = []
        for _ in range(size):
            frac = math.exp(rng.uniform(math.log(sel_lo), math.log(sel_hi)))
            k = int(math.floor(frac * n))
            start = int(rng.integers(0, n))
            rows = np.concatenate([perm[start:start + k], perm[:max(0, start + k - n)]])
            pool.append(bitmap_from_rows(n, rows))
        pools.append(pool)
    return pools


def serving_queries(w: Workload, n_queries: int, rate_qps: float, seed: int = BASE_SEED + 40,
                    min_inst: int = 3, max_inst: int = 6, sel_lo: float = 0.001,
                    sel_hi: float = 0.5, pool: Optional[List[List[np.ndarray]]] = None) -> List[Query]:
    """Poisson arrivals of random connected star subgraphs.

    Each query takes the fact instance plus 2-4 distinct dimension
    instances (3-5 instances); a 6-instance query adds a second instance
    (an alias) of one chosen dimension, joined on the same foreign key.
    Every dimension instance gets a log-uniform selectivity in
    [sel_lo, sel_hi] (drawn from `pool`, see :func:`selection_pool`, when
    one is given).
    """
    rng = _rng(seed)
    t = 0.0
    out = []
    n_dims = len(w.tables) - 1
    for _ in range(n_queries):
        t += rng.exponential(1.0 / rate_qps) if rate_qps > 0 else 0.0
        n_inst = int(rng.integers(min_inst, max_inst + 1))
        n_dim_inst = n_inst - 1
        n_distinct = min(n_dim_inst, n_dims)
        dims = list(rng.choice(n_dims, size=n_distinct, replace=False) + 1)
        while len(dims) < n_dim_inst:
            dims.append(dims[int(rng.integers(0, len(dims)))])
        inst_table = [0] + [int(d) for d in dims]
        sel: List[Optional[np.ndarray]] = [None]
        edges = []
        for j, d in enumerate(dims, start=1):
            m = w.tables[d].n_rows
            if pool is not None:
                sel.append(pool[d][int(rng.integers(0, len(pool[d])))])
            else:
                frac = math.exp(rng.uniform(math.log(sel_lo), math.log(sel_hi)))
                sel.append(selection(rng, m, frac))
            edges.append(Edge(0, (int(d) - 1,), j, (0,)))
        out.append(Query(inst_table, sel, edges, t))
    return out


def random_tiny(seed: int, n_tables: int, max_rows: int = 48, domain: int = 6,
                acyclic: bool = True, int64_mix: bool = True,
                composite_prob: float = 0.0, sel_prob: float = 0.6) -> Workload:
    """Small random join graph for brute-force checks.

    Tables have 1..max_rows rows; every edge adds one fresh column on
    either side (values uniform in [0, domain)), or two for a composite
    key.  ``acyclic`` makes the join graph a random tree; otherwise extra
    edges (a cycle, possibly parallel edges) are added.
    """
    rng = _rng(seed)
    n = [int(rng.integers(1, max_rows + 1)) for _ in range(n_tables)]
    pairs = []
    for v in range(1, n_tables):
        pairs.append((int(rng.integers(0, v)), v))
    if not acyclic:
        for _ in range(int(rng.integers(1, 3))):
            u, v = rng.choice(n_tables, size=2, replace=False)
            pairs.append((int(u), int(v)))
    cols: List[List[np.ndarray]] = [[] for _ in n]
    edges = []
    for (u, v) in pairs:
        nk = 2 if rng.random() < composite_prob else 1
        cu, cv = [], []
        for _ in range(nk):
            dt_u = np.int64 if (int64_mix and rng.random() < 0.5) else np.int32
            dt_v = np.int64 if (int64_mix and rng.random() < 0.5) else np.int32
            # negative values exercise the sign extension of int32 keys
            off = -domain // 2
            cu.append(len(cols[u]))
            cols[u].append((rng.integers(0, domain, n[u]) + off).astype(dt_u))
            cv.append(len(cols[v]))
            cols[v].append((rng.integers(0, domain, n[v]) + off).astype(dt_v))
        edges.append(Edge(u, tuple(cu), v, tuple(cv)))
    tables = []
    for i in range(n_tables):
        s = None
        if rng.random() < sel_prob:
            s = bitmap_from_bools(rng.random(n[i]) < rng.uniform(0.2, 0.9))
        if not cols[i]:
            cols[i].append(np.zeros(n[i], np.int32))
        tables.append(Table(f"t{i}", n[i], cols[i], [f"c{j}" for j in range(len(cols[i]))], s))
    return Workload(f"tiny{seed}", tables, edges, 10, 4, 256, 0)
