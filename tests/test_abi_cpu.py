"""CPU-side checks of the C ABI: the library builds for sm_103a, loads,
exports every function include/pt.h declares, rejects bad input on the
host, and its host-only planner agrees with the oracle's orientation."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2307_15255_b300 import build
    build.build()
    import paper_2307_15255_b300.pt as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(P):
    names = _declared()
    assert "pt_register_table" in names and "pt_run_backward" in names
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(P):
    for n in _declared():
        assert callable(getattr(P, n)), n


def test_abi_version(P):
    assert P.pt_abi_version() >> 16 == 1


def test_create_rejects_bad_config_before_touching_the_device(P):
    for kw in ({"block_bits": 128}, {"k": 0}, {"k": 17}, {"bits_per_key": 0}):
        with pytest.raises(P.PtError) as ei:
            P.pt_create(**kw)
        assert ei.value.status == P.PT_ERR_INVALID


def test_plan_graph_rejects_malformed_graphs(P):
    with pytest.raises(P.PtError) as ei:
        P.pt_plan_graph([10, 20], [(0, (0,), 0, (0,))])          # self edge
    assert ei.value.status == P.PT_ERR_INVALID
    with pytest.raises(P.PtError) as ei:
        P.pt_plan_graph([10, 20], [(0, (0,), 5, (0,))])          # unknown table
    assert ei.value.status == P.PT_ERR_INVALID
    with pytest.raises(P.PtError) as ei:
        P.pt_plan_graph([10, 20], [(0, (0,), 1, (0,), 2)])      # unknown edge flag
    assert ei.value.status == P.PT_ERR_UNSUPPORTED
    # a one-direction (left outer join) edge is accepted and oriented like any other
    assert P.pt_plan_graph([10, 20], [(1, (0,), 0, (0,), 1)])["src"] == [0]


@pytest.mark.parametrize("make", [W.chain3, lambda: W.snowflake(scale=0.01), lambda: W.cyclic5(scale=0.001)])
def test_plan_graph_matches_oracle_orientation(P, oracle_lib, make):
    w = make()
    n = [t.n_rows for t in w.tables]
    edges = [(e.t0, e.c0, e.t1, e.c1) for e in w.edges]
    got = P.pt_plan_graph(n, edges)
    want = oracle_lib.orient(n, w.edges)
    assert got["src"] == want["src"] and got["dst"] == want["dst"] and got["order"] == want["order"]
    for s, d in zip(got["src"], got["dst"]):
        assert got["level"][d] > got["level"][s]


def test_plan_graph_random_graphs(P, oracle_lib):
    rng = np.random.default_rng(0)
    for s in range(200):
        nt = int(rng.integers(1, 9))
        n = [int(x) for x in rng.integers(0, 5, nt)]  # many ties
        ne = int(rng.integers(0, 12)) if nt > 1 else 0
        edges = []
        for _ in range(ne):
            a, b = rng.choice(nt, 2, replace=False)
            edges.append(W.Edge(int(a), (0,), int(b), (0,)))
        got = P.pt_plan_graph(n, [(e.t0, e.c0, e.t1, e.c1) for e in edges])
        want = oracle_lib.orient(n, edges)
        assert got["src"] == want["src"] and got["dst"] == want["dst"] and got["order"] == want["order"]
        # level = longest path from a source of the oriented DAG, by brute force
        # over paths (the probe order and the first-probe schedule use it)
        for v in range(nt):
            preds = [s_ for s_, d in zip(want["src"], want["dst"]) if d == v]

            def depth(u):
                ps = [s_ for s_, d in zip(want["src"], want["dst"]) if d == u]
                return max([1 + depth(x) for x in ps], default=0)

            assert got["level"][v] == depth(v), (s, v)
            assert all(got["level"][v] > got["level"][u] for u in preds)


def test_context_calls_reject_a_null_context(P):
    # every per-context setter and getter answers PT_ERR_INVALID for ctx = NULL
    # on the host, before touching a device
    n = ctypes.c_int32()
    kt = P.pt_kernel_times()
    for name, args in (("pt_set_streams", (None, 1)), ("pt_set_first_probe", (None, 1)),
                       ("pt_set_cluster", (None, 1)), ("pt_set_kernel_timing", (None, 1)),
                       ("pt_set_graph_mode", (None, 1)), ("pt_set_launch", (None, 256, 0, 0)),
                       ("pt_get_kernel_times", (None, ctypes.byref(kt))),
                       ("pt_get_launch_times", (None, 0, None, ctypes.byref(n))),
                       ("pt_run_transfer", (None,)), ("pt_plan", (None, None, None))):
        assert getattr(P.lib, name)(*args) == P.PT_ERR_INVALID, name
