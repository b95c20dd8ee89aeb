"""The oracle's join count (Section 3.3, the join phase): equal to the
brute-force join on tiny trees, and unchanged by predicate transfer (the
transfer keeps every row that takes part in the join)."""
import dataclasses

import numpy as np
import pytest

import workloads as W


def test_join_count_equals_brute_force(oracle_lib):
    for seed in range(40):
        w = W.random_tiny(2000 + seed, 2 + seed % 5, max_rows=14, domain=4, acyclic=True,
                          composite_prob=0.25)
        assert oracle_lib.join_count(w) == oracle_lib.brute_force(w)["n_results"], seed


def test_join_count_of_a_forest_is_a_product(oracle_lib):
    a = W.random_tiny(77, 3, max_rows=12, domain=3)
    b = W.random_tiny(78, 2, max_rows=12, domain=3)
    k = a.n_tables
    w = W.Workload("forest", a.tables + b.tables,
                   a.edges + [dataclasses.replace(e, t0=e.t0 + k, t1=e.t1 + k) for e in b.edges])
    assert oracle_lib.join_count(w) == oracle_lib.join_count(a) * oracle_lib.join_count(b)


@pytest.mark.parametrize("exact", [True, False])
def test_transfer_keeps_the_join_size(oracle_lib, exact):
    for seed in range(25):
        w = W.random_tiny(2100 + seed, 3 + seed % 4, max_rows=80, domain=6, acyclic=True, composite_prob=0.2)
        res = oracle_lib.transfer(w, exact=exact)
        assert oracle_lib.join_count(w, rows=res["surv"][1]) == oracle_lib.join_count(w), seed
        assert oracle_lib.join_count(w, rows=res["surv"][0]) == oracle_lib.join_count(w), seed


def test_chain3_join_size(oracle_lib):
    """R 10k (10% kept) - S 100k - T 10k (20% kept), S's keys uniform over
    R's and T's: about 100k * 0.1 * 0.2 = 2000 joined tuples (one per
    surviving S row: R and T keys are unique), on the selections and on the
    transfer's survivors alike."""
    w = W.chain3()
    n = oracle_lib.join_count(w)
    assert 1800 < n < 2200
    res = oracle_lib.transfer(w)
    assert oracle_lib.join_count(w, rows=res["surv"][1]) == n
    # with unique keys on R and T, each surviving S row of the exact reduction is one tuple
    ex = oracle_lib.transfer(w, exact=True)
    assert ex["count"][1][1] == n


def test_join_count_rejects_cycles_and_one_way_edges(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.join_count(W.cyclic5(scale=0.001))
    w = W.chain3(scale=0.01)
    w = dataclasses.replace(w, edges=[dataclasses.replace(w.edges[0], flags=1), w.edges[1]])
    with pytest.raises(ValueError):
        oracle_lib.join_count(w)
