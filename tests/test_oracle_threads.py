"""The OpenMP build of the oracle (used only to time it on every host core)
gives the same survivors, counts, filters, sizes and sector counts as the
single-threaded build."""
import pytest

import workloads as W


def _same(a, b):
    import numpy as np
    for p in range(2):
        for x, y in zip(a["surv"][p], b["surv"][p]):
            assert np.array_equal(x, y)
        for x, y in zip(a["filters"][p], b["filters"][p]):
            assert np.array_equal(x, y)
    assert a["count"] == b["count"]
    assert a["nblocks"] == b["nblocks"]
    assert a["sectors"] == b["sectors"]


@pytest.mark.parametrize("make", [lambda: W.chain3(),
                                  lambda: W.snowflake(scale=0.05, int64=True, composite=True, zipf=1.1,
                                                      bits_per_key=16),
                                  lambda: W.cyclic5(scale=0.01)],
                         ids=["chain3", "snowflake_x0.05", "cyclic5_x0.01"])
def test_threads_give_identical_results(oracle_lib, make):
    w = make()
    one = oracle_lib.transfer(w)
    _, used = oracle_lib.lib_threads(4)
    assert used == 4
    _same(one, oracle_lib.transfer(w, threads=4))


def test_threads_exact_mode_identical(oracle_lib):
    w = W.chain3()
    _same(oracle_lib.transfer(w, exact=True), oracle_lib.transfer(w, exact=True, threads=3))
