"""Pins of the oracle's blocked Bloom filter: bit layout invariants, the
size rule, no false negatives, and the false-positive rate against the
closed form of the blocked layout."""
import math

import numpy as np
import pytest

from _fpr_model import blocked_km_fpr, textbook_fpr
from workloads import Edge, Table, Workload


@pytest.mark.parametrize("B", [256, 512])
@pytest.mark.parametrize("k", [1, 2, 4, 7, 16])
def test_bit_positions_distinct_and_in_block(oracle_lib, B, k):
    rng = np.random.default_rng(B + k)
    for h in rng.integers(0, 2**63, 300, dtype=np.uint64):
        h = int(h) * 2 + 1
        pos = oracle_lib.bits_of(h, B, k)
        assert len(set(pos)) == k
        assert all(0 <= p < B for p in pos)


@pytest.mark.parametrize("B", [256, 512])
def test_single_insert_sets_k_bits_in_its_block(oracle_lib, B):
    rng = np.random.default_rng(7)
    for nb in (1, 3, 17, 1000):
        for _ in range(20):
            h = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
            w = oracle_lib.filter_build([h], nb, B, 4)
            j = oracle_lib.block_of(h, nb)
            assert 0 <= j < nb
            blk = w.reshape(nb, B // 32)
            assert int(np.unpackbits(blk.view(np.uint8)).sum()) == 4
            assert int(np.unpackbits(blk[j].view(np.uint8)).sum()) == 4


def test_block_index_uses_high_word_multiply_shift(oracle_lib):
    # multiply-shift range reduction: endpoints, independence of the low word, near-uniformity
    for nb in (1, 2, 7, 1000, 2**31 - 1):
        assert oracle_lib.block_of(0x00000000_FFFFFFFF, nb) == 0
        assert oracle_lib.block_of(0xFFFFFFFF_00000000, nb) == nb - 1
    rng = np.random.default_rng(3)
    hs = [int(x) for x in rng.integers(0, 2**63, 2000, dtype=np.uint64)]
    for h in hs[:200]:
        assert oracle_lib.block_of(h, 13) == oracle_lib.block_of(h ^ 0xDEADBEEF, 13)
    counts = np.bincount([oracle_lib.block_of(h << 1 | 1, 7) for h in hs], minlength=7)
    chi2 = ((counts - len(hs) / 7) ** 2 / (len(hs) / 7)).sum()
    assert chi2 < 30  # 6 dof; p < 1e-4 above this


def test_size_rule_values(oracle_lib):
    nb = oracle_lib.nblocks_for
    assert nb(0, 100, 10, 256) == 1          # an empty survivor set still gets one block
    assert nb(100, 50, 10, 256) == 2         # min(c, n_probe) = 50 -> ceil(500 / 256)
    assert nb(1000, 10**6, 10, 256) == 40    # ceil(10000 / 256)
    assert nb(1000, 10**6, 10, 512) == 20
    assert nb(256, 10**6, 16, 256) == 16     # exact multiple
    assert nb(257, 10**6, 16, 256) == 17


def test_no_false_negatives(oracle_lib):
    rng = np.random.default_rng(11)
    hs = [int(x) for x in rng.integers(0, 2**63, 3000, dtype=np.uint64)]
    for B in (256, 512):
        for nb in (1, 5, 64):
            w = oracle_lib.filter_build(hs, nb, B, 4)
            assert oracle_lib.filter_probe(w, nb, B, 4, hs).all()


def _fpr_workload(n, m, bits_per_key, block_bits, seed):
    """Build table A (n distinct keys) -> probe table B (m keys none of which is in A)."""
    rng = np.random.default_rng(seed)
    keys = rng.integers(-2**63, 2**63 - 1, n + m + 1000, dtype=np.int64)
    keys = np.unique(keys)
    rng.shuffle(keys)
    a, b = keys[:n], keys[n:n + m]
    A = Table("A", n, [a], ["k"], None)
    Bt = Table("B", m, [b], ["k"], None)
    return Workload("fpr", [A, Bt], [Edge(0, (0,), 1, (0,))], bits_per_key, 4, block_bits, 0)


@pytest.mark.parametrize("bpk,B", [(8, 256), (10, 256), (16, 256), (10, 512), (16, 512)])
def test_false_positive_rate_matches_blocked_closed_form(oracle_lib, bpk, B):
    n, m = 100_000, 4_000_000
    w = _fpr_workload(n, m, bpk, B, seed=bpk * 1000 + B)
    res = oracle_lib.transfer(w)
    nb = res["nblocks"][0][0]
    assert nb == math.ceil(n * bpk / B)
    measured = res["count"][0][1] / m          # every survivor of B is a false positive
    expect = blocked_km_fpr(n, nb, B, 4)
    sigma = math.sqrt(expect * (1 - expect) / m)
    assert abs(measured - expect) <= 4 * sigma + 0.005 * expect, (measured, expect)
    # the blocked layout is never better than the textbook unblocked rate
    assert measured >= textbook_fpr(n, nb * B, 4) - 4 * sigma
