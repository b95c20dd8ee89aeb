"""Pins of the oracle's key -> block -> bit rule against hand-worked vectors.

The vectors in ``golden/filter_bits_vectors.json`` were worked out by hand
from the written filter rule (block by multiply-shift of the high word;
h1 = lo mod B, h2 = (lo >> 16) | 1, bit i = (h1 + i*h2) mod B; bit t of a
block is bit t mod 32 of word t div 32).  The paper fixes no filter layout
(Section 3.2, "Filter Type"), so these pin the library's own rule: a
shifted h1 or h2, a wrong wrap, or a most-significant-bit-first word order
fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
VEC = json.load(open(os.path.join(HERE, "golden", "filter_bits_vectors.json")))


def _h(v):
    return int(v["h"], 16)


@pytest.mark.parametrize("v", VEC["vectors"], ids=lambda v: v["h"])
def test_block_index(oracle_lib, v):
    for nb, j in v["block"].items():
        assert oracle_lib.block_of(_h(v), int(nb)) == j


@pytest.mark.parametrize("v", VEC["vectors"], ids=lambda v: v["h"])
@pytest.mark.parametrize("B", [256, 512])
@pytest.mark.parametrize("k", [4, 7])
def test_bit_positions_in_order(oracle_lib, v, B, k):
    assert oracle_lib.bits_of(_h(v), B, k) == v["bits7"][str(B)][:k]


@pytest.mark.parametrize("v", VEC["vectors"], ids=lambda v: v["h"])
@pytest.mark.parametrize("B", [256, 512])
def test_single_insert_sets_the_worked_words(oracle_lib, v, B):
    spec = v["words"][str(B)]
    nb = spec["nblocks"]
    got = oracle_lib.filter_build([_h(v)], nb, B, 4)
    want = np.zeros(nb * B // 32, np.uint32)
    for i, x in spec["words"].items():
        want[int(i)] = int(x, 16)
    assert np.array_equal(got, want), {i: hex(int(x)) for i, x in enumerate(got) if x}


@pytest.mark.parametrize("v", VEC["vectors"], ids=lambda v: v["h"])
@pytest.mark.parametrize("B", [256, 512])
def test_probe_reads_the_same_bits(oracle_lib, v, B):
    # the probe accepts the inserted hash, and rejects it as soon as any one
    # of its worked bits is cleared
    spec = v["words"][str(B)]
    nb = spec["nblocks"]
    h = _h(v)
    words = oracle_lib.filter_build([h], nb, B, 4)
    assert oracle_lib.filter_probe(words, nb, B, 4, [h])[0]
    base = v["block"]["5"] * B // 32 if nb == 5 else 0
    for b in v["bits7"][str(B)][:4]:
        w = words.copy()
        w[base + (b >> 5)] &= np.uint32(~(1 << (b & 31)) & 0xFFFFFFFF)
        assert not oracle_lib.filter_probe(w, nb, B, 4, [h])[0]


def test_key_to_bits_through_the_hash(oracle_lib):
    kb = VEC["key_to_bits"]
    h = oracle_lib.hash1(kb["key"], kb["seed"])
    assert h == int(kb["h"], 16)
    for nb, j in kb["block"].items():
        assert oracle_lib.block_of(h, int(nb)) == j
    for B, bl in kb["bits4"].items():
        assert oracle_lib.bits_of(h, int(B), 4) == bl
