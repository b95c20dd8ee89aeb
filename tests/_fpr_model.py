"""Expected false-positive rate of the blocked filter, from its definition.

A key sets k bits of one B-bit block: h1 + i*h2 (mod B), i < k, with h1
uniform in [0, B) and h2 uniform over the odd residues (Kirsch and
Mitzenmacher's double hashing inside one block).  A non-member query hits
a block holding j keys and passes when all k of its own bits are set.
Inclusion-exclusion over the subsets S of the query's bits gives

    P(pass | j) = sum_S (-1)^|S| (1 - p_S)^j,

where p_S is the chance that one key's k bits meet S.  Averaging over the
query's step h2 and over j ~ Binomial(n, 1/nblocks) (the keys' blocks are
uniform; Putze, Sanders, Singler, "Cache-, Hash- and Space-Efficient Bloom
Filters", 2007) gives the expected rate.  Nothing here calls the oracle.
"""
import math
from itertools import combinations

import numpy as np
from scipy.stats import binom


def blocked_km_fpr(n: int, nblocks: int, block_bits: int, k: int) -> float:
    B = block_bits
    odd = np.arange(1, B, 2)
    lam = n / nblocks
    jmax = int(lam + 12 * math.sqrt(lam) + 20)
    js = np.arange(0, jmax + 1)
    pj = binom.pmf(js, n, 1.0 / nblocks)
    shifts = (np.arange(k)[None, :, None] * odd[:, None, None]) % B  # (h2, i, 1)
    total = 0.0
    for h2q in odd:
        q = [(i * int(h2q)) % B for i in range(k)]
        f = np.zeros(len(js))
        for r in range(0, k + 1):
            for S in combinations(q, r):
                if r == 0:
                    f += 1.0
                    continue
                # h1 values whose progression with step h2 meets S: union of S - i*h2
                U = ((np.asarray(S)[None, None, :] - shifts) % B).reshape(len(odd), -1)
                Us = np.sort(U, axis=1)
                distinct = 1 + (np.diff(Us, axis=1) != 0).sum(axis=1)
                p_s = distinct.mean() / B
                f += (-1) ** r * (1.0 - p_s) ** js
        total += float((f * pj).sum())
    return total / len(odd)


def textbook_fpr(n: int, m_bits: int, k: int) -> float:
    """(1 - e^{-kn/m})^k, the unblocked Bloom filter's rate."""
    return (1.0 - math.exp(-k * n / m_bits)) ** k
