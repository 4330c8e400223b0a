"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds parameter presets and seeded generators of plaintext
matrices and matrix shapes.  It contains none of the method's arithmetic: no
transform, no encoding, no ring or scheme operation.  Both the oracle
(``oracle/``) and the product package import it so that the two sides receive
the same inputs; neither side imports the other.

The workloads stand in for the paper's experiments (Section 5: random pairs
with dimensions uniform in [1, 64], a ring of dimension 2^12 in the paper).
The three ring-parameter presets follow the benchmark configurations that the
build is measured on:

* ``tiny``   N=4096,  t=65537, 3 chain primes < 2^30, 1 special prime, dnum=3
* ``medium`` N=8192,  t=65537, 5 chain primes < 2^40, 1 special prime, dnum=5
* ``paper``  N=16384, t=65537, 8 chain primes < 2^50, 2 special primes, dnum=4

and the same three rings under the BFV variant (``tiny_bfv``, ``medium_bfv``,
``paper_bfv``).
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Preset:
    """Ring and RNS-chain parameters.

    Primes are the largest primes below ``2**qbits`` congruent to 1 mod 2N
    (chain first, in descending order, then the next ``K`` primes below them
    as special primes).  ``alpha`` chain primes form one key-switching digit,
    ``dnum = L / alpha``.  ``ms_drop`` is the number of chain primes dropped
    by a modulus switch before each ciphertext product (only the tiny preset
    needs one, its 90-bit modulus cannot absorb the product noise).
    """

    name: str
    logN: int
    t: int
    L: int
    qbits: int
    K: int
    alpha: int
    eta: int = 21
    ms_drop: int = 0
    scheme: int = 0  # 0: BGV, 1: BFV (the paper's scheme; no modulus switch)

    @property
    def N(self) -> int:
        return 1 << self.logN

    @property
    def slots(self) -> int:
        return self.N // 2

    @property
    def dnum(self) -> int:
        return self.L // self.alpha


TINY = Preset("tiny", logN=12, t=65537, L=3, qbits=30, K=1, alpha=1, ms_drop=1)
MEDIUM = Preset("medium", logN=13, t=65537, L=5, qbits=40, K=1, alpha=1)
PAPER = Preset("paper", logN=14, t=65537, L=8, qbits=50, K=2, alpha=2)
# The BFV variant on the same rings (the tiny ring needs no modulus switch
# under BFV: its noise stays about 9 bits below log2(Q / 2t)).
TINY_BFV = Preset("tiny_bfv", logN=12, t=65537, L=3, qbits=30, K=1, alpha=1, scheme=1)
MEDIUM_BFV = Preset("medium_bfv", logN=13, t=65537, L=5, qbits=40, K=1, alpha=1, scheme=1)
PAPER_BFV = Preset("paper_bfv", logN=14, t=65537, L=8, qbits=50, K=2, alpha=2, scheme=1)
PRESETS = {p.name: p for p in (TINY, MEDIUM, PAPER, TINY_BFV, MEDIUM_BFV, PAPER_BFV)}

# Matrix shapes (m, l, n) and entry ranges of the workloads.
TINY_SHAPES: List[Tuple[int, int, int]] = [(4, 8, 6)]
TINY_RANGE = (0, 15)
MEDIUM_SHAPES: List[Tuple[int, int, int]] = [(16, 32, 24), (32, 8, 48)]
MEDIUM_RANGE = (-8, 7)
PAPER_SHAPES: List[Tuple[int, int, int]] = [(64, 64, 64), (32, 128, 16), (128, 16, 64)]
PAPER_RANGE = (0, 255)
BATCH_COUNT = 512
BATCH_RANGE = (0, 15)


def matrices(m: int, l: int, n: int, lo: int, hi: int, seed: int = 0, t: int = 65537):
    """Return (A, B) as int64 arrays with entries uniform in [lo, hi].

    Entries are lifted to [0, t) (negative values wrap mod t), which is the
    plaintext space of the scheme.  A is m x l, B is l x n, row-major.
    """
    rng = np.random.default_rng([seed, m, l, n])
    A = rng.integers(lo, hi + 1, size=(m, l), dtype=np.int64)
    B = rng.integers(lo, hi + 1, size=(l, n), dtype=np.int64)
    return np.mod(A, t), np.mod(B, t)


def batch_shapes(count: int, slots: int, seed: int = 0, lo: int = 4, hi: int = 64):
    """Shapes (m, l, n), each uniform in [lo, hi], redrawn until every one of
    m*l, l*n and m*n is at most ``slots`` (the products fit one slot row)."""
    rng = np.random.default_rng([seed, 0xB47C])
    out = []
    while len(out) < count:
        m, l, n = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        if m * l <= slots and l * n <= slots and m * n <= slots:
            out.append((m, l, n))
    return out


def serving_requests(count: int, rate: float, slots: int, seed: int = 0):
    """Poisson arrival stream of matrix-product requests.

    Returns a list of (arrival_time_s, (m, l, n)).  70% small shapes
    (m, l, n uniform in 1..16), 25% medium (17..64, redrawn until the product
    fits ``slots``), 5% exactly 128 x 16 x 64.
    """
    rng = np.random.default_rng([seed, 0x5E7E])
    gaps = rng.exponential(1.0 / rate, size=count)
    times = np.cumsum(gaps)
    out = []
    for i in range(count):
        u = rng.random()
        if u < 0.70:
            shp = tuple(int(v) for v in rng.integers(1, 17, size=3))
        elif u < 0.95:
            while True:
                m, l, n = (int(v) for v in rng.integers(17, 65, size=3))
                if m * l <= slots and l * n <= slots and m * n <= slots:
                    break
            shp = (m, l, n)
        else:
            shp = (128, 16, 64)
        out.append((float(times[i]), shp))
    return out
