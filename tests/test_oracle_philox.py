"""Pins of the oracle's Philox4x32-10 (reading R1/R2 of the VEGAS+ point draw).

* known-answer vectors published with the generator (tests/golden), which a
  wrong multiplier, Weyl constant, word order or round count fails;
* statistical uniformity of the words and of the derived coordinates;
* avalanche: one flipped counter bit changes about half of the 128 output bits.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_uniform_words(orc):
    rng = np.random.default_rng(1)
    counts = np.zeros(256)
    for _ in range(4096):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        out = orc.philox4x32_10(ctr, [7, 11])
        for w in out:
            counts[int(w) >> 24] += 1
    expected = counts.sum() / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 340.0  # 255 dof; p ~ 3e-4


def test_avalanche(orc):
    rng = np.random.default_rng(2)
    dist = []
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        a = orc.philox4x32_10(ctr, [3, 5])
        bit = int(rng.integers(0, 128))
        ctr2 = ctr.copy()
        ctr2[bit // 32] ^= np.uint64(1 << (bit % 32))
        b = orc.philox4x32_10(ctr2, [3, 5])
        dist.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(dist) < 68
