"""Pins of the oracle's Philox4x32-10 against the generator's published known answers."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for w in rows:
        out = philox.philox4x32_10(w[0:4], w[4:6])
        assert [int(o) for o in out] == w[6:10]


def test_vectorised_matches_scalar():
    ctr = np.arange(64, dtype=np.uint64)
    vec = philox.philox4x32_10((ctr, 7, 3, 1), (123, 456))
    for i in (0, 17, 63):
        sc = philox.philox4x32_10((i, 7, 3, 1), (123, 456))
        assert all(int(v[i]) == int(s) for v, s in zip(vec, sc))


def test_u53_construction():
    assert philox.u53(0, 0) == 0.0
    top = philox.u53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53
    # (x0 >> 5) fills the high 27 bits, (x1 >> 6) the low 26 bits of the 53-bit mantissa
    assert philox.u53(1 << 5, 0) == 2.0 ** 26 * 2.0 ** -53
    assert philox.u53(0, 1 << 6) == 2.0 ** -53


def test_seed_key_split():
    k0, k1 = philox.seed_key(np.uint64(0x0123456789ABCDEF))
    assert int(k0) == 0x89ABCDEF and int(k1) == 0x01234567


def test_uniform_statistics():
    u = philox.uniform(5, np.arange(200000, dtype=np.uint64), 0, 0, philox.PURPOSE_SPIN)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(u))
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = ((hist - len(u) / 20) ** 2 / (len(u) / 20)).sum()
    assert chi2 < 60          # 19 dof; p ~ 1e-6
