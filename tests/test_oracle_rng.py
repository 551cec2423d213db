"""Pins for the oracle's counter-based RNG (Philox4x32-10, Salmon et al. SC'11),
its 53-bit uniforms and its Box-Muller normals."""
import math

import numpy as np
import pytest

from conftest import read_golden


def test_philox_known_answers(orc):
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform53_open_interval_and_resolution(orc):
    lo = orc.uniform53(0, 0)
    hi = orc.uniform53(0xFFFFFFFF, 0xFFFFFFFF)
    assert 0.0 < lo < 1e-15
    assert 1.0 - 1e-15 < hi < 1.0
    assert lo == 2.0 ** -53 and hi == 1.0 - 2.0 ** -53
    # only the top 52 of the 64 bits matter: the low 12 bits of `lo` are ignored
    assert orc.uniform53(0x12345678, 0x9ABCDEF0) == orc.uniform53(0x12345678, 0x9ABCD000)
    # one step in bit 12 moves the value by exactly 2^-52
    a = orc.uniform53(0x12345678, 0x9ABCD000)
    b = orc.uniform53(0x12345678, 0x9ABCE000)
    assert b - a == 2.0 ** -52
    # symmetric about 1/2: complementing the word reflects u -> 1 - u
    assert orc.uniform53(0x0F0F0F0F, 0x12345000) + orc.uniform53(0xF0F0F0F0, 0xEDCBAFFF) == 1.0


def _ks_normal(x):
    x = np.sort(x)
    n = len(x)
    cdf = np.array([0.5 * (1.0 + math.erf(v / math.sqrt(2.0))) for v in x])
    d = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(0, n) / n))
    return d * math.sqrt(n)


def test_box_muller_is_standard_normal(orc):
    z = np.array([orc.normal3(7, s, p, 1) for s in range(4) for p in range(1000)])
    assert z.shape == (4000, 3)
    for c in range(3):
        # Kolmogorov-Smirnov statistic; 1.63 is the 1% critical value
        assert _ks_normal(z[:, c]) < 1.63
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.06
    assert abs(np.corrcoef(z[:, 0], z[:, 2])[0, 1]) < 0.06


def test_accept_uniform_is_uniform_and_keyed(orc):
    u = np.array([orc.accept_uniform(3, s, p) for s in range(4) for p in range(1000)])
    assert np.all((u > 0) & (u < 1))
    us = np.sort(u)
    d = np.max(np.abs(us - (np.arange(len(us)) + 0.5) / len(us)))
    assert d * math.sqrt(len(us)) < 1.63
    # distinct seeds, sweeps, particles and purposes draw distinct numbers
    assert orc.accept_uniform(3, 0, 0) != orc.accept_uniform(4, 0, 0)
    assert orc.accept_uniform(3, 0, 0) != orc.accept_uniform(3, 1, 0)
    assert orc.accept_uniform(3, 0, 0) != orc.accept_uniform(3, 0, 1)
    assert not np.allclose(orc.normal3(3, 0, 0, 1), orc.normal3(3, 0, 0, 0))


def test_seed_high_word_is_part_of_the_key(orc):
    assert orc.accept_uniform(1, 0, 0) != orc.accept_uniform(1 + (1 << 32), 0, 0)
