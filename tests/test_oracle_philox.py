"""Pins of the oracle's Philox4x32-10 and Box-Muller fields (CPU only)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[:4], v[4:6], v[6:]))
    return rows


@pytest.mark.parametrize("ctr,key,out", load_kat())
def test_philox_known_answers(ctr, key, out):
    got = philox.philox4x32_10(np.array([ctr], dtype=np.uint64), tuple(key))[0]
    assert [int(x) for x in got] == out


def test_uniforms_are_exact_53_bit_and_in_unit_interval():
    w = philox.field_words(3, 16, 50, seed=1)
    u = philox.field_uniforms(3, 16, 50, seed=1)
    assert u.min() > 0.0 and u.max() <= 1.0
    k = np.round(u * 2.0 ** 53) - 1
    # the 53-bit integer is rebuilt exactly from the two words it came from
    hi = (w[..., 0].astype(np.uint64) >> np.uint64(5)).astype(np.float64)
    lo = (w[..., 1].astype(np.uint64) >> np.uint64(6)).astype(np.float64)
    assert np.array_equal(k[..., 0], hi * 2.0 ** 26 + lo)
    # extreme words map to the ends of (0, 1]
    assert philox.uniforms53(np.array([0], np.uint32), np.array([0], np.uint32))[0] == 2.0 ** -53
    top = np.array([0xFFFFFFFF], np.uint32)
    assert philox.uniforms53(top, top)[0] == 1.0


def test_counters_distinct_per_step_walker_pair():
    a = philox.field_words(0, 4, 10, seed=1)
    b = philox.field_words(1, 4, 10, seed=1)
    c = philox.field_words(0, 4, 10, seed=2)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    flat = a.reshape(-1, 4)
    assert len({tuple(r) for r in flat}) == flat.shape[0]


def test_gaussian_fields_are_standard_normal():
    xi = philox.gaussian_fields(7, 512, 400, seed=1).ravel()
    assert abs(xi.mean()) < 5.0 / np.sqrt(xi.size)
    assert abs(xi.var() - 1.0) < 8.0 * np.sqrt(2.0 / xi.size)
    assert stats.kstest(xi, "norm").pvalue > 1e-4


def test_odd_field_count_takes_first_of_pair():
    even = philox.gaussian_fields(2, 3, 6, seed=9)
    odd = philox.gaussian_fields(2, 3, 5, seed=9)
    assert np.array_equal(odd, even[:, :5])
