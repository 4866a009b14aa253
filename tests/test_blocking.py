"""Reblocking analysis (host logic) against closed forms: independent data give the
plain standard error sigma / sqrt(n); an AR(1) series x_t = rho x_{t-1} + e_t with
unit variance has the standard error of its mean sqrt((1 + rho) / ((1 - rho) n)) for
long series; each level's block means are the means of consecutive 2^level points."""
import numpy as np
import pytest

from paper_2209_04015_b300.blocking import (block_energies, estimate, optimal_level,
                                            reblock)


def _ar1(n, rho, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n) * np.sqrt(1.0 - rho * rho)
    x = np.empty(n)
    x[0] = rng.standard_normal()
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    return x


def test_levels_are_means_of_consecutive_blocks():
    x = np.random.default_rng(1).standard_normal(1000)
    table = reblock(x)
    for t in table:
        B = t.block
        m = x.size // B
        means = x[: m * B].reshape(m, B).mean(axis=1)
        assert t.n == m
        assert t.mean == pytest.approx(means.mean(), rel=1e-13, abs=1e-15)
        assert t.stderr == pytest.approx(means.std(ddof=1) / np.sqrt(m), rel=1e-12)
    assert table[0].mean == pytest.approx(x.mean(), rel=1e-14, abs=1e-16)


@pytest.mark.parametrize("seed", range(4))
def test_independent_data_give_sigma_over_sqrt_n(seed):
    n, sigma = 2 ** 14, 1.7
    x = 3.0 + sigma * np.random.default_rng(seed).standard_normal(n)
    est = estimate(x)
    # an error estimate from m block means is itself uncertain by 1 / sqrt(2 (m - 1)):
    # allow four of those
    m = est.table[est.level].n
    exact = sigma / np.sqrt(n)
    assert abs(est.error - exact) <= 4 * exact / np.sqrt(2 * (m - 1))
    assert abs(est.mean - 3.0) < 5 * exact


def test_correlated_data_reach_the_ar1_error():
    n, rho = 2 ** 16, 0.8
    exact = np.sqrt((1 + rho) / ((1 - rho) * n))
    errs = []
    for seed in range(6):
        est = estimate(_ar1(n, rho, seed))
        assert est.level is not None and est.level >= 3  # naive level 0 is 3x too small
        errs.append(est.error)
        m = est.table[est.level].n
        # four statistical sigmas of the estimate plus 10% for the finite block length
        assert abs(est.error - exact) <= (4 / np.sqrt(2 * (m - 1)) + 0.1) * exact
    assert np.mean(errs) == pytest.approx(exact, rel=0.12)
    assert reblock(_ar1(n, rho, 0))[0].stderr < 0.5 * exact


def test_discard_and_short_series():
    x = np.concatenate([np.full(50, 10.0), np.random.default_rng(3).standard_normal(4096)])
    est = estimate(x, discard=50)
    assert est.n == 4096 and abs(est.mean) < 0.1
    assert optimal_level(reblock(np.ones(8)), 8) == 0
    with pytest.raises(ValueError):
        estimate(np.ones(3), discard=2)


def test_block_energies_from_sums():
    sums = np.array([[2.0, 0.0, -3.0, 0.5], [4.0, 1.0, -8.0, 2.0]])
    np.testing.assert_allclose(block_energies(sums), [-1.5, ((-8 + 2j) / (4 + 1j)).real])
