"""Pins of the oracle's comb (population control) against what the resampling must
satisfy whatever its implementation: equal weights leave the population alone,
every walker gets floor or ceil of W w_z / T copies, the copy counts are unbiased
over the offset u, zero weights are never copied, the cap bounds the copies, and
estimators keep their expectation.  Brute force on tiny inputs enumerates the teeth
by hand."""
import numpy as np
import pytest

from oracle.afqmc import Oracle
from oracle.population import block_sums, comb_parents, population_control
from paper_2209_04015_b300.synthetic import make_system, perturbed_walkers


def _weights(W, seed, zeros=0):
    rng = np.random.default_rng(seed)
    w = rng.lognormal(0.0, 0.7, W)
    if zeros:
        w[rng.choice(W, zeros, replace=False)] = 0.0
    return w


@pytest.mark.parametrize("u", [0.0, 0.25, 0.5, 0.999999])
def test_equal_weights_keep_every_walker(u):
    for W in (1, 7, 64):
        parents, T = comb_parents(np.full(W, 0.37), u)
        assert np.array_equal(parents, np.arange(W))
        assert T == pytest.approx(0.37 * W, rel=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_copies_are_floor_or_ceil_of_expected(seed):
    W = 50
    w = _weights(W, seed, zeros=6)
    for u in np.random.default_rng(100 + seed).random(8):
        parents, T = comb_parents(w, u)
        n = np.bincount(parents, minlength=W)
        expect = W * w / T
        assert n.sum() == W
        assert np.all(n >= np.floor(expect) - 1e-9) and np.all(n <= np.ceil(expect) + 1e-9)
        assert np.all(n[w == 0.0] == 0)


def test_copy_counts_are_unbiased_over_the_offset():
    """E_u[n_z] = W w_z / T exactly for u uniform on [0, 1); a midpoint grid of
    offsets reproduces it to O(1 / grid)."""
    W = 23
    w = _weights(W, 7, zeros=3)
    grid = (np.arange(4000) + 0.5) / 4000
    counts = np.zeros(W)
    for u in grid:
        parents, T = comb_parents(w, u)
        counts += np.bincount(parents, minlength=W)
    np.testing.assert_allclose(counts / grid.size, W * w / w.sum(), atol=2e-3)


def test_cap_bounds_the_copies_of_a_heavy_walker():
    W = 20
    w = _weights(W, 3)
    w[4] = 1e3
    cap = 2.0
    capped = np.minimum(w, cap)
    for u in (0.1, 0.6):
        parents, T = comb_parents(w, u, w_cap=cap)
        assert T == pytest.approx(capped.sum(), rel=1e-14)
        assert np.sum(parents == 4) <= np.ceil(W * cap / T)
    with pytest.raises(ValueError):
        comb_parents(np.zeros(5), 0.3)


def test_brute_force_teeth_on_tiny_inputs():
    w = np.array([0.0, 2.0, 0.5, 0.0, 1.5])  # T = 4, spacing 0.8
    # teeth at 0.8 (k + u); intervals [0,0) [0,2) [2,2.5) [2.5,2.5) [2.5,4); at u = 0.5
    # the third tooth is 2.5 * 0.8 = 2.0 exactly (in FP64 too), a running sum, so it
    # belongs to the next walker with positive weight
    for u, expect in ((0.0, [1, 1, 1, 2, 4]), (0.5, [1, 1, 2, 4, 4]), (0.9, [1, 1, 2, 4, 4])):
        parents, _ = comb_parents(w, u)
        assert parents.tolist() == expect, (u, parents)


def test_population_control_keeps_estimator_expectation():
    """Over the offset, sum_k (T / W) E_L(parent_k) averages to sum_z w_z E_L,z; the new
    walkers are exact copies of their parents (matrices, overlaps, energies)."""
    s = make_system(9, 2, 2, 12, seed=5, decay="geometric", e0=0.1)
    W = 12
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b)
    orc.init_walkers(perturbed_walkers(s, W, eps=0.4, seed=2), w=_weights(W, 9, zeros=2))
    before = block_sums(orc)
    e = orc.local_energy_of(orc.phi)[:, 3]
    phi0, ov0, w0 = orc.phi.copy(), orc.ovlp.copy(), orc.w.copy()
    acc = 0.0 + 0.0j
    grid = (np.arange(2000) + 0.5) / 2000
    for u in grid:
        parents, T = comb_parents(w0, u)
        acc += np.sum((T / W) * e[parents])
    assert abs(acc / grid.size - (before[2] + 1j * before[3])) < 2e-3 * abs(before[2])
    parents = population_control(orc, 0.3)
    assert np.array_equal(orc.phi, phi0[parents]) and np.array_equal(orc.ovlp, ov0[parents])
    np.testing.assert_allclose(orc.w, np.full(W, w0.sum() / W), rtol=1e-15)
    np.testing.assert_array_equal(orc.local_energy_of(orc.phi)[:, 3], e[parents])
