"""Population control (comb) and the block workflow on the GPU against the oracle,
through the C ABI.

The comb's parent indices are integers decided by FP64 comparisons of running
weight sums: with the same weights on both sides (set explicitly) they must agree
bit for bit, including a tooth that lands exactly on a running sum.  The gathered
walkers are bit-exact copies; steps after the comb (rebuilt theta, determinants and
Coulomb vector) and whole blocks then agree with the oracle at the FP64 tolerance.
"""
import numpy as np
import pytest

from gpu_common import assert_energy_parity, assert_state_parity, make_pair, need_gpu
from oracle import philox
from oracle.population import comb_parents, population_control, run_blocks
from paper_2209_04015_b300.synthetic import (gaussian_fields, make_config, make_system,
                                             perturbed_walkers)

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _system():
    return make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)


def _weights(W, seed):
    rng = np.random.default_rng(seed)
    w = rng.lognormal(0.0, 0.8, W)
    w[rng.choice(W, 3, replace=False)] = 0.0
    return w


def _pair_with_weights(s, W, w, **kw):
    phi = perturbed_walkers(s, W, eps=0.3, seed=5)
    ctx, orc = make_pair(s, W, phi=phi, **kw)
    ctx.init_walkers(W, phi, w)
    orc.init_walkers(phi, w)
    return ctx, orc


@pytest.mark.parametrize("u,w_cap", [(0.0, 0.0), (0.37, 0.0), (0.999, 0.0), (0.5, 1.5)])
def test_comb_parents_bit_exact_and_walkers_copied(u, w_cap):
    s = _system()
    W = 13
    w = _weights(W, 2)
    ctx, orc = _pair_with_weights(s, W, w)
    phi0, ov0 = ctx.get_walkers(), ctx.get_overlaps()
    parents = ctx.comb(u, w_cap)
    ref = population_control(orc, u, w_cap)
    assert np.array_equal(parents, ref)
    assert np.array_equal(ctx.get_walkers(), phi0[parents])
    assert np.array_equal(ctx.get_overlaps(), ov0[parents])
    _, T = comb_parents(w, u, w_cap)
    assert np.array_equal(ctx.get_weights().real, np.full(W, T / W))
    assert_energy_parity(ctx, orc, TOL)


def test_comb_tooth_on_a_running_sum():
    """Weights (0, 2, 0.5, 0, 1.5) at u = 0.5: the third tooth is 2.0 exactly, a
    running sum, and goes to the next walker with positive weight."""
    s = make_system(9, 2, 2, 12, seed=5, decay="geometric", e0=0.1)
    w = np.array([0.0, 2.0, 0.5, 0.0, 1.5])
    ctx, _ = _pair_with_weights(s, 5, w)
    phi = ctx.get_walkers()
    for u, expect in ((0.5, [1, 1, 2, 4, 4]), (0.0, [1, 1, 1, 2, 4])):
        ctx.init_walkers(5, phi, w)
        assert ctx.comb(u).tolist() == expect


def test_steps_after_the_comb_match_the_oracle():
    s = _system()
    W = 11
    ctx, orc = _pair_with_weights(s, W, _weights(W, 6))
    ctx.comb(0.61)
    population_control(orc, 0.61)
    fields = np.stack([gaussian_fields(W, s.X, seed=300 + k) for k in range(6)])
    ctx.propagate(fields, 6)
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_run_blocks_is_the_step_sequence(precision):
    """The native block driver equals the same calls made one by one."""
    s, c = make_config("c1")
    W = c["W"]
    u = np.array([0.3, 0.75, 0.1])
    a, _ = make_pair(s, W, precision=precision)
    b, _ = make_pair(s, W, precision=precision)
    sums = a.run_blocks(3, 4, u=u)
    for k in range(3):
        b.propagate(None, 4)
        e, _ = b.local_energy()
        wb = b.get_weights()
        ref = np.array([wb.sum().real, wb.sum().imag, (wb * e[:, 3]).sum().real,
                        (wb * e[:, 3]).sum().imag])
        np.testing.assert_allclose(sums[k], ref, rtol=1e-13, atol=1e-13)
        b.comb(u[k])
    assert np.array_equal(a.get_walkers(), b.get_walkers())
    assert np.array_equal(a.get_weights(), b.get_weights())


@pytest.mark.parametrize("feedback,cap", [(False, 0.0), (True, 0.0), (True, 1.05)])
def test_run_blocks_matches_oracle_blocks(feedback, cap):
    s, c = make_config("c1")
    W = c["W"]
    u = np.array([0.42, 0.05, 0.9, 0.5])
    ctx, orc = make_pair(s, W, seed=1)
    sums = ctx.run_blocks(4, 5, u=u, w_cap=cap, shift_feedback=feedback)
    ref = run_blocks(orc, lambda k: philox.gaussian_fields(k, W, s.X, 1), 4, 5, u=u,
                     w_cap=cap, shift_feedback=feedback)
    np.testing.assert_allclose(sums, ref, rtol=TOL, atol=TOL * np.abs(ref).max())
    assert_state_parity(ctx, orc, TOL)
    assert ctx.get_e_shift() == pytest.approx(orc.e_shift, rel=TOL)
    if feedback:  # the shift follows the last block, and later steps use it
        expect = ref[-1, 2] / ref[-1, 0] - np.log(ref[-1, 0] / W) / (orc.dt * 5)
        assert orc.e_shift == pytest.approx(expect, rel=1e-14)
        fields = np.stack([gaussian_fields(W, s.X, seed=500 + k) for k in range(3)])
        ctx.propagate(fields, 3)
        orc.propagate(list(fields))
        assert_state_parity(ctx, orc, TOL)


def test_shift_feedback_keeps_the_total_weight_bounded():
    """Without feedback the weights of the synthetic system grow by ~e^{dt steps dE}
    (E_shift = E_HF lies far above the projected energy); with the population feedback
    the total weight stays near W."""
    s, c = make_config("c1")
    W = c["W"]
    a, _ = make_pair(s, W, seed=1)
    b, _ = make_pair(s, W, seed=1)
    u = np.random.default_rng(3).random(40)
    free = a.run_blocks(40, 25, u=u)
    fed = b.run_blocks(40, 25, u=u, shift_feedback=True)
    assert free[-1, 0] > 1e6 * W
    assert np.all(fed[:, 0] < 3 * W) and np.all(fed[1:, 0] > W / 3)


def test_comb_errors_are_reported():
    from paper_2209_04015_b300 import AfqError
    s = _system()
    W = 6
    ctx, _ = _pair_with_weights(s, W, _weights(W, 1))
    for u, cap in ((1.0, 0.0), (-0.1, 0.0), (float("nan"), 0.0), (0.5, -1.0)):
        with pytest.raises(AfqError) as e:
            ctx.comb(u, cap)
        assert e.value.code == 1  # AFQ_ERR_ARG
    phi = ctx.get_walkers()
    ctx.init_walkers(W, phi, np.zeros(W))
    with pytest.raises(AfqError) as e:
        ctx.comb(0.5)
    assert e.value.code == 4  # AFQ_ERR_NAN: no positive total weight
    assert np.array_equal(ctx.get_walkers(), phi)  # walkers kept
    fp, _ = make_pair(s, W, free_projection=True)
    with pytest.raises(AfqError) as e:
        fp.comb(0.5)
    assert e.value.code == 5  # AFQ_ERR_STATE
    with pytest.raises(AfqError) as e:
        ctx.run_blocks(2, 0)
    assert e.value.code == 1


def test_run_blocks_free_projection_with_shift_feedback():
    """Complex weights (free projection): no comb, the shift feedback takes the real
    part of the complex block estimate and |sum w| as the total weight."""
    s, c = make_config("c1")
    W = c["W"]
    ctx, orc = make_pair(s, W, seed=1, free_projection=True, dt=0.01)
    sums = ctx.run_blocks(3, 4, shift_feedback=True)
    ref = run_blocks(orc, lambda k: philox.gaussian_fields(k, W, s.X, 1), 3, 4,
                     shift_feedback=True)
    np.testing.assert_allclose(sums, ref, rtol=TOL, atol=TOL * np.abs(ref).max())
    assert_state_parity(ctx, orc, TOL)
    assert ctx.get_e_shift() == pytest.approx(orc.e_shift, rel=TOL)


def test_comb_single_walker_and_zero_blocks():
    s = _system()
    ctx, orc = _pair_with_weights(s, 1, np.array([2.5]))
    phi = ctx.get_walkers()
    assert ctx.comb(0.7).tolist() == [0]
    assert np.array_equal(ctx.get_walkers(), phi)
    assert ctx.get_weights().real.tolist() == [2.5]
    assert ctx.run_blocks(0, 5).shape == (0, 4)
    assert ctx.get_step() == 0
