"""Split precision at FP64 quality (7 exact digits per operand, and 6) against the
oracle, and its two MMA issue forms against each other (GPU).

With split_slices = prop_slices = 7 every tensor-core contraction (force bias, VHS,
Taylor powers and one-body halves, stored exchange, overlap product) takes 55-bit
digit expansions of both operands with exact integer accumulation, so the split path
is held to the FP64 path's parity bar: walkers element by element, overlaps, weights
and every energy part within 1e-10 relative of the oracle.  6 digits (47 bits) are
held to the same bar.
"""
import numpy as np
import pytest

from gpu_common import assert_energy_parity, assert_state_parity, make_pair, need_gpu, rel, walker_rel
from oracle import philox
from paper_2209_04015_b300.synthetic import (gaussian_fields, make_config, make_system,
                                             perturbed_walkers, trial_walkers)

pytestmark = pytest.mark.gpu
TOL = 1e-10
DIGITS = dict(precision="split_bf16", split_slices=7, prop_slices=7)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("nd", [7, 6])
@pytest.mark.parametrize("shape", [(37, 5, 3, 71, 13), (50, 7, 0, 66, 9), (96, 20, 20, 101, 7)])
def test_seven_digit_split_matches_oracle_at_fp64_tolerance(shape, nd):
    """7 digits (55 bits), and 6 (47 bits, whose truncation lies at the FP64 path's own
    rounding level on these workloads), held to the FP64 parity bar."""
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=M + 3, decay="geometric", e0=0.37)
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc = make_pair(s, W, phi=phi, precision="split_bf16", split_slices=nd,
                         prop_slices=nd)
    assert ctx.exchange_algorithm() == "stored"
    digits, _ = ctx.prop_digits()
    assert digits[0] == digits[-1] == nd
    fields = np.stack([gaussian_fields(W, s.X, seed=70 + k) for k in range(6)])
    ctx.propagate(fields, 6)  # a QR after the fifth step
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


def test_seven_digit_split_c2_full_size_sampled_walkers():
    """The 100-orbital workload at full size (128 walkers, device Philox fields, 6 steps
    with a QR), 5 walkers re-run by the oracle alone."""
    s, c = make_config("c2")
    W, nsteps = c["W"], 6
    ctx, _ = make_pair(s, W, **DIGITS)
    ctx.propagate(None, nsteps)
    e, _ = ctx.local_energy()
    idx = np.array([0, 31, 64, 100, 127])
    from oracle.afqmc import Oracle
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005)
    orc.init_walkers(trial_walkers(s, len(idx)))
    orc.propagate([philox.gaussian_fields(k, W, s.X, 1)[idx] for k in range(nsteps)])
    assert walker_rel(ctx.get_walkers()[idx], orc.phi).max() <= TOL
    assert rel(ctx.get_weights()[idx], orc.w).max() <= TOL
    eref, _ = orc.local_energy()
    for k in range(4):
        scale = np.maximum(np.abs(eref[:, k]), 1e-3 * np.abs(eref[:, 3]))
        assert np.all(np.abs(e[idx, k] - eref[:, k]) <= TOL * scale), k


def test_seven_digits_need_the_stored_exchange():
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.afqmc import AFQ_ERR_ARG, AfqError
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    ctx = AfqContext(exchange="direct", **DIGITS)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    with pytest.raises(AfqError) as e:
        ctx.init_trial(s.psi_a, s.psi_b)
    assert e.value.code == AFQ_ERR_ARG


@pytest.mark.parametrize("shape", [(37, 5, 3, 71, 13), (96, 20, 20, 101, 7)])
def test_seven_digit_mma_forms_are_bit_identical(shape):
    """Every split GEMM at 7 digits with one MMA per A digit over the concatenated B
    digits (the default) against one MMA per digit pair (prop_kernel 'per_pair'): the
    same exact integer sums per TMEM accumulator, so the same bits after 6 steps with
    a QR, and the same energies."""
    from paper_2209_04015_b300 import AfqContext
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=M + 11, decay="geometric", e0=0.2)
    phi = perturbed_walkers(s, W, eps=0.3, seed=5)
    ctxs = []
    for kernel in ("per_pass", "per_pair"):
        ctx = AfqContext(dt=0.005, qr_period=5, prop_kernel=kernel, **DIGITS)
        ctx.init_hamiltonian(s.h1, s.L, s.e0)
        ctx.init_trial(s.psi_a, s.psi_b)
        ctx.init_walkers(W, phi)
        ctxs.append(ctx)
    fields = np.stack([gaussian_fields(W, s.X, seed=40 + k) for k in range(6)])
    for ctx in ctxs:
        ctx.propagate(fields, 6)
    a, b = ctxs
    assert np.array_equal(a.get_walkers(), b.get_walkers())
    assert np.array_equal(a.get_weights(), b.get_weights())
    assert np.array_equal(a.get_overlaps(), b.get_overlaps())
    ea, _ = a.local_energy()
    eb, _ = b.local_energy()
    assert np.array_equal(ea, eb)
    for ctx in ctxs:
        ctx.close()
