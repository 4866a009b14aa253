"""Pins of the oracle's K-step chain gradient (CPU).

The PyTorch restatement of the chain (oracle/chain.py) must give the NumPy
oracle's loss, its autograd gradient must match central finite differences of the
NumPy oracle's loss (eps = 1e-6 within 1e-6 relative; Richardson-extrapolated
eps = 2e-4 / 1e-4 within 1e-8), at
K = 0 it must reduce to the closed-form local-energy gradients, and the loss and
gradient must not depend on where the QR gauge fixing happens.
"""
import numpy as np
import pytest

from oracle import philox
from oracle.afqmc import Oracle
from oracle.chain import chain_loss, chain_vjp
from oracle.gradients import local_energy_vjp
from paper_2209_04015_b300.synthetic import make_system, perturbed_walkers


def setup(M=10, na=3, nb=2, X=13, W=3, K=7, seed=5):
    s = make_system(M, na, nb, X, seed=seed, decay="half", e0=0.3)
    phi0 = perturbed_walkers(s, W, eps=0.3, seed=seed + 1)
    xis = np.stack([philox.gaussian_fields(k, W, X, 1) for k in range(K)]) if K else \
        np.zeros((0, W, X))
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    return s, phi0, xis, g


def _loss(s, phi0, xis, g, h1=None, L=None, qr=3):
    return chain_loss(s.h1 if h1 is None else h1, s.L if L is None else L, s.e0, s.psi_a,
                      s.psi_b, phi0, xis, g, qr_period=qr)


@pytest.mark.parametrize("K", [0, 4, 7])
def test_torch_restatement_gives_the_oracle_loss(K):
    s, phi0, xis, g = setup(K=K)
    ref = _loss(s, phi0, xis, g)
    lt, *_ = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=3)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, e_shift=0.0)
    scale = np.sum(np.abs(g) * np.abs(orc.local_energy_of(phi0)[:, 3]))
    assert abs(lt - ref) <= 1e-12 * scale


@pytest.mark.parametrize("shape", [(10, 3, 2, 13, 3, 7), (8, 2, 0, 9, 2, 5)])
def test_chain_gradient_matches_finite_differences(shape):
    """eps = 1e-6 central differences within 1e-6, and a Richardson-extrapolated pair
    (eps = 2e-4, 1e-4; truncation O(eps^4)) within 1e-8."""
    M, na, nb, X, W, K = shape
    s, phi0, xis, g = setup(M, na, nb, X, W, K)
    _, gh, gL, gp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=3)
    rng = np.random.default_rng(11)

    def fd(f, eps):
        return (f(eps) - f(-eps)) / (2 * eps)

    def check(f, an, what):
        d6 = fd(f, 1e-6)
        assert abs(d6 - an) <= 1e-6 * abs(an), (what, d6, an)
        rich = (4 * fd(f, 1e-4) - fd(f, 2e-4)) / 3
        assert abs(rich - an) <= 1e-8 * abs(an), (what, rich, an)

    for _ in range(2):
        D = rng.standard_normal(s.h1.shape)
        D = D + D.T
        check(lambda e: _loss(s, phi0, xis, g, h1=s.h1 + e * D), np.sum(gh * D), "h1")
        D = rng.standard_normal(s.L.shape)
        D = D + D.transpose(0, 2, 1)
        check(lambda e: _loss(s, phi0, xis, g, L=s.L + e * D), np.sum(gL * D), "L")
        D = rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape)
        check(lambda e: _loss(s, phi0 + e * D, xis, g), np.sum(np.real(np.conj(gp) * D)), "phi")


def test_single_entries_of_phi0():
    s, phi0, xis, g = setup(K=5)
    _, _, _, gp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=3)
    eps = 1e-6
    for (z, p, j) in ((0, 0, 0), (1, 7, 4), (2, 3, 2)):
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            D = np.zeros_like(phi0)
            D[z, p, j] = unit
            fd = (_loss(s, phi0 + eps * D, xis, g) - _loss(s, phi0 - eps * D, xis, g)) / (2 * eps)
            assert abs(fd - part(gp[z, p, j])) <= 1e-6 * max(1.0, abs(fd))


def test_zero_steps_reduce_to_closed_forms():
    s, phi0, xis, g = setup(K=0)
    _, gh, gL, gp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=3)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, e_shift=0.0)
    rh, rL, rp = local_energy_vjp(orc, phi0, g)
    assert np.max(np.abs(gh - 0.5 * (rh + rh.T))) <= 1e-12 * np.max(np.abs(rh))
    assert np.max(np.abs(gL - 0.5 * (rL + rL.transpose(0, 2, 1)))) <= 1e-12 * np.max(np.abs(rL))
    assert np.max(np.abs(gp - rp)) <= 1e-12 * np.max(np.abs(rp))


def test_qr_gauge_does_not_change_loss_or_gradient():
    s, phi0, xis, g = setup(K=6)
    a = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=0)
    b = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=2)
    assert abs(a[0] - b[0]) <= 1e-12 * max(1.0, abs(a[0]))
    for x, y in zip(a[1:], b[1:]):
        assert np.max(np.abs(x - y)) <= 1e-10 * np.max(np.abs(x))
