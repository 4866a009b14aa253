"""Adjoint of the mixed local energy on the GPU against the oracle's closed forms.

The oracle's closed forms (oracle/gradients.py) are pinned by central finite
differences of the oracle's local energy; here the CUDA backward, through the C
ABI, must agree with them to 1e-10 relative (of the largest entry) in FP64.
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu
from oracle.gradients import local_energy_vjp
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _cot(W, seed, zero_except=None):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    if zero_except is not None:
        keep = np.zeros(W, dtype=bool)
        keep[list(zero_except)] = True
        g[~keep] = 0.0
    return g


def _close(a, b, tol=TOL):
    err = np.max(np.abs(a - b)) / np.max(np.abs(b))
    assert err <= tol, err


@pytest.mark.parametrize("shape", [(37, 5, 3, 71, 13), (29, 4, 0, 33, 5), (40, 7, 7, 97, 3)])
@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_backward_matches_closed_forms(shape, precision):
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=11, decay="geometric", e0=0.2)
    phi = perturbed_walkers(s, W, eps=0.4, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, precision=precision)
    g = _cot(W, 5)
    dh, dL, dp = ctx.local_energy_backward(g)
    rh, rL, rp = local_energy_vjp(orc, phi, g)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp, rp)


def test_backward_after_steps_and_qr():
    """Backward at walkers that have been propagated and re-orthonormalised."""
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)
    ctx, orc = make_pair(s, 9, phi=perturbed_walkers(s, 9, eps=0.3, seed=2), qr_period=3)
    ctx.propagate(nsteps=6)  # device Philox fields; the walkers are read back below
    phi = ctx.get_walkers()
    g = _cot(9, 8)
    dh, dL, dp = ctx.local_energy_backward(g)
    rh, rL, rp = local_energy_vjp(orc, phi, g)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp, rp)


def test_backward_c5_sampled_walkers():
    """Full 150-orbital, 750-vector, 256-walker shape; the cotangent is non-zero on
    three walkers only, so the oracle needs only those walkers."""
    s, c = make_config("c5")
    W = c["W"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=9)
    ctx, orc = make_pair(s, W, phi=phi)
    sample = [0, 131, W - 1]
    g = _cot(W, 6, zero_except=sample)
    dh, dL, dp = ctx.local_energy_backward(g)
    rh, rL, rp = local_energy_vjp(orc, phi[sample], g[sample])
    _close(dh, rh)
    _close(dL, rL)
    _close(dp[sample], rp)
    others = np.setdiff1d(np.arange(W), sample)
    assert np.max(np.abs(dp[others])) == 0.0


def test_backward_large_spin_block():
    """n_alpha M = 8400: more entries of theta per spin than one thread block holds,
    and a beta block of a different size."""
    s = make_system(300, 28, 2, 40, seed=1)
    W = 3
    phi = perturbed_walkers(s, W, eps=0.3, seed=5)
    ctx, orc = make_pair(s, W, phi=phi)
    g = _cot(W, 8)
    dh, dL, dp = ctx.local_energy_backward(g)
    rh, rL, rp = local_energy_vjp(orc, phi, g)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp, rp)


def test_torch_autograd_function():
    import torch
    from paper_2209_04015_b300.autograd import local_energy
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)
    W = 6
    phi_np = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc = make_pair(s, W, phi=phi_np)
    dev = torch.device("cuda:0")
    phi = torch.tensor(phi_np, device=dev, requires_grad=True)
    h1 = torch.tensor(s.h1, device=dev, requires_grad=True)
    L = torch.tensor(s.L, device=dev, requires_grad=True)
    E = local_energy(ctx, phi, h1, L)
    ref_e, _ = orc.local_energy()
    assert np.max(np.abs(E.detach().cpu().numpy() - ref_e[:, 3])) <= TOL * np.max(np.abs(ref_e[:, 3]))
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(W), rng.standard_normal(W)
    loss = (torch.tensor(a, device=dev) * E.real + torch.tensor(b, device=dev) * E.imag).sum()
    loss.backward()
    rh, rL, rp = local_energy_vjp(orc, phi_np, a + 1j * b)
    _close(h1.grad.cpu().numpy(), rh)
    _close(L.grad.cpu().numpy(), rL)
    _close(phi.grad.cpu().numpy(), rp)
