"""Adjoint of a K-step chain on the GPU against the oracle's autograd gradient.

The oracle's chain gradient (oracle/chain.py) is pinned on the CPU by finite
differences of the NumPy oracle.  Here the CUDA chain backward, through the C ABI,
must match it within 1e-9 relative (of each output's largest entry), and central
finite differences of the CUDA forward itself (eps = 1e-6) within 1e-6.
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu
from oracle import philox
from oracle.chain import chain_vjp
from oracle.gradients import local_energy_vjp
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _close(a, b, tol=TOL):
    err = np.max(np.abs(a - b)) / np.max(np.abs(b))
    assert err <= tol, err


def _case(M, na, nb, X, W, seed=4):
    s = make_system(M, na, nb, X, seed=seed, decay="geometric", e0=0.37)
    phi0 = perturbed_walkers(s, W, eps=0.3, seed=seed + 1)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    return s, phi0, g


def _fields(K, W, X, seed=1):
    return np.stack([philox.gaussian_fields(k, W, X, seed) for k in range(K)])


@pytest.mark.parametrize("shape,K,qr", [((37, 5, 3, 71, 6), 7, 3), ((29, 4, 0, 33, 5), 9, 0),
                                        ((40, 6, 6, 97, 4), 10, 5)])
def test_chain_backward_matches_oracle(shape, K, qr):
    s, phi0, g = _case(*shape)
    W = shape[4]
    ctx, _ = make_pair(s, W, phi=phi0, qr_period=qr)
    ctx.chain_forward(K)  # device Philox fields of steps 0 .. K-1
    dh, dL, dp = ctx.chain_backward(g)
    xis = _fields(K, W, s.X)
    _, rh, rL, rp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=qr)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp, rp)


def test_chain_energy_and_explicit_fields():
    s, phi0, g = _case(37, 5, 3, 71, 6)
    rng = np.random.default_rng(3)
    xis = rng.standard_normal((6, 6, s.X))
    ctx, orc = make_pair(s, 6, phi=phi0, qr_period=4)
    e = ctx.chain_forward(6, xis)
    orc.propagate(list(xis))
    eref = orc.local_energy_of(orc.phi)
    assert np.max(np.abs(e[:, 3] - eref[:, 3])) <= 1e-10 * np.max(np.abs(eref[:, 3]))
    dh, dL, dp = ctx.chain_backward(g)
    _, rh, rL, rp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, xis, g, qr_period=4)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp, rp)


def test_zero_steps_equal_local_energy_backward():
    s, phi0, g = _case(37, 5, 3, 71, 6)
    ctx, orc = make_pair(s, 6, phi=phi0)
    ctx.chain_forward(0)
    dh, dL, dp = ctx.chain_backward(g)
    rh, rL, rp = local_energy_vjp(orc, phi0, g)
    _close(dh, 0.5 * (rh + rh.T), 1e-10)
    _close(dL, 0.5 * (rL + rL.transpose(0, 2, 1)), 1e-10)
    _close(dp, rp, 1e-10)


def test_chain_gradient_matches_gpu_finite_differences():
    """Central differences (eps = 1e-6) of the CUDA forward along random directions."""
    s, phi0, g = _case(24, 3, 2, 31, 3)
    K, qr, eps = 6, 3, 1e-6
    ctx, _ = make_pair(s, 3, phi=phi0, qr_period=qr)
    ctx.chain_forward(K)
    dh, dL, dp = ctx.chain_backward(g)

    def loss(h1=None, L=None, phi=None):
        from paper_2209_04015_b300 import AfqContext
        c = AfqContext(qr_period=qr)
        c.init_hamiltonian(s.h1 if h1 is None else h1, s.L if L is None else L, s.e0)
        c.init_trial(s.psi_a, s.psi_b)
        c.init_walkers(3, phi0 if phi is None else phi)
        e = c.chain_forward(K)
        c.close()
        return float(np.sum(np.real(np.conj(g) * e[:, 3])))

    rng = np.random.default_rng(2)
    D = rng.standard_normal(s.h1.shape)
    D = D + D.T
    fd = (loss(h1=s.h1 + eps * D) - loss(h1=s.h1 - eps * D)) / (2 * eps)
    assert abs(fd - np.sum(dh * D)) <= 1e-6 * abs(fd)
    D = rng.standard_normal(s.L.shape)
    D = D + D.transpose(0, 2, 1)
    fd = (loss(L=s.L + eps * D) - loss(L=s.L - eps * D)) / (2 * eps)
    assert abs(fd - np.sum(dL * D)) <= 1e-6 * abs(fd)
    D = rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape)
    fd = (loss(phi=phi0 + eps * D) - loss(phi=phi0 - eps * D)) / (2 * eps)
    assert abs(fd - np.sum(np.real(np.conj(dp) * D))) <= 1e-6 * abs(fd)


def test_backward_leaves_the_context_state_alone():
    s, phi0, g = _case(37, 5, 3, 71, 6)
    a, _ = make_pair(s, 6, phi=phi0, qr_period=3)
    b, _ = make_pair(s, 6, phi=phi0, qr_period=3)
    a.chain_forward(5)
    b.chain_forward(5)
    a.chain_backward(g)
    for get in ("get_walkers", "get_weights", "get_overlaps", "get_force_bias"):
        assert np.array_equal(getattr(a, get)(), getattr(b, get)()), get
    a.propagate(nsteps=2)
    b.propagate(nsteps=2)
    assert np.array_equal(a.get_walkers(), b.get_walkers())
    assert np.array_equal(a.local_energy()[0], b.local_energy()[0])


def test_chain_errors():
    from paper_2209_04015_b300.afqmc import AFQ_ERR_ARG, AFQ_ERR_STATE, AfqError
    s, phi0, g = _case(20, 3, 2, 21, 3)
    ctx, _ = make_pair(s, 3, phi=phi0)
    with pytest.raises(AfqError) as e:
        ctx.chain_backward(g)
    assert e.value.code == AFQ_ERR_STATE
    ctx.chain_forward(3)
    ctx.propagate(nsteps=1)
    with pytest.raises(AfqError) as e:
        ctx.chain_backward(g)
    assert e.value.code == AFQ_ERR_STATE
    ctx.chain_forward(2)
    ctx.orthogonalise()
    with pytest.raises(AfqError) as e:
        ctx.chain_backward(g)
    assert e.value.code == AFQ_ERR_STATE
    mixed, _ = make_pair(s, 3, phi=phi0, precision="split_bf16")
    with pytest.raises(AfqError) as e:
        mixed.chain_forward(2)
    assert e.value.code == AFQ_ERR_ARG
    capped, _ = make_pair(s, 3, phi=phi0, fb_cap=1.0)
    with pytest.raises(AfqError) as e:
        capped.chain_forward(2)
    assert e.value.code == AFQ_ERR_ARG


def test_c5_chain_sampled_walkers():
    """150 orbitals, 15+15 electrons, 750 vectors, 256 walkers, K = 20 with QR every 5
    steps; the cotangent is non-zero on two walkers, which the oracle follows alone
    (walkers are independent when the weights are not part of the objective)."""
    s, c = make_config("c5")
    W, K = c["W"], c["steps"]
    phi0 = perturbed_walkers(s, W, eps=0.3, seed=9)
    ctx, _ = make_pair(s, W, phi=phi0, qr_period=5)
    ctx.chain_forward(K)
    sample = [3, W - 2]
    g = np.zeros(W, dtype=np.complex128)
    g[sample] = [0.7 - 0.2j, -0.4 + 1.1j]
    dh, dL, dp = ctx.chain_backward(g)
    xis = _fields(K, W, s.X)[:, sample]
    _, rh, rL, rp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0[sample], xis, g[sample],
                              qr_period=5)
    _close(dh, rh)
    _close(dL, rL)
    _close(dp[sample], rp)
    others = np.setdiff1d(np.arange(W), sample)
    assert np.max(np.abs(dp[others])) == 0.0


def test_torch_chain_function():
    import torch
    from paper_2209_04015_b300.autograd import chain_energy
    s, phi0, g = _case(37, 5, 3, 71, 6)
    K = 6
    ctx, _ = make_pair(s, 6, phi=phi0, qr_period=3)
    dev = torch.device("cuda:0")
    phi = torch.tensor(phi0, device=dev, requires_grad=True)
    h1 = torch.tensor(s.h1, device=dev, requires_grad=True)
    L = torch.tensor(s.L, device=dev, requires_grad=True)
    E = chain_energy(ctx, K, phi, h1, L)
    loss = torch.sum(torch.real(torch.conj(torch.tensor(g, device=dev)) * E))
    loss.backward()
    lref, rh, rL, rp = chain_vjp(s.h1, s.L, s.e0, s.psi_a, s.psi_b, phi0, _fields(K, 6, s.X), g,
                                 qr_period=3)
    assert abs(loss.item() - lref) <= 1e-10 * np.sum(np.abs(g) * np.abs(E.detach().cpu().numpy()))
    _close(h1.grad.cpu().numpy(), rh)
    _close(L.grad.cpu().numpy(), rL)
    _close(phi.grad.cpu().numpy(), rp)
