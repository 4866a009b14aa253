"""The complex-gradient convention the autograd bridge returns, checked on PyTorch
itself (CPU): for a holomorphic f and Loss = Re(conj(g) f(z)), PyTorch's z.grad is
g conj(f'(z)) = dLoss/dRe z + i dLoss/dIm z, and the grad_output it passes for a
complex output E is dLoss/dRe E + i dLoss/dIm E."""
import numpy as np
import torch


def test_holomorphic_vjp_convention():
    rng = np.random.default_rng(0)
    z0 = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    g = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    z = torch.tensor(z0, requires_grad=True)
    f = z ** 3
    loss = (torch.tensor(g).conj() * f).real.sum()
    loss.backward()
    assert np.allclose(z.grad.numpy(), g * np.conj(3 * z0 ** 2), rtol=1e-13, atol=0)


def test_grad_output_convention():
    seen = {}

    class Probe(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            return x.clone()

        @staticmethod
        def backward(ctx, go):
            seen["go"] = go.clone()
            return go

    x = torch.tensor([1.0 + 2.0j, -0.5 + 0.25j], requires_grad=True)
    e = Probe.apply(x)
    (3.0 * e.real + 5.0 * e.imag).sum().backward()
    assert np.allclose(seen["go"].numpy(), [3.0 + 5.0j, 3.0 + 5.0j])
