"""PyTorch autograd bridge for the mixed local energy and K-step chains (FP64).

``local_energy(afq, phi, h1, L)`` returns E_L,z (complex, shape W) of the walkers
held by the context ``afq`` as a differentiable function of the walkers, the
one-body Hamiltonian and the Cholesky vectors (Sec. "Local energy"; the paper
leaves automatic differentiation to future work).  The context owns the values:
``phi``, ``h1`` and ``L`` must be the device tensors it was initialised with (or
hold the same values); they carry the autograd graph.  The backward runs the
closed-form adjoint kernels of libafqmc (afq_local_energy_backward_dev) and gives
PyTorch's complex convention, dLoss/dRe + i dLoss/dIm, for phi.

``chain_energy(afq, K, phi0, h1, L)`` runs K propagation steps from the context's
walkers (fixed fields; Philox by default) and returns E_L at the end; its backward
is afq_chain_backward_dev (checkpointed recomputation), with symmetrised gradients
for h1 and L and the gradient for the starting walkers phi0.
"""
from __future__ import annotations

import torch

from .afqmc import AfqContext


def _join(afq: AfqContext) -> None:
    # work on the context's stream must be complete before PyTorch's stream reads it
    if afq.stream:
        torch.cuda.ExternalStream(afq.stream).synchronize()


def _ptr(t):
    return None if t is None else t.data_ptr()


class LocalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, afq: AfqContext, phi, h1, L):
        W, M, N, X = afq.W, afq.M, afq.N, afq.X
        if tuple(phi.shape) != (W, M, N) or tuple(h1.shape) != (M, M) or \
                tuple(L.shape) != (X, M, M):
            raise ValueError("phi, h1 and L must have the context's shapes")
        e = torch.empty((W, 4), dtype=torch.complex128, device=phi.device)
        afq.local_energy_dev(e.data_ptr(), None)
        _join(afq)
        fctx.afq = afq
        fctx.step = afq.get_step()
        return e[:, 3].clone()

    @staticmethod
    def backward(fctx, gE):
        afq = fctx.afq
        if afq.get_step() != fctx.step:
            raise RuntimeError("the context has stepped since the forward pass")
        _, want_phi, want_h1, want_L = fctx.needs_input_grad
        dev = gE.device
        g = gE.to(torch.complex128).contiguous()
        dphi = torch.empty((afq.W, afq.M, afq.N), dtype=torch.complex128, device=dev) \
            if want_phi else None
        dh1 = torch.empty((afq.M, afq.M), dtype=torch.float64, device=dev) if want_h1 else None
        dL = torch.empty((afq.X, afq.M, afq.M), dtype=torch.float64, device=dev) if want_L \
            else None
        torch.cuda.current_stream(dev).synchronize()  # g is produced on PyTorch's stream
        afq.local_energy_backward_dev(g.data_ptr(), _ptr(dh1), _ptr(dL), _ptr(dphi))
        return None, dphi, dh1, dL


def local_energy(afq: AfqContext, phi, h1, L):
    """Differentiable E_L (complex, W) of the context's current walkers."""
    return LocalEnergy.apply(afq, phi, h1, L)


class ChainEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, afq: AfqContext, K: int, phi0, h1, L, fields=None):
        W, M, N, X = afq.W, afq.M, afq.N, afq.X
        if tuple(phi0.shape) != (W, M, N) or tuple(h1.shape) != (M, M) or \
                tuple(L.shape) != (X, M, M):
            raise ValueError("phi0, h1 and L must have the context's shapes")
        e = torch.empty((W, 4), dtype=torch.complex128, device=phi0.device)
        f = None
        if fields is not None:
            f = fields.to(device=phi0.device, dtype=torch.float64).contiguous()
            torch.cuda.current_stream(phi0.device).synchronize()
        afq.chain_forward_dev(K, _ptr(f), e.data_ptr())
        _join(afq)
        fctx.afq = afq
        return e[:, 3].clone()

    @staticmethod
    def backward(fctx, gE):
        afq = fctx.afq
        _, _, want_phi, want_h1, want_L, _ = fctx.needs_input_grad
        dev = gE.device
        g = gE.to(torch.complex128).contiguous()
        dphi = torch.empty((afq.W, afq.M, afq.N), dtype=torch.complex128, device=dev) \
            if want_phi else None
        dh1 = torch.empty((afq.M, afq.M), dtype=torch.float64, device=dev) if want_h1 else None
        dL = torch.empty((afq.X, afq.M, afq.M), dtype=torch.float64, device=dev) if want_L \
            else None
        torch.cuda.current_stream(dev).synchronize()
        afq.chain_backward_dev(g.data_ptr(), _ptr(dh1), _ptr(dL), _ptr(dphi))
        return None, None, dphi, dh1, dL, None


def chain_energy(afq: AfqContext, K: int, phi0, h1, L, fields=None):
    """Differentiable E_L (complex, W) after K steps from the context's walkers."""
    return ChainEnergy.apply(afq, K, phi0, h1, L, fields)
