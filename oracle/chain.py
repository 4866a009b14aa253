"""Gradient of a K-step phaseless chain (oracle side; test infrastructure only).

The paper leaves automatic differentiation to future work (Sec. "Customized mixed
estimators").  The objective differentiated here is

    Loss = sum_z Re(conj(g_z) E_L(Phi_z^K)),

where Phi^K comes from K steps of the propagation of Sec. "Review of AFQMC"
(B(y) Phi = P T_n(A) P Phi, A = i sqrt(dt) sum_g y_g L_g, y = xi - xbar,
xbar = -i sqrt(dt) (c - vbar), QR every qr_period steps) with the N(0,1) fields xi
held fixed (reparameterisation).  The force bias is a function of Phi and L and is
differentiated through; the weights are not part of the objective (the phaseless
max(0, cos) is not differentiable); vbar, L~ and P are functions of h1 and L.
h1 and L are symmetric, so their gradients are reported symmetrised,
(grad + grad^T) / 2: the gradient with respect to symmetric perturbations.

Two forward implementations live here: ``chain_loss`` drives the NumPy oracle
(oracle.afqmc), and ``chain_vjp`` restates the same steps with PyTorch CPU
operations in float64 / complex128 so that autograd (a library primitive)
supplies the gradient.  Tests pin the second against the first: equal losses,
central finite differences of ``chain_loss``, the closed forms at K = 0, and the
invariance of the loss under the QR gauge.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .afqmc import Oracle


def chain_loss(h1, L, e0, psi_a, psi_b, phi0, xis, g, dt=0.005, order=6, qr_period=5):
    """Loss through the NumPy oracle (fields xis: K x W x X)."""
    orc = Oracle(h1, L, e0, psi_a, psi_b, dt=dt, taylor_order=order, qr_period=qr_period,
                 e_shift=0.0)
    orc.init_walkers(phi0)
    orc.propagate(list(xis))
    e = orc.local_energy_of(orc.phi)[:, 3]
    return float(np.sum(np.real(np.conj(g) * e)))


def _qr_positive(block):
    """Q of the QR of each walker's block with diag(R) real and positive."""
    Q, R = torch.linalg.qr(block, mode="reduced")
    d = torch.diagonal(R, dim1=-2, dim2=-1)
    return Q * (d / d.abs()).unsqueeze(-2)


def _theta(psi, blk):
    S = torch.einsum("pi,zpj->zij", psi.to(blk.dtype), blk)
    return torch.linalg.solve(S.transpose(-1, -2), blk.transpose(-1, -2)).transpose(-1, -2)


def chain_forward_torch(h1, L, e0, psi_a, psi_b, phi0, xis, dt=0.005, order=6, qr_period=5):
    """E_L (W complex) after K steps, as a PyTorch graph in h1, L and phi0."""
    na = psi_a.shape[1]
    pa = torch.as_tensor(psi_a, dtype=torch.float64)
    pb = torch.as_tensor(psi_b, dtype=torch.float64)
    sq = math.sqrt(dt)
    Lt_a = torch.einsum("pi,gpr->gir", pa, L)
    Lt_b = torch.einsum("pi,gpr->gir", pb, L)
    vbar = torch.einsum("gir,ri->g", Lt_a, pa) + torch.einsum("gir,ri->g", Lt_b, pb)
    hpp = h1 - 0.5 * torch.einsum("gpr,grq->pq", L, L) + torch.einsum("g,gpq->pq", vbar, L)
    # P = exp(-dt h''/2) from the eigenpairs of the symmetric h'' (as in the NumPy
    # oracle); autograd differentiates through the eigendecomposition
    evals, U = torch.linalg.eigh(0.5 * (hpp + hpp.T))
    P = ((U * torch.exp(-0.5 * dt * evals)) @ U.T).to(torch.complex128)
    Lc = L.to(torch.complex128)

    def thetas(phi):
        ta = _theta(pa, phi[:, :, :na]) if na else None
        tb = _theta(pb, phi[:, :, na:]) if psi_b.shape[1] else None
        return ta, tb

    def coulomb(ta, tb):
        c = 0
        if ta is not None:
            c = c + torch.einsum("gjp,zpj->zg", Lt_a.to(torch.complex128), ta)
        if tb is not None:
            c = c + torch.einsum("gjp,zpj->zg", Lt_b.to(torch.complex128), tb)
        return c

    phi = phi0
    for k in range(len(xis)):
        ta, tb = thetas(phi)
        c = coulomb(ta, tb)
        xbar = -1j * sq * (c - vbar.to(torch.complex128))
        y = torch.as_tensor(xis[k], dtype=torch.complex128) - xbar
        A = 1j * sq * torch.einsum("zg,gpq->zpq", y, Lc)
        term = P @ phi
        out = term
        for n in range(1, order + 1):
            term = (A @ term) / n
            out = out + term
        phi = P @ out
        if qr_period > 0 and (k + 1) % qr_period == 0:
            blocks = []
            if na:
                blocks.append(_qr_positive(phi[:, :, :na]))
            if psi_b.shape[1]:
                blocks.append(_qr_positive(phi[:, :, na:]))
            phi = torch.cat(blocks, dim=2)
    ta, tb = thetas(phi)
    c = coulomb(ta, tb)
    e1 = 0
    ek = 0
    for psi, th, Lt in ((pa, ta, Lt_a), (pb, tb, Lt_b)):
        if th is None:
            continue
        ht = (psi.T @ h1).to(torch.complex128)
        e1 = e1 + torch.einsum("jq,zqj->z", ht, th)
        T = torch.einsum("gip,zpj->zgij", Lt.to(torch.complex128), th)
        ek = ek - 0.5 * torch.einsum("zgij,zgji->z", T, T)
    ej = 0.5 * torch.sum(c * c, dim=1)
    return e0 + e1 + ej + ek


def chain_vjp(h1, L, e0, psi_a, psi_b, phi0, xis, g, dt=0.005, order=6, qr_period=5):
    """(loss, grad h1 (sym), grad L (sym), grad phi0) by PyTorch autograd.

    grad phi0 follows PyTorch's complex convention dLoss/dRe + i dLoss/dIm.
    """
    th1 = torch.tensor(np.asarray(h1, dtype=np.float64), requires_grad=True)
    tL = torch.tensor(np.asarray(L, dtype=np.float64), requires_grad=True)
    tphi = torch.tensor(np.asarray(phi0, dtype=np.complex128), requires_grad=True)
    e = chain_forward_torch(th1, tL, e0, psi_a, psi_b, tphi, xis, dt, order, qr_period)
    loss = torch.sum(torch.real(torch.conj(torch.as_tensor(g, dtype=torch.complex128)) * e))
    loss.backward()
    gh = th1.grad.numpy()
    gL = tL.grad.numpy()
    return (float(loss.detach()), 0.5 * (gh + gh.T), 0.5 * (gL + gL.transpose(0, 2, 1)),
            tphi.grad.numpy())
