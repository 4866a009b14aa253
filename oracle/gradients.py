"""Gradients of the mixed local energy (oracle side; test infrastructure only).

The paper leaves automatic differentiation to future work (Sec. "Customized mixed
estimators", last paragraph).  These are closed forms derived from the local
energy of Sec. "Local energy" (E_L = e0 + E1 + EJ + EK with theta = Phi
(Psi^T Phi)^-1), written as plainly as possible.  Conventions:

* E_z is complex and holomorphic in Phi_z.  For a cotangent g_z (PyTorch's
  convention: g = dLoss/dRe E + i dLoss/dIm E) the real loss has
    dLoss/dh1   = Re sum_z conj(g_z) dE_z/dh1,
    dLoss/dL_g  = Re sum_z conj(g_z) dE_z/dL_g,
    dLoss/dPhi  = g_z conj(dE_z/dPhi_z)   (dLoss/dRe Phi + i dLoss/dIm Phi).
* h1 and every L_g are treated as unconstrained (entries independent); for
  symmetric inputs a symmetric gradient is (grad + grad^T) / 2.

Closed forms (G^s_pq = sum_j Psi_pj theta_qj, G = G^a + G^b, c_g = <L_g, G>):
    dE/dh1       = G                       (the mixed one-body density matrix)
    dE/dL_g      = c_g G - sum_s G^s L_g^T G^s
    dE/dtheta_s  = Gbar_s = h~_s^T + (sum_g c_g L~_g,s)^T - (sum_g T_g,s L~_g,s)^T,
                   T_g,s = L~_g,s theta_s
    dE/dPhi_s    = (I - Psi_s theta_s^T) Gbar_s S_s^-T,  S_s = Psi_s^T Phi_s
"""
from __future__ import annotations

import numpy as np

from .afqmc import Oracle, coulomb_vector, greens_function, overlap_and_theta


def local_energy_closed_form_derivatives(orc: Oracle, phi: np.ndarray):
    """Per-walker holomorphic derivatives dE/dh1 (W,M,M), dE/dL (W,X,M,M), dE/dPhi (W,M,N)."""
    W, M = phi.shape[0], orc.M
    pa, pb = orc.split(phi)
    _, ta = overlap_and_theta(orc.psi_a, pa)
    _, tb = overlap_and_theta(orc.psi_b, pb)
    c = coulomb_vector(orc.Lt_a, orc.Lt_b, ta, tb)
    Ga = greens_function(orc.psi_a, ta)
    Gb = greens_function(orc.psi_b, tb)
    Gt = Ga + Gb
    dh = Gt.copy()
    dL = np.empty((W, orc.X, M, M), dtype=np.complex128)
    for z in range(W):
        for g in range(orc.X):
            Lg = orc.L[g]
            dL[z, g] = c[z, g] * Gt[z] - Ga[z] @ Lg.T @ Ga[z] - Gb[z] @ Lg.T @ Gb[z]
    dphi = np.empty_like(phi)
    for sl, psi, th, Lt, ht, blk in ((slice(0, orc.na), orc.psi_a, ta, orc.Lt_a, orc.ht_a, pa),
                                     (slice(orc.na, orc.na + orc.nb), orc.psi_b, tb, orc.Lt_b,
                                      orc.ht_b, pb)):
        if psi.shape[1] == 0:
            continue
        for z in range(W):
            theta = th[z]
            gbar = ht.T.astype(np.complex128)
            gbar = gbar + np.einsum("g,gjp->pj", c[z], Lt)
            T = np.einsum("gip,pj->gij", Lt, theta)
            gbar = gbar - np.einsum("gji,gip->pj", T, Lt)
            S = psi.T @ blk[z]
            proj = np.eye(M) - psi @ theta.T
            dphi[z][:, sl] = proj @ gbar @ np.linalg.inv(S).T
    return dh, dL, dphi


def local_energy_vjp(orc: Oracle, phi: np.ndarray, g: np.ndarray):
    """Gradients of Loss = sum_z Re(conj(g_z) E_z) for a cotangent g (W complex)."""
    dh, dL, dphi = local_energy_closed_form_derivatives(orc, phi)
    cg = np.conj(g)
    grad_h = np.real(np.einsum("z,zpq->pq", cg, dh))
    grad_L = np.real(np.einsum("z,zgpq->gpq", cg, dL))
    grad_phi = g[:, None, None] * np.conj(dphi)
    return grad_h, grad_L, grad_phi


def loss(orc: Oracle, phi: np.ndarray, g: np.ndarray, h1: np.ndarray | None = None,
         L: np.ndarray | None = None) -> float:
    """Loss = sum_z Re(conj(g_z) E_L(phi_z)) for (optionally) modified h1 or L."""
    if h1 is not None or L is not None:
        orc = Oracle(orc.h1 if h1 is None else h1, orc.L if L is None else L, orc.e0, orc.psi_a,
                     orc.psi_b, dt=orc.dt, e_shift=orc.e_shift)
    e = orc.local_energy_of(phi)[:, 3]
    return float(np.sum(np.real(np.conj(g) * e)))
