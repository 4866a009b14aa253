"""FP64 oracle of one phaseless-AFQMC step for single-determinant walkers.

TEST INFRASTRUCTURE ONLY (see the package docstring): only tests/, the smoke
check and bench.py's CPU-baseline leg may use this module.

The paper (arXiv:2209.04015) states the method in Sec. "Review of AFQMC" (the
hybrid propagation, Eqs. import, ovl, ph, theta and the weight update) and in
Sec. "Implementational details" (overlap, Green's function, force bias and
local energy for single-determinant trials).  This module takes those steps in
that order, in float64 / complex128 NumPy, looping over walkers where that makes
the correspondence with the equations clearer.

Conventions and readings (the paper leaves these open; each is one choice):

* Spin is written out: alpha and beta determinants share h1 and the Cholesky
  vectors L_g; the Coulomb term couples the spins and exchange is per spin.
* Green's function: G_pq = <a+_p a_q> = sum_j Psi_pj theta_qj with
  theta = Phi (Psi^T Phi)^-1 (Eq. halfgf prints the two sides with p and q swapped;
  for symmetric h1 and L the energy does not depend on the choice).
* Force bias: the mixed estimate of v'_g = i (v_g - vbar_g), scaled by
  -sqrt(dt), so xbar_g = -i sqrt(dt) (c_g - vbar_g) with c_g = sum_pq L_g,pq G_pq
  (Eq. fb is the unscaled c_g).
* Mean-field subtraction: vbar_g = sum_sigma tr(Psi_s^T L_g Psi_s).  The one-body
  operator is h' = h1 - 1/2 sum_g L_g L_g (normal ordering of the two-body term),
  h'' = h' + sum_g vbar_g L_g, and the half-step one-body propagator is
  P = exp(-dt h''/2), applied on both sides of the two-body factor.
* Propagator for shifted fields y = xi - xbar: B(y) Phi = P T_n(A) P Phi with
  A = i sqrt(dt) sum_g y_g L_g and T_n the Taylor series of order n; the scalar
  exp(cmf), cmf = -i sqrt(dt) sum_g y_g vbar_g, belongs to B and enters the
  overlap ratio; the constant exp(-dt (e0 - 1/2 sum vbar^2 - E_shift)) is real.
* Phase: theta_z = arg of the overlap ratio R_z (including exp(cmf)); the force
  bias factor exp(cfb), cfb = xi.xbar - xbar.xbar/2, enters the magnitude only.
* Walkers whose weight drops to zero keep being propagated.
* QR re-orthogonalisation makes diag(R) real and positive, and divides the stored
  overlap by prod_sigma det R_sigma.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# Trial-dependent intermediates (built once)
# ----------------------------------------------------------------------------

def half_rotated_cholesky(L: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """L~_g,ir = sum_p Psi_pi L_g,pr: the half-rotated auxiliary vectors.

    Sec. "One-body Green's function and force bias", the equation defining
    L_ir^alpha from C_psi0^dagger (Psi is real here, so the dagger is a transpose).
    Returns shape (X, N, M).
    """
    X = L.shape[0]
    out = np.empty((X, psi.shape[1], L.shape[1]))
    for g in range(X):
        out[g] = psi.T @ L[g]
    return out


def mean_field(L: np.ndarray, psi_a: np.ndarray, psi_b: np.ndarray) -> np.ndarray:
    """vbar_g = sum_sigma tr(Psi_s^T L_g Psi_s): the trial's expectation of v_g."""
    X = L.shape[0]
    v = np.zeros(X)
    for g in range(X):
        for psi in (psi_a, psi_b):
            v[g] += np.trace(psi.T @ L[g] @ psi)
    return v


def one_body_operators(h1: np.ndarray, L: np.ndarray, vbar: np.ndarray,
                       dt: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """h' = h1 - 1/2 sum_g L_g L_g, h'' = h' + sum_g vbar_g L_g, P = exp(-dt h''/2).

    The normal-ordering term follows from rewriting the two-body part of
    Eq. Habinitio with the Cholesky factorisation as 1/2 sum_g v_g^2; the
    mean-field shift moves vbar_g v_g into the one-body part (Sec. "Review of
    AFQMC", Eq. Bx; the paper defers the details to its cited reviews).  P comes
    from a dense eigendecomposition of the symmetric h''.
    """
    X = L.shape[0]
    hp = h1.copy()
    for g in range(X):
        hp -= 0.5 * (L[g] @ L[g])
    hpp = hp.copy()
    for g in range(X):
        hpp += vbar[g] * L[g]
    hpp = 0.5 * (hpp + hpp.T)
    evals, U = np.linalg.eigh(hpp)
    P = (U * np.exp(-0.5 * dt * evals)) @ U.T
    return hp, hpp, P


# ----------------------------------------------------------------------------
# Overlap, theta, Green's function (Sec. "Overlap" and Eqs. gf, halfgf)
# ----------------------------------------------------------------------------

def overlap_matrix(psi: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """S = Psi^T Phi for each walker (Sec. "Overlap", the einsum of Listing 1).

    psi (M, N) real, phi (W, M, N) complex -> (W, N, N).
    """
    return np.einsum("pi,zpj->zij", psi, phi)


def overlap_and_theta(psi: np.ndarray, phi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """det(Psi^T Phi) and theta = Phi (Psi^T Phi)^-1 per walker (Eq. halfgf).

    Returns (ovlp (W,), theta (W, M, N)).
    """
    S = overlap_matrix(psi, phi)
    ovlp = np.linalg.det(S)
    theta = phi @ np.linalg.inv(S)
    return ovlp, theta


def greens_function(psi: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """G_pq = sum_j Psi_pj theta_qj (Eq. gf through the factorised Eq. halfgf)."""
    return np.einsum("pj,zqj->zpq", psi, theta)


# ----------------------------------------------------------------------------
# Force bias and fields (Sec. "Review of AFQMC"; Eqs. fb, rfb)
# ----------------------------------------------------------------------------

def coulomb_vector(Lt_a: np.ndarray, Lt_b: np.ndarray, theta_a: np.ndarray,
                   theta_b: np.ndarray) -> np.ndarray:
    """c_zg = sum_sigma sum_jp L~_g,jp theta_z,pj (Eq. rfb, both spins).

    This is the mixed estimate of v_g = sum_pr L_g,pr a+_p a_r; it gives the
    force bias and, at the same walker, the Coulomb energy.  Returns (W, X).
    """
    c = np.einsum("gjp,zpj->zg", Lt_a, theta_a)
    c = c + np.einsum("gjp,zpj->zg", Lt_b, theta_b)
    return c


def force_bias(c: np.ndarray, vbar: np.ndarray, dt: float, cap: float = 0.0) -> np.ndarray:
    """xbar = -sqrt(dt) <v'> with v' = i (v - vbar): xbar = -i sqrt(dt) (c - vbar).

    The optimal force bias of Sec. "Review of AFQMC".  With cap > 0 each component
    whose modulus exceeds cap is scaled back to modulus cap (a common safeguard;
    off by default).
    """
    xbar = -1j * np.sqrt(dt) * (c - vbar[None, :])
    if cap > 0.0:
        mag = np.abs(xbar)
        big = mag > cap
        xbar = np.where(big, cap * xbar / np.where(big, mag, 1.0), xbar)
    return xbar


def field_factors(xi: np.ndarray, xbar: np.ndarray, vbar: np.ndarray,
                  dt: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Shifted fields y = xi - xbar and the two per-walker scalars of the step.

    cfb = sum_g (xi_g xbar_g - xbar_g^2 / 2) is the exponent of Eq. import;
    cmf = -i sqrt(dt) sum_g y_g vbar_g is the mean-field scalar carried by B(y).
    """
    y = xi - xbar
    cfb = np.sum(xi * xbar - 0.5 * xbar * xbar, axis=1)
    cmf = -1j * np.sqrt(dt) * (y @ vbar)
    return y, cfb, cmf


# ----------------------------------------------------------------------------
# Propagator (Eq. Bx; the walker update of Sec. "Review of AFQMC")
# ----------------------------------------------------------------------------

def vhs(y: np.ndarray, L: np.ndarray) -> np.ndarray:
    """V = sum_g y_g L_g for one walker's shifted fields y (X,) -> (M, M) complex."""
    V = np.zeros(L.shape[1:], dtype=np.complex128)
    for g in range(L.shape[0]):
        V += y[g] * L[g]
    return V


def taylor_apply(A: np.ndarray, phi: np.ndarray, order: int) -> np.ndarray:
    """T_n(A) phi = sum_{k=0..n} A^k phi / k!, accumulated term by term."""
    out = phi.copy()
    term = phi
    for k in range(1, order + 1):
        term = (A @ term) / k
        out = out + term
    return out


def apply_propagator(phi: np.ndarray, y: np.ndarray, L: np.ndarray, P: np.ndarray,
                     dt: float, order: int, chunk: int = 64) -> np.ndarray:
    """Phi' = P T_n(i sqrt(dt) V(y)) P Phi for a batch of walkers.

    phi (W, M, Na+Nb), y (W, X).  The two-body factor is the same for both spins,
    so it acts on the concatenated walker matrix.  V is built in walker chunks
    (sum over g of y_zg L_g, as in vhs) to bound memory.
    """
    out = np.empty_like(phi)
    for z0 in range(0, phi.shape[0], chunk):
        z1 = min(z0 + chunk, phi.shape[0])
        V = np.einsum("zg,gpq->zpq", y[z0:z1], L)
        A = 1j * np.sqrt(dt) * V
        out[z0:z1] = P @ taylor_apply(A, P @ phi[z0:z1], order)
    return out


# ----------------------------------------------------------------------------
# Local energy (Sec. "Local energy")
# ----------------------------------------------------------------------------

def exchange_energy(Lt: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """E_K = -1/2 sum_g sum_ij T_ij T_ji with T_ij = sum_p L~_g,ip theta_pj.

    Sec. "Local energy": the exchange term of E_L and the intermediate T, formed
    and consumed per walker.  One spin; returns (W,) complex.
    """
    W = theta.shape[0]
    ek = np.zeros(W, dtype=np.complex128)
    for z in range(W):
        T = Lt @ theta[z]
        ek[z] = -0.5 * np.einsum("gij,gji->", T, T)
    return ek


def one_body_energy(ht_a: np.ndarray, ht_b: np.ndarray, theta_a: np.ndarray,
                    theta_b: np.ndarray) -> np.ndarray:
    """E1 = sum_sigma sum_pq h_pq G_pq = sum_sigma sum_jq h~_jq theta_qj."""
    return (np.einsum("jq,zqj->z", ht_a, theta_a)
            + np.einsum("jq,zqj->z", ht_b, theta_b))


# ----------------------------------------------------------------------------
# The oracle driver
# ----------------------------------------------------------------------------

@dataclass
class StepRecord:
    """Intermediates of the last step, for parity tests."""

    c: np.ndarray | None = None
    xbar: np.ndarray | None = None
    y: np.ndarray | None = None
    cfb: np.ndarray | None = None
    cmf: np.ndarray | None = None
    ratio: np.ndarray | None = None
    importance: np.ndarray | None = None


@dataclass
class Oracle:
    """Walker ensemble plus the Hamiltonian and trial intermediates.

    Arrays follow the library's layouts: h1 (M, M), L (X, M, M), psi_* (M, N_s),
    phi (W, M, Na+Nb) complex with the alpha columns first, fields (W, X).
    """

    h1: np.ndarray
    L: np.ndarray
    e0: float
    psi_a: np.ndarray
    psi_b: np.ndarray
    dt: float = 0.005
    taylor_order: int = 6
    qr_period: int = 5
    e_shift: float | None = None
    fb_cap: float = 0.0
    free_projection: bool = False
    phi: np.ndarray | None = None
    w: np.ndarray | None = None
    ovlp: np.ndarray | None = None
    nstep: int = 0
    last: StepRecord = field(default_factory=StepRecord)

    def __post_init__(self):
        self.M = self.h1.shape[0]
        self.X = self.L.shape[0]
        self.na = self.psi_a.shape[1]
        self.nb = self.psi_b.shape[1]
        self.Lt_a = half_rotated_cholesky(self.L, self.psi_a)
        self.Lt_b = half_rotated_cholesky(self.L, self.psi_b)
        self.ht_a = self.psi_a.T @ self.h1
        self.ht_b = self.psi_b.T @ self.h1
        self.vbar = mean_field(self.L, self.psi_a, self.psi_b)
        self.hp, self.hpp, self.P = one_body_operators(self.h1, self.L, self.vbar, self.dt)
        if self.e_shift is None:
            self.e_shift = self.trial_energy()

    # -- walkers --------------------------------------------------------------
    def init_walkers(self, phi: np.ndarray, w: np.ndarray | None = None) -> None:
        self.phi = np.array(phi, dtype=np.complex128)
        W = self.phi.shape[0]
        wdt = np.complex128 if self.free_projection else np.float64
        self.w = np.ones(W, dtype=wdt) if w is None else np.array(w, dtype=wdt)
        self.ovlp = self.overlap(self.phi)
        self.nstep = 0

    def split(self, phi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        return phi[:, :, : self.na], phi[:, :, self.na:]

    def overlap(self, phi: np.ndarray) -> np.ndarray:
        """<Psi_T|phi> = prod_sigma det(Psi_s^T Phi_s) (Sec. "Overlap")."""
        pa, pb = self.split(phi)
        oa, _ = overlap_and_theta(self.psi_a, pa)
        ob, _ = overlap_and_theta(self.psi_b, pb)
        return oa * ob

    def thetas(self, phi: np.ndarray):
        pa, pb = self.split(phi)
        _, ta = overlap_and_theta(self.psi_a, pa)
        _, tb = overlap_and_theta(self.psi_b, pb)
        return ta, tb

    # -- energies ---------------------------------------------------------------
    def trial_energy(self) -> float:
        """E_L of the trial itself (the walker equal to Psi_T)."""
        phi = np.concatenate([self.psi_a, self.psi_b], axis=1)[None].astype(np.complex128)
        return float(self.local_energy_of(phi)[0, 3].real)

    def local_energy_of(self, phi: np.ndarray) -> np.ndarray:
        """Columns E1, EJ, EK, E_L (complex) of the mixed local energy per walker.

        Sec. "Local energy": E_L = <Psi_T|H|phi>/<Psi_T|phi> = e0 + E1 + EJ + EK with
        EJ = 1/2 sum_g c_g^2 (Coulomb, both spins) and EK the per-spin exchange.
        """
        ta, tb = self.thetas(phi)
        c = coulomb_vector(self.Lt_a, self.Lt_b, ta, tb)
        e1 = one_body_energy(self.ht_a, self.ht_b, ta, tb)
        ej = 0.5 * np.sum(c * c, axis=1)
        ek = exchange_energy(self.Lt_a, ta) + exchange_energy(self.Lt_b, tb)
        el = self.e0 + e1 + ej + ek
        return np.stack([e1, ej, ek, el], axis=1)

    def local_energy(self) -> tuple[np.ndarray, float]:
        """Per-walker energies and the weighted estimate sum w Re E_L / sum w."""
        e = self.local_energy_of(self.phi)
        if self.free_projection:
            emix = float((np.sum(self.w * e[:, 3]) / np.sum(self.w)).real)
        else:
            emix = float(np.sum(self.w * e[:, 3].real) / np.sum(self.w))
        return e, emix

    # -- propagation --------------------------------------------------------------
    def step(self, xi: np.ndarray) -> None:
        """One hybrid-propagation step of every walker with the given N(0,1) fields.

        Sec. "Review of AFQMC": force bias, shifted fields, B(x - xbar), overlap
        ratio (Eq. ovl), importance function (Eq. import), phaseless weight
        (Eqs. ph, theta), then the weight and walker update.
        """
        dt = self.dt
        ta, tb = self.thetas(self.phi)
        c = coulomb_vector(self.Lt_a, self.Lt_b, ta, tb)
        xbar = force_bias(c, self.vbar, dt, self.fb_cap)
        y, cfb, cmf = field_factors(xi, xbar, self.vbar, dt)
        new_phi = apply_propagator(self.phi, y, self.L, self.P, dt, self.taylor_order)
        new_ovlp = self.overlap(new_phi)
        ratio = new_ovlp / self.ovlp * np.exp(cmf)
        const = np.exp(-dt * (self.e0 - 0.5 * np.sum(self.vbar ** 2) - self.e_shift))
        importance = ratio * np.exp(cfb) * const
        if self.free_projection:
            self.w = self.w * importance
        else:
            phase = np.angle(ratio)
            self.w = self.w * np.abs(importance) * np.maximum(0.0, np.cos(phase))
        self.phi = new_phi
        self.ovlp = new_ovlp
        self.nstep += 1
        self.last = StepRecord(c=c, xbar=xbar, y=y, cfb=cfb, cmf=cmf, ratio=ratio,
                               importance=importance)

    def orthogonalise(self) -> None:
        """QR of each walker's spin blocks with diag(R) > 0; overlap divided by det R."""
        for z in range(self.phi.shape[0]):
            detr = 1.0
            for lo, hi in ((0, self.na), (self.na, self.na + self.nb)):
                if hi == lo:
                    continue
                Q, R = np.linalg.qr(self.phi[z][:, lo:hi])
                d = np.diag(R)
                ph = d / np.abs(d)
                Q = Q * ph[None, :]
                detr *= np.prod(np.abs(d))
                self.phi[z][:, lo:hi] = Q
            self.ovlp[z] = self.ovlp[z] / detr

    def propagate(self, fields: list[np.ndarray] | np.ndarray) -> None:
        """Steps with the given fields; QR after every qr_period-th step."""
        for xi in fields:
            self.step(xi)
            if self.qr_period > 0 and self.nstep % self.qr_period == 0:
                self.orthogonalise()
