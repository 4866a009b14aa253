"""Mixed estimators other than the energy, plain NumPy (test infrastructure).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and bench.py's CPU legs may
use this module; the library never imports it.

Sec. "Customized mixed estimators" adds <S^2> as its example: S^2 commutes with H,
so its mixed estimate is unbiased, and for a single-determinant trial

    <Psi_T|S^2|phi_z> / <Psi_T|phi_z> = N_beta + M_S (M_S + 1) - tr(G_alpha G_beta)

with G_sigma the walker's one-body Green's function of spin sigma.  Reading: the
printed sum is over G_{p beta, q beta} G_{p alpha, q alpha} while the printed
listing contracts the second index of one with the first of the other; Wick's
theorem on S^2 = S_- S_+ + S_z (S_z + 1), S_+ = sum_p a+_{p alpha} a_{p beta}, gives
<S_- S_+> = N_beta - sum_pq G_alpha,pq G_beta,qp, i.e. the trace of the product
(the two agree for symmetric G, not for a general walker).  M_S = (N_alpha -
N_beta) / 2.
"""
from __future__ import annotations

import numpy as np

from oracle.afqmc import greens_function


def spin_squared_of(orc, phi: np.ndarray) -> np.ndarray:
    """Mixed <S^2> of each walker (complex)."""
    ta, tb = orc.thetas(phi)
    na, nb = orc.na, orc.nb
    ms = 0.5 * (na - nb)
    ga = greens_function(orc.psi_a, ta)  # (W, M, M) each
    gb = greens_function(orc.psi_b, tb)
    return nb + ms * (ms + 1.0) - np.einsum("zpq,zqp->z", ga, gb)


def spin_squared(orc) -> tuple[np.ndarray, float]:
    """Per-walker <S^2> and the weighted estimate Re(sum w S2 / sum w)."""
    s2 = spin_squared_of(orc, orc.phi)
    w = np.asarray(orc.w, dtype=np.complex128)
    return s2, float((np.sum(w * s2) / np.sum(w)).real)


def one_rdm(orc) -> np.ndarray:
    """Weighted mixed one-body density matrix per spin, (2, M, M) complex:
    sum_z w_z G^s_z / sum_z w_z with G_pq = <a+_p a_q> of each walker (reading of
    Eq. halfgf, as for the energy)."""
    ta, tb = orc.thetas(orc.phi)
    w = np.asarray(orc.w, dtype=np.complex128)
    ga = greens_function(orc.psi_a, ta)
    gb = greens_function(orc.psi_b, tb)
    return np.stack([np.einsum("z,zpq->pq", w, ga), np.einsum("z,zpq->pq", w, gb)]) / np.sum(w)
