"""Pins of the oracle's mixed <S^2> estimator: brute force in Fock space with the
operator S^2 = S_- S_+ + S_z (S_z + 1) built from Jordan-Wigner matrices (no Wick's
theorem), on general complex walkers whose Green's functions are not symmetric (so
the index order of the trace is tested); the textbook spin contamination of a
determinant (Szabo and Ostlund, Eq. 2.271); a closed-shell singlet and a high-spin
determinant; invariance under Phi -> Phi C."""
import numpy as np
import pytest

from fockspace import FockSpace
from oracle.afqmc import Oracle
from oracle.estimators import spin_squared, spin_squared_of
from paper_2209_04015_b300.synthetic import make_system, perturbed_walkers


def _orth(M, n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((M, n)))
    return q


def _oracle(s, psi_a, psi_b):
    return Oracle(s.h1, s.L, s.e0, psi_a, psi_b)


def _s2_operator(fs: FockSpace):
    M = fs.M
    splus = sum(fs.cre[fs.so(p, 0)] @ fs.ann[fs.so(p, 1)] for p in range(M))
    sminus = splus.conj().T
    na = sum(fs.cre[fs.so(p, 0)] @ fs.ann[fs.so(p, 0)] for p in range(M))
    nb = sum(fs.cre[fs.so(p, 1)] @ fs.ann[fs.so(p, 1)] for p in range(M))
    sz = 0.5 * (na - nb)
    return sminus @ splus + sz @ sz + sz


@pytest.mark.parametrize("na,nb", [(2, 1), (2, 2), (1, 2), (3, 0)])
def test_mixed_s2_matches_fock_space(na, nb):
    M = 4
    s = make_system(M, na, nb, 3, seed=2, decay="half")
    orc = _oracle(s, s.psi_a, s.psi_b)
    phi = perturbed_walkers(s, 3, eps=0.8, seed=4)
    fs = FockSpace(M)
    S2 = _s2_operator(fs)
    trial = fs.determinant(s.psi_a, s.psi_b)
    got = spin_squared_of(orc, phi)
    for z in range(3):
        v = fs.walker_state(phi[z], na)
        ref = np.vdot(trial, S2 @ v) / np.vdot(trial, v)
        assert abs(got[z] - ref) < 1e-12 * max(1.0, abs(ref)), (z, got[z], ref)


def test_determinant_spin_contamination_closed_form():
    """Walker = trial (different alpha and beta orbitals): S^2 = M_S (M_S + 1) + N_b
    - sum_ij |<a_i|b_j>|^2."""
    M, na, nb = 9, 4, 2
    s = make_system(M, na, nb, 5, seed=3, decay="half")
    pa, pb = _orth(M, na, 11), _orth(M, nb, 12)
    orc = _oracle(s, pa, pb)
    phi = np.concatenate([pa, pb], axis=1)[None].astype(np.complex128)
    ms = 0.5 * (na - nb)
    expect = ms * (ms + 1) + nb - np.sum((pa.T @ pb) ** 2)
    assert spin_squared_of(orc, phi)[0] == pytest.approx(expect, abs=1e-12)


def test_closed_shell_singlet_and_high_spin():
    M = 8
    s = make_system(M, 3, 3, 5, seed=3, decay="half")
    pa = _orth(M, 3, 21)
    rhf = _oracle(s, pa, pa)
    phi = np.concatenate([pa, pa], axis=1)[None].astype(np.complex128)
    assert abs(spin_squared_of(rhf, phi)[0]) < 1e-12
    hs = _oracle(s, pa, pa[:, :1])  # 3 alpha, 1 beta in the same orbitals: M_S = 1
    phi = np.concatenate([pa, pa[:, :1]], axis=1)[None].astype(np.complex128)
    assert spin_squared_of(hs, phi)[0] == pytest.approx(2.0, abs=1e-12)


def test_gauge_invariance_and_weighted_estimate():
    s = make_system(10, 3, 2, 6, seed=5, decay="half")
    orc = _oracle(s, s.psi_a, s.psi_b)
    W = 4
    phi = perturbed_walkers(s, W, eps=0.5, seed=7)
    rng = np.random.default_rng(1)
    c = rng.standard_normal((W, 5, 5)) + 1j * rng.standard_normal((W, 5, 5))
    c[:, :3, 3:] = 0.0
    c[:, 3:, :3] = 0.0  # block diagonal: no spin mixing
    a = spin_squared_of(orc, phi)
    b = spin_squared_of(orc, phi @ c)
    np.testing.assert_allclose(b, a, rtol=1e-11, atol=1e-12)
    orc.init_walkers(phi, w=np.array([0.5, 1.0, 2.0, 0.25]))
    s2, mix = spin_squared(orc)
    assert mix == pytest.approx(float((np.sum(orc.w * s2) / np.sum(orc.w)).real), rel=1e-14)
