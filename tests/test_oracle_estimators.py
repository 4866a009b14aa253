"""Pins of the oracle's mixed <S^2> estimator: brute force in Fock space with the
operator S^2 = S_- S_+ + S_z (S_z + 1) built from Jordan-Wigner matrices (no Wick's
theorem), on general complex walkers whose Green's functions are not symmetric (so
the index order of the trace is tested); the textbook spin contamination of a
determinant (Szabo and Ostlund, Eq. 2.271); a closed-shell singlet and a high-spin
determinant; invariance under Phi -> Phi C.  The weighted mixed one-body density
matrix: its trace, the one-body energy it gives against the local energy's E1, and
Fock-space matrix elements for a single walker."""
import numpy as np
import pytest

from fockspace import FockSpace
from oracle.afqmc import Oracle
from oracle.estimators import one_rdm, spin_squared, spin_squared_of
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


def test_one_rdm_trace_one_body_energy_and_fock_space():
    """The weighted mixed 1-RDM: trace n_s per spin (every walker's G has trace n_s);
    sum_pq h1_pq (G^a + G^b)_pq equals the weighted one-body energy E1 of the local
    energy; with one walker it is <Psi_T|a+_p a_q|phi>/<Psi_T|phi> in Fock space."""
    s = make_system(9, 3, 2, 6, seed=4, decay="half")
    orc = _oracle(s, s.psi_a, s.psi_b)
    W = 5
    orc.init_walkers(perturbed_walkers(s, W, eps=0.5, seed=3), w=np.array([0.3, 1.0, 2.0, 0.7, 1.1]))
    g = one_rdm(orc)
    assert abs(np.trace(g[0]) - 3) < 1e-12 and abs(np.trace(g[1]) - 2) < 1e-12
    e = orc.local_energy_of(orc.phi)
    w = orc.w
    e1 = np.sum(w * e[:, 0]) / np.sum(w)
    assert abs(np.sum(s.h1 * (g[0] + g[1])) - e1) < 1e-11 * max(1.0, abs(e1))
    M = 4
    s4 = make_system(M, 2, 1, 3, seed=2, decay="half")
    o4 = _oracle(s4, s4.psi_a, s4.psi_b)
    phi = perturbed_walkers(s4, 1, eps=0.8, seed=4)
    o4.init_walkers(phi)
    g4 = one_rdm(o4)
    fs = FockSpace(M)
    trial = fs.determinant(s4.psi_a, s4.psi_b)
    v = fs.walker_state(phi[0], 2)
    den = np.vdot(trial, v)
    for sigma in (0, 1):
        for p_ in range(M):
            for q in range(M):
                op = fs.cre[fs.so(p_, sigma)] @ fs.ann[fs.so(q, sigma)]
                ref = np.vdot(trial, op @ v) / den
                assert abs(g4[sigma][p_, q] - ref) < 1e-12, (sigma, p_, q)
