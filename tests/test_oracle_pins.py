"""Pins of the FP64 oracle against closed forms, invariants and brute force (CPU only).

Each test ties one part of oracle.afqmc to something other than itself: the
Jordan-Wigner Fock-space brute force of tests/fockspace.py, the full ERI tensor,
scipy's matrix exponential, exact Gaussian integrals by quadrature, or
invariances that a dropped term, wrong sign or transposed index would break.
"""
import numpy as np
import pytest
import scipy.linalg

from fockspace import FockSpace
from oracle import afqmc
from oracle.afqmc import Oracle
from paper_2209_04015_b300.synthetic import make_system, perturbed_walkers, trial_walkers


def small_oracle(M=4, na=2, nb=1, X=6, seed=3, e0=0.3, dt=0.01, **kw):
    s = make_system(M, na, nb, X, seed=seed, decay="half", e0=e0)
    return s, Oracle(s.h1, s.L, e0, s.psi_a, s.psi_b, dt=dt, **kw)


def random_walkers(s, W, seed=0, eps=0.4):
    return perturbed_walkers(s, W, eps=eps, seed=seed)


# ---------------------------------------------------------------------------- A1

def test_overlap_matches_fock_space():
    s, o = small_oracle()
    F = FockSpace(s.M)
    phi = random_walkers(s, 5)
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    ov = o.overlap(phi)
    for z in range(5):
        assert np.isclose(ov[z], np.vdot(psiT, F.walker_state(phi[z], s.na)), rtol=1e-13)


def test_greens_function_matches_fock_space():
    s, o = small_oracle()
    F = FockSpace(s.M)
    phi = random_walkers(s, 3, seed=4)
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    ta, tb = o.thetas(phi)
    for z in range(3):
        st = F.walker_state(phi[z], s.na)
        den = np.vdot(psiT, st)
        for sigma, psi, th in ((0, s.psi_a, ta), (1, s.psi_b, tb)):
            G = afqmc.greens_function(psi, th[z:z + 1])[0]
            for p in range(s.M):
                for q in range(s.M):
                    op = F.cre[F.so(p, sigma)] @ F.ann[F.so(q, sigma)]
                    ref = np.vdot(psiT, op @ st) / den
                    assert abs(G[p, q] - ref) < 1e-12 * max(1.0, abs(ref))


def test_greens_function_idempotent_with_trace_n():
    s = make_system(8, 3, 2, 24, seed=1, decay="half")
    phi = perturbed_walkers(s, 4, eps=0.5, seed=2)
    for psi, cols in ((s.psi_a, slice(0, 3)), (s.psi_b, slice(3, 5))):
        _, th = afqmc.overlap_and_theta(psi, phi[:, :, cols])
        G = afqmc.greens_function(psi, th)
        assert np.allclose(G @ G, G, atol=1e-12)
        assert np.allclose(np.trace(G, axis1=1, axis2=2), psi.shape[1], atol=1e-12)


def test_gauge_invariance_of_theta_and_overlap_scaling():
    s = make_system(8, 3, 2, 24, seed=1, decay="half")
    phi = perturbed_walkers(s, 2, eps=0.5, seed=5)[:, :, :3]
    rng = np.random.default_rng(0)
    C = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    o1, t1 = afqmc.overlap_and_theta(s.psi_a, phi)
    o2, t2 = afqmc.overlap_and_theta(s.psi_a, phi @ C)
    assert np.allclose(t1, t2, atol=1e-12)
    assert np.allclose(o2, o1 * np.linalg.det(C), rtol=1e-12)


def test_trial_walker_has_unit_overlap_and_zero_force_bias():
    s, o = small_oracle(M=8, na=2, nb=2, X=24, seed=1)
    phi = trial_walkers(s, 3)
    o.init_walkers(phi)
    assert np.allclose(o.ovlp, 1.0, atol=1e-13)
    ta, tb = o.thetas(phi)
    assert np.allclose(ta, s.psi_a[None], atol=1e-14)
    c = afqmc.coulomb_vector(o.Lt_a, o.Lt_b, ta, tb)
    assert np.max(np.abs(afqmc.force_bias(c, o.vbar, o.dt))) < 1e-13


# ---------------------------------------------------------------------------- A2

def test_coulomb_vector_matches_full_g_and_fock_space():
    s, o = small_oracle()
    F = FockSpace(s.M)
    phi = random_walkers(s, 2, seed=8)
    ta, tb = o.thetas(phi)
    c = afqmc.coulomb_vector(o.Lt_a, o.Lt_b, ta, tb)
    Ga = afqmc.greens_function(s.psi_a, ta)
    Gb = afqmc.greens_function(s.psi_b, tb)
    brute = np.einsum("zpq,gpq->zg", Ga + Gb, s.L)
    assert np.allclose(c, brute, rtol=1e-12, atol=1e-13)
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    st = F.walker_state(phi[0], s.na)
    for g in range(s.X):
        vg = F.one_body(s.L[g])
        assert np.isclose(c[0, g], np.vdot(psiT, vg @ st) / np.vdot(psiT, st), rtol=1e-12)


def test_mean_field_is_trial_expectation_fock_space():
    s, o = small_oracle()
    F = FockSpace(s.M)
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    for g in range(s.X):
        ref = np.vdot(psiT, F.one_body(s.L[g]) @ psiT).real
        assert np.isclose(o.vbar[g], ref, rtol=1e-12, atol=1e-14)


def test_force_bias_cancels_linear_field_term():
    """With the optimal force bias, log I has no O(sqrt(dt)) slope in the fields.

    d log I / d xi_g = sqrt(dt) <v'_g> + xbar_g + O(dt |y|); the optimal choice
    cancels the first two, and at xi = 0 the shifted field y = -xbar is itself
    O(sqrt(dt)), so the slope is O(dt^1.5): quartering dt divides it by 8.  A
    wrong sign or scale of xbar leaves an O(sqrt(dt)) slope (a factor of 2).
    """
    slopes = []
    for dt in (4e-4, 1e-4):
        s, o = small_oracle(dt=dt, seed=6)
        phi = random_walkers(s, 1, seed=9)
        o.init_walkers(phi)
        xi0 = np.zeros((1, s.X))
        h = 1e-4
        logi = []
        for d in (-h, h):
            o.init_walkers(phi)
            xi = xi0.copy()
            xi[0, 0] += d
            o.step(xi)
            logi.append(np.log(o.last.importance[0]))
        slopes.append(abs((logi[1] - logi[0]) / (2 * h)))
    ratio = slopes[0] / slopes[1]
    assert 7.0 < ratio < 9.0, ratio


# ---------------------------------------------------------------------------- A4 / A5

def test_taylor_series_matches_expm():
    s = make_system(10, 3, 3, 20, seed=2, decay="half")
    rng = np.random.default_rng(1)
    y = rng.standard_normal(20)
    dt = 1e-3
    A = 1j * np.sqrt(dt) * afqmc.vhs(y, s.L)
    phi = perturbed_walkers(s, 1, seed=3)[0]
    approx = afqmc.taylor_apply(A, phi, 6)
    exact = scipy.linalg.expm(A) @ phi
    nA = np.linalg.norm(A, 2)
    bound = nA ** 7 / 5040 * np.exp(nA) * np.linalg.norm(phi, 2)
    assert np.linalg.norm(approx - exact, 2) <= bound * 1.01 + 1e-15
    assert np.linalg.norm(afqmc.taylor_apply(A, phi, 3) - exact) > 1e-3 * bound * 1e3


def test_vhs_is_sum_of_cholesky_vectors():
    s = make_system(6, 2, 2, 9, seed=2, decay="half")
    y = np.random.default_rng(3).standard_normal(9) + 0.5j
    V = afqmc.vhs(y, s.L)
    assert np.allclose(V, np.tensordot(y, s.L, axes=1))
    assert np.allclose(V, V.T)


def test_one_body_operators_against_eri_and_expm():
    """h' from the ERI tensor: h'_ps = h_ps - 1/2 sum_r (pr|rs); P P = expm(-dt h'')."""
    s, o = small_oracle(M=6, na=2, nb=2, X=8, seed=4, dt=0.05)
    eri = np.einsum("gpr,gqs->prqs", s.L, s.L)
    hp = s.h1 - 0.5 * np.einsum("prrs->ps", eri)
    assert np.allclose(o.hp, hp, atol=1e-13)
    hpp = hp + np.einsum("g,gpq->pq", o.vbar, s.L)
    assert np.allclose(o.hpp, hpp, atol=1e-13)
    assert np.allclose(o.P @ o.P, scipy.linalg.expm(-0.05 * hpp), atol=1e-13)


def test_zero_field_step_is_one_body_evolution():
    s, o = small_oracle(M=8, na=2, nb=2, X=24, seed=1, dt=0.01)
    phi = random_walkers(s, 2, seed=1)
    out = afqmc.apply_propagator(phi, np.zeros((2, s.X)), s.L, o.P, o.dt, 6)
    ref = scipy.linalg.expm(-o.dt * o.hpp) @ phi
    assert np.allclose(out, ref, atol=1e-13)
    # the energy of the evolved walker equals the direct Wick value (see below)
    assert np.allclose(o.local_energy_of(out)[:, 3], wick_energy(s, out), rtol=1e-11)


def test_hs_quadrature_reproduces_exact_propagator():
    """One Cholesky vector and h1 commuting with it: the Trotter split is exact.

    The importance-sampled propagator averaged over the field by Gauss-Hermite
    quadrature must then equal exp(-dt (H - E_shift)) applied to the walker, in
    the representation sum_k q_k I_k |phi'_k> / <Psi_T|phi'_k>.  This pins
    A = i sqrt(dt) y L, cmf, cfb, h', h'', P and the real constant together.
    """
    M, na, nb = 4, 2, 1
    s = make_system(M, na, nb, 1, seed=11, decay="half")
    L = s.L * 1.3
    h1 = 0.7 * L[0] - 0.4 * L[0] @ L[0] + 0.2 * np.eye(M)
    e0, dt = 0.25, 0.05
    o = Oracle(h1, L, e0, s.psi_a, s.psi_b, dt=dt, taylor_order=24, free_projection=True)
    F = FockSpace(M)
    H = F.hamiltonian(h1, L, e0).toarray()
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), na)
    phi = perturbed_walkers(s, 1, eps=0.5, seed=3)
    nodes, qw = np.polynomial.hermite_e.hermegauss(60)
    qw = qw / np.sqrt(2 * np.pi)
    acc = np.zeros(F.dim, dtype=complex)
    for x, q in zip(nodes, qw):
        o.init_walkers(phi)
        o.step(np.array([[x]]))
        st = F.walker_state(o.phi[0], na)
        acc += q * o.last.importance[0] * st / np.vdot(psiT, st)
    st0 = F.walker_state(phi[0], na)
    ref = scipy.linalg.expm(-dt * (H - o.e_shift * np.eye(F.dim))) @ st0 / np.vdot(psiT, st0)
    assert np.linalg.norm(acc - ref) < 1e-10 * np.linalg.norm(ref)
    assert abs(o.last.xbar[0, 0]) > 1e-3   # the force bias is non-trivial here


def test_overlap_ratio_matches_fock_space_propagator():
    """R = <Psi_T|B(y)|phi>/<Psi_T|phi> with B built in Fock space by expm (Thouless)."""
    s, o = small_oracle(dt=0.02, seed=12)
    o.taylor_order = 20
    F = FockSpace(s.M)
    phi = random_walkers(s, 1, seed=2)
    o.init_walkers(phi)
    xi = np.random.default_rng(5).standard_normal((1, s.X))
    o.step(xi)
    y = o.last.y[0]
    A = 1j * np.sqrt(o.dt) * np.tensordot(y, s.L, axes=1)
    B = (F.expm(F.one_body(-0.5 * o.dt * o.hpp)) @ F.expm(F.one_body(A))
         @ F.expm(F.one_body(-0.5 * o.dt * o.hpp)))
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    st = F.walker_state(phi[0], s.na)
    ref = np.vdot(psiT, B @ st) / np.vdot(psiT, st) * np.exp(o.last.cmf[0])
    assert np.isclose(o.last.ratio[0], ref, rtol=1e-11)
    # and the propagated determinant is the Fock-space image of the walker
    assert np.allclose(F.walker_state(o.phi[0], s.na), B @ st, atol=1e-11)


# ---------------------------------------------------------------------------- A6

def test_phaseless_weight_rule():
    """w' = w |I| max(0, cos arg R); walkers with cos < 0 get weight exactly 0."""
    s, o = small_oracle(M=6, na=2, nb=2, X=8, seed=2, dt=0.5)
    o.L = o.L * 4.0
    o.__post_init__()
    o.init_walkers(random_walkers(s, 200, seed=3, eps=0.6))
    w0 = o.w.copy()
    o.step(np.random.default_rng(2).standard_normal((200, s.X)) * 3.0)
    cosv = np.cos(np.angle(o.last.ratio))
    neg = cosv < 0
    assert neg.any() and (~neg).any()
    assert np.all(o.w[neg] == 0.0)
    pos = ~neg
    assert np.allclose(o.w[pos], w0[pos] * np.abs(o.last.importance[pos]) * cosv[pos],
                       rtol=1e-14)


# ---------------------------------------------------------------------------- A7

def wick_energy(s, phi, e0=None):
    """E_L from the full ERI tensor and G (both spins), brute force."""
    e0 = s.e0 if e0 is None else e0
    eri = np.einsum("gpr,gqs->prqs", s.L, s.L)
    out = []
    for z in range(phi.shape[0]):
        Gs = []
        for psi, cols in ((s.psi_a, slice(0, s.na)), (s.psi_b, slice(s.na, s.na + s.nb))):
            _, th = afqmc.overlap_and_theta(psi, phi[z:z + 1, :, cols])
            Gs.append(afqmc.greens_function(psi, th)[0])
        Gt = Gs[0] + Gs[1]
        e = e0 + np.sum(s.h1 * Gt)
        e += 0.5 * np.einsum("prqs,pr,qs->", eri, Gt, Gt)
        for G in Gs:
            e -= 0.5 * np.einsum("prqs,ps,qr->", eri, G, G)
        out.append(e)
    return np.array(out)


def test_local_energy_matches_fock_space_hamiltonian():
    s, o = small_oracle()
    F = FockSpace(s.M)
    H = F.hamiltonian(s.h1, s.L, s.e0)
    psiT = F.walker_state(np.concatenate([s.psi_a, s.psi_b], 1).astype(complex), s.na)
    phi = random_walkers(s, 4, seed=6)
    e = o.local_energy_of(phi)
    for z in range(4):
        st = F.walker_state(phi[z], s.na)
        ref = np.vdot(psiT, H @ st) / np.vdot(psiT, st)
        assert np.isclose(e[z, 3], ref, rtol=1e-12)
    assert np.allclose(e[:, 3], s.e0 + e[:, 0] + e[:, 1] + e[:, 2])


def test_trial_energy_is_slater_condon():
    s = make_system(8, 2, 2, 24, seed=1, decay="half", e0=1.5)
    o = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b)
    eri = np.einsum("gpr,gqs->prqs", s.L, s.L)
    Pa, Pb = s.psi_a @ s.psi_a.T, s.psi_b @ s.psi_b.T
    P = Pa + Pb
    ehf = s.e0 + np.sum(s.h1 * P) + 0.5 * np.einsum("prqs,pr,qs->", eri, P, P)
    for Ps in (Pa, Pb):
        ehf -= 0.5 * np.einsum("prqs,ps,qr->", eri, Ps, Ps)
    assert np.isclose(o.trial_energy(), ehf, rtol=1e-13)


def test_local_energy_matches_wick_with_full_eri():
    s = make_system(8, 3, 2, 24, seed=1, decay="half", e0=-0.7)
    o = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b)
    phi = perturbed_walkers(s, 5, eps=0.5, seed=4)
    assert np.allclose(o.local_energy_of(phi)[:, 3], wick_energy(s, phi), rtol=1e-12)


def test_energy_invariant_under_orbital_rotation_and_gauge():
    s = make_system(8, 3, 2, 24, seed=1, decay="half", e0=0.1)
    o = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b)
    phi = perturbed_walkers(s, 3, eps=0.5, seed=4)
    e = o.local_energy_of(phi)[:, 3]
    U = np.linalg.qr(np.random.default_rng(8).standard_normal((8, 8)))[0]
    Lr = np.einsum("pi,gpq,qj->gij", U, s.L, U)
    orot = Oracle(U.T @ s.h1 @ U, Lr, s.e0, U.T @ s.psi_a, U.T @ s.psi_b)
    assert np.allclose(orot.local_energy_of(np.einsum("pi,zpj->zij", U, phi))[:, 3], e,
                       rtol=1e-12)
    C = np.eye(5, dtype=complex)
    C[:3, :3] += 0.3 * np.random.default_rng(1).standard_normal((3, 3))
    C[3:, 3:] *= 1.7 - 0.2j
    assert np.allclose(o.local_energy_of(phi @ C)[:, 3], e, rtol=1e-12)


def test_exchange_equals_listing_style_sum():
    """E_K = -1/2 sum_g sum_ij T_ij T_ji equals -1/2 sum_g (T ravel) . (T^T ravel)."""
    s = make_system(8, 3, 2, 12, seed=1, decay="half")
    o = Oracle(s.h1, s.L, 0.0, s.psi_a, s.psi_b)
    phi = perturbed_walkers(s, 2, eps=0.5, seed=4)
    ta, _ = o.thetas(phi)
    ek = afqmc.exchange_energy(o.Lt_a, ta)
    for z in range(2):
        acc = 0.0
        for g in range(s.X):
            T = o.Lt_a[g].dot(ta[z].real) + 1j * o.Lt_a[g].dot(ta[z].imag)
            acc += np.dot(T.ravel(), T.T.ravel())
        assert np.isclose(ek[z], -0.5 * acc, rtol=1e-13)


# ---------------------------------------------------------------------------- A8

def test_qr_keeps_energy_theta_and_sets_overlap():
    s, o = small_oracle(M=8, na=3, nb=2, X=24, seed=1)
    o.init_walkers(random_walkers(s, 4, seed=2, eps=0.7))
    o.phi = o.phi * 1.9   # an unnormalised walker, as after a few steps
    o.ovlp = o.overlap(o.phi)
    e1, _ = o.local_energy()
    ta1, tb1 = o.thetas(o.phi)
    o.orthogonalise()
    e2, _ = o.local_energy()
    ta2, tb2 = o.thetas(o.phi)
    assert np.allclose(e1, e2, rtol=1e-12)
    assert np.allclose(ta1, ta2, atol=1e-12) and np.allclose(tb1, tb2, atol=1e-12)
    for cols in (slice(0, 3), slice(3, 5)):
        Q = o.phi[:, :, cols]
        eye = np.eye(Q.shape[2])
        assert np.allclose(np.conj(np.swapaxes(Q, 1, 2)) @ Q, eye[None], atol=1e-13)
    assert np.allclose(o.ovlp, o.overlap(o.phi), rtol=1e-12)


# ---------------------------------------------------------------------------- whole method

def test_free_projection_converges_to_exact_diagonalisation():
    """4 orbitals, 1+1 electrons: free projection against the exact E(tau) and E0.

    The trial is the best product state of the exact ground state.  The walker
    average sum w E_L / sum w must agree with the exact projected energy
    <Psi_T|H e^{-tau H}|Psi_T> / <Psi_T|e^{-tau H}|Psi_T> within 4 jackknife
    standard errors at several tau, and at the last tau with the Fock-sector
    ground state energy.
    """
    M, na, nb, X = 4, 1, 1, 4
    s = make_system(M, na, nb, X, seed=5, decay="half")
    F = FockSpace(M)
    H = F.hamiltonian(s.h1, s.L, 0.0)
    idx = F.sector(na, nb)
    ev, vec = np.linalg.eigh(H.toarray()[np.ix_(idx, idx)].real)
    E0 = ev[0]
    C = np.zeros((M, M))
    for k, st in enumerate(idx):
        p = [b for b in range(M) if st >> b & 1][0]
        q = [b for b in range(M) if st >> (M + b) & 1][0]
        C[p, q] = vec[k, 0]
    u, _, vt = np.linalg.svd(C)
    psi_a, psi_b = u[:, :1], vt[:1].T
    dt, W = 0.02, 3000
    o = Oracle(s.h1, s.L, 0.0, psi_a, psi_b, dt=dt, free_projection=True)
    phi0 = np.concatenate([psi_a, psi_b], 1).astype(complex)
    o.init_walkers(np.repeat(phi0[None], W, 0))
    assert o.trial_energy() - E0 > 0.02   # the test can tell the trial from E0
    Hd = H.toarray()
    psiT = F.walker_state(phi0, na)
    rng = np.random.default_rng(1)
    checks = {20, 40, 60}
    for k in range(1, 61):
        o.step(rng.standard_normal((W, X)))
        if o.nstep % 5 == 0:
            o.orthogonalise()
        if k in checks:
            e, emix = o.local_energy()
            num, den = o.w * e[:, 3], o.w
            G = 20
            gi = np.arange(W) % G
            jk = np.array([(num[gi != g].sum() / den[gi != g].sum()).real for g in range(G)])
            err = np.sqrt((G - 1) / G * np.sum((jk - jk.mean()) ** 2))
            prop = scipy.linalg.expm(-k * dt * Hd) @ psiT
            exact = (np.vdot(psiT, Hd @ prop) / np.vdot(psiT, prop)).real
            assert abs(emix - exact) < 4 * err + 2e-4, (k, emix, exact, err)
    assert abs(emix - E0) < 4 * err + 2e-3
