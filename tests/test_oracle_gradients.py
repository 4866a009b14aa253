"""Pins of the oracle's closed-form local-energy gradients (CPU).

Central finite differences (eps = 1e-6) of the oracle's own E_L, entry by entry,
with no symmetry imposed on the perturbed h1 or L_g; and dE/dh1 equals the mixed
one-body density matrix G = sum_s Psi_s theta_s^T.
"""
import numpy as np

from oracle import afqmc
from oracle.afqmc import Oracle
from oracle.gradients import local_energy_closed_form_derivatives, local_energy_vjp, loss
from paper_2209_04015_b300.synthetic import make_system, perturbed_walkers

EPS = 1e-6


def setup(M=6, na=2, nb=2, X=5, W=3, seed=3):
    s = make_system(M, na, nb, X, seed=seed, decay="half", e0=0.2)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b)
    phi = perturbed_walkers(s, W, eps=0.4, seed=seed + 1)
    g = np.random.default_rng(seed).standard_normal(W) + 1j * np.random.default_rng(seed + 9).standard_normal(W)
    return s, orc, phi, g


def test_dE_dh1_is_mixed_one_body_density():
    s, orc, phi, _ = setup()
    dh, _, _ = local_energy_closed_form_derivatives(orc, phi)
    ta, tb = orc.thetas(phi)
    G = afqmc.greens_function(s.psi_a, ta) + afqmc.greens_function(s.psi_b, tb)
    assert np.allclose(dh, G, atol=1e-14)


def test_grad_h1_matches_finite_differences():
    s, orc, phi, g = setup()
    gh, _, _ = local_energy_vjp(orc, phi, g)
    for p in range(s.M):
        for q in range(s.M):
            hp = s.h1.copy(); hp[p, q] += EPS
            hm = s.h1.copy(); hm[p, q] -= EPS
            fd = (loss(orc, phi, g, h1=hp) - loss(orc, phi, g, h1=hm)) / (2 * EPS)
            assert abs(fd - gh[p, q]) < 1e-7 * max(1.0, abs(gh[p, q])), (p, q, fd, gh[p, q])


def test_grad_L_matches_finite_differences():
    s, orc, phi, g = setup()
    _, gL, _ = local_energy_vjp(orc, phi, g)
    rng = np.random.default_rng(1)
    for _ in range(25):
        gi, p, q = rng.integers(s.X), rng.integers(s.M), rng.integers(s.M)
        Lp = s.L.copy(); Lp[gi, p, q] += EPS
        Lm = s.L.copy(); Lm[gi, p, q] -= EPS
        fd = (loss(orc, phi, g, L=Lp) - loss(orc, phi, g, L=Lm)) / (2 * EPS)
        assert abs(fd - gL[gi, p, q]) < 1e-7 * max(1.0, abs(gL[gi, p, q])), (gi, p, q, fd)


def test_grad_phi_matches_finite_differences():
    s, orc, phi, g = setup(na=3, nb=1)
    _, _, gphi = local_energy_vjp(orc, phi, g)
    for z in range(phi.shape[0]):
        for p in range(s.M):
            for j in range(s.na + s.nb):
                fd = []
                for d in (EPS, 1j * EPS):
                    pp = phi.copy(); pp[z, p, j] += d
                    pm = phi.copy(); pm[z, p, j] -= d
                    fd.append((loss(orc, pp, g) - loss(orc, pm, g)) / (2 * EPS))
                ref = fd[0] + 1j * fd[1]
                assert abs(ref - gphi[z, p, j]) < 1e-7 * max(1.0, abs(ref)), (z, p, j, ref)
