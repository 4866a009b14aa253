"""Mixed <S^2> estimator and the weighted mixed one-body density matrix on the GPU
(through the C ABI) against the oracle, which forms the Green's functions walker by
walker; the oracle itself is pinned by brute force in Fock space.  Tolerance 1e-10
relative (of max(1, |S2|), or of the largest matrix entry), as for every FP64
quantity."""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu
from oracle.estimators import one_rdm, spin_squared
from paper_2209_04015_b300.synthetic import gaussian_fields, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _check(ctx, orc):
    got, mix = ctx.spin_squared()
    ref, rmix = spin_squared(orc)
    scale = np.maximum(1.0, np.abs(ref))
    assert np.max(np.abs(got - ref) / scale) <= TOL, np.max(np.abs(got - ref) / scale)
    assert abs(mix - rmix) <= TOL * max(1.0, abs(rmix))
    return got


@pytest.mark.parametrize("shape", [(37, 5, 3, 71, 13), (29, 4, 0, 33, 5), (90, 40, 36, 45, 3),
                                   (130, 64, 64, 20, 2)])
def test_s2_matches_oracle_after_steps(shape):
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=8, decay="geometric", e0=0.2)
    phi = perturbed_walkers(s, W, eps=0.4, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, qr_period=2)
    _check(ctx, orc)
    fields = np.stack([gaussian_fields(W, s.X, seed=40 + k) for k in range(3)])
    ctx.propagate(fields, 3)  # weights and a QR in between
    orc.propagate(list(fields))
    _check(ctx, orc)


def test_s2_of_a_closed_shell_trial_is_zero_and_split_contexts_agree():
    M, n = 24, 4
    s = make_system(M, n, n, 17, seed=2, decay="geometric")
    s.psi_b = s.psi_a.copy()  # restricted closed shell: a singlet
    ctx, orc = make_pair(s, 3)
    got = _check(ctx, orc)
    assert np.max(np.abs(got)) < 1e-12
    phi = perturbed_walkers(s, 6, eps=0.5, seed=9)
    for precision in ("fp64", "split_bf16"):
        c2, o2 = make_pair(s, 6, phi=phi, precision=precision)
        _check(c2, o2)


@pytest.mark.parametrize("shape,free", [((37, 5, 3, 71, 9), False), ((37, 5, 3, 71, 9), True),
                                        ((29, 4, 0, 33, 5), False)])
def test_one_rdm_matches_oracle(shape, free):
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=8, decay="geometric", e0=0.2)
    phi = perturbed_walkers(s, W, eps=0.4, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, qr_period=2, free_projection=free,
                         dt=0.01 if free else 0.005)
    _one_rdm_after_steps(ctx, orc, s, W, X, na, nb, TOL)


def test_one_rdm_of_a_split_context():
    """A split-precision context's walkers differ from the oracle's after steps (the
    propagation's digits); at the same walkers (set from the oracle) its FP64
    estimator agrees at 1e-10."""
    M, na, nb, X, W = 37, 5, 3, 71, 9
    s = make_system(M, na, nb, X, seed=8, decay="geometric", e0=0.2)
    phi = perturbed_walkers(s, W, eps=0.4, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, precision="split_bf16")
    w = np.linspace(0.5, 1.5, W)
    ctx.init_walkers(W, phi, w)
    orc.init_walkers(phi, w)
    g = ctx.one_rdm()
    ref = one_rdm(orc)
    assert np.max(np.abs(g - ref)) <= TOL * np.max(np.abs(ref))


def _one_rdm_after_steps(ctx, orc, s, W, X, na, nb, tol):
    fields = np.stack([gaussian_fields(W, X, seed=70 + k) for k in range(3)])
    ctx.propagate(fields, 3)  # weights (complex in free projection) and a QR in between
    orc.propagate(list(fields))
    g = ctx.one_rdm()
    ref = one_rdm(orc)
    assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref))
    assert abs(np.trace(g[0]) - na) < 1e-10 and abs(np.trace(g[1]) - nb) < 1e-10
