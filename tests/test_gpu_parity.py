"""GPU (FP64 path) against the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerance: 1e-10 relative per walker for walker matrices, overlaps, weights and
each energy component, as the FP64 target states.  Sizes span several tiles of
every kernel with ragged tails (odd X, N not a multiple of the column chunk,
M not a multiple of 32).
"""
import numpy as np
import pytest

from gpu_common import (assert_energy_parity, assert_state_parity, make_pair, need_gpu, rel,
                        walker_rel)
from oracle import philox
from paper_2209_04015_b300.synthetic import (gaussian_fields, make_config, make_system,
                                             perturbed_walkers, trial_walkers)

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


RAGGED = dict(M=37, na=5, nb=3, X=71, W=13)


def ragged_system(seed=4):
    return make_system(RAGGED["M"], RAGGED["na"], RAGGED["nb"], RAGGED["X"], seed=seed,
                       decay="geometric", e0=0.37)


def test_philox_words_bit_exact_and_fields_match():
    s = make_system(9, 2, 2, 37, seed=1)
    ctx, _ = make_pair(s, 11, seed=123456789012345)
    for step in (0, 7, (1 << 32) + 3):
        words = ctx.philox_words(step)
        ref = philox.field_words(step, 11, 37, 123456789012345)
        assert np.array_equal(words, ref)
        f = ctx.philox_fields(step)
        fr = philox.gaussian_fields(step, 11, 37, 123456789012345)
        assert np.all(np.abs(f - fr) <= 4e-16 * np.maximum(1.0, np.abs(fr)) * 8)


@pytest.mark.parametrize("exchange", ["direct", "stored"])
@pytest.mark.parametrize("cfg", ["c1", "ragged", "c2"])
def test_trial_energy_and_initial_energy(cfg, exchange):
    if cfg == "ragged":
        s, W = ragged_system(), RAGGED["W"]
    else:
        s, c = make_config(cfg)
        W = c["W"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc = make_pair(s, W, phi=phi, exchange=exchange)
    assert ctx.exchange_algorithm() == exchange
    assert abs(ctx.trial_energy() - orc.trial_energy()) <= TOL * abs(orc.trial_energy())
    assert rel(ctx.get_overlaps(), orc.ovlp).max() <= TOL
    assert_energy_parity(ctx, orc, TOL)


@pytest.mark.parametrize("exchange", ["direct", "stored"])
@pytest.mark.parametrize("cfg,nsteps", [("c1", 10), ("ragged", 12), ("c2", 3)])
def test_propagation_with_host_fields(cfg, nsteps, exchange):
    if cfg == "ragged":
        s, W = ragged_system(), RAGGED["W"]
    else:
        s, c = make_config(cfg)
        W = c["W"]
    ctx, orc = make_pair(s, W, exchange=exchange)
    fields = np.stack([gaussian_fields(W, s.X, seed=100 + k) for k in range(nsteps)])
    ctx.propagate(fields, nsteps)
    orc.propagate(list(fields))
    assert ctx.get_step() == nsteps
    assert_state_parity(ctx, orc, TOL)
    xb = ctx.get_force_bias()
    assert np.max(np.abs(xb - orc.last.xbar)) <= TOL * np.max(np.abs(orc.last.xbar))
    assert_energy_parity(ctx, orc, TOL)


def test_device_philox_path_matches_oracle_fields():
    s, c = make_config("c1")
    W = c["W"]
    ctx, orc = make_pair(s, W, seed=1)
    ctx.propagate(None, c["steps"])
    orc.propagate([philox.gaussian_fields(k, W, s.X, 1) for k in range(c["steps"])])
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


def test_free_projection_parity():
    s = ragged_system(seed=6)
    W = 7
    ctx, orc = make_pair(s, W, free_projection=True, dt=0.01)
    fields = np.stack([gaussian_fields(W, s.X, seed=200 + k) for k in range(6)])
    ctx.propagate(fields, 6)
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


def test_force_bias_cap_parity():
    s = make_system(12, 3, 2, 30, seed=8, decay="half")
    s.L[:] *= 6.0
    W = 9
    phi = perturbed_walkers(s, W, eps=0.8, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, fb_cap=0.05, dt=0.02)
    fields = np.stack([gaussian_fields(W, s.X, seed=300 + k) for k in range(3)])
    ctx.propagate(fields, 3)
    orc.propagate(list(fields))
    assert np.max(np.abs(orc.last.xbar)) <= 0.05 + 1e-15
    assert np.sum(np.isclose(np.abs(orc.last.xbar), 0.05)) > 0
    assert_state_parity(ctx, orc, TOL)


@pytest.mark.parametrize("exchange", ["direct", "stored"])
@pytest.mark.parametrize("M,na,nb,X,W", [(6, 3, 0, 5, 4), (5, 1, 1, 1, 1), (33, 1, 2, 2, 3),
                                         (40, 12, 11, 64, 5), (70, 9, 5, 90, 37)])
def test_edge_shapes(M, na, nb, X, W, exchange):
    s = make_system(M, na, nb, X, seed=9, decay="half")
    phi = perturbed_walkers(s, W, eps=0.2, seed=5)
    ctx, orc = make_pair(s, W, phi=phi, qr_period=2, exchange=exchange)
    fields = np.stack([gaussian_fields(W, X, seed=400 + k) for k in range(4)])
    ctx.propagate(fields, 4)
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


@pytest.mark.parametrize("exchange", ["direct", "stored"])
def test_maximum_sizes(exchange):
    """The ABI's limits: 64 electrons per spin, and 1024 orbitals with the direct
    exchange (the FP64 propagator narrows its column chunk to fit shared memory; the
    split path's long rows take the two-pass slicing); the stored exchange at 64 + 64
    electrons on 200 orbitals (its tensor at 1024 orbitals would be (64 x 1024)^2
    doubles per spin)."""
    M = 1024 if exchange == "direct" else 200
    s = make_system(M, 64, 64, 5, seed=9, decay="half")
    W = 2
    phi = perturbed_walkers(s, W, eps=0.2, seed=5)
    ctx, orc = make_pair(s, W, phi=phi, qr_period=2, exchange=exchange)
    assert ctx.exchange_algorithm() == exchange
    fields = np.stack([gaussian_fields(W, s.X, seed=600 + k) for k in range(2)])
    ctx.propagate(fields, 2)
    orc.propagate(list(fields))
    assert_state_parity(ctx, orc, TOL)
    assert_energy_parity(ctx, orc, TOL)


def test_orthogonalise_entry_point():
    s = ragged_system(seed=2)
    W = 5
    phi = perturbed_walkers(s, W, eps=0.5, seed=8) * 1.7
    ctx, orc = make_pair(s, W, phi=phi)
    e_before, _ = ctx.local_energy()
    ctx.orthogonalise()
    orc.orthogonalise()
    assert_state_parity(ctx, orc, TOL)
    e_after, _ = ctx.local_energy()
    assert np.max(rel(e_after[:, 3], e_before[:, 3])) <= TOL


def test_orthogonalise_nearly_dependent_columns():
    """Second columns of each spin block within 1e-4 of the first (condition ~1e4)
    take the Gram-Schmidt reorthogonalisation pass: Q matches the oracle's Householder
    QR and stays orthonormal to working precision (a single classical pass would lose
    orthogonality at ~eps cond^2 ~ 1e-8)."""
    s = ragged_system(seed=3)
    W, na = 6, RAGGED["na"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=11)
    for c0 in (0, na):
        phi[:, :, c0 + 1] = phi[:, :, c0] + 1e-4 * phi[:, :, c0 + 1]
    ctx, orc = make_pair(s, W, phi=phi)
    ctx.orthogonalise()
    orc.orthogonalise()
    assert_state_parity(ctx, orc, TOL)
    q = ctx.get_walkers()
    for cols in (slice(0, na), slice(na, None)):
        qs = q[:, :, cols]
        gram = np.einsum("zpi,zpj->zij", qs.conj(), qs)
        assert np.max(np.abs(gram - np.eye(qs.shape[2]))) <= 1e-13


def test_checkpoint_resume_is_bit_exact():
    s, c = make_config("c1")
    W = c["W"]
    ctx, _ = make_pair(s, W)
    ctx.propagate(None, 3)
    phi, w, ov, st = ctx.get_walkers(), ctx.get_weights(), ctx.get_overlaps(), ctx.get_step()
    ctx.propagate(None, 4)
    ref_phi, ref_w = ctx.get_walkers(), ctx.get_weights()
    ctx2, _ = make_pair(s, W)
    ctx2.set_state(phi, w, ov, st)
    ctx2.propagate(None, 4)
    assert np.array_equal(ctx2.get_walkers(), ref_phi)
    assert np.array_equal(ctx2.get_weights(), ref_w)


def test_errors_are_reported_not_faulted():
    from paper_2209_04015_b300 import AfqContext, AfqError
    s = make_system(8, 2, 2, 6, seed=1, decay="half")
    ctx = AfqContext()
    with pytest.raises(AfqError) as e:
        ctx.propagate(None, 1)
    assert e.value.code == 5  # AFQ_ERR_STATE
    h = s.h1.copy()
    h[0, 1] += 1e-3
    with pytest.raises(AfqError) as e:
        ctx.init_hamiltonian(h, s.L)
    assert e.value.code == 1  # AFQ_ERR_ARG
    ctx.init_hamiltonian(s.h1, s.L)
    ctx.init_trial(s.psi_a, s.psi_b)
    phi = trial_walkers(s, 3)
    phi[1, :, 1] = 0.0          # a walker whose overlap matrix is singular
    with pytest.raises(AfqError) as e:
        ctx.init_walkers(3, phi)
    assert e.value.code == 3  # AFQ_ERR_SINGULAR
    ctx.init_walkers(3, trial_walkers(s, 3))
    ctx.propagate(None, 2)      # the context stays usable after the reported error


def test_c2_full_size_sampled_walkers():
    """c2 at full size in the launch configuration of the benchmark: 128 walkers, device
    Philox fields, QR every 5 steps; 6 walkers re-run by the oracle one set at a time
    (walkers are independent, so a subset with its own field rows gives the same values)."""
    s, c = make_config("c2")
    W, nsteps = c["W"], 6
    ctx, _ = make_pair(s, W)
    ctx.propagate(None, nsteps)
    e, _ = ctx.local_energy()
    idx = np.array([0, 17, 64, 99, 126, 127])
    from oracle.afqmc import Oracle
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=c.get("dt", 0.005))
    orc.init_walkers(trial_walkers(s, len(idx)))
    orc.propagate([philox.gaussian_fields(k, W, s.X, 1)[idx] for k in range(nsteps)])
    phi = ctx.get_walkers()[idx]
    assert walker_rel(phi, orc.phi).max() <= TOL
    assert rel(ctx.get_weights()[idx], orc.w).max() <= TOL
    eref, _ = orc.local_energy()
    assert rel(e[idx, 3], eref[:, 3]).max() <= TOL


def test_c3_fp64_full_size_sampled_walkers():
    """The benchmark's main line: 290 orbitals, 26 + 26 electrons, 1500 Cholesky
    vectors, 640 walkers in FP64, autotuned as the benchmark runs it (the stored
    exchange), device Philox fields, 5 steps ending with a QR, then the local energy;
    3 walkers re-run by the oracle alone (walkers are independent, so a subset with its
    own field rows gives the same values), each energy part, weight and walker element
    within 1e-10."""
    s, c = make_config("c3")
    W, nsteps = c["W"], 5
    ctx, _ = make_pair(s, W)
    ctx.autotune()
    assert ctx.exchange_algorithm() == "stored"
    ctx.propagate(None, nsteps)
    e, _ = ctx.local_energy()
    idx = np.array([0, 333, 639])
    from oracle.afqmc import Oracle
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005)
    orc.init_walkers(trial_walkers(s, len(idx)))
    orc.propagate([philox.gaussian_fields(k, W, s.X, 1)[idx] for k in range(nsteps)])
    assert walker_rel(ctx.get_walkers()[idx], orc.phi).max() <= TOL
    assert rel(ctx.get_weights()[idx], orc.w).max() <= TOL
    eref, _ = orc.local_energy()
    for k in range(4):
        scale = np.maximum(np.abs(eref[:, k]), 1e-3 * np.abs(eref[:, 3]))
        assert np.all(np.abs(e[idx, k] - eref[:, k]) <= TOL * scale), k
    ctx.close()


def test_recreated_contexts_on_reused_memory_are_identical():
    """Contexts destroyed and re-created while others stay alive reuse device memory
    that holds stale values (NaN bit patterns included); no kernel may read memory it
    did not write first (a set-up y = a x + 0 y once turned such NaNs into P)."""
    from paper_2209_04015_b300 import AfqContext
    others = []
    for k in range(3):
        s = make_system(30 + 7 * k, 4, 3, 40, seed=20 + k)
        c = AfqContext(precision="split_bf16" if k % 2 else "fp64")
        c.init_hamiltonian(s.h1, s.L, s.e0)
        c.init_trial(s.psi_a, s.psi_b)
        c.init_walkers(16)
        c.propagate(None, 2)
        others.append(c)
    s = make_system(48, 6, 5, 90, seed=3)
    results = []
    for rep in range(3):
        for prec in ("fp64", "split_bf16"):
            c = AfqContext(precision=prec)
            c.init_hamiltonian(s.h1, s.L, s.e0)
            c.init_trial(s.psi_a, s.psi_b)
            c.init_walkers(24)
            c.propagate(None, 3)
            e, _ = c.local_energy()
            results.append((prec, c.get_walkers(), e))
            c.close()
    for i in range(2, len(results)):
        assert results[i][0] == results[i - 2][0]
        assert np.array_equal(results[i][1], results[i - 2][1])
        assert np.array_equal(results[i][2], results[i - 2][2])


def test_auto_exchange_choice_and_agreement():
    """AUTO takes the stored tensor where it needs fewer multiply-adds (M < 1.5 X) and
    the direct form elsewhere; both give the same energies to rounding."""
    s, c = make_config("c2")
    W = 40
    phi = perturbed_walkers(s, W, eps=0.3, seed=4)
    ctx_a, _ = make_pair(s, W, phi=phi)
    ctx_d, _ = make_pair(s, W, phi=phi, exchange="direct")
    assert ctx_a.exchange_algorithm() == "stored"
    ea, _ = ctx_a.local_energy()
    ed, _ = ctx_d.local_energy()
    assert np.max(np.abs(ea[:, 2] - ed[:, 2])) <= 1e-12 * np.max(np.abs(ed[:, 2]))
    wide = make_system(60, 4, 4, 30, seed=3)
    ctx_w, _ = make_pair(wide, 3)
    assert ctx_w.exchange_algorithm() == "direct"
