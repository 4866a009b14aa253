"""Split-precision (bf16 slices on tcgen05 tensor cores) against FP64 references.

Tolerances: the mixed-precision target is a mixed-energy error of at most 1e-6 Ha
per walker against the FP64 oracle.  The GEMM engine's error, relative to
max|A| max|B| sqrt(K), must fall by 30x from one slice (bf16, 2^-8) to two
(~2^-16); a third slice then meets the FP32 accumulation floor of the tensor core
(measured ~3e-7 at K = 150 and ~9e-7 at K = 1000), so it must stay within 1.5x of
two slices and below 2e-6.
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu, walker_rel
from oracle import philox
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
E_TOL = 1e-6  # Ha per walker


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def split_gemm(A, B, slices):
    import torch
    from paper_2209_04015_b300 import afqmc as binding
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Cd = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float64, device="cuda")
    binding.gemm_split_bf16(A.shape[0], B.shape[0], A.shape[1], slices, Ad.data_ptr(),
                            Bd.data_ptr(), Cd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return Cd.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(300, 200, 150), (128, 300, 64), (77, 16, 1000)])
def test_split_gemm_error_shrinks_with_slices(m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k)) * np.exp(rng.standard_normal((n, 1)))
    ref = A @ B.T
    scale = np.abs(A).max() * np.abs(B).max() * np.sqrt(k)
    errs = [np.abs(split_gemm(A, B, s) - ref).max() / scale for s in (1, 2, 3)]
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 30
    assert errs[2] <= 1.5 * errs[1]
    assert errs[2] < 2e-6, errs


def mixed_vs_oracle(s, W, phi, nsteps, fields=None, **kw):
    ctx, orc = make_pair(s, W, phi=phi, precision="split_bf16", **kw)
    e0, _ = ctx.local_energy()
    e0_ref, _ = orc.local_energy()
    if nsteps:
        if fields is None:
            fields = [philox.gaussian_fields(k, W, s.X, 1) for k in range(nsteps)]
        ctx.propagate(np.stack(fields), nsteps)
        orc.propagate(list(fields))
    e1, _ = ctx.local_energy()
    e1_ref, _ = orc.local_energy()
    return ctx, orc, e0, e0_ref, e1, e1_ref


@pytest.mark.parametrize("exchange", ["direct", "stored"])
@pytest.mark.parametrize("cfg", ["ragged", "wide", "uneven", "one_spin", "c2", "max"])
def test_mixed_energy_within_1e6_of_fp64_oracle(cfg, exchange):
    if cfg == "ragged":
        s = make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)
        W = 13
    elif cfg == "wide":
        # 80 walker columns (two propagation column tiles), 40 electrons per spin
        # (exchange rows beyond one warp), 7 walkers (not a multiple of the exchange
        # walker block)
        s = make_system(96, 40, 40, 101, seed=6, decay="geometric", e0=-0.2)
        W = 7
    elif cfg == "uneven":
        # unequal spins (two exchange launches), one electron in one spin
        s = make_system(45, 9, 1, 57, seed=8, decay="geometric", e0=0.1)
        W = 5
    elif cfg == "one_spin":
        # no beta electrons: the beta blocks of every contraction are empty
        s = make_system(50, 7, 0, 66, seed=12, decay="geometric", e0=0.2)
        W = 9
    elif cfg == "max":
        # 64 electrons per spin; 1024 orbitals with the direct exchange (rows past 512:
        # the two-pass slicing), 200 with the stored one
        s = make_system(1024 if exchange == "direct" else 200, 64, 64, 5, seed=9,
                        decay="half")
        W = 2
    else:
        s, c = make_config("c2")
        W = c["W"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc, e0, e0r, e1, e1r = mixed_vs_oracle(s, W, phi, 2, exchange=exchange)
    assert ctx.exchange_algorithm() == exchange
    for e, er in ((e0, e0r), (e1, e1r)):
        # 1e-6 Ha; the synthetic maximum-size walkers reach |E_L| ~ 1e3 Ha, where the
        # bound is the same relative error as 1e-6 Ha at the 290-orbital energies
        # (2e-8 |E|)
        tol = E_TOL if cfg != "max" else max(E_TOL, 2e-8 * np.max(np.abs(er[:, 3])))
        assert np.max(np.abs(e[:, 3] - er[:, 3])) <= tol
        assert np.max(np.abs(e[:, 2] - er[:, 2])) <= tol   # exchange
        assert np.max(np.abs(e[:, 1] - er[:, 1])) <= tol   # Coulomb
    # propagated in split precision (VHS, Taylor terms and one-body halves on the tensor
    # cores, identity parts in FP64): walkers stay within 1e-6 relative after 2 steps
    dphi = walker_rel(ctx.get_walkers(), orc.phi).max()
    print(f"{cfg} {exchange}: 2-step max rel dPhi {dphi:.2e}, "
          f"max |dE_L| {np.max(np.abs(e1[:, 3] - e1r[:, 3])):.2e}, "
          f"max |dE_K| {np.max(np.abs(e1[:, 2] - e1r[:, 2])):.2e}")
    assert dphi < 1e-6


def test_mixed_trajectory_error_over_20_steps():
    """The split-precision trajectory over 20 steps: energies within 1e-6 Ha of the
    oracle, walkers and weights within 1e-6 relative."""
    s = make_system(37, 5, 3, 71, seed=4, decay="geometric", e0=0.37)
    W = 13
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    ctx, orc, _, _, e1, e1r = mixed_vs_oracle(s, W, phi, 20)
    de = np.max(np.abs(e1[:, 3] - e1r[:, 3]))
    dphi = walker_rel(ctx.get_walkers(), orc.phi).max()
    dw = np.max(np.abs(ctx.get_weights().real - orc.w) / np.abs(orc.w))
    print(f"20 steps: max |dE_L| {de:.2e} Ha, max rel dPhi {dphi:.2e}, max rel dw {dw:.2e}")
    assert de <= E_TOL and dphi <= 1e-6 and dw <= 1e-6


@pytest.mark.parametrize("exchange", ["direct", "stored"])
def test_mixed_c3_shape_sampled_walkers(exchange):
    """The paper's large shape (290 orbitals, 26+26 electrons, 1500 Cholesky vectors,
    640 walkers), one step with device fields; 4 walkers re-run by the oracle."""
    s, c = make_config("c3")
    W = c["W"]
    phi = perturbed_walkers(s, W, eps=0.3, seed=2)
    from paper_2209_04015_b300 import AfqContext
    from oracle.afqmc import Oracle
    ctx = AfqContext(dt=0.005, precision="split_bf16", exchange=exchange)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W, phi)
    e0, _ = ctx.local_energy()
    ctx.propagate(None, 1)
    e1, _ = ctx.local_energy()
    idx = np.array([0, 211, 503, 639])
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005)
    orc.init_walkers(phi[idx])
    e0r, _ = orc.local_energy()
    orc.propagate([philox.gaussian_fields(0, W, s.X, 1)[idx]])
    e1r, _ = orc.local_energy()
    assert ctx.exchange_algorithm() == exchange
    # both exchange algorithms accumulate exactly where it matters: the stored one in
    # exact digit diagonals, the direct one with its leading digit product in an exact
    # accumulator (only the ~2^-8 tail sees the tensor core's biased FP32 sums)
    for e, er in ((e0[idx], e0r), (e1[idx], e1r)):
        assert np.max(np.abs(e[:, 3] - er[:, 3])) <= E_TOL
        assert np.max(np.abs(e[:, 2] - er[:, 2])) <= E_TOL   # exchange
        assert np.max(np.abs(e[:, 1] - er[:, 1])) <= E_TOL   # Coulomb (exact digits)


def test_mixed_c3_100_steps_against_oracle():
    """The paper's large shape (290 orbitals, 26+26 electrons, 1500 Cholesky vectors,
    640 walkers) in split precision for 100 steps with host fields and the QR every 5
    steps; two walkers re-run by the oracle alone (walkers are independent, so a
    subset with its own field rows is the same computation).  After 100 steps every
    energy part stays within 1e-6 Ha of the oracle and every walker element within
    1e-6 of the walker's largest element."""
    from oracle.afqmc import Oracle
    from paper_2209_04015_b300 import AfqContext
    s, c = make_config("c3")
    W, nsteps = c["W"], 100
    idx = np.array([0, 517])
    ctx = AfqContext(dt=0.005, qr_period=5, precision="split_bf16")
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W)
    orc = Oracle(s.h1, s.L, s.e0, s.psi_a, s.psi_b, dt=0.005, qr_period=5)
    orc.init_walkers(ctx.get_walkers()[idx])
    rng = np.random.default_rng(2024)
    sub = []
    for _ in range(nsteps):
        xi = rng.standard_normal((W, s.X))
        ctx.propagate(xi, 1)
        sub.append(xi[idx].copy())
    orc.propagate(sub)
    e, _ = ctx.local_energy()
    eref, _ = orc.local_energy()
    de = np.abs(e[idx] - eref)
    print("c3 100 steps, max |dE| (E1, EJ, EK, E_L):", de.max(axis=0))
    assert de.max() <= E_TOL, de.max(axis=0)
    dphi = walker_rel(ctx.get_walkers()[idx], orc.phi).max()
    assert dphi <= 1e-6, dphi
    ctx.close()


def test_propagation_digit_schedule():
    """The split propagation keeps all prop_slices digits on the two P passes and on
    powers larger than ~1e-3 of Phi, and never more digits on a power than on the
    one before it; an FP64 context has no schedule."""
    from paper_2209_04015_b300 import AfqContext
    from paper_2209_04015_b300.afqmc import AFQ_ERR_STATE, AfqError
    s, c = make_config("c2")
    for slices in (4, 3):
        ctx = AfqContext(dt=0.005, precision="split_bf16", prop_slices=slices)
        ctx.init_hamiltonian(s.h1, s.L, s.e0)
        ctx.init_trial(s.psi_a, s.psi_b)
        digits, x = ctx.prop_digits()
        n = ctx.params.taylor_order
        assert len(digits) == n + 2 and digits[0] == digits[-1] == slices
        powers = digits[1:-1]
        assert all(1 <= d <= slices for d in powers)
        assert all(a >= b for a, b in zip(powers, powers[1:]))
        assert 0.01 < x < 1.0
        import math
        for k, d in enumerate(powers, start=1):
            if x ** k / math.factorial(k) > 1e-3:
                assert d == slices, (k, d)
        ctx.close()
    fp = AfqContext(dt=0.005)
    fp.init_hamiltonian(s.h1, s.L, s.e0)
    fp.init_trial(s.psi_a, s.psi_b)
    with pytest.raises(AfqError) as e:
        fp.prop_digits()
    assert e.value.code == AFQ_ERR_STATE
