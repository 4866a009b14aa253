"""The allocation-free exchange entry point (GPU).

afq_exchange_energy_static serves callers that cannot call cudaMalloc, for
example a host framework whose own pool or fixed arena owns all device memory,
or a latency-critical loop that must avoid cudaMalloc's device synchronisation.
Its partial sums live in the library's static device array instead of an
allocation.

The tests feed it half-rotated Cholesky vectors and theta matrices formed by the
oracle and compare its exchange energies with the oracle's exchange_energy (the
per-walker T_ij T_ji sum of Sec. "Local energy") within the FP64 tolerance of the
other parity tests, on two calls in a row: the second is smaller and uses a
different Cholesky group size, so it reads slots that the first call left filled
with its own values, and would see them if it did not rewrite every slot it reads.
A third test checks that a call never lowers the shared-memory limit of the
exchange kernel that an FP64 context with more electrons relies on.

The file is named to be collected last: it runs after every other test.
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu
from oracle.afqmc import exchange_energy, half_rotated_cholesky, overlap_and_theta
from paper_2209_04015_b300 import afqmc as binding
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-10


def group_size(na, nb):
    """Cholesky vectors per exchange group of the kernel, max(1, 64 / max n_s)."""
    return max(1, 64 // max(na, nb))


def oracle_inputs(s, phi):
    """L~ (X x N x M), theta^T (W x N x M) and the oracle's exchange energy per walker."""
    Lt_a = half_rotated_cholesky(s.L, s.psi_a)
    Lt_b = half_rotated_cholesky(s.L, s.psi_b)
    _, ta = overlap_and_theta(s.psi_a, phi[:, :, :s.na])
    _, tb = overlap_and_theta(s.psi_b, phi[:, :, s.na:])
    ek = exchange_energy(Lt_a, ta)
    if s.nb:
        ek = ek + exchange_energy(Lt_b, tb)
    Lt = np.concatenate([Lt_a, Lt_b], axis=1)
    thetaT = np.concatenate([np.swapaxes(ta, 1, 2), np.swapaxes(tb, 1, 2)], axis=1)
    return np.ascontiguousarray(Lt), np.ascontiguousarray(thetaT), ek


def run_static(s, W, Lt, thetaT):
    import torch
    Lt_d = torch.from_numpy(Lt).cuda()
    th_d = torch.from_numpy(thetaT).cuda()
    ek_d = torch.full((W,), complex("nan"), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    binding.exchange_energy_static(s.M, s.X, s.na, s.nb, W, Lt_d.data_ptr(), th_d.data_ptr(),
                                   ek_d.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return ek_d.cpu().numpy()


def test_static_scratch_exchange_matches_oracle_twice():
    need_gpu()
    big, cbig = make_config("c2")             # 100 orbitals, 10 + 10, X = 400, W = 128
    small = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    cases = [(big, cbig["W"], perturbed_walkers(big, cbig["W"], eps=0.3, seed=5)),
             (small, 13, perturbed_walkers(small, 13, eps=0.3, seed=2))]
    slots = [W * 2 * -(-s.X // group_size(s.na, s.nb)) for s, W, _ in cases]
    # the second call is smaller and groups the Cholesky vectors differently (6 vs 12
    # per group), so every slot it reads holds a value of the first call beforehand
    assert slots[1] < slots[0] <= binding.AFQ_STATIC_EXCHANGE_SLOTS
    assert group_size(big.na, big.nb) != group_size(small.na, small.nb)
    for s, W, phi in cases:
        Lt, thetaT, ref = oracle_inputs(s, phi)
        got = run_static(s, W, Lt, thetaT)
        assert np.all(np.isfinite(got))
        err = np.max(np.abs(got - ref) / np.abs(ref))
        assert err <= TOL, err


def test_static_call_keeps_context_exchange_launchable():
    """An FP64 context with 26 electrons per spin runs the direct exchange kernel with
    ~48 KB of shared memory; a static call for 5 + 3 electrons needs ~23 KB and must
    not lower the kernel's limit under the context's next launch."""
    need_gpu()
    s = make_system(60, 26, 26, 90, seed=7, decay="geometric")
    W = 6
    phi = perturbed_walkers(s, W, eps=0.3, seed=3)
    ctx, orc = make_pair(s, W, phi=phi, exchange="direct")
    assert ctx.exchange_algorithm() == "direct"
    e_before, _ = ctx.local_energy()
    small = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    phs = perturbed_walkers(small, 4, eps=0.3, seed=2)
    Lt, thetaT, ref = oracle_inputs(small, phs)
    got = run_static(small, 4, Lt, thetaT)
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= TOL
    e_after, _ = ctx.local_energy()          # raises AfqError if the launch fails
    assert np.array_equal(e_after[:, 2], e_before[:, 2])
    eref, _ = orc.local_energy()
    assert np.max(np.abs(e_after[:, 2] - eref[:, 2]) / np.abs(eref[:, 2])) <= TOL
    ctx.close()


def test_static_scratch_rejects_oversized_calls():
    need_gpu()
    import torch
    s = make_system(8, 1, 1, 4, seed=1, decay="half")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    too_many_walkers = binding.AFQ_STATIC_EXCHANGE_SLOTS
    with pytest.raises(binding.AfqError) as e:
        binding.exchange_energy_static(s.M, s.X, s.na, s.nb, too_many_walkers, buf.data_ptr(),
                                       buf.data_ptr(), buf.data_ptr(), None)
    assert e.value.code == binding.AFQ_ERR_ARG
