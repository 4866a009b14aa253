"""The allocation-free exchange entry point against the context path (GPU).

afq_exchange_energy_static serves callers that cannot call cudaMalloc, for
example a host framework whose own pool or fixed arena owns all device memory,
or a latency-critical loop that must avoid cudaMalloc's device synchronisation.
Its partial sums live in the library's static device array instead of an
allocation.  This test feeds it the same half-rotated Cholesky vectors and theta
matrices that the context uses and compares its exchange energies with column EK
of afq_local_energy, within the FP64 tolerance of the other parity tests, on two
calls in a row of different sizes (the second call must not see the first
call's leftovers in the shared array).
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu
from oracle.afqmc import half_rotated_cholesky, overlap_and_theta
from paper_2209_04015_b300 import afqmc as binding
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-10


def device_inputs(s, phi):
    """L~ as X x N x M and theta^T as W x N x M complex, on the device."""
    import torch
    Lt = np.concatenate([half_rotated_cholesky(s.L, s.psi_a),
                         half_rotated_cholesky(s.L, s.psi_b)], axis=1)
    _, ta = overlap_and_theta(s.psi_a, phi[:, :, :s.na])
    _, tb = overlap_and_theta(s.psi_b, phi[:, :, s.na:])
    thetaT = np.concatenate([np.swapaxes(ta, 1, 2), np.swapaxes(tb, 1, 2)], axis=1)
    Lt_d = torch.from_numpy(np.ascontiguousarray(Lt)).cuda()
    th_d = torch.from_numpy(np.ascontiguousarray(thetaT)).cuda()
    return Lt_d, th_d


def run_static(s, W, phi):
    import torch
    Lt_d, th_d = device_inputs(s, phi)
    ek_d = torch.full((W,), complex("nan"), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    binding.exchange_energy_static(s.M, s.X, s.na, s.nb, W, Lt_d.data_ptr(), th_d.data_ptr(),
                                   ek_d.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return ek_d.cpu().numpy()


def context_exchange(s, W, phi):
    ctx, _ = make_pair(s, W, phi=phi)
    e, _ = ctx.local_energy()
    return e[:, 2]


def test_static_scratch_exchange_matches_context_path_twice():
    need_gpu()
    cases = []
    s1 = make_system(37, 5, 3, 71, seed=4, decay="geometric")
    cases.append((s1, 13, perturbed_walkers(s1, 13, eps=0.3, seed=2)))
    s2, c2 = make_config("c2")
    cases.append((s2, c2["W"], perturbed_walkers(s2, c2["W"], eps=0.3, seed=5)))
    for s, W, phi in cases:
        got = run_static(s, W, phi)
        ref = context_exchange(s, W, phi)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= TOL


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
