"""The split-precision propagation as one cluster kernel (prop_kernel = 1) and as
per-pass kernels with one MMA per digit pair (prop_kernel = 2) against the default
per-pass kernels, whose passes of up to 4 digits issue one MMA per A digit over the
concatenated B digits (GPU).

Both forms run the same arithmetic (the same digits, row exponents, digit products,
recombination and FP64 updates in the same order), the cluster kernel with every GEMM
pass of a walker in one launch and the exponents exchanged between the CTAs of a
cluster, the per-pass form with separate slicing launches.  So after steps with the
same fields, including a QR, the walkers, overlaps, weights and energies must be
bit-identical; the per-pass form itself is checked against the oracle in
test_gpu_mixed.py.  Shapes: one 128-row slab (clusters of one CTA) with narrow and
wide column tiles, two column tiles per walker, clusters of 3 and of 8 CTAs, an empty
spin, and the 290-orbital shape on a few walkers.
"""
import numpy as np
import pytest

from gpu_common import need_gpu
from paper_2209_04015_b300.synthetic import gaussian_fields, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu


def ctx_for(s, W, phi, kernel, **kw):
    from paper_2209_04015_b300 import AfqContext
    ctx = AfqContext(dt=0.005, qr_period=5, precision="split_bf16", prop_kernel=kernel, **kw)
    ctx.init_hamiltonian(s.h1, s.L, s.e0)
    ctx.init_trial(s.psi_a, s.psi_b)
    ctx.init_walkers(W, phi)
    return ctx


@pytest.mark.parametrize("other", ["fused", "per_pair"])
@pytest.mark.parametrize("shape", [
    (37, 5, 3, 71, 13),      # one slab, 16-column tile
    (100, 10, 10, 400, 24),  # one slab, 32-column tile
    (96, 40, 40, 101, 7),    # two 64-column tiles per walker
    (300, 26, 26, 150, 9),   # clusters of 3 slabs (the 290-orbital tiling)
    (50, 7, 0, 66, 9),       # no beta electrons
    (1024, 64, 64, 5, 2),    # clusters of 8 slabs, two column tiles
])
def test_other_kernels_are_bit_identical_to_per_pass(shape, other):
    """The same digits, row exponents and exact integer sums per TMEM accumulator in
    every form, so the same bits after 6 steps with a QR."""
    need_gpu()
    M, na, nb, X, W = shape
    s = make_system(M, na, nb, X, seed=M + na, decay="geometric", e0=0.1)
    phi = perturbed_walkers(s, W, eps=0.3, seed=3)
    fused = ctx_for(s, W, phi, other)
    ref = ctx_for(s, W, phi, "per_pass")
    nsteps = 6  # a QR after the fifth
    fields = np.stack([gaussian_fields(W, s.X, seed=90 + k) for k in range(nsteps)])
    fused.propagate(fields, nsteps)
    ref.propagate(fields, nsteps)
    assert np.array_equal(fused.get_walkers(), ref.get_walkers())
    assert np.array_equal(fused.get_overlaps(), ref.get_overlaps())
    assert np.array_equal(fused.get_weights(), ref.get_weights())
    e, _ = fused.local_energy()
    er, _ = ref.local_energy()
    assert np.array_equal(e, er)
    assert np.all(np.isfinite(e))
    fused.close()
    ref.close()


def test_cluster_kernel_device_fields_and_launch_count():
    """Device Philox fields; the cluster kernel takes one launch per step where the
    per-pass form takes 2 n + 5 (n = 6 Taylor terms)."""
    need_gpu()
    s = make_system(300, 26, 26, 150, seed=5, decay="geometric")
    W = 12
    phi = perturbed_walkers(s, W, eps=0.3, seed=4)
    fused = ctx_for(s, W, phi, "fused")
    ref = ctx_for(s, W, phi, "per_pass")
    n0f, n0r = fused.launch_count(), ref.launch_count()
    fused.propagate(None, 3)
    ref.propagate(None, 3)
    # per step the per-pass form launches the transpose, Phi's slicing, 8 GEMM passes
    # and 7 Taylor slicing passes (17) where the cluster kernel launches once
    assert (ref.launch_count() - n0r) - (fused.launch_count() - n0f) == 3 * 16
    assert np.array_equal(fused.get_walkers(), ref.get_walkers())
    fused.close()
    ref.close()
