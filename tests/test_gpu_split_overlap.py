"""Split precision: the quantities the FP64-quality parts of the step produce (GPU).

In a split-precision context the overlap matrix S = Psi^T Phi and H = h~ Phi are
formed on the tensor cores with 7 exact digits, det S and S^-1 by double-float
Gauss-Jordan elimination, and the one-body energy as E1 = tr(S^-1 H) (Sec. "Overlap",
Eq. halfgf, and the one-body term of Sec. "Local energy"), while theta itself is cut to
the force bias's digit count.  So the overlaps and E1 must meet the FP64 path's bar
against the oracle (1e-10 relative), whatever theta's digits; EJ and EK go through
the digit GEMMs and meet the split-precision bar (1e-6 Ha).  Shapes: ragged, equal
spins with two theta K blocks (40 electrons), no beta electrons, and the 100-orbital
workload.
"""
import numpy as np
import pytest

from gpu_common import make_pair, need_gpu, rel
from paper_2209_04015_b300.synthetic import make_config, make_system, perturbed_walkers

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_HA = 1e-6


def _shape(name):
    if name == "c2":
        s, c = make_config("c2")
        return s, c["W"]
    M, na, nb, X, W, seed = {"ragged": (37, 5, 3, 71, 13, 4), "wide": (96, 40, 40, 101, 5, 6),
                             "one_spin": (50, 7, 0, 66, 6, 12)}[name]
    return make_system(M, na, nb, X, seed=seed, decay="geometric", e0=0.2), W


@pytest.mark.parametrize("name", ["ragged", "wide", "one_spin", "c2"])
def test_split_overlaps_and_e1_at_fp64_quality(name):
    need_gpu()
    s, W = _shape(name)
    phi = perturbed_walkers(s, W, eps=0.3, seed=5)
    ctx, orc = make_pair(s, W, phi=phi, precision="split_bf16")
    e, _ = ctx.local_energy()
    eref, _ = orc.local_energy()
    assert rel(ctx.get_overlaps(), orc.ovlp).max() <= TOL, rel(ctx.get_overlaps(), orc.ovlp).max()
    scale = np.max(np.abs(eref[:, 0]))
    assert np.max(np.abs(e[:, 0] - eref[:, 0])) <= TOL * scale, \
        np.max(np.abs(e[:, 0] - eref[:, 0])) / scale
    assert np.max(np.abs(e[:, 1] - eref[:, 1])) <= TOL_HA
    assert np.max(np.abs(e[:, 2] - eref[:, 2])) <= TOL_HA
    ctx.close()
