"""Population control and the block workflow, plain NumPy (test infrastructure).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and bench.py's CPU legs may
use this module; the library never imports it.

The paper counts population control among the computationally light parts of
AFQMC (Sec. "Introduction") without fixing an algorithm, and runs production
calculations as blocks: a number of propagation steps (typically 25) followed by
one energy evaluation, with the block energies reblocked afterwards (the example
workflow in Sec. "Interface with PySCF").  Readings taken here:

* Population control is the comb (systematic resampling): with the phaseless
  weights w_z >= 0, their running sums C_z = w_0 + ... + w_z (left to right) and
  T = C_{W-1}, one offset u in [0, 1) drawn by the caller places W teeth at
  t_k = (k + u) (T / W), k = 0..W-1.  New walker k copies the walker z with
  C_{z-1} <= t_k < C_z (walker matrix and stored overlap), and every new walker
  has weight T / W.  A tooth that rounding puts at or above C_{W-1} goes to the
  last walker with positive weight.
* Weight cap: before the comb each weight is replaced by min(w_z, w_cap) when
  w_cap > 0 (off by default, as the paper states none).
* Block energy: the block's sums (sum_z w_z, sum_z w_z E_L,z) after its last step;
  the block estimate is Re(sum w E_L / sum w).
* Energy-shift feedback (optional): after each block the shift E_shift of the weight
  factor exp(-dt (e0 - 1/2 sum vbar^2 - E_shift)) becomes E_b - ln(T_b / W) / (dt n),
  E_b the block's estimate, T_b its total weight and n its steps (the population
  control of diffusion Monte Carlo), so the total weight stays near W over long runs;
  every weight of a step gets the same factor, so ratio estimators do not change.
"""
from __future__ import annotations

import numpy as np


def comb_parents(w: np.ndarray, u: float, w_cap: float = 0.0) -> tuple[np.ndarray, float]:
    """Parent index of every new walker and the total weight T, by the comb above."""
    w = np.array(w, dtype=np.float64)
    if w_cap > 0.0:
        w = np.minimum(w, w_cap)
    W = w.shape[0]
    C = np.empty(W)
    s = 0.0
    for z in range(W):  # running sums in index order
        s = s + w[z]
        C[z] = s
    T = C[W - 1]
    if not (T > 0.0 and np.isfinite(T)):
        raise ValueError("total weight is not positive and finite")
    spacing = T / W
    last = max(z for z in range(W) if w[z] > 0.0)
    parents = np.empty(W, dtype=np.int64)
    for k in range(W):
        t = (k + u) * spacing
        z = 0
        while z < W and C[z] <= t:  # first walker whose running sum passes the tooth
            z += 1
        parents[k] = min(z, last)
    return parents, float(T)


def population_control(orc, u: float, w_cap: float = 0.0) -> np.ndarray:
    """Applies the comb to an Oracle's walkers in place; returns the parents."""
    if orc.free_projection:
        raise ValueError("the comb needs the phaseless (real, non-negative) weights")
    parents, T = comb_parents(orc.w, u, w_cap)
    W = orc.phi.shape[0]
    orc.phi = orc.phi[parents].copy()
    orc.ovlp = orc.ovlp[parents].copy()
    orc.w = np.full(W, T / W)
    return parents


def block_sums(orc) -> np.ndarray:
    """(sum_z w_z, sum_z w_z E_L,z) of the current walkers, as [Re, Im, Re, Im]."""
    e = orc.local_energy_of(orc.phi)[:, 3]
    w = np.asarray(orc.w, dtype=np.complex128)
    den = np.sum(w)
    num = np.sum(w * e)
    return np.array([den.real, den.imag, num.real, num.imag])


def run_blocks(orc, fields_of_step, nblocks: int, steps_per_block: int,
               u: np.ndarray | None = None, w_cap: float = 0.0,
               shift_feedback: bool = False) -> np.ndarray:
    """The block workflow: per block, steps_per_block steps (QR at the Oracle's
    cadence) with the fields fields_of_step(global step index), then the block sums,
    then (shift_feedback) E_shift <- the block's Re(sum w E_L / sum w), then the comb
    with offset u[b] when u is given.  Returns (nblocks, 4)."""
    out = np.empty((nblocks, 4))
    for b in range(nblocks):
        n0 = orc.nstep
        orc.propagate([fields_of_step(n0 + k) for k in range(steps_per_block)])
        out[b] = block_sums(orc)
        if shift_feedback:
            W = orc.phi.shape[0]
            if orc.free_projection:
                den = out[b, 0] + 1j * out[b, 1]
                eb = ((out[b, 2] + 1j * out[b, 3]) / den).real
                tb = abs(den)
            else:
                eb = out[b, 2] / out[b, 0]
                tb = out[b, 0]
            e = eb - np.log(tb / W) / (orc.dt * steps_per_block)
            if np.isfinite(e):
                orc.e_shift = float(e)
        if u is not None:
            population_control(orc, float(u[b]), w_cap)
    return out
