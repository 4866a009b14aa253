"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmarks.

This module holds no arithmetic of the AFQMC method itself: it only draws random
Hamiltonian pieces, trial orbitals and walker matrices with the shapes and value
distributions described below, so that the CUDA library and the CPU oracle can be
fed identical inputs.  It imports numpy only.

Recipe (the paper's molecules need integral files that are not available, so
these stand in for them, with the sizes of the paper's largest single-determinant
space, 52 electrons in 290 orbitals with 640 walkers and dt = 0.005):

* h1: symmetric; off-diagonal entries N(0,1) symmetrised and scaled by 0.1, the
  diagonal set to sorted N(0,1) draws times sqrt(M), so the diagonal dominates.
* L_g (g = 0..X-1): symmetric Gaussian matrices, each normalised to unit Frobenius
  norm, then scaled either by 0.5**(g/4) ("half" decay) or geometrically by r**g
  with r chosen so that ||L_{X-1}|| / ||L_0|| = 1e-4 ("geometric" decay).
* trial: for each spin the Q factor of a seeded Gaussian M x N_sigma matrix.
* walkers: copies of the trial (complex128), or the trial plus a seeded complex
  perturbation when a test wants walkers that differ from it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SyntheticSystem:
    """One seeded system: Hamiltonian pieces and a trial determinant."""

    M: int
    na: int
    nb: int
    X: int
    h1: np.ndarray  # (M, M) float64, symmetric
    L: np.ndarray  # (X, M, M) float64, each symmetric
    e0: float
    psi_a: np.ndarray  # (M, na) float64, orthonormal columns
    psi_b: np.ndarray  # (M, nb) float64, orthonormal columns

    @property
    def N(self) -> int:
        return self.na + self.nb


# The five workloads: orbital count, electrons per spin, Cholesky count, walkers,
# steps, norm decay of the Cholesky vectors.
CONFIGS = {
    "c1": dict(M=8, na=2, nb=2, X=24, W=10, steps=10, decay="half"),
    "c2": dict(M=100, na=10, nb=10, X=400, W=128, steps=200, decay="geometric"),
    "c3": dict(M=290, na=26, nb=26, X=1500, W=640, steps=100, decay="geometric"),
    "c5": dict(M=150, na=15, nb=15, X=750, W=256, steps=20, decay="geometric"),
}
# Batched uneven systems: orbitals, electrons per spin = round(0.2 M), X = 5 M.
C4_ORBITALS = (48, 64, 80, 100, 120, 150, 180, 220)
C4_WALKERS = (512, 256, 256, 128, 128, 64, 64, 32)


def make_system(M: int, na: int, nb: int, X: int, seed: int = 1,
                decay: str = "geometric", e0: float = 0.0) -> SyntheticSystem:
    """Draw a seeded Hamiltonian (h1, L) and trial following the module recipe."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((M, M))
    h1 = 0.1 * 0.5 * (a + a.T)
    h1[np.diag_indices(M)] = np.sort(rng.standard_normal(M)) * np.sqrt(M)
    if decay == "half":
        scale = 0.5 ** (np.arange(X) / 4.0)
    elif decay == "geometric":
        r = (1e-4) ** (1.0 / max(X - 1, 1))
        scale = r ** np.arange(X)
    else:
        raise ValueError(f"unknown decay {decay!r}")
    L = np.empty((X, M, M))
    for g in range(X):
        b = rng.standard_normal((M, M))
        b = 0.5 * (b + b.T)
        L[g] = b * (scale[g] / np.linalg.norm(b))
    psi_a = np.linalg.qr(rng.standard_normal((M, na)))[0]
    psi_b = np.linalg.qr(rng.standard_normal((M, nb)))[0]
    return SyntheticSystem(M, na, nb, X, h1, L, float(e0), psi_a, psi_b)


def make_config(name: str, seed: int = 1) -> tuple[SyntheticSystem, dict]:
    """System and run parameters of one of the named workloads (c1, c2, c3, c5)."""
    c = dict(CONFIGS[name])
    sysm = make_system(c["M"], c["na"], c["nb"], c["X"], seed=seed, decay=c["decay"])
    return sysm, c


def make_c4(seed0: int = 1) -> list[tuple[SyntheticSystem, int]]:
    """The eight uneven systems of the batched workload with their walker counts."""
    out = []
    for k, (M, W) in enumerate(zip(C4_ORBITALS, C4_WALKERS)):
        n = int(round(0.2 * M))
        out.append((make_system(M, n, n, 5 * M, seed=seed0 + k), W))
    return out


def trial_walkers(sysm: SyntheticSystem, W: int) -> np.ndarray:
    """W copies of the trial determinant, shape (W, M, na+nb), complex128."""
    phi = np.concatenate([sysm.psi_a, sysm.psi_b], axis=1).astype(np.complex128)
    return np.repeat(phi[None], W, axis=0).copy()


def perturbed_walkers(sysm: SyntheticSystem, W: int, eps: float = 0.3,
                      seed: int = 7) -> np.ndarray:
    """Trial walkers plus a seeded complex Gaussian perturbation of size eps."""
    rng = np.random.default_rng(seed)
    phi = trial_walkers(sysm, W)
    noise = rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape)
    return phi + eps * noise / np.sqrt(sysm.M)


def gaussian_fields(W: int, X: int, seed: int = 11) -> np.ndarray:
    """Seeded N(0,1) auxiliary fields, shape (W, X), for runs that pass fields in."""
    return np.random.default_rng(seed).standard_normal((W, X))
