"""Block statistics of serially correlated Monte Carlo data (host side, NumPy).

The paper's workflow samples blocks (propagation steps followed by one energy
evaluation), discards the first blocks for equilibration and reblocks the rest to
get the energy and its error bar, citing Flyvbjerg and Petersen, J. Chem. Phys. 91,
461 (1989) (Sec. "Interface with PySCF").  This module is that analysis:

* ``reblock``: the blocking transformation x'_i = (x_{2i} + x_{2i+1}) / 2 applied
  repeatedly (a trailing odd element is dropped); at each level the standard error
  of the mean, sqrt(c0 / (n - 1)) with c0 the biased variance of the n block means,
  and its own uncertainty, that error / sqrt(2 (n - 1)) (Flyvbjerg and Petersen).
* ``optimal_level``: the smallest level whose block length B = 2^level satisfies
  B^3 > 2 n (s_level / s_0)^4, n the number of data points and s the standard error
  (Lee, Needs and Drummond, Phys. Rev. B 83, 125114 (2011)); None if no level does.
* ``estimate``: mean and error bar of a series after discarding equilibration data.
* ``block_energies``: the per-block mixed-energy estimate Re(sum w E_L / sum w) from
  the sums that ``AfqContext.run_blocks`` returns.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class BlockLevel:
    level: int        # number of blocking transformations applied
    block: int        # data points per block, 2^level
    n: int            # block means at this level
    mean: float
    stderr: float     # standard error of the mean from this level's block means
    stderr_err: float


def reblock(x: np.ndarray) -> list[BlockLevel]:
    """Flyvbjerg-Petersen blocking table of a 1-D series (levels while n >= 2)."""
    y = np.asarray(x, dtype=np.float64).ravel()
    out = []
    level = 0
    while y.size >= 2:
        n = y.size
        c0 = float(np.mean((y - y.mean()) ** 2))
        se = float(np.sqrt(c0 / (n - 1)))
        out.append(BlockLevel(level, 2 ** level, n, float(y.mean()), se,
                              se / float(np.sqrt(2.0 * (n - 1)))))
        m = n // 2
        y = 0.5 * (y[0:2 * m:2] + y[1:2 * m:2])
        level += 1
    return out


def optimal_level(table: list[BlockLevel], n: int) -> int | None:
    """Smallest level with B^3 > 2 n (s_B / s_0)^4, or None (series too short)."""
    if not table or table[0].stderr == 0.0:
        return 0 if table else None
    s0 = table[0].stderr
    for t in table:
        if float(t.block) ** 3 > 2.0 * n * (t.stderr / s0) ** 4:
            return t.level
    return None


@dataclass
class Estimate:
    mean: float
    error: float
    level: int | None   # chosen blocking level (None: not converged, last level used)
    n: int              # data points analysed
    table: list[BlockLevel]


def estimate(x: np.ndarray, discard: int = 0) -> Estimate:
    """Mean and error bar of x[discard:] from the blocking table at the optimal level
    (the last level when no level meets the criterion)."""
    y = np.asarray(x, dtype=np.float64).ravel()[discard:]
    if y.size < 2:
        raise ValueError("need at least two data points after the discarded ones")
    table = reblock(y)
    lev = optimal_level(table, y.size)
    row = table[lev] if lev is not None else table[-1]
    return Estimate(float(y.mean()), row.stderr, lev, int(y.size), table)


def block_energies(sums: np.ndarray) -> np.ndarray:
    """Re(sum w E_L / sum w) per block from rows (Re sum w, Im sum w, Re sum w E_L,
    Im sum w E_L)."""
    s = np.asarray(sums, dtype=np.float64)
    den = s[:, 0] + 1j * s[:, 1]
    num = s[:, 2] + 1j * s[:, 3]
    return (num / den).real
