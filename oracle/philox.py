"""Philox4x32-10 and Gaussian auxiliary fields (oracle side; test infrastructure only).

The paper does not name its random number generator.  Fields here come from the
counter-based Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11), implemented from that paper's definition:

* state: four 32-bit counter words c0..c3 and two 32-bit key words k0, k1;
* one round: (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as 64-bit products,
  then c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
* between rounds the key is bumped by the Weyl constants (k0 += W0, k1 += W1);
* ten rounds.

Field layout (the same definition is written independently in the CUDA library):
counter = (step mod 2^32, walker, g // 2, step >> 32), key = (seed mod 2^32,
seed >> 32).  The four output words give two 53-bit uniforms in (0, 1],
u = (k + 1) 2^-53 with k = (w0 >> 5) 2^26 + (w1 >> 6) (and w2, w3 for the second),
and Box-Muller turns (u1, u2) into the fields for g = 2m and 2m + 1:
r = sqrt(-2 ln u1), xi_2m = r cos(2 pi u2), xi_2m+1 = r sin(2 pi u2).
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Apply Philox4x32-10 to an (n, 4) array of uint32 counters; returns (n, 4) uint32."""
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0 = np.uint64(key[0] & 0xFFFFFFFF)
    k1 = np.uint64(key[1] & 0xFFFFFFFF)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def uniforms53(wa: np.ndarray, wb: np.ndarray) -> np.ndarray:
    """Two uint32 words -> one float64 uniform in (0, 1] with 53 random bits."""
    k = (wa.astype(np.uint64) >> np.uint64(5)) * np.uint64(1 << 26) \
        + (wb.astype(np.uint64) >> np.uint64(6))
    return (k + np.uint64(1)).astype(np.float64) * 2.0 ** -53


def field_counters(step: int, W: int, X: int) -> np.ndarray:
    """Counters for every (walker, g-pair) of one step, shape (W * ceil(X/2), 4)."""
    npair = (X + 1) // 2
    z, m = np.meshgrid(np.arange(W, dtype=np.uint64), np.arange(npair, dtype=np.uint64),
                       indexing="ij")
    ctr = np.empty((W * npair, 4), dtype=np.uint64)
    ctr[:, 0] = step & 0xFFFFFFFF
    ctr[:, 1] = z.ravel()
    ctr[:, 2] = m.ravel()
    ctr[:, 3] = (step >> 32) & 0xFFFFFFFF
    return ctr


def field_words(step: int, W: int, X: int, seed: int) -> np.ndarray:
    """Raw Philox words of one step, shape (W, ceil(X/2), 4) uint32."""
    out = philox4x32_10(field_counters(step, W, X), (seed & 0xFFFFFFFF, seed >> 32))
    return out.reshape(W, (X + 1) // 2, 4)


def field_uniforms(step: int, W: int, X: int, seed: int) -> np.ndarray:
    """The two uniforms per (walker, g-pair), shape (W, ceil(X/2), 2)."""
    w = field_words(step, W, X, seed)
    u1 = uniforms53(w[..., 0], w[..., 1])
    u2 = uniforms53(w[..., 2], w[..., 3])
    return np.stack([u1, u2], axis=-1)


def gaussian_fields(step: int, W: int, X: int, seed: int) -> np.ndarray:
    """N(0,1) auxiliary fields xi of one step, shape (W, X), by Box-Muller."""
    u = field_uniforms(step, W, X, seed)
    r = np.sqrt(-2.0 * np.log(u[..., 0]))
    ang = 2.0 * np.pi * u[..., 1]
    g = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=-1).reshape(W, -1)
    return np.ascontiguousarray(g[:, :X])
