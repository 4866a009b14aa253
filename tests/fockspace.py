"""Brute-force second quantisation on a tiny Fock space, used to pin the oracle.

Nothing here uses Wick's theorem, Slater-Condon rules or determinant formulas:
states are vectors over occupation bitstrings, operators are Jordan-Wigner sparse
matrices, and the Hamiltonian of Eq. Habinitio is assembled term by term from
a+ a+ a a products.  Spin orbital (p, sigma) has index p + sigma * M.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg
import scipy.sparse as sp


class FockSpace:
    def __init__(self, M: int):
        self.M = M
        self.n = 2 * M
        self.dim = 1 << self.n
        self.ann = [self._annihilator(k) for k in range(self.n)]
        self.cre = [a.T.tocsr() for a in self.ann]

    def _annihilator(self, k: int) -> sp.csr_matrix:
        rows, cols, vals = [], [], []
        for s in range(self.dim):
            if s >> k & 1:
                sign = -1.0 if bin(s & ((1 << k) - 1)).count("1") % 2 else 1.0
                rows.append(s ^ (1 << k))
                cols.append(s)
                vals.append(sign)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))

    def so(self, p: int, sigma: int) -> int:
        return p + sigma * self.M

    # -- states -------------------------------------------------------------------
    def vacuum(self) -> np.ndarray:
        v = np.zeros(self.dim, dtype=np.complex128)
        v[0] = 1.0
        return v

    def determinant(self, cols_a: np.ndarray, cols_b: np.ndarray) -> np.ndarray:
        """c+(phi_1) ... c+(phi_N)|0> with the alpha orbitals first."""
        orbs = [(cols_a[:, j], 0) for j in range(cols_a.shape[1])]
        orbs += [(cols_b[:, j], 1) for j in range(cols_b.shape[1])]
        v = self.vacuum()
        for coef, sigma in reversed(orbs):
            op = sum(complex(coef[p]) * self.cre[self.so(p, sigma)] for p in range(self.M))
            v = op @ v
        return v

    def walker_state(self, phi: np.ndarray, na: int) -> np.ndarray:
        return self.determinant(phi[:, :na], phi[:, na:])

    # -- operators ----------------------------------------------------------------
    def one_body(self, K: np.ndarray, spins=(0, 1)) -> sp.csr_matrix:
        """sum_{pq, sigma in spins} K_pq a+_{p sigma} a_{q sigma}."""
        out = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for sigma in spins:
            for p, q in itertools.product(range(self.M), repeat=2):
                if K[p, q] != 0:
                    out = out + K[p, q] * (self.cre[self.so(p, sigma)] @ self.ann[self.so(q, sigma)])
        return out

    def hamiltonian(self, h1: np.ndarray, L: np.ndarray, e0: float) -> sp.csr_matrix:
        """e0 + sum h_pq a+a + 1/2 sum (pr|qs) a+_p a+_q a_s a_r over both spin pairs."""
        M = self.M
        eri = np.einsum("gpr,gqs->prqs", L, L)
        H = e0 * sp.identity(self.dim, format="csr", dtype=np.complex128)
        H = H + self.one_body(h1)
        cc = {}
        aa = {}
        for i, j in itertools.product(range(self.n), repeat=2):
            cc[i, j] = self.cre[i] @ self.cre[j]
            aa[i, j] = self.ann[i] @ self.ann[j]
        for s1, s2 in itertools.product((0, 1), repeat=2):
            for p, q, r, s in itertools.product(range(M), repeat=4):
                v = eri[p, r, q, s]
                if v == 0.0:
                    continue
                H = H + 0.5 * v * (cc[self.so(p, s1), self.so(q, s2)]
                                   @ aa[self.so(s, s2), self.so(r, s1)])
        return H.tocsr()

    def sector(self, na: int, nb: int) -> np.ndarray:
        amask = (1 << self.M) - 1
        idx = [s for s in range(self.dim)
               if bin(s & amask).count("1") == na and bin(s >> self.M).count("1") == nb]
        return np.array(idx)

    def ground_energy(self, H: sp.csr_matrix, na: int, nb: int) -> float:
        idx = self.sector(na, nb)
        Hs = H.toarray()[np.ix_(idx, idx)]
        return float(np.linalg.eigvalsh(0.5 * (Hs + Hs.conj().T))[0])

    @staticmethod
    def expm(op) -> np.ndarray:
        return scipy.linalg.expm(op.toarray() if sp.issparse(op) else op)
