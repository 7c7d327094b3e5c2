"""Brute-force second quantisation on tiny systems (a pin for the oracle).

Independent of the oracle: it builds the Hamiltonian of Eq. (1) literally from
creation and annihilation operators in the Jordan-Wigner representation of the
fixed-particle-number sectors, with V_ijkl = sum_g L_g,ij L_g,kl, and
expands Slater determinants into determinant coefficients (minors).  It uses no
Green's function, no Wick theorem and no Monte Carlo form.

Mode q = s*N + i (s = 0 spin up, 1 spin down).  Basis state of an occupied set
q1 < q2 < ... is c+_q1 c+_q2 ... |0>; so c_q carries the sign (-1)^(number of
occupied modes below q), and the coefficient of (up set I, down set J) in the
determinant with orbitals (phi_up, phi_dn) is det(phi_up[I]) det(phi_dn[J]).
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def sector_states(N: int, n_up: int, n_dn: int) -> np.ndarray:
    ups = [sum(1 << i for i in c) for c in itertools.combinations(range(N), n_up)]
    dns = [sum(1 << (N + i) for i in c) for c in itertools.combinations(range(N), n_dn)]
    return np.array(sorted(u | d for u in ups for d in dns), dtype=np.int64)


def _popcount_below(s: np.ndarray, q: int) -> np.ndarray:
    m = s & ((1 << q) - 1)
    c = np.zeros_like(m)
    while np.any(m):
        c += m & 1
        m >>= 1
    return c


def annihilator(q: int, src: np.ndarray, dst: np.ndarray) -> sp.csr_matrix:
    """Matrix of c_q from the span of ``src`` states to the span of ``dst``."""
    occ = (src >> q) & 1 == 1
    cols = np.nonzero(occ)[0]
    new = src[cols] ^ (1 << q)
    rows = np.searchsorted(dst, new)
    assert np.all(dst[rows] == new)
    sign = np.where(_popcount_below(src[cols], q) % 2 == 0, 1.0, -1.0)
    return sp.csr_matrix((sign, (rows, cols)), shape=(dst.size, src.size))


class FockSpace:
    def __init__(self, N: int, n_up: int, n_dn: int):
        self.N, self.n_up, self.n_dn = N, n_up, n_dn
        self.states = sector_states(N, n_up, n_dn)
        self._sectors = {}
        self._ann = {}

    def sector(self, nu, nd):
        key = (nu, nd)
        if key not in self._sectors:
            self._sectors[key] = sector_states(self.N, nu, nd)
        return self._sectors[key]

    def c(self, i: int, s: int, nu: int, nd: int) -> sp.csr_matrix:
        """c_{i,s} acting on sector (nu, nd)."""
        key = (i, s, nu, nd)
        if key not in self._ann:
            src = self.sector(nu, nd)
            dst = self.sector(nu - (s == 0), nd - (s == 1))
            self._ann[key] = annihilator(s * self.N + i, src, dst)
        return self._ann[key]

    def _pattern(self, nu: int, nd: int):
        """(rows, cols, sign, k, l) of every nonzero of every c+_{k s} c_{l s}."""
        key = ("pattern", nu, nd)
        if key not in self._ann:
            src = self.sector(nu, nd)
            parts = []
            for s, ns in ((0, nu), (1, nd)):
                if ns == 0:
                    continue
                for k in range(self.N):
                    for l in range(self.N):
                        E = (self.c(k, s, nu, nd).T @ self.c(l, s, nu, nd)).tocoo()
                        parts.append((E.row, E.col, E.data, np.full(E.nnz, k), np.full(E.nnz, l)))
            self._ann[key] = tuple(np.concatenate(a) for a in zip(*parts)) + (src.size,)
        return self._ann[key]

    def one_body(self, M: np.ndarray, nu: int, nd: int) -> sp.csr_matrix:
        """sum_s sum_kl M_kl c+_{k s} c_{l s} on sector (nu, nd)."""
        rows, cols, sign, k, l, dim = self._pattern(nu, nd)
        return sp.csr_matrix((sign * M[k, l], (rows, cols)), shape=(dim, dim))

    def hamiltonian(self, h: np.ndarray, L: np.ndarray) -> sp.csr_matrix:
        """H = sum_ij h_ij c+_i c_j + 1/2 sum_ijkl V_ijkl c+_i c+_k c_l c_j
        (both spin sums), V_ijkl = sum_g L_g,ij L_g,kl, built literally as
        1/2 sum_g sum_s sum_ij L_g,ij c+_is (sum_kl,t L_g,kl c+_kt c_lt) c_js."""
        nu, nd = self.n_up, self.n_dn
        H = self.one_body(h, nu, nd)
        for g in range(L.shape[0]):
            for s, (mu, md) in ((0, (nu - 1, nd)), (1, (nu, nd - 1))):
                if (s == 0 and nu == 0) or (s == 1 and nd == 0):
                    continue
                A = self.one_body(L[g], mu, md)
                for i in range(self.N):
                    ci = self.c(i, s, nu, nd)
                    B = sum(L[g, i, j] * self.c(j, s, nu, nd) for j in range(self.N))
                    H = H + 0.5 * (ci.T @ (A @ B))
        return H.tocsr()

    def determinant(self, phi_up: np.ndarray, phi_dn: np.ndarray) -> np.ndarray:
        """Coefficients of the Slater determinant in the sector basis (minors)."""
        N = self.N
        out = np.empty(self.states.size, dtype=np.result_type(phi_up, phi_dn, np.float64))
        for idx, s in enumerate(self.states):
            I = [i for i in range(N) if (s >> i) & 1]
            J = [j for j in range(N) if (s >> (N + j)) & 1]
            du = np.linalg.det(phi_up[I, :]) if I else 1.0
            dd = np.linalg.det(phi_dn[J, :]) if J else 1.0
            out[idx] = du * dd
        return out
