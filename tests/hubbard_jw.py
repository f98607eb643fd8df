"""Brute-force Jordan-Wigner construction of the 1D Hubbard chain (Eq. HUBB).

Test fixture, independent of both the oracle and the CUDA library.  Modes
are ordered 1up, 1dn, 2up, 2dn, ...; the annihilator of mode p acts as
c_p |n> = (-1)^(sum_{p'<p} n_p') n_p |n - e_p>.  A Fock state of L sites has
index sum_site s_site * 4^(L-1-site) with the local digit s = n_up + 2 n_dn,
i.e. local states (0, up, down, up-down) and the first site slowest.  With
this numbering the first L-1 sites form the block B and the last site the
added site a, and the [B a] index is (block index) * 4 + s, the convention
r = i*d + s of the library.
"""
from __future__ import annotations

import itertools

import numpy as np


def _occupations(L: int):
    """All occupation tuples (n_1up, n_1dn, ..., n_Lup, n_Ldn) with their index."""
    for digits in itertools.product(range(4), repeat=L):
        occ = []
        for s in digits:
            occ += [s & 1, (s >> 1) & 1]
        idx = 0
        for s in digits:
            idx = idx * 4 + s
        yield tuple(occ), idx


def annihilators(L: int):
    """Dense c_p for p = 2*site + spin (spin 0 = up, 1 = down), dim 4^L."""
    dim = 4 ** L
    ops = [np.zeros((dim, dim)) for _ in range(2 * L)]
    for occ, idx in _occupations(L):
        for p in range(2 * L):
            if occ[p] == 0:
                continue
            new = list(occ)
            new[p] = 0
            sign = -1.0 if sum(occ[:p]) % 2 else 1.0
            jdx = 0
            for site in range(L):
                jdx = jdx * 4 + new[2 * site] + 2 * new[2 * site + 1]
            ops[p][jdx, idx] = sign
    return ops


def hubbard_hamiltonian(L: int, t: float, U: float, c=None) -> np.ndarray:
    """H = -t sum_{i,s} (c+_{i+1 s} c_{i s} + h.c.) + (U/2) sum_{i,s} n_{i s} n_{i sbar}
    with open boundaries (Eq. HUBB)."""
    c = annihilators(L) if c is None else c
    dim = 4 ** L
    H = np.zeros((dim, dim))
    for i in range(L - 1):
        for s in range(2):
            a, b = c[2 * (i + 1) + s], c[2 * i + s]
            H += -t * (a.T @ b + b.T @ a)
    for i in range(L):
        n_up = c[2 * i].T @ c[2 * i]
        n_dn = c[2 * i + 1].T @ c[2 * i + 1]
        H += 0.5 * U * (n_up @ n_dn + n_dn @ n_up)
    return H


def number_ops(L: int, c=None):
    """(N_up, N_dn) total number operators (diagonal)."""
    c = annihilators(L) if c is None else c
    Nu = sum(c[2 * i].T @ c[2 * i] for i in range(L))
    Nd = sum(c[2 * i + 1].T @ c[2 * i + 1] for i in range(L))
    return Nu, Nd


def sector_basis(L: int):
    """For every Fock index, its (N_up, N_dn)."""
    out = np.zeros((4 ** L, 2), dtype=np.int64)
    for occ, idx in _occupations(L):
        out[idx] = (sum(occ[0::2]), sum(occ[1::2]))
    return out
