"""Numerical vacuum eigenstates for the oracle (test infrastructure only).

(For the isotropic KSU potential, V below is the vacuum Cornell potential with string breaking
instead of the Coulomb term, and each state is signed positive at its first significant point.)

The discretised singlet vacuum Hamiltonian of angular momentum l on the trajectory grid (Sec. 2.5,
the computed eigenstates of initType 100 / ProjType 1), written out as a dense matrix on the interior
points r_j = j dr, j = 1 .. N-1:

    H = diag(V) + S diag(K) S (2/N),   S_jk = sin(pi j k / N),
    V_j = -C_F alpha_s / r_j + l(l+1) / (M r_j^2),
    K_k = (pi k / L)^2 / M            (derivType 1: 2 [1 - cos(pi k dr / L)] / (M dr^2)),

i.e. the potential and the kinetic factor of the split-step propagator (S (2/N) is the inverse of
the sine transform S).  numpy's symmetric eigensolver diagonalises it; the eigenvectors are
normalised with the discrete norm dr sum u^2 = 1 and signed to overlap positively with the analytic
Coulomb state of the same (n, l).
"""
from __future__ import annotations

import numpy as np

from . import core

BASIS_NL = ((1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2))


KSU_A, KSU_SIGMA, KSU_RSB = 0.409, 0.21, 1.25 / 0.1973269804   # App. E: a, sigma (GeV^2), r_SB (GeV^-1)


def vacuum_potential(g: core.Grid, r: np.ndarray) -> np.ndarray:
    """The singlet vacuum potential: -C_F alpha_s / r (the OQS+pNRQCD potential), or for the KSU
    potential the Cornell potential -a/r + sigma r, constant beyond the string-breaking distance
    r_SB (App. E, Eq. vvac)."""
    if g.potential == 1:
        return np.where(r <= KSU_RSB, -KSU_A / r + KSU_SIGMA * r, -KSU_A / KSU_RSB + KSU_SIGMA * KSU_RSB)
    CF = (g.Nc * g.Nc - 1.0) / (2.0 * g.Nc)
    return -CF * g.alpha_s / r


def hamiltonian(g: core.Grid, l: int) -> np.ndarray:
    N, L = g.N, g.L
    dr = L / N
    j = np.arange(1, N)
    r = j * dr
    V = vacuum_potential(g, r) + l * (l + 1) / (g.M * r * r)
    p = np.pi * j / L
    K = p * p / g.M if g.deriv_type == 0 else 2.0 * (1.0 - np.cos(p * dr)) / (g.M * dr * dr)
    S = np.sin(np.pi * np.outer(j, j) / N)
    return np.diag(V) + (S * K) @ S * (2.0 / N)


def vacuum_eigenstates(g: core.Grid, l: int, m: int):
    """(eigenvalues, states (m, N)) of the m lowest eigenstates of angular momentum l, n = l+1 .. l+m."""
    w, v = np.linalg.eigh(hamiltonian(g, l))
    dr = g.L / g.N
    out = np.zeros((m, g.N))
    for k in range(m):
        u = np.zeros(g.N)
        u[1:] = v[:, k] / np.sqrt(dr)
        if g.potential == 1:
            # sign: the first point where |u| exceeds 1e-3 of its maximum is positive
            first = np.nonzero(np.abs(u) > 1e-3 * np.abs(u).max())[0][0]
            if u[first] < 0:
                u = -u
        else:
            ref = core.eigenstate(g, l + 1 + k, l)
            if np.dot(u, ref) < 0:
                u = -u
        out[k] = u
    return w[:m], out


def numerical_basis(g: core.Grid) -> np.ndarray:
    """The six basis states 1S 2S 1P 3S 2P 1D as numerical eigenstates, (6, N)."""
    b = np.zeros((len(BASIS_NL), g.N))
    for l, m in ((0, 3), (1, 2), (2, 1)):
        _, v = vacuum_eigenstates(g, l, m)
        for k in range(m):
            b[BASIS_NL.index((l + 1 + k, l))] = v[k]
    return b
