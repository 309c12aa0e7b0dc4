"""Exact results for the periodic 2D Ising model used to pin the oracle.

Independent of the oracle's C code: plain numpy / mpmath.
  * enumerate_g(L): density of states g(E) by enumerating all 2^(L*L) states
    (L <= 4), with the energy evaluated by array rolls.
  * transfer_g(L): g(E) by a row-to-row transfer matrix with energy-indexed
    count vectors (exact integers; L <= 6).
  * kaufman_Z(L, K): B. Kaufman's closed-form partition function of the
    finite L x L periodic lattice (Phys. Rev. 76 (1949) 1232), the formula the
    paper's exact curves (Ferdinand and Fisher 1969, Fig. 1) are built on.
  * exact_thermo(L, beta): E, C, F, S per Sec. 4.1 from Kaufman's Z.
Levels: E = -2N + 4m, m in [0, N].
"""
from __future__ import annotations

import mpmath as mp
import numpy as np


def energies_of_states(L: int) -> np.ndarray:
    N = L * L
    states = np.arange(2 ** N, dtype=np.uint64)
    bits = ((states[:, None] >> np.arange(N, dtype=np.uint64)) & np.uint64(1)).astype(np.int8)
    s = (2 * bits - 1).reshape(-1, L, L)          # s[state, y, x], bit y*L+x
    return -(s * (np.roll(s, -1, axis=2) + np.roll(s, -1, axis=1))).sum(axis=(1, 2))


def enumerate_g(L: int) -> np.ndarray:
    assert L <= 4
    N = L * L
    E = energies_of_states(L)
    return np.bincount((E + 2 * N) // 4, minlength=N + 1).astype(object)


def transfer_g(L: int) -> list[int]:
    """g(E) by transfer matrix over rows: exact Python integers."""
    N = L * L
    R = 1 << L
    rows = np.array([[1 if (r >> x) & 1 else -1 for x in range(L)] for r in range(R)])
    # bonds inside a row (to the right neighbour, periodic) and between rows
    e_in = -(rows * np.roll(rows, -1, axis=1)).sum(axis=1)              # [R]
    e_between = -(rows[:, None, :] * rows[None, :, :]).sum(axis=2)       # [R, R]
    off = 2 * N
    size = 4 * N + 1
    g = [0] * (N + 1)
    for first in range(R):
        # vec[r][E + off]: number of partial configurations with current row r
        vec = np.zeros((R, size), dtype=object)
        vec[first, e_in[first] + off] = 1
        for _ in range(L - 1):
            new = np.zeros((R, size), dtype=object)
            for prev in range(R):
                row = vec[prev]
                nz = np.nonzero(row)[0]
                if nz.size == 0:
                    continue
                for cur in range(R):
                    sh = int(e_between[prev, cur] + e_in[cur])
                    new[cur, nz + sh] += row[nz]
            vec = new
        for last in range(R):
            sh = int(e_between[last, first])       # close the column ring
            nz = np.nonzero(vec[last])[0]
            for idx in nz:
                E = idx - off + sh
                g[(E + 2 * N) // 4] += int(vec[last, idx])
    return g


def kaufman_Z(L: int, K, dps: int = 60):
    """Partition function of the L x L periodic lattice at coupling K = beta J."""
    with mp.workdps(max(dps, mp.mp.dps)):
        K = mp.mpf(K)
        c = mp.cosh(2 * K) * mp.coth(2 * K)

        def gam(k):
            if k == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(mp.pi * k / L))

        Z1 = Z2 = Z3 = Z4 = mp.mpf(1)
        for r in range(L):
            g1, g0 = gam(2 * r + 1), gam(2 * r)
            Z1 *= 2 * mp.cosh(L * g1 / 2)
            Z2 *= 2 * mp.sinh(L * g1 / 2)
            Z3 *= 2 * mp.cosh(L * g0 / 2)
            Z4 *= 2 * mp.sinh(L * g0 / 2)
        return mp.mpf(1) / 2 * (2 * mp.sinh(2 * K)) ** (mp.mpf(L * L) / 2) * (Z1 + Z2 + Z3 + Z4)


def exact_thermo(L: int, beta: float, dps: int = 60):
    """E, C, F, S (Sec. 4.1 definitions) from ln Z by numerical differentiation
    in high precision: E = -d lnZ/d beta, C = beta^2 d^2 lnZ/d beta^2."""
    with mp.workdps(dps):
        b = mp.mpf(beta)
        f = lambda x: mp.log(kaufman_Z(L, x, dps))
        lnZ = f(b)
        E = -mp.diff(f, b)
        C = b ** 2 * mp.diff(f, b, 2)
        F = -lnZ / b
        S = b * (E - F)
        return float(E), float(C), float(F), float(S)


def thermo_from_g(g, L: int, beta: float):
    """The same four quantities summed over a density of states."""
    N = L * L
    with mp.workdps(60):
        b = mp.mpf(beta)
        Es = [mp.mpf(-2 * N + 4 * m) for m in range(N + 1)]
        w = [mp.mpf(int(g[m])) * mp.e ** (-b * Es[m]) for m in range(N + 1)]
        Z = mp.fsum(w)
        E = mp.fsum(w[m] * Es[m] for m in range(N + 1)) / Z
        E2 = mp.fsum(w[m] * Es[m] ** 2 for m in range(N + 1)) / Z
        C = b ** 2 * (E2 - E ** 2)
        F = -mp.log(Z) / b
        S = b * (E - F)
        return float(E), float(C), float(F), float(S)
