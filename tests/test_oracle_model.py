"""Pins for the oracle's Ising model (Sec. 4.1): energy, density of states,
initial configurations, threshold table.

The energy function is pinned by closed forms (ordered, checkerboard and
stripe states) and, through the density of states it produces on every L=2
and L=4 configuration, by Kaufman's exact finite-lattice partition function.
"""
import mpmath as mp
import numpy as np
import pytest

import exact
import oracle


@pytest.mark.parametrize("L", [2, 4, 6, 8, 32, 64])
def test_energy_closed_forms(L):
    N = L * L
    up = np.ones((L, L), np.int8)
    assert oracle.energy(up) == -2 * N
    assert oracle.energy(-up) == -2 * N
    y, x = np.mgrid[0:L, 0:L]
    checker = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy(checker) == 2 * N
    stripes = np.where(x % 2 == 0, 1, -1).astype(np.int8)          # vertical stripes
    assert oracle.energy(stripes) == 0
    one = up.copy()
    one[L // 2, L // 3] = -1
    assert oracle.energy(one) == -2 * N + 8          # dE = 2 s (4 neighbour slots)


@pytest.mark.parametrize("L", [2, 4])
def test_density_of_states_matches_kaufman(L):
    N = L * L
    g = np.zeros(N + 1, dtype=np.int64)
    for state in range(2 ** N):
        bits = (state >> np.arange(N)) & 1
        s = (2 * bits - 1).astype(np.int8).reshape(L, L)
        E = oracle.energy(s)
        assert (E + 2 * N) % 4 == 0
        g[oracle.level(E, L)] += 1
    assert g.sum() == 2 ** N
    assert list(g) == list(g[::-1])                 # E -> -E symmetry (even L)
    for K in (0.05, 0.3, 0.4406868, 0.8, 2.0):
        with mp.workdps(50):
            Zg = mp.fsum(int(g[m]) * mp.exp(-mp.mpf(K) * (-2 * N + 4 * m)) for m in range(N + 1))
            Zk = exact.kaufman_Z(L, K)
            assert abs(Zg / Zk - 1) < mp.mpf(10) ** -40
    if L == 4:
        assert g[1] == 0 and g[N - 1] == 0 and g[0] == 2 and g[2] == 2 * N


def test_transfer_matrix_g_matches_kaufman_L6():
    g = exact.transfer_g(6)
    N = 36
    assert sum(g) == 2 ** N
    for K in (0.2, 0.4406868, 1.1):
        with mp.workdps(50):
            Zg = mp.fsum(g[m] * mp.exp(-mp.mpf(K) * (-2 * N + 4 * m)) for m in range(N + 1))
            assert abs(Zg / exact.kaufman_Z(6, K) - 1) < mp.mpf(10) ** -40


def test_init_all_up():
    s = oracle.init_lattice(8, 123, 5, 0)
    assert (s == 1).all()


@pytest.mark.parametrize("L,chain,seed", [(8, 0, 1), (32, 77, 2), (48, 3, 3), (128, 1023, 99)])
def test_init_random_bits_come_from_philox_tag2(L, chain, seed):
    s = oracle.init_lattice(L, seed, chain, 1)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    N = L * L
    words = {}
    for site in range(N):
        q = site >> 5
        if q not in words:
            words[q] = oracle.philox((q >> 2, 0, chain, 2), key)[q & 3]
        want = 1 if (words[q] >> (site & 31)) & 1 else -1
        assert s[site // L, site % L] == want
    assert abs(s.mean()) < 0.2


def test_table_definition():
    rng = np.random.default_rng(7)
    L = 6
    N = L * L
    W = rng.normal(0, 3, N + 1)
    T = oracle.build_table(W, L)
    for m in range(N + 1):
        for a in range(5):
            mp_ = m + a - 2
            want = 0 if (mp_ < 0 or mp_ > N) else oracle.threshold(W[mp_] - W[m])
            assert T[m, a] == want
    Tz = oracle.build_table(np.zeros(N + 1), L)
    assert (Tz[2:N - 1] == 0xFFFFFFFF).all()
