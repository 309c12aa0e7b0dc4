"""Pins for the oracle's Markov dynamics (Sec. 2 step 2, Sec. 4.2 Metropolis).

* W = 0 makes every flip certain, so the first round is a closed form that a
  direct simulation (flip each site in typewriter order, recompute the energy
  from scratch) reproduces.
* The tracked energy always equals the energy recomputed from the lattice.
* Under the exact multicanonical weight W = -ln g(E) the energy histogram is
  flat, under W = -beta E the mean energy and specific heat equal the exact
  canonical values (g from enumeration / transfer matrix, both pinned to
  Kaufman's closed form).
* L = 2: the exact one-sweep transition matrix built from the oracle's
  thresholds leaves pi ~ 1/g(E) stationary to 2^-32.
* The recursion of Eq. (new_weight) drives W towards -ln g + const.
"""
from fractions import Fraction

import numpy as np
import pytest

import exact
import oracle


def _direct_energy(s):
    return int(-(s * (np.roll(s, -1, axis=1) + np.roll(s, -1, axis=0))).sum())


@pytest.mark.parametrize("L,p,start,S", [(8, 3, 0, 2), (6, 2, 1, 3), (4, 5, 1, 4)])
def test_first_round_at_zero_weight_is_closed_form(L, p, start, S):
    N = L * L
    seed = 1
    job = oracle.Job(L, p, seed, start)
    job.run_round(S)
    samples = job.samples
    M = S * N
    for c in range(p):
        s = oracle.init_lattice(L, seed, c, start).astype(np.int64)
        E0 = _direct_energy(s)
        want = []
        for k in range(M):
            site = k % N
            s[site // L, site % L] *= -1                    # every flip accepted
            want.append((_direct_energy(s) + 2 * N) // 4)
            if site == N - 1:
                assert _direct_energy(s) == E0               # a full sweep flips all spins
        assert list(samples[c]) == want
        assert (job.spins[c] == s).all()
    joined = job.join()
    assert joined == p * M
    assert (job.k == 1).all()
    h = sum(np.bincount(samples[c], minlength=N + 1) for c in range(p))
    assert (job.hist == h).all()


def test_tracked_energy_equals_lattice_energy():
    L, p = 6, 5
    job = oracle.Job(L, p, 9, 1)
    rng = np.random.default_rng(0)
    job.weights = rng.normal(0, 2.0, L * L + 1)
    for _ in range(3):
        job.run_round(40, nthreads=2)
        job.join()
        for c in range(p):
            assert job.levels[c] == oracle.level(oracle.energy(job.spins[c]), L)
        assert (job.trace[-1] == job.levels).all()


def test_streaming_chain_equals_job_chain():
    L, p, seed = 6, 3, 21
    W = np.random.default_rng(1).normal(0, 1.5, L * L + 1)
    job = oracle.Job(L, p, seed, 1)
    job.weights = W
    s0 = job.spins.copy()
    m0 = job.levels.copy()
    job.run_round(30)
    for c in range(p):
        s, m, trace, hist, samples = oracle.chain_round(L, seed, c, 0, 30, W, s0[c], m0[c],
                                                        want_samples=True)
        assert (s == job.spins[c]).all() and m == job.levels[c]
        assert (samples == job.samples[c]).all()
        assert (trace == job.trace[:, c]).all()
        assert (hist == np.bincount(samples, minlength=L * L + 1)).all()


def _exact_ln_g(L):
    g = np.array(exact.enumerate_g(L) if L <= 4 else exact.transfer_g(L), dtype=float)
    W = np.zeros_like(g)
    W[g > 0] = -np.log(g[g > 0])
    return g, W


def test_flat_histogram_under_exact_multicanonical_weight():
    L, p, S = 4, 16, 20000
    g, W = _exact_ln_g(L)
    reach = g > 0
    fr = []
    for c in range(p):
        s0 = oracle.init_lattice(L, 31, c, 1)
        m0 = oracle.level(oracle.energy(s0), L)
        _, _, _, hist, _ = oracle.chain_round(L, 31, c, 0, S, W, s0, m0, want_trace=False)
        assert (hist[~reach] == 0).all()
        fr.append(hist[reach] / hist.sum())
    fr = np.array(fr)
    mean = fr.mean(axis=0)
    err = fr.std(axis=0, ddof=1) / np.sqrt(p)
    target = 1.0 / reach.sum()
    assert (np.abs(mean - target) < 5 * err + 1e-4).all(), (mean, err)
    assert np.abs(mean / target - 1).max() < 0.05


@pytest.mark.parametrize("L,beta,S", [(4, 0.3, 20000), (6, 0.44, 6000)])
def test_canonical_energy_and_specific_heat(L, beta, S):
    N = L * L
    g, _ = _exact_ln_g(L)
    Em = np.array([-2 * N + 4 * m for m in range(N + 1)], dtype=float)
    W = -beta * Em
    p = 16
    E1, E2 = [], []
    for c in range(p):
        s0 = oracle.init_lattice(L, 5, c, 1)
        m0 = oracle.level(oracle.energy(s0), L)
        _, _, _, hist, _ = oracle.chain_round(L, 5, c, 0, S, W, s0, m0, want_trace=False)
        P = hist / hist.sum()
        E1.append((P * Em).sum())
        E2.append((P * Em ** 2).sum())
    E1, E2 = np.array(E1), np.array(E2)
    Ee, Ce, _, _ = exact.thermo_from_g(g, L, beta)
    E_est, E_err = E1.mean(), E1.std(ddof=1) / np.sqrt(p)
    assert abs(E_est - Ee) < 5 * E_err, (E_est, Ee, E_err)
    C_est = beta ** 2 * (E2.mean() - E_est ** 2)
    assert abs(C_est / Ce - 1) < 0.1, (C_est, Ce)


def test_L2_sweep_matrix_leaves_multicanonical_law_stationary():
    L, N = 2, 4
    g, W = _exact_ln_g(L)
    T = oracle.build_table(W, L)
    states = range(16)

    def spins(st):
        return np.array([1 if (st >> q) & 1 else -1 for q in range(N)]).reshape(L, L)

    def level_of(st):
        return (_direct_energy(spins(st)) + 2 * N) // 4

    def site_matrix(q):
        P = [[Fraction(0)] * 16 for _ in states]
        x, y = q % L, q // L
        for st in states:
            s = spins(st)
            nb = s[y, (x + 1) % L] + s[y, (x - 1) % L] + s[(y + 1) % L, x] + s[(y - 1) % L, x]
            dE = 2 * s[y, x] * nb
            m = level_of(st)
            pa = Fraction(int(T[m, dE // 4 + 2]) + 1, 2 ** 32)
            P[st][st ^ (1 << q)] += pa
            P[st][st] += 1 - pa
        return P

    def matmul(A, B):
        return [[sum(A[i][k] * B[k][j] for k in states) for j in states] for i in states]

    P = site_matrix(0)
    for q in range(1, N):
        P = matmul(P, site_matrix(q))
    pi = [Fraction(1, int(g[level_of(st)])) for st in states]
    Z = sum(pi)
    pi = [v / Z for v in pi]
    piP = [sum(pi[i] * P[i][j] for i in states) for j in states]
    assert max(abs(a - b) for a, b in zip(piP, pi)) <= Fraction(8, 2 ** 32) * max(pi)
    marg = {}
    for st in states:
        marg[level_of(st)] = marg.get(level_of(st), 0) + pi[st]
    assert sorted(marg) == [0, 2, 4] and all(v == Fraction(1, 3) for v in marg.values())


def test_weight_recursion_converges_to_minus_ln_g():
    L = 4
    g, _ = _exact_ln_g(L)
    reach = g > 0
    job = oracle.Job(L, 8, 11, 1)
    devs = []
    for it in range(10):
        job.iteration(20000, 0, nthreads=4)
        W = job.weights
        assert (W[~reach] == 0).all()                  # never visited, never updated
        d = W[reach] + np.log(g[reach])
        devs.append(np.abs(d - d.mean()).max())
    assert devs[0] > 1.0                                 # W=0 start is far off
    assert max(devs[-5:]) < 0.06, devs


def test_rounds_of_any_length_compose():
    # Sec. 2 step 2 with rounds that are not whole sweeps (Fig. 2's M_node =
    # 100 < N): the chains' dynamics do not depend on where rounds end, so
    # rounds of 100 attempts concatenate to the same samples, lattices and
    # levels as whole sweeps; the trace records the level where sweeps end
    L, p = 20, 5
    N = L * L
    W = np.random.default_rng(5).normal(0, 3.0, N + 1)
    a = oracle.Job(L, p, 31, 1)
    b = oracle.Job(L, p, 31, 1)
    a.weights = W
    b.weights = W
    a.run_round(2, 2)
    sa, ta = a.samples, a.trace
    parts, traces = [], []
    for _ in range(8):                         # 8 x 100 attempts = 2 sweeps
        b.run_attempts(100, 2)
        parts.append(b.samples)
        traces.append(b.trace)
    assert np.array_equal(np.concatenate(parts, axis=1), sa)
    assert np.array_equal(np.concatenate(traces, axis=0), ta)
    assert [t.shape[0] for t in traces] == [0, 0, 0, 1, 0, 0, 0, 1]
    assert np.array_equal(a.spins, b.spins) and np.array_equal(a.levels, b.levels) and a.t == b.t
