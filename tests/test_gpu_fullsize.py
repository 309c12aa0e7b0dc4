"""Full-size runs (every chain, the benchmark's launch configuration) checked
on sampled chains that the oracle replays one by one, plus the properties
that hold at any size.

For a sampled chain c the oracle starts from the GPU's round-start lattice
and level, the same attempt counter and the same weights, and reproduces
its whole round (Sec. 2 step 2): final lattice, final level and the energy
after every sweep must be identical.  Its first kept sample k_c (Sec. 2
step 4) is recomputed for the input level the GPU's own results imply (the
last level of the nearest earlier chain that kept samples, else the carry
of the previous round).  Over all chains: sum h = joined length =
sum(M - k + 1), offsets = exclusive scan, unreachable levels empty, and the
weight update (Eq. new_weight in logs) and threshold table equal the
oracle's for the GPU's histogram, bit for bit.

The oracle replays run in host threads (the C calls release the GIL).
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import BATCH_GROUPS, WORKLOADS, canonical_weights, random_weights

pytestmark = pytest.mark.gpu

BETA_C = 0.4406867935097715  # ln(1 + sqrt 2) / 2: weights of the critical Boltzmann law


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()
    oracle.build()


def _sample_chains(p, n, seed):
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(2, p - 2), size=max(0, n - 4), replace=False)
    return sorted(set([0, 1, p - 2, p - 1] + [int(c) for c in mid]))


class _RoundStart:
    """What the oracle needs to replay chains of the next round."""

    def __init__(self, g):
        info = g.info()
        self.L, self.N, self.p = g.L, g.L * g.L, g.p
        self.t0 = info["attempts_per_chain"]
        self.r = info["rounds_joined"]
        self.carry = oracle.level(info["carry_energy"], g.L) if info["carry_valid"] else -1
        self.spins = oracle.unpack_spins(g.spin_words, g.L)
        self.levels = (g.energies.astype(np.int64) + 2 * self.N) // 4
        self.W = g.weights
        self.hist = g.hist   # earlier rounds of the same weight iteration


def _check_round(g, rs, S, seed, chains, with_trace=True):
    """After g ran and joined one round from round start rs."""
    L, N, p = rs.L, rs.N, rs.p
    M = S * N
    k = g.k
    off = g.offsets
    h = g.hist
    lv = (g.energies.astype(np.int64) + 2 * N) // 4
    words = g.spin_words.reshape(p, -1)
    info = g.info()
    joined = info["last_joined"]
    # properties over every chain
    assert ((k >= 0) & (k <= M)).all()
    kept = np.where(k > 0, M - k + 1, 0)
    assert joined == kept.sum() == (h - rs.hist).sum()
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(kept)[:-1]]))
    assert (h >= 0).all() and h[1] == 0 and h[N - 1] == 0
    assert ((lv >= 0) & (lv <= N)).all()
    if rs.carry < 0:
        assert k[0] == 1
    # input level of each sampled chain, from the GPU's own results
    last_acc = np.where(k > 0, np.arange(p), -1)
    last_acc = np.maximum.accumulate(np.concatenate([[-1], last_acc[:-1]]))

    def replay(c):
        s1, m1, tr, _, _ = oracle.chain_round(L, g.seed, c, rs.t0, S, rs.W, rs.spins[c], int(rs.levels[c]),
                                              want_trace=with_trace)
        i = last_acc[c]
        x = int(lv[i]) if i >= 0 else rs.carry
        kc = 1 if x < 0 else oracle.chain_first_accept(L, g.seed, c, rs.t0, S, rs.W, rs.spins[c],
                                                       int(rs.levels[c]), x, rs.r)
        return c, oracle.pack_spins(s1[None]).reshape(-1), m1, tr, kc

    workers = min(len(chains), os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        for c, w1, m1, tr, kc in ex.map(replay, chains):
            assert np.array_equal(words[c], w1), f"lattice of chain {c}"
            assert lv[c] == m1, f"level of chain {c}"
            if with_trace:
                assert np.array_equal(g.trace_chain(c), 4 * tr - 2 * N), f"trace of chain {c}"
            assert k[c] == kc, f"first kept sample of chain {c}"
    # weight update and thresholds against the oracle's, for the GPU's histogram
    W0 = g.weights
    g.update_weights()
    W1 = W0.copy()
    for m in np.nonzero(h)[0]:
        W1[m] = W0[m] - oracle.log_det(float(h[m]))
    assert np.array_equal(g.weights, W1)
    assert np.array_equal(g.table, oracle.build_table(W1, L))


def _full_single(name, S, n_sample, weights):
    w = WORKLOADS[name]
    S = S or w.sweeps
    g = mc.Job(w.L, w.chains, w.seed, w.start)
    g.set_trace(True)
    g.weights = weights(w.L)
    # a short round first, so that the checked round starts from a carry
    g.run_sweeps(2)
    g.join()
    rs = _RoundStart(g)
    g.run_sweeps(S)
    g.join()
    _check_round(g, rs, S, w.seed, _sample_chains(w.chains, n_sample, w.seed))


def test_L32_p16384_full_round_sampled():
    # every chain, 1e5 sweeps, default launch shape (the benchmark's)
    _full_single("L32_p16384", 0, 32, lambda L: canonical_weights(L, BETA_C))


def test_L64_p4096_full_round_sampled():
    _full_single("L64_p4096", 0, 8, lambda L: canonical_weights(L, BETA_C))


def test_L128_p1024_every_chain_sampled():
    # every chain; 2e3 of the workload's 2e5 sweeps so that each sampled
    # replay stays within seconds on the host
    _full_single("L128_p1024", 2000, 8, lambda L: random_weights(L, 3, 3.0))


def test_batch_uneven_fused_graph_sampled():
    # all five groups at full chain counts in the fused, graph-captured
    # launch; 5e3 of the 5e4 sweeps per iteration
    S = 5000
    jobs = []
    for L, p, seed in BATCH_GROUPS:
        g = mc.Job(L, p, seed, 1)
        g.weights = random_weights(L, seed, 2.0)
        jobs.append(g)
    mc.mc_batch_run([g.h for g in jobs], 1, 2, 2)   # one short iteration; weights updated
    starts = [_RoundStart(g) for g in jobs]
    mc.mc_batch_run([g.h for g in jobs], 1, S, 2)
    # mc_batch_run updated the weights; check the round against the
    # round-start weights, then the update separately
    for g, rs, (L, p, seed) in zip(jobs, starts, BATCH_GROUPS):
        N = L * L
        M = S * N
        k = g.k
        kept = np.where(k > 0, M - k + 1, 0)
        assert g.info()["last_joined"] == kept.sum()
        lv = (g.energies.astype(np.int64) + 2 * N) // 4
        words = g.spin_words.reshape(p, -1)
        chains = _sample_chains(p, 4, seed)
        last_acc = np.where(k > 0, np.arange(p), -1)
        last_acc = np.maximum.accumulate(np.concatenate([[-1], last_acc[:-1]]))

        def replay(c, g=g, rs=rs, L=L):
            s1, m1, _, _, _ = oracle.chain_round(L, g.seed, c, rs.t0, S, rs.W, rs.spins[c], int(rs.levels[c]),
                                                 want_trace=False)
            i = last_acc[c]
            x = int(lv[i]) if i >= 0 else rs.carry
            kc = oracle.chain_first_accept(L, g.seed, c, rs.t0, S, rs.W, rs.spins[c], int(rs.levels[c]), x, rs.r)
            return c, oracle.pack_spins(s1[None]).reshape(-1), m1, kc

        with ThreadPoolExecutor(min(len(chains), os.cpu_count() or 1)) as ex:
            for c, w1, m1, kc in ex.map(replay, chains):
                assert np.array_equal(words[c], w1)
                assert lv[c] == m1
                assert k[c] == kc


@pytest.mark.parametrize("name,S,iters", [("L32_p16384", 10, 3), ("L64_p4096", 2, 3), ("L128_p1024", 1, 2)])
def test_all_chains_bit_exact_at_full_chain_count(name, S, iters):
    # every chain of the workload (its L, p, seed and start) against the
    # oracle, with the sweeps per round cut so that the oracle keeps every
    # sample of the round in memory: spins, energies, traces, k, histograms,
    # weights.  The energies also equal a from-scratch recomputation from the
    # GPU's own lattices (the trace's last entry is the chain's energy).
    w = WORKLOADS[name]
    L, p, N = w.L, w.chains, w.N
    g = mc.Job(L, p, w.seed, w.start)
    g.set_trace(True)
    o = oracle.Job(L, p, w.seed, w.start)
    threads = os.cpu_count() or 1
    for _ in range(iters):
        g.run_sweeps(S)
        o.run_round(S, threads)
        assert np.array_equal(g.spin_words, oracle.pack_spins(o.spins))
        E = g.energies
        assert np.array_equal(E, 4 * o.levels - 2 * N)
        tr = g.trace
        assert np.array_equal(tr, 4 * o.trace - 2 * N)
        assert np.array_equal(tr[-1], E)
        spins = oracle.unpack_spins(g.spin_words, L)
        for c in (0, p // 2, p - 1):
            assert oracle.energy(spins[c]) == E[c]
        assert g.join() == o.join()
        assert np.array_equal(g.k, o.k)
        assert np.array_equal(g.hist, o.hist)
        g.update_weights()
        o.update_weights()
        assert np.array_equal(g.weights, o.weights)
