"""Pins for the oracle's joint (Sec. 2, steps 3-6) and weight update
(Sec. 3.1, Eq. new_weight; Sec. 4.2, logarithms).

Hand-made energy sequences with weights chosen so that every Metropolis test
is certain (d >= 0) or fails unless its uniform is exactly 0 (d <= -23; the
test checks that no such uniform is drawn) give expected keep-indices, carries
and histograms that follow from the algorithm's text by hand.  The uniforms
themselves come from the Philox counters the oracle documents, evaluated with
the Philox that cuRAND pins.
"""
import numpy as np
import pytest

import exact
import oracle

SEED = 77


def _ju(r, i, k, seed=SEED):
    """joint uniform of sample k (1-based) of chain i in round r"""
    q = k - 1
    return oracle.philox((q >> 2, r, i, 1), (seed & 0xFFFFFFFF, seed >> 32))[q & 3]


def test_joint_scan_certain_and_impossible():
    N = 16
    W = np.zeros(N + 1)
    lv = np.array([3, 4, 5, 6, 7, 8, 9, 10] * 2, np.int32)
    assert oracle.joint_scan(lv, W, 5, SEED, 0, 0) == 1          # flat weight: first sample kept
    W[:] = -40.0
    W[9] = 0.0                                                    # only the carry's level is heavy
    assert all(_ju(0, 2, k) != 0 for k in range(1, 17))
    assert oracle.joint_scan(lv, W, 9, SEED, 0, 2) == 7           # first sample at level 9
    lv2 = lv.copy()
    lv2[lv2 == 9] = 8
    assert oracle.joint_scan(lv2, W, 9, SEED, 0, 2) == 0          # no acceptable sample


@pytest.mark.parametrize("r,i", [(0, 0), (3, 5), (11, 1000)])
def test_joint_scan_half_probability(r, i):
    N = 16
    W = np.zeros(N + 1)
    W[2] = -np.log(2.0)                                           # ratio 1/2 for level 2
    lv = np.full(64, 2, np.int32)
    T = oracle.threshold(W[2] - W[7])
    want = next((k for k in range(1, 65) if _ju(r, i, k) <= T), 0)
    assert oracle.joint_scan(lv, W, 7, SEED, r, i) == want
    assert T == 2**31 - 1


def _crafted_job(p, S, L=4):
    job = oracle.Job(L, p, SEED, 1)
    return job, S * L * L


def test_join_keeps_rejects_and_passes_the_carry():
    L, N, p, S = 4, 16, 4, 1
    job, M = _crafted_job(p, S)
    # round 0 (first joint of the job): chain 0 is kept whole (nothing to check)
    W = np.full(N + 1, -40.0)
    W[8] = 0.0
    W[10] = 0.0
    job.weights = W
    samp = np.zeros((p, M), np.int32)
    samp[0] = 6; samp[0, -1] = 8          # passes on level 8
    samp[1] = 5                           # never reaches a heavy level -> rejected
    samp[2] = 7; samp[2, 4:] = 10         # first heavy sample at k=5; passes on 10
    samp[3] = 10; samp[3, :2] = 4         # first heavy at k=3
    for i in (1, 2, 3):
        assert all(_ju(0, i, k) != 0 for k in range(1, M + 1))
    job.set_samples(S, samp)
    joined = job.join()
    k = list(job.k)
    assert k == [1, 0, 5, 3]
    assert joined == M + (M - 4) + (M - 2)
    h = np.bincount(samp[0], minlength=N + 1) + np.bincount(samp[2, 4:], minlength=N + 1) \
        + np.bincount(samp[3, 2:], minlength=N + 1)
    assert (job.hist == h).all()
    assert job.carry == 10
    # round 1: chain 0 checks against what chain 3 passed on (level 10)
    samp2 = np.full((p, M), 5, np.int32)
    samp2[0, 9:] = 8                      # k=10 for chain 0
    samp2[1, :] = 5                       # rejected: carry stays chain 0's last (8)
    samp2[2, 0] = 8                       # accepted at once, passes on 5
    samp2[3, :] = 5                       # carry level 5 now: W equal -> accepted at k=1
    for i in range(p):
        assert all(_ju(1, i, kk) != 0 for kk in range(1, M + 1))
    job.set_samples(S, samp2)
    j2 = job.join()
    assert list(job.k) == [10, 0, 1, 1]
    assert j2 == (M - 9) + M + M
    assert job.carry == 5
    assert job.round == 2


def test_no_accept_in_first_chain_keeps_previous_carry():
    L, N, p, S = 4, 16, 3, 1
    job, M = _crafted_job(p, S)
    W = np.full(N + 1, -40.0)
    W[12] = 0.0
    job.weights = W
    samp = np.full((p, M), 3, np.int32)
    samp[0, -1] = 12
    job.set_samples(S, samp)
    job.join()                            # chain 0 kept whole; carry 12; chains 1, 2 rejected
    assert list(job.k) == [1, 0, 0] and job.carry == 12
    samp = np.full((p, M), 3, np.int32)
    samp[2, 7] = 12
    job.set_samples(S, samp)
    job.join()
    assert list(job.k) == [0, 0, 8] and job.carry == 3


def test_streaming_first_accept_equals_stored_scan():
    L, seed = 6, 5
    N = L * L
    rng = np.random.default_rng(3)
    W = rng.normal(0, 1.0, N + 1)
    for c in range(6):
        s0 = oracle.init_lattice(L, seed, c, 1)
        m0 = oracle.level(oracle.energy(s0), L)
        S = 20
        _, _, _, _, samples = oracle.chain_round(L, seed, c, 4 * N, S, W, s0, m0, want_samples=True)
        for x in rng.integers(0, N + 1, 4):
            for r in (0, 7):
                k_scan = oracle.joint_scan(samples, W, int(x), seed, r, c)
                k_rep, ph = oracle.chain_first_accept(L, seed, c, 4 * N, S, W, s0, m0, int(x), r,
                                                      want_prefix_hist=True)
                assert k_rep == k_scan
                upto = (k_scan - 1) if k_scan else samples.size
                assert (ph == np.bincount(samples[:upto], minlength=N + 1)).all()


def test_invariants_over_iterations():
    L, p, S = 6, 12, 30
    N = L * L
    job = oracle.Job(L, p, 8, 1)
    for it in range(5):
        W0 = job.weights
        job.run_round(S, nthreads=3)
        joined = job.join()
        h = job.hist
        assert h.sum() == joined <= p * S * N
        assert (h >= 0).all()
        assert h[1] == 0 and h[N - 1] == 0            # unreachable levels
        k = job.k
        assert ((k == 0) | ((k >= 1) & (k <= S * N))).all()
        assert joined == sum(S * N - kk + 1 for kk in k if kk > 0)
        job.update_weights()
        W1 = job.weights
        assert (job.hist == 0).all()
        assert (W1[h == 0] == W0[h == 0]).all()
        nz = h > 0
        assert np.allclose(W1[nz], W0[nz] - np.log(h[nz]), rtol=0, atol=1e-12)
        assert (job.table == oracle.build_table(W1, L)).all()


def test_rounds_repeat_until_M_total():
    L, p, S = 4, 4, 10
    M = S * L * L
    job = oracle.Job(L, p, 2, 1)
    total = job.iteration(S, M_total=int(2.5 * p * M))
    assert job.round == 3 or total >= 2.5 * p * M
    assert total >= 2.5 * p * M
    assert job.t == job.round * M


def test_naive_join_keeps_everything():
    L, p, S = 4, 5, 7
    job = oracle.Job(L, p, 4, 1)
    job.weights = np.random.default_rng(0).normal(0, 3, L * L + 1)
    job.run_round(S)
    samples = job.samples
    assert job.join_naive() == p * S * L * L
    assert (job.k == 1).all()
    assert (job.hist == np.bincount(samples.reshape(-1), minlength=L * L + 1)).all()


def test_joined_chain_is_flat_under_exact_weights():
    L, p, S = 4, 16, 250
    N = L * L
    g = np.array(exact.enumerate_g(L), dtype=float)
    reach = g > 0
    W = np.zeros(N + 1)
    W[reach] = -np.log(g[reach])
    job = oracle.Job(L, p, 13, 1)
    job.weights = W
    job.run_round(50)                      # equilibrate, then start counting
    job.join()
    job.update_weights()
    job.weights = W
    per_round = []
    for _ in range(24):
        before = job.hist.copy()
        job.run_round(S, nthreads=4)
        job.join()
        d = job.hist - before
        per_round.append(d[reach] / d.sum())
    per_round = np.array(per_round)
    mean = per_round.mean(axis=0)
    err = per_round.std(axis=0, ddof=1) / np.sqrt(len(per_round))
    target = 1.0 / reach.sum()
    assert (np.abs(mean - target) < 5 * err + 1e-4).all(), (mean, err)


def test_energy_ordered_joint_hand_made():
    # W rises steeply with the level: a joint to a lower level fails (d <= -30,
    # threshold 0, and no uniform is 0), to an equal or higher level it passes
    L, N, p, S = 4, 16, 5, 1
    levels = [5, 1, 4, 2, 3]
    W = 30.0 * np.arange(N + 1)
    results = {}
    for mode in (0, 1):
        job, M = _crafted_job(p, S, L)
        job.set_join_order(mode)
        job.weights = W
        samp = np.array([[lv] * M for lv in levels], np.int32)
        for i in range(p):
            assert all(_ju(0, i, k) != 0 for k in range(1, M + 1))
        job.set_samples(S, samp)
        results[mode] = (job.join(), list(job.k), list(job.order), job.carry, job.hist.copy())
    # index order: chain 0 (level 5) kept whole, every later chain lies below the carry
    assert results[0][:4] == (M, [1, 0, 0, 0, 0], [0, 1, 2, 3, 4], 5)
    # ascending final energy: 1, 3, 4, 2, 0 -- each joint goes up, all kept whole
    assert results[1][:4] == (p * M, [1, 1, 1, 1, 1], [1, 3, 4, 2, 0], 5)
    assert (results[1][4] == np.bincount(levels, minlength=N + 1) * M).all()


def test_energy_order_ties_and_invariants():
    L, p, S = 6, 12, 3
    N = L * L
    o = oracle.Job(L, p, 21, 1)
    o.set_join_order(1)
    o.weights = np.random.default_rng(4).normal(0, 2.0, N + 1)
    for _ in range(4):
        o.run_round(S, 4)
        last = o.levels.copy()
        joined = o.join()
        order = o.order
        assert list(order) == list(np.lexsort((np.arange(p), last)))   # by level, ties by index
        k = o.k
        M = S * N
        assert joined == sum(M - kk + 1 for kk in k if kk > 0) == o.hist.sum()
        kept_in_order = [c for c in order if k[c] > 0]
        if kept_in_order:
            assert o.carry == last[kept_in_order[-1]]
        o.update_weights()


def test_adaptive_rounds_follow_the_rule():
    # W = 0: every sample is kept, so round sizes follow from the rule by hand
    L, p, S = 4, 6, 10
    N = L * L
    o = oracle.Job(L, p, 3, 1)
    per_round = p * S * N
    joined, sweeps = o.iteration_adaptive(S, int(2.5 * per_round), 2)
    assert sweeps == [S, S, 5]                 # remaining 0.5 p S N at rate p N per sweep
    assert joined == 2 * per_round + p * 5 * N
    # the rule clamps to [1, S]: a tiny remainder still takes one sweep
    o2 = oracle.Job(L, p, 3, 1)
    joined2, sweeps2 = o2.iteration_adaptive(S, per_round + 1, 2)
    assert sweeps2 == [S, 1] and joined2 == per_round + p * N
    # an M_total already met after one round: one round
    o3 = oracle.Job(L, p, 3, 1)
    assert o3.iteration_adaptive(S, 1, 2)[1] == [S]


def test_adaptive_iteration_invariants_under_rejections():
    L, p, S = 6, 10, 4
    N = L * L
    o = oracle.Job(L, p, 8, 1)
    o.weights = np.random.default_rng(2).normal(0, 6.0, N + 1)
    M_total = 3 * p * S * N // 2
    joined, sweeps = o.iteration_adaptive(S, M_total, 4, max_rounds=200)
    assert joined >= M_total or len(sweeps) == 200
    assert all(1 <= s <= S for s in sweeps) and sweeps[0] == S
    assert o.round == len(sweeps)


def test_acceptance_from_per_level_minimum_uniforms():
    # The identity the GPU's exact scan relies on (Sec. 2 step 4): a chain
    # keeps samples for input x iff some visited level m has
    # min{u_k : m_k = m} <= thr(W[m] - W[x]).  Checked against the oracle's
    # literal scan on random sequences, weights and inputs.
    rng = np.random.default_rng(11)
    N = 36
    for trial in range(60):
        M = int(rng.integers(8, 200))
        lv = np.clip(np.cumsum(rng.integers(-2, 3, M)) + int(rng.integers(5, 30)), 0, N).astype(np.int32)
        W = rng.normal(0, float(rng.choice([0.5, 3.0, 12.0])), N + 1)
        x = int(rng.integers(0, N + 1))
        r, i = int(rng.integers(0, 5)), int(rng.integers(0, 50))
        umin = {}
        for k in range(1, M + 1):
            u = _ju(r, i, k)
            umin[int(lv[k - 1])] = min(umin.get(int(lv[k - 1]), 0xFFFFFFFF), u)
        accept = any(u <= oracle.threshold(W[m] - W[x]) for m, u in umin.items())
        assert accept == (oracle.joint_scan(lv, W, x, SEED, r, i) > 0), trial
