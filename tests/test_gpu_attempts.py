"""Rounds that are not whole sweeps (Sec. 2 step 2 with Fig. 2's M_node =
100 < N): the GPU's per-attempt path and its joint -- over the recorded
levels with each chain's samples tested in parallel, or by serial replay
when the record is off -- against the oracle, bit for bit, alone and mixed
with sweep rounds."""
import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import random_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()
    oracle.build()


def _same(g, o, L):
    N = L * L
    assert np.array_equal(g.spin_words, oracle.pack_spins(o.spins))
    assert np.array_equal(g.energies, 4 * o.levels - 2 * N)


@pytest.mark.parametrize("order,naive,record", [(0, False, True), (1, False, True), (0, True, True),
                                                (0, False, False), (1, False, False)])
def test_fig2_rounds_match_the_oracle(order, naive, record):
    L, p, n = 20, 32, 100                      # Fig. 2: L = 20, p = 32, M_node = 100
    W = random_weights(L, 20, 4.0)
    g = mc.Job(L, p, 10, 1)
    if not record:
        g.set_partial_record(0)                # serial replay joint
    o = oracle.Job(L, p, 10, 1)
    g.weights = W
    o.weights = W
    g.set_join_order(order)
    o.set_join_order(order)
    for _ in range(3):
        for _ in range(5):
            g.run_attempts(n)
            o.run_attempts(n, 4)
            _same(g, o, L)
            jg = g.join_naive() if naive else g.join()
            jo = o.join_naive() if naive else o.join()
            assert jg == jo
            assert np.array_equal(g.k, o.k)
            assert np.array_equal(g.hist, o.hist)
            assert g.info()["carry_energy"] == 4 * o.carry - 2 * L * L
        g.update_weights()
        o.update_weights()
        assert np.array_equal(g.weights, o.weights)


@pytest.mark.parametrize("record", [True, False])
def test_mixed_round_lengths(record):
    L, p = 16, 10
    N = L * L
    W = random_weights(L, 3, 6.0)
    g = mc.Job(L, p, 4, 1)
    if not record:
        g.set_partial_record(0)
    o = oracle.Job(L, p, 4, 1)
    g.weights = W
    o.weights = W
    plan = [("s", 1), ("a", 48), ("s", 2), ("a", 3 * N - 48), ("s", 1), ("a", 7), ("a", N - 7)]
    for kind, v in plan:
        if kind == "s":
            g.run_sweeps(v)
            o.run_attempts(v * N, 4)
        else:
            g.run_attempts(v)
            o.run_attempts(v, 4)
        _same(g, o, L)
        assert g.join() == o.join()
        assert np.array_equal(g.k, o.k)
        assert np.array_equal(g.hist, o.hist)
        assert g.info()["attempts_per_chain"] == o.t
    g.update_weights()
    o.update_weights()
    assert np.array_equal(g.weights, o.weights)


def test_batch_refuses_jobs_inside_a_sweep():
    g = mc.Job(8, 4, 1, 1)
    g.run_attempts(10)
    g.join()
    with pytest.raises(mc.McError) as e:
        mc.mc_batch_run([g], 1, 1, 1)
    assert e.value.code == mc.MC_EINVAL


def test_long_partial_rounds_with_late_first_passes():
    # rounds of 3000 attempts (> one block of threads per chain) under rough
    # weights, so first passing samples fall in later blocks or never
    L, p, n = 12, 24, 3000
    W = random_weights(L, 31, 12.0)
    g = mc.Job(L, p, 13, 1)
    o = oracle.Job(L, p, 13, 1)
    g.weights = W
    o.weights = W
    g.run_attempts(7)                           # inside a sweep from now on
    o.run_attempts(7, 4)
    assert g.join() == o.join()
    late = 0
    for _ in range(4):
        g.run_attempts(n)
        o.run_attempts(n, 4)
        _same(g, o, L)
        assert g.join() == o.join()
        k = g.k
        assert np.array_equal(k, o.k)
        assert np.array_equal(g.hist, o.hist)
        late += int(((k > 1024) | (k == 0)).sum())
    assert late > 0
    assert g.info()["device_bytes"] >= p * n * 4


def test_partial_record_argument_checks():
    g = mc.Job(8, 4, 1, 1)
    g.run_attempts(10)
    with pytest.raises(mc.McError) as e:
        g.set_partial_record(100)
    assert e.value.code == mc.MC_ESTATE
    g.join()
    g.set_partial_record(-1)
