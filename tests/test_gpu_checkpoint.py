"""Checkpoint / resume: a job saved between rounds and loaded into a new job
continues exactly as the uninterrupted job (spins, levels, k, histograms,
weights, carry, counters)."""
import numpy as np
import pytest

import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import random_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()


def _state(g):
    info = g.info()
    return (g.spin_words.copy(), g.energies.copy(), g.weights.copy(), g.hist.copy(), g.visited.copy(),
            info["attempts_per_chain"], info["rounds_joined"], info["carry_valid"], info["carry_energy"],
            info["total_joined"])


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


@pytest.mark.parametrize("L,p,S,order", [(16, 50, 3, 0), (32, 70, 2, 1), (64, 9, 1, 0)])
def test_resume_is_exact(tmp_path, L, p, S, order):
    W = random_weights(L, 7, 6.0)

    def make():
        g = mc.Job(L, p, 99, 1)
        g.weights = W
        g.set_join_order(order)
        return g

    a = make()
    b = make()
    for _ in range(2):
        for g in (a, b):
            g.run_sweeps(S); g.join(); g.update_weights()
    # mid-iteration: one round joined, weights not yet updated
    for g in (a, b):
        g.run_sweeps(S); g.join()
    path = str(tmp_path / "job.bin")
    b.save(path)
    b.close()
    c = mc.Job.load(path)
    _same(_state(a), _state(c))
    for _ in range(2):
        ka = []
        for g in (a, c):
            g.run_sweeps(S); g.join()
            ka.append(g.k.copy())
            g.update_weights()
        assert np.array_equal(ka[0], ka[1])
        _same(_state(a), _state(c))


def test_save_refused_while_a_round_is_pending(tmp_path):
    g = mc.Job(8, 4, 1, 1)
    g.run_sweeps(1)
    with pytest.raises(mc.McError) as e:
        g.save(str(tmp_path / "x.bin"))
    assert e.value.code == mc.MC_ESTATE
