"""Batched weight iterations (mc_batch_run) give, job by job, exactly what
running every job alone gives: one launch per job, one fused launch per
round, and the fused loop captured as a CUDA graph."""
import numpy as np
import pytest

import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import random_weights

pytestmark = pytest.mark.gpu

GROUPS = [(8, 40, 11), (16, 70, 12), (48, 9, 13), (24, 33, 14), (12, 10, 15)]  # (L, chains, seed); 12: no fused form


def _jobs(trace):
    js = []
    for L, p, seed in GROUPS:
        j = mc.Job(L, p, seed, 1)
        j.weights = random_weights(L, seed, 2.0)
        if trace:
            j.set_trace(True)
        js.append(j)
    return js


def _state(j):
    return (j.spin_words.copy(), j.energies.copy(), j.weights.copy(), j.k.copy(), j.info()["total_joined"])


@pytest.fixture(scope="module")
def reference():
    mc.build()
    js = _jobs(trace=False)
    S, iters = 3, 3
    for _ in range(iters):
        for j in js:
            j.run_sweeps(S)
            j.join()
            j.update_weights()
    return [_state(j) for j in js]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_modes_match_single_jobs(reference, mode):
    js = _jobs(trace=(mode == 2))
    mc.mc_batch_run(js, 3, 3, mode)
    for j, ref in zip(js, reference):
        got = _state(j)
        for a, b in zip(got[:4], ref[:4]):
            assert np.array_equal(a, b)
        assert got[4] == ref[4]
        assert j.info()["rounds_joined"] == 3


@pytest.mark.parametrize("mode", [1, 2])
def test_autotuned_batch_matches_single_jobs(reference, mode):
    # shapes picked by timing whole fused launches; the chains are the same
    js = _jobs(trace=False)
    mc.mc_batch_autotune(js, 2, use_cache=False)
    shapes = [mc.mc_batch_shape(j) for j in js]
    assert all(w == 4 for (_, _, w, _) in shapes)
    assert [f for (*_, f) in shapes] == [True, True, True, True, False]   # L = 12 keeps its own launch
    mc.mc_batch_autotune(js, 2, use_cache=True)                          # cached: same shapes
    assert [mc.mc_batch_shape(j) for j in js] == shapes
    mc.mc_batch_run(js, 3, 3, mode)
    for j, ref in zip(js, reference):
        got = _state(j)
        for a, b in zip(got[:4], ref[:4]):
            assert np.array_equal(a, b)
        assert got[4] == ref[4]


def test_batch_autotune_argument_checks():
    js = _jobs(trace=False)
    with pytest.raises(mc.McError) as e:
        mc.mc_batch_autotune(js, 0)
    assert e.value.code == mc.MC_EINVAL
    js[0].run_sweeps(1)
    with pytest.raises(mc.McError) as e:
        mc.mc_batch_autotune(js, 1)
    assert e.value.code == mc.MC_ESTATE


def test_batch_rejects_pending_and_duplicates():
    js = _jobs(trace=False)
    with pytest.raises(mc.McError):
        mc.mc_batch_run([js[0], js[0]], 1, 1, 1)
    js[1].run_sweeps(1)
    with pytest.raises(mc.McError) as e:
        mc.mc_batch_run(js, 1, 1, 1)
    assert e.value.code == mc.MC_ESTATE
