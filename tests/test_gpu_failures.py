"""Failure handling on the host: an allocation that fails (injected on the host
before any CUDA call, as an out-of-memory would) is reported as MC_ENOMEM,
releases what the call had allocated, and leaves the job -- or the server
and its other jobs -- usable.  Nothing here faults, traps or hangs the GPU."""
import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()
    yield
    mc.mc_inject_alloc_failure(-1)


def _allocations_of_init(L, p):
    live0 = mc.mc_live_allocations()
    g = mc.Job(L, p, 1, 1)
    n = mc.mc_live_allocations() - live0
    g.close()
    assert mc.mc_live_allocations() == live0
    return n


def test_every_allocation_of_mc_init_can_fail_without_leaking():
    L, p = 16, 64
    n = _allocations_of_init(L, p)
    assert n >= 10
    live0 = mc.mc_live_allocations()
    for k in range(n):
        mc.mc_inject_alloc_failure(k)
        with pytest.raises(mc.McError) as e:
            mc.mc_init(L, p, 5, 1)
        assert e.value.code == mc.MC_ENOMEM
        assert mc.mc_live_allocations() == live0, k
    mc.mc_inject_alloc_failure(-1)
    g = mc.Job(L, p, 5, 1)          # and the next one works
    g.close()
    assert mc.mc_live_allocations() == live0


@pytest.mark.parametrize("trace", [False, True])
def test_round_allocation_failure_leaves_the_job_usable(trace):
    # the first round allocates the checkpoint segments (and the trace): make
    # each of those fail once; the job then runs on and matches the oracle
    L, p, S, seed = 8, 30, 4, 41
    live0 = mc.mc_live_allocations()
    g = mc.Job(L, p, seed, 1)
    g.set_trace(trace)
    o = oracle.Job(L, p, seed, 1)
    for k in range(3):                   # (k = 0 is the trace when it is on)
        mc.mc_inject_alloc_failure(k)
        with pytest.raises(mc.McError) as e:
            g.run_sweeps(S)
        assert e.value.code == mc.MC_ENOMEM
        assert g.info()["round_pending"] == 0
    mc.mc_inject_alloc_failure(-1)
    for _ in range(2):
        g.run_sweeps(S)
        o.run_round(S)
        assert g.join() == o.join()
        assert np.array_equal(g.k, o.k)
        assert np.array_equal(g.hist, o.hist)
        g.update_weights()
        o.update_weights()
        assert np.array_equal(g.weights, o.weights)
    g.close()
    assert mc.mc_live_allocations() == live0


def _alone(L, p, seed, iters, S):
    g = mc.Job(L, p, seed, 1)
    for _ in range(iters):
        g.run_sweeps(S)
        g.join()
        g.update_weights()
    W = g.weights
    g.close()
    return W


def test_server_admission_failure_ends_that_job_only():
    jobs = [(16, 128, 61, 3, 2), (32, 64, 62, 3, 2), (24, 100, 63, 2, 3)]
    live0 = mc.mc_live_allocations()
    with mc.Server(4 * GB, max_slots=1) as srv:
        mc.mc_inject_alloc_failure(3)        # inside the first job's admission (mc_init)
        ids = [srv.submit(*j) for j in jobs]
        with pytest.raises(mc.McError) as e:
            srv.wait(ids[0])
        assert e.value.code == mc.MC_ENOMEM
        res = [srv.wait(i) for i in ids[1:]]
        info = srv.info()
    mc.mc_inject_alloc_failure(-1)
    assert info["bytes_in_use"] == 0 and info["active"] == 0
    assert info["completed"] == 3                 # the failed one counts as ended
    for (L, p, seed, iters, S), (W, st) in zip(jobs[1:], res):
        assert st["status"] == mc.MC_OK
        assert np.array_equal(W, _alone(L, p, seed, iters, S))
    assert mc.mc_live_allocations() == live0


def test_thermo_buffer_failure():
    g = mc.Job(8, 16, 3, 1)
    g.run_sweeps(2)
    g.join()
    g.update_weights()
    live = mc.mc_live_allocations()
    mc.mc_inject_alloc_failure(0)
    with pytest.raises(mc.McError) as e:
        g.thermo([0.3])
    assert e.value.code == mc.MC_ENOMEM
    assert mc.mc_live_allocations() == live
    mc.mc_inject_alloc_failure(-1)
    assert np.isfinite(g.thermo([0.3])).all()
    g.close()
