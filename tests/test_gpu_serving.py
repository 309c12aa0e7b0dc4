"""Serving (continuous batching): every job's result is the same alone and in
the mix, bit for bit; admission respects slots and the memory budget."""
import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()


def _alone(L, p, seed, iters, S, start=1):
    g = mc.Job(L, p, seed, start)
    for _ in range(iters):
        g.run_sweeps(S)
        g.join()
        g.update_weights()
    W = g.weights
    joined = g.info()["total_joined"]
    dev = g.info()["device_bytes"]
    g.close()
    return W, joined, dev


MIX = [(16, 256, 1001, 5, 4), (32, 512, 1002, 4, 3), (48, 300, 1003, 3, 2), (64, 256, 1004, 3, 2),
       (96, 64, 1005, 2, 1), (128, 40, 1006, 2, 1), (8, 33, 1007, 6, 5), (24, 1000, 1008, 4, 3)]


def test_results_identical_alone_and_in_the_mix():
    with mc.Server(40 * GB, max_slots=4) as srv:
        ids = [srv.submit(L, p, seed, iters, S) for (L, p, seed, iters, S) in MIX]
        got = [srv.wait(j) for j in ids]
        info = srv.info()
    assert info["completed"] == len(MIX) and info["active"] == 0 and info["queued"] == 0
    # continuous batching: several jobs were resident and running at once
    assert 2 <= info["peak_active"] <= 4
    spans = [(st["t_admit"], st["t_done"]) for _, st in got]
    overlapping = [(a, b) for a in range(len(spans)) for b in range(a + 1, len(spans))
                   if max(spans[a][0], spans[b][0]) < min(spans[a][1], spans[b][1])]
    assert overlapping, spans
    for (L, p, seed, iters, S), (W, st) in zip(MIX, got):
        W_alone, joined, dev = _alone(L, p, seed, iters, S)
        assert np.array_equal(W, W_alone), f"L={L}"
        assert st["joined"] == joined
        assert st["attempts"] == p * iters * S * L * L
        assert st["device_bytes"] == dev == mc.mc_job_device_bytes(L, p, S)
        assert st["t_submit"] <= st["t_admit"] <= st["t_done"]


def test_served_job_matches_the_oracle():
    L, p, seed, iters, S = 8, 20, 77, 4, 3
    with mc.Server(1 * GB, max_slots=2) as srv:
        W, _ = srv.wait(srv.submit(L, p, seed, iters, S))
    o = oracle.Job(L, p, seed, 1)
    for _ in range(iters):
        o.iteration(S, 0, 4)
    assert np.array_equal(W, o.weights)


def test_budget_admits_one_job_at_a_time():
    jobs = [(32, 128, 2001 + i, 3, 2) for i in range(4)]
    need = mc.mc_job_device_bytes(32, 128, 2)
    with mc.Server(need + need // 2, max_slots=4) as srv:
        ids = [srv.submit(*j) for j in jobs]
        res = [srv.wait(i) for i in ids]
        info = srv.info()
        assert info["peak_active"] == 1
        assert info["peak_bytes"] == need
        with pytest.raises(mc.McError) as e:
            srv.submit(64, 4096, 1, 1, 1)      # alone larger than the budget
        assert e.value.code == mc.MC_ENOMEM
    # serialised by the budget: admissions follow completions
    for a, b in zip(res, res[1:]):
        assert a[1]["t_done"] <= b[1]["t_admit"]
    for (L, p, seed, iters, S), (W, _) in zip(jobs, res):
        assert np.array_equal(W, _alone(L, p, seed, iters, S)[0])


def test_bad_requests():
    with mc.Server(1 * GB, max_slots=1) as srv:
        for spec in [(6, 10, 1, 1, 1), (8, 0, 1, 1, 1), (8, 10, 1, 0, 1), (8, 10, 1, 1, 0)]:
            with pytest.raises(mc.McError) as e:
                srv.submit(*spec)
            assert e.value.code == mc.MC_EINVAL
        with pytest.raises(mc.McError) as e:
            mc.mc_server_poll(srv.h, 12345)
        assert e.value.code == mc.MC_EINVAL
        j = srv.submit(8, 4, 1, 1, 1)
        W, st = srv.wait(j)
        assert st["status"] == mc.MC_OK and W.shape == (65,)
        with pytest.raises(mc.McError) as e:
            mc.mc_server_wait(srv.h, j, 65)     # already collected
        assert e.value.code == mc.MC_EINVAL


def test_free_with_work_in_flight():
    srv = mc.Server(4 * GB, max_slots=1)
    for i in range(4):
        srv.submit(32, 256, 3000 + i, 2, 5)
    srv.close()                                 # cancels the queued ones, finishes the admitted one
