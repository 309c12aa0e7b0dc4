"""GPU path (through the C ABI) against the CPU oracle, element by element.

Bit-exact: spins, energies, per-sweep traces, first kept samples k_i, joined
lengths, carries, histograms, thresholds.  W after each update: identical
bits expected (same IEEE operations in the same order); the required bound
is 1e-12 absolute.
"""
import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import WORKLOADS, random_weights

pytestmark = pytest.mark.gpu

W_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()


def _compare_state(g, o, L):
    N = L * L
    assert np.array_equal(g.spin_words, oracle.pack_spins(o.spins))
    assert np.array_equal(g.energies, 4 * o.levels - 2 * N)


def _compare_weights(g, o):
    Wg, Wo = g.weights, o.weights
    assert np.abs(Wg - Wo).max() <= W_TOL
    assert np.array_equal(Wg, Wo)            # same operations, same order: same bits
    assert np.array_equal(g.table, o.table)
    assert np.array_equal(g.visited, o.visited)


def _run_parity(L, p, S, iters, start, seed, weights=None, shape=None, M_total=0, order=0, policy=None,
                seg=None, record=None):
    N = L * L
    g = mc.Job(L, p, seed, start)
    if record is False:
        g.set_round_record(0)       # the joint replays the chains from checkpoints
    elif record:
        g.set_round_record(1 << 29)  # the joint reads the round's record of levels
    if policy is not None:
        g.set_join_policy(*policy)
    if seg is not None:
        g.set_segment_samples(seg)
    if shape is not None:
        g.set_launch_shape(*shape)
    g.set_trace(True)
    o = oracle.Job(L, p, seed, start)
    if order:
        g.set_join_order(order)
        o.set_join_order(order)
    if weights is not None:
        g.weights = weights
        o.weights = weights
    _compare_state(g, o, L)
    _compare_weights(g, o)
    mism = 0
    for it in range(iters):
        tot_g = tot_o = 0
        while True:
            g.run_sweeps(S)
            o.run_round(S, nthreads=8)
            _compare_state(g, o, L)
            assert np.array_equal(g.trace, 4 * o.trace - 2 * N)
            jg, jo = g.join(), o.join()
            assert jg == jo
            assert np.array_equal(g.k, o.k)
            assert np.array_equal(g.order, o.order)
            info = g.info()
            mism += info["last_mismatch"]
            assert info["carry_valid"] == 1
            assert info["carry_energy"] == 4 * o.carry - 2 * N
            hg = g.hist
            assert np.array_equal(hg, o.hist)
            tot_g += jg
            tot_o += jo
            if tot_o >= M_total:
                break
        g.update_weights()
        o.update_weights()
        _compare_weights(g, o)
    return g, o, mism


@pytest.mark.parametrize("L,p,S,iters,start", [
    (4, 5, 3, 4, 1), (8, 37, 7, 4, 1), (12, 33, 5, 3, 1), (16, 100, 4, 3, 1), (20, 32, 2, 4, 1),
    (24, 50, 3, 3, 1), (28, 17, 2, 3, 1), (32, 130, 3, 4, 1), (36, 40, 2, 3, 1), (48, 33, 2, 3, 1),
    (64, 20, 2, 3, 1), (100, 9, 1, 3, 1), (128, 6, 1, 2, 1), (32, 3, 2, 3, 0),
])
def test_weight_iterations_bit_exact(L, p, S, iters, start):
    _run_parity(L, p, S, iters, start, seed=1000 + L)


@pytest.mark.parametrize("record", [True, False])
@pytest.mark.parametrize("L,p,S,iters", [(8, 37, 7, 3), (32, 130, 3, 3), (64, 20, 2, 2), (100, 7, 1, 2),
                                         (128, 6, 1, 2)])
def test_weight_iterations_bit_exact_record_and_replay(L, p, S, iters, record):
    # the joint reading the round's record of levels, and replaying every
    # sample from the checkpoints (the default records rounds this small)
    _run_parity(L, p, S, iters, 1, seed=2000 + L, weights=random_weights(L, L + 3, 6.0), record=record)


@pytest.mark.parametrize("L,p,S", [(8, 40, 5), (32, 70, 2), (64, 12, 1)])
def test_rugged_weight_rejections_and_resolution(L, p, S):
    # a rough weight makes many chains keep nothing, so speculated joint
    # inputs are often wrong and the resolution passes must fix them
    W = random_weights(L, seed=L, scale=12.0)
    g, o, mism = _run_parity(L, p, S, 3, 1, seed=77, weights=W)
    assert mism > 0


@pytest.mark.parametrize("shape", [(0, 27, 4), (0, 32, 1), (0, 5, 3), (1, 8, 2), (1, 32, 4), (1, 1, 1)])
def test_launch_shape_does_not_change_results(shape):
    _run_parity(32, 130, 2, 3, 1, seed=5, weights=random_weights(32, 3, 4.0), shape=shape)


@pytest.mark.parametrize("shape", [(1, 3, 4), (1, 16, 1)])
def test_launch_shape_large_lattice(shape):
    _run_parity(64, 21, 1, 2, 1, seed=6, shape=shape)


@pytest.mark.parametrize("L,p,shape", [(96, 9, (2, 9, 1)), (96, 21, (2, 3, 4)), (100, 7, (2, 7, 1)),
                                        (128, 6, (2, 2, 3)), (128, 40, (2, 32, 2)),
                                        (96, 9, (1, 9, 1)), (128, 6, (1, 2, 3))])
def test_lattice_placement_above_L64(L, p, shape):
    # placement 2 (the default here): generation with the lattice in global
    # memory, rows streamed through registers; 1: in shared memory.  Lane
    # groups of 4 at most 8 chains a warp.  The joint replays in shared memory.
    _run_parity(L, p, 1, 2, 1, seed=40 + L, shape=shape, weights=random_weights(L, L + 1, 6.0))
    g = mc.Job(L, p, 1, 1)
    g.set_launch_shape(*shape)
    assert g.info()["placement"] == shape[0]


def test_rounds_until_M_total():
    _run_parity(16, 20, 2, 3, 1, seed=9, M_total=int(2.5 * 20 * 2 * 256))


@pytest.mark.parametrize("L,p,S,scale", [(8, 40, 3, 12.0), (16, 300, 2, 6.0), (32, 130, 2, 4.0), (64, 20, 1, 8.0)])
def test_energy_ordered_joint_matches_oracle(L, p, S, scale):
    # energy-ordered joining (end of Sec. 2): chains joined by ascending final
    # level; rough weights so that both resolution paths run
    W = random_weights(L, seed=3 * L, scale=scale)
    g, o, mism = _run_parity(L, p, S, 3, 1, seed=500 + L, weights=W, order=1)
    order = g.order
    lv = (g.energies.astype(np.int64) + 2 * L * L) // 4
    assert list(order) == list(np.lexsort((np.arange(p), lv)))


@pytest.mark.parametrize("record", [True, False])
@pytest.mark.parametrize("policy", [(0, 0, 0), (-1, 0, 0), (0, 0, 64), (-1, 1, 3)])
@pytest.mark.parametrize("L,p,S", [(8, 40, 3), (32, 70, 2)])
def test_every_resolution_path_gives_the_serial_rule(policy, L, p, S, record):
    # (0,0,0): no passes, no scan -- the one-block fallback resolves all;
    # (-1,0,0): straight to the summary replay and exact scan;
    # (0,0,64): speculative passes only; (-1,1,3): one pass, then the scan;
    # each reading the round's record of levels, or replaying the chains
    W = random_weights(L, seed=L + 9, scale=10.0)
    g, o, mism = _run_parity(L, p, S, 3, 1, seed=900 + L, weights=W, policy=policy, record=record)
    assert mism > 0


@pytest.mark.parametrize("record", [True, False])
@pytest.mark.parametrize("L,p,S,scale", [(8, 300, 2, 40.0), (16, 200, 1, 30.0)])
def test_exact_scan_long_runs_of_rejecting_chains(L, p, S, scale, record):
    # straight to the summary and the exact scan, with weights so rough that
    # most chains keep nothing: inputs then come from many positions back
    # (beyond the scan's precomputed candidates), and the scan carries them
    W = random_weights(L, seed=L + 40, scale=scale)
    g, o, mism = _run_parity(L, p, S, 3, 1, seed=700 + L, weights=W, policy=(-1, 0, 0), record=record)
    assert mism > 0
    run = best = 0
    for k in g.k:   # joint order is index order here
        run = run + 1 if k == 0 else 0
        best = max(best, run)
    assert best > 8, best      # a run of rejecting chains longer than the candidate window


@pytest.mark.parametrize("L,p,S,seg,K,C", [
    (8, 40, 200, 64 * 3, 67, 3),     # multi-sweep segments, many of them
    (8, 40, 200, 1, 200, 1),         # one sweep each
    (16, 64, 96, 256, 96, 1),
    (32, 70, 64, 1024, 64, 1),
    (16, 64, 60, 256 * 7, 30, 2),    # too few at 7 sweeps: at least 32 (here 30 of 2)
])
def test_segment_lengths_give_the_serial_rule(L, p, S, seg, K, C):
    # the joint's replays run one checkpoint segment per lane; with rough
    # weights the first accepted samples fall in late segments of their
    # chains, where the search skips and stops segments behind an earlier hit
    W = random_weights(L, seed=L + 21, scale=10.0)
    g, o, mism = _run_parity(L, p, S, 2, 1, seed=300 + L, weights=W, seg=seg)
    info = g.info()
    assert (info["segments"], info["segment_sweeps"]) == (K, C)
    k = g.k
    M = S * L * L
    assert ((k > C * L * L) & (k <= M)).any()      # some hits beyond the first segment


@pytest.mark.parametrize("L,p,S,seg", [(8, 40, 200, 64 * 3), (32, 70, 64, 1024)])
def test_segment_lengths_with_the_replay_joint(L, p, S, seg):
    W = random_weights(L, seed=L + 21, scale=10.0)
    _run_parity(L, p, S, 2, 1, seed=300 + L, weights=W, seg=seg, record=False)


def test_round_record_limit_and_memory():
    L, p, S = 96, 5, 2            # rounds this small are recorded by default
    g = mc.Job(L, p, 3, 1)
    g.run_sweeps(S)
    g.join()
    with_rec = g.info()["device_bytes"]
    assert with_rec == mc.mc_job_device_bytes(L, p, S)
    h = mc.Job(L, p, 3, 1)
    h.set_round_record(p * S * L * L - 1)        # one sample too many: replayed
    h.run_sweeps(S)
    h.join()
    # 2 bytes a sample; the record's chains are padded to whole tiles of 32
    assert with_rec - h.info()["device_bytes"] == 2 * (-(-p // 32) * 32) * S * L * L
    assert np.array_equal(g.k, h.k) and np.array_equal(g.hist, h.hist)
    with pytest.raises(mc.McError) as e:
        h.run_sweeps(S)
        h.set_round_record(0)
    assert e.value.code == mc.MC_ESTATE


def test_segment_length_argument_checks():
    g = mc.Job(8, 4, 1, 1)
    with pytest.raises(mc.McError) as e:
        g.set_segment_samples(-1)
    assert e.value.code == mc.MC_EINVAL
    g.run_sweeps(1)
    with pytest.raises(mc.McError) as e:
        g.set_segment_samples(100)
    assert e.value.code == mc.MC_ESTATE
    g.join()
    g.set_segment_samples(0)


def test_naive_join_matches_oracle():
    L, p, S = 16, 24, 3
    g = mc.Job(L, p, 4, 1)
    o = oracle.Job(L, p, 4, 1)
    W = random_weights(L, 8, 5.0)
    g.weights = W
    o.weights = W
    for _ in range(2):
        g.run_sweeps(S)
        o.run_round(S)
        assert g.join_naive() == o.join_naive() == p * S * L * L
        assert np.array_equal(g.hist, o.hist)
        assert (g.k == 1).all()
        g.update_weights()
        o.update_weights()
        _compare_weights(g, o)


def test_config_L8_p64_all_iterations():
    w = WORKLOADS["L8_p64"]
    _run_parity(w.L, w.chains, w.sweeps, w.iterations, w.start, w.seed)


def test_offsets_are_exclusive_scan_of_kept_lengths():
    L, p, S = 8, 50, 3
    g = mc.Job(L, p, 12, 1)
    g.weights = random_weights(L, 1, 8.0)
    g.run_sweeps(S)
    joined = g.join()
    k, off = g.k, g.offsets
    M = S * L * L
    kept = np.where(k > 0, M - k + 1, 0)
    assert joined == kept.sum() == g.hist.sum()
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(kept)[:-1]]))


def test_call_order_and_argument_errors():
    g = mc.Job(8, 4, 1, 1)
    with pytest.raises(mc.McError) as e:
        g.join()
    assert e.value.code == mc.MC_ESTATE
    g.run_sweeps(1)
    with pytest.raises(mc.McError) as e:
        g.run_sweeps(1)
    assert e.value.code == mc.MC_ESTATE
    with pytest.raises(mc.McError) as e:
        g.update_weights()
    assert e.value.code == mc.MC_ESTATE
    g.join()
    with pytest.raises(mc.McError) as e:
        mc.mc_set_weights(g.h, np.zeros(5))
    assert e.value.code == mc.MC_EINVAL
    with pytest.raises(mc.McError) as e:
        g.set_launch_shape(0, 33, 1)
    assert e.value.code == mc.MC_EINVAL
    with pytest.raises(mc.McError) as e:
        mc.mc_run_sweeps(g.h, 0)
    assert e.value.code == mc.MC_EINVAL


def test_set_spins_roundtrip_and_energy():
    L, p = 48, 3
    g = mc.Job(L, p, 2, 0)
    rng = np.random.default_rng(0)
    s = rng.choice(np.array([-1, 1], np.int8), size=(p, L, L))
    g.spin_words = oracle.pack_spins(s)
    assert np.array_equal(g.spin_words, oracle.pack_spins(s))
    assert list(g.energies) == [oracle.energy(s[c]) for c in range(p)]


def test_autotune_picks_a_supported_shape_and_keeps_results():
    L, p, S = 32, 200, 2
    g = mc.Job(L, p, 31, 1)
    W = random_weights(L, 5, 3.0)
    g.weights = W
    shape = g.autotune(probe_sweeps=2, use_cache=False)
    assert shape[0] in (0, 1) and 1 <= shape[1] <= 32 and 1 <= shape[2] <= 4
    info = g.info()
    assert (info["placement"], info["chains_per_warp"], info["warps_per_block"]) == shape
    o = oracle.Job(L, p, 31, 1)
    o.weights = W
    _compare_state(g, o, L)         # tuning did not move the chains
    g.run_sweeps(S)
    o.run_round(S, nthreads=8)
    _compare_state(g, o, L)
    assert g.join() == o.join()
    assert np.array_equal(g.hist, o.hist)
    assert mc.mc_autotune(g.h, 2, True) == shape   # cached


@pytest.mark.parametrize("L,p,S,adapt", [(8, 30, 4, True), (16, 50, 3, True), (32, 40, 2, False)])
def test_iteration_with_m_total_matches_oracle(L, p, S, adapt):
    # step 6: rounds until h holds M_total samples, adaptive round lengths
    N = L * L
    W = random_weights(L, seed=L + 1, scale=6.0)
    g = mc.Job(L, p, 700 + L, 1)
    o = oracle.Job(L, p, 700 + L, 1)
    g.weights = W
    o.weights = W
    M_total = 5 * p * S * N // 2
    for _ in range(3):
        jg, rg = g.iteration(S, M_total, adapt=adapt, max_rounds=50)
        if adapt:
            jo, sweeps = o.iteration_adaptive(S, M_total, 8, max_rounds=50)
            assert rg == len(sweeps)
        else:
            jo = o.iteration(S, M_total, 8)
        assert jg == jo
        _compare_state(g, o, L)
        _compare_weights(g, o)


@pytest.mark.parametrize("L,start", [(4, 0), (12, 1), (64, 1)])
def test_single_chain(L, start):
    # p = 1: the joint has one chain; after the first round it checks against
    # its own last level of the previous round
    _run_parity(L, 1, 3, 3, start, seed=60 + L, weights=random_weights(L, L, 5.0))


def test_first_iteration_closed_form_on_the_gpu():
    # W = 0: every flip is accepted, so one sweep flips every spin in order and
    # returns to the starting energy; every chain is kept whole (k = 1)
    L, p, S = 8, 37, 3
    N = L * L
    g = mc.Job(L, p, 3, 0)                      # all up: E = -2N
    g.set_trace(True)
    g.run_sweeps(S)
    assert (g.trace == -2 * N).all()
    assert g.join() == p * S * N
    assert (g.k == 1).all()
    assert g.hist.sum() == p * S * N


def test_round_length_limit():
    g = mc.Job(128, 2, 1, 1)
    with pytest.raises(mc.McError) as e:
        mc.mc_run_sweeps(g.h, (1 << 34) // (128 * 128))    # M = S N would reach 2^34
    assert e.value.code == mc.MC_EINVAL
