"""CPU model of sharding one job's chains over several GPUs (gloo ranks).

Each rank owns a contiguous range of chains and generates them (Sec. 2 step
2, here with the oracle).  The joint (steps 3-5) then needs one exchange:
an all-gather of every chain's last level and of its first accepted sample
under the speculated input (the last level of the chain before it); every
rank runs the same serial fix-up over those summaries, and only where the
actual input differs from the speculated one does the chain's owner search
again and broadcast the answer.  The kept samples' histograms are summed by
an all-reduce, and every rank applies the same weight update (Eq.
new_weight), so no weights are broadcast.  The model must reproduce the
single-process oracle's k_i, h and W bit for bit, round after round.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _owner(q, p, world):
    per = (p + world - 1) // world
    return q // per


def _shard_job(rank, world, L, p, seed, start, S, rounds, W0, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle

    N = L * L
    M = S * N
    per = (p + world - 1) // world
    lo, hi = rank * per, min(p, (rank + 1) * per)
    mine = range(lo, hi)
    spins = {c: oracle.init_lattice(L, seed, c, start) for c in mine}
    lev = {c: oracle.level(oracle.energy(spins[c]), L) for c in mine}
    W = np.array(W0, dtype=np.float64)
    h = np.zeros(N + 1, np.int64)
    carry = -1                                   # nothing passed on before the first joint
    record = []
    for r in range(rounds):
        # generation, own chains only
        samples, hists = {}, {}
        for c in mine:
            s, m, _, hist, smp = oracle.chain_round(L, seed, c, r * M, S, W, spins[c], lev[c], want_samples=True,
                                                    want_trace=False)
            spins[c], lev[c], samples[c], hists[c] = s, m, smp, hist
        # exchange 1: every chain's last level
        last = torch.zeros(p, dtype=torch.int64)
        for c in mine:
            last[c] = lev[c]
        dist.all_reduce(last)                    # ranges are disjoint: the sum is the gather
        last = last.numpy()
        # speculation: chain q receives the last level of chain q - 1
        spec = torch.zeros(p, dtype=torch.int64)
        for c in mine:
            x = carry if c == 0 else int(last[c - 1])
            spec[c] = 1 if x < 0 else oracle.joint_scan(samples[c], W, x, seed, r, c)
        dist.all_reduce(spec)
        spec = spec.numpy()
        # serial fix-up, the same on every rank; the owner answers a mismatch
        k = np.zeros(p, np.int64)
        x_in = carry
        for q in range(p):
            x_spec = carry if q == 0 else int(last[q - 1])
            if x_in == x_spec:
                k[q] = spec[q]
            else:
                t = torch.zeros(1, dtype=torch.int64)
                if _owner(q, p, world) == rank:
                    t[0] = 1 if x_in < 0 else oracle.joint_scan(samples[q], W, x_in, seed, r, q)
                dist.broadcast(t, src=_owner(q, p, world))
                k[q] = int(t[0])
            if k[q] > 0:
                x_in = int(last[q])
        if x_in >= 0:
            carry = x_in
        # kept samples' histogram: own chains, then one all-reduce
        hr = torch.zeros(N + 1, dtype=torch.int64)
        for c in mine:
            if k[c] > 0:
                hr += torch.from_numpy(np.bincount(samples[c][k[c] - 1:], minlength=N + 1).astype(np.int64))
        dist.all_reduce(hr)
        h += hr.numpy()
        record.append((k.copy(), h.copy()))
        # weight update (Eq. new_weight in logarithms), identical everywhere
        for m in np.nonzero(h)[0]:
            W[m] = W[m] - oracle.log_det(float(h[m]))
        h[:] = 0
        record.append(W.copy())
    if rank == 0:
        out.put(record)
    dist.barrier()


def _rank_main(rank, world, port, args, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _shard_job(rank, world, *args, out)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_joint_matches_the_single_process_oracle(world):
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import oracle
    from paper_0812_2964_gb300.workloads import random_weights

    oracle.build()
    L, p, seed, start, S, rounds = 8, 13, 71, 1, 2, 4
    W0 = random_weights(L, seed=7, scale=40.0)    # rough: rejections, so speculation fails somewhere
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    args = (L, p, seed, start, S, rounds, W0)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, args, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    record = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0

    o = oracle.Job(L, p, seed, start)
    o.weights = W0
    mism = 0
    for r in range(rounds):
        o.run_round(S)
        o.join()
        k, h = record[2 * r]
        assert np.array_equal(k, o.k), f"round {r}"
        assert np.array_equal(h, o.hist), f"round {r}"
        o.update_weights()
        assert np.array_equal(record[2 * r + 1], o.weights), f"round {r}"
        # how often the speculation (chain q-1 kept samples) was wrong
        mism += int(((k[:-1] == 0)).sum())
    assert mism > 0
