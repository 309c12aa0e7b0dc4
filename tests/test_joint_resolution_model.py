"""The GPU joint's resolution scheme, modelled in plain Python on small
random rounds and compared with the oracle's literal serial joint (Sec. 2
steps 3-5).  The scheme: speculate that every chain receives the last level
of its predecessor, search all chains, then resolution passes (a chain is
re-searched when its actual input -- the last level of the nearest earlier
chain that kept samples, else the carry -- differs from the input its k was
found for; passes may defer when many chains are pending), then the exact
scan over per-level minimum joint uniforms, a search of the chains that keep
samples under a new input, more passes, and the serial fallback.  Every
policy must give the serial rule's k exactly."""
import numpy as np
import pytest

import oracle

SEED = 91


def _ju(r, i, k):
    q = k - 1
    return oracle.philox((q >> 2, r, i, 1), (SEED & 0xFFFFFFFF, SEED >> 32))[q & 3]


def _first(lv, U, W, x):
    """first k (1-based) with u_k <= thr(W[m_k] - W[x]); 0 if none; x < 0: 1"""
    if x < 0:
        return 1
    for k, (m, u) in enumerate(zip(lv, U), start=1):
        if u <= oracle.threshold(W[m] - W[x]):
            return k
    return 0


def _inputs(k, last, carry):
    """actual input of each chain from the current k's"""
    x, out = carry, []
    for i in range(len(k)):
        out.append(x)
        if k[i] > 0:
            x = last[i]
    return out


def _resolve(lv, U, W, carry, passes_before, passes_after, scan, defer):
    p = len(lv)
    last = [int(l[-1]) for l in lv]
    xused = [carry] + last[:-1]
    k = [_first(lv[i], U[i], W, xused[i]) for i in range(p)]

    def mark():
        xs = _inputs([max(v, 0) for v in k], last, carry)
        pend = []
        for i in range(p):
            if xs[i] != xused[i]:
                xused[i] = xs[i]
                k[i] = -1
                pend.append(i)
            elif k[i] < 0:
                pend.append(i)
        return pend

    def passes(n, may_defer):
        for _ in range(n):
            pend = mark()
            if may_defer and len(pend) > p // 16 and defer:
                continue                       # left to the scan
            for i in pend:
                k[i] = _first(lv[i], U[i], W, xused[i])

    if scan:
        passes(passes_before, True)
        pend = mark()
        if pend:
            f = min(pend)
            umin = [{} for _ in range(p)]
            for i in range(f, p):
                for m, u in zip(lv[i], U[i]):
                    umin[i][int(m)] = min(umin[i].get(int(m), 0xFFFFFFFF), u)
            x = _inputs([max(v, 0) for v in k], last, carry)[f]
            listed = []
            for i in range(f, p):
                known = x == xused[i] and k[i] >= 0
                if known:
                    acc = k[i] > 0
                elif x < 0:
                    acc, k[i] = True, 1
                else:
                    acc = any(u <= oracle.threshold(W[m] - W[x]) for m, u in umin[i].items())
                    xused[i] = x
                    k[i] = -1 if acc else 0
                    if acc:
                        listed.append(i)
                if acc:
                    x = last[i]
            for i in listed:
                k[i] = _first(lv[i], U[i], W, xused[i])
        passes(passes_before, False)
    else:
        passes(passes_after, False)
    # serial fallback until nothing changes
    fallback = 0
    while True:
        pend = mark()
        if not pend:
            break
        fallback += 1
        for i in pend:
            k[i] = _first(lv[i], U[i], W, xused[i])
    return k, fallback


@pytest.mark.parametrize("policy", [(2, 10, True, True), (2, 10, True, False), (0, 0, True, True),
                                    (0, 0, False, False), (1, 3, True, True), (0, 64, False, False)])
def test_every_policy_gives_the_serial_rule(policy):
    rng = np.random.default_rng(7)
    L = 4
    N = L * L
    for trial in range(25):
        p = int(rng.integers(2, 40))
        M = int(rng.integers(4, 60))
        W = rng.normal(0, float(rng.choice([1.0, 6.0, 15.0])), N + 1)
        lv = [np.clip(np.cumsum(rng.integers(-2, 3, M)) + int(rng.integers(2, N - 2)), 0, N) for _ in range(p)]
        r = int(rng.integers(0, 4))
        U = [[_ju(r, i, kk) for kk in range(1, M + 1)] for i in range(p)]
        carry = int(rng.integers(-1, N + 1)) if trial % 3 else -1
        # the serial rule
        want, x = [], carry
        for i in range(p):
            kk = _first(lv[i], U[i], W, x)
            want.append(kk)
            if kk > 0:
                x = int(lv[i][-1])
        got, fallback = _resolve(lv, U, W, carry, *policy)
        assert got == want, (trial, policy)
        if policy[2]:
            assert fallback == 0, (trial, policy)   # the exact scan settles everything by itself
