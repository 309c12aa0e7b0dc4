"""Pins of the oracle's statistical averages (Sec. 3.2, Eq. reweighting2;
E, C, F, S of Sec. 4.1): with W = -ln g(E) + c over the levels that exist,
the reweighted averages must equal the exact finite-lattice thermodynamics
of Kaufman's closed-form partition function (which the paper's Fig. 1
curves are built on), computed independently in mpmath."""
import numpy as np
import pytest

import oracle
from exact import enumerate_g, exact_thermo, transfer_g

BETAS = [0.05, 0.2, 0.35, 0.4406867935097715, 0.55, 0.8, 1.5, 4.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _weights_from_g(g, shift):
    g = np.array([int(x) for x in g], dtype=object)
    vis = np.array([1 if x > 0 else 0 for x in g], dtype=np.uint8)
    W = np.zeros(len(g))
    for m, x in enumerate(g):
        if x > 0:
            W[m] = -float(np.log(float(x))) + shift
    return W, vis


@pytest.mark.parametrize("L,gfun", [(4, enumerate_g), (6, transfer_g)])
def test_reweighting_with_exact_weights_reproduces_kaufman(L, gfun):
    g = gfun(L)
    W, vis = _weights_from_g(g, shift=3.25)
    out = oracle.thermo(L, W, vis, BETAS)
    for b, row in zip(BETAS, out):
        E, C, F, S = exact_thermo(L, b)
        assert row[0] == pytest.approx(E, rel=1e-11, abs=1e-9)
        assert row[1] == pytest.approx(C, rel=1e-9, abs=1e-9)
        assert row[2] == pytest.approx(F, rel=1e-11)
        assert row[3] == pytest.approx(S, rel=1e-10, abs=1e-10)


def test_limits():
    L = 4
    N = L * L
    W, vis = _weights_from_g(enumerate_g(L), shift=0.0)
    hot, cold = oracle.thermo(L, W, vis, [1e-6, 30.0])
    # beta -> 0: <H> = 0 by symmetry, S -> N ln 2; beta -> inf: two ground states
    assert abs(hot[0]) < 1e-3 and hot[3] == pytest.approx(N * np.log(2.0), rel=1e-6)
    assert cold[0] == pytest.approx(-2 * N) and cold[3] == pytest.approx(np.log(2.0), rel=1e-9)
    assert cold[1] == pytest.approx(0.0, abs=1e-9)


def test_shift_invariance_and_mask():
    L = 4
    W, vis = _weights_from_g(enumerate_g(L), shift=0.0)
    a = oracle.thermo(L, W, vis, BETAS)
    b = oracle.thermo(L, W + 123.5, vis, BETAS)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
    # the unreachable levels (m = 1, N - 1) hold W = 0: counting them is wrong
    vis_all = np.ones_like(vis)
    c = oracle.thermo(L, W, vis_all, BETAS)
    assert not np.allclose(a, c, rtol=1e-6)


def test_visited_mask_of_a_job():
    L, p = 4, 8
    o = oracle.Job(L, p, 5, 1)
    assert not o.visited.any()
    o.iteration(3, 0, 2)
    v = o.visited
    assert v[1] == 0 and v[L * L - 1] == 0 and v.sum() > 0
    W = o.weights
    assert (W[v == 0] == 0).all()
