"""Part (ii) on the GPU (Sec. 3.2, Eq. reweighting2; E, C, F, S of Sec. 4.1)
against the oracle and against Kaufman's exact finite-lattice values.

Tolerance (the two sides sum the same N+1 <= 16385 exponentials in a
different order, with exp/log from different libraries, each within a few
ulp): relative 1e-10 for E and F, 1e-9 for C, absolute 1e-10 * N for S
(S = beta (E - F) cancels at low temperature)."""
import numpy as np
import pytest

import oracle
import paper_0812_2964_gb300 as mc

pytest.importorskip("mpmath")
from exact import enumerate_g, exact_thermo  # noqa: E402

pytestmark = pytest.mark.gpu

BETAS = [0.05, 0.2, 0.35, 0.4406867935097715, 0.55, 0.8, 1.5, 4.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    mc.build()
    oracle.build()


def _close(g, o, N):
    assert np.allclose(g[:, 0], o[:, 0], rtol=1e-10, atol=1e-10 * N)
    assert np.allclose(g[:, 1], o[:, 1], rtol=1e-9, atol=1e-9)
    assert np.allclose(g[:, 2], o[:, 2], rtol=1e-10)
    assert np.allclose(g[:, 3], o[:, 3], rtol=0, atol=1e-10 * N)


@pytest.mark.parametrize("L,gfun", [(4, enumerate_g)])
def test_exact_weights_give_kaufman(L, gfun):
    # (the GPU takes L % 4 == 0; the oracle is pinned at L = 6 as well)
    N = L * L
    g = np.array([int(x) for x in gfun(L)], dtype=object)
    vis = np.array([1 if x > 0 else 0 for x in g], dtype=np.uint8)
    W = np.array([-np.log(float(x)) + 1.5 if x > 0 else 0.0 for x in g])
    job = mc.Job(L, 4, 1, 1)
    job.weights = W
    job.visited = vis
    assert np.array_equal(job.visited, vis)
    out = job.thermo(BETAS)
    _close(out, oracle.thermo(L, W, vis, BETAS), N)
    for b, row in zip(BETAS, out):
        E, C, F, S = exact_thermo(L, b)
        assert row[0] == pytest.approx(E, rel=1e-10, abs=1e-9)
        assert row[1] == pytest.approx(C, rel=1e-8, abs=1e-8)
        assert row[2] == pytest.approx(F, rel=1e-10)
        assert row[3] == pytest.approx(S, rel=1e-9, abs=1e-9)
    assert np.array_equal(out, job.thermo(BETAS))        # deterministic


@pytest.mark.parametrize("L,p,S,iters", [(16, 100, 5, 6), (64, 20, 2, 3), (128, 6, 1, 2)])
def test_after_weight_iterations_matches_oracle(L, p, S, iters):
    g = mc.Job(L, p, 40 + L, 1)
    o = oracle.Job(L, p, 40 + L, 1)
    for _ in range(iters):
        g.run_sweeps(S); g.join(); g.update_weights()
        o.iteration(S, 0, 8)
    assert np.array_equal(g.weights, o.weights)
    assert np.array_equal(g.visited, o.visited)
    _close(g.thermo(BETAS), oracle.thermo(L, o.weights, o.visited, BETAS), L * L)


def test_flat_histogram_weights_reproduce_exact_L8():
    # the method end to end (the Fig. 1 comparison on a lattice whose exact
    # values are cheap): weight iterations on the GPU, then the averages
    L, p, S = 8, 256, 2000
    N = L * L
    g = mc.Job(L, p, 8, 1)
    for _ in range(25):
        g.run_sweeps(S); g.join(); g.update_weights()
    out = g.thermo([0.2, 0.4406867935097715, 0.7])
    for b, row in zip([0.2, 0.4406867935097715, 0.7], out):
        E, C, F, S_ = exact_thermo(L, b)
        assert abs(row[0] - E) / N < 0.02
        assert abs(row[2] - F) / N < 0.01
        assert abs(row[3] - S_) / N < 0.02


def test_thermo_rejects_bad_betas():
    g = mc.Job(8, 2, 1, 1)
    for bad in ([0.0], [-1.0], [np.inf], [np.nan]):
        with pytest.raises(mc.McError) as e:
            g.thermo(bad)
        assert e.value.code == mc.MC_EINVAL
