"""mc_generate_noalloc (one round of generation on caller-owned device
buffers, no device allocation) gives exactly what the job API gives for the
same chains: same spins, same levels, same per-level sample counts, on two
rounds in a row.  This file is collected last on purpose: the entry point's
scratch is shared process-wide, so it also runs after every other test."""
import numpy as np
import pytest

import paper_0812_2964_gb300 as mc
from paper_0812_2964_gb300.workloads import random_weights

pytestmark = pytest.mark.gpu


# L = 100 and 128 read the threshold table straight from the fixed scratch
# (it does not fit in shared memory); 128 fills the whole scratch.  L = 96,
# and L = 128 with more than 8 chains a warp (4900 chains over 608 warps),
# sweep their lattices in place in the caller's spin buffer.
@pytest.mark.parametrize("L,p,S", [(32, 300, 3), (48, 40, 2), (8, 70, 5), (100, 8, 1), (128, 8, 1),
                                   (96, 40, 1), (128, 4900, 1)])
def test_noalloc_generation_matches_job_api(L, p, S):
    torch = pytest.importorskip("torch")
    mc.build()
    N = L * L
    M = S * N
    seed = 4242 + L
    W = random_weights(L, seed=L, scale=3.0)
    job = mc.Job(L, p, seed, 1)
    job.weights = W
    spins0 = job.spin_words.copy()
    levels0 = (job.energies + 2 * N) // 4

    dev = torch.device("cuda")
    d_spins = torch.from_numpy(spins0.reshape(-1).view(np.int32).copy()).to(dev)
    d_levels = torch.from_numpy(levels0.astype(np.int32)).to(dev)
    d_W = torch.from_numpy(W.astype(np.float64)).to(dev)
    d_hist = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()

    h_prev = np.zeros(N + 1, np.int64)
    for r in range(2):
        # the job API: one round, chains concatenated whole, so h grows by
        # exactly this round's samples
        job.run_sweeps(S)
        job.join_naive()
        h_now = job.hist
        want_hist = h_now - h_prev
        h_prev = h_now
        want_spins = job.spin_words.reshape(-1)
        want_levels = (job.energies + 2 * N) // 4

        mc.mc_generate_noalloc(L, p, seed, r * M, S, d_spins.data_ptr(), d_levels.data_ptr(),
                               d_W.data_ptr(), d_hist.data_ptr(), None)
        torch.cuda.synchronize()
        got_spins = d_spins.cpu().numpy().view(np.uint32)
        assert np.array_equal(got_spins, want_spins), f"round {r}: spins differ"
        assert np.array_equal(d_levels.cpu().numpy(), want_levels), f"round {r}: levels differ"
        assert np.array_equal(d_hist.cpu().numpy(), want_hist), f"round {r}: histograms differ"
        assert want_hist.sum() == p * M
    job.close()


def test_noalloc_rejects_oversized_lattice():
    mc.build()
    with pytest.raises(mc.McError) as e:
        mc.mc_generate_noalloc(132, 4, 1, 0, 1, 16, 16, 16, 16, None)
    assert e.value.code == mc.MC_EINVAL
    assert "128" in str(e.value)
