"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
runs: named workloads (lattice size, number of chains, sweeps per round,
weight iterations, seed, start) and seeded weight arrays.  Nothing here
computes any part of the method.

The workloads follow the Ising runs of the paper (Table 1: L = 100, p = 32,
M_total = 1e8, I = 1300; Fig. 2: L = 20, p = 32, M_node = 100) scaled to
thousands of chains on one GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    chains: int
    sweeps: int            # sweeps per chain per round (M = sweeps * L^2 samples)
    iterations: int        # weight iterations
    seed: int
    start: int = 1         # 0 all up, 1 random
    notes: str = ""

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def attempts_per_iteration(self) -> int:
        return self.chains * self.sweeps * self.N


WORKLOADS = {
    # 64 short chains on a small lattice, ordered start
    "L8_p64": Workload("L8_p64", 8, 64, 10_000, 10, 1, 0, "small case; the oracle runs it whole"),
    # thousands of chains, one per thread, lattice rows in registers
    "L32_p16384": Workload("L32_p16384", 32, 16384, 100_000, 50, 2, 1, "headline throughput case"),
    # larger lattices, lattice in shared memory, per-sweep energy trace
    "L64_p4096": Workload("L64_p4096", 64, 4096, 200_000, 100, 3, 1),
    "L128_p1024": Workload("L128_p1024", 128, 1024, 200_000, 100, 3, 1),
    # the paper's own lattice sizes
    "L100_p32": Workload("L100_p32", 100, 32, 313, 1300, 9, 1,
                         "Table 1: M_node = M_total / p = 3.125e6 samples, rounded up to whole sweeps"),
    "L20_p32": Workload("L20_p32", 20, 32, 1, 10, 10, 1, "Fig. 2 lattice"),
}


def workload(name: str) -> Workload:
    """A named workload, or an ad-hoc one named L<L>_p<chains> (20 sweeps a
    round, seed 11, random start) -- the size of one served job."""
    if name in WORKLOADS:
        return WORKLOADS[name]
    import re
    m = re.fullmatch(r"L(\d+)_p(\d+)", name)
    if not m:
        raise KeyError(f"unknown workload {name!r}")
    return Workload(name, int(m.group(1)), int(m.group(2)), 20, 10, 11, 1, "ad hoc")


# uneven sizes in one batch
BATCH_GROUPS = [(16, 8192, 4), (24, 4096, 5), (32, 4096, 6), (48, 2048, 7), (64, 1024, 8)]


def random_weights(L: int, seed: int, scale: float = 2.0) -> np.ndarray:
    """A seeded, smooth-plus-noise log-weight over the N+1 energy levels."""
    N = L * L
    rng = np.random.default_rng(seed)
    m = np.arange(N + 1)
    smooth = scale * np.sin(2 * np.pi * m / max(N, 1) * rng.uniform(0.5, 3.0))
    return smooth + rng.normal(0.0, scale * 0.25, N + 1)


def canonical_weights(L: int, beta: float) -> np.ndarray:
    """W(E) = -beta E on the levels E = -2N + 4m (a Boltzmann weight)."""
    N = L * L
    E = -2 * N + 4 * np.arange(N + 1)
    return -beta * E.astype(np.float64)


@dataclass(frozen=True)
class ServedJob:
    arrival: float   # seconds after the stream starts
    L: int
    chains: int
    iterations: int
    sweeps: int
    seed: int


SERVING_SIZES = (16, 32, 48, 64, 96, 128)


def serving_stream(n_jobs: int, rate: float = 20.0, sweeps: int = 20, seed: int = 5) -> list[ServedJob]:
    """Poisson arrivals (mean `rate` jobs/s) of weight-estimation jobs: L
    uniform over SERVING_SIZES, chains uniform over 256, 512, ..., 4096,
    weight iterations uniform over 20..60, `sweeps` sweeps per iteration,
    job seed 1000 + index."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n_jobs):        # job by job, so a shorter stream is a prefix of a longer one
        t += float(rng.exponential(1.0 / rate))
        L = int(rng.choice(np.array(SERVING_SIZES)))
        p = 256 * int(rng.integers(1, 17))
        its = int(rng.integers(20, 61))
        out.append(ServedJob(t, L, p, its, sweeps, 1000 + i))
    return out
