"""Stored fixtures: the paper's Table 1 parameters (cited) behind the
L100_p32 workload, and the oracle's regression anchor written by
tests/golden/make_golden.py."""
import os

import oracle
from paper_0812_2964_gb300.workloads import WORKLOADS

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table1():
    out = {}
    for line in open(os.path.join(HERE, "paper_table1.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = int(value)
    return out


def test_table1_workload():
    t = _table1()
    w = WORKLOADS["L100_p32"]
    assert (w.L, w.chains, w.iterations) == (t["L"], t["p"], t["I"])
    # M_node = M_total / p samples per chain per iteration, rounded up to whole sweeps of N
    assert w.sweeps == -(-t["M_total"] // (t["p"] * w.N))


def test_oracle_matches_its_stored_anchor():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    oracle.build()
    stored = [l.rstrip("\n") for l in open(os.path.join(HERE, "oracle_L4_p8_seed7.txt")) if not l.startswith("#")]
    now = [f"{n} {i} {v}" for n, i, v in mod.compute()]
    assert stored == now
