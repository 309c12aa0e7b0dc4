"""Writes oracle_L4_p8_seed7.txt: the oracle's weights, histogram-free state
and joint results after three weight iterations of a small job (L = 4,
8 chains, 3 sweeps per round, random start, seed 7).  Calls only oracle/.
A regression anchor for the oracle (its pins against the paper and exact
results are in tests/test_oracle_*.py).  Run: python tests/golden/make_golden.py"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def compute():
    o = oracle.Job(4, 8, 7, 1)
    rows = []
    for it in range(3):
        o.run_round(3, 1)
        joined = o.join()
        rows.append(("joined", it, joined))
        rows.append(("k", it, " ".join(str(int(x)) for x in o.k)))
        o.update_weights()
    rows.append(("W", 3, " ".join(repr(float(w)) for w in o.weights)))
    rows.append(("levels", 3, " ".join(str(int(m)) for m in o.levels)))
    return rows


if __name__ == "__main__":
    oracle.build()
    with open(os.path.join(HERE, "oracle_L4_p8_seed7.txt"), "w") as f:
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        for name, it, val in compute():
            f.write(f"{name} {it} {val}\n")
