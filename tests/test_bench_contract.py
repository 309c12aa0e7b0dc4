"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line with the contract's keys; the serving stream has the shape of its
description.  CPU only."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "L32_p16384"


def test_serving_stream_shape():
    sys.path.insert(0, ROOT)
    from paper_0812_2964_gb300.workloads import SERVING_SIZES, serving_stream

    s = serving_stream(2000)
    t = np.array([j.arrival for j in s])
    assert np.all(np.diff(t) > 0)
    assert abs(len(s) / t[-1] - 20.0) < 1.5                  # mean 20 arrivals per second
    assert {j.L for j in s} == set(SERVING_SIZES)
    assert all(j.chains % 256 == 0 and 256 <= j.chains <= 4096 for j in s)
    assert all(20 <= j.iterations <= 60 and j.sweeps == 20 for j in s)
    mean_attempts = np.mean([j.chains * j.L ** 2 * j.sweeps * j.iterations for j in s])
    assert 8e9 < mean_attempts < 12e9                        # about 9.7e9 attempts per job
    assert serving_stream(50) == serving_stream(2000)[:50]   # the same seeded stream


def test_workload_names():
    # named workloads, and one job of any size as L<L>_p<chains> (the size of a served job)
    sys.path.insert(0, ROOT)
    from paper_0812_2964_gb300.workloads import WORKLOADS, workload

    assert workload("L32_p16384") is WORKLOADS["L32_p16384"]
    w = workload("L96_p2048")
    assert (w.L, w.chains, w.sweeps, w.N) == (96, 2048, 20, 96 * 96)
    with pytest.raises(KeyError):
        workload("L96")
