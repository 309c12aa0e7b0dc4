"""The GPU row sweep (bit-parallel neighbour counts, Philox prefetch,
dwell-time histogram) and the joint's replay hooks (per-word joint
uniforms, first accepted sample, per-level minimum uniforms) compiled for
the host and checked against the oracle for every supported lattice size,
before any of it runs on a GPU."""
import os
import shutil
import subprocess

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_sweep_row_matches_oracle_on_host(tmp_path):
    exe = tmp_path / "emu"
    obj = tmp_path / "oracle.o"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-c",
                           os.path.join(ROOT, "oracle", "mc_oracle.c"), "-o", str(obj)])
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-include", os.path.join(HERE, "host_emu", "cuda_stub.h"),
                           "-I", os.path.join(ROOT, "paper_0812_2964_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "oracle"),
                           os.path.join(HERE, "host_emu", "sweep_row_vs_oracle.cpp"), str(obj),
                           "-o", str(exe), "-lm", "-pthread"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(": ok") == 13
