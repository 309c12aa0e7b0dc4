"""The GPU row sweep (bit-parallel neighbour counts, Philox prefetch,
dwell-time histogram) and the joint's replay hooks (per-word joint
uniforms, first accepted sample, per-level minimum uniforms) compiled for
the host and checked against the oracle for every supported lattice size,
before any of it runs on a GPU; the round record's layout checked against
the oracle's per-sample levels; and the joint's exact-scan state machine
checked against the serial rule it stands for."""
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


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_scan_state_machine_matches_the_serial_rule_on_host(tmp_path):
    """The exact scan's per-position transition functions (compiled for the
    host), composed one by one and through the block scan's ranges and
    Hillis-Steele prefix, give every position the input the serial rule of
    Sec. 2 passes to it; kFar and kStop begin exactly where they should."""
    exe = tmp_path / "fsm"
    subprocess.check_call(["g++", "-O2", "-std=c++17",
                           "-include", os.path.join(HERE, "host_emu", "cuda_stub.h"),
                           "-I", os.path.join(ROOT, "paper_0812_2964_gb300", "csrc"),
                           os.path.join(HERE, "host_emu", "scan_fsm_vs_serial.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "algebra: ok" in r.stdout and "serial rule: ok" in r.stdout, r.stdout


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_round_record_layout_matches_oracle_samples_on_host(tmp_path):
    """Generation in recording mode (compiled for the host) stores every
    sample's level where the joint's recorded-round kernels read it
    (rec_index), equal to the oracle's level of that sample, for 37 chains
    (a full and a ragged tile of 32) at L = 8 ... 100; padding lanes and
    the space past the record stay unwritten."""
    exe = tmp_path / "rec"
    obj = tmp_path / "oracle.o"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-c",
                           os.path.join(ROOT, "oracle", "mc_oracle.c"), "-o", str(obj)])
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-include", os.path.join(HERE, "host_emu", "cuda_stub.h"),
                           "-I", os.path.join(HERE, "host_emu", "include"),
                           "-I", os.path.join(ROOT, "paper_0812_2964_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "oracle"),
                           os.path.join(HERE, "host_emu", "record_vs_oracle.cpp"), str(obj),
                           "-o", str(exe), "-lm", "-pthread"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("record: ok") == 6, r.stdout
