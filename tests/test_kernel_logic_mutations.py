"""The host checks of the GPU kernels' logic are sensitive: each plausible
mistake below, planted in a copy of a kernel header (on the CPU; the
library's sources are never changed), makes its host check fail -- the row
sweep and the joint's replay hooks against the oracle, the round record's
layout against the oracle's per-sample levels, the exact scan's state
machine against the serial rule -- while the unchanged headers pass."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_0812_2964_gb300", "csrc")

# host checks: harness source, extra include directory, expected "ok" lines
SWEEP = ("sweep_row_vs_oracle.cpp", None, 13)
RECORD = ("record_vs_oracle.cpp", os.path.join(HERE, "host_emu", "include"), 6)
SCAN = ("scan_fsm_vs_serial.cpp", None, 2)

# (name, host check, header, text in it, its replacement); each text occurs once
MUTATIONS = [
    ("threshold of the wrong outcome of the previous site", SWEEP, "mc_chain.cuh",
     "const uint32_t thr = f ? t1 : t0;", "const uint32_t thr = f ? t0 : t1;"),
    ("left neighbour's change of agreement with the wrong sign", SWEEP, "mc_chain.cuh",
     "D[q] = 0x04040404u + 0xF8u * b2;", "D[q] = 0xFCFCFCFCu + 0x08u * b2;"),
    ("left neighbour dropped from the packed counts", SWEEP, "mc_chain.cuh",
     "A0[q] = 4u * b0 + 8u * b1 + 4u * b2;", "A0[q] = 4u * b0 + 8u * b1;"),
    ("carry of the bit-sliced adder wrong", SWEEP, "mc_chain.cuh",
     "s1[w] = (eu[w] & ed[w]) | (er[w] & (eu[w] ^ ed[w]));", "s1[w] = (eu[w] & ed[w]) | (er[w] & eu[w]);"),
    ("periodic wrap of the right neighbour missing", SWEEP, "mc_chain.cuh",
     ": ((c >> 1) | ((cur[0] & 1u) << (lw - 1)));", ": (c >> 1);"),
    ("last site of a row ignores the flip of site 0", SWEEP, "mc_chain.cuh",
     "(((er[w] >> b) & 1u) ^ f0)", "((er[w] >> b) & 1u)"),
    ("threshold for the flipped outcome loaded at the unflipped level", SWEEP, "mc_chain.cuh",
     "const int off1 = off0 + nd4 * np1 + dl;", "const int off1 = off0 + nd4 * np1;"),
    ("Philox block counter advanced by half a word", SWEEP, "mc_chain.cuh",
     "pf.blk += static_cast<uint64_t>(nb_next / 4);", "pf.blk += static_cast<uint64_t>(nb_next / 8);"),
    ("late histogram count parked in the wrong slot", SWEEP, "mc_chain.cuh",
     "pend[b % D] = m4;", "pend[(b + 1) % D] = m4;"),
    ("joint search: sample index off by one", SWEEP, "mc_chain.cuh",
     "const int64_t kk = kw + b + 1;", "const int64_t kk = kw + b;"),
    ("summary replay: per-level maximum instead of minimum uniform", SWEEP, "mc_chain.cuh",
     "} else {\n      run_min = min(run_min, u);", "} else {\n      run_min = max(run_min, u);"),
    ("record: second sample of a pair shifted by 15 bits", RECORD, "mc_chain.cuh",
     "if (b & 1) pk[q] |= lv << 16;", "if (b & 1) pk[q] |= lv << 15;"),
    ("record: groups of a chain 31 chains apart instead of 32", RECORD, "mc_chain.cuh",
     "constexpr int kRecGroupStride = 4 * 32;", "constexpr int kRecGroupStride = 4 * 31;"),
    ("record: chain and sample swapped inside a group", RECORD, "mc_internal.h",
     "static_cast<size_t>(c % kRecTile)) *\n             4 +\n         static_cast<size_t>(k & 3);",
     "static_cast<size_t>(k & 3)) *\n             4 +\n         static_cast<size_t>(c % kRecTile);"),
    ("scan: transition functions composed in the wrong order", SCAN, "mc_scan_fsm.cuh",
     "tr_at(B, tr_at(A, s))", "tr_at(A, tr_at(B, s))"),
    ("scan: an answer already known read as unknown", SCAN, "mc_scan_fsm.cuh",
     "(c == kAnsYes || c == kAnsKnownYes) ? 1", "(c == kAnsYes) ? 1"),
    ("scan: an undecidable answer read as an input from far back", SCAN, "mc_scan_fsm.cuh",
     ": kStop;\n    r |=", ": kFar;\n    r |="),
]


def _run(tmp, tag, check, header, header_src, oracle_obj):
    harness, extra_inc, _ = check
    d = os.path.join(tmp, tag)
    os.makedirs(d, exist_ok=True)
    for n in os.listdir(CSRC):
        if n.endswith((".cuh", ".h")):
            shutil.copy(os.path.join(CSRC, n), d)
    if header:
        with open(os.path.join(d, header), "w") as f:
            f.write(header_src)
    exe = os.path.join(d, "emu")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-include", os.path.join(HERE, "host_emu", "cuda_stub.h")]
    if extra_inc:
        cmd += ["-I", extra_inc]
    cmd += ["-I", d, "-I", os.path.join(ROOT, "oracle"), os.path.join(HERE, "host_emu", harness), oracle_obj,
            "-o", exe, "-lm", "-pthread"]
    subprocess.check_call(cmd)
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return -1, "timeout"
    return r.returncode, r.stdout[-1500:]


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_each_planted_kernel_mistake_fails_the_host_check(tmp_path):
    obj = str(tmp_path / "oracle.o")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-c",
                           os.path.join(ROOT, "oracle", "mc_oracle.c"), "-o", obj])
    jobs = [(f"unchanged: {c[0]}", c, None, "") for c in (SWEEP, RECORD, SCAN)]
    for name, check, header, old, new in MUTATIONS:
        with open(os.path.join(CSRC, header)) as f:
            src = f.read()
        assert src.count(old) == 1, f"mutation target not found once: {name}"
        jobs.append((name, check, header, src.replace(old, new)))
    with cf.ThreadPoolExecutor(max_workers=6) as ex:
        futs = {name: ex.submit(_run, str(tmp_path), f"v{n}", check, header, src, obj)
                for n, (name, check, header, src) in enumerate(jobs)}
        results = {name: f.result() for name, f in futs.items()}
    for check in (SWEEP, RECORD, SCAN):
        rc, out = results.pop(f"unchanged: {check[0]}")
        assert rc == 0 and out.count(": ok") == check[2], out
    survivors = [name for name, (rc, out) in results.items() if rc == 0]
    assert not survivors, "mistakes the host checks did not catch: " + "; ".join(survivors)
