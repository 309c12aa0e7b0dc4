"""The host checks of the GPU row sweep and the joint's replay hooks are
sensitive: each plausible mistake below, planted in a copy of the kernels'
header (on the CPU; the library's sources are never changed), makes the
host emulation against the oracle fail, while the unchanged header passes."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_0812_2964_gb300", "csrc")
HEADER = "mc_chain.cuh"

# (name, text in mc_chain.cuh, its replacement); each text occurs once
MUTATIONS = [
    ("threshold of the wrong outcome of the previous site",
     "const uint32_t thr = f ? t1 : t0;", "const uint32_t thr = f ? t0 : t1;"),
    ("left neighbour's change of agreement with the wrong sign",
     "D[q] = 0x04040404u + 0xF8u * b2;", "D[q] = 0xFCFCFCFCu + 0x08u * b2;"),
    ("left neighbour dropped from the packed counts",
     "A0[q] = 4u * b0 + 8u * b1 + 4u * b2;", "A0[q] = 4u * b0 + 8u * b1;"),
    ("carry of the bit-sliced adder wrong",
     "s1[w] = (eu[w] & ed[w]) | (er[w] & (eu[w] ^ ed[w]));", "s1[w] = (eu[w] & ed[w]) | (er[w] & eu[w]);"),
    ("periodic wrap of the right neighbour missing",
     ": ((c >> 1) | ((cur[0] & 1u) << (lw - 1)));", ": (c >> 1);"),
    ("last site of a row ignores the flip of site 0",
     "(((er[w] >> b) & 1u) ^ f0)", "((er[w] >> b) & 1u)"),
    ("threshold for the flipped outcome loaded at the unflipped level",
     "const int off1 = off0 + nd4 * np1 + dl;", "const int off1 = off0 + nd4 * np1;"),
    ("Philox block counter advanced by half a word",
     "pf.blk += static_cast<uint64_t>(nb_next / 4);", "pf.blk += static_cast<uint64_t>(nb_next / 8);"),
    ("late histogram count parked in the wrong slot",
     "pend[b % D] = m4;", "pend[(b + 1) % D] = m4;"),
    ("joint search: sample index off by one",
     "const int64_t kk = kw + b + 1;", "const int64_t kk = kw + b;"),
    ("summary replay: per-level maximum instead of minimum uniform",
     "} else {\n      run_min = min(run_min, u);", "} else {\n      run_min = max(run_min, u);"),
]


def _run(tmp, tag, header_src, oracle_obj):
    d = os.path.join(tmp, tag)
    os.makedirs(d, exist_ok=True)
    for n in os.listdir(CSRC):
        if n.endswith((".cuh", ".h")):
            shutil.copy(os.path.join(CSRC, n), d)
    with open(os.path.join(d, HEADER), "w") as f:
        f.write(header_src)
    exe = os.path.join(d, "emu")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-include", os.path.join(HERE, "host_emu", "cuda_stub.h"),
                           "-I", d, "-I", os.path.join(ROOT, "oracle"),
                           os.path.join(HERE, "host_emu", "sweep_row_vs_oracle.cpp"), oracle_obj,
                           "-o", exe, "-lm", "-pthread"])
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
    with open(os.path.join(CSRC, HEADER)) as f:
        src = f.read()
    variants = [("unchanged", src)]
    for name, old, new in MUTATIONS:
        assert src.count(old) == 1, f"mutation target not found once: {name}"
        variants.append((name, src.replace(old, new)))
    with cf.ThreadPoolExecutor(max_workers=6) as ex:
        futs = {name: ex.submit(_run, str(tmp_path), f"v{n}", s, obj) for n, (name, s) in enumerate(variants)}
        results = {name: f.result() for name, f in futs.items()}
    rc, out = results.pop("unchanged")
    assert rc == 0 and out.count(": ok") == 13, out
    survivors = [name for name, (rc, out) in results.items() if rc == 0]
    assert not survivors, "mistakes the host check did not catch: " + "; ".join(survivors)
