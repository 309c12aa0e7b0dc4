"""The oracle's pins are sensitive: each plausible mistake below, planted in
a copy of the oracle's C source (on the CPU; the oracle itself is never
changed), makes the pin suites fail, while the unchanged source built the
same way passes them.  The stored regression anchor (tests/golden) is left
out on purpose: it compares the oracle with its own earlier output, and the
point is that the independent pins catch each mistake."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "mc_oracle.c")
PINS = ["test_oracle_primitives.py", "test_oracle_model.py", "test_oracle_dynamics.py",
        "test_oracle_joint.py", "test_oracle_thermo.py"]

# (name, text in the source, its replacement); the first occurrence is changed
MUTATIONS = [
    ("Metropolis table: sign of the weight difference (Sec. 4.2)",
     "or_threshold(W[mp] - W[m])", "or_threshold(W[m] - W[mp])"),
    ("a neighbour dropped from the energy change (Sec. 4.1)",
     "SPIN(s, L, x, y - 1) + SPIN(s, L, x, y + 1);", "SPIN(s, L, x, y - 1);"),
    ("site order transposed (typewriter order, x fastest)",
     "int x = site % L, y = site / L;", "int y = site % L, x = site / L;"),
    ("energy sign (Sec. 4.1 Hamiltonian)",
     "E -= SPIN(s, L, x, y) *", "E += SPIN(s, L, x, y) *"),
    ("joint test: sign of the weight difference (Sec. 2 step 4)",
     "or_threshold(W[levels[k - 1]] - W[x_level])", "or_threshold(W[x_level] - W[levels[k - 1]])"),
    ("joined chain: first kept sample dropped (Sec. 2 step 4)",
     "for (int64_t t = k - 1; t < M; ++t) j->h[lev[t]] += 1;",
     "for (int64_t t = k; t < M; ++t) j->h[lev[t]] += 1;"),
    ("carry: first instead of last kept configuration passed on (Sec. 2 step 4)",
     "j->carry = lev[M - 1];", "j->carry = lev[0];"),
    ("weight update: sign of ln h (Eq. new_weight)",
     "j->W[m] = j->W[m] - or_log_det(", "j->W[m] = j->W[m] + or_log_det("),
    ("exp: Taylor series truncated after 7 terms",
     "double poly = EXP_C[13];\n    for (int j = 12;", "double poly = EXP_C[6];\n    for (int j = 5;"),
    ("ln: atanh series truncated after 5 terms",
     "double q = LOG_C[10];\n    for (int j = 9;", "double q = LOG_C[4];\n    for (int j = 3;"),
    ("threshold: ceil(2^32 e^d) instead of ceil(...) - 1",
     "return (uint32_t)(ceil(x) - 1.0);", "return (uint32_t)ceil(x);"),
    ("Philox: one multiplier digit changed (SC'11 constants)",
     "#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F57u"),
]


def _build(tmp, tag, src):
    d = os.path.join(tmp, tag)
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "mc_oracle.c"), "w") as f:
        f.write(src)
    shutil.copy(os.path.join(ROOT, "oracle", "mc_oracle.h"), d)
    so = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", so, os.path.join(d, "mc_oracle.c"), "-lm"])
    return so


def _pins(so):
    env = dict(os.environ, MC_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *[os.path.join(HERE, f) for f in PINS]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_each_planted_mistake_fails_the_pins(tmp_path):
    with open(SRC) as f:
        src = f.read()
    builds = [("unchanged", _build(str(tmp_path), "unchanged", src))]
    for n, (name, old, new) in enumerate(MUTATIONS):
        assert src.count(old) >= 1, f"mutation target not found: {name}"
        builds.append((name, _build(str(tmp_path), f"m{n}", src.replace(old, new, 1))))
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        results = dict(zip([b[0] for b in builds], ex.map(lambda b: _pins(b[1]), builds)))
    rc, out = results.pop("unchanged")
    assert rc == 0, "the unchanged source built the same way must pass the pins:\n" + out
    survivors = [name for name, (rc, out) in results.items() if rc != 1]
    assert not survivors, "mistakes the pins did not catch (or that broke the run): " + "; ".join(
        f"{name}: rc {results[name][0]}\n{results[name][1]}" for name in survivors)
