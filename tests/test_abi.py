"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute calls: no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_0812_2964_gb300 as mc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(mc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return mc.build()


def test_header_declares_the_core_calls():
    d = _declared()
    for name in ("mc_init", "mc_run_sweeps", "mc_join", "mc_histogram", "mc_update_weights"):
        assert name in d


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    for n in _declared():
        assert hasattr(mc, n), n


def test_no_gpu_call_without_device(libpath):
    # loading is fine; the launch counter is a pure host query
    assert mc.mc_kernel_launches() >= 0
    assert isinstance(mc.mc_last_error(), str)


def test_init_rejects_bad_arguments(libpath):
    # argument checks happen before any CUDA call
    for L, p, start in [(3, 4, 0), (6, 4, 0), (132, 4, 0), (8, 0, 0), (8, 4, 2)]:
        with pytest.raises(mc.McError) as e:
            mc.mc_init(L, p, 1, start)
        assert e.value.code == mc.MC_EINVAL


def test_job_device_bytes_is_a_host_query(libpath):
    assert mc.mc_job_device_bytes(6, 10, 1) == 0 and mc.mc_job_device_bytes(8, 0, 1) == 0
    a = mc.mc_job_device_bytes(32, 100, 10)
    assert a > 0
    assert mc.mc_job_device_bytes(32, 200, 10) > a      # more chains, more memory
    assert mc.mc_job_device_bytes(64, 100, 10) > a      # larger lattice, more memory


def test_job_device_bytes_counts_the_round_record(libpath):
    # a whole-sweep round of at most 2^33 samples is recorded, 2 bytes a
    # sample for every chain of a tile of 32: one chain past a full tile adds
    # a whole tile's record
    M = 10 * 32 * 32
    grow = mc.mc_job_device_bytes(32, 33, 10) - mc.mc_job_device_bytes(32, 32, 10)
    assert grow >= 32 * M * 2
    assert mc.mc_job_device_bytes(32, 34, 10) - mc.mc_job_device_bytes(32, 33, 10) < M * 2
    # above 2^33 samples the round is replayed instead: no record (16.8 GB at
    # 500 sweeps of 1024 chains at L = 128, 8.4e9 samples; none at 600 sweeps)
    assert 1024 * 500 * 128 * 128 <= 2 ** 33 < 1024 * 600 * 128 * 128
    with_rec = mc.mc_job_device_bytes(128, 1024, 500)
    without = mc.mc_job_device_bytes(128, 1024, 600)
    assert with_rec - without > 1024 * 500 * 128 * 128 * 2 * 0.9


def test_load_rejects_missing_and_foreign_files(libpath, tmp_path):
    # checked before any CUDA call
    with pytest.raises(mc.McError) as e:
        mc.mc_load(str(tmp_path / "missing.job"))
    assert e.value.code == mc.MC_EINVAL
    bad = tmp_path / "foreign.job"
    bad.write_bytes(b"not a saved job at all" * 4)
    with pytest.raises(mc.McError) as e:
        mc.mc_load(str(bad))
    assert e.value.code == mc.MC_EINVAL


def test_last_error_is_per_thread(libpath):
    # argument errors come back before any CUDA call: no GPU needed
    import threading

    msgs = {}

    def fail_in_thread():
        with pytest.raises(mc.McError):
            mc.mc_init(3, 4, 1, 0)
        msgs["other"] = mc.mc_last_error()

    def fresh_thread():
        msgs["fresh"] = mc.mc_last_error()

    t = threading.Thread(target=fail_in_thread)
    t.start()
    t.join()
    t = threading.Thread(target=fresh_thread)
    t.start()
    t.join()
    assert "L=3" in msgs["other"], msgs["other"]
    assert msgs["fresh"] == ""


def test_job_device_bytes_caps_the_checkpoints(libpath):
    # rounds too large to record keep lattice checkpoints for the joint's
    # replays, fewer and longer segments once they would pass 4 GiB: a job's
    # memory stops growing with the round length
    for L, p in [(32, 16384), (64, 4096), (128, 1024)]:
        b1 = mc.mc_job_device_bytes(L, p, 200_000)
        b2 = mc.mc_job_device_bytes(L, p, 1_000_000)   # (S N < 2^34 at L = 128)
        assert b1 < 4 * 2 ** 30 + 200_000_000
        assert abs(b2 - b1) < 0.05 * b1
