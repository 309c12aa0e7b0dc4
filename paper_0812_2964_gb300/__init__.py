"""Python binding of libmcgpu (include/mc.h): parallel multicanonical Ising
chains joined by detailed balance, on one GB300 (sm_103a).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  If the library has not been built (``build()``) or cannot be
loaded, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build

__all__ = ["build", "McError", "mc_info", "Job", "lib", "mc_kernel_launches"] + [
    "mc_init", "mc_free", "mc_set_stream", "mc_set_trace", "mc_run_sweeps", "mc_join",
    "mc_join_naive", "mc_histogram", "mc_update_weights", "mc_get_weights", "mc_set_weights",
    "mc_get_table", "mc_get_spins", "mc_set_spins", "mc_get_energies", "mc_get_trace",
    "mc_get_trace_chain", "mc_get_visited", "mc_set_visited", "mc_thermo", "mc_set_join_order",
    "mc_get_order", "mc_save", "mc_load", "mc_iteration", "mc_set_join_policy", "mc_run_attempts",
    "mc_set_segment_samples", "mc_set_partial_record", "mc_set_round_record", "mc_inject_alloc_failure", "mc_live_allocations",
    "mc_get_join", "mc_get_info", "mc_set_launch_shape", "mc_sync", "mc_last_error",
    "mc_generate_noalloc", "mc_autotune", "mc_batch_run", "mc_batch_autotune", "mc_batch_shape",
    "mc_job_device_bytes", "mc_server_create", "mc_server_submit", "mc_server_poll", "mc_server_wait",
    "mc_server_get_info", "mc_server_clock", "mc_server_free", "Server"]

# revision of the generation kernel; bump when it changes (profiles record it)
KERNEL_REV = "gen-6"

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ESTATE, MC_ETIMEOUT = 0, -1, -2, -3, -4, -5
_NAMES = {MC_EINVAL: "MC_EINVAL", MC_ENOMEM: "MC_ENOMEM", MC_ECUDA: "MC_ECUDA",
          MC_ESTATE: "MC_ESTATE", MC_ETIMEOUT: "MC_ETIMEOUT"}


class McError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class mc_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("N", ctypes.c_int), ("n_chains", ctypes.c_int),
                ("words_per_row", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("attempts_per_chain", ctypes.c_uint64), ("rounds_joined", ctypes.c_uint32),
                ("last_sweeps", ctypes.c_int64), ("round_pending", ctypes.c_int),
                ("carry_valid", ctypes.c_int), ("carry_energy", ctypes.c_int),
                ("last_joined", ctypes.c_int64), ("last_rejected", ctypes.c_int64),
                ("last_mismatch", ctypes.c_int64), ("last_passes", ctypes.c_int64),
                ("last_searched", ctypes.c_int64), ("total_joined", ctypes.c_int64),
                ("placement", ctypes.c_int),
                ("chains_per_warp", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("last_scanned", ctypes.c_int64),
                ("segments", ctypes.c_int), ("segment_sweeps", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mc_jobspec(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_chains", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("start", ctypes.c_int), ("iterations", ctypes.c_int), ("sweeps", ctypes.c_int64)]


class mc_jobstats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("slot", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("attempts", ctypes.c_int64),
                ("joined", ctypes.c_int64), ("device_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mc_server_info(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("queued", ctypes.c_int), ("active", ctypes.c_int),
                ("finished", ctypes.c_int), ("budget_bytes", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("peak_active", ctypes.c_int), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    """Load libmcgpu.so (built in-tree by ``build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: run paper_0812_2964_gb300.build() first")
        L = ctypes.CDLL(_LIB_PATH)
        sig = {
            "mc_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                       ctypes.POINTER(_vp)]),
            "mc_free": (None, [_vp]),
            "mc_set_stream": (ctypes.c_int, [_vp, _vp]),
            "mc_set_trace": (ctypes.c_int, [_vp, ctypes.c_int]),
            "mc_run_sweeps": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "mc_run_attempts": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "mc_join": (ctypes.c_int, [_vp, _i64p]),
            "mc_join_naive": (ctypes.c_int, [_vp, _i64p]),
            "mc_histogram": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_update_weights": (ctypes.c_int, [_vp]),
            "mc_get_weights": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_set_weights": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_get_table": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_get_spins": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
            "mc_set_spins": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
            "mc_get_energies": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_get_trace": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
            "mc_get_trace_chain": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t]),
            "mc_get_visited": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_set_visited": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_thermo": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
            "mc_set_join_order": (ctypes.c_int, [_vp, ctypes.c_int]),
            "mc_set_join_policy": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
            "mc_set_segment_samples": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "mc_set_partial_record": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "mc_set_round_record": (ctypes.c_int, [_vp, ctypes.c_int64]),
            "mc_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
            "mc_iteration": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                            _i64p, ctypes.POINTER(ctypes.c_int)]),
            "mc_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
            "mc_get_order": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
            "mc_get_join": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
            "mc_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(mc_info)]),
            "mc_set_launch_shape": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            "mc_sync": (ctypes.c_int, [_vp]),
            "mc_batch_run": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int64, ctypes.c_int]),
            "mc_batch_autotune": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int64, ctypes.c_int]),
            "mc_batch_shape": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
            "mc_autotune": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
            "mc_generate_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                   ctypes.c_uint64, ctypes.c_int64, _vp, _vp, _vp,
                                                   _vp, _vp]),
            "mc_job_device_bytes": (ctypes.c_uint64, [ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
            "mc_server_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(_vp)]),
            "mc_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(mc_jobspec), ctypes.POINTER(ctypes.c_uint64)]),
            "mc_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
            "mc_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.c_int,
                                              ctypes.POINTER(mc_jobstats)]),
            "mc_server_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(mc_server_info)]),
            "mc_server_clock": (ctypes.c_double, [_vp]),
            "mc_server_free": (None, [_vp]),
            "mc_kernel_launches": (ctypes.c_uint64, []),
            "mc_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int64]),
            "mc_live_allocations": (ctypes.c_int64, []),
            "mc_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != MC_OK:
        raise McError(rc, lib().mc_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------ C-ABI names
def mc_init(L: int, n_chains: int, seed: int, start: int = 1):
    h = _vp()
    _check(lib().mc_init(L, n_chains, seed, start, ctypes.byref(h)))
    return h


def mc_free(job):
    lib().mc_free(job)


def mc_set_stream(job, stream_handle: int | None):
    _check(lib().mc_set_stream(job, _vp(stream_handle or 0)))


def mc_set_trace(job, enabled: bool):
    _check(lib().mc_set_trace(job, 1 if enabled else 0))


def mc_run_sweeps(job, n_sweeps: int):
    _check(lib().mc_run_sweeps(job, n_sweeps))


def mc_run_attempts(job, n_attempts: int):
    _check(lib().mc_run_attempts(job, n_attempts))


def mc_join(job, want_length: bool = True):
    v = ctypes.c_int64(0)
    _check(lib().mc_join(job, ctypes.byref(v) if want_length else None))
    return int(v.value) if want_length else None


def mc_join_naive(job, want_length: bool = True):
    v = ctypes.c_int64(0)
    _check(lib().mc_join_naive(job, ctypes.byref(v) if want_length else None))
    return int(v.value) if want_length else None


def mc_histogram(job, out: np.ndarray):
    assert out.dtype == np.int64 and out.flags.c_contiguous
    _check(lib().mc_histogram(job, _ptr(out), out.size))
    return out


def mc_update_weights(job):
    _check(lib().mc_update_weights(job))


def mc_get_weights(job, out: np.ndarray):
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(lib().mc_get_weights(job, _ptr(out), out.size))
    return out


def mc_set_weights(job, w: np.ndarray):
    w = np.ascontiguousarray(w, dtype=np.float64)
    _check(lib().mc_set_weights(job, _ptr(w), w.size))


def mc_get_table(job, out: np.ndarray):
    assert out.dtype == np.uint32 and out.flags.c_contiguous
    _check(lib().mc_get_table(job, _ptr(out), out.size))
    return out


def mc_get_spins(job, out: np.ndarray):
    assert out.dtype == np.uint32 and out.flags.c_contiguous
    _check(lib().mc_get_spins(job, _ptr(out), out.size))
    return out


def mc_set_spins(job, words: np.ndarray):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    _check(lib().mc_set_spins(job, _ptr(w), w.size))


def mc_get_energies(job, out: np.ndarray):
    assert out.dtype == np.int32 and out.flags.c_contiguous
    _check(lib().mc_get_energies(job, _ptr(out), out.size))
    return out


def mc_get_trace(job, out: np.ndarray):
    assert out.dtype == np.int32 and out.flags.c_contiguous
    _check(lib().mc_get_trace(job, _ptr(out), out.size))
    return out


def mc_get_trace_chain(job, chain: int, out: np.ndarray):
    assert out.dtype == np.int32 and out.flags.c_contiguous
    _check(lib().mc_get_trace_chain(job, int(chain), _ptr(out), out.size))
    return out


def mc_get_visited(job, out: np.ndarray):
    assert out.dtype == np.uint8 and out.flags.c_contiguous
    _check(lib().mc_get_visited(job, _ptr(out), out.size))
    return out


def mc_set_visited(job, v: np.ndarray):
    v = np.ascontiguousarray(v, dtype=np.uint8)
    _check(lib().mc_set_visited(job, _ptr(v), v.size))


def mc_iteration(job, n_sweeps: int, m_total: int = 0, adapt: bool = False, max_rounds: int = 1_000_000):
    """One weight iteration; returns (joined, rounds)."""
    joined = ctypes.c_int64(0)
    rounds = ctypes.c_int(0)
    _check(lib().mc_iteration(job, n_sweeps, m_total, 1 if adapt else 0, max_rounds, ctypes.byref(joined),
                              ctypes.byref(rounds)))
    return joined.value, rounds.value


def mc_save(job, path: str):
    _check(lib().mc_save(job, os.fsencode(path)))


def mc_load(path: str):
    h = _vp()
    _check(lib().mc_load(os.fsencode(path), ctypes.byref(h)))
    return h


def mc_set_join_policy(job, scan_max_samples: int = -1, passes_before_scan: int = 2,
                       passes_without_scan: int = 10):
    _check(lib().mc_set_join_policy(job, scan_max_samples, passes_before_scan, passes_without_scan))


def mc_set_round_record(job, max_samples: int):
    _check(lib().mc_set_round_record(job, int(max_samples)))


def mc_set_partial_record(job, max_entries: int):
    _check(lib().mc_set_partial_record(job, int(max_entries)))


def mc_set_segment_samples(job, samples: int):
    _check(lib().mc_set_segment_samples(job, int(samples)))


def mc_set_join_order(job, mode: int):
    _check(lib().mc_set_join_order(job, int(mode)))


def mc_get_order(job, out: np.ndarray):
    assert out.dtype == np.int32 and out.flags.c_contiguous
    _check(lib().mc_get_order(job, _ptr(out), out.size))
    return out


def mc_thermo(job, betas) -> np.ndarray:
    b = np.ascontiguousarray(betas, dtype=np.float64).reshape(-1)
    out = np.zeros((b.size, 4), np.float64)
    _check(lib().mc_thermo(job, _ptr(b), b.size, _ptr(out)))
    return out


def mc_get_join(job, k: np.ndarray | None, offsets: np.ndarray | None, n: int):
    _check(lib().mc_get_join(job, _ptr(k) if k is not None else None,
                             _ptr(offsets) if offsets is not None else None, n))


def mc_get_info(job) -> mc_info:
    info = mc_info()
    _check(lib().mc_get_info(job, ctypes.byref(info)))
    return info


def mc_set_launch_shape(job, placement: int, chains_per_warp: int, warps_per_block: int):
    _check(lib().mc_set_launch_shape(job, placement, chains_per_warp, warps_per_block))


def mc_autotune(job, probe_sweeps: int, use_cache: bool = True):
    pl, c, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mc_autotune(job, probe_sweeps, 1 if use_cache else 0, ctypes.byref(pl),
                             ctypes.byref(c), ctypes.byref(w)))
    return int(pl.value), int(c.value), int(w.value)


def mc_batch_run(jobs, iterations: int, n_sweeps: int, mode: int):
    """jobs: list of handles (or Job objects)."""
    hs = [j.h if isinstance(j, Job) else j for j in jobs]
    arr = (_vp * len(hs))(*[h.value if isinstance(h, _vp) else h for h in hs])
    _check(lib().mc_batch_run(arr, len(hs), iterations, n_sweeps, mode))


def _handles(jobs):
    hs = [j.h if isinstance(j, Job) else j for j in jobs]
    return (_vp * len(hs))(*[h.value if isinstance(h, _vp) else h for h in hs]), len(hs)


def mc_batch_autotune(jobs, probe_sweeps: int, use_cache: bool = True):
    arr, n = _handles(jobs)
    _check(lib().mc_batch_autotune(arr, n, probe_sweeps, 1 if use_cache else 0))


def mc_batch_shape(job):
    # (placement, chains per warp, warps per block, has a fused form) of a job in a fused launch
    pl, c, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = lib().mc_batch_shape(job.h if isinstance(job, Job) else job, ctypes.byref(pl), ctypes.byref(c),
                              ctypes.byref(w))
    if rc < 0:
        _check(rc)
    return int(pl.value), int(c.value), int(w.value), bool(rc)


def mc_sync(job):
    _check(lib().mc_sync(job))


def mc_generate_noalloc(L: int, n_chains: int, seed: int, t0: int, n_sweeps: int, d_spins: int,
                        d_levels: int, d_weights: int, d_hist: int, stream: int | None = None):
    """Device pointers (ints) in, nothing allocated; see include/mc.h."""
    _check(lib().mc_generate_noalloc(L, n_chains, seed, t0, n_sweeps, _vp(d_spins), _vp(d_levels),
                                     _vp(d_weights), _vp(d_hist), _vp(stream or 0)))


def mc_last_error() -> str:
    return lib().mc_last_error().decode(errors="replace")


def mc_kernel_launches() -> int:
    return int(lib().mc_kernel_launches())


def mc_inject_alloc_failure(after: int):
    _check(lib().mc_inject_alloc_failure(int(after)))


def mc_live_allocations() -> int:
    return int(lib().mc_live_allocations())


# ------------------------------------------------------------ convenience
class Job:
    """One weight-estimation job (numpy in, numpy out)."""

    def __init__(self, L: int, n_chains: int, seed: int, start: int = 1):
        self.L, self.p, self.seed = L, n_chains, seed
        self.N = L * L
        self.wd = (L + 31) // 32
        self.h = mc_init(L, n_chains, seed, start)

    def close(self):
        if getattr(self, "h", None):
            mc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_trace(self, on=True):
        mc_set_trace(self.h, on)

    def set_stream(self, handle):
        mc_set_stream(self.h, handle)

    def set_launch_shape(self, placement, cpw, wpb):
        mc_set_launch_shape(self.h, placement, cpw, wpb)

    def autotune(self, probe_sweeps: int, use_cache: bool = True):
        return mc_autotune(self.h, probe_sweeps, use_cache)

    def run_sweeps(self, S: int):
        mc_run_sweeps(self.h, S)

    def join(self, want_length=True):
        return mc_join(self.h, want_length)

    def join_naive(self, want_length=True):
        return mc_join_naive(self.h, want_length)

    def update_weights(self):
        mc_update_weights(self.h)

    @property
    def hist(self):
        return mc_histogram(self.h, np.zeros(self.N + 1, np.int64))

    @property
    def weights(self):
        return mc_get_weights(self.h, np.zeros(self.N + 1, np.float64))

    @weights.setter
    def weights(self, w):
        mc_set_weights(self.h, w)

    @property
    def table(self):
        """Thresholds as [m][a] (a = aligned neighbours)."""
        t = mc_get_table(self.h, np.zeros(5 * (self.N + 1), np.uint32))
        return t.reshape(5, self.N + 1).T.copy()

    @property
    def spin_words(self):
        return mc_get_spins(self.h, np.zeros(self.p * self.L * self.wd, np.uint32)).reshape(
            self.p, self.L, self.wd)

    @spin_words.setter
    def spin_words(self, w):
        mc_set_spins(self.h, np.asarray(w, np.uint32).reshape(-1))

    @property
    def energies(self):
        return mc_get_energies(self.h, np.zeros(self.p, np.int32))

    @property
    def trace(self):
        S = self.info()["last_sweeps"]
        return mc_get_trace(self.h, np.zeros(S * self.p, np.int32)).reshape(S, self.p)

    @property
    def visited(self):
        return mc_get_visited(self.h, np.zeros(self.N + 1, np.uint8))

    @visited.setter
    def visited(self, v):
        mc_set_visited(self.h, v)

    def iteration(self, n_sweeps: int, m_total: int = 0, adapt: bool = False, max_rounds: int = 1_000_000):
        return mc_iteration(self.h, n_sweeps, m_total, adapt, max_rounds)

    def save(self, path: str):
        mc_save(self.h, path)

    @classmethod
    def load(cls, path: str) -> "Job":
        h = mc_load(path)
        job = cls.__new__(cls)
        job.h = h
        info = mc_info()
        _check(lib().mc_get_info(h, ctypes.byref(info)))
        job.L, job.p, job.seed = info.L, info.n_chains, info.seed
        job.N = job.L * job.L
        job.wd = (job.L + 31) // 32
        return job

    def run_attempts(self, n_attempts: int):
        mc_run_attempts(self.h, n_attempts)

    def set_join_policy(self, scan_max_samples: int = -1, passes_before_scan: int = 2,
                        passes_without_scan: int = 10):
        mc_set_join_policy(self.h, scan_max_samples, passes_before_scan, passes_without_scan)

    def set_join_order(self, mode: int):
        mc_set_join_order(self.h, mode)

    def set_segment_samples(self, samples: int):
        mc_set_segment_samples(self.h, samples)

    def set_partial_record(self, max_entries: int):
        mc_set_partial_record(self.h, max_entries)

    def set_round_record(self, max_samples: int):
        mc_set_round_record(self.h, max_samples)

    @property
    def order(self):
        return mc_get_order(self.h, np.zeros(self.p, np.int32))

    def thermo(self, betas):
        """E, C, F, S (columns) at each beta, from the current weight."""
        return mc_thermo(self.h, betas)

    def trace_chain(self, chain: int):
        S = self.info()["last_sweeps"]
        return mc_get_trace_chain(self.h, chain, np.zeros(S, np.int32))

    @property
    def k(self):
        k = np.zeros(self.p, np.int64)
        mc_get_join(self.h, k, None, self.p)
        return k

    @property
    def offsets(self):
        o = np.zeros(self.p, np.int64)
        mc_get_join(self.h, None, o, self.p)
        return o

    def info(self):
        return mc_get_info(self.h).as_dict()

    def sync(self):
        mc_sync(self.h)


# ------------------------------------------------------------ serving
def mc_job_device_bytes(L: int, n_chains: int, sweeps: int) -> int:
    return int(lib().mc_job_device_bytes(L, n_chains, sweeps))


def mc_server_create(budget_bytes: int, max_slots: int):
    h = _vp()
    _check(lib().mc_server_create(budget_bytes, max_slots, ctypes.byref(h)))
    return h


def mc_server_submit(srv, L: int, n_chains: int, seed: int, start: int, iterations: int, sweeps: int) -> int:
    spec = mc_jobspec(L, n_chains, seed, start, iterations, sweeps)
    jid = ctypes.c_uint64()
    _check(lib().mc_server_submit(srv, ctypes.byref(spec), ctypes.byref(jid)))
    return jid.value


def mc_server_poll(srv, jid: int) -> bool:
    done = ctypes.c_int()
    _check(lib().mc_server_poll(srv, jid, ctypes.byref(done)))
    return bool(done.value)


def mc_server_wait(srv, jid: int, n_levels: int | None):
    """Block until job jid is done; returns (W or None, stats dict).  Raises
    McError with the job's own status if it failed."""
    st = mc_jobstats()
    W = np.zeros(n_levels, np.float64) if n_levels else None
    rc = lib().mc_server_wait(srv, jid, _ptr(W) if W is not None else None, n_levels or 0, ctypes.byref(st))
    _check(rc)
    return W, st.as_dict()


def mc_server_get_info(srv) -> dict:
    info = mc_server_info()
    _check(lib().mc_server_get_info(srv, ctypes.byref(info)))
    return info.as_dict()


def mc_server_clock(srv) -> float:
    return float(lib().mc_server_clock(srv))


def mc_server_free(srv):
    lib().mc_server_free(srv)


class Server:
    """Continuous-batching server for weight-estimation jobs (numpy out)."""

    def __init__(self, budget_bytes: int, max_slots: int = 16):
        self.h = mc_server_create(budget_bytes, max_slots)
        self._levels = {}

    def submit(self, L: int, n_chains: int, seed: int, iterations: int, sweeps: int, start: int = 1) -> int:
        jid = mc_server_submit(self.h, L, n_chains, seed, start, iterations, sweeps)
        self._levels[jid] = L * L + 1
        return jid

    def poll(self, jid: int) -> bool:
        return mc_server_poll(self.h, jid)

    def wait(self, jid: int):
        return mc_server_wait(self.h, jid, self._levels.pop(jid))

    def clock(self) -> float:
        return mc_server_clock(self.h)

    def info(self) -> dict:
        return mc_server_get_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            mc_server_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
