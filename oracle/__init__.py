"""Plain sequential CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The GPU library never imports
it and shares no code with it.

The arithmetic lives in ``mc_oracle.c`` (plain C, built with gcc
``-ffp-contract=off``); this module only compiles it and marshals arguments
through ctypes.  Paper sections followed: Sec. 2 (the algorithm, steps 1-6),
Sec. 3.1 (Eq. new_weight), Sec. 4.1 (the Hamiltonian), Sec. 4.2 (weights kept
as logarithms; Metropolis test at the joints).

``MC_ORACLE_LIB`` names a prebuilt library to load instead of compiling
``mc_oracle.c``; only the mutation test sets it, to run the pins against
deliberately broken builds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library to load instead (nothing is compiled then): the
# mutation test uses it to run the pins against deliberately broken builds.
_LIB_OVERRIDE = os.environ.get("MC_ORACLE_LIB", "")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-pthread"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (gcc; x86_64 or aarch64)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "mc_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                L = ctypes.CDLL(_LIB_OVERRIDE)
            else:
                build()
                L = ctypes.CDLL(_LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _declare(L):
    c = ctypes
    sig = {
        "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "or_exp_det": (c.c_double, [c.c_double]),
        "or_log_det": (c.c_double, [c.c_double]),
        "or_threshold": (c.c_uint32, [c.c_double]),
        "or_const": (c.c_double, [c.c_int]),
        "or_energy": (c.c_int, [_i8p, c.c_int]),
        "or_init_lattice": (None, [_i8p, c.c_int, c.c_uint64, c.c_uint32, c.c_int]),
        "or_build_table": (None, [_dp, c.c_int, _u32p]),
        "or_chain_round": (c.c_int, [c.c_int, c.c_uint64, c.c_uint32, c.c_uint64, c.c_int64,
                                     _u32p, _i8p, _i32p, _i32p, _i64p, _i32p]),
        "or_chain_first_accept": (c.c_int64, [c.c_int, c.c_uint64, c.c_uint32, c.c_uint64,
                                              c.c_int64, _u32p, _dp, _i8p, c.c_int32,
                                              c.c_int32, c.c_uint32, _i64p]),
        "or_joint_scan": (c.c_int64, [_i32p, c.c_int64, _dp, c.c_int32, c.c_uint64,
                                      c.c_uint32, c.c_uint32]),
        "or_create": (c.c_void_p, [c.c_int, c.c_int, c.c_uint64, c.c_int]),
        "or_free": (None, [c.c_void_p]),
        "or_run_round": (c.c_int, [c.c_void_p, c.c_int64, c.c_int]),
        "or_run_attempts": (c.c_int, [c.c_void_p, c.c_int64, c.c_int]),
        "or_get_last_M": (c.c_int64, [c.c_void_p]),
        "or_join": (c.c_int64, [c.c_void_p]),
        "or_join_naive": (c.c_int64, [c.c_void_p]),
        "or_update_weights": (None, [c.c_void_p]),
        "or_iteration": (c.c_int64, [c.c_void_p, c.c_int64, c.c_int64, c.c_int]),
        "or_iteration_adaptive": (c.c_int64, [c.c_void_p, c.c_int64, c.c_int64, c.c_int, c.c_int,
                                              c.POINTER(c.c_int), _i64p]),
        "or_get_weights": (None, [c.c_void_p, _dp]),
        "or_set_weights": (None, [c.c_void_p, _dp]),
        "or_get_table": (None, [c.c_void_p, _u32p]),
        "or_get_hist": (None, [c.c_void_p, _i64p]),
        "or_get_spins": (None, [c.c_void_p, _i8p]),
        "or_get_levels": (None, [c.c_void_p, _i32p]),
        "or_get_trace": (None, [c.c_void_p, _i32p]),
        "or_get_k": (None, [c.c_void_p, _i64p]),
        "or_get_carry": (c.c_int32, [c.c_void_p, c.POINTER(c.c_int)]),
        "or_get_t": (c.c_uint64, [c.c_void_p]),
        "or_get_round": (c.c_uint32, [c.c_void_p]),
        "or_get_last_S": (c.c_int64, [c.c_void_p]),
        "or_get_samples": (None, [c.c_void_p, _i32p]),
        "or_set_samples": (c.c_int, [c.c_void_p, c.c_int64, _i32p]),
        "or_get_visited": (None, [c.c_void_p, _u8p]),
        "or_set_join_order": (None, [c.c_void_p, c.c_int]),
        "or_get_order": (None, [c.c_void_p, _i32p]),
        "or_thermo": (None, [c.c_int, _dp, _u8p, _dp, c.c_int, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def exp_det(d: float) -> float:
    return lib().or_exp_det(float(d))


def log_det(x: float) -> float:
    return lib().or_log_det(float(x))


def threshold(d: float) -> int:
    return int(lib().or_threshold(float(d)))


def const(which: int) -> float:
    return lib().or_const(int(which))


def energy(spins: np.ndarray) -> int:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    L = s.shape[-1]
    return int(lib().or_energy(_p(s, _i8p), L))


def init_lattice(L: int, seed: int, chain: int, start: int) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    lib().or_init_lattice(_p(s, _i8p), L, seed, chain, start)
    return s


def build_table(W: np.ndarray, L: int) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    T = np.zeros((L * L + 1) * 5, dtype=np.uint32)
    lib().or_build_table(_p(W, _dp), L, _p(T, _u32p))
    return T.reshape(L * L + 1, 5)


def level(E: int, L: int) -> int:
    return (E + 2 * L * L) // 4


def chain_round(L, seed, chain, t0, S, W, spins, m, want_samples=False, want_trace=True):
    """One chain, one round (streaming).  Returns (spins, m, trace, hist, samples)."""
    N = L * L
    T = np.ascontiguousarray(build_table(W, L).reshape(-1))
    s = np.array(spins, dtype=np.int8, copy=True).reshape(L, L)
    mm = ctypes.c_int32(int(m))
    trace = np.zeros(S, dtype=np.int32) if want_trace else None
    hist = np.zeros(N + 1, dtype=np.int64)
    samples = np.zeros(S * N, dtype=np.int32) if want_samples else None
    lib().or_chain_round(L, seed, chain, t0, S, _p(T, _u32p), _p(s, _i8p), ctypes.byref(mm),
                         _p(trace, _i32p), _p(hist, _i64p), _p(samples, _i32p))
    return s, int(mm.value), trace, hist, samples


def chain_first_accept(L, seed, chain, t0, S, W, spins_start, m_start, x_level, r,
                       want_prefix_hist=False):
    N = L * L
    W = np.ascontiguousarray(W, dtype=np.float64)
    T = np.ascontiguousarray(build_table(W, L).reshape(-1))
    s = np.ascontiguousarray(spins_start, dtype=np.int8).reshape(L, L)
    ph = np.zeros(N + 1, dtype=np.int64) if want_prefix_hist else None
    k = lib().or_chain_first_accept(L, seed, chain, t0, S, _p(T, _u32p), _p(W, _dp), _p(s, _i8p),
                                    int(m_start), int(x_level), r, _p(ph, _i64p))
    return (int(k), ph) if want_prefix_hist else int(k)


def joint_scan(levels, W, x_level, seed, r, i):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    W = np.ascontiguousarray(W, dtype=np.float64)
    return int(lib().or_joint_scan(_p(lv, _i32p), lv.size, _p(W, _dp), int(x_level), seed, r, i))


def thermo(L, W, visited, betas):
    """E, C, F, S at each beta (columns), from ln-weights W over the visited
    levels (Eq. reweighting2).  Returns an array [len(betas)][4]."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    v = np.ascontiguousarray(visited, dtype=np.uint8)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    assert W.size == v.size == L * L + 1
    out = np.zeros((b.size, 4), dtype=np.float64)
    lib().or_thermo(L, _p(W, _dp), _p(v, _u8p), _p(b, _dp), b.size, _p(out, _dp))
    return out


# ---------------------------------------------------------------- a whole job
class Job:
    """A multicanonical weight-estimation job run by the oracle."""

    def __init__(self, L: int, p: int, seed: int, start: int = 1):
        self.L, self.p, self.seed = L, p, seed
        self.N = L * L
        self._h = lib().or_create(L, p, seed, start)
        if not self._h:
            raise ValueError(f"oracle rejects L={L} p={p}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_free(h)
            self._h = None

    def run_round(self, S: int, nthreads: int = 1):
        rc = lib().or_run_round(self._h, S, nthreads)
        if rc != 0:
            raise MemoryError("oracle round failed")

    def run_attempts(self, n: int, nthreads: int = 1):
        if lib().or_run_attempts(self._h, n, nthreads) != 0:
            raise MemoryError

    def join(self) -> int:
        return int(lib().or_join(self._h))

    def join_naive(self) -> int:
        return int(lib().or_join_naive(self._h))

    def update_weights(self):
        lib().or_update_weights(self._h)

    def iteration(self, S: int, M_total: int = 0, nthreads: int = 1) -> int:
        return int(lib().or_iteration(self._h, S, M_total, nthreads))

    def iteration_adaptive(self, S: int, M_total: int, nthreads: int = 1, max_rounds: int = 1000):
        """Returns (joined, [sweeps of each round])."""
        rounds = ctypes.c_int(0)
        sw = np.zeros(max_rounds, dtype=np.int64)
        joined = int(lib().or_iteration_adaptive(self._h, S, M_total, nthreads, max_rounds,
                                                   ctypes.byref(rounds), _p(sw, _i64p)))
        return joined, [int(x) for x in sw[:rounds.value]]

    @property
    def weights(self):
        W = np.zeros(self.N + 1, dtype=np.float64)
        lib().or_get_weights(self._h, _p(W, _dp))
        return W

    @weights.setter
    def weights(self, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.size == self.N + 1
        lib().or_set_weights(self._h, _p(W, _dp))

    @property
    def table(self):
        T = np.zeros((self.N + 1) * 5, dtype=np.uint32)
        lib().or_get_table(self._h, _p(T, _u32p))
        return T.reshape(self.N + 1, 5)

    @property
    def hist(self):
        h = np.zeros(self.N + 1, dtype=np.int64)
        lib().or_get_hist(self._h, _p(h, _i64p))
        return h

    @property
    def spins(self):
        s = np.zeros((self.p, self.L, self.L), dtype=np.int8)
        lib().or_get_spins(self._h, _p(s, _i8p))
        return s

    @property
    def levels(self):
        m = np.zeros(self.p, dtype=np.int32)
        lib().or_get_levels(self._h, _p(m, _i32p))
        return m

    @property
    def trace(self):
        S = int(lib().or_get_last_S(self._h))
        tr = np.zeros((S, self.p), dtype=np.int32)
        if S:
            lib().or_get_trace(self._h, _p(tr, _i32p))
        return tr

    @property
    def k(self):
        k = np.zeros(self.p, dtype=np.int64)
        lib().or_get_k(self._h, _p(k, _i64p))
        return k

    @property
    def carry(self):
        v = ctypes.c_int(0)
        c = lib().or_get_carry(self._h, ctypes.byref(v))
        return (int(c) if v.value else None)

    @property
    def t(self):
        return int(lib().or_get_t(self._h))

    def set_join_order(self, mode: int):
        lib().or_set_join_order(self._h, int(mode))

    @property
    def order(self):
        out = np.zeros(self.p, dtype=np.int32)
        lib().or_get_order(self._h, _p(out, _i32p))
        return out

    @property
    def visited(self):
        out = np.zeros(self.N + 1, dtype=np.uint8)
        lib().or_get_visited(self._h, _p(out, _u8p))
        return out

    @property
    def round(self):
        return int(lib().or_get_round(self._h))

    def set_samples(self, S: int, samples):
        sm = np.ascontiguousarray(samples, dtype=np.int32)
        assert sm.size == self.p * S * self.N
        if lib().or_set_samples(self._h, S, _p(sm, _i32p)) != 0:
            raise MemoryError

    @property
    def samples(self):
        M = int(lib().or_get_last_M(self._h))
        out = np.zeros((self.p, M), dtype=np.int32)
        lib().or_get_samples(self._h, _p(out, _i32p))
        return out


def pack_spins(spins: np.ndarray) -> np.ndarray:
    """Bit-pack int8 +-1 lattices [..., L, L] into the row-word layout
    [..., L, ceil(L/32)] uint32 (bit x%32 of word x//32 of row y is site (x, y),
    1 meaning +1).  Layout conversion only."""
    s = np.asarray(spins)
    L = s.shape[-1]
    Wd = (L + 31) // 32
    bits = (s > 0).astype(np.uint64)
    out = np.zeros(s.shape[:-1] + (Wd,), dtype=np.uint64)
    for x in range(L):
        out[..., x // 32] |= bits[..., x] << np.uint64(x % 32)
    return out.astype(np.uint32)


def unpack_spins(words: np.ndarray, L: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32)
    out = np.zeros(w.shape[:-1] + (L,), dtype=np.int8)
    for x in range(L):
        b = (w[..., x // 32] >> np.uint32(x % 32)) & np.uint32(1)
        out[..., x] = np.where(b == 1, 1, -1)
    return out
