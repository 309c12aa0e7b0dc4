"""Pins for the oracle's primitives: Philox4x32-10, deterministic exp/log and
the Metropolis threshold.  None of these is checked against the oracle
itself: Philox against NVIDIA cuRAND's host generator (an independent
implementation, run on the CPU), exp/log/threshold against mpmath at 40+
digits, the constants against exact rational arithmetic.
"""
import ctypes
import ctypes.util
import math
import os
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

import oracle


# ------------------------------------------------------------------ Philox
def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


def _curand_stream(seed: int, n: int, offset: int = 0) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return buf


# cuRAND's host Philox4_32_10 generator emits 4-word block b of its stream as
# Philox(counter = (b // 65536 (64-bit, split lo/hi), b % 65536, 0),
#        key = (lo32(seed), hi32(seed))).
CURAND_LANES = 65536


def _curand_block_counter(b: int):
    q = b // CURAND_LANES
    return (q & 0xFFFFFFFF, q >> 32, b % CURAND_LANES, 0)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand(seed):
    nblocks = CURAND_LANES + 64
    out = _curand_stream(seed, 4 * nblocks).reshape(-1, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = list(range(0, 300)) + list(range(CURAND_LANES - 5, nblocks)) + \
        list(rng.integers(0, nblocks, 300))
    for b in picks:
        assert oracle.philox(_curand_block_counter(int(b)), key) == [int(v) for v in out[b]], b


def test_philox_high_counter_word_matches_curand():
    # an offset of 2^50 words puts 2^32 into the counter's first two words
    seed = 0xDEADBEEFCAFEF00D
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for offset in (1 << 50, (1 << 50) + (5 << 18) * 4 + 12, (1 << 62)):
        out = _curand_stream(seed, 16, offset).reshape(-1, 4)
        for j in range(4):
            b = offset // 4 + j
            assert oracle.philox(_curand_block_counter(b), key) == [int(v) for v in out[j]]


def test_philox_tag_word_changes_output():
    key = (5, 6)
    outs = {tuple(oracle.philox((7, 0, 9, tag), key)) for tag in range(4)}
    assert len(outs) == 4


# ------------------------------------------------------------------ constants
def _nearest(fr: Fraction) -> float:
    return float(fr)   # Fraction -> float rounds to nearest


def test_constants_exact_definitions():
    with mp.workdps(80):
        ln2 = Fraction(mp.nstr(mp.log(2), 75))
        inv = Fraction(mp.nstr(1 / mp.log(2), 75))
        sqh = Fraction(mp.nstr(mp.sqrt(mp.mpf(1) / 2), 75))
    LN2_HI, LN2_LO, INV_LN2, SQRT_HALF = (oracle.const(i) for i in range(4))
    # LN2_HI: ln 2 truncated to 32 significant bits
    assert Fraction(LN2_HI) == Fraction(math.floor(ln2 * 2**33), 2**33)
    assert LN2_LO == _nearest(ln2 - Fraction(LN2_HI))
    assert INV_LN2 == _nearest(inv)
    assert SQRT_HALF == _nearest(sqh)
    for j in range(14):
        assert oracle.const(100 + j) == _nearest(Fraction(1, math.factorial(j)))
    for j in range(11):
        assert oracle.const(200 + j) == _nearest(Fraction(1, 2 * j + 1))


# ------------------------------------------------------------------ exp / log
def _ulps(got: float, exact) -> float:
    return float(abs(mp.mpf(got) - exact) / mp.mpf(math.ulp(float(exact))))


def test_exp_det_within_two_ulp():
    rng = np.random.default_rng(1)
    ds = np.concatenate([rng.uniform(-23, 0, 6000), rng.uniform(-700, 700, 1500),
                         -np.logspace(-14, 1.36, 800), [-23.0, -22.18, -1e-300, 0.0]])
    with mp.workdps(40):
        worst = max(_ulps(oracle.exp_det(float(d)), mp.exp(mp.mpf(float(d)))) for d in ds)
    assert worst <= 2.0, worst


def test_log_det_within_one_ulp():
    rng = np.random.default_rng(2)
    xs = np.concatenate([np.arange(2, 5001), rng.integers(2, 2**53, 3000).astype(float),
                         2.0 ** np.arange(1, 63)])
    assert oracle.log_det(1.0) == 0.0
    with mp.workdps(40):
        worst = max(_ulps(oracle.log_det(float(x)), mp.log(mp.mpf(float(x)))) for x in xs)
    assert worst <= 1.0, worst


# ------------------------------------------------------------------ threshold
def _thr_exact(d: float):
    """ceil(2^32 exp(d)) - 1 exactly, and the distance of 2^32 exp(d) to the
    nearest integer."""
    with mp.workdps(60):
        x = mp.ldexp(mp.exp(mp.mpf(d)), 32)
        c = int(mp.ceil(x))
        dist = float(min(x - mp.floor(x), mp.ceil(x) - x))
        return c - 1, dist


def test_threshold_special_values():
    assert oracle.threshold(0.0) == 0xFFFFFFFF
    assert oracle.threshold(-0.0) == 0xFFFFFFFF
    assert oracle.threshold(3.5) == 0xFFFFFFFF
    assert oracle.threshold(-23.0) == 0
    assert oracle.threshold(-500.0) == 0
    assert oracle.threshold(-22.2) == 0          # 2^32 e^-22.2 < 1


def test_threshold_is_ceil_of_scaled_exp():
    rng = np.random.default_rng(3)
    ds = np.concatenate([rng.uniform(-23, 0, 4000), -np.logspace(-10, 0, 300),
                         -rng.uniform(0, 1e-6, 200)])
    for d in ds:
        d = float(d)
        T = oracle.threshold(d)
        Te, dist = _thr_exact(d)
        Te = min(Te, 0xFFFFFFFF)
        # exp_det is within 2 ulp (< 2^-51 relative), so only values of
        # 2^32 exp(d) within 2^-19 of an integer can round across it
        if dist > 2.0 ** -19:
            assert T == max(Te, 0), (d, T, Te)
        else:
            assert abs(T - Te) <= 1


def test_threshold_acceptance_probability_bound():
    # P(u <= T) = (T+1)/2^32 must be within 2^-32 of min(1, e^d)
    rng = np.random.default_rng(4)
    for d in np.concatenate([rng.uniform(-30, 2, 3000), [-22.18, -22.17, -1e-12]]):
        d = float(d)
        p_acc = (oracle.threshold(d) + 1) / 2.0**32
        with mp.workdps(40):
            p = min(mp.mpf(1), mp.exp(mp.mpf(d)))
            assert abs(mp.mpf(p_acc) - p) <= mp.mpf(2) ** -32 * (1 + 1e-9)


def test_threshold_monotone():
    ds = np.sort(np.random.default_rng(5).uniform(-24, 1, 5000))
    T = [oracle.threshold(float(d)) for d in ds]
    assert all(a <= b for a, b in zip(T, T[1:]))
