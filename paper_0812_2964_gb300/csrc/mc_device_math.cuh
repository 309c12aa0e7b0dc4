// Device-side counter RNG and deterministic FP64 exp / log / threshold.
//
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11 -- 10 rounds, each two 32x32->64-bit multiplies (one
// mul.wide per multiply), the key bumped by the Weyl constants between rounds.
//
// exp/log: Cody-Waite argument reduction with a Taylor (exp) or atanh (log)
// series, every operation an explicitly rounded IEEE add/mul/div
// (__dadd_rn, __dmul_rn, ...), so no fused multiply-add can be formed and the
// results are reproducible bit for bit by any IEEE-754 double implementation
// that performs the same operations in the same order.  The acceptance test
// of the Metropolis method (Sec. 4.2) compares a 32-bit uniform with
// thr(d) = ceil(2^32 exp(d)) - 1 (0xFFFFFFFF for d >= 0, 0 for d <= -23).
#pragma once
#include <cstdint>

namespace mcgpu {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Counter words: [0..1] = 64-bit block index, [2] = chain, [3] = stream tag.
constexpr uint32_t kTagFlip = 0u;
constexpr uint32_t kTagJoint = 1u;
constexpr uint32_t kTagInit = 2u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint32_t uint4_word(const uint4 v, uint32_t w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------- FP64
// ln 2 truncated to 32 significant bits (n * kLn2Hi exact for |n| < 2^21),
// the remainder rounded to nearest, 1/ln 2 and sqrt(1/2) rounded to nearest.
constexpr double kLn2Hi = 0x1.62e42fefp-1;
constexpr double kLn2Lo = 0x1.473de6af278edp-34;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

// 2^k for integer k in the normal range, built from the exponent bits.
__device__ __forceinline__ double pow2i(int k) {
  return __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}

// 1/j! (j = 0..13) and 1/(2j+1) (j = 0..10), each the correctly rounded
// quotient of two exactly representable integers (folded at compile time).
__constant__ double kExpCoef[14] = {
    1.0 / 1.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0,
    1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0,
    1.0 / 479001600.0, 1.0 / 6227020800.0};
__constant__ double kLogCoef[11] = {
    1.0 / 1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0, 1.0 / 11.0,
    1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0};

// exp(d) for |d| <= 700: n = rint(d / ln2), r = (d - n ln2_hi) - n ln2_lo,
// exp(r) = sum_{j=0..13} r^j / j! by Horner, exp(d) = exp(r) 2^n.
__device__ __forceinline__ double exp_det(double d) {
  const double n = rint(__dmul_rn(d, kInvLn2));
  const double r = __dsub_rn(__dsub_rn(d, __dmul_rn(n, kLn2Hi)), __dmul_rn(n, kLn2Lo));
  double poly = kExpCoef[13];
#pragma unroll
  for (int j = 12; j >= 0; --j) poly = __dadd_rn(__dmul_rn(poly, r), kExpCoef[j]);
  const int ni = static_cast<int>(n);
  // scale by 2^n in two exact steps so that each power of two stays normal
  const int n1 = ni / 2, n2 = ni - n1;
  return __dmul_rn(__dmul_rn(poly, pow2i(n1)), pow2i(n2));
}

// ln(x) for finite x >= 1: x = f 2^e with f in [sqrt(1/2), sqrt(2)),
// s = (f-1)/(f+1), ln f = 2 s sum_{j=0..10} s^(2j)/(2j+1) by Horner in s^2,
// ln x = e ln2_hi + (e ln2_lo + ln f).
__device__ __forceinline__ double log_det(double x) {
  const long long bits = __double_as_longlong(x);
  int e = static_cast<int>((bits >> 52) & 0x7FF) - 1022;           // x = f 2^e, f in [1/2, 1)
  double f = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FE0000000000000LL);
  if (f < kSqrtHalf) {
    f = __dmul_rn(f, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
  const double z = __dmul_rn(s, s);
  double q = kLogCoef[10];
#pragma unroll
  for (int j = 9; j >= 0; --j) q = __dadd_rn(__dmul_rn(q, z), kLogCoef[j]);
  const double series = __dmul_rn(__dmul_rn(2.0, s), q);
  const double ed = static_cast<double>(e);
  return __dadd_rn(__dmul_rn(ed, kLn2Hi), __dadd_rn(__dmul_rn(ed, kLn2Lo), series));
}

// Threshold of the Metropolis test for a log-weight change d: a uniform u
// is accepted iff u <= thr(d).  P(accept) = (thr + 1) / 2^32.
__device__ __forceinline__ uint32_t threshold_det(double d) {
  if (d >= 0.0) return 0xFFFFFFFFu;
  if (d <= -23.0) return 0u;
  const double x = __dmul_rn(exp_det(d), 4294967296.0);   // exact scaling by 2^32
  if (x <= 1.0) return 0u;
  return static_cast<uint32_t>(__dsub_rn(ceil(x), 1.0));
}

}  // namespace mcgpu
