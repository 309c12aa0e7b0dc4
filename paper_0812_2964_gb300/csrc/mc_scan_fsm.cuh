// The exact scan of the joint (Sec. 2 steps 3-5, in chain order) as a state
// machine over joint positions.
//
// The serial rule passes to chain q the last level of the nearest earlier
// chain that kept samples (else the carry of the previous round; with
// neither, chain q is kept whole).  Most of the time that chain is one of the
// few just before q, so the state entering position q is d = how many
// positions back the input came from: 0 no input yet, 1..kScanCand the chain
// d positions back (position -1 is the carry), kFar further back, kStop an
// answer that the per-level summary cannot give.  Each position's answers
// under the kScanCand nearest inputs (one byte each, see below) define its
// transition function; transition functions compose associatively, so a
// block-wide prefix scan gives every position's entering state at once.
#pragma once
#include <cstdint>

namespace mcgpu {

constexpr int kScanCand = 8;
constexpr int kFar = kScanCand + 1, kStop = kScanCand + 2, kStates = kScanCand + 3;

// Answer codes, one byte per (position, d): 0 keeps nothing, 1 keeps
// samples, 2 undecidable (the scan stops there), 3 no such input, 4 / 5 as
// 0 / 1 but k is already known for this input (nothing to write).
constexpr int kAnsNo = 0, kAnsYes = 1, kAnsUndecided = 2, kAnsNone = 3, kAnsKnownNo = 4, kAnsKnownYes = 5;

// A transition function: the next state of every state, in 4-bit fields.
using Trans = unsigned long long;
static_assert(kScanCand == 8 && kStates <= 16, "answer codes in one 64-bit word, states in 4 bits");

__device__ __forceinline__ int tr_at(Trans T, int s) { return static_cast<int>((T >> (4 * s)) & 15u); }

__device__ __forceinline__ Trans tr_identity() {
  Trans r = 0;
#pragma unroll
  for (int s = 0; s < kStates; ++s) r |= static_cast<Trans>(s) << (4 * s);
  return r;
}

// B after A
__device__ __forceinline__ Trans tr_then(Trans A, Trans B) {
  Trans r = 0;
#pragma unroll
  for (int s = 0; s < kStates; ++s) r |= static_cast<Trans>(tr_at(B, tr_at(A, s))) << (4 * s);
  return r;
}

// The transition of one position from its answer codes (byte d - 1 = the
// answer under the input d positions back): no input keeps the chain whole
// (next state 1); an input under which the chain keeps samples makes it the
// next one's input (1); one under which it keeps nothing passes the same
// input on, one position further back (kFar past kScanCand); an undecidable
// answer stops.  kFar and kStop are absorbing.
__device__ __forceinline__ Trans tr_position(unsigned long long codes) {
  Trans r = static_cast<Trans>(1) | (static_cast<Trans>(kFar) << (4 * kFar)) |
            (static_cast<Trans>(kStop) << (4 * kStop));
#pragma unroll
  for (int d = 1; d <= kScanCand; ++d) {
    const int c = static_cast<int>((codes >> (8 * (d - 1))) & 0xFFu);
    const int next = (c == kAnsYes || c == kAnsKnownYes) ? 1
                     : (c == kAnsNo || c == kAnsKnownNo) ? (d == kScanCand ? kFar : d + 1)
                                                        : kStop;
    r |= static_cast<Trans>(next) << (4 * d);
  }
  return r;
}

}  // namespace mcgpu
