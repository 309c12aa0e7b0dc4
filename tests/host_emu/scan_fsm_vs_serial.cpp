// CPU check of the exact scan's state machine (mc_scan_fsm.cuh, compiled for
// the host) against the serial rule of the joint that it replaces (Sec. 2
// steps 3-5): chain q takes the last level of the nearest earlier chain
// that kept samples, else the carry, else it is kept whole.
//
// Each trial draws, for every joint position q and every possible input
// source (position -1 = the carry, 0..q-1 a chain), whether chain q keeps
// samples under that input (yes / no / undecidable, plain or "already
// known").  The serial walk gives the input of every position; the state
// machine must give, at every position, the same source (state d = q - src),
// kFar exactly from the first position whose source lies more than
// kScanCand positions back, and kStop exactly after the first undecidable
// answer.  The block-wide prefix scan of scan_kernel (ranges per thread, a
// Hillis-Steele scan over the ranges' compositions) is replayed with the
// same functions and must give every range's entering state.  tr_then must
// be associative and tr_identity neutral.
#include <random>

#include "mc_scan_fsm.cuh"
using namespace mcgpu;

namespace {

constexpr int kNoSource = -2;   // no carry and no earlier chain kept samples

struct Trial {
  int P = 0, f = 0, last0 = kNoSource;
  std::vector<std::vector<uint8_t>> ans;   // ans[q][src + 1]
};

Trial draw(std::mt19937_64& g, int P, double p_yes, double p_und, double p_known) {
  Trial t;
  t.P = P;
  std::uniform_real_distribution<double> U(0.0, 1.0);
  t.f = static_cast<int>(g() % static_cast<uint64_t>(P));
  const int r = static_cast<int>(g() % 4);
  // the nearest earlier chain that kept samples: none, the carry, just
  // before f, or far before f
  t.last0 = r == 0 ? kNoSource : r == 1 ? -1 : r == 2 ? t.f - 1 : t.f - 1 - static_cast<int>(g() % 20);
  if (t.last0 < -1 && r != 0) t.last0 = -1;
  t.ans.resize(P);
  for (int q = 0; q < P; ++q) {
    t.ans[q].resize(q + 1);
    for (int s = 0; s <= q; ++s) {
      const double u = U(g);
      int a = u < p_und ? kAnsUndecided : (u < p_und + p_yes ? kAnsYes : kAnsNo);
      if (a != kAnsUndecided && U(g) < p_known) a = (a == kAnsYes) ? kAnsKnownYes : kAnsKnownNo;
      t.ans[q][s] = static_cast<uint8_t>(a);
    }
  }
  return t;
}

unsigned long long codes_of(const Trial& t, int q) {
  unsigned long long c = 0;
  for (int d = 1; d <= kScanCand; ++d) {
    const int src = q - d;
    const int a = src >= -1 ? t.ans[q][src + 1] : kAnsNone;
    c |= static_cast<unsigned long long>(a) << (8 * (d - 1));
  }
  return c;
}

// the state entering each position q = f..P (P: after the last), by the serial rule
std::vector<int> serial_states(const Trial& t) {
  std::vector<int> st(t.P + 1 - t.f);
  int last = t.last0;
  bool stopped = false, far = false;
  for (int q = t.f; q <= t.P; ++q) {
    int s;
    if (stopped) s = kStop;
    else if (far || (last != kNoSource && q - last > kScanCand)) { far = true; s = kFar; }
    else s = last == kNoSource ? 0 : q - last;
    st[q - t.f] = s;
    if (q == t.P || stopped || far) continue;
    if (last == kNoSource) { last = q; continue; }   // kept whole
    const int a = t.ans[q][last + 1];
    if (a == kAnsUndecided) stopped = true;
    else if (a == kAnsYes || a == kAnsKnownYes) last = q;
  }
  return st;
}

// the source the serial rule passes to chain q (for the kFar hand-over)
int serial_last_before(const Trial& t, int q_end) {
  int last = t.last0;
  for (int q = t.f; q < q_end; ++q) {
    if (last == kNoSource) { last = q; continue; }
    const int a = t.ans[q][last + 1];
    if (a == kAnsYes || a == kAnsKnownYes) last = q;
  }
  return last;
}

int entering_state(const Trial& t) {
  return t.last0 == kNoSource ? 0 : std::min(t.f - t.last0, kFar);
}

int fails = 0;
#define CHECK(c, ...)                 \
  do {                                \
    if (!(c)) {                       \
      if (fails < 20) printf(__VA_ARGS__); \
      ++fails;                        \
    }                                 \
  } while (0)

}  // namespace

int main() {
  std::mt19937_64 g(20240531);

  // algebra: identity and associativity on random transition functions
  std::uniform_int_distribution<int> S(0, kStates - 1);
  auto rnd = [&]() {
    Trans r = 0;
    for (int s = 0; s < kStates; ++s) r |= static_cast<Trans>(S(g)) << (4 * s);
    return r;
  };
  for (int i = 0; i < 20000; ++i) {
    const Trans A = rnd(), B = rnd(), C = rnd();
    CHECK(tr_then(tr_identity(), A) == A && tr_then(A, tr_identity()) == A, "identity\n");
    CHECK(tr_then(tr_then(A, B), C) == tr_then(A, tr_then(B, C)), "associativity\n");
    for (int s = 0; s < kStates; ++s) CHECK(tr_at(tr_then(A, B), s) == tr_at(B, tr_at(A, s)), "order\n");
  }
  printf("algebra: %s\n", fails ? "FAIL" : "ok");
  const int f0 = fails;

  // the serial rule, position by position and through the block scan
  const double regimes[][3] = {{0.9, 0.0, 0.2}, {0.5, 0.0, 0.2}, {0.1, 0.0, 0.3}, {0.02, 0.0, 0.3},
                               {0.3, 0.002, 0.2}, {0.05, 0.001, 0.5}, {0.6, 0.05, 0.0}};
  const int threads[] = {1, 3, 32, 1024};
  long far_seen = 0, stop_seen = 0, handovers = 0;
  for (int trial = 0; trial < 700; ++trial) {
    const auto& rg = regimes[trial % 7];
    const int P = 1 + static_cast<int>(g() % 600);
    const Trial t = draw(g, P, rg[0], rg[1], rg[2]);
    const std::vector<int> want = serial_states(t);
    // one position at a time
    int s = entering_state(t);
    CHECK(s == want[0], "trial %d: entering state %d, serial %d\n", trial, s, want[0]);
    for (int q = t.f; q < t.P; ++q) {
      const int prev = s;
      s = tr_at(tr_position(codes_of(t, q)), s);
      CHECK(s == want[q + 1 - t.f], "trial %d q %d: state %d, serial %d\n", trial, q + 1, s, want[q + 1 - t.f]);
      if (s == kFar && prev != kFar) {
        // the kernel hands over to one chain at a time with the input of the
        // chain kFar positions before the first position entered in kFar
        ++handovers;
        CHECK(serial_last_before(t, q + 1) == q + 1 - kFar, "trial %d: kFar hand-over at %d\n", trial, q + 1);
      }
    }
    far_seen += want.back() == kFar;
    stop_seen += want.back() == kStop;
    // the block scan: each thread composes a range, a Hillis-Steele scan
    // gives the inclusive prefixes, each range starts from the one before
    const int nt = threads[trial % 4], len = t.P - t.f, per = (len + nt - 1) / nt;
    std::vector<Trans> tr(nt);
    for (int th = 0; th < nt; ++th) {
      Trans agg = tr_identity();
      const int lo = std::min(t.P, t.f + th * per), hi = std::min(t.P, lo + per);
      for (int q = lo; q < hi; ++q) agg = tr_then(agg, tr_position(codes_of(t, q)));
      tr[th] = agg;
    }
    for (int off = 1; off < nt; off <<= 1) {
      std::vector<Trans> nx(tr);
      for (int th = off; th < nt; ++th) nx[th] = tr_then(tr[th - off], tr[th]);
      tr.swap(nx);
    }
    const int st0 = entering_state(t);
    for (int th = 0; th < nt; ++th) {
      const int lo = std::min(t.P, t.f + th * per);
      const int s_in = tr_at(th > 0 ? tr[th - 1] : tr_identity(), st0);
      CHECK(s_in == want[lo - t.f], "trial %d thread %d: range enters in %d, serial %d\n", trial, th, s_in,
            want[lo - t.f]);
    }
    CHECK(tr_at(tr[nt - 1], st0) == want.back(), "trial %d: final state\n", trial);
  }
  printf("serial rule: %s (%ld trials end in kFar, %ld in kStop, %ld kFar hand-overs)\n",
         fails == f0 ? "ok" : "FAIL", far_seen, stop_seen, handovers);
  if (far_seen == 0 || stop_seen == 0 || handovers == 0) {
    printf("coverage: FAIL\n");
    return 1;
  }
  return fails ? 1 : 0;
}
