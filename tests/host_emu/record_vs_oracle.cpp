// CPU check of the round record (compiled for the host): every chain swept
// with sweep_row and the generation hook in recording mode stores, at
// rec_index(c, k, M), the level of its sample k -- the layout the joint's
// recorded-round kernels read -- and the oracle's or_chain_round gives the
// same level for every sample.  37 chains make a full tile of 32 and a
// ragged one; the padding lanes' entries stay untouched, and no store falls
// outside rec_entries(p, M).
#include "mc_chain.cuh"
#include "mc_internal.h"
extern "C" {
#include "mc_oracle.h"
}
using namespace mcgpu;

template <int WD>
int run(int L, int p, int64_t S, uint64_t seed, const double* W) {
  const int N = L * L, np1 = N + 1;
  const int64_t M = S * N;
  std::vector<uint32_t> Tor(5 * np1), T(5 * np1);
  or_build_table(W, L, Tor.data());
  for (int m = 0; m < np1; ++m) for (int a = 0; a < 5; ++a) T[a * np1 + m] = Tor[m * 5 + a];
  const size_t n_rec = static_cast<size_t>(rec_entries(p, M));
  // one guard group past the end: a store there is an out-of-range write
  std::vector<uint16_t> rec(n_rec + 4, 0xFFFFu);
  int bad = 0;
  for (int c = 0; c < p; ++c) {
    std::vector<int8_t> s(N);
    or_init_lattice(s.data(), L, seed, c, 1);
    int m = (or_energy(s.data(), L) + 2 * N) / 4;
    const int m0 = m;
    std::vector<uint32_t> lat(L * WD, 0);
    for (int y = 0; y < L; ++y) for (int x = 0; x < L; ++x) if (s[y * L + x] > 0) lat[y * WD + x / 32] |= 1u << (x % 32);
    std::vector<uint32_t> hist(np1 + 3, 0u);
    GenHook<WD == 1 ? 32 : 8, true> hk;
    hk.init(hist.data(), 1u, np1);
    hk.rec = rec.data() + rec_index(c, 0, M);
    hk.rec_on = true;
    Prefetch pf;
    prefetch_init<WD>(pf, L, 0, (uint32_t)c, (uint32_t)seed, (uint32_t)(seed >> 32));
    for (int64_t sw = 0; sw < S; ++sw)
      for (int y = 0; y < L; ++y) {
        const int ym = (y + L - 1) % L, yp = (y + 1) % L;
        uint32_t cur[WD], up[WD], dn[WD];
        for (int w = 0; w < WD; ++w) { cur[w] = lat[y * WD + w]; up[w] = lat[ym * WD + w]; dn[w] = lat[yp * WD + w]; }
        sweep_row<WD>(cur, up, dn, L, m, T.data(), np1, pf, (uint32_t)c, (uint32_t)seed, (uint32_t)(seed >> 32), hk);
        for (int w = 0; w < WD; ++w) lat[y * WD + w] = cur[w];
      }
    std::vector<int32_t> samples(M);
    int32_t mo = m0;
    or_chain_round(L, seed, c, 0, S, Tor.data(), s.data(), &mo, nullptr, nullptr, samples.data());
    int64_t diff = 0;
    for (int64_t k = 0; k < M; ++k) diff += rec[rec_index(c, k, M)] != static_cast<uint16_t>(samples[k]);
    if (diff || mo != m) {
      ++bad;
      if (bad < 3) printf("L=%d chain %d: %lld samples differ (level %d vs %d)\n", L, c, (long long)diff, m, mo);
    }
  }
  // padding lanes of the last tile and the guard group: never written
  int64_t touched = 0;
  for (int c = p; c < (p + kRecTile - 1) / kRecTile * kRecTile; ++c)
    for (int64_t k = 0; k < M; ++k) touched += rec[rec_index(c, k, M)] != 0xFFFFu;
  for (size_t q = n_rec; q < rec.size(); ++q) touched += rec[q] != 0xFFFFu;
  if (touched) {
    ++bad;
    printf("L=%d: %lld entries outside the chains' samples written\n", L, (long long)touched);
  }
  return bad;
}

int main() {
  int total_bad = 0;
  const int Ls[] = {8, 16, 32, 36, 64, 100};
  for (int L : Ls) {
    const int N = L * L;
    std::vector<double> W(N + 1);
    srand(7 * L);
    for (int i = 0; i <= N; ++i) W[i] = 3.0 * ((double)rand() / RAND_MAX - 0.5) + 2.0 * sin(i * 0.013);
    const int64_t S = L <= 36 ? 2 : 1;
    const int wd = (L + 31) / 32;
    const uint64_t seed = 0xABCDEF12345ull + L;
    int bad;
    if (wd == 1) bad = run<1>(L, 37, S, seed, W.data());
    else if (wd == 2) bad = run<2>(L, 37, S, seed, W.data());
    else bad = run<4>(L, 37, S, seed, W.data());
    printf("L=%d record: %s\n", L, bad ? "FAIL" : "ok");
    total_bad += bad;
  }
  return total_bad ? 1 : 0;
}
