// CPU check of the GPU row sweep (mc_chain.cuh, compiled for the host):
// every chain is swept with sweep_row and with the oracle's or_chain_round
// from the same start; lattices, levels, per-sweep levels and dwell-time
// histograms must agree exactly, and the level index must stay in [0, N].
// The joint's replay hooks are checked too: SearchHook finds the oracle's
// first accepted sample for an input level, and SummaryHook's per-level
// minimum uniforms decide acceptance exactly as that search does.

#include "mc_chain.cuh"
extern "C" {
#include "mc_oracle.h"
}
using namespace mcgpu;

// replay S sweeps of one chain from (lat, m) with a hook (early: stop after
// the row in which hk.done became true)
template <int WD, class Hook>
void replay(int L, int64_t S, std::vector<uint32_t> lat, int m, const uint32_t* T, int np1, uint64_t seed,
            uint32_t c, Hook& hk, bool early) {
  Prefetch pf;
  prefetch_init<WD>(pf, L, 0, c, (uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t sw = 0; sw < S; ++sw)
    for (int y = 0; y < L; ++y) {
      int ym = (y + L - 1) % L, yp = (y + 1) % L;
      uint32_t cur[WD], up[WD], dn[WD];
      for (int w = 0; w < WD; ++w) { cur[w] = lat[y * WD + w]; up[w] = lat[ym * WD + w]; dn[w] = lat[yp * WD + w]; }
      sweep_row<WD>(cur, up, dn, L, m, T, np1, pf, c, (uint32_t)seed, (uint32_t)(seed >> 32), hk);
      for (int w = 0; w < WD; ++w) lat[y * WD + w] = cur[w];
      if (early && hk.done) return;
    }
}

template <int WD>
int run(int L, int p, int64_t S, uint64_t seed, const double* W, int start) {
  const int N = L * L, np1 = N + 1;
  std::vector<uint32_t> Tor(5 * np1), T(5 * np1);
  or_build_table(W, L, Tor.data());
  for (int m = 0; m < np1; ++m) for (int a = 0; a < 5; ++a) T[a * np1 + m] = Tor[m * 5 + a];
  int bad = 0;
  for (int c = 0; c < p; ++c) {
    std::vector<int8_t> s(N);
    or_init_lattice(s.data(), L, seed, c, start);
    int m_or = (or_energy(s.data(), L) + 2 * N) / 4;
    // pack
    std::vector<uint32_t> lat(L * WD, 0);
    for (int y = 0; y < L; ++y) for (int x = 0; x < L; ++x) if (s[y * L + x] > 0) lat[y * WD + x / 32] |= 1u << (x % 32);
    int m = m_or;
    std::vector<uint32_t> hist(np1, 0);
    hist.resize(np1 + 3, 0u);          // (scratch counter of the delayed counts past the last level)
    GenHook<WD == 1 ? 32 : 8> hk;
    hk.init(hist.data(), 1u, np1);
    Prefetch pf; prefetch_init<WD>(pf, L, 0, (uint32_t)c, (uint32_t)seed, (uint32_t)(seed >> 32));
    std::vector<int32_t> tr_g(S);
    for (int64_t sw = 0; sw < S; ++sw) {
      for (int y = 0; y < L; ++y) {
        int ym = (y + L - 1) % L, yp = (y + 1) % L;
        uint32_t cur[WD], up[WD], dn[WD];
        for (int w = 0; w < WD; ++w) { cur[w] = lat[y * WD + w]; up[w] = lat[ym * WD + w]; dn[w] = lat[yp * WD + w]; }
        sweep_row<WD>(cur, up, dn, L, m, T.data(), np1, pf, (uint32_t)c, (uint32_t)seed, (uint32_t)(seed >> 32), hk);
        if (m < 0 || m > N) { printf("m out of range %d\n", m); return 1; }
        for (int w = 0; w < WD; ++w) lat[y * WD + w] = cur[w];
      }
      tr_g[sw] = m;
    }
    hk.flush(m);
    // oracle
    std::vector<int32_t> tr(S); std::vector<int64_t> h(np1, 0);
    int32_t mo = m_or;
    or_chain_round(L, seed, c, 0, S, Tor.data(), s.data(), &mo, tr.data(), h.data(), nullptr);
    std::vector<uint32_t> lat2(L * WD, 0);
    for (int y = 0; y < L; ++y) for (int x = 0; x < L; ++x) if (s[y * L + x] > 0) lat2[y * WD + x / 32] |= 1u << (x % 32);
    bool ok = (lat == lat2) && (mo == m);
    for (int64_t sw = 0; sw < S; ++sw) ok = ok && tr[sw] == tr_g[sw];
    for (int q = 0; q < np1; ++q) ok = ok && (int64_t)hist[q] == h[q];
    if (!ok) { ++bad; if (bad < 3) printf("L=%d chain %d mismatch (m %d vs %d)\n", L, c, m, mo); }
    // joint hooks, for inputs at, below and above the chain's start level
    std::vector<int8_t> s0(N);
    or_init_lattice(s0.data(), L, seed, c, start);
    std::vector<uint32_t> lat0(L * WD, 0);
    for (int y = 0; y < L; ++y) for (int x = 0; x < L; ++x) if (s0[y * L + x] > 0) lat0[y * WD + x / 32] |= 1u << (x % 32);
    const int xs[3] = {m_or, m_or / 2, (m_or + N) / 2};
    for (int xi = 0; xi < 3; ++xi) {
      const int x = xs[xi];
      const uint32_t r = 3 + xi;
      std::vector<uint32_t> tj(np1);
      for (int q = 0; q < np1; ++q) tj[q] = or_threshold(W[q] - W[x]);
      SearchHook sh;
      sh.tj = tj.data(); sh.k = 0; sh.M = S * N; sh.found = 0; sh.chain = (uint32_t)c; sh.r = r;
      sh.k0 = (uint32_t)seed; sh.k1 = (uint32_t)(seed >> 32); sh.done = false;
      replay<WD>(L, S, lat0, m_or, T.data(), np1, seed, (uint32_t)c, sh, true);
      const int64_t k_or = or_chain_first_accept(L, seed, (uint32_t)c, 0, S, Tor.data(), W, s0.data(), m_or, x, r,
                                                 nullptr);
      std::vector<uint32_t> umin(np1, 0xFFFFFFFFu);
      SummaryHook<> su;
      su.umin = umin.data(); su.k = 0; su.chain = (uint32_t)c; su.r = r; su.k0 = (uint32_t)seed;
      su.k1 = (uint32_t)(seed >> 32); su.cur = -1; su.lo = 0x7FFFFFFF; su.hi = -1; su.run_min = 0xFFFFFFFFu;
      su.flag = false; su.done = false;
      replay<WD>(L, S, lat0, m_or, T.data(), np1, seed, (uint32_t)c, su, false);
      su.flush();
      // the same summary through a window of 8 levels (most levels fall
      // outside it, so both paths run): the same row once drained, and the
      // window empty again
      std::vector<uint32_t> umin_w(np1, 0xFFFFFFFFu), win(8 * kWinStride, 0xFFFFFFFFu);
      SummaryHook<8> sw;
      sw.umin = umin_w.data(); sw.k = 0; sw.chain = (uint32_t)c; sw.r = r; sw.k0 = (uint32_t)seed;
      sw.k1 = (uint32_t)(seed >> 32); sw.cur = -1; sw.lo = 0x7FFFFFFF; sw.hi = -1; sw.run_min = 0xFFFFFFFFu;
      sw.flag = false; sw.done = false; sw.win = win.data() + 5;
      replay<WD>(L, S, lat0, m_or, T.data(), np1, seed, (uint32_t)c, sw, false);
      sw.flush();
      sw.drain();
      bool win_ok = umin_w == umin && sw.lo == su.lo && sw.hi == su.hi && sw.flag == su.flag;
      for (uint32_t v : win) win_ok = win_ok && v == 0xFFFFFFFFu;
      bool acc = false;
      for (int q = su.lo; q <= su.hi; ++q) acc = acc || (umin[q] != 0xFFFFFFFFu && umin[q] <= tj[q]);
      if (sh.found != k_or || acc != (k_or > 0) || su.k != S * N || !win_ok) {
        ++bad;
        if (bad < 3) printf("L=%d chain %d joint hooks: search %lld vs %lld, summary %d\n", L, c,
                            (long long)sh.found, (long long)k_or, (int)acc);
      }
    }
  }
  return bad;
}
int main() {
  int total_bad = 0;
  int Ls[] = {4, 8, 12, 16, 20, 24, 28, 32, 36, 48, 64, 100, 128};
  for (int L : Ls) {
    int N = L * L;
    std::vector<double> W(N + 1);
    srand(L);
    for (int i = 0; i <= N; ++i) W[i] = 3.0 * ((double)rand() / RAND_MAX - 0.5) + 2.0 * sin(i * 0.01);
    int64_t S = L <= 32 ? 20 : 4;
    int p = L <= 32 ? 8 : 3;
    int wd = (L + 31) / 32, bad = 0;
    for (int start = 0; start < 2; ++start) {
      if (wd == 1) bad += run<1>(L, p, S, 0x1234567890ull + L, W.data(), start);
      else if (wd == 2) bad += run<2>(L, p, S, 0x1234567890ull + L, W.data(), start);
      else if (wd == 3) bad += run<3>(L, p, S, 0x1234567890ull + L, W.data(), start);
      else bad += run<4>(L, p, S, 0x1234567890ull + L, W.data(), start);
    }
    printf("L=%d: %s\n", L, bad ? "MISMATCH" : "ok");
    total_bad += bad;
  }
  return total_bad != 0;
}
