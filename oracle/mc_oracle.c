/*
 * mc_oracle.c -- plain, slow, sequential CPU oracle (test infrastructure).
 *
 * This file is the reference the GPU library is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it;
 * the GPU library shares no code with it.  Everything is written to be read
 * against the paper:
 *   Sec. 2, "Algorithm", steps 1-6 ......... or_run_round / or_run_attempts /
 *                                             or_join / or_iteration
 *   Sec. 2, step 6 with M_node adjusted ..... or_iteration_adaptive
 *   Sec. 2, energy-ordered joining .......... or_set_join_order (opt-in)
 *   Sec. 5, Fig. 2 control (no balance) ..... or_join_naive
 *   Sec. 3.1, Eq. (new_weight) .............. or_update_weights
 *   Sec. 3.2, Eq. (reweighting2), Sec. 4.1 .. or_thermo (E, C, F, S)
 *   Sec. 4.1, the Hamiltonian ............... or_energy
 *   Sec. 4.2, weights kept as logarithms .... W = ln w, W -= ln h
 *   Sec. 4.2, "The Metropolis method" ....... or_threshold (flips and joints)
 * The random-number generator (Philox4x32-10, Salmon, Moraes, Dror and Shaw,
 * SC'11) and the deterministic exp/log are not in the paper; they fix every
 * draw and every rounding so that two implementations can agree bit for bit.
 *
 * Build with -ffp-contract=off: exp/log below must round every operation
 * separately (no fused multiply-add), on x86_64 and aarch64 alike.
 */
#include "mc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64    */
/* multiplies; key bumped by the Weyl constants between rounds.        */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t c3, unsigned word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[word & 3u];
}

/* uniform for flip attempt t (0-based count since the job started) of chain c */
static uint32_t flip_uniform(uint64_t seed, uint32_t c, uint64_t t)
{
    uint64_t b = t >> 2;
    return philox_word(seed, (uint32_t)b, (uint32_t)(b >> 32), c, 0u, (unsigned)(t & 3u));
}

/* uniform for the joint test of sample k (1-based) of chain i in round r */
static uint32_t joint_uniform(uint64_t seed, uint32_t r, uint32_t i, int64_t k)
{
    uint64_t q = (uint64_t)(k - 1);
    return philox_word(seed, (uint32_t)(q >> 2), r, i, 1u, (unsigned)(q & 3u));
}

/* ------------------------------------------------------------------ */
/* Deterministic exp and log: only IEEE +, -, *, / (each rounded to    */
/* nearest), rint, frexp, ldexp.                                       */
/* ------------------------------------------------------------------ */
/* ln 2 cut to 32 significant bits, so n*LN2_HI is exact for |n| < 2^21 */
static const double LN2_HI = 0x1.62e42fefp-1;
/* the rest of ln 2, rounded to nearest */
static const double LN2_LO = 0x1.473de6af278edp-34;
/* 1/ln 2 rounded to nearest */
static const double INV_LN2 = 0x1.71547652b82fep+0;
/* sqrt(1/2) rounded to nearest */
static const double SQRT_HALF = 0x1.6a09e667f3bcdp-1;

/* 1/j!, j = 0..13, each the nearest double (j! is exact in a double) */
static const double EXP_C[14] = {
    1.0 / 1.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0,
    1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0,
    1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0};

/* 1/(2j+1), j = 0..10, each the nearest double */
static const double LOG_C[11] = {
    1.0 / 1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0, 1.0 / 11.0,
    1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0};

double or_const(int which)
{
    switch (which) {
    case 0: return LN2_HI;
    case 1: return LN2_LO;
    case 2: return INV_LN2;
    case 3: return SQRT_HALF;
    default:
        if (which >= 100 && which < 114) return EXP_C[which - 100];
        if (which >= 200 && which < 211) return LOG_C[which - 200];
        return 0.0;
    }
}

/*
 * exp(d) for |d| <= 700 (Cody & Waite 1980 reduction + Taylor polynomial):
 *   n = rint(d / ln 2),  r = (d - n LN2_HI) - n LN2_LO,  |r| <~ ln2 / 2,
 *   exp(r) = sum_{j=0}^{13} r^j / j!  (Horner),  exp(d) = 2^n exp(r).
 * The truncated tail is below 5e-18 relative.
 */
double or_exp_det(double d)
{
    double n = rint(d * INV_LN2);
    double r = (d - n * LN2_HI) - n * LN2_LO;
    double poly = EXP_C[13];
    for (int j = 12; j >= 0; --j)
        poly = poly * r + EXP_C[j];
    return ldexp(poly, (int)n);
}

/*
 * ln(x) for finite x >= 1 (used on integer counts h(E)):
 *   x = f 2^e with f in [sqrt(1/2), sqrt(2)),  s = (f-1)/(f+1),
 *   ln f = 2 s sum_{j=0}^{10} s^(2j) / (2j+1)  (|s| <= 0.1716; tail < 1e-18),
 *   ln x = e LN2_HI + (e LN2_LO + ln f).
 */
double or_log_det(double x)
{
    int e;
    double f = frexp(x, &e);          /* x = f * 2^e, f in [1/2, 1) */
    if (f < SQRT_HALF) {
        f = f * 2.0;
        e = e - 1;
    }
    double s = (f - 1.0) / (f + 1.0);
    double z = s * s;
    double q = LOG_C[10];
    for (int j = 9; j >= 0; --j)
        q = q * z + LOG_C[j];
    double series = (2.0 * s) * q;
    double ed = (double)e;
    return ed * LN2_HI + (ed * LN2_LO + series);
}

/*
 * Metropolis acceptance threshold for a move with log-weight change d
 * (Sec. 4.2: the weight is kept as its logarithm, so the Metropolis ratio
 * w'/w is exp(d)).  A 32-bit uniform u is accepted iff u <= thr(d):
 *   d >= 0            -> 0xFFFFFFFF (always accepted, exactly);
 *   d <= -23          -> 0 (exp(-23) < 2^-32);
 *   otherwise x = 2^32 exp(d):  x <= 1 -> 0,  else ceil(x) - 1.
 * P(accept) = (thr+1)/2^32 is within 2^-32 of min(1, exp(d)).
 */
uint32_t or_threshold(double d)
{
    if (d >= 0.0) return 0xFFFFFFFFu;
    if (d <= -23.0) return 0u;
    double x = ldexp(or_exp_det(d), 32);
    if (x <= 1.0) return 0u;
    return (uint32_t)(ceil(x) - 1.0);
}

/* ------------------------------------------------------------------ */
/* The 2D Ising model (Sec. 4.1)                                       */
/* ------------------------------------------------------------------ */
#define SPIN(s, L, x, y) ((int)(s)[(size_t)(((y) + (L)) % (L)) * (size_t)(L) + (size_t)(((x) + (L)) % (L))])

/* H = -sum over nearest-neighbour pairs of s_i s_j, periodic: each site bonds
 * to its right and lower neighbour, 2N bonds in all. */
int or_energy(const int8_t *s, int L)
{
    int E = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            E -= SPIN(s, L, x, y) * (SPIN(s, L, x + 1, y) + SPIN(s, L, x, y + 1));
    return E;
}

static int level_of(int E, int N) { return (E + 2 * N) / 4; }

/* Step 1: initial configuration C_1^{(i)}; start 0 = all up, 1 = random. */
void or_init_lattice(int8_t *s, int L, uint64_t seed, uint32_t chain, int start)
{
    int N = L * L;
    for (int site = 0; site < N; ++site) {
        if (start == 0) {
            s[site] = 1;
        } else {
            uint32_t q = (uint32_t)site >> 5;          /* 32-bit word of the packed lattice */
            uint32_t word = philox_word(seed, q >> 2, 0u, chain, 2u, q & 3u);
            uint32_t bit = (word >> (site & 31)) & 1u;
            s[site] = bit ? 1 : -1;
        }
    }
}

/* Table of flip thresholds: T[m*5 + a] for a move from level m to m + a - 2
 * (dE = 4(a - 2)); moves that leave [0, N] never occur and get 0. */
void or_build_table(const double *W, int L, uint32_t *T)
{
    int N = L * L;
    for (int m = 0; m <= N; ++m)
        for (int a = 0; a < 5; ++a) {
            int mp = m + a - 2;
            T[m * 5 + a] = (mp < 0 || mp > N) ? 0u : or_threshold(W[mp] - W[m]);
        }
}

/*
 * Step 2 for one chain: S sweeps (M = S*N single-spin-flip Metropolis
 * attempts in typewriter order) under the weight behind T.  *m_io is the
 * level before the round and after it.  Optional outputs: trace[s] = level
 * after sweep s; hist[m] += number of samples at level m; samples[k-1] =
 * level of sample k (the configuration after attempt k).
 */
/* n consecutive attempts of one chain from its attempt t0: attempt t visits
 * site t mod N (typewriter order continues across rounds), so a round need
 * not start or end on a sweep.  trace gets the level at the end of every
 * sweep completed inside the attempts. */
int or_chain_attempts(int L, uint64_t seed, uint32_t chain, uint64_t t0, int64_t n,
                      const uint32_t *T, int8_t *s, int32_t *m_io,
                      int32_t *trace, int64_t *hist, int32_t *samples)
{
    int N = L * L;
    int m = *m_io;
    int64_t n_tr = 0;
    for (int64_t k = 0; k < n; ++k) {
        const uint64_t t = t0 + (uint64_t)k;
        const int site = (int)(t % (uint64_t)N);
        int x = site % L, y = site / L;
        int sv = SPIN(s, L, x, y);
        int nb = SPIN(s, L, x - 1, y) + SPIN(s, L, x + 1, y) + SPIN(s, L, x, y - 1) + SPIN(s, L, x, y + 1);
        int dE = 2 * sv * nb;
        int a = dE / 4 + 2;
        uint32_t u = flip_uniform(seed, chain, t);
        if (u <= T[m * 5 + a]) {
            s[y * L + x] = (int8_t)(-sv);
            m += dE / 4;
        }
        if (hist) hist[m] += 1;
        if (samples) samples[k] = m;
        if (trace && site == N - 1) trace[n_tr++] = m;
    }
    *m_io = m;
    return 0;
}

int or_chain_round(int L, uint64_t seed, uint32_t chain, uint64_t t0, int64_t S,
                   const uint32_t *T, int8_t *s, int32_t *m_io,
                   int32_t *trace, int64_t *hist, int32_t *samples)
{
    return or_chain_attempts(L, seed, chain, t0, S * (int64_t)L * L, T, s, m_io, trace, hist, samples);
}

/*
 * Step 4 for one chain on its stored samples: the first k in 1..M whose
 * configuration passes the Metropolis test against the previous node's last
 * configuration (level x), or 0 if none does.
 */
int64_t or_joint_scan(const int32_t *levels, int64_t M, const double *W,
                      int32_t x_level, uint64_t seed, uint32_t r, uint32_t i)
{
    for (int64_t k = 1; k <= M; ++k) {
        uint32_t u = joint_uniform(seed, r, i, k);
        if (u <= or_threshold(W[levels[k - 1]] - W[x_level]))
            return k;
    }
    return 0;
}

/*
 * The same first-accept search without stored samples: chain `chain` is
 * regenerated from its round-start state (s_start, m_start) with the round's
 * flip counters and each sample is tested as it appears.  prefix_hist (if
 * given) receives the levels of the discarded samples 1..k-1 (all M if none
 * is accepted).
 */
int64_t or_chain_first_accept(int L, uint64_t seed, uint32_t chain, uint64_t t0,
                              int64_t S, const uint32_t *T, const double *W,
                              const int8_t *s_start, int32_t m_start,
                              int32_t x_level, uint32_t r, int64_t *prefix_hist)
{
    int N = L * L;
    int8_t *s = (int8_t *)malloc((size_t)N);
    memcpy(s, s_start, (size_t)N);
    int m = m_start;
    uint64_t t = t0;
    int64_t k = 0, found = 0;
    for (int64_t sweep = 0; sweep < S && !found; ++sweep) {
        for (int site = 0; site < N; ++site) {
            int x = site % L, y = site / L;
            int sv = SPIN(s, L, x, y);
            int nb = SPIN(s, L, x - 1, y) + SPIN(s, L, x + 1, y) + SPIN(s, L, x, y - 1) + SPIN(s, L, x, y + 1);
            int dE = 2 * sv * nb;
            int a = dE / 4 + 2;
            uint32_t u = flip_uniform(seed, chain, t);
            t += 1;
            if (u <= T[m * 5 + a]) {
                s[y * L + x] = (int8_t)(-sv);
                m += dE / 4;
            }
            k += 1;
            uint32_t uj = joint_uniform(seed, r, chain, k);
            if (uj <= or_threshold(W[m] - W[x_level])) {
                found = k;
                break;
            }
            if (prefix_hist) prefix_hist[m] += 1;
        }
    }
    free(s);
    return found;
}

/* ------------------------------------------------------------------ */
/* A whole job: p chains, the joint, the weight recursion              */
/* ------------------------------------------------------------------ */
struct or_job {
    int L, N, p;
    uint64_t seed;
    int8_t *spins;      /* [p][N] */
    int32_t *m;         /* [p] current level */
    uint64_t t;         /* attempts per chain since the job started */
    double *W;          /* [N+1] ln w */
    uint32_t *T;        /* [(N+1)*5] flip thresholds under W */
    int64_t *h;         /* [N+1] total histogram of the joined chain */
    int32_t carry;      /* level of the last configuration passed on */
    int carry_valid;
    uint32_t r;         /* rounds joined so far */
    int64_t last_S;     /* sweeps completed inside the last round (trace entries) */
    int64_t last_M;     /* attempts (samples) per chain of the last round */
    int32_t *samples;   /* [p][M] levels of the last round's samples */
    int32_t *trace;     /* [p][S] level after each sweep */
    int64_t *k;         /* [p] first kept sample of the last joint (0 = none) */
    uint8_t *visited;   /* [N+1] 1 once a weight update has seen h > 0 there */
    int join_order;     /* 0: chains joined in index order; 1: by final energy */
    int32_t *order;     /* [p] chain at each position of the last joint */
};

or_job *or_create(int L, int p, uint64_t seed, int start)
{
    if (L < 2 || L > 256 || (L & 1) || p < 1) return NULL;
    or_job *j = (or_job *)calloc(1, sizeof(or_job));
    j->L = L;
    j->N = L * L;
    j->p = p;
    j->seed = seed;
    j->spins = (int8_t *)malloc((size_t)p * (size_t)j->N);
    j->m = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    j->W = (double *)calloc((size_t)j->N + 1, sizeof(double));      /* w^(1) = 1 */
    j->T = (uint32_t *)malloc(sizeof(uint32_t) * 5 * ((size_t)j->N + 1));
    j->h = (int64_t *)calloc((size_t)j->N + 1, sizeof(int64_t));     /* step 1: h(E) = 0 */
    j->k = (int64_t *)calloc((size_t)p, sizeof(int64_t));
    j->visited = (uint8_t *)calloc((size_t)j->N + 1, 1);
    j->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)p);
    for (int c = 0; c < p; ++c) j->order[c] = c;
    for (int c = 0; c < p; ++c) {
        int8_t *s = j->spins + (size_t)c * j->N;
        or_init_lattice(s, L, seed, (uint32_t)c, start);
        j->m[c] = level_of(or_energy(s, L), j->N);
    }
    or_build_table(j->W, L, j->T);
    return j;
}

void or_free(or_job *j)
{
    if (!j) return;
    free(j->spins); free(j->m); free(j->W); free(j->T); free(j->h);
    free(j->samples); free(j->trace); free(j->k); free(j->visited); free(j->order);
    free(j);
}

typedef struct {
    or_job *j;
    int64_t n, n_tr;
    int tid, nthreads;
} round_arg;

static void *round_worker(void *vp)
{
    round_arg *a = (round_arg *)vp;
    or_job *j = a->j;
    for (int c = a->tid; c < j->p; c += a->nthreads)
        or_chain_attempts(j->L, j->seed, (uint32_t)c, j->t, a->n, j->T,
                          j->spins + (size_t)c * j->N, &j->m[c],
                          j->trace + (size_t)c * (size_t)a->n_tr, NULL,
                          j->samples + (size_t)c * (size_t)a->n);
    return NULL;
}

/* Step 2 for every chain: n attempts each (a round need not be whole sweeps). */
int or_run_attempts(or_job *j, int64_t n, int nthreads)
{
    if (n < 1) return -1;
    const uint64_t N = (uint64_t)j->N;
    /* sweeps completed inside the round: attempts t with t mod N = N - 1 */
    const int64_t n_tr = (int64_t)((j->t + (uint64_t)n) / N - j->t / N);
    free(j->samples);
    free(j->trace);
    j->samples = (int32_t *)malloc(sizeof(int32_t) * (size_t)j->p * (size_t)n);
    j->trace = (int32_t *)malloc(sizeof(int32_t) * (size_t)j->p * (size_t)(n_tr > 0 ? n_tr : 1));
    if (!j->samples || !j->trace) return -2;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > j->p) nthreads = j->p;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    round_arg *args = (round_arg *)malloc(sizeof(round_arg) * (size_t)nthreads);
    for (int q = 0; q < nthreads; ++q) {
        args[q].j = j; args[q].n = n; args[q].n_tr = n_tr; args[q].tid = q; args[q].nthreads = nthreads;
        pthread_create(&th[q], NULL, round_worker, &args[q]);
    }
    for (int q = 0; q < nthreads; ++q) pthread_join(th[q], NULL);
    free(th);
    free(args);
    j->t += (uint64_t)n;
    j->last_S = n_tr;
    j->last_M = n;
    return 0;
}

int or_run_round(or_job *j, int64_t S, int nthreads)
{
    if (S < 1) return -1;
    return or_run_attempts(j, S * (int64_t)j->N, nthreads);
}

/*
 * Steps 3-5: i = 0..p-1 in order.  Node i checks the detailed balance of its
 * configurations C_k (k = 1, 2, ...) against the last configuration passed on
 * by node (i-1+p) mod p; the first accepted one and all after it are kept and
 * added to h, and node i passes on its own last configuration.  If none is
 * accepted the configuration passed on stays the one node i received, and
 * none of node i's configurations is kept.  Node 0 checks against what node
 * p-1 passed on in the previous round; in the job's first round there is
 * nothing to check against and node 0's chain is kept whole.
 * Returns the number of configurations kept in this round.
 */
/* Order of the chains at the joint.  Index order, or (the energy-ordered
 * joining the paper proposes at the end of Sec. 2 to raise acceptance, with
 * the order left open there) ascending by the energy of each chain's last
 * generated configuration, equal energies in index order. */
static const int32_t *g_sort_levels;
static int cmp_by_level(const void *a, const void *b)
{
    const int32_t ia = *(const int32_t *)a, ib = *(const int32_t *)b;
    const int32_t la = g_sort_levels[ia], lb = g_sort_levels[ib];
    if (la != lb) return la < lb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

static void joint_order(or_job *j, int64_t M)
{
    for (int c = 0; c < j->p; ++c) j->order[c] = c;
    if (j->join_order != 1) return;
    int32_t *last = (int32_t *)malloc(sizeof(int32_t) * (size_t)j->p);
    for (int c = 0; c < j->p; ++c) last[c] = j->samples[(size_t)c * (size_t)M + (size_t)(M - 1)];
    g_sort_levels = last;
    qsort(j->order, (size_t)j->p, sizeof(int32_t), cmp_by_level);
    g_sort_levels = NULL;
    free(last);
}

int64_t or_join(or_job *j)
{
    int64_t M = j->last_M;
    int64_t joined = 0;
    joint_order(j, M);
    for (int q = 0; q < j->p; ++q) {
        const int i = j->order[q];
        const int32_t *lev = j->samples + (size_t)i * (size_t)M;
        int64_t k;
        if (!j->carry_valid)
            k = 1;
        else
            k = or_joint_scan(lev, M, j->W, j->carry, j->seed, j->r, (uint32_t)i);
        j->k[i] = k;
        if (k > 0) {
            for (int64_t t = k - 1; t < M; ++t) j->h[lev[t]] += 1;   /* h += h_local */
            joined += M - k + 1;
            j->carry = lev[M - 1];
            j->carry_valid = 1;
        }
    }
    j->r += 1;
    return joined;
}

/* The control experiment of Sec. 5 (Fig. 2): chains concatenated whole,
 * without the detailed-balance test at the joints. */
int64_t or_join_naive(or_job *j)
{
    int64_t M = j->last_M;
    joint_order(j, M);
    for (int q = 0; q < j->p; ++q) {
        const int i = j->order[q];
        const int32_t *lev = j->samples + (size_t)i * (size_t)M;
        j->k[i] = 1;
        for (int64_t t = 0; t < M; ++t) j->h[lev[t]] += 1;
        j->carry = lev[M - 1];
        j->carry_valid = 1;
    }
    j->r += 1;
    return M * (int64_t)j->p;
}

void or_set_join_order(or_job *j, int mode) { j->join_order = mode; }
void or_get_order(const or_job *j, int32_t *order) { memcpy(order, j->order, sizeof(int32_t) * (size_t)j->p); }

/* Eq. (new_weight) in logarithms: w <- w / h where h > 0, i.e. W -= ln h;
 * then h is cleared for the next iteration. */
void or_update_weights(or_job *j)
{
    for (int m = 0; m <= j->N; ++m) {
        if (j->h[m] > 0) {
            j->W[m] = j->W[m] - or_log_det((double)j->h[m]);
            j->visited[m] = 1;
        }
        j->h[m] = 0;
    }
    or_build_table(j->W, j->L, j->T);
}

/* Steps 2-6 under one weight, then the weight update: rounds are repeated
 * while h holds fewer than M_total configurations. */
int64_t or_iteration(or_job *j, int64_t S, int64_t M_total, int nthreads)
{
    int64_t total = 0;
    do {
        if (or_run_round(j, S, nthreads) != 0) return -1;
        total += or_join(j);
    } while (total < M_total);
    or_update_weights(j);
    return total;
}

/* Step 6 with "M_node adjusted appropriately": after a round that leaves h
 * short of M_total, the next round's sweeps are those that the last round's
 * rate of kept samples per sweep needs for the remainder,
 *   S_next = ceil(remaining * S_last / joined_last), within [1, S],
 * and S when the last round kept nothing.  rounds_out (may be NULL) gets the
 * number of rounds; sweeps_out (may be NULL, room for max_rounds) their S. */
int64_t or_iteration_adaptive(or_job *j, int64_t S, int64_t M_total, int nthreads, int max_rounds,
                              int *rounds_out, int64_t *sweeps_out)
{
    int64_t total = 0, s_cur = S;
    int rounds = 0;
    for (;;) {
        if (or_run_round(j, s_cur, nthreads) != 0) return -1;
        const int64_t got = or_join(j);
        total += got;
        if (sweeps_out && rounds < max_rounds) sweeps_out[rounds] = s_cur;
        ++rounds;
        if (total >= M_total || rounds >= max_rounds) break;
        const int64_t remaining = M_total - total;
        int64_t nxt = S;
        if (got > 0) {
            nxt = (remaining * s_cur + got - 1) / got;
            if (nxt < 1) nxt = 1;
            if (nxt > S) nxt = S;
        }
        s_cur = nxt;
    }
    or_update_weights(j);
    if (rounds_out) *rounds_out = rounds;
    return total;
}

int or_get_L(const or_job *j) { return j->L; }
int or_get_p(const or_job *j) { return j->p; }
void or_get_weights(const or_job *j, double *W) { memcpy(W, j->W, sizeof(double) * ((size_t)j->N + 1)); }
void or_set_weights(or_job *j, const double *W)
{
    memcpy(j->W, W, sizeof(double) * ((size_t)j->N + 1));
    or_build_table(j->W, j->L, j->T);
}
void or_get_table(const or_job *j, uint32_t *T) { memcpy(T, j->T, sizeof(uint32_t) * 5 * ((size_t)j->N + 1)); }
void or_get_hist(const or_job *j, int64_t *h) { memcpy(h, j->h, sizeof(int64_t) * ((size_t)j->N + 1)); }
void or_get_spins(const or_job *j, int8_t *s) { memcpy(s, j->spins, (size_t)j->p * (size_t)j->N); }
void or_get_levels(const or_job *j, int32_t *m) { memcpy(m, j->m, sizeof(int32_t) * (size_t)j->p); }
void or_get_trace(const or_job *j, int32_t *trace)
{
    /* out[sweep][chain] */
    for (int c = 0; c < j->p; ++c)
        for (int64_t s = 0; s < j->last_S; ++s)
            trace[(size_t)s * (size_t)j->p + (size_t)c] = j->trace[(size_t)c * (size_t)j->last_S + (size_t)s];
}
void or_get_k(const or_job *j, int64_t *k) { memcpy(k, j->k, sizeof(int64_t) * (size_t)j->p); }
int32_t or_get_carry(const or_job *j, int *valid) { if (valid) *valid = j->carry_valid; return j->carry; }
uint64_t or_get_t(const or_job *j) { return j->t; }
void or_get_visited(const or_job *j, uint8_t *v) { memcpy(v, j->visited, (size_t)j->N + 1); }
uint32_t or_get_round(const or_job *j) { return j->r; }
int64_t or_get_last_S(const or_job *j) { return j->last_S; }
int64_t or_get_last_M(const or_job *j) { return j->last_M; }
/* Test hook: install hand-made samples for the last round (S sweeps), so that
 * the joint can be checked on crafted energy sequences. */
int or_set_samples(or_job *j, int64_t S, const int32_t *samples)
{
    if (S < 1) return -1;
    int64_t M = S * (int64_t)j->N;
    free(j->samples);
    j->samples = (int32_t *)malloc(sizeof(int32_t) * (size_t)j->p * (size_t)M);
    if (!j->samples) return -2;
    memcpy(j->samples, samples, sizeof(int32_t) * (size_t)j->p * (size_t)M);
    j->last_S = S;
    j->last_M = M;
    return 0;
}

void or_get_samples(const or_job *j, int32_t *samples)
{
    memcpy(samples, j->samples, sizeof(int32_t) * (size_t)j->p * (size_t)j->last_M);
}

/* ------------------------------------------------------------------ */
/* Statistical averages at inverse temperature beta (Sec. 3.2, Eq.     */
/* reweighting2; Sec. 4.1 for E, C, F, S).  With W = ln w and the       */
/* density of states D(E) proportional to 1/w(E), over the levels the   */
/* weight iteration has visited:                                        */
/*   <O> = sum_E O(E) e^{-W(E) - beta E} / sum_E e^{-W(E) - beta E},     */
/* every exponential taken relative to the largest exponent (the        */
/* logarithmic evaluation Sec. 4.2 asks for).  E = <H>,                  */
/* C = beta^2 (<H^2> - <H>^2) summed as beta^2 <(H - <H>)^2>.  D is      */
/* normalised so that it counts all 2^N states:                          */
/*   ln Z = N ln 2 + ln sum_E e^{-W - beta E} - ln sum_E e^{-W},         */
/* F = -ln Z / beta, S = beta (E - F).                                   */
/* out[4 b + 0..3] = E, C, F, S at betas[b].  Plain libm exp/log: these */
/* averages are compared with a tolerance, not bit for bit.             */
/* ------------------------------------------------------------------ */
void or_thermo(int L, const double *W, const uint8_t *visited, const double *betas, int nb, double *out)
{
    const int N = L * L;
    double bmax = -INFINITY;
    for (int m = 0; m <= N; ++m)
        if (visited[m] && -W[m] > bmax) bmax = -W[m];
    double sg = 0.0;
    for (int m = 0; m <= N; ++m)
        if (visited[m]) sg += exp(-W[m] - bmax);
    const double ln_norm = bmax + log(sg);           /* ln sum_E e^{-W} */
    for (int b = 0; b < nb; ++b) {
        const double beta = betas[b];
        double amax = -INFINITY;
        for (int m = 0; m <= N; ++m) {
            if (!visited[m]) continue;
            const double E = (double)(4 * m - 2 * N);
            const double a = -W[m] - beta * E;
            if (a > amax) amax = a;
        }
        double z = 0.0, e1 = 0.0;
        for (int m = 0; m <= N; ++m) {
            if (!visited[m]) continue;
            const double E = (double)(4 * m - 2 * N);
            const double wgt = exp(-W[m] - beta * E - amax);
            z += wgt;
            e1 += E * wgt;
        }
        const double Eav = e1 / z;
        double v = 0.0;
        for (int m = 0; m <= N; ++m) {
            if (!visited[m]) continue;
            const double E = (double)(4 * m - 2 * N);
            const double wgt = exp(-W[m] - beta * E - amax);
            v += (E - Eav) * (E - Eav) * wgt;
        }
        const double lnZ = (double)N * log(2.0) + amax + log(z) - ln_norm;
        const double F = -lnZ / beta;
        out[4 * b + 0] = Eav;
        out[4 * b + 1] = beta * beta * (v / z);
        out[4 * b + 2] = F;
        out[4 * b + 3] = beta * (Eav - F);
    }
}
