/*
 * mc_oracle.h -- plain sequential CPU oracle for parallel multicanonical
 * Ising chains joined by detailed balance (Sugihara, Higo, Nakamura,
 * "Parallelization of Markov Chain Generation and its Application to the
 * Multicanonical Method").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * includes, links or calls anything here, and this file shares no code with
 * it.
 *
 * Conventions (the readings the oracle takes where the paper is silent):
 *   - Lattice: L x L periodic square lattice, N = L*L sites, spin s(x,y) in
 *     {-1,+1} stored as int8 at index y*L + x.  L even, 2 <= L <= 256.
 *   - Energy (Sec. 4.1): E = -sum_{x,y} s(x,y) [s(x+1,y) + s(x,y+1)], indices
 *     mod L (2N bonds).  E = -2N + 4m, level m in [0, N].
 *   - One sample = the configuration after one single-spin-flip attempt.
 *     Attempts visit sites in typewriter order (x fastest), so a round of
 *     S sweeps is M = S*N attempts per chain.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (lo32(seed),
 *     hi32(seed)).  Counter words: flips (lo32(t>>2), hi32(t>>2), c, 0) word
 *     t&3 with t the chain's attempt count since job start; joints
 *     ((k-1)>>2, r, i, 1) word (k-1)&3 for sample k of chain i in round r;
 *     random start: word q of the bit-packed lattice is
 *     Philox((q>>2, 0, c, 2)) word q&3, bit (site & 31) of word (site >> 5),
 *     1 meaning +1.
 *   - Acceptance of a move from level m to m' (flip or joint, Metropolis):
 *     d = W[m'] - W[m]; accept iff u <= thr(d) (see or_threshold).
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- primitives ---- */
void     or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   or_exp_det(double d);
double   or_log_det(double x);
uint32_t or_threshold(double d);
double   or_const(int which);

/* ---- lattice ---- */
int  or_energy(const int8_t *s, int L);
void or_init_lattice(int8_t *s, int L, uint64_t seed, uint32_t chain, int start);
void or_build_table(const double *W, int L, uint32_t *T);

/* ---- one chain, one round (streaming; nothing stored per sample unless asked) ---- */
int  or_chain_round(int L, uint64_t seed, uint32_t chain, uint64_t t0, int64_t S,
                    const uint32_t *T, int8_t *s, int32_t *m_io,
                    int32_t *trace, int64_t *hist, int32_t *samples);
int64_t or_chain_first_accept(int L, uint64_t seed, uint32_t chain, uint64_t t0,
                              int64_t S, const uint32_t *T, const double *W,
                              const int8_t *s_start, int32_t m_start,
                              int32_t x_level, uint32_t r, int64_t *prefix_hist);
int64_t or_joint_scan(const int32_t *levels, int64_t M, const double *W,
                      int32_t x_level, uint64_t seed, uint32_t r, uint32_t i);

/* ---- a whole job (Sec. 2 algorithm + Sec. 3 weight recursion) ---- */
typedef struct or_job or_job;
or_job *or_create(int L, int p, uint64_t seed, int start);
void    or_free(or_job *j);
int     or_run_round(or_job *j, int64_t S, int nthreads);
/* a round of n attempts per chain (attempt t visits site t mod N) */
int     or_run_attempts(or_job *j, int64_t n, int nthreads);
int64_t or_join(or_job *j);
int64_t or_join_naive(or_job *j);
/* joint order: 0 chain index (default), 1 ascending final energy (ties by index) */
void    or_set_join_order(or_job *j, int mode);
void    or_get_order(const or_job *j, int32_t *order);   /* [p] chain at each position */
void    or_update_weights(or_job *j);
int64_t or_iteration(or_job *j, int64_t S, int64_t M_total, int nthreads);
/* rounds with adjusted sweeps until h holds M_total samples (or max_rounds) */
int64_t or_iteration_adaptive(or_job *j, int64_t S, int64_t M_total, int nthreads, int max_rounds,
                              int *rounds_out, int64_t *sweeps_out);

int     or_get_L(const or_job *j);
int     or_get_p(const or_job *j);
void    or_get_weights(const or_job *j, double *W);
void    or_set_weights(or_job *j, const double *W);
void    or_get_table(const or_job *j, uint32_t *T);
void    or_get_hist(const or_job *j, int64_t *h);
void    or_get_spins(const or_job *j, int8_t *s);
void    or_get_levels(const or_job *j, int32_t *m);
void    or_get_trace(const or_job *j, int32_t *trace);
void    or_get_k(const or_job *j, int64_t *k);
int32_t or_get_carry(const or_job *j, int *valid);
uint64_t or_get_t(const or_job *j);
void    or_get_visited(const or_job *j, uint8_t *visited);
uint32_t or_get_round(const or_job *j);
int64_t or_get_last_S(const or_job *j);
int64_t or_get_last_M(const or_job *j);
void    or_get_samples(const or_job *j, int32_t *samples);
int     or_set_samples(or_job *j, int64_t S, const int32_t *samples);

/* ---- part (ii): statistical averages from a weight (Eq. reweighting2) ---- */
/* out[4b..4b+3] = E, C, F, S at betas[b] over the levels with visited[m] */
void or_thermo(int L, const double *W, const uint8_t *visited, const double *betas, int nb, double *out);

#ifdef __cplusplus
}
#endif
#endif
