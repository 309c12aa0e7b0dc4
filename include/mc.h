/*
 * mc.h -- C ABI of the GB300 library for parallel multicanonical Ising
 * chains joined by detailed balance (T. Sugihara, J. Higo, H. Nakamura,
 * "Parallelization of Markov Chain Generation and its Application to the
 * Multicanonical Method").
 *
 * One job = p independent single-spin-flip Metropolis chains on the periodic
 * L x L Ising model (Sec. 4.1, J = 1) under a common multicanonical weight
 * w(E) = exp(W(E)) (Sec. 3.1; the library stores W = ln w, Sec. 4.2).  The
 * weight-estimation loop of Sec. 2 / Sec. 3.1 is
 *
 *     mc_init -> repeat { mc_run_sweeps -> mc_join  [until h holds M_total]
 *                         -> mc_histogram (optional) -> mc_update_weights }
 *
 * Conventions shared by every call:
 *   - Energies E = -sum_<ij> s_i s_j = -2N + 4m, N = L*L; arrays indexed by
 *     energy have N + 1 entries, entry m for E = -2N + 4m.
 *   - One sample = the configuration after one single-spin-flip attempt;
 *     sites are visited in typewriter order, so a round of S sweeps is
 *     M = S*N samples per chain.
 *   - Random numbers are Philox4x32-10 with key = seed; every draw has a
 *     fixed counter, so results do not depend on launch shape, GPU or run.
 *   - Spins are bit-packed: row y of chain c is ceil(L/32) uint32 words at
 *     [(c*L + y)*ceil(L/32)]; bit x%32 of word x/32 is site (x, y), 1 = +1.
 *   - All pointers in this header are HOST pointers owned by the caller and
 *     only read or written during the call, unless stated otherwise.  The
 *     job owns all its device memory.  Work is queued on the job's CUDA
 *     stream; calls that return data synchronise that stream.
 *   - A job handle is not thread-safe: use one handle per host thread.
 *   - Every call returns MC_OK or a negative status; mc_last_error() gives a
 *     message for the calling thread.  Nothing throws across the ABI.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_EINVAL (-1)   /* bad argument (size, range, null pointer) */
#define MC_ENOMEM (-2)   /* device or host allocation failed */
#define MC_ECUDA (-3)    /* a CUDA call failed (message has the CUDA error) */
#define MC_ESTATE (-4)   /* call out of order (e.g. mc_join without a round) */
#define MC_ETIMEOUT (-5) /* reserved: no call waits on the device without a bound */

typedef struct mc_job mc_job;

typedef struct mc_info {
  int L, N, n_chains, words_per_row;
  uint64_t seed;
  uint64_t attempts_per_chain; /* attempts each chain has made since mc_init */
  uint32_t rounds_joined;      /* joints done so far */
  int64_t last_sweeps;         /* sweeps of the most recent round */
  int round_pending;           /* 1 between mc_run_sweeps and mc_join */
  int carry_valid;             /* 0 until the first joint */
  int carry_energy;            /* energy passed on to the next round's chain 0 */
  int64_t last_joined;         /* samples kept by the most recent joint */
  int64_t last_rejected;       /* chains of the most recent joint with none kept */
  int64_t last_mismatch;       /* chains whose speculated joint input was wrong */
  int64_t last_passes;         /* resolution passes of the most recent joint */
  int64_t last_searched;       /* samples replayed while resolving */
  int64_t total_joined;        /* samples kept by all joints of the job */
  int placement;               /* 0: lattice in registers, 1: in shared memory, 2: in global memory */
  int chains_per_warp, warps_per_block;
  size_t device_bytes;         /* device memory held by the job */
  int64_t last_scanned;        /* chains the exact scan settled (0: speculation sufficed) */
  int segments;                /* checkpoint segments of the most recent whole-sweep round */
  int segment_sweeps;          /* sweeps per segment of that round */
} mc_info;

/* Create a job: Sec. 2 step 1 (h = 0, initial configurations C_1) and
 * Sec. 3.1 (w^(1) = 1, i.e. W = 0).  4 <= L <= 128 with L % 4 == 0;
 * 1 <= n_chains <= 2^24; start 0 = all spins up, 1 = random (Philox
 * counter (q>>2, 0, chain, 2), word q&3 holds linear sites 32q..32q+31).
 * Allocates all device memory of the job on the current device.  On error
 * *out is NULL. */
int mc_init(int L, int n_chains, uint64_t seed, int start, mc_job **out);

/* Release the job and its device memory (NULL is accepted). */
void mc_free(mc_job *job);

/* Queue the job's work on this CUDA stream (cudaStream_t passed as void*;
 * NULL restores the job's own stream).  The caller keeps ownership. */
int mc_set_stream(mc_job *job, void *cuda_stream);

/* Enable (1) or disable (0) the per-sweep energy trace (int32 per chain per
 * sweep, kept in device memory; read with mc_get_trace).  Default off. */
int mc_set_trace(mc_job *job, int enabled);

/* Sec. 2 step 2: every chain makes n_sweeps * N single-spin-flip Metropolis
 * attempts under the current weight, continuing from its own last
 * configuration (chains are never replaced).  Asynchronous on the job's
 * stream.  MC_ESTATE if the previous round has not been joined.
 * n_sweeps >= 1 and n_sweeps * N < 2^34. */
int mc_run_sweeps(mc_job *job, int64_t n_sweeps);

/* Sec. 2 step 2 with M_node = n_attempts, which need not be whole sweeps
 * (Fig. 2 uses M_node = 100 < N at L = 20): attempt t of a chain (counted
 * from mc_init) visits site t mod N, so the typewriter order simply
 * continues across rounds.  Whole sweeps from a sweep boundary take the
 * mc_run_sweeps path; any other round (and any mc_run_sweeps while the
 * chains are inside a sweep) runs one thread per chain on its lattice in
 * global memory (meant for short rounds) and records the level of every
 * sample (p * n_attempts int32, see mc_set_partial_record), from which
 * mc_join applies the serial rule chain by chain, each chain's samples
 * tested in parallel; rounds too large to record are joined by replaying
 * each chain in one thread.  No trace is recorded for such a round, and
 * mc_batch_run refuses jobs inside a sweep.  1 <= n_attempts < 2^34.
 * Asynchronous; MC_ESTATE if the previous round has not been joined. */
int mc_run_attempts(mc_job *job, int64_t n_attempts);

/* Largest whole-sweep round (p * M samples) whose levels generation records,
 * 2 bytes a sample, for the joint to read instead of replaying the chains
 * from checkpoints (performance and memory only: both give the serial
 * rule's result).  The default is 2^33 (16 GiB of record); max_samples < 0
 * restores it, 0 turns the record off.  The record holds p rounded up to a
 * multiple of 32 chains.
 * Rounds of mc_batch_run are not recorded.  MC_ESTATE while a round is
 * pending. */
int mc_set_round_record(mc_job *job, int64_t max_samples);

/* Largest record (p * n_attempts entries, int32 each) that a round of
 * mc_run_attempts keeps for its joint; larger rounds are joined by serial
 * replay (performance and memory only: both give the serial rule's result).
 * max_entries < 0 restores the default 2^26.  MC_ESTATE while a round is
 * pending. */
int mc_set_partial_record(mc_job *job, int64_t max_entries);

/* Sec. 2 steps 3-5 for the last round: chain i (in order; see
 * mc_set_join_order) keeps its samples from the first one that passes the
 * Metropolis test against the energy passed on by the chains before it
 * (chain 0: by the previous round; in the job's first round chain 0 is kept
 * whole); a chain with no such sample keeps nothing and passes on what it
 * received.  Kept samples are added to h.  The serial rule is evaluated in
 * parallel: speculative searches over the round's samples (read from its
 * record, or replayed from lattice checkpoints), resolution passes, an exact
 * scan over per-level summaries when speculation does not settle (a
 * recorded round goes straight to it when the job's previous joint rejected
 * more than p/16 chains); the result is that of the serial rule.
 * Asynchronous; if joined_len is not NULL the call synchronises and stores
 * the number of samples kept in this round.  MC_ESTATE without a pending
 * round. */
int mc_join(mc_job *job, int64_t *joined_len);

/* The control of Sec. 5 / Fig. 2: concatenate the last round's chains whole,
 * without the detailed-balance test at the joints.  Same contract as
 * mc_join. */
int mc_join_naive(mc_job *job, int64_t *joined_len);

/* Copy the total histogram h(E) of the joined chain for the current weight
 * (int64, n_bins must be N + 1) into out.  Synchronises. */
int mc_histogram(mc_job *job, int64_t *out, int n_bins);

/* Sec. 3.1 Eq. (new_weight) in logarithms (Sec. 4.2): W(E) -= ln h(E) where
 * h(E) > 0, unchanged elsewhere; then h = 0 and the acceptance-threshold
 * table is rebuilt.  MC_ESTATE while a round is pending.  Asynchronous. */
int mc_update_weights(mc_job *job);

/* One weight iteration (Sec. 2 step 6, then Sec. 3.1): rounds of n_sweeps
 * sweeps, each joined, until the iteration's histogram holds m_total
 * samples (at least one round; at most max_rounds), then mc_update_weights.
 * adapt != 0 adjusts M_node as step 6 allows: after a round that leaves h
 * short, the next round has ceil(remaining * S_last / joined_last) sweeps,
 * clamped to [1, n_sweeps] (n_sweeps if the last round kept nothing).
 * *joined (may be NULL) = samples kept, *rounds (may be NULL) = rounds run.
 * Synchronises after every round (the loop needs each joined length). */
int mc_iteration(mc_job *job, int64_t n_sweeps, int64_t m_total, int adapt, int max_rounds,
                 int64_t *joined, int *rounds);

/* W = ln w (double, n = N + 1).  mc_set_weights rebuilds the thresholds;
 * MC_ESTATE while a round is pending.  mc_get_weights synchronises. */
int mc_get_weights(mc_job *job, double *out, int n);
int mc_set_weights(mc_job *job, const double *w, int n);

/* How the joint resolves wrong speculations (performance only: every
 * policy gives the serial rule's result).  Rounds of at most
 * scan_max_samples samples (all chains; < 0: the default 2e10) run
 * passes_before_scan speculative passes, then the summary replay and the
 * exact scan if chains are still pending, then passes_before_scan passes
 * more; larger rounds run passes_without_scan passes; whatever is left goes
 * to the one-block fallback.  Passes in 0..64 (defaults 2 and 10).
 * MC_ESTATE while a round is pending. */
int mc_set_join_policy(mc_job *job, int64_t scan_max_samples, int passes_before_scan, int passes_without_scan);

/* Length of the checkpoint segments the joint replays (performance only:
 * every length gives the serial rule's result).  Generation stores each
 * chain's lattice every C sweeps; every replay of the joint (Sec. 2 step 4:
 * the search for a chain's first accepted sample, the summary of its
 * levels, the count of its discarded prefix) runs one segment per GPU lane,
 * so the segment length bounds the joint's critical path.  The library
 * aims at segments of about `samples` attempts (whole sweeps; 0 restores
 * the default of 2^16), keeps at least min(32, S) segments and at most
 * 2^24 samples per segment, and takes fewer, longer segments where their
 * checkpoints would exceed 4 GiB.  mc_get_info reports the choice of the
 * last round.  MC_EINVAL for samples < 0, MC_ESTATE while a round is
 * pending. */
int mc_set_segment_samples(mc_job *job, int64_t samples);

/* Checkpoint / resume (no counterpart in the paper).  mc_save writes the
 * job's whole resumable state -- L, n_chains, seed, start, join order,
 * attempts per chain, rounds joined, the carry, the bit-packed spins, W,
 * the current iteration's histogram h and the visited mask -- to a file
 * (MC_ESTATE while a round is pending; MC_EINVAL if the file cannot be
 * written).  mc_load creates a new job on the current device from such a
 * file (MC_EINVAL for a missing, foreign or truncated file, before any CUDA
 * call); continuing it gives exactly the results the saved job would have
 * given.  Launch shapes and traces are not saved.  Both synchronise. */
int mc_save(mc_job *job, const char *path);
int mc_load(const char *path, mc_job **out);

/* Order of the chains at the joint (Sec. 2 steps 3-5).  mode 0 (default):
 * chain index.  mode 1: energy-ordered joining, which the end of Sec. 2
 * proposes to raise the acceptance at the joints and leaves unspecified --
 * here the chains are joined in ascending order of the energy of their last
 * generated configuration, equal energies by chain index; the joint's
 * uniforms keep their chain's index.  It changes which samples are kept (a
 * different, still exact, dynamics).  MC_EINVAL for another mode, MC_ESTATE
 * while a round is pending.  mc_get_order: out[q] = chain at position q of
 * the last joint (n = n_chains; synchronises). */
int mc_set_join_order(mc_job *job, int mode);
int mc_get_order(mc_job *job, int32_t *out, int n);

/* Levels the weight iteration has visited: out[m] = 1 once a weight update
 * (mc_update_weights) saw h[m] > 0, else 0; n = N+1.  These are the
 * energies the statistical averages sum over.  mc_set_visited restores a
 * saved mask (nonzero = 1; MC_ESTATE while a round is pending).  Both
 * synchronise. */
int mc_get_visited(mc_job *job, uint8_t *out, int n);
int mc_set_visited(mc_job *job, const uint8_t *in, int n);

/* Part (ii) of the paper (Sec. 3.2, Eq. reweighting2; quantities of
 * Sec. 4.1): statistical averages of the Ising model at inverse
 * temperatures betas[0..n_beta-1] (each > 0, 1 <= n_beta <= 65535) from the
 * job's current weight, with the density of states taken as
 * D(E) ~ 1/w(E) = e^{-W(E)} over the visited levels and normalised to 2^N
 * states: out[4b + 0..3] = E = <H>, C = beta^2 (<H^2> - <H>^2),
 * F = -ln Z / beta, S = beta (E - F) (J = k_B = 1).  Evaluated in FP64
 * relative to the largest exponent; deterministic.  Host arrays;
 * synchronises. */
int mc_thermo(mc_job *job, const double *betas, int n_beta, double *out);

/* Acceptance thresholds, planar: out[a*(N+1) + m] for the move from level m
 * to m + a - 2 (a = number of aligned neighbours), n = 5*(N+1).  A uniform
 * u is accepted iff u <= threshold.  Synchronises. */
int mc_get_table(mc_job *job, uint32_t *out, int n);

/* Bit-packed spins of all chains, n_words = n_chains * L * ceil(L/32).
 * mc_set_spins masks unused high bits, recomputes the energies and is
 * refused (MC_ESTATE) while a round is pending.  Both synchronise. */
int mc_get_spins(mc_job *job, uint32_t *out, size_t n_words);
int mc_set_spins(mc_job *job, const uint32_t *in, size_t n_words);

/* Current energy of every chain (n = n_chains).  Synchronises. */
int mc_get_energies(mc_job *job, int32_t *out, int n);

/* Energy after each sweep of the last round, out[s*n_chains + c];
 * n >= last_sweeps * n_chains; MC_ESTATE if the trace was off.  Syncs. */
int mc_get_trace(mc_job *job, int32_t *out, size_t n);

/* Energy after each sweep of the last round for one chain: out[s] for
 * s < last_sweeps (n >= last_sweeps).  A strided device-to-host copy of
 * the same buffer mc_get_trace reads; MC_EINVAL for a chain out of range,
 * MC_ESTATE if the trace was off.  Synchronises. */
int mc_get_trace_chain(mc_job *job, int chain, int32_t *out, size_t n);

/* Result of the last joint: k[i] = first kept sample of chain i (1..M) or 0
 * if none was kept; offsets[i] = position of chain i's kept segment in the
 * joined chain of that round.  Either pointer may be NULL.  Synchronises. */
int mc_get_join(mc_job *job, int64_t *k, int64_t *offsets, int n);

/* Job state and statistics of the last joint.  Synchronises. */
int mc_get_info(mc_job *job, mc_info *info);

/* Choose how chains map to the GPU (placement 0 = lattice rows in
 * registers, L <= 32; 1 = shared memory; 2 = global memory with the rows
 * streamed through registers, L = 96, 100, 128 -- the default at L = 96,
 * where the threshold table then fits in shared memory, and with more than
 * 8 chains a warp at L = 100, 128; the joint's replays of such a job use
 * shared memory), chains per warp 1..32, warps per block 1..4.  The
 * dynamics and all results are independent of this choice. */
int mc_set_launch_shape(mc_job *job, int placement, int chains_per_warp, int warps_per_block);

/* `iterations` weight iterations (round of n_sweeps sweeps, joint, weight
 * update -- Sec. 2 and Eq. new_weight) of n_jobs independent jobs, queued on
 * the first job's stream.  mode 0: one generation launch per job and round;
 * mode 1: one fused generation launch per round for all jobs whose lattice
 * size has a fused form (L = 8, 16, 24, 32 in registers; 24, 32, 48, 64 in
 * shared memory; up to 8 jobs), each with the shape mc_batch_autotune chose
 * for it, or by rule (full warps; shared memory at L = 24, 32, 48, 64), the
 * others keep their own launch; mode 2: mode 1 with the whole loop captured
 * once as a CUDA graph and launched.  The
 * chains, and so every result, are the same in all modes.  Synchronises.
 * No round may be pending on any job.  The paper has no counterpart: a
 * scheduling form of running independent weight estimations together. */
int mc_batch_run(mc_job **jobs, int n_jobs, int iterations, int64_t n_sweeps, int mode);

/* Launch shapes of the jobs in a fused batch launch (mc_batch_run modes 1
 * and 2), by measurement: each job's candidate shapes (lattice in registers
 * or shared memory where the fused kernel has that form, 4..32 chains per
 * warp, lane groups of 4 for shared-memory lattices above L = 32 with at
 * most 8 chains a warp) are tried in turn, longest chains first, each trial
 * timed as one whole fused generation launch of all n_jobs jobs of
 * probe_sweeps sweeps on scratch copies of their chains (CUDA events; the
 * jobs' own chains do not move); only combinations whose blocks are all
 * resident on the GPU at once are considered, and a change is kept if it
 * shortens the launch by more than 1 %.  The result is stored in every job
 * and used by mc_batch_run; with use_cache != 0 a result found earlier for
 * the same device and the same (L, n_chains) list is reused without timing.
 * The chains, and so every result, are the same under any shape.  The paper
 * has no counterpart (launch tuning).  1 <= n_jobs <= 8; allocates and frees
 * temporary device memory; synchronises.  mc_batch_shape reports the shape
 * a job gets in a fused launch and returns 1 if it has a fused form (0 if it
 * keeps its own launch), or a negative status. */
int mc_batch_autotune(mc_job **jobs, int n_jobs, int64_t probe_sweeps, int use_cache);
int mc_batch_shape(mc_job *job, int *placement, int *chains_per_warp, int *warps_per_block);

/* Pick the launch shape by measurement: every supported combination of
 * placement, chains per warp and warps per block is timed on a scratch copy
 * of the job's chains (probe_sweeps sweeps each, CUDA events on the job's
 * stream; the job's own chains do not move) and the fastest is kept for the
 * job.  With use_cache != 0 a shape found earlier for the same device, L and
 * n_chains is reused without timing.  The chosen shape is returned through
 * the (nullable) out pointers.  The paper has no counterpart (launch tuning).
 * Allocates and frees temporary device memory; synchronises. */
int mc_autotune(mc_job *job, int64_t probe_sweeps, int use_cache, int *placement,
                int *chains_per_warp, int *warps_per_block);

/* Wait for the job's queued work. */
int mc_sync(mc_job *job);

/* One round of chain generation (what mc_run_sweeps does for a job) on
 * caller-owned DEVICE buffers, without allocating any device memory.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * while they run (a host function inside a stream, a process whose device
 * memory is fully reserved up front, a pool that forbids foreign
 * allocations).
 *   d_spins   [n_chains][L][ceil(L/32)] uint32, read and overwritten;
 *   d_levels  [n_chains] int32, level m = (E + 2N)/4 of each lattice, updated;
 *   d_weights [N+1] double, W = ln w (read);
 *   d_hist    [N+1] int64, zeroed, then the number of this round's samples
 *             at each level;
 *   t0        attempts each chain made before this round (multiple of 4),
 *             so that round r of a job started at t0 = 0 uses t0 = r*M.
 * Work is queued on cuda_stream (NULL = legacy default stream); returns
 * without waiting.  The launch shape is the library's default for L and
 * n_chains (see mc_set_launch_shape; at L = 96, and at L = 100, 128 with
 * more than 8 chains a warp, the lattices are swept in place in d_spins).
 * Scratch: the threshold table lives in one fixed
 * 320 KiB device array (L <= 128) that the library holds on every device
 * until the process exits; L > 128 is rejected with MC_EINVAL.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress)
 * and must therefore come before any stream capture on that device.  All
 * calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller. */
int mc_generate_noalloc(int L, int n_chains, uint64_t seed, uint64_t t0, int64_t n_sweeps,
                        uint32_t *d_spins, int32_t *d_levels, const double *d_weights,
                        int64_t *d_hist, void *cuda_stream);

/* Failure injection for tests of the error paths (no counterpart in the
 * paper).  After `after` more device allocations by this library (job state,
 * checkpoint segments, traces, statistical-average buffers; those a server
 * makes when it admits a job count too), the next one fails on the host
 * before any CUDA call, as an out-of-memory would, and the calling entry
 * point returns MC_ENOMEM after releasing what it had allocated; later
 * allocations succeed again.  after < 0 disarms it.  Process-wide.
 * mc_live_allocations: device allocations this library holds right now (a
 * leak check: it returns to its old value once the jobs are freed). */
int mc_inject_alloc_failure(int64_t after);
int64_t mc_live_allocations(void);

/* Number of kernels this library has launched since it was loaded. */
uint64_t mc_kernel_launches(void);

/* Message of the last failed call on this thread ("" if none). */
const char *mc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
