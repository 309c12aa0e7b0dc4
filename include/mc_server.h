/* Serving: a request loop that runs many multicanonical weight-estimation
 * jobs (Sec. 3: W^(n) -> W^(n+1) by Eq. new_weight, each iteration one
 * round of Sec. 2 steps 2-4) side by side on one GPU.
 *
 * The paper runs one job on many processes; it has no serving layer.  Here
 * jobs of different lattice sizes arrive over time.  A job is admitted when
 * a slot is free and its device memory fits in the server's budget
 * (first fit in arrival order); its lattices, counters, W(E) and histogram
 * stay resident on the device until it finishes.  Every slot has its own
 * CUDA stream, so the work of admitted jobs overlaps on the device; a host
 * thread of the server keeps each slot at most two iterations ahead of the
 * GPU and admits new jobs as slots and memory free up.  Each job runs with
 * its chains packed into as few warps as possible (a round takes as long
 * as with the chains spread out, since one chain's latency sets it), so
 * that concurrent jobs share the SMs.  The dynamics of a
 * job do not depend on what else runs: its result is identical to the same
 * job run alone through mc.h.
 *
 * Thread safety: every call below may be made from any host thread.
 */
#ifndef MC_SERVER_H
#define MC_SERVER_H

#include "mc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mc_server mc_server;

/* One weight-estimation job: mc_init(L, n_chains, seed, start), then
 * `iterations` times { mc_run_sweeps(sweeps); mc_join; mc_update_weights }. */
typedef struct mc_jobspec {
  int L;              /* 4 <= L <= 128, L % 4 == 0 */
  int n_chains;       /* >= 1 */
  uint64_t seed;      /* Philox key of the job */
  int start;          /* 0 all up, 1 random */
  int iterations;     /* weight iterations, >= 1 */
  int64_t sweeps;     /* sweeps per chain per iteration, >= 1 */
} mc_jobspec;

typedef struct mc_jobstats {
  int status;           /* MC_OK, or the error code that ended the job */
  int slot;             /* slot (stream) it ran on, -1 if never admitted */
  double t_submit;      /* seconds on the server clock (mc_server_clock) */
  double t_admit;
  double t_done;
  int64_t attempts;     /* n_chains * iterations * sweeps * N */
  int64_t joined;       /* kept samples over all iterations */
  uint64_t device_bytes;/* device memory the job held */
} mc_jobstats;

typedef struct mc_server_info {
  int max_slots;
  int queued, active, finished;   /* finished: done and not yet collected */
  uint64_t budget_bytes, bytes_in_use, peak_bytes;
  int peak_active;
  uint64_t admitted, completed;
} mc_server_info;

/* Device memory a job of this shape holds while resident (what admission
 * charges against the budget), trace off. */
uint64_t mc_job_device_bytes(int L, int n_chains, int64_t sweeps);

/* Create a server on the current device with `max_slots` (1..64) slots and
 * a device-memory budget in bytes; starts its host thread.  MC_EINVAL for
 * bad arguments, MC_ECUDA / MC_ENOMEM on device errors. */
int mc_server_create(uint64_t budget_bytes, int max_slots, mc_server **out);

/* Queue a job; *id identifies it in mc_server_poll / mc_server_wait.
 * MC_EINVAL for a bad spec, MC_ENOMEM if the job alone exceeds the budget,
 * MC_ESTATE after mc_server_free started. */
int mc_server_submit(mc_server *srv, const mc_jobspec *spec, uint64_t *id);

/* *done = 1 when the job has finished (successfully or not). MC_EINVAL for
 * an unknown (or already collected) id. */
int mc_server_poll(mc_server *srv, uint64_t id, int *done);

/* Block until the job has finished, then collect it: W_out (may be NULL
 * when n == 0) receives its final weights W(E) (n must be N+1 otherwise)
 * and *stats (may be NULL) its record; the id is released.  Returns the
 * job's status (MC_OK or its error), or MC_EINVAL for an unknown id or a
 * wrong n (the job is then not collected). */
int mc_server_wait(mc_server *srv, uint64_t id, double *W_out, int n, mc_jobstats *stats);

/* Counters of the server (a snapshot). */
int mc_server_get_info(mc_server *srv, mc_server_info *info);

/* Seconds since the server was created (steady clock). */
double mc_server_clock(mc_server *srv);

/* Stop accepting jobs, cancel the queued ones that were not admitted yet,
 * let the admitted ones finish, then free every resource (uncollected
 * results are dropped).  NULL is accepted. */
void mc_server_free(mc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* MC_SERVER_H */
