/*
 * tauleap.h -- C ABI of the B300 batched stochastic-simulation engine.
 *
 * The engine runs many independent stochastic simulations of one
 * mass-action reaction network at once, each with its own kinetic constants
 * and initial molecule counts.  This is the parameter-sweep workload of the
 * paper's "Aims and motivation" section, where all simulations of a sweep are
 * mutually independent (Methods, last paragraph).  One CUDA thread group
 * advances one simulation.
 *
 * Method, per simulation (Methods section: X(t) is a continuous-time Markov
 * chain over molecule counts, sampled by Gillespie's algorithm):
 *   - tau-leaping with the step-size selection of Cao, Gillespie & Petzold
 *     (J. Chem. Phys. 124, 044109, 2006) and the critical-reaction rule of
 *     Cao, Gillespie & Petzold (J. Chem. Phys. 123, 054104, 2005),
 *   - falling back to blocks of exact SSA steps (direct method) when the
 *     admissible leap is shorter than a few mean reaction times,
 *   - or exact SSA only (SSA_MODE_EXACT),
 *   - or tau-leaping with Langevin (normal) increments for large leap means
 *     (SSA_MODE_CLE).
 * Random numbers come from Philox4x32-10 counter-based streams.  A
 * simulation's stream is keyed by (seed, global simulation index), so results
 * do not depend on batch composition, launch shape or sharding.
 *
 * Conventions
 *   - Every entry point returns SSA_OK (0) or a negative SSA_E* code.
 *     ssa_last_error() then holds a message for the calling thread.
 *   - Per-simulation failures (step cap, count overflow) are not call
 *     errors: they are reported in ssa_sim_stats.status.  The samples after
 *     a failure repeat the last valid state.
 *   - Index arrays are int32 and rates / times are IEEE double.  All
 *     arrays are dense, row-major and C-contiguous.
 *   - Handles are not shared between threads without external locking.
 *     Different handles may be used concurrently.
 *   - Any CUDA failure is reported as SSA_ECUDA with the CUDA error string.
 */
#ifndef TAULEAP_H
#define TAULEAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSA_ABI_VERSION 2

/* return codes */
#define SSA_OK 0
#define SSA_EINVAL (-1)       /* bad argument or model */
#define SSA_ENOMEM (-2)       /* the job's HBM footprint does not fit */
#define SSA_EBUSY (-3)        /* job still running (ssa_poll-based callers) */
#define SSA_ECUDA (-4)        /* CUDA runtime error */
#define SSA_EUNSUPPORTED (-5) /* option combination not built */

/* per-simulation status (ssa_sim_stats.status) */
#define SSA_STATUS_OK 0
#define SSA_STATUS_STEP_LIMIT 1   /* max_attempts leap attempts + SSA steps used */
#define SSA_STATUS_OVERFLOW 2     /* a count passed 2^31-1 or a leap drew > 2^40 */
#define SSA_STATUS_REJECT_LIMIT 3 /* max_halvings negativity retries in one leap */
#define SSA_STATUS_INVALID 4      /* the propensity sum a0 was not finite (bad rates) */

/* job / request states (ssa_poll, ssa_server_poll) */
#define SSA_JOB_QUEUED 0
#define SSA_JOB_RUNNING 1
#define SSA_JOB_DONE 2
#define SSA_JOB_FAILED 3

/* ssa_options.mode */
#define SSA_MODE_TAU_LEAP 0 /* CGP tau-leaping with critical reactions + SSA fallback */
#define SSA_MODE_EXACT 1    /* Gillespie direct method only */
#define SSA_MODE_CLE 2      /* as TAU_LEAP, but a noncritical reaction whose leap mean is >= 1000 fires
                               max(0, round(mean + sqrt(mean) z)) times, z ~ N(0,1) (chemical Langevin
                               increment, Marsaglia's polar method on the same stream); lane layout only */

/* ssa_options.precision */
#define SSA_FP64_REF 0 /* bit-identical to the FP64 reference algorithm */
#define SSA_FAST 1     /* FP32 propensities, Poisson means and sampler; FP64 clock, a0, tau' */

/* ssa_options.layout */
#define SSA_LAYOUT_AUTO 0
#define SSA_LAYOUT_WARP 1 /* one warp (32 lanes) per simulation throughout */
#define SSA_LAYOUT_LANE 2 /* one simulation per lane for SSA steps; warp-cooperative leaps */

typedef struct ssa_model *ssa_model_t;
typedef struct ssa_job *ssa_job_t;

/*
 * A reaction network (Methods: reactions fire between species and change
 * the state vector X of molecule counts).  This is reaction-major CSR.
 * Reaction j consumes react_coef[e] molecules of species react_species[e]
 * for e in [react_ptr[j], react_ptr[j+1]), and produces products in the same
 * way.  The reaction order (sum of reactant coefficients) must be <= 2.
 * Coefficients are >= 1, and product coefficients are <= 100.  A species
 * appears at most once per row.  Arrays are caller-owned and are read only
 * during ssa_load_model.
 */
typedef struct {
    int32_t n_species;   /* N, 1..16384 */
    int32_t n_reactions; /* M, 1..16384 */
    const int32_t *react_ptr, *react_species, *react_coef;
    const int32_t *prod_ptr, *prod_species, *prod_coef;
} ssa_model_desc;

typedef struct {
    int32_t mode;         /* SSA_MODE_* (default TAU_LEAP) */
    int32_t precision;    /* SSA_FP64_REF or SSA_FAST */
    double eps;           /* CGP error-control parameter epsilon (0.03) */
    int32_t n_c;          /* critical threshold: L_j < n_c (10) */
    int32_t ssa_block;    /* SSA steps per fallback block (100) */
    double ssa_factor;    /* fall back when tau' < ssa_factor / a0 (10) */
    int32_t max_halvings; /* negativity retries per leap (64) */
    int32_t layout;       /* SSA_LAYOUT_* (AUTO) */
    int64_t max_attempts; /* per-simulation cap on leap attempts + SSA steps (1e8) */
    int32_t block_warps;  /* warps per CTA, 0 = automatic */
    int32_t sims_per_warp; /* lane layout: lanes of a warp that own a simulation (1..32, 0 = 32) */
    int32_t ctas_per_sm;   /* lane layout: resident CTAs per SM (0 = as many as fit); with fewer, the
                              shared-memory carve-out is sized to them and the rest of each SM's
                              on-chip memory serves as L1 cache for the rate constants */
    int32_t reg_cap;       /* lane layout: register budget of the kernel build: 0 = up to 255 registers per
                              thread, 1 = the build limited to 168 so that three CTAs of at most 4 warps
                              fit per SM when shared memory allows (block_warps must be <= 4) */
    uint64_t *work_counters; /* optional DEVICE array of SSA_WORK_COUNTERS uint64 that the launch adds
                                its work to (lane layout, tau-leaping modes; see below); NULL = none */
} ssa_options;

/* Work the method performed in a launch, for measurement (ssa_options.
 * work_counters; the counts are added to the array, which the caller
 * clears).  Exact SSA events and leap attempts are in ssa_sim_stats.
 * Counted: step selections (propensities, a0, critical set and tau' of a
 * state; CGP 2006), terms of the mu / sigma^2 sums of the species that bound
 * tau' and those species, tau'' evaluations (attempts with a critical
 * reaction), Poisson means formed (noncritical reactions per attempt),
 * inversion draws and the sum of their results (cdf terms after the first),
 * PTRS draws, their iterations and their acceptance tests after the
 * squeeze (Hormann 1993).  Langevin increments are not counted. */
#define SSA_WORK_SELECTIONS 0
#define SSA_WORK_TAU_TERMS 1
#define SSA_WORK_TAU_SPECIES 2
#define SSA_WORK_TAU2 3
#define SSA_WORK_MEANS 4
#define SSA_WORK_INV_DRAWS 5
#define SSA_WORK_INV_TERMS 6
#define SSA_WORK_PTRS_DRAWS 7
#define SSA_WORK_PTRS_ITERS 8
#define SSA_WORK_PTRS_TESTS 9
#define SSA_WORK_COUNTERS 10

/* Per-simulation counters and status (56 bytes). */
typedef struct {
    int32_t status;    /* SSA_STATUS_* */
    int32_t reserved;
    int64_t leaps;     /* accepted tau-leaps */
    int64_t rejected;  /* leap attempts undone because a count went negative */
    int64_t ssa_steps; /* reactions fired by exact SSA steps */
    int64_t firings;   /* total reaction firings (leap Poisson counts + SSA events) */
    int64_t attempts;  /* random-stream attempt counter at exit */
    double t_final;    /* simulated time reached */
} ssa_sim_stats;

/* Fill *opts with the defaults listed above. */
void ssa_default_options(ssa_options *opts);

/* Validate a network and upload it to the current CUDA device.  On success
 * *out is a handle that owns the device copy; free it with ssa_free_model.
 * Fails with SSA_EINVAL for order > 2, a species index out of range, a
 * coefficient out of range, or a repeated species in one row. */
int ssa_load_model(const ssa_model_desc *desc, ssa_model_t *out);
int ssa_free_model(ssa_model_t model);
int ssa_model_info(ssa_model_t model, int32_t *n_species, int32_t *n_reactions);

/* Enqueue n_sims simulations on `stream` (a cudaStream_t, NULL = legacy
 * default stream).  All array arguments are DEVICE pointers on the model's
 * device, caller-owned, and must stay valid until the stream reaches this
 * work:
 *   params       [n_sims][M] double  stochastic rate constants c_j (>= 0)
 *   x0           [n_sims][N] int32   initial counts (>= 0)
 *   sample_times [n_samples] double  non-decreasing, within [0, t_end]
 *   samples      [n_sims][n_samples][N] int32 output: X at each sample time
 *   stats        [n_sims] ssa_sim_stats output (may be NULL)
 * Simulation r uses the random stream of global index sim_offset + r
 * (sim_offset + n_sims <= 2^32).  Returns as soon as the launch is queued;
 * the function allocates a small stream-ordered work counter and frees it
 * on the same stream; in fast mode (lane layout) it also allocates the FP32
 * images of params (4 * n_sims * M bytes), forms them with a conversion
 * kernel on `stream` and frees them there.  The first launch on each device also copies the
 * logarithm table (6 KB, built on the host) into device memory on `stream`
 * and waits for that copy, so make one launch on a device before capturing
 * launches into a CUDA graph.  The library keeps per-device state for the
 * life of the process (that table); after a cudaDeviceReset the device must
 * not be used through this library again. */
int ssa_simulate_dev(ssa_model_t model, int64_t n_sims, int64_t sim_offset,
                     const double *params, const int32_t *x0, double t_end,
                     const double *sample_times, int32_t n_samples, uint64_t seed,
                     const ssa_options *opts, int32_t *samples, ssa_sim_stats *stats,
                     void *stream);

/* Sweep moments instead of trajectories (the sweep post-processing of the
 * paper's "Aims and motivation": parameter sweeps summarised across
 * replicates).  Simulates like ssa_simulate_dev (same arguments, same random
 * streams, lane layout) but writes no samples array: while recording, every
 * count x of sample k, species i is added to exact integer sums S1 = sum x
 * and S2 = sum x^2 over the n_sims simulations, and the call ends with
 *   mean[k][i] = RN(RN(S1) / RN(n_sims)),
 *   var[k][i]  = RN(RN(n_sims S2 - S1^2) / RN(n_sims (n_sims - 1)))
 * (unbiased variance, 0 when n_sims < 2), DEVICE arrays [n_samples][N] of
 * double, caller-owned.  The results are fixed functions of the integer
 * sums, whatever order the simulations finish in.  This avoids the
 * n_sims * n_samples * N * 4-byte trajectory array when only moments are
 * needed.  Allocates (stream-ordered) 24 * n_samples * N bytes of
 * accumulators and frees them on `stream`.  SSA_EINVAL for n_sims < 1,
 * n_samples < 1 or null mean/var; SSA_EUNSUPPORTED with the warp layout. */
int ssa_simulate_moments_dev(ssa_model_t model, int64_t n_sims, int64_t sim_offset,
                             const double *params, const int32_t *x0, double t_end,
                             const double *sample_times, int32_t n_samples, uint64_t seed,
                             const ssa_options *opts, double *mean, double *var, ssa_sim_stats *stats,
                             void *stream);

/* Sweep histograms instead of trajectories (the same sweep post-processing):
 * simulates like ssa_simulate_dev (same arguments, same random streams, lane
 * layout) but writes no samples array; every recorded count x of sample k,
 * species i adds 1 to one bin of the cell's histogram:
 *   counts[k][i][0]          x < bin_lo (underflow),
 *   counts[k][i][1 + b]      bin_lo + b bin_width <= x < bin_lo + (b+1) bin_width,
 *                            b = 0..n_bins-1,
 *   counts[k][i][n_bins + 1] x >= bin_lo + n_bins bin_width (overflow).
 * counts is a DEVICE array [n_samples][N][n_bins + 2] of uint64, caller-owned;
 * the launch ADDS to it (zero it first, or accumulate several batches), so
 * every cell's bins sum to the simulations recorded into it.  The counts are
 * exact integers whatever order simulations finish in.  SSA_EINVAL for
 * n_bins < 1, bin_width < 1, n_samples < 1, a null counts array or more
 * than 2^34 bins; SSA_EUNSUPPORTED with the warp layout. */
int ssa_simulate_histograms_dev(ssa_model_t model, int64_t n_sims, int64_t sim_offset,
                                const double *params, const int32_t *x0, double t_end,
                                const double *sample_times, int32_t n_samples, uint64_t seed,
                                const ssa_options *opts, int32_t bin_lo, int32_t bin_width, int32_t n_bins,
                                uint64_t *counts, ssa_sim_stats *stats, void *stream);

/* Deterministic counterpart of a sweep: the reaction-rate equations (the
 * paper's Methods section: for abundant species the state follows
 * dX/dt = sum_j nu_j a_j(X) with continuous X; a 2X reaction has the
 * mean-field propensity c x^2/2), one ODE system per parameter set,
 * integrated by the Dormand-Prince 5(4) pair with a power-of-two step
 * controller: h starts at sample_times[n_samples-1] / 64; a step is accepted
 * when max_i |e_i| / (atol + rtol max(|x_i|, |x_new_i|)) <= 1, after which h
 * doubles when that error is <= 2^-6 (unless the step was shortened to land
 * on a sample time); a rejected step halves the step it tried.  DEVICE
 * arrays: params [n_sims][M], x0 [n_sims][N] int32 (initial amounts),
 * sample_times [n_samples] non-decreasing and >= 0, out [n_sims][n_samples][N]
 * double, stats [n_sims] (may be NULL; leaps = accepted steps, rejected =
 * rejected steps; status STEP_LIMIT after max_steps steps, INVALID for a
 * non-finite state, after which the samples repeat the last state).
 * SSA_EINVAL for rtol or atol not finite and > 0 or max_steps < 1. */
int ssa_integrate_rre_dev(ssa_model_t model, int64_t n_sims, const double *params, const int32_t *x0,
                          const double *sample_times, int32_t n_samples, double rtol, double atol,
                          int64_t max_steps, double *out, ssa_sim_stats *stats, void *stream);

/* Same as ssa_simulate_dev, for callers that cannot allocate device memory
 * (for example code that runs inside an allocator's callbacks, or programs
 * that reserve all device memory up front).  It calls no cudaMalloc,
 * cudaFree or other allocating routine; in fast mode the kernel converts
 * each rate constant to FP32 where it uses it (the same values as the
 * staged images of ssa_simulate_dev).  The one piece of scratch memory the
 * kernel needs, its 8-byte work counter, lives in a 256-byte static device
 * array that every GPU loading this library keeps until process exit; a
 * launch needing more scratch than that is rejected with SSA_EINVAL.  Each
 * call looks up the array's device address on the model's device (this
 * allocates nothing); the first call on a device also uploads the logarithm
 * table as ssa_simulate_dev does, so make that first call before any stream
 * capture.  All calls share the array: the
 * counter is cleared on `stream` before each launch, and calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it and must be serialised by the caller.  The paper has no counterpart to
 * this entry point. */
int ssa_simulate_dev_noalloc(ssa_model_t model, int64_t n_sims, int64_t sim_offset,
                             const double *params, const int32_t *x0, double t_end,
                             const double *sample_times, int32_t n_samples, uint64_t seed,
                             const ssa_options *opts, int32_t *samples, ssa_sim_stats *stats,
                             void *stream);

/* One group of a multi-network launch: a loaded network and its batch.
 * Array members are DEVICE pointers with the layouts of ssa_simulate_dev;
 * all models must live on the same device. */
typedef struct {
    ssa_model_t model;
    int64_t n_sims;
    int64_t sim_offset;           /* global index of the group's first simulation (RNG identity) */
    const double *params;         /* [n_sims][M] */
    const int32_t *x0;            /* [n_sims][N] */
    double t_end;
    const double *sample_times;   /* [n_samples] */
    int32_t n_samples;
    int32_t reserved;
    uint64_t seed;
    int32_t *samples;             /* [n_sims][n_samples][N] output */
    ssa_sim_stats *stats;         /* [n_sims] output, may be NULL */
} ssa_group;

/* Heterogeneous batch in ONE persistent launch: lanes take simulations from
 * all groups through a single work counter, in the order the groups are
 * given (put the most expensive groups first to shorten the tail), each
 * lane running its own group's network, read from global memory.  The
 * per-warp workspace is sized for the largest network.  Results per
 * simulation are identical to ssa_simulate_dev of its group with the same
 * options and seed.  opts->precision applies to every group; the lane
 * layout is used.  Allocates (stream-ordered) the group table and the work
 * counter, in fast mode also the FP32 images of every group's params, and
 * frees them on `stream`. */
int ssa_simulate_multi_dev(int32_t n_groups, const ssa_group *groups, const ssa_options *opts, void *stream);

/* Host-buffer form.  Copies the HOST inputs to device memory that the job
 * owns and enqueues the simulation on `stream` (NULL = a stream the job
 * creates).  The inputs may be reused once this returns.  Fails with
 * SSA_ENOMEM if the job's device footprint exceeds the free HBM.  Complete the
 * job with ssa_poll / ssa_wait and ssa_fetch, then free it with
 * ssa_release_job. */
int ssa_submit_batch(ssa_model_t model, int64_t n_sims, const double *params,
                     const int32_t *x0, double t_end, const double *sample_times,
                     int32_t n_samples, uint64_t seed, const ssa_options *opts,
                     void *stream, ssa_job_t *out);

/* Non-blocking: *state = SSA_JOB_RUNNING, SSA_JOB_DONE or SSA_JOB_FAILED. */
int ssa_poll(ssa_job_t job, int32_t *state);
/* Block until the job's work is complete. */
int ssa_wait(ssa_job_t job);
/* Wait for the job, then copy its results to HOST buffers:
 * samples [n_sims][n_samples][N] int32, stats [n_sims] (either may be NULL). */
int ssa_fetch(ssa_job_t job, int32_t *samples, ssa_sim_stats *stats);
/* Wait for the job and free everything it owns. */
int ssa_release_job(ssa_job_t job);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of simulation requests                   */
/* ------------------------------------------------------------------ */
/* A request is one network and one batch of simulations, with HOST inputs.
 * A dispatcher thread admits queued requests in arrival order whenever one
 * of n_streams stream slots is free and the request's device footprint
 * (inputs + outputs) fits the HBM budget still unused; the requests
 * admitted together run as one multi-network launch, and launches on
 * different slots overlap on the device.  Results stay resident in device
 * memory until ssa_server_fetch copies them out and frees them, returning
 * their bytes to the budget (a client that never fetches keeps its memory).
 * Simulation r of a request uses the random stream (request seed, r), so a
 * request's result is the same alone and in any mix. */
typedef struct ssa_server *ssa_server_t;

typedef struct {
    int64_t max_device_bytes; /* HBM budget for admitted requests; 0 = 80% of free memory at creation */
    int32_t n_streams;        /* launches in flight (1..16), default 4 */
    int32_t max_batch;        /* requests per launch (1..256), default 16 */
    ssa_options opts;         /* applied to every request; default precision SSA_FAST */
} ssa_server_config;

typedef struct {
    int32_t state;      /* SSA_JOB_QUEUED, _RUNNING, _DONE or _FAILED */
    int32_t batch_size; /* requests in the launch that ran this one */
    double t_submit;    /* seconds since server creation */
    double t_admit;     /* -1 until admitted */
    double t_done;      /* -1 until the launch completed */
} ssa_request_info;

void ssa_server_default_config(ssa_server_config *cfg);
/* Create a server on the current device (models submitted to it must live there). */
int ssa_server_create(const ssa_server_config *cfg, ssa_server_t *out);
/* Queue a request; inputs are copied before the call returns.  *ticket
 * identifies it.  SSA_ENOMEM if its footprint exceeds the whole budget. */
int ssa_server_submit(ssa_server_t srv, ssa_model_t model, int64_t n_sims, const double *params,
                      const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                      uint64_t seed, int64_t *ticket);
int ssa_server_poll(ssa_server_t srv, int64_t ticket, ssa_request_info *info);
int ssa_server_wait(ssa_server_t srv, int64_t ticket, ssa_request_info *info);
/* Wait for the request, copy samples [n_sims][n_samples][N] and stats
 * [n_sims] (either may be NULL) to HOST memory, free its device memory and
 * forget the ticket. */
int ssa_server_fetch(ssa_server_t srv, int64_t ticket, int32_t *samples, ssa_sim_stats *stats);
/* Launches issued so far, requests waiting for admission, admitted bytes. */
int ssa_server_stats(ssa_server_t srv, int64_t *launches, int64_t *queued, int64_t *device_bytes_in_use);
/* Finish queued and running requests, free everything. */
int ssa_server_destroy(ssa_server_t srv);
const char *ssa_server_last_error(void);

/* ------------------------------------------------------------------ */
/* Measurement                                                           */
/* ------------------------------------------------------------------ */
/* Issue-rate microbenchmark of the current device, the denominator of the
 * simulation kernels' roofline (they are bound by FP64 and FP32 instruction
 * issue, not by memory bandwidth or tensor cores; the paper has no
 * counterpart).  Launches, on `stream`, one full-device grid in which every
 * thread runs 8 independent chains of 4,096 dependent adds (double, then
 * float; no fused multiply-add), and one warp with a single dependent chain
 * of double adds timed with the SM clock.  Writes the best of three timed
 * launches as adds per second (*fp64_adds_per_s, *fp32_adds_per_s) and the
 * SM cycles per dependent double add (*fp64_add_latency_cycles); any output
 * pointer may be NULL.  Allocates and frees a few MB of stream-ordered
 * scratch and synchronises `stream`.  SSA_ECUDA on any CUDA failure. */
int ssa_measure_issue_rates(void *stream, double *fp64_adds_per_s, double *fp32_adds_per_s,
                            double *fp64_add_latency_cycles);

/* Message describing the last failed call on this thread ("" if none). */
const char *ssa_last_error(void);
int ssa_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TAULEAP_H */
