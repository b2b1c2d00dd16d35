/*
 * fs.h -- C ABI of libflashstep: the renewal (age-dependent hazard) Bernoulli
 * tau-leaping step of SIR/SEIR on a CSR contact graph, on one GB300 GPU
 * (sm_103a). Method: FlashSpread, arXiv 2604.22092 -- Section 3 (Eqs. 1-3:
 * state (X, tau), rate decomposition, inducer influence), Section 5.1
 * (Proposition 1: stable log-normal hazard), Section 5.2 (Bernoulli
 * tau-leap), Section 5.4 (Algorithm 3: the fused step; Algorithm 2: capture
 * of b steps in a CUDA Graph), Section 5.5 (degree-aware traversal),
 * Section 5.7 (storage precision).
 *
 * General rules for every entry point
 *   - Every function returns an fs_status; FS_OK is 0. On any other value
 *     fs_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread). No C++ exception crosses this boundary.
 *   - Argument errors are detected on the host before any device work and
 *     leave every handle unchanged (FS_EINVAL).
 *   - Host arrays passed in are read during the call only; the caller keeps
 *     ownership. Device memory is allocated and owned by the library.
 *   - A CUDA error moves the handle to a failed state: the call returns
 *     FS_ECUDA and later calls on that handle return FS_ESTATE.
 *   - Handles are not thread-safe; use one handle from one thread at a time.
 *   - Node ids are the caller's (original) ids everywhere in this API. The
 *     library may relabel nodes internally; random numbers are always keyed
 *     by original ids, so results never depend on the internal layout.
 *
 * Conventions
 *   compartments: FS_S = 0, FS_E = 1, FS_I = 2, FS_R = 3 (SIR leaves E empty)
 *   CSR: row i lists the in-neighbours j of node i (each j -> i edge once);
 *        row_ptr int64[n+1] nondecreasing with row_ptr[0] = 0,
 *        col_ind int32[row_ptr[n]] with 0 <= col_ind[e] < n.
 *        Undirected graphs list every edge in both rows.
 *   uniforms: u = (w >> 8) * 2^-24 with w = word (replicate mod 4) of
 *        Philox4x32-10(counter = (node, step, replicate / 4, 0),
 *                      key = (seed mod 2^32, seed / 2^32)); a node fires
 *        when u < p, p = 1 - exp(-lambda * dt) computed in FP32.
 */
#ifndef FLASHSTEP_FS_H
#define FLASHSTEP_FS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_EINVAL = 1,        /* invalid argument (detected before device work)   */
    FS_ENOMEM = 2,        /* device or host allocation failed / over budget   */
    FS_ECUDA = 3,         /* a CUDA call or kernel failed                      */
    FS_ETIMEOUT = 4,      /* a bounded device wait ran out                     */
    FS_EBUSY = 5,         /* the object is still referenced                    */
    FS_ESTATE = 6,        /* the handle is in a failed state                   */
    FS_EUNSUPPORTED = 7   /* valid request this build does not implement       */
} fs_status;

enum { FS_S = 0, FS_E = 1, FS_I = 2, FS_R = 3 };
enum { FS_SIR = 0, FS_SEIR = 1, FS_SIS = 2 };
enum { FS_AGE_F32 = 0, FS_AGE_F16 = 1, FS_AGE_BF16 = 2 };
enum { FS_DISPATCH_AUTO = 0, FS_DISPATCH_THREAD = 1, FS_DISPATCH_MERGE = 2, FS_DISPATCH_TUNE = 3 };
/* How a realisation obtains the infection pressure of its S nodes (the count
 * c_i of in-neighbours in I, lambda_i = beta c_i; Eq. 3 with unit weights and
 * constant shedding), passed in fs_sim_params.flags:
 *   FS_PRESSURE_GATHER: every step, every S node counts the I bits of its
 *     row in an infectious bitmap (the paper's gather, Algorithm 3).
 *   FS_PRESSURE_PUSH: every node keeps c_i; a node entering I adds 1 to the
 *     count of each node whose row lists it, a node leaving I subtracts 1
 *     (along the transposed CSR, built on the graph's first push-form sim).
 *     Same integer counts, so the same trajectory bit for bit; the work per
 *     step no longer grows with the edges of S rows. Needs every node of the
 *     one-thread-per-node class to have in-degree <= 255 (true for every
 *     dispatch except FS_DISPATCH_THREAD on graphs with d_max > 255).
 *   FS_PRESSURE_AUTO (0): for a single realisation (fs_sim_*), PUSH where
 *     it is available, else GATHER; for a packed ensemble (also in batches
 *     and the server), PUSH where it is available for ensembles of up to 8
 *     realisations and GATHER for 9 to 32: a packed gather reads each column
 *     once for all the replicates of a node while pushes are paid per
 *     replicate, and on GB300 the gather measured faster at 16 and 32
 *     replicate lanes, the push at 8. A shedding profile always takes
 *     GATHER. FS_PRESSURE_PUSH / _GATHER force a form there too (every
 *     realisation of an ensemble or request must pass the same flags). */
enum { FS_PRESSURE_AUTO = 0, FS_PRESSURE_GATHER = 1, FS_PRESSURE_PUSH = 2 };
/* Active-node compaction (Section 5.6), a flag ORed into fs_sim_params.flags
 * of a single realisation: at the start of every launch sequence (each CUDA
 * Graph replay of the step loop, and the directly launched remainder) the
 * units that still hold a non-R node are listed (SELL slices of 32 nodes in
 * the gather form, groups of 8 nodes and merge-class nodes in the push form)
 * and the steps of that sequence visit only them. R is absorbing, so a unit
 * dropped at a refresh never needs a step again; units that reach R inside a
 * sequence stay on the list until the next refresh. The list is used only
 * once at least half the nodes are R (before that the refresh writes "all
 * units" and returns). Trajectories are identical with and without it.
 * Merge-class chunks of the gather form are edge-partitioned and not listed.
 * Packed ensembles, batches, the server and fs_step_noalloc reject it. */
#define FS_ACTIVE_LIST 0x4
#define FS_PRESSURE_MASK 0x3

/* Holding-time law of a nodal transition (Section 5.1; hazard h = f/S).
 *   FS_LAW_EXP:       a = rate gamma                  h = gamma
 *   FS_LAW_LOGNORMAL: a = mu, b = sigma (log-days)    h = sqrt(2/pi)/(tau sigma erfcx(z)),
 *                                                     z = (ln tau - mu)/(sigma sqrt 2)
 *   FS_LAW_WEIBULL:   a = shape k >= 1, b = scale s   h = (k/s)(tau/s)^(k-1)
 *   FS_LAW_ERLANG:    k = stages >= 1, a = rate r     h = r (r tau)^(k-1)/(k-1)! / sum_{n<k} (r tau)^n/n!
 * Hazards are evaluated in FP32 at the begin-of-step age; h(0) = 0 for the
 * log-normal, for Weibull with k > 1 and for Erlang with k > 1. */
typedef enum {
    FS_LAW_NONE = 0, FS_LAW_EXP = 1, FS_LAW_LOGNORMAL = 2, FS_LAW_WEIBULL = 3, FS_LAW_ERLANG = 4
} fs_law_kind;

typedef struct {
    int32_t kind;        /* fs_law_kind */
    int32_t k;           /* Erlang stages */
    double a, b;
} fs_law;

/* Shedding profile s(tau) of the source-node infectivity (Section 5.3,
 * Eq. 8): an I node of infection age tau exerts beta * s(tau) on each of its
 * out-neighbours.
 *   FS_SHED_NONE:    s = 1 (Markovian edges; the pressure is beta x the
 *                    number of infectious in-neighbours, an integer count)
 *   FS_SHED_HAZARD:  s = the hazard of the `shedding` law (e.g. the
 *                    infectious law itself: beta h_IR(tau))
 *   FS_SHED_DENSITY: s = the density of the `shedding` law (e.g. a
 *                    log-normal viral-load profile)
 * With a profile, every step writes beta s(tau') of each node that is I after
 * it (tau' its new age), FP32 rounded to the sim's age storage type, and an S
 * node's pressure is the FP32 sum of those values over its infectious
 * in-neighbours, in a fixed order (row order in the one-lane-per-node class;
 * segmented warp sums folded by warp, then by chunk, in the merge class), so
 * a run is reproducible bit for bit. Gather form only (the adaptive step,
 * eps > 0, combines with it): FS_PRESSURE_PUSH and fs_step_noalloc need
 * FS_SHED_NONE (FS_EUNSUPPORTED). Packed ensembles, batches and the server
 * take it in the gather form when every realisation of the ensemble (or
 * request) has a profile: each replicate keeps its own infectivities and
 * sums them in the same order as alone (row order; in the merge class the
 * windows, warp ranges and chunks of the single-realisation kernel), so its
 * trajectory is the one it has alone. */
typedef enum { FS_SHED_NONE = 0, FS_SHED_HAZARD = 1, FS_SHED_DENSITY = 2 } fs_shed_mode;

/* One realisation (Section 3; Algorithm 3 with a fixed step dt). */
typedef struct {
    int32_t model;       /* FS_SIR or FS_SEIR                                     */
    int32_t age_dtype;   /* FS_AGE_F32, FS_AGE_F16 or FS_AGE_BF16 (age storage)    */
    fs_law latent;       /* E -> I law (SEIR only; ignored for SIR)                */
    fs_law infectious;   /* I -> R law                                             */
    double beta;         /* hazard per infectious in-neighbour (1/day) > 0         */
    double dt;           /* fixed step (days) > 0; with eps > 0, the cap dt_max    */
    uint64_t seed;       /* Philox key                                             */
    uint32_t replicate;  /* realisation index in the key's stream                  */
    int32_t index_state; /* compartment of the index cases: FS_E (SEIR) or FS_I    */
    int32_t flags;       /* FS_PRESSURE_AUTO / _GATHER / _PUSH, optionally | FS_ACTIVE_LIST;
                            other bits invalid                                    */
    int32_t shed_mode;   /* fs_shed_mode (0: s = 1)                                */
    /* Adaptive step (Section 5.2): with eps > 0 step k advances by
     *   dt_k = min(dt, eps / (lambda*_{k-1} + delta))
     * where lambda*_{k-1} is the largest rate of any node in step k-1 (S:
     * beta x infectious in-neighbours, E/I: the hazard at the begin-of-step
     * age) and the first step after init or set_state uses dt. Computed in
     * FP32 on the device; ages advance by that value; hazards are evaluated
     * directly (no memoised tables, since ages leave the fixed-step
     * sequence). Single realisations, in either pressure form and with or
     * without a shedding profile; packed ensembles, batches and the server
     * (each realisation with its own step size and clock, fs_ens_time; every
     * realisation of an ensemble or request adaptive, or none);
     * fs_step_noalloc needs eps = 0. */
    double eps;          /* 0: fixed step; > 0: the tolerance (the paper uses 0.01-0.05) */
    double delta;        /* added to lambda*; 0 = 1e-12                            */
    fs_law shedding;     /* the law of s(tau) when shed_mode != FS_SHED_NONE       */
    /* Markovian engine (Section 4, Algorithm 1), selected by theta > 0: all
     * rates constant (infectious law, and latent law for SEIR, must be
     * FS_LAW_EXP; SIS: I -> S, SIR / SEIR: I -> R); step k has the size
     *   tau_k = min(theta N / Lambda, p_max / max_i lambda_i, dt)
     * from the rates of the state at its start (Lambda = their sum; a term is
     * skipped when its denominator is 0), computed in double from integer
     * reductions (exact, schedule-independent) and applied as a float. The
     * infection counts are exact integers kept for every node and updated
     * after each step by +-1 along the transposed CSR from the nodes that
     * entered or left I (Inertial Mode) or recounted from the rows (Control
     * Mode); markov_mode picks: 0 by memory touched, 1 inertial, 2 control.
     * Single realisations only (packed ensembles, the server and
     * fs_step_noalloc reject it); eps, shedding and FS_ACTIVE_LIST must be
     * off; the flags' pressure form is ignored. FS_SIS needs theta > 0. */
    double theta;        /* 0: renewal engine; > 0: Algorithm 1 (the paper uses 0.01) */
    double p_max;        /* largest per-step probability (0 = 0.1, the paper's)   */
    int32_t markov_mode; /* 0 auto, 1 inertial, 2 control                          */
    int32_t reserved2_;  /* must be 0                                              */
} fs_sim_params;

/* Graph construction options (all fields may be 0 for the defaults). */
typedef struct {
    int32_t dispatch;        /* FS_DISPATCH_*: AUTO picks the class split from the
                                degree profile by a fixed rule (Section 5.5
                                auto-dispatch); TUNE times short trial runs
                                from an early-phase state (1% I) and from a
                                mid-epidemic mix of states for each
                                candidate split (thresholds 31, 63, 127, 255
                                below d_max) and keeps the fastest (the AUTO
                                split unless beaten by > 2%), caching the choice
                                per degree profile
                                (ceil log2 N, ceil log2 d_max, round d_avg) for
                                the process; graphs with d_max <= 64 need no
                                trial. THREAD / MERGE force one class.          */
    int32_t thread_max_deg;  /* rows of degree <= this go to the one-thread-per-node
                                class; larger rows go to the edge-partitioned
                                merge class. 0 = chosen by the tuner; >= 31        */
    int32_t device_input;    /* 1: row_ptr/col_ind are device pointers             */
    int32_t reserved_;
} fs_graph_opts;

typedef struct {
    int64_t n, nnz, d_max;
    double d_avg, rho;        /* rho = d_max / d_avg (Section 5.5)                 */
    int64_t n_thread;         /* nodes in the one-thread-per-node (SELL-32) class  */
    int64_t n_merge;          /* nodes in the edge-partitioned merge class         */
    int64_t sell_entries;     /* SELL-32 column entries incl. padding              */
    int64_t merge_chunks;     /* edge chunks of the merge class per step           */
    int32_t thread_max_deg;   /* class threshold in use                            */
    int32_t identity_layout;  /* 1 when internal ids equal original ids            */
    int64_t device_bytes;     /* device memory held by the graph                   */
} fs_graph_info_t;

typedef struct fs_graph fs_graph;
typedef struct fs_sim fs_sim;

/* Library version string, e.g. "flashstep 0.1 sm_103a". Never NULL. */
const char* fs_version(void);
/* Message for the last non-OK status on this thread ("" if none). */
const char* fs_last_error(void);

/* ---------------------------------------------------------------------------
 * fs_graph_create -- ingest a CSR graph (Appendix D.1 layout; Section 5.5
 * degree inspection). Copies the CSR to the device (or reads it there when
 * opts->device_input = 1), computes degrees, d_max, rho, splits the nodes
 * into the thread class and the merge class, relabels nodes by degree
 * (stable), and builds the SELL-32 column blocks of the thread class and the
 * chunk tables of the merge class. Runs on `stream` (a cudaStream_t, NULL =
 * a library stream) and returns after the ingest has completed.
 *   n        number of nodes, 1 <= n < 2^31
 *   row_ptr  int64[n+1] (see CSR above)
 *   col_ind  int32[row_ptr[n]]
 *   weights  must be NULL (unit edge weights; other weights: FS_EUNSUPPORTED)
 *   opts     NULL for the defaults
 *   out      receives the handle; destroy with fs_graph_destroy
 * Errors: FS_EINVAL (bad sizes, row_ptr[0] != 0, non-monotone row_ptr,
 *         col_ind out of range; row_ptr[0] and row_ptr[n] are read on the
 *         host, the rest is checked on the device after the copy, for host
 *         and device input alike), FS_ENOMEM, FS_ECUDA, FS_EUNSUPPORTED.
 * ------------------------------------------------------------------------- */
fs_status fs_graph_create(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                          const float* weights, const fs_graph_opts* opts,
                          void* stream, fs_graph** out);
/* The graph's sizes, degree profile and the class split in use (Section
 * 5.5: d_max, rho = d_max / d_avg). fs_graph_info_get is the same call.
 * Errors: FS_EINVAL (NULL argument). */
fs_status fs_graph_info(const fs_graph* g, fs_graph_info_t* out);
fs_status fs_graph_info_get(const fs_graph* g, fs_graph_info_t* out);
/* FS_EBUSY while a simulation created on the graph is alive. */
fs_status fs_graph_destroy(fs_graph* g);

/* ---------------------------------------------------------------------------
 * fs_sim_init -- one realisation on a graph (Algorithm 2: persistent state
 * X, tau and the step counter). Every node starts in S with age 0; the
 * listed index nodes start in params->index_state with age 0; the step
 * counter starts at 0.
 *   index_nodes  host int32[n_index] of distinct original ids in [0, n)
 *   stream       cudaStream_t used by every later call on the sim (NULL = a
 *                library-owned non-blocking stream)
 * Errors: FS_EINVAL (bad params: model, laws, beta, dt, dtype, index list),
 *         FS_ENOMEM, FS_ECUDA.
 * ------------------------------------------------------------------------- */
fs_status fs_sim_init(fs_graph* g, const fs_sim_params* params,
                      const int32_t* index_nodes, int64_t n_index, void* stream,
                      fs_sim** out);

/* One fused step (Algorithm 3); counts_out (host uint32[4], may be NULL)
 * receives [S, E, I, R] after the step. Synchronous. */
fs_status fs_sim_step(fs_sim* s, uint32_t* counts_out);

/* `steps` fused steps; the step loop runs as replays of a CUDA Graph of
 * `graph_steps` steps (Algorithm 2; captured on first use, 0 = 50) plus
 * directly launched remainder steps. counts_out: host uint32[(steps+1)*4],
 * row 0 = the counts before the first step, row t = after step t. May be
 * NULL. Synchronous. */
fs_status fs_sim_run(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_out);

/* Asynchronous form of fs_sim_run for callers that keep results on the
 * device: enqueues the steps on the sim's stream and returns. counts_dev:
 * device uint32[(steps+1)*4] written when the stream reaches it, or NULL.
 * Call fs_sim_sync before reading results or issuing host calls that read
 * the state. */
fs_status fs_sim_run_async(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_dev);
/* Waits for the sim's stream and reports device-side errors. */
fs_status fs_sim_sync(fs_sim* s);

/* fs_sim_run_async + fs_sim_sync with CUDA events recorded on the sim's
 * stream around every graph replay: replay_ms (host float[steps/K + 1])
 * receives the duration of each K-step replay (step kernels, the launch gaps
 * between them and the replay's epilogue) and, last, of the directly
 * launched remainder (0 if none); *n_replays = steps/K + 1. */
fs_status fs_sim_run_timed(fs_sim* s, int64_t steps, int32_t graph_steps, uint32_t* counts_dev,
                           float* replay_ms, int64_t* n_replays);

/* Number of kernels enqueued so far by step loops of this process (graph
 * replays count their kernels). */
fs_status fs_kernel_launches(uint64_t* count);

/* Dispatch autotuner (FS_DISPATCH_TUNE): trial runs timed so far, graph
 * creations answered from the cache, and degree profiles cached. The paper
 * has no autotuner; its dispatch is a fixed rule on rho. */
fs_status fs_tune_stats(int64_t* trials, int64_t* cache_hits, int64_t* profiles);
/* Forgets every cached choice and zeroes the statistics. */
fs_status fs_tune_reset(void);

/* Host copies of the state in original node order: state uint8[n], age
 * (float / binary16 / bfloat16 bits per age_dtype)[n], step (next step
 * index). Any pointer may be NULL. Synchronous. */
fs_status fs_sim_get_state(fs_sim* s, uint8_t* state, void* age, int64_t* step);
/* Replace the state (resume from a checkpoint; original node order). The
 * ages must be storage values of the sim's age dtype; S and R ages must be
 * 0. Synchronous. */
fs_status fs_sim_set_state(fs_sim* s, const uint8_t* state, const void* age, int64_t step);

/* Simulated time (the clock of Algorithm 2 / Algorithm 1, Section 5.2):
 * *elapsed (may be NULL) = the sum of the step sizes of the
 * steps run since init or set_state; *next_dt (may be NULL) = the size of the
 * next step (dt for a fixed step; 0 for the Markovian engine, whose next
 * step size depends on the rates of the state it starts from). Synchronous. */
fs_status fs_sim_time(const fs_sim* s, double* elapsed, float* next_dt);

/* Active-node compaction accounting (FS_ACTIVE_LIST, Section 5.6): *listed = the sum over
 * the launch sequences run since init or set_state of the units each one
 * visited (all units while the list is not in use), *units = the number of
 * units (SELL slices in the gather form, push items in the push form; 0
 * without FS_ACTIVE_LIST). Synchronous. */
fs_status fs_sim_active_units(const fs_sim* s, uint64_t* listed, uint64_t* units);

/* *total = the node transitions (S -> E/I, E -> I, I -> R/S) of the steps
 * run since init or set_state (the Markovian engine's "events", Section 4).
 * Synchronous. */
fs_status fs_sim_transitions(const fs_sim* s, uint64_t* total);

/* The infectivity the next step reads (Eq. 8): rho[i] = beta s(tau_i) as
 * stored (age_dtype storage: float / binary16 / bfloat16 bits, n elements,
 * original node order) for I nodes and 0 elsewhere. Needs shed_mode !=
 * FS_SHED_NONE (else FS_EUNSUPPORTED). Synchronous. */
fs_status fs_sim_infectivity_get(fs_sim* s, void* rho);

/* The pressure form the sim runs (FS_PRESSURE_GATHER or FS_PRESSURE_PUSH).
 * The Markovian engine keeps its own exact counts (updated by pushes or
 * recounts, see markov_mode) and reports FS_PRESSURE_GATHER. */
fs_status fs_sim_pressure_get(const fs_sim* s, int32_t* pressure);

/* Work accounting for the roofline model: the sum over all steps run so far
 * of sum_{i in S at step start} deg(i), and of |S at step start|. */
fs_status fs_sim_work(const fs_sim* s, uint64_t* s_degree_sum, uint64_t* s_node_sum, int64_t* steps_run);

fs_status fs_sim_destroy(fs_sim* s);

/* ---------------------------------------------------------------------------
 * Diagnostics that run the same device functions the step uses.
 * fs_eval_hazard: h_dev[i] = hazard(law, tau_dev[i]) in FP32, device arrays
 * of n floats, on `stream` (asynchronous).
 * fs_eval_uniforms: u_dev[i] = the step's uniform for (seed, replicate,
 * step, nodes_dev[i]) as a float, device arrays (asynchronous).
 * ------------------------------------------------------------------------- */
fs_status fs_eval_hazard(const fs_law* law, const float* tau_dev, float* h_dev, int64_t n, void* stream);
/* f_dev[i] = the probability density of `law` at tau_dev[i] in FP32 (the
 * shedding profile of FS_SHED_DENSITY); asynchronous. */
fs_status fs_eval_density(const fs_law* law, const float* tau_dev, float* f_dev, int64_t n, void* stream);
fs_status fs_eval_uniforms(uint64_t seed, uint32_t replicate, int64_t step, const int32_t* nodes_dev,
                           float* u_dev, int64_t n, void* stream);

/* ---------------------------------------------------------------------------
 * Packed ensembles and batches (the fused step of Algorithm 3 applied to many
 * realisations at once). An ensemble holds 1..32 realisations of one graph
 * stored node-major (the state of replicate r of node i next to the other
 * replicates of node i), so every column read and neighbour-mask gather of a
 * step serves all of them. Each realisation keeps its own parameters (beta,
 * laws, seed, replicate index), so it draws exactly the uniforms it would
 * draw alone: an ensemble's results are identical to running each
 * realisation on its own with fs_sim_*. A batch (the segment table) steps
 * every live ensemble added to it with one kernel launch per step;
 * ensembles may join and leave between launches.
 * ------------------------------------------------------------------------- */
typedef struct fs_ens fs_ens;
typedef struct fs_batch fs_batch;

/* params[n_real]: every entry must share model, age_dtype and index_state;
 * the index nodes (host int32[n_index], distinct original ids) are the same
 * for every realisation. Either every realisation takes the adaptive step
 * (eps > 0, Section 5.2; each replicate then has its own step size and
 * clock: its trajectory is the one it has alone through fs_sim_*) or none;
 * likewise every realisation has a shedding profile (Section 5.3, each its
 * own law, gather form) or none.
 * Errors: FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_EUNSUPPORTED (FS_ACTIVE_LIST,
 * theta > 0, a shedding profile with FS_PRESSURE_PUSH). */
fs_status fs_ens_create(fs_graph* g, const fs_sim_params* params, int32_t n_real, const int32_t* index_nodes,
                        int64_t n_index, fs_ens** out);
/* Runs the ensemble alone for `steps` steps (a batch of one).
 * counts_out: host uint32[(steps+1)][n_real][4] or NULL. Synchronous. */
fs_status fs_ens_run(fs_ens* e, int64_t steps, int32_t graph_steps, uint32_t* counts_out);
/* Host copies of realisation r's state (original node order) and the number
 * of steps the ensemble has run. Synchronous. */
fs_status fs_ens_get_state(fs_ens* e, int32_t r, uint8_t* state, void* age, int64_t* step);
/* Per realisation r < n_real (host arrays, each may be NULL): the simulated
 * time its steps have covered, and the size of its next step (the adaptive
 * rule, Section 5.2; the fixed dt otherwise). Synchronous. */
fs_status fs_ens_time(fs_ens* e, double* elapsed, float* next_dt);
/* *pressure = FS_PRESSURE_GATHER or FS_PRESSURE_PUSH: the form the
 * ensemble runs (FS_PRESSURE_AUTO resolves by replicate width). */
fs_status fs_ens_pressure_get(const fs_ens* e, int32_t* pressure);
/* FS_EBUSY while the ensemble is a live member of a batch. */
fs_status fs_ens_destroy(fs_ens* e);

/* A batch steps ensembles of one age storage type together. stream: a
 * cudaStream_t or NULL for a library stream. */
fs_status fs_batch_create(int32_t age_dtype, int32_t max_members, void* stream, fs_batch** out);
/* Adds an ensemble that will run `steps` further steps, starting at the
 * batch's next launch. counts_out: host uint32[(steps+1)][n_real][4] or NULL,
 * written when the member completes (row 0 = counts when it joins). */
fs_status fs_batch_add(fs_batch* b, fs_ens* e, int64_t steps, uint32_t* counts_out);
/* Launches `launches` steps of every live member (replays of a captured
 * graph of graph_steps launches; 0 = 50), then retires the members that have
 * completed (their counts are copied out). Synchronous. */
fs_status fs_batch_run(fs_batch* b, int64_t launches, int32_t graph_steps);
/* Live members and the launches still needed to complete all of them. */
fs_status fs_batch_status(const fs_batch* b, int32_t* live, int64_t* launches_to_finish);
fs_status fs_batch_destroy(fs_batch* b);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of forecast ensembles. A server owns a batch
 * and a host thread. A request asks for n_scen x replicates realisations of
 * one resident graph (realisation (s, r) uses scenarios[s] with replicate
 * index scenarios[s].replicate + r), run for `steps` steps. Requests are
 * admitted first come, first served while their device memory fits the
 * budget and the work in flight stays under a cap; admitted requests join
 * the running batch at the next quantum of `quantum` launches, so work of
 * requests that arrive while others run overlaps on the device; finished
 * requests leave the batch and free their memory. Every running request
 * advances one step per launch, so a launch costs the sum of their sizes:
 * the cap keeps enough work in flight to fill the GPU while letting the
 * requests at the head of the queue finish early instead of all sharing the
 * device until the end. Results are identical to running each realisation
 * alone.
 * Graphs must outlive the requests that use them.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t hbm_budget_bytes;  /* device memory for request state; 0 = 80% of free memory */
    int32_t max_members;       /* ensembles in flight (segment table rows); 0 = 4096        */
    int32_t quantum;           /* launches between admissions and retirements; 0 = 10      */
    int32_t age_dtype;         /* age storage of every request                               */
    int32_t reserved_;         /* must be 0                                                  */
    int64_t max_inflight;      /* cap on node x realisation updates per launch summed over
                                  running requests; the queue head waits while admitting it
                                  would pass the cap, unless nothing runs. 0 = 2^25, -1 = none */
    double wait_limit_s;       /* longest time a request may wait in the queue; a request
                                  not admitted by then is retired alone: fs_server_poll
                                  reports done with FS_ETIMEOUT, the others run on.
                                  0 = no limit; must be >= 0                                  */
} fs_server_cfg;

typedef struct {
    int64_t submitted, completed, queued, running;
    int64_t launches;          /* step launches so far                                       */
    int64_t node_updates;      /* realisation-node-steps completed                           */
    int64_t device_bytes;      /* request state held on the device now                       */
    double busy_seconds;       /* time with at least one request in flight                   */
} fs_server_stats;

typedef struct fs_server fs_server;

fs_status fs_server_create(const fs_server_cfg* cfg, fs_server** out);
/* Validates and queues a request (host arrays are copied). Scenarios share
 * model, index_state and flags; every scenario takes the adaptive step or
 * none, and every scenario has a shedding profile (gather form) or none.
 * FS_EINVAL for bad arguments, FS_ENOMEM if the request alone exceeds the
 * budget, FS_EUNSUPPORTED for FS_ACTIVE_LIST, theta > 0, or a shedding
 * profile with FS_PRESSURE_PUSH. */
fs_status fs_server_submit(fs_server* s, fs_graph* g, const fs_sim_params* scenarios, int32_t n_scen,
                           int32_t replicates, const int32_t* index_nodes, int64_t n_index, int64_t steps,
                           uint64_t* request_id);
/* *done = 1 when the request has finished; then counts_out (host uint32
 * [(steps+1)][n_scen*replicates][4], may be NULL) receives its counts and
 * *seconds (may be NULL) its time from submission to completion. A request
 * retired by the wait limit sets *done = 1 and returns FS_ETIMEOUT. */
fs_status fs_server_poll(fs_server* s, uint64_t request_id, int32_t* done, uint32_t* counts_out,
                         double* seconds);
/* Blocks until every submitted request has finished or `timeout_s` passes
 * (FS_ETIMEOUT). */
fs_status fs_server_drain(fs_server* s, double timeout_s);
fs_status fs_server_stats_get(fs_server* s, fs_server_stats* out);
/* Stops the thread (finishing nothing further) and frees everything. */
fs_status fs_server_destroy(fs_server* s);

/* ---------------------------------------------------------------------------
 * Device memory. Graphs, simulations, ensembles, batches and their scratch
 * take device memory from the library's allocator. By default it keeps the
 * blocks that are freed (after a device-wide synchronisation, so no launched
 * work still uses them) and hands them out again for the same size, so that
 * objects created and destroyed in a loop do not pay for cudaMalloc and
 * cudaFree each time; when the device runs out of memory the cache is
 * released and the allocation retried. (The paper's engine allocates through
 * PyTorch; this boundary has no PyTorch types.)
 *   fs_set_allocator      routes every later allocation to alloc(bytes, ctx)
 *                         (it must return device memory of the current device,
 *                         aligned to at least 256 bytes, or NULL when out of
 *                         memory) and its release to free_fn(ptr, ctx), called
 *                         after a device-wide synchronisation; the library
 *                         then caches nothing. NULL, NULL restores the
 *                         library's own allocator. A block is always released
 *                         through the functions that allocated it. Both
 *                         functions or neither, else FS_EINVAL.
 *   fs_release_cached_memory  frees the cached blocks of the current device.
 *   fs_cached_memory      bytes cached and blocks in use on the current device
 *                         (the library's own allocator only).
 * ------------------------------------------------------------------------- */
typedef void* (*fs_alloc_fn)(size_t bytes, void* ctx);
typedef void (*fs_free_fn)(void* ptr, void* ctx);
fs_status fs_set_allocator(fs_alloc_fn alloc, fs_free_fn free_fn, void* ctx);
fs_status fs_release_cached_memory(void);
fs_status fs_cached_memory(uint64_t* cached_bytes, uint64_t* live_blocks);

/* ---------------------------------------------------------------------------
 * Failure-detection test hooks. The paper has no counterpart: these let the
 * tests make the library's own bounded device waits and bounds checks fire
 * without faulting the GPU. They affect only simulations created while the
 * setting is in force (the setting is copied at fs_sim_init); 0 turns it off.
 *   FS_TEST_WAIT_TIMEOUT  value = a wait limit in polls (1 .. 2^20): the
 *                         merge-class chunks of the gather form arm their
 *                         mbarrier but issue no bulk copy, so the bounded
 *                         wait runs out with nothing in flight; the step then
 *                         sets the device error word and returns, and the
 *                         next synchronising call reports FS_ETIMEOUT (the
 *                         simulation then answers FS_ESTATE; other handles
 *                         and the CUDA context stay usable).
 *   FS_TEST_BOUNDS_SHRINK value = how far below the end of the transposed
 *                         CSR the bounds check of its column reads is put
 *                         (the reads it rejects are still inside the buffer);
 *                         only in the bounds-checked build (FS_DEBUG_BOUNDS),
 *                         else FS_EUNSUPPORTED.
 * In the bounds-checked build the step kernels check the indices of their
 * main accesses; the first index out of range is recorded with its check's
 * site, the access is skipped, and the call reports FS_ECUDA with "bounds
 * check failed: site S, index I" in fs_last_error.
 * ------------------------------------------------------------------------- */
enum { FS_TEST_WAIT_TIMEOUT = 1, FS_TEST_BOUNDS_SHRINK = 2 };
fs_status fs_test_inject(int32_t what, int64_t value);
/* *enabled = 1 in the bounds-checked build, else 0. */
fs_status fs_debug_bounds_build(int32_t* enabled);

/* ---------------------------------------------------------------------------
 * fs_step_noalloc -- one fused step that allocates no device memory. The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc while they step -- code running inside CUDA stream capture
 * (where cudaMalloc is not allowed), and applications whose device memory is
 * owned by their own pool or arena and must not be grown behind its back. The
 * graph is created beforehand with fs_graph_create (which does allocate); the
 * caller owns and passes every other buffer.
 *
 * The step's only scratch -- the merge class's cross-chunk partial counts and
 * tickets, a 256-byte control block and a 1 KiB row of per-warp delta slots
 * -- lives in one fixed array inside the library, sized for at most 65,536
 * merge-class rows (512 KiB + 1.25 KiB, held on every GPU that loads the
 * library until the process exits). A graph with more merge-class rows is
 * rejected with FS_EINVAL.
 *   g               graph from fs_graph_create. The buffers below are in the
 *                   graph's internal node order, which is the caller's order
 *                   when fs_graph_info_get reports identity_layout = 1.
 *   params          the realisation, as for fs_sim_init (index_state unused).
 *                   The pressure form in params->flags is ignored: this step
 *                   always counts infectious neighbours by the gather over the
 *                   bitmap (the push form keeps per-node counts, which would be
 *                   more caller-owned state); both forms give the same counts.
 *   step            step index k (keys the uniforms), 0 <= k < 2^32
 *   state_dev       device uint8[n], read and updated in place
 *   age_dev         device ages[n] of params->age_dtype, updated in place
 *   bitmap_cur_dev  device uint32[n/32 + 1]: bit i = (state[i] == FS_I) at
 *                   the start of the step, other bits 0
 *   bitmap_next_dev device uint32[n/32 + 1], receives that bitmap after the
 *                   step (must not alias bitmap_cur_dev)
 *   deltas_dev      device uint64[5], receives [nodes that left S, E -> I,
 *                   I -> R, sum of degrees of the nodes that left S, device
 *                   error word (0 = ok)]
 *   stream          cudaStream_t (NULL = the legacy default stream); the call
 *                   only enqueues work and returns
 * Set-up: the first call on each device looks up the device address of the
 * scratch array (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. Every call shares the one array and
 * clears what must start at zero; calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Errors: FS_EINVAL (NULL pointers, bad params or step, too many merge-class
 * rows), FS_EUNSUPPORTED (eps > 0, a shedding profile, FS_ACTIVE_LIST,
 * theta > 0, or a current device ordinal of 64 or more), FS_ESTATE (the graph
 * is in a failed state), FS_ECUDA.
 * ------------------------------------------------------------------------- */
fs_status fs_step_noalloc(const fs_graph* g, const fs_sim_params* params, int64_t step,
                          uint8_t* state_dev, void* age_dev, const uint32_t* bitmap_cur_dev,
                          uint32_t* bitmap_next_dev, uint64_t* deltas_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
