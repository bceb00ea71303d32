/*
 * steps_gpu.h -- C ABI of the GB300 operator-splitting reaction-diffusion
 * library (Parallel STEPS method, Chen & De Schutter).
 *
 * The method (§2, Algorithm 1): a tetrahedral mesh, a set of species with
 * diffusion constants and a set of mass-action reactions. Time advances in
 * windows of constant length tau = 1 / max_{S,tet} d_{S,tet} (§2.1). In every
 * window each tet first runs its own reactions by Gillespie's SSA for tau,
 * tracking each species' time-averaged occupancy; then, for every diffusive
 * species, a binomial number of molecules leaves the tet and is split over
 * its face neighbours in proportion to the face rates D*A/(V*d) (Algorithm 1,
 * diffusion operator). All tets advance together on one GPU.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative STEPS_ERR_* code; nothing aborts.
 *     steps_last_error() returns a thread-local message for the last failure.
 *   - Arrays passed in are owned by the caller and copied before the call
 *     returns (unless stated otherwise); handles are owned by the library
 *     until the matching *_destroy.
 *   - Tet indices are always the caller's original order (the library may
 *     reorder tets internally for locality; results do not depend on it).
 *   - Host pointers, except arguments whose names start with d_ (CUDA device
 *     pointers, e.g. d_counts of steps_run_noalloc, d_out of steps_run_record).
 *   - A NULL handle or array, or a size out of range, gives STEPS_ERR_ARG.
 *   - Units: metres, seconds, m^2/s; rate constants in SI (order 0: M/s,
 *     order 1: 1/s, order 2: 1/(M s)).
 */
#ifndef STEPS_GPU_H
#define STEPS_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STEPS_OK 0
#define STEPS_ERR_ARG (-1)     /* bad argument */
#define STEPS_ERR_MESH (-2)    /* invalid mesh (degenerate tet, face of 3+ tets, bad index) */
#define STEPS_ERR_MODEL (-3)   /* invalid model (order > 2, negative rate, too many species) */
#define STEPS_ERR_OOM (-4)     /* device or host allocation failed */
#define STEPS_ERR_CUDA (-5)    /* a CUDA call failed */
#define STEPS_ERR_TIMEOUT (-6) /* a bounded device wait ran out: the window's results are not valid, and a bulk
                                  copy may still be in flight, so the simulation (every member, for a batch) is
                                  closed: later runs return STEPS_ERR_STATE until it is destroyed and rebuilt */
#define STEPS_ERR_STATE (-7)   /* device-side check failed (negative count) or bad call order */

#define STEPS_MAX_SPECIES 32
#define STEPS_MAX_REACTIONS 32

typedef struct steps_mesh steps_mesh;
typedef struct steps_model steps_model;
typedef struct steps_sim steps_sim;

/* Occupancy modes of the trial count fed to the diffusion operator. */
#define STEPS_OCC_MEAN 1 /* Algorithm 1: mean occupancy Nbar = O_S / tau, stochastically rounded (default) */
#define STEPS_OCC_END 0  /* end-of-reaction-phase count */

/* Leave law of the diffusion operator's binomial(Nbar, tau, d). */
#define STEPS_LEAVE_EULER 0 /* p = tau d (the default) */
#define STEPS_LEAVE_EXP 1   /* p = 1 - exp(-tau d): an exponential leaving time of rate d inside the window; runs on
                               the model-specialised kernel only (specialize 0 or 1; creation forces it) */

/* Internal tet order. */
#define STEPS_REORDER_NONE 0
#define STEPS_REORDER_MORTON 1 /* Morton (Z-order) of barycentres (default) */
#define STEPS_REORDER_RCM 2    /* reverse Cuthill-McKee of the face adjacency (face neighbours a few positions apart) */

typedef struct steps_options {
    int32_t occupancy;   /* STEPS_OCC_MEAN or STEPS_OCC_END */
    int32_t reorder;     /* STEPS_REORDER_* */
    int32_t block;       /* threads per block of the step kernel; 0 = default (256) */
    int32_t use_graph;   /* 1 = replay full windows from a captured CUDA graph (default), 0 = plain launches */
    int32_t specialize;  /* step kernel compiled for this model at run time (NVRTC): 0 = when the mesh has at
                            least 65,536 tets and NVRTC is available (default), 1 = always (sim creation fails
                            with STEPS_ERR_CUDA if it cannot be built), -1 = never (the generic kernel) */
    int32_t leave_law;   /* STEPS_LEAVE_EULER (default) or STEPS_LEAVE_EXP */
    int32_t flow;        /* launch form of a run's consecutive full windows. Flow: one launch for all of them,
                            in which each tile of a window starts as soon as the tiles holding its face
                            neighbours have finished the previous window (the model-specialised kernel at any
                            block size, the generic kernel at block 256). Window launches: one launch per
                            window (graph replay as use_graph says). 0 (default): the first run with at least
                            72 full windows times, on its own windows, window launches, flow launches of
                            `block`-tet tiles and (specialised, block < 512) of 512-tet tiles, and keeps the
                            fastest (steps_sim_flow reports it); 1: flow at `block` where a flow kernel exists;
                            -1: window launches. The results are the same bits in every form. */
    int32_t reserved[1]; /* set to 0 */
} steps_options;

/* Fill *opt with the defaults. */
void steps_options_default(steps_options *opt);

/*
 * Mesh from vertices and tets (§2.1: the geometry every process is given).
 *   verts_xyz: [nv*3] float64, metres, row-major (x, y, z).
 *   tets:      [nt*4] int32, 0-based vertex indices. Local face f of a tet is
 *              the face opposite its local vertex f.
 * Builds face adjacency (faces matched by vertex triple), volumes V, face
 * areas A and barycentre distances d, and the geometric face rates
 * g_f = A_f / (V d_f) in float64. Boundary faces are reflective.
 * Errors: STEPS_ERR_ARG (nv < 4, nt < 1, NULL), STEPS_ERR_MESH (index out of
 * range, zero-volume tet, a face shared by more than two tets).
 */
int steps_mesh_create(const double *verts_xyz, int64_t nv, const int32_t *tets, int64_t nt,
                      steps_mesh **out);
void steps_mesh_destroy(steps_mesh *mesh);
/* Number of tets of the mesh. */
int steps_mesh_num_tets(const steps_mesh *mesh, int64_t *nt);

/*
 * Model: species and mass-action reactions (§2.1 "biochemical model").
 *   diff_m2_per_s: [n_species] diffusion constants, 0 = immobile.
 *   lhs, rhs:      [n_reac * n_species] int32 reactant / product molecule
 *                  counts of each reaction (row r = reaction r).
 *   k:             [n_reac] rate constants (order 0: M/s, 1: 1/s, 2: 1/(M s)).
 * Propensities per tet of volume V (litres V_L): order 0 a = k N_A V_L;
 * order 1 a = k N_X; order 2 a = k/(N_A V_L) N_X N_Y, and for X + X,
 * a = k/(N_A V_L) N_X (N_X - 1).
 * Errors: STEPS_ERR_ARG (n_species not in [1, 32], n_reac not in [0, 32]),
 * STEPS_ERR_MODEL (negative D, k or stoichiometry, reaction order > 2, more
 * than 6 species changed by one reaction).
 */
int steps_model_create(int32_t n_species, const double *diff_m2_per_s, int32_t n_reac,
                       const int32_t *lhs, const int32_t *rhs, const double *k, steps_model **out);
void steps_model_destroy(steps_model *model);

/*
 * Simulation of `model` on `mesh`, state resident on the current CUDA device.
 *   seed:        key of the counter-based Philox4x32-10 stream; every draw is
 *                addressed by (window, original tet id, purpose, index), so
 *                results do not depend on tet order, launch shape or batching.
 *   opt:         NULL = defaults.
 *   cuda_stream: cudaStream_t to launch on (NULL = the legacy default stream).
 * Computes tau = 1 / (max_S D_S * max_tet G_tet) over diffusive species
 * (§2.1; +inf when nothing can diffuse, in which case every steps_run call
 * is a single reaction window), the fixed-point face thresholds and the
 * per-tet volume factors, and uploads them. Counts start at zero.
 * The mesh and model may be destroyed after this call.
 */
int steps_sim_create(const steps_mesh *mesh, const steps_model *model, uint64_t seed,
                     const steps_options *opt, void *cuda_stream, steps_sim **out);
void steps_sim_destroy(steps_sim *sim);

/*
 * A new simulation with the mesh, model, options, region masks and device
 * tables of `src` (copied on the device, no host-side rebuilding), its own
 * seed and stream, zero counts and time 0. For serving many jobs that share
 * a mesh and model.
 */
int steps_sim_clone(const steps_sim *src, uint64_t seed, void *cuda_stream, steps_sim **out);
/* Device memory a simulation holds, in bytes (for admission by memory budget). */
int steps_sim_device_bytes(const steps_sim *sim, int64_t *bytes);

/* Counts of one species in every tet: counts[nt] int32 >= 0, original tet order (host). */
int steps_set_counts(steps_sim *sim, int32_t species, const int32_t *counts);
int steps_get_counts(const steps_sim *sim, int32_t species, int32_t *out);
/* All species at once: [n_species * nt] int32, species-major (host). */
int steps_set_counts_all(steps_sim *sim, const int32_t *counts);
int steps_get_counts_all(const steps_sim *sim, int32_t *out);

/*
 * Restrict reaction `reac` to the tets with active[tet] != 0 (original tet
 * order, [nt] uint8; NULL = active everywhere). Used for region-limited
 * sources such as a zero-order influx.
 */
int steps_set_reac_mask(steps_sim *sim, int32_t reac, const uint8_t *active);

/*
 * Advance from the current time t to t_end (Algorithm 1 main loop).
 * Full windows of tau while t + tau <= t_end (within 1e-9 tau); a shorter
 * last window tau_k = t_end - t if time remains; tau is unchanged for later
 * calls (a run that stops off the window grid restarts the grid at t_end).
 * Time is t_base + k tau, recomputed, not accumulated. t_end <= t is a no-op.
 * Returns STEPS_ERR_ARG for a non-finite t_end and STEPS_ERR_STATE if a
 * device-side check failed (a negative count, or a tet that fired more than
 * 2^24 reactions in one window, which stops that tet's reaction phase).
 * The call returns after the work is enqueued on the stream and the error
 * word read back (so it synchronises with the stream once per call).
 */
int steps_run(steps_sim *sim, double t_end);

/*
 * Set the rate constant of reaction `reac` (SI units as in
 * steps_model_create) for the windows that follow. The paper drives its
 * calcium-burst runs with influx rates that change over time per region
 * (§3.2); a caller changes the rate between steps_run calls (or between
 * recording runs) to follow such a profile. The kernels use (float)k.
 * Errors: STEPS_ERR_ARG for a reaction out of range or a rate that is
 * negative or not finite. The next run re-captures its CUDA graphs.
 */
int steps_set_reac_rate(steps_sim *sim, int32_t reac, double k);

/*
 * Advance to t_end like steps_run and record, at every time t0 + k dt_rec
 * (k = 1, 2, ... while <= t_end; t0 = the time at the call; times
 * recomputed, not accumulated), the counts of n_species species (indices
 * `species`) at n_tets tets (original ids `tets`) into d_out, the way the
 * paper records concentrations at fixed intervals (§3.2). Each recording
 * time is a window boundary: the run stops there like steps_run(t) would
 * (a shortened window when dt_rec is not a multiple of tau), so the
 * recorded counts equal those of successive steps_run calls, bit for bit.
 * d_out: caller-owned DEVICE memory of at least max_records * n_species *
 * n_tets int32, recording k - 1 at offset (k - 1) n_species n_tets, laid
 * out [species][tet] in the order given. The snapshots are taken on the
 * device with no host synchronisation between them; the call synchronises
 * once at the end. *n_records (may be NULL) receives the number written.
 * The selection is copied to a small device buffer the simulation keeps.
 * Errors: STEPS_ERR_ARG for bad species/tet indices, a non-positive dt_rec
 * or more recordings than max_records (checked before anything runs); the
 * errors of steps_run otherwise.
 */
int steps_run_record(steps_sim *sim, double t_end, double dt_rec, int32_t n_species, const int32_t *species,
                     int32_t n_tets, const int32_t *tets, int32_t *d_out, int64_t max_records, int64_t *n_records);

/* *specialized = 1 when the simulation runs a step kernel compiled for its
 * model (see steps_options.specialize), else 0. The two kernels give the same
 * results bit for bit; the specialised one takes fewer instructions. */
int steps_sim_specialized(const steps_sim *sim, int32_t *specialized);

/* *flow_block = the tile size (threads per block) of the flow launches the simulation's full windows
 * run as (steps_options.flow), or 0 when they run as window launches. tune_ms (may be NULL): [3] ms per
 * window measured by the tuning run for window launches, flow launches at the simulation's block size
 * and flow launches of 512-tet tiles (0 for a form not timed, and before the tuning run). */
int steps_sim_flow(const steps_sim *sim, int32_t *flow_block, float *tune_ms);

/* Tets and species of a simulation (either output may be NULL). */
int steps_sim_shape(const steps_sim *sim, int64_t *nt, int32_t *n_species);

int steps_get_time(const steps_sim *sim, double *t);
int steps_get_tau(const steps_sim *sim, double *tau);
/* Windows run so far (the RNG window index) and kernel launches issued. */
int steps_get_windows(const steps_sim *sim, uint64_t *windows, uint64_t *launches);

/* ---------------------------------------------------------------------- */
/* Batched form: one launch per window advances many simulations.         */
/* ---------------------------------------------------------------------- */
typedef struct steps_batch steps_batch;

typedef struct steps_batch_options {
    int32_t block;       /* threads per block; 0 = autotune over 128/256/512 on the first run (default) */
    int32_t use_graph;   /* 1 = replay windows from a captured CUDA graph (default) */
    int32_t specialize;  /* batched kernel compiled at run time for the members' model: 0 = when all members
                            share one model structure (species, reactions, stoichiometry, diffusive set; rates
                            may differ), they hold at least 65,536 tets together and NVRTC is available
                            (default), 1 = always (creation fails with STEPS_ERR_ARG if the members differ in
                            structure, the first run with STEPS_ERR_CUDA if it cannot be built), -1 = never */
    int32_t flow;        /* 0 (default): one launch per window for all members. 1: on the specialised batched
                            kernel, a run's full windows go through one launch per group of consecutive members
                            whose tables fit in about half of L2, in which each tile of a window starts once the
                            tiles holding its face neighbours have finished the previous window. The members'
                            results are the same bits; the groups' windows run from L2 (far fewer DRAM bytes),
                            at a few per cent lower throughput on an issue-bound batch. */
    int32_t reserved[4]; /* set to 0 */
} steps_batch_options;

void steps_batch_options_default(steps_batch_options *opt);

/*
 * A batch of n existing simulations (independent replicates or different
 * meshes, seeds, time windows and models, on the current device). Each
 * window launch covers every member's tiles; a member's model and window
 * arguments are read from a device table, and its window counter and buffer
 * parity advance on the device, so the whole step loop replays from a CUDA
 * graph. Results are the same bits as running each member alone with
 * steps_run (the random numbers are addressed by member seed, window and
 * original tet). The batch does not own the members: they must outlive it,
 * and must not be run or changed by other calls while a batch call runs.
 * cuda_stream: stream of the batch's launches (NULL = legacy default stream).
 */
int steps_batch_create(steps_sim *const *members, int32_t n, const steps_batch_options *opt, void *cuda_stream,
                       steps_batch **out);
void steps_batch_destroy(steps_batch *batch);

/*
 * Advance member j to t_end[j] (absolute seconds, [n] host array) by the
 * window rule of steps_run: full windows of the member's own tau, then a
 * shortened last window where time remains. Members with fewer windows sit
 * out the later launches. With block autotuning, the first run times three
 * windows at each candidate block size (real windows: results do not depend
 * on the block size) and keeps the fastest. Synchronises with the batch's
 * stream once. Errors as steps_run.
 */
int steps_batch_run(steps_batch *batch, const double *t_end);

/* Block size in use, kernel launches issued so far, and the autotuner's
 * milliseconds per window for blocks 128/256/512 (tune_ms[3], zeros if not run). */
int steps_batch_info(const steps_batch *batch, int32_t *block, uint64_t *launches, float *tune_ms);

/* *specialized = 1 when the batch runs the model-specialised batched kernel. */
int steps_batch_specialized(const steps_batch *batch, int32_t *specialized);

/* ---------------------------------------------------------------------- */
/* Served form: continuous batching of simulation jobs on one GPU.        */
/* ---------------------------------------------------------------------- */
typedef struct steps_server steps_server;

typedef struct steps_server_options {
    int64_t device_budget; /* bytes of device memory the running jobs may hold; 0 = no limit (default) */
    int32_t max_jobs;      /* jobs advanced together; default 64 */
    int32_t wave_windows;  /* windows of its own tau a job advances per round; default 16 */
    int32_t block;         /* threads per block of the batched kernel; default 256 (fixed: batches re-form
                              whenever jobs come and go, so no autotuning) */
    int32_t specialize;    /* -1 (default): all running jobs in one batch on the generic batched kernel.
                              0 or 1: jobs grouped by model structure, one batch per group, the groups'
                              batches running at the same time on streams the server creates; each
                              batch takes steps_batch_options.specialize = this value (1: the kernel
                              compiled for the group's model; create the prototypes with
                              steps_options.specialize = 1 so that it is compiled then, once per model
                              structure, and never between requests) */
    int32_t reserved[2];   /* set to 0 */
} steps_server_options;

void steps_server_options_default(steps_server_options *opt);

/*
 * A server that advances many independent jobs together with batched
 * launches (the batched form above), admitting and retiring jobs between
 * rounds. Jobs are admitted first come first served while a slot is free and
 * the job's device memory fits the budget (a job is always admitted when none
 * runs). Because every random number is addressed by (job seed, window,
 * original tet), a job's result is the same bits as the same simulation run
 * alone with steps_run, whatever else runs beside it.
 * cuda_stream: stream of the server's launches with specialize = -1, and of
 * every job's set-up and result copies (NULL = legacy default stream).
 * Errors: STEPS_ERR_ARG (NULL, max_jobs < 1, wave_windows < 1, bad block).
 */
int steps_server_create(const steps_server_options *opt, void *cuda_stream, steps_server **out);
/* Frees every job's device memory and results. */
void steps_server_destroy(steps_server *srv);

/*
 * Queue a job: a simulation with the mesh, model, options, region masks and
 * device tables of `proto` (steps_sim_clone: no host-side rebuilding), the
 * job's own seed, initial counts `counts` ([n_species * nt] int32, species-
 * major, original tet order, host; copied here) at time 0, run to t_end
 * seconds. `proto` must stay alive until the job is admitted (see
 * steps_server_job_state). *job: the job's id (0, 1, 2, ... in submission
 * order). Errors: STEPS_ERR_ARG (NULL, t_end not finite or < 0).
 */
int steps_server_submit(steps_server *srv, const steps_sim *proto, uint64_t seed, const int32_t *counts,
                        double t_end, int64_t *job);

/*
 * One round: admit queued jobs; advance every running job by up to
 * wave_windows windows on its own window grid, stopping at its t_end (one
 * batched run; the batch is re-formed only when the set of running jobs
 * changed); retire the jobs that reached t_end (final counts copied to the
 * host, device memory freed). *running: jobs running after the round;
 * *finished: jobs that finished in this round (either may be NULL).
 * Synchronises with the server's stream. Errors as steps_batch_run; jobs
 * keep their state.
 */
int steps_server_step(steps_server *srv, int32_t *running, int32_t *finished);

/* State of a job: 0 queued, 1 running, 2 finished (result held), 3 result
 * taken; its windows run so far and its simulated time. Any output may be
 * NULL. Errors: STEPS_ERR_ARG (unknown job). */
int steps_server_job_state(const steps_server *srv, int64_t job, int32_t *state, uint64_t *windows, double *t);

/* Final counts of a finished job ([n_species * nt] int32, original tet order,
 * host, caller-owned, sized by the job's prototype); the server then frees
 * its copy. counts_out may be NULL to free it unread. Errors: STEPS_ERR_ARG
 * (unknown job), STEPS_ERR_STATE (not finished, or already taken). */
int steps_server_take_result(steps_server *srv, int64_t job, int32_t *counts_out);

/* Rounds run, batch re-formations, batched kernel launches, jobs queued and
 * running now, and the device bytes the running jobs hold. Any output may be
 * NULL. */
int steps_server_stats(const steps_server *srv, uint64_t *rounds, uint64_t *rebuilds, uint64_t *launches,
                       int32_t *queued, int32_t *running, int64_t *device_bytes);

/*
 * Advance `sim` to t_end on counts held in a caller-owned device buffer,
 * without allocating any memory. The paper has no counterpart: this serves
 * callers that cannot let a library call cudaMalloc -- an application that
 * owns all device memory through its own pool or a fixed per-job budget, or
 * one that must not allocate once it is running. The simulation must still be
 * created beforehand (that call allocates its tables).
 *   d_counts: [n_species * nt] int32 device pointer, species-major, original
 *             tet order; in: counts at the current time; out: counts at t_end.
 * Runs the same windows as steps_run (same results, bit for bit) with plain
 * launches. The simulation's clock advances; its own count buffers are
 * neither read nor written, so do not mix this call with steps_run on one
 * simulation without setting the counts again.
 * Scratch: a fixed device array in the library, two count buffers of at most
 * 4,194,304 int32 each (n_species * (nt rounded up to a multiple of 32)) plus
 * two error words: 32 MiB held on every GPU that loads the library until exit.
 * Larger problems get STEPS_ERR_ARG. The array is shared by every call and
 * keeps the last call's contents (each call clears it first); calls that
 * overlap on the GPU, on any stream or thread, race on it. The device the
 * simulation was created on must be current (else STEPS_ERR_ARG). The first
 * call on a device looks up the array's address with that device current;
 * make that first call before any stream capture. Synchronises with the
 * simulation's stream before returning.
 * Errors: d_counts holding a negative count gives STEPS_ERR_ARG before
 * anything changes (clock and d_counts as before the call); so does a
 * simulation under STEPS_LEAVE_EXP (a shortened window would need a table
 * built on the host); otherwise as steps_run.
 */
int steps_run_noalloc(steps_sim *sim, int32_t *d_counts, double t_end);

const char *steps_last_error(void);

/* ---------------------------------------------------------------------- */
/* Test hooks: run one device building block on host arrays.              */
/* ---------------------------------------------------------------------- */

/* Philox4x32-10 on the device: out[4*i..] = philox(key = seed, counter =
 * ctr[4*i..]), n counters. Host arrays in and out. */
int steps_debug_philox(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out);
/* The step kernel's float natural logarithm on the device, n values. */
int steps_debug_logf(const float *x, int64_t n, float *out);
/* The step kernel's bounded wait for its bulk copies, on its own (a test of
 * the failure path). One thread arms a barrier for a 16-byte copy: with
 * deliver != 0 it issues the copy and the wait completes (STEPS_OK); with
 * deliver = 0 nothing completes it, and the wait gives up after limit_cycles
 * clock cycles (STEPS_ERR_TIMEOUT). No copy is in flight when the kernel
 * ends, so the device stays usable. limit_cycles: 1 .. 2^31 (about a second
 * at most); else STEPS_ERR_ARG. */
int steps_debug_wait(int32_t deliver, int64_t limit_cycles);
/* The flow launch's bounded wait for the tiles a tile depends on, on its own
 * (a test of the failure path). One warp waits for 40 listed tiles to have
 * finished window 4: with deliver != 0 they all have (STEPS_OK); with
 * deliver = 0 one has not, and the wait gives up after limit_cycles clock
 * cycles (STEPS_ERR_TIMEOUT). limit_cycles: 1 .. 2^31; else STEPS_ERR_ARG. */
int steps_debug_flow_wait(int32_t deliver, int64_t limit_cycles);
/* The host-side set-up of steps_sim_create alone, with no device work (for
 * tests of the host logic without a GPU): *tau (§2.1), the cumulative face
 * thresholds of every tet at the full window ([nt*4] uint32, 2^31 fixed
 * point, caller's tet order) and, if perm is not NULL, the internal tet order
 * ([nt] int32: device index -> caller's tet id). reorder: STEPS_REORDER_*.
 * Errors: STEPS_ERR_ARG (NULL mesh, model, tau or thr; bad reorder). */
int steps_debug_host_tables(const steps_mesh *mesh, const steps_model *model, int32_t reorder, double *tau,
                            uint32_t *thr, int32_t *perm);

#ifdef __cplusplus
}
#endif

#endif /* STEPS_GPU_H */
