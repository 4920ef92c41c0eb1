/*
 * mpc.h -- C ABI of the GB300 multiparticle-collision-dynamics (MPC) step library.
 *
 * One MPC time step (Westphal, Goh, Winkler, Gompper, arXiv 2406.15236, Sec. II):
 *   streaming              r_i <- r_i + h v_i                       (Eq. 1)
 *   boundary conditions    periodic, or bounce-back walls at z = 0, Lz with phantom
 *                          particles in the wall part of cut cells  (Sec. II, "Boundary
 *                          conditions")
 *   body force             v_i <- v_i + g h before streaming        (Sec. II, "External fields")
 *   random lattice shift   one uniform vector in [0, a)^3 per step  (Sec. II, after Eq. 2)
 *   collision per cell     SRD rotation v_i <- v_cm + D(alpha)(v_i - v_cm)   (Eq. 2)
 *                          or MPC-AT+a (angular-momentum-conserving Andersen-thermostat
 *                          MPC of the reference cited with Eqs. 3-4)
 *   thermostat             Maxwell-Boltzmann scaling, kappa = sqrt(2E_k / sum m v_ic^2),
 *                          E_k ~ Gamma(3(N_c-1)/2, kT)              (Eqs. 5-7)
 *   reorder                particles are binned by collision cell every step
 *                          (Sec. III.B.3, permanent exchange / spatial reorder)
 *
 * State contract (shared by every entry point):
 *   - Positions are 32-bit unsigned fixed point per axis with F fraction bits per cell
 *     length a = 1, F = 31 - ceil(log2(max L)); X in [0, L << F).
 *   - Velocities are float32.  Arrays are structure-of-arrays: X = {x[N], y[N], z[N]},
 *     V = {vx[N], vy[N], vz[N]}; id[N] is a persistent particle tag (Sec. III.C,
 *     "Fluid Particle ID") that keys per-particle random draws.
 *   - Random numbers are Philox4x32-10 keyed by (seed) with counter
 *     (index, step, tag << 24 | sub-draw, box_id), so results do not depend on the
 *     order of particles in memory.
 *
 * Errors: every call returns an mpc_status; nothing aborts.  mpc_last_error() gives the
 * text of the last error on a handle (or of the last failed mpc_create when NULL).
 * Threading: a handle may be used by one host thread at a time.
 * Streams: work is enqueued on the CUDA stream given to mpc_create (a cudaStream_t
 * passed as void*, NULL for the legacy default stream); calls that return data to
 * the host synchronise that stream.
 */
#ifndef MPC_H
#define MPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpc_s* mpc_handle;

typedef enum {
  MPC_SRD = 0,    /* stochastic rotation dynamics, Eq. (2) */
  MPC_AT_A = 1,   /* Andersen-thermostat MPC with angular-momentum conservation */
  MPC_SRD_A = 2   /* SRD with angular-momentum conservation, Eqs. (3)-(4) */
} mpc_variant;

typedef enum {
  MPC_OK = 0,
  MPC_EINVAL = 1,    /* invalid argument or parameter combination */
  MPC_ENOMEM = 2,    /* device or host allocation failed */
  MPC_ECUDA = 3,     /* a CUDA call failed (text in mpc_last_error) */
  MPC_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  MPC_ESTATE = 5     /* state inconsistent (e.g. a particle outside the box) */
} mpc_status;

enum {
  MPC_FLAG_OBSERVABLES = 1u,  /* accumulate observables inside every step */
  MPC_FLAG_DEBUG_CELLS = 2u,  /* keep each particle's collision cell and per-cell counts */
  /* Bit-reproducible trajectories (Sec. III.B, "Reproducibility"): every per-cell sum and
   * every observable is accumulated in 64-bit fixed point (cell sums: 32 fraction bits;
   * observables: 24), so results do not depend on the order of particles in memory,
   * on the brick geometry, the threads per cell, or on which other boxes share a batch.
   * Range: each summed per-particle term (a velocity component, a squared relative
   * speed, a component of r x v) must stay below 2^15 in magnitude; a larger term makes
   * the next synchronising call return MPC_ESTATE.  Sums of the observables must stay
   * below 2^39 in magnitude. */
  MPC_FLAG_DETERMINISTIC = 4u
};

typedef struct {
  int32_t L[3];          /* box edge lengths in collision cells, each in [2, 1024] */
  double a;              /* collision-cell size; must be 1.0 (lengths are in units of a) */
  double n_c;            /* mean particles per cell <N_c>; N = round(Lx Ly Lz n_c) */
  double h;              /* time step, > 0 */
  double alpha_deg;      /* SRD rotation angle in degrees (SRD, SRD+a) */
  double kT;             /* thermal energy k_B T, > 0 */
  double m;              /* particle mass, > 0 */
  int32_t variant;       /* mpc_variant */
  int32_t thermostat;    /* 1: MBS thermostat after the collision (MPC_SRD only) */
  int32_t walls_z;       /* walls at z = 0 and z = Lz (Sec. II, Boundary conditions):
                            0 none (periodic in z); 1 no-slip (bounce-back, phantom
                            particles in cut cells); 2 slip (specular reflection) */
  double gravity[3];     /* body-force acceleration g */
  uint64_t seed;         /* Philox key */
  uint32_t box_id;       /* Philox counter word 3 (distinguishes boxes with one seed) */
  uint32_t flags;        /* MPC_FLAG_* */
  int32_t capacity;      /* particles per brick buffer; 0 = chosen from n_c */
  int32_t graph_steps;   /* steps per captured CUDA graph; 0 = default (16) */
  int32_t tile_particles;   /* target mean particles per brick (the on-chip sort tile);
                               0 = 640; see mpc_autotune */
  int32_t threads_per_cell; /* threads that reduce one cell: 0 (auto) or a power of two
                               <= 32; see mpc_autotune */
  int32_t obs_ring;         /* rows of the per-step observables ring; 0 = 1024 */
  int32_t reserved;         /* must be 0 */
  double wall_u[2];         /* x velocity of the no-slip walls at z = 0 and z = Lz (shear
                               flow between moving walls); 0 unless walls_z = 1 */
} mpc_params;

/* Device-memory provider.  alloc returns device memory of `bytes` (>= 256-byte aligned)
 * usable on `stream`, or NULL; release returns it.  Passing NULL to mpc_create uses
 * cudaMalloc/cudaFree. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*release)(void* ctx, void* ptr, size_t bytes, void* stream);
} mpc_allocator;

typedef struct {
  double momentum[3];    /* sum m v after the last step */
  double ekin;           /* sum m v^2 / 2 */
  double temperature;    /* m sum |v - <v>|^2 / (3 (N - 1)), k_B = 1 */
  double stress_kin[3];  /* -(m/V) sum v_a v_b with the streaming velocity: xy, yz, zx */
  double stress_col[6];  /* -(m/(V h)) sum dv_a rho_b (collisional): xy, yx, yz, zy, zx, xz */
  int64_t n_particles;
  int64_t step;          /* number of completed steps */
  int32_t has_stress;    /* 1 if the stresses were accumulated inside the last step */
  int32_t reserved;
} mpc_obs;

typedef struct {
  int64_t n_particles;
  int64_t n_cells;       /* Lx Ly (Lz + walls_z): cells of the shifted lattice */
  int64_t step;          /* completed steps */
  int32_t fixed_bits;    /* F */
  int32_t capacity;      /* particles per brick buffer */
  int32_t brick[3];      /* cells per brick along x, y, z */
  int32_t n_bricks[3];
  uint64_t device_bytes; /* device memory held by the handle */
  int32_t recoveries;    /* capacity overflows repaired so far */
  int32_t threads_per_cell;
} mpc_info;

/* Create a box, initialise it (Sec. II: uniform positions, Maxwell-Boltzmann velocities
 * with the net momentum removed, ids 0..N-1) and bin it for step 0.
 * p: parameters (copied).  stream: cudaStream_t or NULL.  alloc: NULL or a provider
 * that must outlive the handle.  out: receives the handle.  Synchronises the stream. */
mpc_status mpc_create(const mpc_params* p, void* stream, const mpc_allocator* alloc,
                      mpc_handle* out);

/* Release every device buffer of the handle (after finishing its queued work). */
mpc_status mpc_destroy(mpc_handle h);

/* Enqueue nsteps >= 0 MPC steps (graph-captured in chunks); asynchronous.  A capacity
 * overflow inside the queued steps stops the chain at a consistent step; the next
 * synchronising call repairs it and runs the remaining steps. */
mpc_status mpc_step(mpc_handle h, int64_t nsteps);

/* Wait for queued steps, repair capacity overflows, report device-side errors. */
mpc_status mpc_synchronize(mpc_handle h);

/* Copy the state out, ordered by unshifted cell index (Sec. III.G.2: checkpoints are
 * sorted by unshifted cell), arbitrary order inside a cell.
 * X: 3N uint32, V: 3N float, id: N uint32 or NULL, cell: N uint32 or NULL (collision
 * cell of each particle in the last step; needs MPC_FLAG_DEBUG_CELLS), step: or NULL.
 * device_ptrs = 0: host buffers; 1: device buffers.  Synchronises. */
mpc_status mpc_get_state(mpc_handle h, uint32_t* X, float* V, uint32_t* id, uint32_t* cell,
                         int64_t* step, int device_ptrs);

/* Replace the state (N particles, same N as the handle) and the step counter.
 * X values must lie in [0, L << F) (MPC_EINVAL otherwise).  Synchronises. */
mpc_status mpc_set_state(mpc_handle h, const uint32_t* X, const float* V, const uint32_t* id,
                         int64_t step, int device_ptrs);

/* Per-cell particle counts of the last step (n_cells uint32; MPC_FLAG_DEBUG_CELLS). */
mpc_status mpc_get_cell_counts(mpc_handle h, uint32_t* counts, int device_ptrs);

/* Observables after the last completed step (Sec. II: conserved momentum and energy;
 * stress for Green-Kubo viscosity).  Synchronises. */
mpc_status mpc_observables(mpc_handle h, mpc_obs* out);

/* Up to `count` most recent per-step rows (oldest first) of the observables ring
 * (needs MPC_FLAG_OBSERVABLES): row = {px,py,pz, 2 ekin/m, skin xy,yz,zx, scol xy,yx,
 * yz,zy,zx,xz, step, 0, 0} as raw sums (see mpc_obs for the scalings).  Returns the
 * number of rows written in *written.  Synchronises. */
mpc_status mpc_observable_series(mpc_handle h, double* rows, int64_t count, int64_t* written);

/* Velocity profile across the box along z (Sec. II, "External fields" and "Boundary
 * conditions": the flow between walls under a body force): the box [0, L_z) is cut into
 * nbins equal slabs; out (host, 4 nbins doubles) receives per slab the number of
 * particles and the sums of v_x, v_y and v_z over them, at the positions and velocities
 * of the current state (those mpc_get_state returns).  nbins in [1, 65536], else
 * MPC_EINVAL.  Allocates a 32 nbins-byte device buffer for the call.  Synchronises. */
mpc_status mpc_velocity_profile(mpc_handle h, int32_t nbins, double* out);

mpc_status mpc_get_info(mpc_handle h, mpc_info* out);

/* Timing support (no counterpart in the paper beyond its per-partial-step timers,
 * Fig. 3): when enabled, CUDA events bracket every launch of the fused step kernel on
 * the handle's stream (inside captured graphs too).  mpc_profile_step_kernel returns
 * the mean duration in ms over the most recent (up to graph_steps) recorded launches
 * and the number of launches averaged; it synchronises the stream. */
mpc_status mpc_set_profiling(mpc_handle h, int enable);
mpc_status mpc_profile_step_kernel(mpc_handle h, double* mean_ms, int32_t* samples);

/* Checkpoint ordering without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when they need
 * it -- e.g. a serving loop whose memory pool owns all of HBM, or code that must not
 * trigger the device-wide synchronisation of cudaFree while other streams run.
 * It sorts n particles by unshifted cell index (the order mpc_get_state produces;
 * arbitrary order inside a cell) using only the caller's arrays plus a fixed scratch
 * area compiled into the library (8.4 MB per device, held until the process exits).
 * L: box edges (each in [2, 1024]) with Lx Ly Lz <= 2,097,152 cells, else MPC_EINVAL.
 * X, V (3n each, SoA, the state contract above), id (n) or NULL: device inputs;
 * X_out, V_out, id_out (NULL exactly when id is NULL): device outputs, not aliasing the
 * inputs.  Positions outside [0, L << F) are rejected with MPC_EINVAL before sorting.
 * stream: cudaStream_t or NULL; the call synchronises it before returning.
 * The first call on a device looks up the scratch area's device address for that
 * device (cudaGetSymbolAddress); make that first call before any stream capture.  The
 * address is kept for the rest of the process: resetting a device (cudaDeviceReset) in
 * a process that has called this entry point on it is not supported.
 * All calls in the process share the one scratch area: calls that overlap on the GPU
 * (different streams or threads, not ordered) race and corrupt each other's results.
 * Errors are reported through mpc_last_error(NULL). */
mpc_status mpc_sort_by_cell_noalloc(const int32_t L[3], int64_t n, const uint32_t* X,
                                    const float* V, const uint32_t* id, uint32_t* X_out,
                                    float* V_out, uint32_t* id_out, void* stream);

/* Checkpoint files (Sec. III.G.2, "Input/Output"): parameters and the step count in a
 * text file `<prefix>.txt` (one "key = value" per line), all particle data in binary in
 * `<prefix>.particles` -- x[N], y[N], z[N] (u32 fixed point, the state contract), vx[N],
 * vy[N], vz[N] (f32), id[N] (u32), ordered by unshifted cell index -- and per unshifted
 * cell its particle count and the offset of its first particle in `<prefix>.cells`
 * (u32 count[C], then u32 offset[C], or u64 offsets when N >= 2^32; C = Lx Ly Lz), all
 * little-endian.  The paper also stores a random seed per cell; here random numbers are
 * counter-based (Philox keyed by the run's seed, the step and the cell), so the seed in
 * the text file is all a reader needs.  Writing synchronises the handle's stream and
 * needs 32 B of host memory per particle; returns MPC_EINVAL when a file cannot be
 * written. */
mpc_status mpc_checkpoint_write(mpc_handle h, const char* prefix);

/* Create a box from a checkpoint written by mpc_checkpoint_write (parameters, step count
 * and state), on `stream` with `alloc` as in mpc_create.  MPC_EINVAL for a missing,
 * malformed or inconsistent file set (counts that do not match the particles' cells,
 * positions outside the box, unknown format version). */
mpc_status mpc_checkpoint_read(const char* prefix, void* stream, const mpc_allocator* alloc,
                               mpc_handle* out);

/* Stop the box at step `limit`: later steps (single or batched) leave it unchanged.
 * limit must not lie before the steps already requested (MPC_EINVAL).  Asynchronous.
 * The paper runs one system per job and has no counterpart; batches and the serving
 * loop use it to end each job at its own step count inside a shared step chain. */
mpc_status mpc_set_step_limit(mpc_handle h, int64_t limit);

/* Device bytes a box with parameters p holds while it lives (steady) and at most during
 * mpc_create (peak), on the current device.  No allocation; MPC_EINVAL as mpc_create. */
mpc_status mpc_footprint(const mpc_params* p, uint64_t* steady_bytes, uint64_t* peak_bytes);

/* Picks tile_particles and threads_per_cell for boxes like p by timing the fused step
 * kernel on a cubic box with p's physics and about 8M particles: tiles of about 320,
 * 640 and 1280 particles whose shared memory per CTA stays within max_smem_bytes (0: no
 * bound), each with the thread splits that finalise a brick in at most four passes.
 * Results are written to *tile_particles, *threads_per_cell and *ns_per_particle_step
 * (the best time); the parameters chosen change only speed (with
 * MPC_FLAG_DETERMINISTIC not even the rounding).  Allocates and frees device memory
 * with cudaMalloc; synchronises `stream`. */
mpc_status mpc_autotune(const mpc_params* p, void* stream, uint64_t max_smem_bytes,
                        int32_t* tile_particles, int32_t* threads_per_cell,
                        double* ns_per_particle_step);

/* ---- Batches: many independent boxes advanced together ----------------------------
 * The paper runs one system per job; a batch advances many boxes (any L, variant,
 * alpha, h, n_c, seed) together, inside CUDA graphs of graph_steps steps.  Per step,
 * small boxes are packed by variant into persistent launches (up to 48 boxes each, the
 * CTAs claiming the boxes' bricks from one work list); boxes with at least two GPU
 * waves of bricks get their own single-box launch in the same step.
 * Member boxes are ordinary handles (mpc_get_state, mpc_observables, ... work on them)
 * created and destroyed through the batch; their device memory comes from the batch's
 * arena when it has one.  A batch and its members are used by one host thread. */
typedef struct mpc_batch_s* mpc_batch;

enum {
  MPC_BATCH_DETERMINISTIC = 1u,  /* members get MPC_FLAG_DETERMINISTIC */
  MPC_BATCH_AUTOTUNE = 2u,       /* members without explicit tile_particles /
                                    threads_per_cell are tuned per class (variant,
                                    n_c, thermostat, walls, flags) with mpc_autotune */
  MPC_BATCH_PACK_ALL = 4u        /* pack every member, whatever its size; by default
                                    members with at least two GPU waves of bricks
                                    (2 x 5 x SMs) get their own single-box launch */
};

typedef struct {
  uint64_t arena_bytes;  /* device memory for all members, allocated once; admission
                            fails with MPC_ENOMEM when a box does not fit.  0: members
                            allocate with cudaMalloc */
  int32_t graph_steps;   /* batch steps per captured graph; 0 = 100 */
  uint32_t flags;        /* MPC_BATCH_* */
  int32_t max_boxes;     /* 0 = 4096 (the maximum) */
  int32_t reserved;      /* must be 0 */
} mpc_batch_config;

typedef struct {
  int32_t n_boxes;
  int32_t work_items;       /* bricks of the packed members */
  int64_t n_particles;
  uint64_t arena_bytes, arena_used, arena_largest_free;
  int32_t grid;             /* CTAs of the packed launches of one step, summed */
  int32_t ctas_per_sm;      /* largest occupancy of a packed launch */
  int32_t smem_bytes;       /* largest dynamic shared memory per CTA of a packed launch */
  int32_t graph_builds;
  int32_t tuned_classes;
  int32_t solo_boxes;       /* members stepped by their own single-box launch */
  int32_t packed_launches;  /* persistent launches per step for the packed members */
  float plan_ms;            /* host time spent re-planning steps and capturing graphs */
} mpc_batch_info;

/* Create an empty batch on `stream` (cudaStream_t or NULL). */
mpc_status mpc_batch_create(const mpc_batch_config* cfg, void* stream, mpc_batch* out);

/* Destroy the batch and every member box (after finishing queued work). */
mpc_status mpc_batch_destroy(mpc_batch b);

/* Create a box (as mpc_create) and make it a member.  Its creation runs on a side
 * stream of the batch, overlapping steps already queued; the box joins the steps
 * enqueued after this call, starting from its step 0.  MPC_ENOMEM (nothing created)
 * when the arena cannot hold it; MPC_EINVAL when the batch is full. */
mpc_status mpc_batch_add(mpc_batch b, const mpc_params* p, mpc_handle* out);

/* Remove a member and release it.  Its memory returns to the arena once the work
 * queued before this call has finished; no synchronisation. */
mpc_status mpc_batch_remove(mpc_batch b, mpc_handle h);

/* Enqueue nsteps batch steps: every member advances by one step per batch step until
 * it reaches its step limit (mpc_set_step_limit).  Asynchronous. */
mpc_status mpc_batch_step(mpc_batch b, int64_t nsteps);

/* Wait for queued steps, repair members whose brick capacity overflowed (they finish
 * their steps alone), and report the first member error. */
mpc_status mpc_batch_synchronize(mpc_batch b);

mpc_status mpc_batch_get_info(mpc_batch b, mpc_batch_info* out);

/* Text of the last error of a batch call (NULL: of the last failed mpc_batch_create). */
const char* mpc_batch_last_error(mpc_batch b);

/* ---- Serving: a continuous-batching request loop ----------------------------------
 * The paper runs one system per job; a server takes simulation jobs (a box, a step
 * count) with arrival times, admits each as soon as it has arrived and its device
 * footprint fits the HBM budget (later small jobs may pass a head job that does not
 * fit), keeps admitted jobs resident as members of one batch, advances them together
 * in chunks of steps, stops each at its own step count, and retires it:
 * its observables give a Green-Kubo shear viscosity, its memory returns to the budget,
 * and waiting jobs are admitted between chunks while the next chunk runs on the GPU.
 * MPC_SERVER_SEQUENTIAL runs the same jobs one at a time through mpc_create/mpc_step
 * instead (the plain path, for comparison).  A server is used by one host thread. */
typedef struct mpc_server_s* mpc_server;

enum {
  MPC_SERVER_DETERMINISTIC = 1u,  /* every job gets MPC_FLAG_DETERMINISTIC: a job's
                                     results do not depend on the other jobs */
  MPC_SERVER_SEQUENTIAL = 2u,     /* one job at a time on the plain single-box path */
  MPC_SERVER_SHARE_ALL = 4u,      /* every resident job steps in every chunk */
  MPC_SERVER_FIRST_COME = 8u,     /* pick stepping jobs in arrival order instead of by
                                     least remaining work */
  MPC_SERVER_AGED = 16u,          /* pick stepping jobs by remaining time (at the
                                     measured particle-step rate) minus the time waited
                                     since arrival: least remaining work for fresh jobs,
                                     arrival order for jobs that have waited as long as
                                     they still need */
  MPC_SERVER_BACKFILL = 32u,      /* jobs of at most a sixteenth of the fill step in every
                                     chunk, beyond the fill: small jobs progress beside a
                                     large one at little cost to it */
  MPC_SERVER_PRIORITY_HEAD = 64u  /* the oldest resident job steps on its own stream of the
                                     highest priority, outside the batch, all its remaining
                                     steps enqueued at once: the GPU's block scheduler serves
                                     its launches first and the other jobs use what it leaves
                                     (the stepping order applies to them) */
};
/* By default a chunk steps the resident jobs with the least remaining work (steps x
 * particles) until they hold fill_kparticles thousand particles (default 16M: enough
 * jobs that their launches overlap and keep every SM busy) and holds the others at their
 * current step.  Short jobs then finish early (low median latency) while the GPU stays
 * full (throughput, and with it the longest latency under load). */

enum { MPC_JOB_QUEUED = 0, MPC_JOB_RUNNING = 1, MPC_JOB_DONE = 2, MPC_JOB_FAILED = 3 };
enum { MPC_JOB_KEEP_SERIES = 1u, MPC_JOB_KEEP_STATE = 2u };

typedef struct {
  uint64_t hbm_budget_bytes;  /* device memory for resident jobs (one arena), > 0 */
  int32_t chunk_steps;        /* most steps per scheduling round (graph size); 0 = 100 */
  int32_t max_active;         /* most resident jobs; 0 = 4096 */
  uint32_t flags;             /* MPC_SERVER_* */
  int32_t fill_kparticles;    /* particles (in thousands) the stepping jobs of a chunk
                                 should hold; 0 = 16000 */
} mpc_server_config;

typedef struct {
  mpc_params params;          /* the box; MPC_FLAG_OBSERVABLES is added and the
                                 observables ring holds every step */
  int64_t steps;              /* steps to run, >= 1 */
  double arrival_s;           /* seconds after the first mpc_server_run call */
  uint32_t keep;              /* MPC_JOB_KEEP_*: keep the per-step observables and / or
                                 the final state on the host for the caller */
  int32_t reserved;           /* must be 0 */
} mpc_job;

typedef struct {
  int32_t status;             /* MPC_JOB_* */
  int32_t error;              /* mpc_status of a failed job */
  double arrival_s, admit_s, finish_s;  /* finish: results on the host */
  int64_t steps;
  int64_t n_particles;
  double eta_gk;              /* Green-Kubo shear viscosity, (V h / kT) [C(0)/2 +
                                 sum_k C(k)] over the six off-diagonal stresses */
  double temperature;         /* mean kinetic temperature over the run */
} mpc_job_result;

typedef struct {
  int64_t chunks;        /* chunks enqueued by the batched loop */
  int64_t chunk_steps;   /* batch steps in them */
  double gpu_ms;         /* device time of the chunks (CUDA events) */
  double host_gap_ms;    /* wall time the device waited for the host between chunks */
  double plan_ms;        /* host time re-planning launches and capturing graphs */
  int32_t graph_builds;
  int32_t reserved;
} mpc_server_stats;

mpc_status mpc_server_create(const mpc_server_config* cfg, void* stream, mpc_server* out);
mpc_status mpc_server_destroy(mpc_server s);

/* Queue a job; *job_id receives its index (0, 1, ...).  No device work. */
mpc_status mpc_server_submit(mpc_server s, const mpc_job* job, int64_t* job_id);

/* Run the loop until every submitted job has finished or failed, or until timeout_s
 * seconds of this call have passed (MPC_ETIMEOUT; running jobs stay resident and a
 * later call continues).  Jobs that cannot fit the budget even alone fail with
 * MPC_ENOMEM. */
mpc_status mpc_server_run(mpc_server s, double timeout_s);

mpc_status mpc_server_job(mpc_server s, int64_t job_id, mpc_job_result* out);
mpc_status mpc_server_get_stats(mpc_server s, mpc_server_stats* out);

/* The observables rows (16 doubles per step, as mpc_observable_series) of a finished
 * job submitted with MPC_JOB_KEEP_SERIES; count >= its steps. */
mpc_status mpc_server_job_series(mpc_server s, int64_t job_id, double* rows, int64_t count);

/* The final state (host buffers: X 3N, V 3N, id N, sorted by unshifted cell) of a
 * finished job submitted with MPC_JOB_KEEP_STATE. */
mpc_status mpc_server_job_state(mpc_server s, int64_t job_id, uint32_t* X, float* V,
                                uint32_t* id);

const char* mpc_server_last_error(mpc_server s);

/* Text of the last error on h (or of the last failed create when h is NULL). */
const char* mpc_last_error(mpc_handle h);

/* Library version string. */
const char* mpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPC_H */
