/*
 * sbs.h - C ABI of the B300 sample-based stochastic (SBS) predictive controller.
 *
 * The library implements the data-parallel hot path of the SBS locomotion
 * controller of Turrisi et al., "On the Benefits of GPU Sample-Based Stochastic
 * Predictive Controllers for Legged Locomotion" (IROS 2024):
 *   - batched forward rollout of K sampled foot-force sequences over H steps
 *     through the single-rigid-body model (Eq. (1), Alg. 2), each sample with its
 *     own step frequency and contact schedule (Sec. IV-C);
 *   - per-step tracking, force and friction-cone cost (Sec. V, Sec. IV-B);
 *   - the distribution update: MPPI weighted mean (Sec. III-C, Alg. 5), elite
 *     mean and diagonal variance refit (Alg. 1, Alg. 4) and the Naive best-sample
 *     rule (Sec. III-B, Alg. 3), also with the step frequency drawn uniformly
 *     from a discrete set and one force Gaussian per frequency (Sec. V);
 *   - one warm-started iteration per control tick (Sec. III-A).
 * Every step runs in the library's own CUDA kernels (sm_103a).
 *
 * Conventions
 *   State x = [p (3, world, m), roll/pitch/yaw (3, rad, ZYX), v (3, world, m/s),
 *              omega (3, body, rad/s)].
 *   Forces: 4 legs (FL, FR, RL, RR) x 3 world-frame components, N.
 *   Decision vector theta of one sample: the force part first (nf = 12 values per
 *   step, step-major, for the per-step policy; 12 values per knot, knot-major,
 *   for the spline policy), then the step frequency in Hz when the gait is
 *   adaptive.  The distribution (mean and variance, length D each) has the same
 *   layout, except that a discrete frequency set of n values holds n force
 *   blocks of nf values, block b for set entry b: D = n nf.
 *   Gait phases are integers in units of 1e-9 cycle (1e9 = one cycle).
 *   Random numbers: Philox4x32-10 keyed by (seed, controller_id), counter
 *   (sample, draw, iteration low, iteration high); draw 0 is the frequency
 *   (Box-Muller on the top 24 bits of words 0, 1); draw 1 + n/6 holds force
 *   normal n: six 21-bit integers per 128-bit block (the top 21 bits of each word,
 *   then the low 11 bits of words 0 and 2 joined to the low 10 bits of words 1
 *   and 3), Box-Muller on the pairs (u0, u1), (u2, u3), (u4, u5).
 *   With a discrete frequency set of n values, sample k takes entry
 *   floor(n u / 2^24), u the top 24 bits of draw 0's first word.
 *
 * Errors: every call returns an int status (SBS_OK = 0, negative on error).  No
 * C++ exception crosses the boundary.  A call that fails validation leaves the
 * handle unchanged.  Errors found on the device (all costs non-finite) are
 * reported in sbs_result.status.  A handle must not be used by two host threads
 * at once.
 *
 * Memory: the library owns its device state (mean, variance, costs, partial
 * sums, counters), allocated at creation through the caller's allocator (or
 * cudaMalloc when none is given) and released by sbs_destroy.  Input and output
 * buffers belong to the caller; the library keeps no pointer to them after the
 * work it enqueued has run.
 */
#ifndef SBS_H
#define SBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define SBS_OK 0
#define SBS_PENDING 1
#define SBS_ERR_INVALID_ARG (-1)
#define SBS_ERR_OOM (-2)
#define SBS_ERR_BUDGET (-3)
#define SBS_ERR_CUDA (-4)
#define SBS_ERR_TIMEOUT (-5)
#define SBS_ERR_DIVERGED (-6)

/* ---------------------------------------------------------------- methods */
#define SBS_MPPI 0  /* weighted mean, covariance unchanged (Alg. 5) */
#define SBS_ELITE 1 /* elite mean + diagonal variance refit (Alg. 1 Update) */
#define SBS_NAIVE 2 /* best sample as the new mean, covariance unchanged (Alg. 3) */

/* ---------------------------------------------------------------- limits */
#define SBS_MAX_H 128         /* horizon steps */
#define SBS_MAX_K (1 << 24)   /* samples per controller */
#define SBS_MAX_TILE 256      /* samples per tile (threads per block) */
#define SBS_MAX_FREQ 8        /* values of a discrete step-frequency set */

/* ---------------------------------------------------------------- buffers for sbs_read */
#define SBS_BUF_MEAN 0      /* float[D]  current mean */
#define SBS_BUF_VAR 1       /* float[D]  current diagonal variance */
#define SBS_BUF_COST 2      /* float[K]  costs of the last iteration (+inf when not finite) */
#define SBS_BUF_FREQ 3      /* int32[K]  quantised step frequency of each sample, mHz */
#define SBS_BUF_ELITE 4     /* int32[K_e] elite sample indices of the last elite iteration, ascending;
                             Naive: int32[n + 1], the winning sample of each set entry (-1: none
                             with a finite cost) then the entry of the best sample (n = 1 without
                             a set) */
#define SBS_BUF_MPPI_MEAN 5 /* float[D]  MPPI mean from the first iteration's samples (compare_mppi) */

/* Single rigid body model of Eq. (1). */
typedef struct sbs_model {
    float mass;         /* kg, > 0 */
    float inertia[3];   /* principal body inertia (diagonal tensor), kg m^2, > 0 */
    float foot[4][3];   /* body-frame foot positions relative to the CoM, m */
    float gravity[3];   /* world gravity, m/s^2 (e.g. 0, 0, -9.81) */
} sbs_model;

/* Stage cost r(u, x, x_ref) (Sec. V) plus the friction-cone penalty and the
 * step-frequency regulariser:
 *   r = sum_c Q_c (x_c - xref_c)^2 + sum_legs sum_a R_a Gamma_a^2
 *     + w_fc sum_stance [max(0, |Gamma_xy| - mu Gamma_z)^2 + max(0, -Gamma_z)^2]
 *   J = sum_{j<H} r(u_j, x_j, xref_j) (+ rho (f - f_nominal)^2 when the step
 *   frequency is sampled, from a Gaussian or from a discrete set). */
typedef struct sbs_cost {
    float Q[12];
    float R[3];
    float w_fc;
    float mu;
    float rho;
    float f_nominal; /* Hz */
    float w_terminal; /* >= 0: adds w_terminal sum_c Q_c (x_H - xref_{H-1})^2 for the state after the
                         last step (Alg. 2 leaves it uncosted; 0 follows the paper) */
} sbs_cost;

typedef struct sbs_config {
    int32_t K;            /* samples, 1..SBS_MAX_K */
    int32_t H;            /* horizon steps, 1..SBS_MAX_H */
    int32_t P;            /* 0: one force per step; 2..8: spline knots per force axis (Sec. IV-B) */
    int32_t method;       /* SBS_MPPI / SBS_ELITE / SBS_NAIVE */
    int32_t iterations;   /* sampling iterations per solve, >= 1 */
    int32_t elite_count;  /* K_e for SBS_ELITE, 1..K */
    int32_t adaptive;     /* 1: the step frequency is sampled (Sec. IV-C) */
    int32_t compare_mppi; /* 1: elite/naive solves also form the MPPI mean of iteration 0 */
    uint32_t dt_us;       /* time step, microseconds */
    uint32_t q_init;      /* initial / fixed step frequency, mHz */
    uint32_t seed;        /* Philox key word 0 */
    uint32_t controller_id; /* Philox key word 1 */
    float lambda;         /* MPPI temperature, > 0 */
    float f_min, f_max;   /* step-frequency clip, Hz */
    float sigma_init;     /* initial force standard deviation, N */
    float sigma_min;      /* elite force standard-deviation floor, N */
    float sigma_f_init;   /* initial frequency standard deviation, Hz */
    float sigma_f_min;    /* elite frequency standard-deviation floor, Hz */
    int32_t tile;         /* samples per tile (64..SBS_MAX_TILE, multiple of 32); 0: default 128 */
    sbs_model model;
    sbs_cost cost;
    /* Discrete step-frequency set (Sec. V): 0, or 1..SBS_MAX_FREQ values drawn
     * uniformly per sample, each with its own force Gaussian.  Requires
     * method SBS_NAIVE, adaptive 0 and compare_mppi 0; q_init, f_min and f_max
     * are then unused (each block's nominal schedule uses its own frequency). */
    int32_t n_freq;
    uint32_t freq_set[SBS_MAX_FREQ]; /* mHz, distinct, 1..10000 */
    /* 0: the foot lever arms are the body-frame offsets model.foot (fixed to the
     * body).  1: stance feet stay fixed on the flat ground z = 0 and the lever arm
     * of leg i is p_f,i - p_c (Eq. (1)); a leg touching down inside the horizon
     * lands at the foothold of Sec. IV-D, p_hip + (T_st / 2) v^d + sqrt(p_c,z / g)
     * (v_c - v^d), with the hip at R (foot x, foot y, 0) from the CoM, T_st the
     * stance time of the sample's frequency and v^d the reference's planar
     * velocity at that step.  sbs_problem.feet gives the feet at t_0. */
    int32_t world_feet;
    /* 0: the friction cone is a penalty in the stage cost (w_fc).  1: the policy's
     * stance forces are projected orthogonally onto the cone |Gamma_xy| <= mu Gamma_z
     * before they act (Sec. IV-B), and the penalty is dropped; the samples (and
     * the distribution update) stay on the unprojected decision variables. */
    int32_t friction_project;
} sbs_config;

/* Periodic gait (Sec. IV-C): leg i is in stance while its phase
 * (phase0 + offset[i] + f t) mod 1 is below the duty factor. */
typedef struct sbs_gait {
    uint32_t offset[4]; /* per-leg phase offset, 1e-9 cycle, < 1e9 */
    uint32_t duty;      /* duty factor D_f, 1e-9 cycle, <= 1e9 */
    uint32_t phase0;    /* gait phase at the first step of the horizon, 1e-9 cycle, < 1e9 */
} sbs_gait;

/* One solve's inputs.  host_memory = 0: x0, xref, f_ext and the result are device
 * pointers read/written by the enqueued kernels (they must stay valid until the
 * stream reaches the work).  host_memory = 1: they are host pointers; inputs are
 * copied to the device before the call returns (pinned memory makes the copy
 * asynchronous) and the result is copied back on the stream (synchronize before
 * reading it). */
typedef struct sbs_problem {
    const float* x0;    /* [12] current state estimate */
    const float* xref;  /* [H][12] reference states x^r_0 .. x^r_{H-1} */
    const float* f_ext; /* [3] known external world force on the body, or NULL (zero) */
    sbs_gait gait;
    int32_t shift;      /* warm start: steps elapsed since the previous solve (0 = none) */
    int32_t host_memory;
    const float* feet;  /* world_feet: [4][2] ground (x, y) of the feet at t_0 (legs FL, FR, RL, RR; a
                           leg in stance at t_0 stays there until it lifts off); else NULL */
} sbs_problem;

/* Result of a solve, written by the device. */
typedef struct sbs_result {
    float u0[12];      /* first control of the new mean: forces at t_0, zero on swing legs */
    float cost_min;    /* best sample cost of the last iteration */
    float ess;         /* MPPI effective sample size 1 / sum w^2 (K_e for elite/naive) */
    float f_mean;      /* mean step frequency after the update, Hz */
    int32_t q_freq;    /* that frequency quantised to mHz */
    int32_t status;    /* SBS_OK or SBS_ERR_DIVERGED (no finite cost; mean kept) */
    int32_t n_finite;  /* samples with a finite cost in the last iteration */
    uint32_t iter_lo;  /* Philox iteration counter of the last iteration */
    uint32_t iter_hi;
} sbs_result;

/* Caller-supplied device allocator (e.g. a framework's caching allocator). */
typedef struct sbs_allocator {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} sbs_allocator;

typedef struct sbs_handle sbs_handle;
typedef struct sbs_batch sbs_batch;

/* Create a controller.  Validates cfg (SBS_ERR_INVALID_ARG), allocates its device
 * state through alloc (NULL: cudaMalloc; SBS_ERR_OOM on failure) on the current
 * device.  The distribution is initialised on the first solve (or sbs_reset).
 * The scratch of plain solves (sbs_workspace_bytes) is allocated through the
 * same allocator on the first sbs_solve; controllers solved only through
 * batches or a server never allocate it. */
int sbs_create(const sbs_config* cfg, const sbs_allocator* alloc, sbs_handle** out);
void sbs_destroy(sbs_handle* h);

/* Allocate the handle's plain-solve workspace now instead of on the first
 * sbs_solve (for callers that must not allocate while they control). */
int sbs_prepare(sbs_handle* h);

/* Length D of the mean (and of the variance): n_blocks 12 (H or P) + adaptive,
 * n_blocks = n_freq when a discrete frequency set is configured, else 1. */
int sbs_dim(const sbs_handle* h);

/* Bytes of device memory the handle holds (state, tables and its own workspace). */
size_t sbs_device_bytes(const sbs_handle* h);

/* Bytes of scratch one solve of this controller needs in a batch workspace
 * (costs, sampled deviations, partial sums, elite indices). */
size_t sbs_workspace_bytes(const sbs_handle* h);

/* The same for a batch in the given deviation mode (SBS_THETA_STORE or
 * SBS_THETA_REGENERATE): a tick that regenerates the sampled deviations needs no
 * room for them (K x nt x 48 bytes less). */
size_t sbs_workspace_bytes_mode(const sbs_handle* h, int theta_mode);

/* Reset the distribution to its initial value for the given gait (hover forces
 * m|g| / n_stance per step, sigma_init; frequency q_init, sigma_f_init) and the
 * iteration counter to iter. Enqueued on stream (a cudaStream_t; NULL = default). */
int sbs_reset(sbs_handle* h, const sbs_gait* gait, uint64_t iter, void* stream);

/* One controller tick (Alg. 4): warm shift by prob->shift steps, then
 * `iterations` rounds of sample / roll out / evaluate / update, enqueued on
 * stream.  The first solve after creation resets the distribution with the
 * problem's gait and ignores the shift. */
int sbs_solve(sbs_handle* h, const sbs_problem* prob, sbs_result* result, void* stream);

/* Copy a device buffer of the handle (SBS_BUF_*) to dst (host_dst: host memory),
 * bytes must equal the buffer's size.  Enqueued on stream.  The cost, frequency
 * and elite buffers are those of the last plain sbs_solve. */
int sbs_read(const sbs_handle* h, int which, void* dst, size_t bytes, int host_dst, void* stream);

/* Checkpoint: the distribution and iteration counter as an opaque byte blob.
 * sbs_state_size gives its size; get/set synchronize the stream. */
size_t sbs_state_size(const sbs_handle* h);
int sbs_get_state(const sbs_handle* h, void* buf, size_t bytes, void* stream);
int sbs_set_state(sbs_handle* h, const void* buf, size_t bytes, void* stream);

/* ---------------------------------------------------------------- allocation-free solve
 * The paper has no counterpart to this entry point; it serves callers that may
 * not allocate device memory when they solve (a real-time control thread that
 * must not block on an allocator, a host application or plug-in that owns all
 * device memory).  It runs one MPPI iteration of the per-step policy
 * (method SBS_MPPI, P = 0, iterations = 1) with all of its per-solve scratch in
 * one file-scope device array of SBS_STATIC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc or
 * cudaFree and creates no handle.
 *   cfg        validated like sbs_create.
 *   prob       device pointers only (host_memory = 0); shift is the warm-start
 *              shift applied to state_in.
 *   state_in   device [mean (D) | variance (D)] of the distribution to sample;
 *              D = 12 H (+1 when adaptive), as sbs_dim reports for a handle of
 *              the same cfg (a discrete frequency set, which would multiply the
 *              12 H, needs the Naive method and is refused here).  Use
 *              sbs_reset / sbs_read of a handle, or your own initial values, for
 *              the first call.
 *   state_out  device [mean | variance] written with the updated distribution;
 *              must not alias state_in.
 *   iter       the Philox iteration counter of this solve.
 *   result     device sbs_result.
 * Returns SBS_ERR_BUDGET when the solve's scratch exceeds the array, and
 * SBS_ERR_INVALID_ARG when `stream` is capturing (the parameter block is copied
 * from memory that does not outlive the call).  The first call on a device, and
 * the first after a device reset, looks the array's device address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All
 * calls share the one
 * array and it keeps the previous call's contents (the completion counters are
 * cleared by every call): calls whose work overlaps on the GPU - on different
 * streams, or from different threads - race and corrupt each other. */
#define SBS_STATIC_SCRATCH_BYTES (64u << 20)
int sbs_solve_mppi_static(const sbs_config* cfg, const sbs_problem* prob, const float* state_in,
                          float* state_out, uint64_t iter, sbs_result* result, void* stream);

/* ---------------------------------------------------------------- sample sharding
 * One controller's K samples split over `world` ranks (a process and a GPU
 * each), by tiles: rank r rolls out tiles [r ntiles / world, (r + 1) ntiles /
 * world).  The samples are independent (Alg. 1 Sampling and Rollout, Alg. 4);
 * the updates (Alg. 1 Update, Alg. 3, Alg. 5) need every sample's cost, so one
 * iteration is
 *   sbs_shard_rollout on every rank (same problem, own rank),
 *   an element-wise SUM over ranks of the exchange buffer taken as int32 words
 *     (an all-reduce; each word is written by at most one rank and is zero on
 *     all others, so the sum is the written bits exactly),
 *   sbs_shard_update on every rank with the summed buffer.
 * Every rank then holds the distribution, result, costs, frequencies and elite
 * list an unsharded sbs_solve of the same controller gives, bit for bit: the
 * MPPI combine runs over the same tile rows in tile order, the selection over
 * the same costs, and the refit regenerates the elite deviations from their
 * Philox counters.  A solve of `iterations` rounds is `iterations` such rounds
 * (the warm-start shift applies to the first).  The library calls no
 * collective: the caller brings its own (NCCL, or gloo through host memory). */

/* Bytes of the exchange buffer: 32-bit words, costs [K] at word 0, quantised
 * frequencies [K] at word Kp, MPPI tile rows [ntiles][12 nt + 8] at word 2 Kp,
 * where Kp = K rounded up to a multiple of 64. */
size_t sbs_shard_exchange_bytes(const sbs_handle* h);

/* Tiles of the controller (ceil(K / tile)), the units sbs_shard_range splits. */
int sbs_shard_tiles(const sbs_handle* h);

/* Host only: the tiles [*begin, *end) of rank `rank` of `world` (contiguous,
 * sizes differing by at most one, empty when world > ntiles).
 * SBS_ERR_INVALID_ARG unless 0 <= rank < world and ntiles >= 0. */
int sbs_shard_range(int ntiles, int rank, int world, int* begin, int* end);

/* This rank's part of one iteration, enqueued on stream: zeroes the exchange
 * buffer xbuf (device, 16-byte aligned, sbs_shard_exchange_bytes) and writes
 * this rank's samples' costs and frequencies and its tiles' MPPI rows into it.
 * prob: device pointers only (host_memory = 0).  The first call after creation
 * resets the distribution with the problem's gait, as sbs_solve does.
 * SBS_ERR_INVALID_ARG while a rollout of this handle waits for its
 * sbs_shard_update (and sbs_solve refuses the handle meanwhile). */
int sbs_shard_rollout(sbs_handle* h, const sbs_problem* prob, int rank, int world, void* xbuf, void* stream);

/* The update of the iteration from the summed exchange buffer (device,
 * unchanged), enqueued on stream; result is a device sbs_result. */
int sbs_shard_update(sbs_handle* h, const void* xbuf, sbs_result* result, void* stream);

/* ---------------------------------------------------------------- batching
 * Many controllers of uneven K and H solved in one set of launches per tick
 * (one block per (controller, tile) item, or a persistent launch pulling items
 * from a device work queue); the tick is captured in a CUDA graph and replayed.
 * Every controller's result equals its own sbs_solve (same tile size), bit for
 * bit. */
/* A batch context for up to max_instances controllers per tick and up to
 * `inflight` (1..8) of its ticks in flight at once.  workspace_bytes is the
 * device-memory budget of its solves' scratch, split evenly between the
 * in-flight ticks: each tick's controllers must fit workspace_bytes / inflight.
 * Each tick also has 24 max_instances + min(w / 8192, 2^24) + 1024 zero-when-idle
 * counter words, w = workspace_bytes / inflight: a controller takes a few, an
 * elite controller selecting from more than 32 768 costs 65 792 (histograms); a
 * tick over either budget is refused with SBS_ERR_BUDGET.
 * A tick reuses the slot of the tick `inflight` calls earlier and waits for
 * that tick on the host first.  The batch owns one non-blocking CUDA stream on
 * which a replayed tick copies its records to the device while the tick before
 * still runs; the caller's stream waits for that copy through an event, so a
 * batched tick cannot be recorded by the caller's own stream capture.
 * sbs_batch_destroy synchronises the device first. */
int sbs_batch_create(int max_instances, int inflight, size_t workspace_bytes, const sbs_allocator* alloc,
                     sbs_batch** out);
void sbs_batch_destroy(sbs_batch* b);

/* Solve n controllers (one iteration each; controllers configured with
 * iterations > 1 are rejected) on stream.  probs[i] must use device memory
 * (host_memory = 0) and results is a device array of n sbs_result.  All
 * controllers must share the tile size and the policy (P), and appear once.
 * Returns SBS_ERR_BUDGET, with nothing enqueued, when their workspaces together
 * exceed the batch workspace.  What follows from the list of controllers alone
 * (their checks, tile order and launch sizes) is kept from the previous call
 * when the same handles come in the same order (a handle destroyed and another
 * created at its address does not match); the problems are checked every call.
 * One thread at a time per batch. */
int sbs_batch_solve(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                    sbs_result* results, void* stream);

/* The same tick from host memory, end to end: probs[i] in host memory
 * (host_memory = 1 for every controller) and `results` a host array of n
 * sbs_result.  The library gathers every controller's x0, reference, f_ext and
 * feet into one pinned staging buffer it owns, copies it to the device in one
 * transfer on `stream`, runs the tick of sbs_batch_solve on those copies, copies
 * the n results back in one transfer and waits for it: on return the results are
 * in `results`.  It first waits for the batch's earlier ticks.  The staging
 * buffers (pinned host and device, through the batch's allocator) grow on demand
 * and are freed by sbs_batch_destroy; SBS_ERR_OOM if they cannot grow.  Errors
 * as sbs_batch_solve. */
int sbs_batch_solve_host(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                         sbs_result* results, void* stream);

/* Inputs written in place for sbs_batch_solve_host: fills probs[i] (host_memory
 * = 1) with pointers into the batch's pinned staging buffer, laid out as that
 * call gathers these controllers in this order: x0 [12], xref [H][12], f_ext [3]
 * when with_fext, feet [4][2] for ground-fixed feet.  A caller that writes its
 * inputs there and passes these problems (same controllers, same order) saves
 * the gather copy; the solve still copies the buffer to the device each tick.
 * The pointers stay valid until a call with more or larger controllers grows
 * the buffer, or sbs_batch_destroy.  Waits for the batch's ticks in flight.
 * SBS_ERR_OOM if the buffer cannot grow. */
int sbs_batch_host_inputs(sbs_batch* b, int n, sbs_handle* const* handles, int with_fext, sbs_problem* probs);

/* Launch mode of a batch.  SBS_BATCH_GRID (default): one block per item, the
 * hardware block scheduler dispatching items in order, heaviest controllers
 * first.  SBS_BATCH_PERSISTENT: as many blocks as fit on the GPU pull items from
 * device queues (atomic heads).  Both give identical results. */
#define SBS_BATCH_GRID 1
#define SBS_BATCH_PERSISTENT 0
int sbs_batch_set_mode(sbs_batch* b, int mode);
int sbs_batch_get_mode(const sbs_batch* b);

/* Samples per thread of a batch's rollout launches: 1, 2, or 0 (the default,
 * one; sbs_batch_autotune measures both and keeps the faster).  Two samples per
 * thread apply to the per-step policy on the ordinary model (no spline, no
 * frequency set, no ground-fixed feet, no friction projection) with tiles of a
 * multiple of 64 samples; each thread then carries two samples whose FP32
 * arithmetic issues as packed FP32x2 instructions, with half the threads and
 * twice the registers per thread.  Other launches keep one.  Results are bit for
 * bit the same either way: this is a launch shape, not a change of method. */
int sbs_batch_set_samples_per_thread(sbs_batch* b, int spt);
int sbs_batch_get_samples_per_thread(const sbs_batch* b);

/* The same choice for a handle's plain solves (sbs_solve); 0 (the default) is
 * one sample per thread.  Plain solves also take SBS_SPT_NOISE_WARPS: one
 * sample per thread and a second thread per sample that draws the sample's
 * normals one step ahead (2T threads per tile: the Philox and Box-Muller work
 * runs on other warps than the model step), for controllers too small to fill
 * the GPU, whose rollout is bound by each sample's chain of dependent
 * instructions; same bits.  Spline controllers take one sample per thread. */
#define SBS_SPT_NOISE_WARPS 3
int sbs_set_samples_per_thread(sbs_handle* h, int spt);

/* Sampled deviations (Alg. 1 Sampling): the update needs sigma * eps of the
 * samples it weights or selects.  SBS_THETA_STORE (the default): the rollout
 * writes every sample's deviations (48 bytes per sample-step, step-major) to
 * the workspace and the update reads them.  SBS_THETA_REGENERATE: nothing is
 * written; the MPPI tile sums and the elite / Naive refit regenerate the
 * deviations of the samples they use from the same Philox counters, with the
 * same operations.  Results are bit for bit the same either way; regeneration
 * trades the stores for Philox and Box-Muller work proportional to the samples
 * of nonzero MPPI weight and the elites.  sbs_batch_autotune measures both. */
#define SBS_THETA_STORE 0
#define SBS_THETA_REGENERATE 1
int sbs_set_theta_mode(sbs_handle* h, int mode);
int sbs_get_theta_mode(const sbs_handle* h);
int sbs_get_samples_per_thread(const sbs_handle* h);
int sbs_batch_set_theta_mode(sbs_batch* b, int mode);
int sbs_batch_get_theta_mode(const sbs_batch* b);

/* Autotuner of a handle's plain solves: times `ticks` solves of prob (after one
 * warm-up solve per setting; real solves, they advance the controller) at one
 * sample per thread, two where the controller can take them and the noise warps
 * (SBS_SPT_NOISE_WARPS) where they apply, each storing and regenerating the
 * sampled deviations, and keeps the fastest setting.  ms_out[2 (spt - 1) + mode]
 * gets the mean solve time in ms of each setting (-1 where not measured).
 * Synchronises the stream. */
int sbs_autotune(sbs_handle* h, const sbs_problem* prob, sbs_result* result, int ticks, float ms_out[6],
                 void* stream);

/* Autotuner: runs `ticks` profiled ticks in each launch mode, with one and (where
 * the launch can take them) two samples per thread, storing and regenerating the
 * sampled deviations, on these controllers and problems (real solves: they
 * advance the controllers), keeps the setting with the shortest mean tick and
 * reports each mode's best mean tick time in ms_out[0] (grid) and ms_out[1]
 * (persistent; 1e30 where nothing was measured).  A setting whose workspace does
 * not fit the batch's arena (stored deviations in an arena sized by
 * sbs_workspace_bytes_mode(h, SBS_THETA_REGENERATE)) is skipped; SBS_ERR_BUDGET
 * when none fits. */
int sbs_batch_autotune(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                       sbs_result* results, int ticks, float ms_out[2], void* stream);

/* Tracing: with profiling on, a batch launches its three stages (rollout,
 * selection, refit) as separate kernels bracketed by CUDA events instead of
 * replaying its graph; sbs_batch_stage_ms waits for the last tick and gives the
 * three stage durations in milliseconds. */
int sbs_batch_set_profiling(sbs_batch* b, int on);
int sbs_batch_stage_ms(sbs_batch* b, float ms[3]);

/* ---------------------------------------------------------------- serving
 * A request loop with continuous batching.  Callers submit solves of their
 * controllers as they arrive (host-memory inputs, copied at submission).  A
 * dispatcher thread admits waiting requests into the next free tick slot while
 * earlier ticks are still running on the GPU: a request joins a tick when its
 * controller has no solve in flight and its workspace fits the slot's share of
 * the device-memory budget; the tick is one batched launch (sbs_batch_solve) on
 * the slot's own stream, so the work of consecutive ticks overlaps on the
 * device.  Controllers keep their warm-start distribution and RNG counter on
 * the device between requests.  With plain = 1 the dispatcher instead solves
 * one request at a time with sbs_solve (one launch set per solve), for
 * comparison.  A controller must not be used by the caller while it has a
 * request outstanding; requests of one controller are served in order. */
typedef struct sbs_server sbs_server;

typedef struct sbs_server_config {
    int32_t slots;         /* ticks in flight (streams), 1..8 */
    int32_t max_batch;     /* controllers per tick, >= 1 */
    int32_t max_pending;   /* outstanding requests accepted, >= 1 */
    int32_t plain;         /* 1: serve one request per sbs_solve instead of batching */
    size_t budget_bytes;   /* device workspace budget shared by the slots */
    int32_t samples_per_thread;  /* the slots' batches: 0 (default) or 1, or 2 (sbs_batch_set_samples_per_thread) */
    int32_t theta_mode;    /* the slots' batches: SBS_THETA_STORE (default) or SBS_THETA_REGENERATE; admission
                              counts each request's workspace in this mode (sbs_workspace_bytes_mode) */
} sbs_server_config;

typedef struct sbs_server_stats {
    uint64_t completed;    /* requests finished */
    uint64_t ticks;        /* batched launches (or plain solves) issued */
    double p50_us, p99_us, max_us, mean_us;  /* submit-to-completion latency of finished requests */
    double mean_batch;     /* mean controllers per tick */
    uint64_t admission_waits;  /* times a ready request waited for budget or a slot */
    uint64_t max_inflight;     /* most ticks that were in flight at once */
} sbs_server_stats;

int sbs_server_create(const sbs_server_config* cfg, const sbs_allocator* alloc, sbs_server** out);
void sbs_server_destroy(sbs_server* s);
/* Submit n requests: probs[i] (host memory) for handles[i]; tickets[i] receives
 * each request's ticket.  SBS_ERR_BUDGET: a request whose workspace can never fit
 * a slot; SBS_PENDING: the queue is full (nothing submitted). */
int sbs_server_submit(sbs_server* s, int n, sbs_handle* const* handles, const sbs_problem* probs,
                      uint64_t* tickets);
/* Collect finished requests: status[i] = SBS_OK (result copied into results[i],
 * the ticket retired), SBS_PENDING, or SBS_ERR_INVALID_ARG (unknown ticket). */
int sbs_server_poll(sbs_server* s, int n, const uint64_t* tickets, sbs_result* results, int32_t* status);
/* Latency and throughput statistics since creation (or the last reset). */
int sbs_server_stats_get(sbs_server* s, sbs_server_stats* out, int reset);

/* ---------------------------------------------------------------- utilities */
const char* sbs_status_str(int status);

/* Philox4x32-10 blocks (Salmon et al., SC'11): out[4i..4i+3] = Philox(ctr[4i..],
 * key[2i..]) for i < n.  Device arrays; enqueued on stream. */
int sbs_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* stream);

/* The standard normals the controller with key (seed, ctrl) draws in iteration
 * iter (Alg. 1 Sampling): for samples k0 .. k0 + nk - 1, out[i (nn + 1)] is the
 * frequency normal (draw 0) and out[i (nn + 1) + 1 + n] force normal n < nn
 * (draw 1 + n/6).  Device output of nk (nn + 1) floats; enqueued on stream.
 * Precision: the angle uses the hardware sine/cosine (a normal moves by at most
 * 3e-6); the frequency normal's radius uses the accurate logarithm, the force
 * normals' radius the hardware base-2 logarithm (error at most 2^-22 on
 * [0.5, 2]), which moves the radius r by at most min(2e/r, sqrt(2e)) with
 * e = 2^-22 ln 2: about 1e-6 at typical radii, at most 5.7e-4 at the smallest;
 * their square root is sbs_sqrt_hw's (relative error below 1.1e-7, under one ulp). */
int sbs_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out, void* stream);

/* The square root the rollout takes of the normals' radius and of the friction
 * cone's |Gamma_xy|: y[i] = the hardware approximation of sqrt(x[i]) for i < n
 * (device arrays, enqueued on stream); for tests of its error bound. */
int sbs_sqrt_hw(const float* x, float* y, int n, void* stream);

/* The sine and cosine the model step takes of the attitude angles (Eq. (1):
 * rotation and Euler-rate map): a Cody-Waite reduction by pi/2 and fitted
 * polynomials on [-pi/4, pi/4]; beyond |x| = 65536 and for non-finite x (a
 * diverged rollout) the hardware approximation.  out: 8 n floats = [sin | cos]
 * of the one-sample form, [sin | cos] of the two-sample (packed) form on lane
 * pairs (2m, 2m + 1), [sin | cos] of the library's accurate sincosf and [sin |
 * cos] of the hardware approximation, for tests of the error bound and of the
 * two forms' equality.  Device arrays, enqueued on stream. */
int sbs_sincos(const float* x, float* out, int n, void* stream);

/* Measure the FP32 FMA throughput of the current device with a register-resident
 * FMA chain kernel; returns FLOP/s (2 per FMA) in *flops, or an error. */
int sbs_fp32_peak(double* flops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBS_H */
