// Internal layout shared by the host API and the kernels of libsbs.
#pragma once

#include <cstddef>
#include <cstdint>

#include "sbs.h"  // include/ is on the include path

namespace sbs {

constexpr uint32_t kPhaseOne = 1000000000u;  // one gait cycle in 1e-9 cycle
constexpr int kMaxKnots = 8;
constexpr int kPartHeader = 8;               // floats ahead of the per-dimension sums in a partial row
constexpr int kGroup = 16;                   // tiles whose partial rows one block combines
constexpr int kRefitThreads = 256;       // plain solves: few controllers, possibly many elites per step
constexpr int kRefitLanesMax = 1024;     // virtual lanes of a refit with a large elite set

// Virtual lanes of a refit (the order of its sums, the same for every block
// size): more lanes for a large elite set shorten each lane's chain of loads.
__host__ __device__ inline int refit_lanes(int Ke) { return Ke > 2048 ? kRefitLanesMax : kRefitThreads; }
// Refit items of a batched controller.  An elite set of at most 2048 (one pass of
// kRefitThreads virtual lanes per step) takes several consecutive steps per item,
// about 4096 elite rows each, so one block's set-up serves them all; a larger set
// and Naive take one step per item.  An adaptive controller's frequency entry is
// one more item.  Each step's sums are formed in the same order either way.
constexpr int kRefitChunk = 8;  // steps whose sums a multi-step refit block holds at once
__host__ __device__ inline int refit_steps_per_item(int method, int Ke, int nt)
{
    if (method != SBS_ELITE || Ke > 2048) return 1;
    const int s = 4096 / (Ke > 0 ? Ke : 1);
    return s < 1 ? 1 : (s > nt ? nt : s);
}
__host__ __device__ inline int refit_items(int method, int Ke, int nt, int adaptive)
{
    const int s = refit_steps_per_item(method, Ke, nt);
    return (nt + s - 1) / s + (adaptive ? 1 : 0);
}
constexpr int kBatchRefitThreads = 128;  // batched ticks: thousands of small refit items (8 blocks per SM)
constexpr int kSelectThreads = 1024;
// Selection blocks of a graph-replayed batched tick: the registers of two rollout
// blocks, so a selection starts as soon as two rollout blocks of an SM finish and
// runs beside the rest of the rollout (a 1024-thread block waits for a whole SM).
constexpr int kBatchSelectThreads = 512;
constexpr int kSelectSmemMaxK = 32768;       // costs staged in shared memory up to this K
constexpr size_t kMaxDynamicSmem = 220 * 1024;  // dynamic shared memory one block may use (below the 227 KB
                                                 // opt-in limit, which also covers the static part)

// Per-controller constants and persistent device state.  Lives in device
// memory; every kernel copies it into shared memory before use.
struct InstParams {
    int32_t K, H, P, D;
    int32_t nt;        // H (per-step policy) or P (spline knots)
    int32_t nf;        // 12 * nt: length of the force part of theta
    int32_t method, adaptive, Ke, T, ntiles, ngroups, compare_mppi;
    int32_t part_stride;  // floats per partial row: kPartHeader + nf
    int32_t n_freq;       // discrete step-frequency set size (0: none)
    int32_t nb;           // force blocks of the distribution: n_freq, else 1
    uint32_t freq[SBS_MAX_FREQ];  // the set, mHz
    // model and cost constants read at every step, in 16-byte groups
    float Q[12];
    float R[3], w_fc;
    float foot[12];
    float gyro[3], inv_mass;  // gyro[a] = (I_{a+1} - I_{a+2}) / I_a (indices mod 3)
    float inv_inertia[3], dt;
    float gravity[3], mu;
    int32_t world_feet;   // 1: stance feet fixed on the ground, footholds at touchdown
    float inv_g;          // 1 / |g_z| (foothold rule)
    int32_t friction_project;  // 1: stance forces projected onto the friction cone, no penalty
    float inv_1pmu2;      // 1 / (1 + mu^2)
    float w_terminal;     // terminal state cost weight (0: none)
    uint32_t dt_us, q_init, seed, ctrl;
    float lambda, inv_lambda, weight_z;
    float rho, f_nominal, f_min, f_max;
    float var_init, var_min, var_f_init, var_f_min;
    float* state[2];   // ping-pong distribution: mean[D] then var[D] (nb force blocks of nf, then the frequency)
    float* mppi_mean;  // [D]
    const float* Bsp;  // [H][P] spline basis
    const float* Ssp;  // [P][P] spline shift-by-one-step map
    int32_t pad1[2];
};

// Scratch of one in-flight solve.  Counters are zero whenever no launch uses them.
struct Workspace {
    float* J;          // [K] costs
    int32_t* q;        // [K] quantised step frequencies
    float* theta;      // [nt][K][12] sampled deviations sigma * eps of every sample
    float* part;       // [ntiles][part_stride] tile partial sums (MPPI)
    float* gpart;      // [ngroups][part_stride] group partial sums
    int32_t* elite;    // [Ke] elite indices, ascending; Naive: [nb] per-block winners (-1: none), best block
    unsigned* counters;  // [ngroups + 1] completion counters
    unsigned* hist;    // [65536 + 256] histograms of the top 16 and top 8 cost-key bits (large elite
                       // selections), or null
    unsigned long long* best;  // Naive: [nb] complemented (cost key, index) of each block's best sample, or null
    unsigned* nfin;    // Naive: samples with a finite cost, or null
    uint32_t* cand;    // large elite selections: [K] keys of the threshold bin (low 16 bits), or null
    int32_t* bcnt;     // large elite selections: [2 ceil(K / 2048)] keys below / equal to the threshold per block
    uint32_t* sel;     // large elite selections: [8] selection scratch
};

// Per-solve, per-iteration arguments.
struct TickArgs {
    const float* x0;
    const float* xref;
    const float* fext;   // may be null
    const float* feet;   // world_feet: [4][2] ground (x, y) of the feet at t_0
    uint32_t offset[4];
    uint32_t duty, phase0;
    int32_t shift;       // warm-start shift applied while staging (first iteration only)
    int32_t src;         // current state buffer; the update writes state[1 - src]
    uint64_t iter;       // Philox iteration counter
    int32_t partials;    // 1: this iteration forms MPPI partial sums and combines them; 2: the tile
                         // rows only (a sharded solve combines all ranks' rows afterwards)
    int32_t mppi_to_state;  // 1: the MPPI combine is the update; 0: it goes to mppi_mean
    int32_t regen;       // 1: the sampled deviations are not stored; their readers regenerate them
    int32_t tile_base;   // first tile of a plain rollout launch (a shard of the controller's tiles)
    sbs_result* result;
    Workspace ws;
};

// One controller of a batched tick: its tick arguments, its parameters and the
// first item of its tiles / selection / refit blocks in the launch's numbering.
struct InstRec {
    TickArgs t;
    const InstParams* dP;
    int32_t tile_begin;
    int32_t select_begin;
    int32_t refit_begin;
    int32_t pad[1];
};

static_assert(sizeof(InstRec) % 16 == 0, "InstRec must be a multiple of 16 bytes");
static_assert(sizeof(InstParams) % 16 == 0, "InstParams must be a multiple of 16 bytes");
static_assert(sizeof(TickArgs) % 8 == 0, "TickArgs must be a multiple of 8 bytes");

// Dynamic shared memory of one rollout item (bytes); nb force blocks.
__host__ __device__ inline size_t rollout_smem_bytes(int H, int P, int T, int nb = 1, bool pair = false)
{
    int nt = P > 0 ? P : H;
    int nf = 12 * nt;
    int nwarps = T / 32;
    size_t floats = 3 * (size_t)nb * nf   // mean, variance, standard deviation (shifted)
                  + 12 * (size_t)H   // reference
                  + (P > 0 ? (size_t)H * 4 * ((P + 3) / 4) + 12 * (size_t)nb * H : 0)  // spline basis, mean forces
                  + (P > 0 ? (size_t)48 * ((P + 3) / 4) * T : 0)  // per-thread knot deviations
                  + (P > 0 ? (size_t)nwarps * nf  // per-warp partial sums, then the combined row
                           : (size_t)(6 * T > nf + kPartHeader ? 6 * T : nf + kPartHeader));  // weight list and slice sums, then the combined row
    if (pair)  // duplicated pairs: reference, mean and deviation rows (per-step policy); basis rows (spline)
        floats = ((floats + 3) & ~(size_t)3) + (P > 0 ? 8 * (size_t)((P + 3) / 4) * H : 72 * (size_t)H);
    return floats * sizeof(float);
}

inline size_t select_smem_bytes(int K) { return 4 * (size_t)(K < kSelectSmemMaxK ? K : kSelectSmemMaxK); }

// Byte layout of a workspace inside one allocation (256-byte aligned pieces),
// and the word layout of its zero-when-idle counter block (an even number of
// words starting 8-byte aligned): Naive best keys (2 nb words) and finite count
// (2 words), completion counters (ngroups + 1), histogram.
struct WsLayout {
    size_t J, q, theta, part, gpart, elite, cand, bcnt, sel, bytes;
    size_t theta_bytes;  // the sampled deviations' region; absent when a tick regenerates them
    int ntiles, ngroups, counters;  // counters: zero-when-idle words
    int c_groups, c_hist;           // word offsets of the completion counters and the histogram
    int naive_nb;                   // Naive force blocks (0: not Naive)
    bool hist;
};

constexpr int kHistBins = 65536;

// hist: the solve selects elites from more costs than fit in shared memory, so
// the rollout tiles also build a histogram of the top 16 key bits.  naive_nb:
// the Naive method's force blocks (the rollout keeps each block's best sample).
inline WsLayout ws_layout(int K, int H, int P, int T, int Ke, bool hist = false, int naive_nb = 0)
{
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const int nt = P > 0 ? P : H, nf = 12 * nt;
    WsLayout L;
    L.ntiles = (K + T - 1) / T;
    L.ngroups = (L.ntiles + kGroup - 1) / kGroup;
    L.hist = hist;
    L.naive_nb = naive_nb;
    L.c_groups = naive_nb > 0 ? 2 * naive_nb + 2 : 0;
    L.c_hist = L.c_groups + L.ngroups + 1;
    L.counters = L.c_hist + (hist ? kHistBins + 256 : 0);
    L.counters += L.counters & 1;
    if (naive_nb + 1 > Ke) Ke = naive_nb + 1;
    const size_t PS = kPartHeader + nf;
    size_t o = 0;
    L.J = o; o = up(o + 4 * (size_t)K);
    L.q = o; o = up(o + 4 * (size_t)K);
    L.theta = o; o = up(o + 4 * (size_t)K * nf);
    L.theta_bytes = o - L.theta;
    L.part = o; o = up(o + 4 * (size_t)L.ntiles * PS);
    L.gpart = o; o = up(o + 4 * (size_t)L.ngroups * PS);
    L.elite = o; o = up(o + 4 * (size_t)(Ke > 0 ? Ke : 1));
    const size_t nblk = ((size_t)K + 2047) / 2048;  // blocks of the multi-block selection
    L.cand = o; o = up(o + (hist ? 4 * (size_t)K : 0));
    L.bcnt = o; o = up(o + (hist ? 8 * nblk : 0));
    L.sel = o; o = up(o + (hist ? 32 : 0));
    L.bytes = o;
    return L;
}

// Bytes of a workspace: without the deviations' region when they are regenerated.
inline size_t ws_bytes(const WsLayout& L, bool regen = false) { return L.bytes - (regen ? L.theta_bytes : 0); }

// A workspace at base.  With regen the deviations' region is left out: the
// regions after it move down by its size and theta is null (never read or written).
inline Workspace ws_at(const WsLayout& L, char* base, unsigned* counters, bool regen = false)
{
    Workspace w;
    const size_t sh = regen ? L.theta_bytes : 0;
    w.J = (float*)(base + L.J);
    w.q = (int32_t*)(base + L.q);
    w.theta = regen ? nullptr : (float*)(base + L.theta);
    base -= sh;  // the regions below follow theta
    w.part = (float*)(base + L.part);
    w.gpart = (float*)(base + L.gpart);
    w.elite = (int32_t*)(base + L.elite);
    w.counters = counters + L.c_groups;
    w.hist = L.hist ? counters + L.c_hist : nullptr;
    w.best = L.naive_nb > 0 ? reinterpret_cast<unsigned long long*>(counters) : nullptr;
    w.nfin = L.naive_nb > 0 ? counters + 2 * L.naive_nb : nullptr;
    w.cand = L.hist ? (uint32_t*)(base + L.cand) : nullptr;
    w.bcnt = L.hist ? (int32_t*)(base + L.bcnt) : nullptr;
    w.sel = L.hist ? (uint32_t*)(base + L.sel) : nullptr;
    return w;
}

// Host-side configuration helpers (defined in sbs_api.cu).
int validate_config(const sbs_config* c);
int validate_gait(const sbs_gait* g);
void fill_params(const sbs_config* cfg, InstParams* out);

// Rollout kernel variant of a launch: the policy's knot count (0: per-step
// forces), plus kExtVariant when a controller of the launch uses an extended
// model feature (a discrete step-frequency set, stance feet fixed on the
// ground).  The batched launchers take a variant where they say P.
constexpr int kExtVariant = 256;
constexpr int kPairVariant = 512;    // two samples per thread
constexpr int kRegenVariant = 1024;  // deviations regenerated by the refit (not stored)
constexpr int kAdaptVariant = 2048;  // two samples per thread: a controller of the launch samples its frequency
inline int rollout_variant(int P, bool ext, bool pair = false, bool regen = false, bool adapt = true)
{
    return P | (ext ? kExtVariant : 0) | (pair ? kPairVariant : 0) | (regen ? kRegenVariant : 0) |
           (pair && adapt && P == 0 ? kAdaptVariant : 0);
}
// Launches that can carry two samples per thread: the ordinary model (per-step or
// spline policy), with tiles of a multiple of 64 samples (whole warps of pairs).
inline bool pair_capable(int P, bool ext, int T) { (void)P; return !ext && T % 64 == 0; }
// Dynamic shared memory of a warp-specialised tile: the per-step layout and a
// double buffer of the normals of T samples.
inline size_t ws_smem_bytes(int H, int T, int nb) { return rollout_smem_bytes(H, 0, T, nb) + 96 * (size_t)T; }
// Plain launches that can take the noise warps: the per-step policy (ordinary or
// extended model), whole warps of samples, 2T threads within the block limit.
inline bool ws_capable(int P, bool ext, int H, int T, int nb)
{
    (void)ext;
    return P == 0 && T % 32 == 0 && 2 * T <= 2 * SBS_MAX_TILE && ws_smem_bytes(H, T, nb) <= kMaxDynamicSmem;
}
// ... and whose duplicated rows fit the shared memory of a block.
inline bool pair_fits(int H, int P, int T, int nb) { return rollout_smem_bytes(H, P, T, nb, true) <= kMaxDynamicSmem; }

// Host-side launchers (defined in sbs_kernels.cu).
int launch_init(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_rollout(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream, int spt = 1,
                   int tiles = -1);
int launch_shard_finish(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_cost_keys(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_select(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_refit(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
// A batched tick's device header: two count blocks of 8 ints (the first rollout
// launch, select and refit read the first; a second rollout launch over the MPPI
// controllers' tiles reads the second), then the records.
constexpr int kBatchCountsB = 8;
constexpr size_t kBatchHeader = 64;
// grids: rollout, select, refit, and the second rollout launch (0: none).
int launch_batch(int P, int mode, const InstRec* dRecs, const int* dCounts, int* dHeads, size_t smem,
                 size_t sel_smem, int T, const int grids[4], void* stream, void* const* events);
int batch_grid(int P, int mode, size_t smem, size_t sel_smem, int T, const int counts[4], int grids[3]);
const void* batch_rollout_fn(int P, int mode);
const void* batch_select_fn(int mode);
const void* batch_refit_fn(int mode, bool regen);
int launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* stream);
int launch_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out, void* stream);
int launch_sqrt_hw(const float* x, float* y, int n, void* stream);
int launch_sincos(const float* x, float* out, int n, void* stream);
int launch_fma_peak(float* out, int iters, int blocks, int threads, void* stream);

}  // namespace sbs

// A controller (opaque in the C ABI).
struct sbs_handle {
    sbs_config cfg;
    sbs::InstParams hP;    // host copy (device pointers filled in)
    sbs::InstParams* dP;   // device copy
    char* dev_base;
    size_t dev_bytes;
    sbs_allocator alloc;
    bool has_alloc;
    int device;
    int cur;               // current state buffer
    uint64_t iter;         // Philox iteration counter of the next iteration
    bool initialized;
    sbs::WsLayout wsl;     // layout of one solve's workspace
    sbs::Workspace ws;     // the handle's own workspace (plain solves), allocated on first use
    char* ws_base;         // its allocation (null until the first plain solve)
    float* dev_in;         // device staging of host inputs: x0 (12) | f_ext (3) | pad | feet (8) | xref (12 H)
    sbs_result* res_dev;   // device result for host-memory solves
    float* pin_in;         // pinned host staging of inputs
    void* in_done;         // cudaEvent_t: last copy out of pin_in has run
    bool in_pending;
    uint64_t uid;          // creation number, unique over the process (a reused address gets a new one)
    int spt;               // samples per thread of plain solves: 0 (default: one), 1 or 2
    int regen;             // 1: plain solves do not store the sampled deviations (readers regenerate them)
    bool shard_pending;    // a sample-sharded rollout waits for its update
    int shard_it;          // iteration of the sharded solve in progress (0: its first)
    sbs::TickArgs shard_t; // that rollout's tick arguments
};


