// Internal layout shared by the host API and the kernels of libsbs.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/sbs.h"

namespace sbs {

constexpr uint32_t kPhaseOne = 1000000000u;  // one gait cycle in 1e-9 cycle
constexpr int kMaxKnots = 8;
constexpr int kPartHeader = 8;               // floats ahead of the per-dimension sums in a partial row
constexpr int kRefitThreads = 256;

// Per-controller constants and device buffers.  Lives in device memory; every
// kernel copies it into shared memory before use.
struct InstParams {
    int32_t K, H, P, D;
    int32_t nt;        // H (per-step policy) or P (spline knots)
    int32_t nf;        // 12 * nt: length of the force part of theta
    int32_t method, adaptive, Ke, T, ntiles, compare_mppi;
    int32_t part_stride;  // floats per partial row: kPartHeader + nf
    uint32_t dt_us, q_init, seed, ctrl;
    float dt, lambda, inv_lambda, inv_mass, weight_z;
    float inertia[3], inv_inertia[3], foot[12], gravity[3];
    float Q[12], R[3], w_fc, mu, rho, f_nominal, f_min, f_max;
    float var_init, var_min, var_f_init, var_f_min;
    // device buffers owned by the handle
    float* state[2];   // ping-pong distribution: mean[D] then var[D]
    float* J;          // [K]
    int32_t* q;        // [K]
    float* part;       // [ntiles][part_stride]
    int32_t* elite;    // [max(Ke, 1)]
    unsigned* counter; // tiles finished in the current launch
    float* mppi_mean;  // [D]
    const float* Bsp;  // [H][P] spline basis
    const float* Ssp;  // [P][P] spline shift-by-one-step map
};

// Per-solve, per-iteration arguments.
struct TickArgs {
    const float* x0;
    const float* xref;
    const float* fext;   // may be null
    uint32_t offset[4];
    uint32_t duty, phase0;
    int32_t shift;       // warm-start shift applied while staging (first iteration only)
    int32_t src;         // current state buffer; the update writes state[1 - src]
    uint64_t iter;       // Philox iteration counter
    int32_t partials;    // 1: this iteration forms MPPI partial sums
    int32_t mppi_to_state;  // 1: the MPPI combine is the update; 0: it goes to mppi_mean
    sbs_result* result;
};

// One controller of a batched tick: its tick arguments, its parameters and the
// first item of its tiles / refit blocks in the launch's item numbering.
struct InstRec {
    TickArgs t;
    const InstParams* dP;
    int32_t tile_begin;
    int32_t refit_begin;
};

static_assert(sizeof(InstRec) % 16 == 0, "InstRec must be a multiple of 16 bytes");
static_assert(sizeof(InstParams) % 16 == 0, "InstParams must be a multiple of 16 bytes");
static_assert(sizeof(TickArgs) % 8 == 0, "TickArgs must be a multiple of 8 bytes");

// Dynamic shared memory of one rollout item (bytes).
inline size_t rollout_smem_bytes(int H, int P, int T)
{
    int nt = P > 0 ? P : H;
    int nf = 12 * nt;
    int nwarps = T / 32;
    size_t floats = 3 * (size_t)nf   // mean, variance, standard deviation (shifted)
                  + 12 * (size_t)H   // reference
                  + (P > 0 ? (size_t)H * P + 12 * (size_t)H : 0)  // spline basis, mean forces
                  + (size_t)T         // weights
                  + (size_t)nwarps * nf;  // per-warp partial sums
    return floats * sizeof(float);
}

// Host-side launchers (defined in sbs_kernels.cu).
int launch_init(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_rollout(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_refit(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream);
int launch_batch(int P, const InstRec* dRecs, const int* dCounts, int* dHeads, size_t smem, int T, int grid1,
                 int grid2, void* stream);
int batch_grid(int P, size_t smem, int T, int* grid1, int* grid2);
const void* batch_rollout_fn(int P);
const void* batch_refit_fn();
int launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* stream);
int launch_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out, void* stream);
int launch_fma_peak(float* out, int iters, int blocks, int threads, void* stream);

}  // namespace sbs
