// Kernels of the SBS controller hot path (sm_103a).
//
//  k_rollout   one block per tile of T samples: stage the (warm-shifted) mean,
//              deviation and reference in shared memory, roll every sample out
//              in registers (Alg. 2 with Eq. (1)), accumulate its cost with Kahan
//              compensation and store its sampled deviations sigma * eps.  For
//              MPPI the tile forms max-shifted partial sums of w and
//              w (theta - mean); the last tile of each group of 16 combines the
//              group, the last group the whole controller (Alg. 5).
//              Naive keeps each force block's best (cost, index) with 64-bit
//              atomics instead.  <NP, EXT>: spline knots (0: one force per step);
//              the extended model features (frequency set, ground-fixed feet,
//              friction projection).
//  k_select    one block per elite/naive controller (1024 threads; 512 in a
//              graph-replayed batched tick): radix select of
//              the K_e lowest (cost, index) pairs and their ordered list (Alg. 1
//              Sorting); Naive reads the per-block best keys.
//  k_sel_*     the same selection spread over many blocks, for one controller
//              with more costs than fit in shared memory (plain solves).
//  k_refit     one block per step (or knot): elite mean and diagonal variance
//              (Alg. 1 Update) or the best sample per force block (Alg. 3) from
//              the stored or regenerated deviations; batched ticks give an
//              elite set of at most 2048 several steps per block.
//  k_grid_* / k_batch_*  the same three stages for many controllers: one block
//              per item, or persistent blocks pulling items from device queues.
//  k_init      the initial distribution.
//  k_philox, k_normals  the random numbers the controller draws (tests).
//  k_sqrt_hw  the hardware square root the rollout uses (tests).
//  k_sincos   the attitude sine and cosine of the model step (tests).
//  k_fma_peak  FP32 FMA-chain microbenchmark for the roofline denominator.
#include <cuda_runtime.h>

#include <cstdint>

#include "sbs_device.cuh"

namespace sbs {

constexpr float kInf = __builtin_huge_valf();

struct __align__(16) BlockShared {
    InstParams P;
    TickArgs t;
    float x0[12];
    float fe[3];
    float feet[8];
    float mu_f, var_f, sig_f;
    float red[32][4];
    int item;
    int last;
    int hist[256];
    int wtot[32], wtot2[32];
    unsigned selkmin[32];  // a selection's staging pass: per-warp best key and finite count
    int selnf[32];
    int digit, below, count;
    unsigned char sched[SBS_MAX_H];  // stance legs of every step when all samples share the frequency
    float mu12[12], vr12[12], dbar[12], sd12[12];
    float wacc[32][12];
    float wacc2[kRefitLanesMax / 32][12];
    PairConsts pc;  // model and cost constants as duplicated pairs (two samples per thread)
};

// A shared-memory vector load the compiler may not hoist out of the step loop
// (keeping the knot deviations in shared memory instead of 48 registers).
__device__ __forceinline__ float4 lds4(const float4* p)
{
    float4 r;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(a));
    return r;
}

struct Views {
    float *mu, *vr, *sd, *xr, *Bs, *Mb, *acc;
    float4* dsm;  // spline: per-thread knot deviations [12][nq][T] as float4 (knots padded to 4)
};

// mu, vr, sd: nb force blocks of nf; Mb: nb blocks of 12 H.
__device__ __forceinline__ Views carve(float* base, int H, int P, int nf, int T, int nb)
{
    Views v;
    v.mu = base;
    v.vr = v.mu + nb * nf;
    v.sd = v.vr + nb * nf;
    v.xr = v.sd + nb * nf;
    float* p = v.xr + 12 * H;
    v.dsm = nullptr;
    if (P > 0) {
        const int nq = (P + 3) / 4;
        v.Bs = p;  // [H][4 nq], zero padded
        p += H * 4 * nq;
        v.Mb = p;
        p += 12 * H * nb;
        v.dsm = reinterpret_cast<float4*>(p);
        p += 48 * nq * T;
    } else {
        v.Bs = v.Mb = nullptr;
    }
    v.acc = p;
    return v;
}

__device__ __forceinline__ void load_params(const InstParams* src, BlockShared& sh)
{
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(&sh.P);
    for (int i = threadIdx.x; i < (int)(sizeof(InstParams) / 16); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ void load_tick(const TickArgs* src, BlockShared& sh)
{
    const long long* s = reinterpret_cast<const long long*>(src);
    long long* d = reinterpret_cast<long long*>(&sh.t);
    for (int i = threadIdx.x; i < (int)(sizeof(TickArgs) / 8); i += blockDim.x) d[i] = s[i];
}

// Initial value of force entry idx (reset rule of the warm start, Sec. III-A):
// every leg's mean force at step j is (0, 0, m|g| / n_j), n_j the stance legs of
// the nominal schedule (of the entry's block frequency for a discrete set);
// spline knots carry m|g| / (4 D_f).
__device__ __forceinline__ void init_entry(const InstParams& P, const TickArgs& t, int idx, float& m,
                                           float& v)
{
    const int blk = idx / P.nf, local = idx - blk * P.nf;
    const int axis = local % 3;
    double fz;
    if (P.P > 0) {
        fz = (double)P.weight_z / (4.0 * (double)t.duty / (double)kPhaseOne);
    } else {
        const int j = local / 12;
        const uint32_t q = P.n_freq > 0 ? P.freq[blk] : P.q_init;
        int n = 0;
        for (int i = 0; i < 4; ++i) n += stance_at(t, i, q, P.dt_us, j);
        fz = n > 0 ? (double)P.weight_z / n : 0.0;
    }
    m = axis == 2 ? (float)fz : 0.0f;
    v = P.var_init;
}

// Force entry idx of the distribution after this tick's warm shift (each force
// block moves on its own).
__device__ __forceinline__ void shifted_entry(const InstParams& P, const TickArgs& t, const float* sm,
                                              const float* sv, int idx, float& m, float& v)
{
    if (t.shift <= 0) {
        m = sm[idx];
        v = sv[idx];
        return;
    }
    const int blk = idx / P.nf, local = idx - blk * P.nf;
    if (P.P > 0) {  // spline: knots re-evaluated one step later (shift is 1)
        const int p = local / 12, c = local % 12;
        const float* smb = sm + blk * P.nf;
        float s = 0.0f;
        for (int r = 0; r < P.P; ++r) s = fmaf(P.Ssp[p * P.P + r], smb[12 * r + c], s);
        m = s;
        v = sv[idx];
        return;
    }
    const int j = local / 12;
    if (j + t.shift < P.H) {
        m = sm[idx + 12 * t.shift];
        v = sv[idx + 12 * t.shift];
    } else {
        init_entry(P, t, idx, m, v);
    }
}

// Stage the shifted distribution, the reference, x0 and f_ext.
__device__ void stage(BlockShared& sh, const Views& v, int P_knots)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const float* sm = P.state[t.src];
    const float* sv = sm + P.D;
    for (int i = threadIdx.x; i < P.nb * P.nf; i += blockDim.x) {
        float m, var;
        shifted_entry(P, t, sm, sv, i, m, var);
        v.mu[i] = m;
        v.vr[i] = var;
        v.sd[i] = sqrtf(var);
    }
    for (int i = threadIdx.x; i < 12 * P.H; i += blockDim.x) v.xr[i] = t.xref[i];
    if (P_knots > 0) {
        const int w4 = 4 * ((P_knots + 3) / 4);
        for (int i = threadIdx.x; i < P.H * w4; i += blockDim.x) {
            const int j = i / w4, p = i % w4;
            v.Bs[i] = p < P_knots ? P.Bsp[j * P_knots + p] : 0.0f;
        }
    }

    if (threadIdx.x < 12) sh.x0[threadIdx.x] = t.x0[threadIdx.x];
    if (threadIdx.x < 3) sh.fe[threadIdx.x] = t.fext ? t.fext[threadIdx.x] : 0.0f;
    if (threadIdx.x < 8) sh.feet[threadIdx.x] = P.world_feet ? t.feet[threadIdx.x] : 0.0f;
    if (threadIdx.x == 0) {
        if (P.adaptive) {
            sh.mu_f = sm[P.D - 1];
            sh.var_f = sv[P.D - 1];
        } else {
            sh.mu_f = P.q_init * 0.001f;
            sh.var_f = 0.0f;
        }
        sh.sig_f = sqrtf(sh.var_f);
    }
    if (P_knots == 0 && !P.adaptive && P.n_freq == 0) {  // one contact schedule for every sample
        const uint64_t step = (uint64_t)P.q_init * P.dt_us;
        for (int j = threadIdx.x; j < P.H; j += blockDim.x) {
            unsigned st = 0;
            for (int i = 0; i < 4; ++i) {
                const uint32_t p0 = t.phase0 + t.offset[i];
                const uint64_t ph = ((uint64_t)(p0 >= kPhaseOne ? p0 - kPhaseOne : p0) + (uint64_t)j * step) % kPhaseOne;
                st |= (ph < t.duty ? 1u : 0u) << i;
            }
            sh.sched[j] = (unsigned char)st;
        }
    }
    __syncthreads();
    if (P_knots > 0) {  // mean force trajectory of each block's spline mean
        for (int i = threadIdx.x; i < 12 * P.H * P.nb; i += blockDim.x) {
            const int blk = i / (12 * P.H), r = i - blk * 12 * P.H;
            const int j = r / 12, c = r % 12;
            const float* mub = v.mu + blk * P.nf;
            float s = 0.0f;
            for (int p = 0; p < P_knots; ++p) s = fmaf(v.Bs[j * 4 * ((P_knots + 3) / 4) + p], mub[12 * p + c], s);
            v.Mb[i] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Block-wide helpers (blockDim a multiple of 32, at most 1024)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float block_min(BlockShared& sh, float v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_min(v);
    __syncthreads();
    if (lane == 0) sh.red[warp][0] = v;
    __syncthreads();
    float m = sh.red[0][0];
    for (int w = 1; w < nw; ++w) m = fminf(m, sh.red[w][0]);
    __syncthreads();
    return m;
}

// Exclusive prefix of per-thread counts over the block in thread order; *total
// gets the block sum.
__device__ __forceinline__ int block_scan(BlockShared& sh, int v, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) sh.wtot[warp] = incl;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        const int x = sh.wtot[w];
        if (w < warp) off += x;
        tot += x;
    }
    __syncthreads();
    *total = tot;
    return off + incl - v;
}

// Sum of 12 per-thread values over the block in a fixed order: warp transpose
// sums, then the warps' totals in warp order.  Threads < 12 receive component
// threadIdx.x in *out_c.
__device__ __forceinline__ float block_sum12(BlockShared& sh, const float v[12])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float o[3];
    const int c0 = warp_sum12(v, o);
    __syncthreads();
    if ((lane & 7) == 0) {
        sh.wacc[warp][c0] = o[0];
        sh.wacc[warp][c0 + 1] = o[1];
        sh.wacc[warp][c0 + 2] = o[2];
    }
    __syncthreads();
    float tot = 0.0f;
    if (threadIdx.x < 12)
        for (int w = 0; w < nw; ++w) tot += sh.wacc[w][threadIdx.x];
    __syncthreads();
    return tot;
}

// ---------------------------------------------------------------------------
// Combine nrows partial rows (stride PS) in row order (Alg. 5 with max shift):
// m = min_t m_t; each row scaled by exp(-(m_t - m) / lambda) (squared for the
// sum of squared weights, none for the finite count); Kahan sums per column.
// out (nf + kPartHeader floats, shared memory) gets the combined row.
// ---------------------------------------------------------------------------
__device__ void combine_rows(BlockShared& sh, const float* rows, int nrows, int PS, int nf, float inv_lambda,
                             float* out)
{
    const int tid = threadIdx.x, T = blockDim.x;
    float m = kInf;
    for (int i = tid; i < nrows; i += T) m = fminf(m, __ldcg(rows + (size_t)i * PS));
    m = block_min(sh, m);
    const int ncol = nf + 4;
    for (int col = tid; col < ncol; col += T) {
        const int off = col < 4 ? 1 + col : kPartHeader + (col - 4);
        float s = 0.0f, c = 0.0f;
        for (int i0 = 0; i0 < nrows; i0 += 8) {
            float mt[8], x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u;
                mt[u] = i < nrows ? __ldcg(rows + (size_t)i * PS) : kInf;
                x[u] = i < nrows ? __ldcg(rows + (size_t)i * PS + off) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (i0 + u < nrows) {
                    const float sc = mt[u] < kInf ? expf(-(mt[u] - m) * inv_lambda) : 0.0f;
                    const float term = col == 3 ? x[u] : (col == 1 ? x[u] * sc * sc : x[u] * sc);
                    kahan_add(s, c, term);
                }
            }
        }
        out[off] = s;
    }
    if (tid == 0) {
        out[0] = m;
        out[5] = out[6] = out[7] = 0.0f;
    }
    __syncthreads();
}

// The MPPI update from the combined row: mean = mu + A / S, variance kept
// (Alg. 5: the covariance is unchanged), and the result record.
__device__ void mppi_finish(BlockShared& sh, const Views& v, const float* row, bool to_state)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, T = blockDim.x;
    const float m = row[0], S = row[1];
    const bool ok = S > 0.0f && m < kInf;
    const float invS = ok ? 1.0f / S : 0.0f;
    float* out_mean = to_state ? P.state[1 - t.src] : P.mppi_mean;
    float* out_var = P.state[1 - t.src] + P.D;
    for (int d = tid; d < P.nf; d += T) {
        out_mean[d] = ok ? v.mu[d] + row[kPartHeader + d] * invS : v.mu[d];
        if (to_state) out_var[d] = v.vr[d];
    }
    const float fmean = P.adaptive ? (ok ? row[3] * invS : sh.mu_f) : sh.mu_f;
    if (tid == 0 && P.adaptive) {
        out_mean[P.D - 1] = fmean;
        if (to_state) out_var[P.D - 1] = sh.var_f;
    }
    if (to_state) {
        sbs_result* r = t.result;
        if (tid < 12) {
            const uint32_t ph = (t.phase0 + t.offset[tid / 3]) % kPhaseOne;
            const float md = ok ? v.mu[tid] + row[kPartHeader + tid] * invS : v.mu[tid];
            r->u0[tid] = ph < t.duty ? md : 0.0f;
        }
        if (tid == 0) {
            r->cost_min = m;
            r->ess = ok ? S * S / row[2] : 0.0f;
            r->f_mean = fmean;
            r->q_freq = (int32_t)quantise_mhz(fmean, P.f_min, P.f_max);
            r->status = ok ? SBS_OK : SBS_ERR_DIVERGED;
            r->n_finite = (int32_t)row[4];
            r->iter_lo = (uint32_t)t.iter;
            r->iter_hi = (uint32_t)(t.iter >> 32);
        }
    }
    __syncthreads();
}

// One listed sample's contribution w d to a float4 column of a tile's row, with
// Kahan compensation (the weighted mean of Alg. 5 summed over the tile).
__device__ __forceinline__ void kahan_wsum4(float4& s, float4& c, float w, float4 d)
{
    kahan_add(s.x, c.x, __fmul_rn(w, d.x));
    kahan_add(s.y, c.y, __fmul_rn(w, d.y));
    kahan_add(s.z, c.z, __fmul_rn(w, d.z));
    kahan_add(s.w, c.w, __fmul_rn(w, d.w));
}

// ---- hierarchical combine: the last tile of a group of kGroup tiles combines
// the group's rows in tile order; the last group combines the group rows, and the
// last block of all finishes the MPPI update.
__device__ void group_combine(BlockShared& sh, const Views& v, int g);

__device__ void tile_combine(BlockShared& sh, const Views& v, int tile)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int g = tile / kGroup;
    const int gsize = min(kGroup, P.ntiles - g * kGroup);
    unsigned* counters = t.ws.counters;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&counters[g], 1u);
        sh.last = prev == (unsigned)gsize - 1u;
    }
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    group_combine(sh, v, g);
}

// Group g's rows combined in tile order (every row of the group written); the
// last group to finish combines the group rows and finishes the update.
__device__ void group_combine(BlockShared& sh, const Views& v, int g)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, T = blockDim.x;
    const int PS = P.part_stride;
    const int gsize = min(kGroup, P.ntiles - g * kGroup);
    unsigned* counters = t.ws.counters;
    float* comb = v.acc;  // nf + kPartHeader floats (blockDim >= 64 leaves room)
    const float* src_rows = t.ws.part + (size_t)g * kGroup * PS;
    combine_rows(sh, src_rows, gsize, PS, P.nf, P.inv_lambda, comb);
    if (P.ngroups > 1) {
        float* grow = t.ws.gpart + (size_t)g * PS;
        for (int i = tid; i < PS; i += T) grow[i] = comb[i];
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            counters[g] = 0u;
            const unsigned prev = atomicAdd(&counters[P.ngroups], 1u);
            sh.last = prev == (unsigned)P.ngroups - 1u;
        }
        __syncthreads();
        if (!sh.last) return;
        __threadfence();
        combine_rows(sh, t.ws.gpart, P.ngroups, PS, P.nf, P.inv_lambda, comb);
        if (tid == 0) counters[P.ngroups] = 0u;
    } else if (tid == 0) {
        counters[g] = 0u;
    }
    mppi_finish(sh, v, comb, t.mppi_to_state != 0);
}

// Reference, mean and deviation rows as duplicated pairs for the two-sample
// rollout ([12 H] float2 each), after the per-step layout (16-byte aligned).
__device__ __forceinline__ float2* pair_ref(const Views& v, const InstParams& P, int T)
{
    const int acc = 6 * T > P.nf + kPartHeader ? 6 * T : P.nf + kPartHeader;
    return reinterpret_cast<float2*>(v.acc + ((acc + 3) & ~3));
}

// Optional terminal cost of the state after the last step: w_T sum_c Q_c
// (x_H - x^r_{H-1})^2.
__device__ __forceinline__ float terminal_cost(const InstParams& P, const float x[12], const float* xr)
{
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float e = __fsub_rn(x[c], xr[c]);
        r = __fmaf_rn(__fmul_rn(P.Q[c], e), e, r);
    }
    return __fmul_rn(P.w_terminal, r);
}

// Step-frequency regulariser rho (q / 1000 - f_n)^2 (Sec. V).
__device__ __forceinline__ float freq_regulariser(const InstParams& P, uint32_t q)
{
    const float d = __fsub_rn(__fdiv_rn((float)q, 1000.0f), P.f_nominal);
    return __fmul_rn(__fmul_rn(P.rho, d), d);
}

// ---------------------------------------------------------------------------
// One tile of T samples.  NP = 0: per-step forces; NP > 0: NP spline knots.
// EXT: the launch may hold controllers with the extended model features: a
// discrete step-frequency set (each sample reads the force Gaussian of its
// draw) or stance feet fixed on the ground (per-sample footholds).  Without it
// every sample reads block 0 at addresses uniform across the warp and uses the
// body-fixed lever arms (a separate instantiation: per-thread addressing alone
// costs the common case ~3 %).
// ---------------------------------------------------------------------------
template <int NP, bool EXT>
__device__ void rollout_tile(BlockShared& sh, float* dyn, int tile)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const Views v = carve(dyn, P.H, NP, P.nf, T, P.nb);
    stage(sh, v, NP);

    const int K = P.K;
    const uint32_t k = (uint32_t)tile * (uint32_t)T + (uint32_t)tid;
    const bool valid = k < (uint32_t)K;
    const uint32_t seed = P.seed, ctrl = P.ctrl;
    const uint64_t iter = t.iter;
    float* theta = t.ws.theta;
    uint32_t q = P.q_init;
    int blk = 0;  // force block: the sample's entry of a discrete frequency set
    if (P.adaptive) {
        q = sample_freq(k, iter, seed, ctrl, sh.mu_f, sh.sig_f, P.f_min, P.f_max);
    } else if constexpr (EXT) {
        if (P.n_freq > 0) {
            blk = freq_block(k, iter, seed, ctrl, P.n_freq);
            q = P.freq[blk];
        }
    }
    const float* mu = v.mu + blk * P.nf;  // this sample's Gaussian
    const float* sd = v.sd + blk * P.nf;

    float x[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) x[c] = sh.x0[c];
    const float fe[3] = {sh.fe[0], sh.fe[1], sh.fe[2]};
    uint32_t ph[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t p0 = t.phase0 + t.offset[i];
        ph[i] = p0 >= kPhaseOne ? p0 - kPhaseOne : p0;
    }
    const uint32_t step = q * P.dt_us;
    const bool uniform_q = NP == 0 && !P.adaptive && P.n_freq == 0;
    const uint32_t duty = t.duty;
    // world-fixed feet: ground positions, last step's stance flags, T_st / 2
    float fx[4], fy[4];
    unsigned prev = 0xfu;  // legs in stance at t_0 keep the given feet
    float tsh = 0.0f;
    if constexpr (EXT) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            fx[i] = sh.feet[2 * i];
            fy[i] = sh.feet[2 * i + 1];
        }
        tsh = (0.5e-6f * (float)duty) / (float)q;
    }

    constexpr int NQ = NP > 0 ? (NP + 3) / 4 : 1;
    if constexpr (NP > 0) {
        float* dsf = reinterpret_cast<float*>(v.dsm);
#pragma unroll 1
        for (int p = 0; p < 4 * NQ; ++p) {
            float e[12];
            if (p < NP) {
                normals12(k, p, iter, seed, ctrl, e);
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = __fmul_rn(sd[12 * p + c], e[c]);
                if (valid && !t.regen) {
                    float4* o = reinterpret_cast<float4*>(theta + ((size_t)p * K + k) * 12);
                    o[0] = make_float4(e[0], e[1], e[2], e[3]);
                    o[1] = make_float4(e[4], e[5], e[6], e[7]);
                    o[2] = make_float4(e[8], e[9], e[10], e[11]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) dsf[(((size_t)c * NQ + p / 4) * T + tid) * 4 + (p & 3)] = e[c];
        }
    }

    float J = 0.0f, Jc = 0.0f;
    const PhiloxPre pp = philox_pre(k, iter, seed, ctrl);
    for (int j = 0; j < P.H; ++j) {
        float G[12];
        if constexpr (NP == 0) {
            float e[12];
            normals12(pp, j, e);
            const float4* m4 = reinterpret_cast<const float4*>(mu + 12 * j);  // 16-byte aligned rows
            const float4* s4 = reinterpret_cast<const float4*>(sd + 12 * j);
            // force mu + sigma eps (one rounding); the deviation sigma eps itself only
            // where it is stored
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 ma = m4[q], sa = s4[q];
                const float mv[4] = {ma.x, ma.y, ma.z, ma.w}, sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) G[4 * q + i] = __fmaf_rn(sv[i], e[4 * q + i], mv[i]);
            }
            if (!t.regen) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float4 sa = s4[q];
                    const float sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) e[4 * q + i] = __fmul_rn(sv[i], e[4 * q + i]);
                }
                if (valid) {
                    float4* o = reinterpret_cast<float4*>(theta + ((size_t)j * K + k) * 12);
                    o[0] = make_float4(e[0], e[1], e[2], e[3]);
                    o[1] = make_float4(e[4], e[5], e[6], e[7]);
                    o[2] = make_float4(e[8], e[9], e[10], e[11]);
                }
            }
        } else {
            const float4* b4 = reinterpret_cast<const float4*>(v.Bs + j * 4 * NQ);
            const float4* m4 = reinterpret_cast<const float4*>(v.Mb + blk * 12 * P.H + 12 * j);  // 16-byte aligned
            const float4 ma = m4[0], mb = m4[1], mc = m4[2];
            const float mrow[12] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w, mc.x, mc.y, mc.z, mc.w};
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                float s = mrow[c];
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) {
                    const float4 b = b4[qq];
                    const float4 d = lds4(v.dsm + (c * NQ + qq) * T + tid);
                    s = fmaf(b.x, d.x, s);
                    s = fmaf(b.y, d.y, s);
                    s = fmaf(b.z, d.z, s);
                    s = fmaf(b.w, d.w, s);
                }
                G[c] = s;
            }
        }
        // legs in swing on the whole warp skip their terms (per-step forces only:
        // the spline kernel runs faster without the branches); swing forces are
        // zeroed only where a leg is live on the warp but swings on some lanes
        unsigned st, live, all;
        if (uniform_q) {  // the block-wide schedule
            st = sh.sched[j];
            live = NP == 0 ? st : 0xfu;
            all = st;
        } else {
            st = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) st |= (ph[i] < duty ? 1u : 0u) << i;
            live = NP == 0 ? __reduce_or_sync(kFull, st) : 0xfu;
            all = NP == 0 ? __reduce_and_sync(kFull, st) : st;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ph[i] += step;
                if (ph[i] >= kPhaseOne) ph[i] -= kPhaseOne;
            }
        }
        if (live != all) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (!(st & (1u << i))) G[3 * i] = G[3 * i + 1] = G[3 * i + 2] = 0.0f;
        }
        bool penalty = true;
        if constexpr (EXT) {
            if (P.friction_project) {  // the policy output constrained to the cone (Sec. IV-B)
#pragma unroll
                for (int i = 0; i < 4; ++i) cone_project(P.mu, P.inv_1pmu2, G[3 * i], G[3 * i + 1], G[3 * i + 2]);
                penalty = false;
            }
        }
        kahan_add(J, Jc, stage_cost(P, x, v.xr + 12 * j, G, live, penalty));
        if constexpr (EXT) {
            if (P.world_feet) {
                const unsigned touch = st & ~prev;  // legs landing at this step
                prev = st;
                srbd_step_world(P, x, G, fe, live, fx, fy, touch, v.xr[12 * j + 6], v.xr[12 * j + 7], tsh);
            } else {
                srbd_step(P, x, G, fe, live);
            }
        } else {
            srbd_step(P, x, G, fe, live);
        }
    }
    if (P.w_terminal > 0.0f) kahan_add(J, Jc, terminal_cost(P, x, v.xr + 12 * (P.H - 1)));
    if (P.adaptive || P.n_freq > 0) kahan_add(J, Jc, freq_regulariser(P, q));
    if (!isfinite(J)) J = kInf;
    if (valid) {
        t.ws.J[k] = J;
        t.ws.q[k] = (int32_t)q;
    }
    if (t.ws.hist) {
        // histograms of the top 16 and top 8 key bits for a large elite selection
        // (one atomic per distinct bin and warp)
        const uint32_t bin = cost_key(J) >> 16;
        const unsigned act = __ballot_sync(kFull, valid);
        if (valid) {
            const unsigned peers = __match_any_sync(act, bin);
            if (lane == __ffs(peers) - 1) atomicAdd(t.ws.hist + bin, (unsigned)__popc(peers));
            const unsigned peers8 = __match_any_sync(act, bin >> 8);
            if (lane == __ffs(peers8) - 1) atomicAdd(t.ws.hist + kHistBins + (bin >> 8), (unsigned)__popc(peers8));
        }
    }
    if (t.ws.best) {
        // Naive: each force block's best finite (cost, index), kept as the maximum of
        // the complemented 64-bit key; one atomic per warp and block present
        const bool fin = valid && J < kInf;
        const unsigned long long key = fin ? ~(((unsigned long long)cost_key(J) << 32) | k) : 0ull;
        unsigned todo = __reduce_or_sync(kFull, fin ? 1u << blk : 0u);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            unsigned long long m = blk == b ? key : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long x = __shfl_xor_sync(kFull, m, o);
                m = x > m ? x : m;
            }
            if (lane == 0) atomicMax(t.ws.best + b, m);
        }
        const unsigned nfw = __popc(__ballot_sync(kFull, fin));
        if (lane == 0 && nfw) atomicAdd(t.ws.nfin, nfw);
    }
    if (!t.partials) return;

    // ---- MPPI partial sums of this tile, shifted by the tile's best cost
    const bool fin = valid && J < kInf;
    const float mt = block_min(sh, fin ? J : kInf);
    const float w = (fin && mt < kInf) ? expf(-(J - mt) * P.inv_lambda) : 0.0f;
    const float f = (float)q / 1000.0f;
    {
        const float s0 = warp_sum(w), s1 = warp_sum(w * w), s2 = warp_sum(w * f), s3 = warp_sum(fin ? 1.0f : 0.0f);
        if (lane == 0) {
            sh.red[warp][0] = s0;
            sh.red[warp][1] = s1;
            sh.red[warp][2] = s2;
            sh.red[warp][3] = s3;
        }
    }
    const int PS = P.part_stride;
    float* row = t.ws.part + (size_t)tile * PS;
    if constexpr (NP == 0) {
        // Weighted deviation sums over the tile's samples of nonzero weight (the rest
        // underflowed, are non-finite or lie past K).  Those samples are listed in
        // shared memory in sample order; thread i then owns float4 column c = i mod 3H
        // of the tile's row (step c / 3, forces 4 (c mod 3) .. +3) and slice
        // s = i / 3H of the list (every nsl-th entry), so each deviation row is read
        // once, by three threads, with no cross-lane reduction; the slices' sums
        // are added in slice order.
        float2* lst = reinterpret_cast<float2*>(v.acc);  // (weight, sample) per listed sample
        const unsigned nzb = __ballot_sync(kFull, w != 0.0f);
        if (lane == 0) sh.wtot[warp] = __popc(nzb);
        __syncthreads();
        int pos = 0, nnz = 0;
        for (int g = 0; g < nw; ++g) {
            const int c = sh.wtot[g];
            pos += g < warp ? c : 0;
            nnz += c;
        }
        if (w != 0.0f) lst[pos + __popc(nzb & ((1u << lane) - 1u))] = make_float2(w, __int_as_float(tid));
        __syncthreads();
        const int ncol = 3 * P.H;
        const int nsl = ncol < T ? T / ncol : 1;
        float4* slice_sum = reinterpret_cast<float4*>(v.acc + 2 * T);  // [nsl][ncol] when nsl > 1
        const float4* th4 = reinterpret_cast<const float4*>(theta) + (size_t)tile * T * 3;
        float4* row4 = reinterpret_cast<float4*>(row + kPartHeader);
        for (int it = tid; it < nsl * ncol; it += T) {
            const int sl = it / ncol, c = it - sl * ncol, j = c / 3;
            const float4* src = th4 + (size_t)j * K * 3 + (c - 3 * j);
            const float4 sd4 = reinterpret_cast<const float4*>(v.sd + 12 * j)[c - 3 * j];
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ac = a;
            if (t.regen) {  // the listed samples' deviations regenerated from their draws
#pragma unroll 1
                for (int e = sl; e < nnz; e += nsl) {
                    const float2 we = lst[e];
                    const float4 d = regen_quad((uint32_t)(tile * T + __float_as_int(we.y)), j, c - 3 * j, t.iter,
                                                P.seed, P.ctrl, sd4);
                    kahan_wsum4(a, ac, we.x, d);
                }
            } else {
#pragma unroll 4
                for (int e = sl; e < nnz; e += nsl) {
                    const float2 we = lst[e];
                    const float4 d = src[3 * __float_as_int(we.y)];
                    kahan_wsum4(a, ac, we.x, d);
                }
            }
            if (nsl == 1) row4[c] = a;
            else slice_sum[it] = a;
        }
        if (nsl > 1) {
            __syncthreads();
            for (int c = tid; c < ncol; c += T) {
                float4 a = slice_sum[c];
                for (int sl = 1; sl < nsl; ++sl) {
                    const float4 b = slice_sum[sl * ncol + c];
                    a.x += b.x;
                    a.y += b.y;
                    a.z += b.z;
                    a.w += b.w;
                }
                row4[c] = a;
            }
        }
    } else {
        // A warp whose weights all underflowed to zero contributes exact zeros.
        const bool warp_live = __any_sync(kFull, w != 0.0f);
        const float* dsf = reinterpret_cast<const float*>(v.dsm);
        if (!warp_live) {
            for (int d = lane; d < P.nf; d += 32) v.acc[warp * P.nf + d] = 0.0f;
        } else {
#pragma unroll 1
            for (int p = 0; p < NP; ++p) {
                float vv[12], o[3];
#pragma unroll
                for (int c = 0; c < 12; ++c) vv[c] = __fmul_rn(w, dsf[(((size_t)c * NQ + p / 4) * T + tid) * 4 + (p & 3)]);
                const int c0 = warp_sum12(vv, o);
                if ((lane & 7) == 0) {
                    float* a = v.acc + warp * P.nf + 12 * p + c0;
                    a[0] = o[0];
                    a[1] = o[1];
                    a[2] = o[2];
                }
            }
        }
        __syncthreads();
        for (int d = tid; d < P.nf; d += T) {
            float s = 0.0f;
            for (int ww = 0; ww < nw; ++ww) s += v.acc[ww * P.nf + d];
            row[kPartHeader + d] = s;
        }
    }
    if (tid == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int ww = 0; ww < nw; ++ww) {
            a0 += sh.red[ww][0];
            a1 += sh.red[ww][1];
            a2 += sh.red[ww][2];
            a3 += sh.red[ww][3];
        }
        row[0] = mt;
        row[1] = a0;
        row[2] = a1;
        row[3] = a2;
        row[4] = a3;
    }

    if (t.partials == 1) tile_combine(sh, v, tile);
}

// ---------------------------------------------------------------------------
// One tile of T samples with two samples per thread: the per-step policy on the
// ordinary model (no spline, no extended feature).  Thread i of the T / 2
// threads carries samples i and i + T / 2 of the tile as the two lanes of float2
// values, so the FP32 arithmetic of the model step, the stage cost, Box-Muller
// and the Kahan sum issues as packed FP32x2 instructions; the Philox rounds, the
// transcendentals and the stores stay per sample.  Every sample sees the same
// operations in the same order as in rollout_tile<0, false>, and the tile's
// reductions run over the same samples in the same order (virtual warp
// s (T / 64) + w holds samples 32 (s (T / 64) + w) ..), so the results are
// bit-identical to the one-sample-per-thread launch on the same tile.  ADAPT:
// the launch may hold a controller that samples its step frequency; without it
// every sample takes the block's contact table and the per-sample phase counter
// is not compiled (fewer registers, no spills).  With it, each sample carries
// one gait phase and forms its legs' phases from the block's offsets at every
// step (one register instead of four).  Each step forms the attitude and the
// state part of the stage cost (which read the state only) ahead of the draws,
// in the same straight-line block, so that their dependency chains interleave
// with the sampler's (3.5 % off the 256-controller tick).
// ---------------------------------------------------------------------------
template <bool ADAPT>
__device__ void rollout_tile_pair(BlockShared& sh, float* dyn, int tile)
{
    using L = Lane<float2>;
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int T2 = blockDim.x, T = 2 * T2, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw2 = T2 >> 5;
    const Views v = carve(dyn, P.H, 0, P.nf, T, P.nb);
    float2* xr2 = pair_ref(v, P, T);  // reference, mean and deviation rows as duplicated pairs
    float2* mu2 = xr2 + 12 * P.H;
    float2* sd2 = mu2 + 12 * P.H;
    stage(sh, v, 0);
    for (int i = tid; i < 12 * P.H; i += T2) {
        xr2[i] = make_float2(v.xr[i], v.xr[i]);
        mu2[i] = make_float2(v.mu[i], v.mu[i]);
        sd2[i] = make_float2(v.sd[i], v.sd[i]);
    }
    fill_pair_consts(sh.pc, P, sh.fe);
    __syncthreads();
    const Consts<float2> Kc{sh.pc};

    const int K = P.K;
    const uint32_t seed = P.seed, ctrl = P.ctrl;
    const uint64_t iter = t.iter;
    float* theta = t.ws.theta;
    uint32_t k[2], q[2];
    bool valid[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        k[l] = (uint32_t)tile * (uint32_t)T + (uint32_t)(l * T2 + tid);
        valid[l] = k[l] < (uint32_t)K;
        q[l] = (ADAPT && P.adaptive) ? sample_freq(k[l], iter, seed, ctrl, sh.mu_f, sh.sig_f, P.f_min, P.f_max)
                                     : P.q_init;
    }
    const float* sd = v.sd;

    float2 x[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) x[c] = L::bc(sh.x0[c]);
    const float2 fe[3] = {sh.pc.fe[0], sh.pc.fe[1], sh.pc.fe[2]};
    const bool uniform_q = !ADAPT || !P.adaptive;
    uint32_t ph[2], step[2];
    if constexpr (ADAPT) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            step[l] = q[l] * P.dt_us;
            ph[l] = t.phase0;
        }
    }
    const uint32_t duty = t.duty;

    float2 J = L::bc(0.0f), Jc = L::bc(0.0f);
    const PhiloxPre pp0 = philox_pre(k[0], iter, seed, ctrl), pp1 = philox_pre(k[1], iter, seed, ctrl);
    for (int j = 0; j < P.H; ++j) {
        const Attitude<float2> A = attitude_v<float2>(x);
        const float2 cost_x = stage_state_cost_v<float2>(Kc, x, xr2 + 12 * j);
        float2 z[12];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const uint4 w[2] = {philox_draw(pp0, 1u + 2u * (uint32_t)j + (uint32_t)d),
                                philox_draw(pp1, 1u + 2u * (uint32_t)j + (uint32_t)d)};
            normals6_v<float2>(w, z + 6 * d);
        }
        // forces mu + sigma eps as lane pairs (one rounding, packed); the deviations
        // sigma eps per sample only where they are stored (48 B per sample)
        float2 G[12];
        {
            const float4* m2 = reinterpret_cast<const float4*>(mu2 + 12 * j);  // duplicated pairs
            const float4* s2 = reinterpret_cast<const float4*>(sd2 + 12 * j);
#pragma unroll
            for (int qq = 0; qq < 6; ++qq) {
                const float4 ma = m2[qq], sa = s2[qq];
                G[2 * qq] = L::fma(make_float2(sa.x, sa.y), z[2 * qq], make_float2(ma.x, ma.y));
                G[2 * qq + 1] = L::fma(make_float2(sa.z, sa.w), z[2 * qq + 1], make_float2(ma.z, ma.w));
            }
        }
        if (!t.regen) {
            const float4* s4 = reinterpret_cast<const float4*>(sd + 12 * j);  // 16-byte aligned rows
            float eA[12], eB[12];
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
                const float4 sa = s4[qq];
                const float sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    eA[4 * qq + i] = __fmul_rn(sv[i], z[4 * qq + i].x);
                    eB[4 * qq + i] = __fmul_rn(sv[i], z[4 * qq + i].y);
                }
            }
            if (valid[0]) {
                float4* o = reinterpret_cast<float4*>(theta + ((size_t)j * K + k[0]) * 12);
                o[0] = make_float4(eA[0], eA[1], eA[2], eA[3]);
                o[1] = make_float4(eA[4], eA[5], eA[6], eA[7]);
                o[2] = make_float4(eA[8], eA[9], eA[10], eA[11]);
            }
            if (valid[1]) {
                float4* o = reinterpret_cast<float4*>(theta + ((size_t)j * K + k[1]) * 12);
                o[0] = make_float4(eB[0], eB[1], eB[2], eB[3]);
                o[1] = make_float4(eB[4], eB[5], eB[6], eB[7]);
                o[2] = make_float4(eB[8], eB[9], eB[10], eB[11]);
            }
        }
        // stance: legs in swing on every sample of the warp skip their terms; swing
        // forces are zeroed where a leg is live on the warp but swings on a sample
        unsigned st[2], live, all;
        if (uniform_q) {
            st[0] = st[1] = live = all = sh.sched[j];
        } else if constexpr (ADAPT) {
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                st[l] = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint32_t pi = ph[l] + sh.t.offset[i];
                    if (pi >= kPhaseOne) pi -= kPhaseOne;
                    st[l] |= (pi < duty ? 1u : 0u) << i;
                }
                ph[l] += step[l];
                if (ph[l] >= kPhaseOne) ph[l] -= kPhaseOne;
            }
            live = __reduce_or_sync(kFull, st[0] | st[1]);
            all = __reduce_and_sync(kFull, st[0] & st[1]);
        }
        if (live != all) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (!(st[0] & (1u << i))) G[3 * i].x = G[3 * i + 1].x = G[3 * i + 2].x = 0.0f;
                if (!(st[1] & (1u << i))) G[3 * i].y = G[3 * i + 1].y = G[3 * i + 2].y = 0.0f;
            }
        }
        kahan_add_v<float2>(J, Jc, stage_force_cost_v<float2>(Kc, cost_x, G, live, true));
        srbd_step_att_v<float2>(Kc, x, G, fe, live, A);
    }
    float Jv[2] = {J.x, J.y}, Jcv[2] = {Jc.x, Jc.y};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        if (P.w_terminal > 0.0f) {
            float xl[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) xl[c] = L::get(x[c], l);
            kahan_add(Jv[l], Jcv[l], terminal_cost(P, xl, v.xr + 12 * (P.H - 1)));
        }
        if (ADAPT && P.adaptive) kahan_add(Jv[l], Jcv[l], freq_regulariser(P, q[l]));
        if (!isfinite(Jv[l])) Jv[l] = kInf;
        if (valid[l]) {
            t.ws.J[k[l]] = Jv[l];
            t.ws.q[k[l]] = (int32_t)q[l];
        }
    }
    if (t.ws.hist) {
        // histograms of the top 16 and top 8 key bits for a large elite selection
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const uint32_t bin = cost_key(Jv[l]) >> 16;
            const unsigned act = __ballot_sync(kFull, valid[l]);
            if (valid[l]) {
                const unsigned peers = __match_any_sync(act, bin);
                if (lane == __ffs(peers) - 1) atomicAdd(t.ws.hist + bin, (unsigned)__popc(peers));
                const unsigned peers8 = __match_any_sync(act, bin >> 8);
                if (lane == __ffs(peers8) - 1) atomicAdd(t.ws.hist + kHistBins + (bin >> 8), (unsigned)__popc(peers8));
            }
        }
    }
    if (t.ws.best) {
        // Naive: the best finite (cost, index) of the one force block
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool fin = valid[l] && Jv[l] < kInf;
            unsigned long long m = fin ? ~(((unsigned long long)cost_key(Jv[l]) << 32) | k[l]) : 0ull;
            if (__any_sync(kFull, fin)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long xo = __shfl_xor_sync(kFull, m, o);
                    m = xo > m ? xo : m;
                }
                if (lane == 0) atomicMax(t.ws.best, m);
            }
            const unsigned nfw = __popc(__ballot_sync(kFull, fin));
            if (lane == 0 && nfw) atomicAdd(t.ws.nfin, nfw);
        }
    }
    if (!t.partials) return;

    // ---- MPPI partial sums of this tile, shifted by the tile's best cost
    bool fin[2];
    fin[0] = valid[0] && Jv[0] < kInf;
    fin[1] = valid[1] && Jv[1] < kInf;
    const float mt = block_min(sh, fminf(fin[0] ? Jv[0] : kInf, fin[1] ? Jv[1] : kInf));
    float w[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        w[l] = (fin[l] && mt < kInf) ? expf(-(Jv[l] - mt) * P.inv_lambda) : 0.0f;
        const float f = (float)q[l] / 1000.0f;
        const float s0 = warp_sum(w[l]), s1 = warp_sum(w[l] * w[l]), s2 = warp_sum(w[l] * f),
                    s3 = warp_sum(fin[l] ? 1.0f : 0.0f);
        if (lane == 0) {
            float* r = sh.red[l * nw2 + warp];
            r[0] = s0;
            r[1] = s1;
            r[2] = s2;
            r[3] = s3;
        }
    }
    const int PS = P.part_stride;
    float* row = t.ws.part + (size_t)tile * PS;
    {
        // the tile's samples of nonzero weight listed in sample order, then one
        // float4 column of the row per thread over a slice of the list (as in
        // rollout_tile)
        float2* lst = reinterpret_cast<float2*>(v.acc);
        unsigned nzb[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            nzb[l] = __ballot_sync(kFull, w[l] != 0.0f);
            if (lane == 0) sh.wtot[l * nw2 + warp] = __popc(nzb[l]);
        }
        __syncthreads();
        const int nw = 2 * nw2;
        int pos[2] = {0, 0}, nnz = 0;
        for (int g = 0; g < nw; ++g) {
            const int c = sh.wtot[g];
            pos[0] += g < warp ? c : 0;
            pos[1] += g < nw2 + warp ? c : 0;
            nnz += c;
        }
#pragma unroll
        for (int l = 0; l < 2; ++l)
            if (w[l] != 0.0f)
                lst[pos[l] + __popc(nzb[l] & ((1u << lane) - 1u))] = make_float2(w[l], __int_as_float(l * T2 + tid));
        __syncthreads();
        const int ncol = 3 * P.H;
        const int nsl = ncol < T ? T / ncol : 1;
        float4* slice_sum = reinterpret_cast<float4*>(v.acc + 2 * T);
        const float4* th4 = reinterpret_cast<const float4*>(theta) + (size_t)tile * T * 3;
        float4* row4 = reinterpret_cast<float4*>(row + kPartHeader);
        for (int it = tid; it < nsl * ncol; it += T2) {
            const int sl = it / ncol, c = it - sl * ncol, j = c / 3;
            const float4* src = th4 + (size_t)j * K * 3 + (c - 3 * j);
            const float4 sd4 = reinterpret_cast<const float4*>(v.sd + 12 * j)[c - 3 * j];
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ac = a;
            if (t.regen) {  // the listed samples' deviations regenerated from their draws
#pragma unroll 1
                for (int e = sl; e < nnz; e += nsl) {
                    const float2 we = lst[e];
                    const float4 d = regen_quad((uint32_t)(tile * T + __float_as_int(we.y)), j, c - 3 * j, t.iter,
                                                P.seed, P.ctrl, sd4);
                    kahan_wsum4(a, ac, we.x, d);
                }
            } else {
#pragma unroll 4
                for (int e = sl; e < nnz; e += nsl) {
                    const float2 we = lst[e];
                    const float4 d = src[3 * __float_as_int(we.y)];
                    kahan_wsum4(a, ac, we.x, d);
                }
            }
            if (nsl == 1) row4[c] = a;
            else slice_sum[it] = a;
        }
        if (nsl > 1) {
            __syncthreads();
            for (int c = tid; c < ncol; c += T2) {
                float4 a = slice_sum[c];
                for (int sl = 1; sl < nsl; ++sl) {
                    const float4 b = slice_sum[sl * ncol + c];
                    a.x += b.x;
                    a.y += b.y;
                    a.z += b.z;
                    a.w += b.w;
                }
                row4[c] = a;
            }
        }
    }
    if (tid == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int ww = 0; ww < 2 * nw2; ++ww) {
            a0 += sh.red[ww][0];
            a1 += sh.red[ww][1];
            a2 += sh.red[ww][2];
            a3 += sh.red[ww][3];
        }
        row[0] = mt;
        row[1] = a0;
        row[2] = a1;
        row[3] = a2;
        row[4] = a3;
    }
    if (t.partials == 1) tile_combine(sh, v, tile);
}

// The spline basis as duplicated pairs for the two-sample spline rollout, after
// the spline layout's per-warp sums (16-byte aligned): bs2 [H][4 ceil(P / 4)].
// The reference and the mean force trajectory stay single floats, broadcast to
// both lanes when read: duplicated, they would take the shared memory of a third
// block per SM (8 warps instead of 12; 0.436 against 0.421 ms per solve of the
// 262 144-sample spline workload).
__device__ __forceinline__ float2* pair_spline_rows(const Views& v, const InstParams& P, int T)
{
    return reinterpret_cast<float2*>(v.acc + (size_t)(T / 32) * P.nf);
}

// Float index of knot p, force component c of lane l (0: sample i, 1: sample
// i + T / 2) of thread i in the two-sample knot-deviation planes: plane
// (c ceil(NP / 4) + p / 4) 2 + (p mod 4) / 2 holds, per thread, the float4
// (A_p', B_p', A_p'+1, B_p'+1) with p' = p - p mod 2 (A, B: the thread's two
// samples), so that a 16-byte load gives two knots as lane pairs and a warp's
// loads are contiguous.
template <int NP>
__device__ __forceinline__ size_t pair_knot_index(int c, int p, int l, int T2, int tid)
{
    constexpr int NQ = (NP + 3) / 4;
    return ((((size_t)c * NQ + p / 4) * 2 + ((p & 3) >> 1)) * T2 + tid) * 4 + 2 * (p & 1) + l;
}

// ---------------------------------------------------------------------------
// One tile of T samples with two samples per thread and the spline policy of NP
// knots (ordinary model): the knot deviations of both samples are drawn once,
// as in rollout_tile<NP, false>, and kept in shared memory as lane pairs; each
// step evaluates both samples' forces from the basis with packed FMAs, and the
// stage cost and model step run on float2 lanes.  Every sample sees the
// operations of rollout_tile<NP, false> in the same order, and the tile's
// reductions run over virtual warps in the same order, so the results are
// bit-identical to the one-sample launch on the same tile.  Each step forms the
// attitude and the state part of the stage cost ahead of the force evaluation
// (1 % here; in the one-sample kernel the same change was 8 % slower).
// ---------------------------------------------------------------------------
template <int NP>
__device__ void rollout_tile_pair_spline(BlockShared& sh, float* dyn, int tile)
{
    using L = Lane<float2>;
    constexpr int NQ = (NP + 3) / 4;
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int T2 = blockDim.x, T = 2 * T2, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw2 = T2 >> 5;
    const Views v = carve(dyn, P.H, NP, P.nf, T, P.nb);
    float2* bs2 = pair_spline_rows(v, P, T);
    stage(sh, v, NP);
    for (int i = tid; i < 4 * NQ * P.H; i += T2) bs2[i] = make_float2(v.Bs[i], v.Bs[i]);
    fill_pair_consts(sh.pc, P, sh.fe);

    const int K = P.K;
    const uint32_t seed = P.seed, ctrl = P.ctrl;
    const uint64_t iter = t.iter;
    float* theta = t.ws.theta;
    uint32_t k[2], q[2];
    bool valid[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        k[l] = (uint32_t)tile * (uint32_t)T + (uint32_t)(l * T2 + tid);
        valid[l] = k[l] < (uint32_t)K;
        q[l] = P.adaptive ? sample_freq(k[l], iter, seed, ctrl, sh.mu_f, sh.sig_f, P.f_min, P.f_max) : P.q_init;
    }
    const float* sd = v.sd;
    // the knots' deviations sigma eps (stored for the update in store mode)
    float* dsf = reinterpret_cast<float*>(v.dsm);
#pragma unroll 1
    for (int p = 0; p < 4 * NQ; ++p) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            float e[12];
            if (p < NP) {
                normals12(k[l], p, iter, seed, ctrl, e);
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = __fmul_rn(sd[12 * p + c], e[c]);
                if (valid[l] && !t.regen) {
                    float4* o = reinterpret_cast<float4*>(theta + ((size_t)p * K + k[l]) * 12);
                    o[0] = make_float4(e[0], e[1], e[2], e[3]);
                    o[1] = make_float4(e[4], e[5], e[6], e[7]);
                    o[2] = make_float4(e[8], e[9], e[10], e[11]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) dsf[pair_knot_index<NP>(c, p, l, T2, tid)] = e[c];
        }
    }
    __syncthreads();
    const Consts<float2> Kc{sh.pc};

    float2 x[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) x[c] = L::bc(sh.x0[c]);
    const float2 fe[3] = {sh.pc.fe[0], sh.pc.fe[1], sh.pc.fe[2]};
    uint32_t ph[2], step[2];  // each sample's gait phase; the legs' phases add the block's offsets
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        ph[l] = t.phase0;
        step[l] = q[l] * P.dt_us;
    }
    const uint32_t duty = t.duty;
    const float4* dsm = v.dsm;

    float2 J = L::bc(0.0f), Jc = L::bc(0.0f);
    for (int j = 0; j < P.H; ++j) {
        const Attitude<float2> A = attitude_v<float2>(x);
        const float2 cost_x = stage_state_cost_bc(Kc, x, v.xr + 12 * j);
        // forces: the mean trajectory plus the basis-weighted knot deviations, in
        // knot order (packed FMAs over both samples)
        float2 G[12];
        {
            const float4* m4 = reinterpret_cast<const float4*>(v.Mb + 12 * j);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const float4 m = m4[cc];
                G[4 * cc] = L::bc(m.x);
                G[4 * cc + 1] = L::bc(m.y);
                G[4 * cc + 2] = L::bc(m.z);
                G[4 * cc + 3] = L::bc(m.w);
            }
            const float4* b4 = reinterpret_cast<const float4*>(bs2 + j * 4 * NQ);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                float2 g = G[c];
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) {
                    const float4 ba = b4[2 * qq], bb = b4[2 * qq + 1];
                    const float4 da = lds4(dsm + ((size_t)(c * NQ + qq) * 2) * T2 + tid);
                    const float4 db = lds4(dsm + ((size_t)(c * NQ + qq) * 2 + 1) * T2 + tid);
                    g = L::fma(make_float2(ba.x, ba.y), make_float2(da.x, da.y), g);
                    g = L::fma(make_float2(ba.z, ba.w), make_float2(da.z, da.w), g);
                    g = L::fma(make_float2(bb.x, bb.y), make_float2(db.x, db.y), g);
                    g = L::fma(make_float2(bb.z, bb.w), make_float2(db.z, db.w), g);
                }
                G[c] = g;
            }
        }
        // each sample's stance legs; a swing leg's force is zeroed on its lane (every
        // leg's terms are then summed, as in the one-sample spline kernel)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            unsigned st = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t pi = ph[l] + sh.t.offset[i];
                if (pi >= kPhaseOne) pi -= kPhaseOne;
                st |= (pi < duty ? 1u : 0u) << i;
            }
            ph[l] += step[l];
            if (ph[l] >= kPhaseOne) ph[l] -= kPhaseOne;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (!(st & (1u << i))) {
                    L::set(G[3 * i], l, 0.0f);
                    L::set(G[3 * i + 1], l, 0.0f);
                    L::set(G[3 * i + 2], l, 0.0f);
                }
        }
        kahan_add_v<float2>(J, Jc, stage_force_cost_v<float2>(Kc, cost_x, G, 0xfu, true));
        srbd_step_att_v<float2>(Kc, x, G, fe, 0xfu, A);
    }
    float Jv[2] = {J.x, J.y}, Jcv[2] = {Jc.x, Jc.y};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        if (P.w_terminal > 0.0f) {
            float xl[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) xl[c] = L::get(x[c], l);
            kahan_add(Jv[l], Jcv[l], terminal_cost(P, xl, v.xr + 12 * (P.H - 1)));
        }
        if (P.adaptive) kahan_add(Jv[l], Jcv[l], freq_regulariser(P, q[l]));
        if (!isfinite(Jv[l])) Jv[l] = kInf;
        if (valid[l]) {
            t.ws.J[k[l]] = Jv[l];
            t.ws.q[k[l]] = (int32_t)q[l];
        }
    }
    if (t.ws.hist) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const uint32_t bin = cost_key(Jv[l]) >> 16;
            const unsigned act = __ballot_sync(kFull, valid[l]);
            if (valid[l]) {
                const unsigned peers = __match_any_sync(act, bin);
                if (lane == __ffs(peers) - 1) atomicAdd(t.ws.hist + bin, (unsigned)__popc(peers));
                const unsigned peers8 = __match_any_sync(act, bin >> 8);
                if (lane == __ffs(peers8) - 1) atomicAdd(t.ws.hist + kHistBins + (bin >> 8), (unsigned)__popc(peers8));
            }
        }
    }
    if (t.ws.best) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool fin = valid[l] && Jv[l] < kInf;
            unsigned long long m = fin ? ~(((unsigned long long)cost_key(Jv[l]) << 32) | k[l]) : 0ull;
            if (__any_sync(kFull, fin)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long xo = __shfl_xor_sync(kFull, m, o);
                    m = xo > m ? xo : m;
                }
                if (lane == 0) atomicMax(t.ws.best, m);
            }
            const unsigned nfw = __popc(__ballot_sync(kFull, fin));
            if (lane == 0 && nfw) atomicAdd(t.ws.nfin, nfw);
        }
    }
    if (!t.partials) return;

    // ---- MPPI partial sums of this tile, shifted by the tile's best cost, over
    // virtual warps (lane 0 of warp w: virtual warp w; lane 1: nw2 + w)
    bool fin[2];
    fin[0] = valid[0] && Jv[0] < kInf;
    fin[1] = valid[1] && Jv[1] < kInf;
    const float mt = block_min(sh, fminf(fin[0] ? Jv[0] : kInf, fin[1] ? Jv[1] : kInf));
    float w[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        w[l] = (fin[l] && mt < kInf) ? expf(-(Jv[l] - mt) * P.inv_lambda) : 0.0f;
        const float f = (float)q[l] / 1000.0f;
        const float s0 = warp_sum(w[l]), s1 = warp_sum(w[l] * w[l]), s2 = warp_sum(w[l] * f),
                    s3 = warp_sum(fin[l] ? 1.0f : 0.0f);
        if (lane == 0) {
            float* r = sh.red[l * nw2 + warp];
            r[0] = s0;
            r[1] = s1;
            r[2] = s2;
            r[3] = s3;
        }
    }
    const int PS = P.part_stride;
    float* row = t.ws.part + (size_t)tile * PS;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        // a virtual warp whose weights all underflowed to zero contributes exact zeros
        float* acc = v.acc + (size_t)(l * nw2 + warp) * P.nf;
        if (!__any_sync(kFull, w[l] != 0.0f)) {
            for (int d = lane; d < P.nf; d += 32) acc[d] = 0.0f;
        } else {
#pragma unroll 1
            for (int p = 0; p < NP; ++p) {
                float vv[12], o[3];
#pragma unroll
                for (int c = 0; c < 12; ++c) vv[c] = __fmul_rn(w[l], dsf[pair_knot_index<NP>(c, p, l, T2, tid)]);
                const int c0 = warp_sum12(vv, o);
                if ((lane & 7) == 0) {
                    float* a = acc + 12 * p + c0;
                    a[0] = o[0];
                    a[1] = o[1];
                    a[2] = o[2];
                }
            }
        }
    }
    __syncthreads();
    for (int d = tid; d < P.nf; d += T2) {
        float s = 0.0f;
        for (int ww = 0; ww < 2 * nw2; ++ww) s += v.acc[ww * P.nf + d];
        row[kPartHeader + d] = s;
    }
    if (tid == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int ww = 0; ww < 2 * nw2; ++ww) {
            a0 += sh.red[ww][0];
            a1 += sh.red[ww][1];
            a2 += sh.red[ww][2];
            a3 += sh.red[ww][3];
        }
        row[0] = mt;
        row[1] = a0;
        row[2] = a1;
        row[3] = a2;
        row[4] = a3;
    }
    if (t.partials == 1) tile_combine(sh, v, tile);
}

// ---------------------------------------------------------------------------
// One tile of T samples on 2T threads (warp-specialised; the per-step policy;
// EXT as in rollout_tile), for controllers too small to fill the GPU, whose rollout
// is bound by each sample's chain of dependent instructions: thread s < T
// integrates sample s, thread T + s draws that sample's 12 normals one step
// ahead into a double buffer in shared memory, so the Philox and Box-Muller
// work runs on other warps than the model step.  The two halves meet at one
// named barrier per step, which every thread passes H + 1 times.  The consumer
// does the operations of rollout_tile<0, EXT> in the same order, and in the
// tile's reductions the producers count as samples past K (weight zero, cost
// +inf), which adds only zero terms: the results are bit-identical to the
// one-sample launch on the same tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ws_barrier(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// The double buffer of normals after the per-step layout: [2][12][T] floats.
__device__ __forceinline__ float* ws_ring(float* dyn, const InstParams& P, int T)
{
    return dyn + rollout_smem_bytes(P.H, 0, T, P.nb) / sizeof(float);
}

template <bool EXT>
__device__ void rollout_tile_ws(BlockShared& sh, float* dyn, int tile)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int NT = blockDim.x, T = NT >> 1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
    const bool producer = tid >= T;
    const int s = producer ? tid - T : tid;  // the sample's place in the tile
    const Views v = carve(dyn, P.H, 0, P.nf, T, P.nb);
    float* ring = ws_ring(dyn, P, T);
    stage(sh, v, 0);

    const int K = P.K;
    const uint32_t k = (uint32_t)tile * (uint32_t)T + (uint32_t)s;
    const bool valid = !producer && k < (uint32_t)K;  // a producer carries no sample of its own
    const uint32_t seed = P.seed, ctrl = P.ctrl;
    const uint64_t iter = t.iter;
    float* theta = t.ws.theta;
    uint32_t q = P.q_init;
    int blk = 0;  // force block: the sample's entry of a discrete frequency set
    if (P.adaptive) {
        q = sample_freq(k, iter, seed, ctrl, sh.mu_f, sh.sig_f, P.f_min, P.f_max);
    } else if constexpr (EXT) {
        if (P.n_freq > 0) {
            blk = freq_block(k, iter, seed, ctrl, P.n_freq);
            q = P.freq[blk];
        }
    }

    float J = kInf, Jc = 0.0f;
    float x[12];
    if (producer) {
        const PhiloxPre pp = philox_pre(k, iter, seed, ctrl);
        float e[12];
        normals12(pp, 0, e);
#pragma unroll
        for (int c = 0; c < 12; ++c) ring[c * T + s] = e[c];
        ws_barrier(NT);
        for (int j = 0; j < P.H; ++j) {
            if (j + 1 < P.H) {
                normals12(pp, j + 1, e);
                float* r = ring + ((j + 1) & 1) * 12 * T;
#pragma unroll
                for (int c = 0; c < 12; ++c) r[c * T + s] = e[c];
            }
            ws_barrier(NT);
        }
    } else {
        const float* mu = v.mu + blk * P.nf;  // this sample's Gaussian
        const float* sd = v.sd + blk * P.nf;
#pragma unroll
        for (int c = 0; c < 12; ++c) x[c] = sh.x0[c];
        const float fe[3] = {sh.fe[0], sh.fe[1], sh.fe[2]};
        uint32_t ph[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t p0 = t.phase0 + t.offset[i];
            ph[i] = p0 >= kPhaseOne ? p0 - kPhaseOne : p0;
        }
        const uint32_t step = q * P.dt_us;
        const bool uniform_q = !P.adaptive && P.n_freq == 0;
        const uint32_t duty = t.duty;
        // world-fixed feet: ground positions, last step's stance flags, T_st / 2
        float fx[4], fy[4];
        unsigned prev = 0xfu;  // legs in stance at t_0 keep the given feet
        float tsh = 0.0f;
        if constexpr (EXT) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fx[i] = sh.feet[2 * i];
                fy[i] = sh.feet[2 * i + 1];
            }
            tsh = (0.5e-6f * (float)duty) / (float)q;
        }
        J = 0.0f;
        ws_barrier(NT);  // step 0's normals
        for (int j = 0; j < P.H; ++j) {
            const float* r = ring + (j & 1) * 12 * T;
            float e[12], G[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) e[c] = r[c * T + s];
            const float4* m4 = reinterpret_cast<const float4*>(mu + 12 * j);
            const float4* s4 = reinterpret_cast<const float4*>(sd + 12 * j);
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
                const float4 ma = m4[qq], sa = s4[qq];
                const float mv[4] = {ma.x, ma.y, ma.z, ma.w}, sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) G[4 * qq + i] = __fmaf_rn(sv[i], e[4 * qq + i], mv[i]);
            }
            if (!t.regen) {
#pragma unroll
                for (int qq = 0; qq < 3; ++qq) {
                    const float4 sa = s4[qq];
                    const float sv[4] = {sa.x, sa.y, sa.z, sa.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) e[4 * qq + i] = __fmul_rn(sv[i], e[4 * qq + i]);
                }
                if (valid) {
                    float4* o = reinterpret_cast<float4*>(theta + ((size_t)j * K + k) * 12);
                    o[0] = make_float4(e[0], e[1], e[2], e[3]);
                    o[1] = make_float4(e[4], e[5], e[6], e[7]);
                    o[2] = make_float4(e[8], e[9], e[10], e[11]);
                }
            }
            unsigned st, live, all;
            if (uniform_q) {
                st = live = all = sh.sched[j];
            } else {
                st = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) st |= (ph[i] < duty ? 1u : 0u) << i;
                live = __reduce_or_sync(kFull, st);
                all = __reduce_and_sync(kFull, st);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ph[i] += step;
                    if (ph[i] >= kPhaseOne) ph[i] -= kPhaseOne;
                }
            }
            if (live != all) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (!(st & (1u << i))) G[3 * i] = G[3 * i + 1] = G[3 * i + 2] = 0.0f;
            }
            bool penalty = true;
            if constexpr (EXT) {
                if (P.friction_project) {  // the policy output constrained to the cone (Sec. IV-B)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        cone_project(P.mu, P.inv_1pmu2, G[3 * i], G[3 * i + 1], G[3 * i + 2]);
                    penalty = false;
                }
            }
            kahan_add(J, Jc, stage_cost(P, x, v.xr + 12 * j, G, live, penalty));
            if constexpr (EXT) {
                if (P.world_feet) {
                    const unsigned touch = st & ~prev;  // legs landing at this step
                    prev = st;
                    srbd_step_world(P, x, G, fe, live, fx, fy, touch, v.xr[12 * j + 6], v.xr[12 * j + 7], tsh);
                } else {
                    srbd_step(P, x, G, fe, live);
                }
            } else {
                srbd_step(P, x, G, fe, live);
            }
            ws_barrier(NT);
        }
        if (P.w_terminal > 0.0f) kahan_add(J, Jc, terminal_cost(P, x, v.xr + 12 * (P.H - 1)));
        if (P.adaptive || P.n_freq > 0) kahan_add(J, Jc, freq_regulariser(P, q));
        if (!isfinite(J)) J = kInf;
        if (valid) {
            t.ws.J[k] = J;
            t.ws.q[k] = (int32_t)q;
        }
    }
    if (t.ws.hist) {
        // histograms of the top 16 and top 8 key bits for a large elite selection
        const uint32_t bin = cost_key(J) >> 16;
        const unsigned act = __ballot_sync(kFull, valid);
        if (valid) {
            const unsigned peers = __match_any_sync(act, bin);
            if (lane == __ffs(peers) - 1) atomicAdd(t.ws.hist + bin, (unsigned)__popc(peers));
            const unsigned peers8 = __match_any_sync(act, bin >> 8);
            if (lane == __ffs(peers8) - 1) atomicAdd(t.ws.hist + kHistBins + (bin >> 8), (unsigned)__popc(peers8));
        }
    }
    if (t.ws.best) {
        // Naive: each force block's best finite (cost, index), kept as the maximum of
        // the complemented 64-bit key; one atomic per warp and block present
        const bool fin = valid && J < kInf;
        const unsigned long long key = fin ? ~(((unsigned long long)cost_key(J) << 32) | k) : 0ull;
        unsigned todo = __reduce_or_sync(kFull, fin ? 1u << blk : 0u);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            unsigned long long m = blk == b ? key : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long xo = __shfl_xor_sync(kFull, m, o);
                m = xo > m ? xo : m;
            }
            if (lane == 0) atomicMax(t.ws.best + b, m);
        }
        const unsigned nfw = __popc(__ballot_sync(kFull, fin));
        if (lane == 0 && nfw) atomicAdd(t.ws.nfin, nfw);
    }
    if (!t.partials) return;

    // ---- MPPI partial sums of this tile, shifted by the tile's best cost (the
    // producers' warps add zero rows to the warp sums, after the consumers')
    const bool fin = valid && J < kInf;
    const float mt = block_min(sh, fin ? J : kInf);
    const float w = (fin && mt < kInf) ? expf(-(J - mt) * P.inv_lambda) : 0.0f;
    const float f = (float)q / 1000.0f;
    {
        const float s0 = warp_sum(w), s1 = warp_sum(w * w), s2 = warp_sum(w * f), s3 = warp_sum(fin ? 1.0f : 0.0f);
        if (lane == 0) {
            sh.red[warp][0] = s0;
            sh.red[warp][1] = s1;
            sh.red[warp][2] = s2;
            sh.red[warp][3] = s3;
        }
    }
    const int PS = P.part_stride;
    float* row = t.ws.part + (size_t)tile * PS;
    {
        // the samples of nonzero weight listed in sample order; the consumers then
        // sum one float4 column of the row each over a slice of the list (as in
        // rollout_tile, with the tile's T samples)
        float2* lst = reinterpret_cast<float2*>(v.acc);
        const unsigned nzb = __ballot_sync(kFull, w != 0.0f);
        if (lane == 0) sh.wtot[warp] = __popc(nzb);
        __syncthreads();
        int pos = 0, nnz = 0;
        for (int g = 0; g < nw; ++g) {
            const int c = sh.wtot[g];
            pos += g < warp ? c : 0;
            nnz += c;
        }
        if (w != 0.0f) lst[pos + __popc(nzb & ((1u << lane) - 1u))] = make_float2(w, __int_as_float(s));
        __syncthreads();
        const int ncol = 3 * P.H;
        const int nsl = ncol < T ? T / ncol : 1;
        float4* slice_sum = reinterpret_cast<float4*>(v.acc + 2 * T);  // [nsl][ncol] when nsl > 1
        const float4* th4 = reinterpret_cast<const float4*>(theta) + (size_t)tile * T * 3;
        float4* row4 = reinterpret_cast<float4*>(row + kPartHeader);
        if (!producer) {
            for (int it = tid; it < nsl * ncol; it += T) {
                const int sl = it / ncol, c = it - sl * ncol, j = c / 3;
                const float4* src = th4 + (size_t)j * K * 3 + (c - 3 * j);
                const float4 sd4 = reinterpret_cast<const float4*>(v.sd + 12 * j)[c - 3 * j];
                float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ac = a;
                if (t.regen) {  // the listed samples' deviations regenerated from their draws
#pragma unroll 1
                    for (int e = sl; e < nnz; e += nsl) {
                        const float2 we = lst[e];
                        const float4 d = regen_quad((uint32_t)(tile * T + __float_as_int(we.y)), j, c - 3 * j,
                                                    t.iter, P.seed, P.ctrl, sd4);
                        kahan_wsum4(a, ac, we.x, d);
                    }
                } else {
#pragma unroll 4
                    for (int e = sl; e < nnz; e += nsl) {
                        const float2 we = lst[e];
                        const float4 d = src[3 * __float_as_int(we.y)];
                        kahan_wsum4(a, ac, we.x, d);
                    }
                }
                if (nsl == 1) row4[c] = a;
                else slice_sum[it] = a;
            }
        }
        if (nsl > 1) {
            __syncthreads();
            if (!producer) {
                for (int c = tid; c < ncol; c += T) {
                    float4 a = slice_sum[c];
                    for (int sl = 1; sl < nsl; ++sl) {
                        const float4 b = slice_sum[sl * ncol + c];
                        a.x += b.x;
                        a.y += b.y;
                        a.z += b.z;
                        a.w += b.w;
                    }
                    row4[c] = a;
                }
            }
        }
    }
    if (tid == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int ww = 0; ww < nw; ++ww) {
            a0 += sh.red[ww][0];
            a1 += sh.red[ww][1];
            a2 += sh.red[ww][2];
            a3 += sh.red[ww][3];
        }
        row[0] = mt;
        row[1] = a0;
        row[2] = a1;
        row[3] = a2;
        row[4] = a3;
    }
    if (t.partials == 1) tile_combine(sh, v, tile);
}

// Cost of an order-preserving key (inverse of cost_key).
__device__ __forceinline__ float key_cost(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------------------
// Naive selection (Alg. 3 Sorting) per force block: the rollout left each
// block's best (cost, index) as a complemented key.  Warp 0 reads and clears
// them, lists each block's winner (-1: no finite cost) followed by the block of
// the overall best, and writes the result record.
// ---------------------------------------------------------------------------
__device__ void naive_select(BlockShared& sh)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x;
    if (tid >= 32) return;
    unsigned long long key = ~0ull;  // no finite sample
    if (tid < P.nb) {
        const unsigned long long c = __ldcg(t.ws.best + tid);
        t.ws.best[tid] = 0ull;
        key = ~c;
        t.ws.elite[tid] = c ? (int32_t)(uint32_t)key : -1;
    }
    unsigned long long m = key;
    int b = tid;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long om = __shfl_xor_sync(kFull, m, o);
        const int ob = __shfl_xor_sync(kFull, b, o);
        if (om < m || (om == m && ob < b)) {
            m = om;
            b = ob;
        }
    }
    if (tid == 0) {
        const bool any = m != ~0ull;
        t.ws.elite[P.nb] = any ? b : 0;
        const unsigned nfin = __ldcg(t.ws.nfin);
        *t.ws.nfin = 0u;
        sbs_result* r = t.result;
        r->cost_min = any ? key_cost((uint32_t)(m >> 32)) : kInf;
        r->ess = 1.0f;
        r->status = any ? SBS_OK : SBS_ERR_DIVERGED;
        r->n_finite = (int32_t)nfin;
        r->iter_lo = (uint32_t)t.iter;
        r->iter_hi = (uint32_t)(t.iter >> 32);
    }
}

// ---------------------------------------------------------------------------
// Elite selection (Alg. 1 Sorting) by one block: the Ke smallest (cost, index)
// pairs, listed by ascending index.  A radix select on the order-preserving cost
// key gives the threshold key thr (the Ke-th smallest) and need_eq, the number of
// keys equal to thr that belong to the elite (ties go to the lowest indices); an
// ordered compaction then lists the elite.
//  * K <= kSelectSmemMaxK: the keys are staged in shared memory; four 8-bit passes.
//  * larger K: the rollout built histograms of the top 8 and top 16 key bits.
//    They give the 16-bit bin holding rank Ke; that bin's keys are gathered into
//    shared memory and two 8-bit passes finish there (two passes over all keys
//    in global memory if the bin holds more keys than fit).
// ---------------------------------------------------------------------------

// The four staged keys i0 .. i0 + 3 from shared memory (the largest key at and
// past end); i0 a multiple of 4.
__device__ __forceinline__ void load4k(const uint32_t* k, int i0, int end, uint32_t c[4])
{
    if (i0 + 4 <= end) {
        const uint4 q = *reinterpret_cast<const uint4*>(k + i0);
        c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = i0 + u < end ? k[i0 + u] : 0xffffffffu;
    }
}

// The four costs of keys i0 .. i0 + 3 (+inf at and past end); i0 a multiple of 4.
__device__ __forceinline__ void load4(const float* J, int i0, int end, float c[4])
{
    if (i0 + 4 <= end) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(J + i0));
        c[0] = q.x; c[1] = q.y; c[2] = q.z; c[3] = q.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = i0 + u < end ? __ldcg(J + i0 + u) : kInf;
    }
}

// The digit of the 256-bin histogram in shared memory holding rank (1-based):
// sets sh.digit and sh.below (keys in lower digits).  Warp 0, 8 bins per lane.
__device__ __forceinline__ void find_digit(BlockShared& sh, const int* hist, int rank)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    int local = 0;
    for (int b = 0; b < 8; ++b) local += hist[8 * lane + b];
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += u;
    }
    const int excl = incl - local;
    const unsigned hit = __ballot_sync(kFull, excl < rank && rank <= incl);
    if (lane == __ffs(hit) - 1) {
        int c = excl;
        for (int b = 0; b < 8; ++b) {
            const int h = hist[8 * lane + b];
            if (c + h >= rank) {
                sh.digit = 8 * lane + b;
                sh.below = c;
                break;
            }
            c += h;
        }
    }
}

// One 8-bit radix pass over n keys: the histogram of digit (key >> shift) & 255
// among keys matching prefix under mask, then the digit holding rank; narrows
// prefix, mask and rank.  SMEM: keys in shared memory; else costs in global memory.
template <bool SMEM>
__device__ void radix_pass(BlockShared& sh, const uint32_t* skeys, const float* J, int n, int shift,
                           uint32_t& prefix, uint32_t& mask, int& rank)
{
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < 256; i += T) sh.hist[i] = 0;
    __syncthreads();
    if constexpr (SMEM) {
        for (int i = tid; i < n; i += T) {
            const uint32_t key = skeys[i];
            if ((key & mask) == prefix) atomicAdd(&sh.hist[(key >> shift) & 255u], 1);
        }
    } else {
        constexpr int KPT = 16;  // keys per thread per iteration
        for (int base = 0; base < n; base += KPT * T) {
            uint32_t keys[KPT];
            bool ok[KPT];
            if (base + KPT * T <= n) {
                // 16-byte loads: thread tid covers keys base + 4 (tid + T u') + 0..3
                const float4* J4 = reinterpret_cast<const float4*>(J + base);
#pragma unroll
                for (int u = 0; u < KPT / 4; ++u) {
                    const float4 v = __ldcg(J4 + tid + u * T);
                    keys[4 * u] = cost_key(v.x);
                    keys[4 * u + 1] = cost_key(v.y);
                    keys[4 * u + 2] = cost_key(v.z);
                    keys[4 * u + 3] = cost_key(v.w);
                }
#pragma unroll
                for (int u = 0; u < KPT; ++u) ok[u] = true;
            } else {
#pragma unroll
                for (int u = 0; u < KPT; ++u) {
                    const int i = base + u * T + tid;
                    ok[u] = i < n;
                    keys[u] = ok[u] ? cost_key(__ldcg(J + i)) : 0u;
                }
            }
#pragma unroll
            for (int u = 0; u < KPT; ++u)
                if (ok[u] && (keys[u] & mask) == prefix) atomicAdd(&sh.hist[(keys[u] >> shift) & 255u], 1);
        }
    }
    __syncthreads();
    find_digit(sh, sh.hist, rank);
    __syncthreads();
    rank -= sh.below;
    prefix |= (uint32_t)sh.digit << shift;
    mask |= 255u << shift;
    __syncthreads();
}

// Threshold key and tie count for K > kSelectSmemMaxK from the rollout's
// histograms (which it clears for the next solve); cand: shared-memory space for
// kSelectSmemMaxK keys.
// The 16-bit key bin holding rank Ke, from the rollout's histograms: the bin, the
// rank within it and its key count.  clear: also clear the histograms for the
// next solve (else the caller's next kernel does).
__device__ void find_bin16(BlockShared& sh, uint32_t& b16_out, int& rank_out, int& ncand_out, bool clear = true)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, T = blockDim.x;
    unsigned* hist16 = t.ws.hist;
    unsigned* hist8 = hist16 + kHistBins;
    int rank = P.Ke;
    // the top-8-bit bin holding rank Ke, then its 16-bit sub-bin
    for (int i = tid; i < 256; i += T) sh.hist[i] = (int)__ldcg(hist8 + i);
    __syncthreads();
    find_digit(sh, sh.hist, rank);
    __syncthreads();
    const int b8 = sh.digit;
    rank -= sh.below;
    __syncthreads();
    const int v = tid < 256 ? (int)__ldcg(hist16 + b8 * 256 + tid) : 0;
    int tot;
    const int excl = block_scan(sh, v, &tot);
    if (tid < 256 && excl < rank && rank <= excl + v) {
        sh.digit = b8 * 256 + tid;
        sh.below = excl;
        sh.count = v;
    }
    __syncthreads();
    const uint32_t b16 = (uint32_t)sh.digit;
    rank -= sh.below;
    const int ncand = sh.count;
    __syncthreads();
    if (clear) {
        for (int i = tid; i < 256; i += T) hist8[i] = 0u;
        for (int i = tid; i < kHistBins; i += T) hist16[i] = 0u;
    }
    b16_out = b16;
    rank_out = rank;
    ncand_out = ncand;
}

__device__ void large_threshold(BlockShared& sh, uint32_t* cand, uint32_t& thr, int& need_eq)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x;
    const int K = P.K;
    const float* J = t.ws.J;
    uint32_t b16;
    int rank, ncand;
    find_bin16(sh, b16, rank, ncand);
    uint32_t prefix = b16 << 16, mask = 0xffff0000u;
    if (ncand > kSelectSmemMaxK) {  // the bin does not fit: finish over all keys
        radix_pass<false>(sh, nullptr, J, K, 8, prefix, mask, rank);
        radix_pass<false>(sh, nullptr, J, K, 0, prefix, mask, rank);
        thr = prefix;
        need_eq = rank;
        return;
    }
    // gather the low 16 bits of the bin's keys (order does not matter for the
    // threshold; the compaction takes ties by index)
    if (tid == 0) sh.count = 0;
    __syncthreads();
    constexpr int R = 4;  // 16-byte loads in flight per thread
    for (int base = 0; base < K; base += 4 * R * T) {
        float c[4 * R];
#pragma unroll
        for (int r = 0; r < R; ++r) load4(J, base + 4 * (tid + r * T), K, c + 4 * r);
#pragma unroll
        for (int u = 0; u < 4 * R; ++u) {
            const int i = base + 4 * (tid + (u / 4) * T) + (u & 3);
            const uint32_t key = cost_key(c[u]);
            const bool m = i < K && (key >> 16) == b16;
            const unsigned bal = __ballot_sync(kFull, m);
            if (bal) {
                int at = 0;
                if (lane == __ffs(bal) - 1) at = atomicAdd(&sh.count, __popc(bal));
                at = __shfl_sync(kFull, at, __ffs(bal) - 1);
                const int pos = at + __popc(bal & ((1u << lane) - 1u));
                if (m && pos < kSelectSmemMaxK) cand[pos] = key & 0xffffu;
            }
        }
    }
    __syncthreads();
    const int n = min(sh.count, kSelectSmemMaxK);
    uint32_t p2 = 0, m2 = 0;
    radix_pass<true>(sh, cand, nullptr, n, 8, p2, m2, rank);
    radix_pass<true>(sh, cand, nullptr, n, 0, p2, m2, rank);
    thr = (b16 << 16) | p2;
    need_eq = rank;
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_excl_scan(int v, int* total)
{
    const int lane = threadIdx.x & 31;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += u;
    }
    *total = __shfl_sync(kFull, incl, 31);
    return incl - v;
}

// List the keys of [begin, end) below thr and the first need_eq keys equal to
// thr, by ascending index, into out from position out0 on (never past Ke).
// begin is a multiple of 4.  Warp w owns a contiguous sub-range (a multiple of
// 128 long, read as 16-byte loads); a first pass counts, the warps' offsets
// follow from one scan over the warps' counts, a second pass writes.  Each
// thread also returns its part of the best cost and of the number of finite
// costs.  R: rounds of 128 keys per warp whose loads are in flight together
// (more only pays when every warp has that many rounds).  KEYS: the keys come
// from skeys, staged in shared memory, instead of the costs in global memory;
// the best cost and finite count are then the caller's (from its staging pass).
template <int R, bool KEYS = false>
__device__ void compact_range(BlockShared& sh, uint32_t thr, int need_eq, int begin, int end, int out0,
                              float* bmin_out, int* nf_out, const uint32_t* skeys = nullptr)
{
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int Ke = sh.P.Ke;
    const float* J = t.ws.J;
    int32_t* out = t.ws.elite;
    const int n = end - begin;
    const int Cw = ((n + nw - 1) / nw + 127) / 128 * 128;
    const int c0 = min(end, begin + warp * Cw), c1 = min(end, c0 + Cw);
    int lt = 0, eq = 0, nf = 0;
    float bmin = kInf;
    for (int base = c0; base < c1; base += 128 * R) {
        float c[4 * R];
        uint32_t kk[4 * R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (KEYS) load4k(skeys, base + 128 * r + 4 * lane, c1, kk + 4 * r);
            else load4(J, base + 128 * r + 4 * lane, c1, c + 4 * r);
        }
#pragma unroll
        for (int u = 0; u < 4 * R; ++u) {
            if (base + 128 * (u / 4) + 4 * lane + (u & 3) < c1) {
                uint32_t key;
                if constexpr (KEYS) key = kk[u];
                else key = cost_key(c[u]);
                lt += key < thr ? 1 : 0;
                eq += key == thr ? 1 : 0;
                if constexpr (!KEYS) {
                    bmin = fminf(bmin, c[u]);
                    nf += c[u] < kInf ? 1 : 0;
                }
            }
        }
    }
    lt = warp_sum_int(lt);
    eq = warp_sum_int(eq);
    if (lane == 0) {
        sh.wtot[warp] = lt;
        sh.wtot2[warp] = eq;
    }
    __syncthreads();
    // this warp's offset: the keys below thr in the warps before it, plus the ties
    // those warps take (ties go to the lowest indices, so they take min(need_eq,
    // their ties)); both counts are prefix sums over the warps, one scan per warp
    const int lt_w = lane < nw ? sh.wtot[lane] : 0, eq_w = lane < nw ? sh.wtot2[lane] : 0;
    int lt_in = lt_w, eq_in = eq_w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(kFull, lt_in, o), b = __shfl_up_sync(kFull, eq_in, o);
        if (lane >= o) {
            lt_in += a;
            eq_in += b;
        }
    }
    const int eqb = __shfl_sync(kFull, eq_in - eq_w, warp);  // ties in the warps before this one
    int off = out0 + __shfl_sync(kFull, lt_in - lt_w, warp) + max(0, min(need_eq, eqb));
    const int take_eq = min(eq, max(0, need_eq - eqb));  // this warp's ties, in index order
    int eq_seen = 0;
    for (int base0 = c0; base0 < c1; base0 += 128 * R) {
        float cr[4 * R];
        uint32_t kr[4 * R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (KEYS) load4k(skeys, base0 + 128 * r + 4 * lane, c1, kr + 4 * r);
            else load4(J, base0 + 128 * r + 4 * lane, c1, cr + 4 * r);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i0 = base0 + 128 * r + 4 * lane;
            const float* c = cr + 4 * r;
            bool is_lt[4], is_eq[4];
            int ne = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                uint32_t key;
                if constexpr (KEYS) key = kr[4 * r + u];
                else key = cost_key(c[u]);
                is_lt[u] = i0 + u < c1 && key < thr;
                is_eq[u] = i0 + u < c1 && key == thr;
                ne += is_eq[u] ? 1 : 0;
            }
            int ne_tot;
            int er = eq_seen + warp_excl_scan(ne, &ne_tot);  // ties before this lane's keys
            bool take[4];
            int nt = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                take[u] = is_lt[u] || (is_eq[u] && er < take_eq);
                er += is_eq[u] ? 1 : 0;
                nt += take[u] ? 1 : 0;
            }
            int nt_tot;
            int pos = off + warp_excl_scan(nt, &nt_tot);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (take[u]) {
                    if (pos < Ke) out[pos] = i0 + u;  // never past the Ke-sized output
                    ++pos;
                }
            }
            off += nt_tot;
            eq_seen += ne_tot;
        }
    }
    *bmin_out = bmin;
    *nf_out = nf;
}

__device__ void select_block(BlockShared& sh, uint32_t* skeys)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    if (P.method == SBS_NAIVE) {
        naive_select(sh);
        return;
    }
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const int K = P.K;
    const float* J = t.ws.J;
    const bool staged = K <= kSelectSmemMaxK;
    uint32_t thr;
    int need_eq;
    if (staged) {
        // staging fused with the first pass's histogram (top 8 key bits), the best
        // key and the finite count (per warp, combined when the record is written)
        for (int i = tid; i < 256; i += T) sh.hist[i] = 0;
        __syncthreads();
        const uint32_t kinf = cost_key(kInf);
        uint32_t kmin = 0xffffffffu;
        int nfk = 0;
        for (int i = tid; i < K; i += T) {
            const uint32_t key = cost_key(__ldcg(J + i));
            skeys[i] = key;
            atomicAdd(&sh.hist[key >> 24], 1);
            kmin = min(kmin, key);
            nfk += key < kinf ? 1 : 0;
        }
        kmin = __reduce_min_sync(kFull, kmin);
        nfk = __reduce_add_sync(kFull, (unsigned)nfk);
        if (lane == 0) {
            sh.selkmin[warp] = kmin;
            sh.selnf[warp] = nfk;
        }
        __syncthreads();
        int rank = P.Ke;
        find_digit(sh, sh.hist, rank);
        __syncthreads();
        rank -= sh.below;
        uint32_t prefix = (uint32_t)sh.digit << 24, mask = 255u << 24;
        __syncthreads();
        for (int pass = 1; pass < 4; ++pass) radix_pass<true>(sh, skeys, nullptr, K, 24 - 8 * pass, prefix, mask, rank);
        thr = prefix;
        need_eq = rank;
    } else if (t.ws.hist) {
        large_threshold(sh, skeys, thr, need_eq);
    } else {  // larger K always comes with the histograms; kept for completeness
        uint32_t prefix = 0, mask = 0;
        int rank = P.Ke;
        for (int pass = 0; pass < 4; ++pass) radix_pass<false>(sh, nullptr, J, K, 24 - 8 * pass, prefix, mask, rank);
        thr = prefix;
        need_eq = rank;
    }
    float bm, beta;
    int nf, nfin;
    if (staged) {  // the list from the staged keys; best cost and finite count from the staging pass
        if (K >= 16384) compact_range<4, true>(sh, thr, need_eq, 0, K, 0, &bm, &nf, skeys);
        else compact_range<1, true>(sh, thr, need_eq, 0, K, 0, &bm, &nf, skeys);
        // warp 0 combines the staging pass's per-warp best keys and finite counts
        // (thread 0 writes the record)
        uint32_t kmin = 0xffffffffu;
        nfin = 0;
        if (warp == 0) {
            kmin = __reduce_min_sync(kFull, lane < nw ? sh.selkmin[lane] : 0xffffffffu);
            nfin = (int)__reduce_add_sync(kFull, lane < nw ? (unsigned)sh.selnf[lane] : 0u);
        }
        beta = key_cost(kmin);
    } else {
        if (K >= 16384) compact_range<4>(sh, thr, need_eq, 0, K, 0, &bm, &nf);
        else compact_range<1>(sh, thr, need_eq, 0, K, 0, &bm, &nf);
        beta = block_min(sh, bm);
        block_scan(sh, nf, &nfin);
    }
    if (tid == 0) {
        sbs_result* r = t.result;
        r->cost_min = beta;
        r->ess = (float)P.Ke;
        r->status = nfin > 0 ? SBS_OK : SBS_ERR_DIVERGED;
        r->n_finite = nfin;
        r->iter_lo = (uint32_t)t.iter;
        r->iter_hi = (uint32_t)(t.iter >> 32);
    }
}

// ---------------------------------------------------------------------------
// Naive refit (Alg. 3) of step (or knot) j in every force block: the block's
// winner becomes its mean (shifted mean + the winner's stored deviation), the
// variance is kept; a block without a finite-cost sample keeps its mean.  u0
// and the reported frequency come from the block of the overall best (the first
// block when no cost is finite).
// ---------------------------------------------------------------------------
template <bool REGEN>
__device__ void naive_refit(BlockShared& sh, int j)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const float* sm = P.state[t.src];
    const float* sv = sm + P.D;
    float* dm = P.state[1 - t.src];
    float* dv = dm + P.D;
    sbs_result* r = t.result;
    const bool diverged = __ldcg(&r->status) != SBS_OK;
    const int bstar = diverged ? 0 : __ldcg(t.ws.elite + P.nb);
    for (int i = threadIdx.x; i < 12 * P.nb; i += blockDim.x) {
        const int blk = i / 12, c = i - 12 * blk;
        const int idx = blk * P.nf + 12 * j + c;
        float m, var;
        shifted_entry(P, t, sm, sv, idx, m, var);
        const int kb = diverged ? -1 : __ldcg(t.ws.elite + blk);
        if (kb >= 0) {
            float d;
            if (REGEN) {  // the winner's deviation, regenerated (its block's standard deviation)
                float e[12];
                normals12((uint32_t)kb, j, t.iter, P.seed, P.ctrl, e);
                float ec = e[0];
#pragma unroll
                for (int i = 1; i < 12; ++i) ec = i == c ? e[i] : ec;  // no local-memory indexing
                d = __fmul_rn(sqrtf(var), ec);
            } else {
                d = __ldcg(t.ws.theta + ((size_t)j * P.K + kb) * 12 + c);
            }
            m += d;
        }
        dm[idx] = m;
        dv[idx] = var;
        if (j == 0 && blk == bstar) {
            const uint32_t ph = (t.phase0 + t.offset[c / 3]) % kPhaseOne;
            r->u0[c] = ph < t.duty ? m : 0.0f;
        }
    }
    if (j == 0 && threadIdx.x == 0 && !P.adaptive) {
        const uint32_t q = P.n_freq > 0 ? P.freq[bstar] : P.q_init;
        r->f_mean = q * 0.001f;
        r->q_freq = (int32_t)q;
    }
}

// ---------------------------------------------------------------------------
// Elite / Naive refit of one step (or knot) b, or of the frequency (b == nt).
// With d = theta - mu the stored deviations of the elites: mean = mu + mean(d),
// var = mean((d - mean(d))^2) floored (Alg. 1 Update, two passes); Naive
// (Alg. 3): the best sample, variance kept.
// ---------------------------------------------------------------------------
template <bool REGEN>
__device__ void refit_block(BlockShared& sh, int b)
{
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, lane = tid & 31;
    const float* sm = P.state[t.src];
    const float* sv = sm + P.D;
    float* dm = P.state[1 - t.src];
    float* dv = dm + P.D;
    const int K = P.K;
    const int Ke = P.method == SBS_NAIVE ? 1 : P.Ke;
    const int V = refit_lanes(Ke);  // virtual lanes: the order of the sums
    const int32_t* elite = t.ws.elite;
    sbs_result* r = t.result;
    const bool diverged = __ldcg(&r->status) != SBS_OK;
    if (b < P.nt && P.method == SBS_NAIVE) {
        naive_refit<REGEN>(sh, b);
        return;
    }
    if (b < P.nt) {
        // the thread's first elite index (virtual lane tid of the first pass), loaded
        // alongside the distribution entries
        const int kfirst = tid < Ke ? __ldcg(elite + tid) : 0;
        if (tid < 12) {
            float m, var;
            shifted_entry(P, t, sm, sv, 12 * b + tid, m, var);
            sh.mu12[tid] = m;
            sh.vr12[tid] = var;
            if (REGEN) sh.sd12[tid] = sqrtf(var);
        } else if (tid >= 32 && tid < 44 && !diverged && !REGEN) {  // the first elite's deviation, alongside
            sh.dbar[tid - 32] = __ldcg(t.ws.theta + ((size_t)b * K + __ldcg(elite)) * 12 + (tid - 32));
        }
        __syncthreads();
        // deviations not stored: regenerated from their draws.  Each thread's first
        // elite row is drawn before the shift is known; thread 0's row is the first
        // elite's, the shift itself.
        float d0[12];
        if (REGEN && !diverged) {
            if (tid < Ke) {
                regen_row((uint32_t)kfirst, b, t.iter, P.seed, P.ctrl, sh.sd12, d0);
                if (tid == 0) {
#pragma unroll
                    for (int c = 0; c < 12; ++c) sh.dbar[c] = d0[c];
                }
            }
            __syncthreads();
        }
        float mean_c = 0.0f, var_c = 0.0f;  // valid in threads < 12
        if (diverged) {
            if (tid < 12) {
                mean_c = sh.mu12[tid];
                var_c = sh.vr12[tid];
            }
        } else {
            // one pass: sums of the deviations and of their squares, both taken
            // about the first elite's deviation d0 (keeps the cancellation small).
            // The order of the sums is that of V virtual lanes (lane v takes elites
            // v, v + V, ...; warp totals in warp order), so a block of any size that
            // divides V gives the same bits.
            for (int v0 = 0; v0 < V; v0 += blockDim.x) {
                const int vl = v0 + tid, vw = vl >> 5;  // virtual lane and warp
                float s[12], s2[12];
#pragma unroll
                for (int c = 0; c < 12; ++c) s[c] = s2[c] = 0.0f;
                int kb = vl < Ke ? __ldcg(elite + vl) : 0;
                if (REGEN) {  // deviations regenerated from their draws
                    for (int e = vl; e < Ke; e += V) {
                        float d[12];
                        if (e == tid) {  // drawn above
#pragma unroll
                            for (int c = 0; c < 12; ++c) d[c] = d0[c];
                        } else {
                            regen_row((uint32_t)kb, b, t.iter, P.seed, P.ctrl, sh.sd12, d);
                        }
                        kb = e + V < Ke ? __ldcg(elite + e + V) : 0;
#pragma unroll
                        for (int c = 0; c < 12; ++c) {
                            const float q = d[c] - sh.dbar[c];
                            s[c] += q;
                            s2[c] = fmaf(q, q, s2[c]);
                        }
                    }
                } else {
                    for (int e = vl; e < Ke; e += V) {
                        // the next elite's index is loaded before this one's row is used
                        const int kn = e + V < Ke ? __ldcg(elite + e + V) : 0;
                        const float4* src = reinterpret_cast<const float4*>(t.ws.theta + ((size_t)b * K + kb) * 12);
                        const float4 a = __ldcg(src), bb = __ldcg(src + 1), cc = __ldcg(src + 2);
                        const float d[12] = {a.x, a.y, a.z, a.w, bb.x, bb.y, bb.z, bb.w, cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                        for (int c = 0; c < 12; ++c) {
                            const float q = d[c] - sh.dbar[c];
                            s[c] += q;
                            s2[c] = fmaf(q, q, s2[c]);
                        }
                        kb = kn;
                    }
                }
                float o[3];
                int c0 = warp_sum12(s, o);
                if ((lane & 7) == 0)
                    for (int i = 0; i < 3; ++i) sh.wacc[vw][c0 + i] = o[i];
                c0 = warp_sum12(s2, o);
                if ((lane & 7) == 0)
                    for (int i = 0; i < 3; ++i) sh.wacc2[vw][c0 + i] = o[i];
            }
            __syncthreads();
            float tot = 0.0f, tot2 = 0.0f;
            if (tid < 12)
                for (int w = 0; w < V / 32; ++w) {
                    tot += sh.wacc[w][tid];
                    tot2 += sh.wacc2[w][tid];
                }
            if (tid < 12) {
                const float m = tot / (float)Ke;
                var_c = fmaxf(fmaf(-m, m, tot2 / (float)Ke), P.var_min);
                mean_c = sh.mu12[tid] + (sh.dbar[tid] + m);
            }
            __syncthreads();
        }
        if (tid < 12) {
            dm[12 * b + tid] = mean_c;
            dv[12 * b + tid] = var_c;
            if (b == 0) {
                const uint32_t ph = (t.phase0 + t.offset[tid / 3]) % kPhaseOne;
                r->u0[tid] = ph < t.duty ? mean_c : 0.0f;
            }
        }
        if (b == 0 && tid == 0 && !P.adaptive) {
            r->f_mean = P.q_init * 0.001f;
            r->q_freq = (int32_t)P.q_init;
        }
    } else {
        // frequency entry (adaptive controllers only)
        const float mu_f = sm[P.D - 1], var_f = sv[P.D - 1];
        float mean_f = mu_f, vf = var_f;
        if (!diverged) {
            if (P.method == SBS_NAIVE) {
                mean_f = (float)__ldcg(t.ws.q + __ldcg(elite)) / 1000.0f;
            } else {
                // two passes over V virtual lanes (the order is
                // independent of the block size, as above)
                __syncthreads();
                for (int v0 = 0; v0 < V; v0 += blockDim.x) {
                    const int vl = v0 + tid;
                    float s = 0.0f;
                    for (int e = vl; e < Ke; e += V) s += (float)__ldcg(t.ws.q + __ldcg(elite + e)) / 1000.0f;
                    s = warp_sum(s);
                    if (lane == 0) sh.red[vl >> 5][0] = s;
                }
                __syncthreads();
                float tot = 0.0f;
                for (int w = 0; w < V / 32; ++w) tot += sh.red[w][0];
                mean_f = tot / (float)Ke;
                for (int v0 = 0; v0 < V; v0 += blockDim.x) {
                    const int vl = v0 + tid;
                    float s2 = 0.0f;
                    for (int e = vl; e < Ke; e += V) {
                        const float d = (float)__ldcg(t.ws.q + __ldcg(elite + e)) / 1000.0f - mean_f;
                        s2 = fmaf(d, d, s2);
                    }
                    s2 = warp_sum(s2);
                    if (lane == 0) sh.red[vl >> 5][1] = s2;
                }
                __syncthreads();
                float tot2 = 0.0f;
                for (int w = 0; w < V / 32; ++w) tot2 += sh.red[w][1];
                vf = fmaxf(tot2 / (float)Ke, P.var_f_min);
            }
        }
        if (tid == 0) {
            dm[P.D - 1] = mean_f;
            dv[P.D - 1] = vf;
            r->f_mean = mean_f;
            r->q_freq = (int32_t)quantise_mhz(mean_f, P.f_min, P.f_max);
        }
    }
}

// Refit of steps b0 .. b1 - 1 of an elite controller whose set fits one pass of
// kRefitThreads virtual lanes per step (Ke <= 2048): the steps' sums are those of
// refit_block (the same virtual lanes, each step's sums about its first elite's
// row), formed kRefitChunk steps at a time with one block barrier per chunk
// instead of several per step, so one block's set-up serves many steps.  Warps
// of virtual lanes past Ke hold exact zeros and skip their reductions.
template <bool REGEN>
__device__ void refit_steps(BlockShared& sh, int b0, int b1)
{
    constexpr int S = kRefitChunk, V = kRefitThreads, NW = V / 32;
    __shared__ float cw[S][NW][12], cw2[S][NW][12];  // per-step totals of the virtual warps
    __shared__ float cmu[S * 12], cvr[S * 12], csd[S * 12], cdb[S * 12];
    const InstParams& P = sh.P;
    const TickArgs& t = sh.t;
    const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x;
    const float* sm = P.state[t.src];
    const float* sv = sm + P.D;
    float* dm = P.state[1 - t.src];
    float* dv = dm + P.D;
    const int K = P.K, Ke = P.Ke;
    const int32_t* elite = t.ws.elite;
    sbs_result* r = t.result;
    const bool diverged = __ldcg(&r->status) != SBS_OK;
    const int e0 = __ldcg(elite);  // the first elite: each step's shift
    for (int c0 = b0; c0 < b1; c0 += S) {
        const int ns = min(S, b1 - c0);
        for (int x = tid; x < 12 * ns; x += T) {
            float m, var;
            shifted_entry(P, t, sm, sv, 12 * c0 + x, m, var);
            cmu[x] = m;
            cvr[x] = var;
            if (REGEN) csd[x] = sqrtf(var);
            else if (!diverged) cdb[x] = __ldcg(t.ws.theta + ((size_t)(c0 + x / 12) * K + e0) * 12 + x % 12);
        }
        __syncthreads();
        if (REGEN && !diverged) {
            for (int jj = tid; jj < ns; jj += T) {
                float d[12];
                regen_row((uint32_t)e0, c0 + jj, t.iter, P.seed, P.ctrl, csd + 12 * jj, d);
#pragma unroll
                for (int c = 0; c < 12; ++c) cdb[12 * jj + c] = d[c];
            }
            __syncthreads();
        }
        if (!diverged) {
            for (int v0 = 0; v0 < V; v0 += T) {
                const int vl = v0 + tid, vw = vl >> 5;
                if (v0 + (tid & ~31) >= Ke) {  // no elite on this virtual warp: zero totals
                    if (lane < 12)
                        for (int jj = 0; jj < ns; ++jj) cw[jj][vw][lane] = cw2[jj][vw][lane] = 0.0f;
                    continue;
                }
                for (int jj = 0; jj < ns; ++jj) {
                    const int j = c0 + jj;
                    const float* db = cdb + 12 * jj;
                    float s[12], s2[12];
#pragma unroll
                    for (int c = 0; c < 12; ++c) s[c] = s2[c] = 0.0f;
                    for (int e = vl; e < Ke; e += V) {
                        const int kb = __ldcg(elite + e);
                        float d[12];
                        if (REGEN) {
                            regen_row((uint32_t)kb, j, t.iter, P.seed, P.ctrl, csd + 12 * jj, d);
                        } else {
                            const float4* src = reinterpret_cast<const float4*>(t.ws.theta + ((size_t)j * K + kb) * 12);
                            const float4 a = __ldcg(src), bb = __ldcg(src + 1), cc = __ldcg(src + 2);
                            d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
                            d[4] = bb.x; d[5] = bb.y; d[6] = bb.z; d[7] = bb.w;
                            d[8] = cc.x; d[9] = cc.y; d[10] = cc.z; d[11] = cc.w;
                        }
#pragma unroll
                        for (int c = 0; c < 12; ++c) {
                            const float q = d[c] - db[c];
                            s[c] += q;
                            s2[c] = fmaf(q, q, s2[c]);
                        }
                    }
                    float o[3];
                    int cc0 = warp_sum12(s, o);
                    if ((lane & 7) == 0)
                        for (int i = 0; i < 3; ++i) cw[jj][vw][cc0 + i] = o[i];
                    cc0 = warp_sum12(s2, o);
                    if ((lane & 7) == 0)
                        for (int i = 0; i < 3; ++i) cw2[jj][vw][cc0 + i] = o[i];
                }
            }
            __syncthreads();
        }
        for (int x = tid; x < 12 * ns; x += T) {
            const int jj = x / 12, c = x - 12 * jj, j = c0 + jj;
            float mean_c, var_c;
            if (diverged) {
                mean_c = cmu[x];
                var_c = cvr[x];
            } else {
                float tot = 0.0f, tot2 = 0.0f;
                for (int w = 0; w < NW; ++w) {
                    tot += cw[jj][w][c];
                    tot2 += cw2[jj][w][c];
                }
                const float m = tot / (float)Ke;
                var_c = fmaxf(fmaf(-m, m, tot2 / (float)Ke), P.var_min);
                mean_c = cmu[x] + (cdb[x] + m);
            }
            dm[12 * j + c] = mean_c;
            dv[12 * j + c] = var_c;
            if (j == 0) {
                const uint32_t ph = (t.phase0 + t.offset[c / 3]) % kPhaseOne;
                r->u0[c] = ph < t.duty ? mean_c : 0.0f;
            }
        }
        if (c0 == 0 && tid == 0 && !P.adaptive) {
            r->f_mean = P.q_init * 0.001f;
            r->q_freq = (int32_t)P.q_init;
        }
        __syncthreads();
    }
}

// Refit item q of a batched controller (refit_items of them).
template <bool REGEN>
__device__ void refit_item(BlockShared& sh, int q)
{
    const InstParams& P = sh.P;
    const int spi = refit_steps_per_item(P.method, P.Ke, P.nt);
    const int nq = (P.nt + spi - 1) / spi;
    if (q >= nq) {
        refit_block<REGEN>(sh, P.nt);  // the frequency entry
    } else if (spi == 1) {
        refit_block<REGEN>(sh, q);
    } else {
        refit_steps<REGEN>(sh, q * spi, min(q * spi + spi, P.nt));
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
template <int NP, bool EXT>
__device__ __forceinline__ void rollout_plain(const InstParams* __restrict__ dP, const TickArgs& t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    rollout_tile<NP, EXT>(sh, reinterpret_cast<float*>(dyn4), blockIdx.x + t.tile_base);
}

template <int NP, bool EXT>
__global__ void __launch_bounds__(SBS_MAX_TILE) k_rollout(const InstParams* __restrict__ dP, TickArgs t)
{
    rollout_plain<NP, EXT>(dP, t);
}

// The ordinary per-step rollout with a register cap that fits 8 blocks of 128
// threads per SM (64 registers, no spills; -1.2 % per batched tick).  The spline
// and extended kernels spill at that cap and keep the compiler's choice.
__global__ void __launch_bounds__(SBS_MAX_TILE, 4) k_rollout_lean(const InstParams* __restrict__ dP, TickArgs t)
{
    rollout_plain<0, false>(dP, t);
}

// Two samples per thread (per-step policy, ordinary model): T / 2 threads per
// tile of T samples, at most 128 registers.
template <bool ADAPT>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2, 4) k_rollout_pair(const InstParams* __restrict__ dP, TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    rollout_tile_pair<ADAPT>(sh, reinterpret_cast<float*>(dyn4), blockIdx.x + t.tile_base);
}

// Two samples per thread with the spline policy: at most 168 registers (the
// knot deviations' shared memory allows three blocks per SM).
template <int NP>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2, 3) k_rollout_pair_spline(const InstParams* __restrict__ dP,
                                                                             TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    rollout_tile_pair_spline<NP>(sh, reinterpret_cast<float*>(dyn4), blockIdx.x + t.tile_base);
}

// Warp-specialised one-sample rollout: 2T threads per tile of T samples.
template <bool EXT>
__global__ void __launch_bounds__(2 * SBS_MAX_TILE) k_rollout_ws(const InstParams* __restrict__ dP, TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    rollout_tile_ws<EXT>(sh, reinterpret_cast<float*>(dyn4), blockIdx.x + t.tile_base);
}

__global__ void __launch_bounds__(kSelectThreads) k_select(const InstParams* __restrict__ dP, TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    select_block(sh, reinterpret_cast<uint32_t*>(dyn4));
}

template <bool REGEN>
__global__ void __launch_bounds__(kRefitLanesMax) k_refit(const InstParams* __restrict__ dP, TickArgs t)
{
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    refit_block<REGEN>(sh, blockIdx.x);
}

// ---- sample sharding: one controller's tiles split over ranks.  Each rank's
// rollout writes its tiles' costs, frequencies and MPPI rows (t.partials = 2: no
// combine); once every rank holds all of them, each runs the update below and
// the selection / refit of the unsharded solve, on the same bits.

// The MPPI combine over every tile's row (Alg. 5 with the per-tile max shift):
// block g combines group g, the last group finishes, as the last tile of each
// group does in an unsharded rollout.  Only the shifted mean and variance are
// staged (the update reads nothing else of the rollout's staging).
__global__ void __launch_bounds__(256) k_shard_combine(const InstParams* __restrict__ dP, TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    const InstParams& P = sh.P;
    const float* sm = P.state[t.src];
    const float* sv = sm + P.D;
    Views v;
    v.mu = reinterpret_cast<float*>(dyn4);
    v.vr = v.mu + P.nb * P.nf;
    v.acc = v.vr + P.nb * P.nf;
    v.sd = v.xr = v.Bs = v.Mb = nullptr;
    v.dsm = nullptr;
    for (int i = threadIdx.x; i < P.nb * P.nf; i += blockDim.x) {
        float m, var;
        shifted_entry(P, sh.t, sm, sv, i, m, var);
        v.mu[i] = m;
        v.vr[i] = var;
    }
    if (threadIdx.x == 0) {
        sh.mu_f = P.adaptive ? sm[P.D - 1] : P.q_init * 0.001f;
        sh.var_f = P.adaptive ? sv[P.D - 1] : 0.0f;
    }
    __syncthreads();
    group_combine(sh, v, blockIdx.x);
}

// The selection's side data from the full cost array: the key histograms of a
// large elite selection, and Naive's best complemented (cost key, index) per
// force block with its finite count.  Integer sums and maxima: the same words
// as the rollout tiles' atomics leave, whatever the order.
__global__ void __launch_bounds__(256) k_cost_keys(const InstParams* __restrict__ dP, TickArgs t)
{
    const int K = dP->K, n_freq = dP->n_freq, adaptive = dP->adaptive;
    const uint32_t seed = dP->seed, ctrl = dP->ctrl;
    const int lane = threadIdx.x & 31;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < (uint32_t)K;
    const float J = valid ? __ldcg(t.ws.J + k) : kInf;
    if (t.ws.hist) {
        const uint32_t bin = cost_key(J) >> 16;
        const unsigned act = __ballot_sync(kFull, valid);
        if (valid) {
            const unsigned peers = __match_any_sync(act, bin);
            if (lane == __ffs(peers) - 1) atomicAdd(t.ws.hist + bin, (unsigned)__popc(peers));
            const unsigned peers8 = __match_any_sync(act, bin >> 8);
            if (lane == __ffs(peers8) - 1) atomicAdd(t.ws.hist + kHistBins + (bin >> 8), (unsigned)__popc(peers8));
        }
    }
    if (t.ws.best) {
        const int blk = (valid && !adaptive && n_freq > 0) ? freq_block(k, t.iter, seed, ctrl, n_freq) : 0;
        const bool fin = valid && J < kInf;
        const unsigned long long key = fin ? ~(((unsigned long long)cost_key(J) << 32) | k) : 0ull;
        unsigned todo = __reduce_or_sync(kFull, fin ? 1u << blk : 0u);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            unsigned long long m = blk == b ? key : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long x = __shfl_xor_sync(kFull, m, o);
                m = x > m ? x : m;
            }
            if (lane == 0) atomicMax(t.ws.best + b, m);
        }
        const unsigned nfw = __popc(__ballot_sync(kFull, fin));
        if (lane == 0 && nfw) atomicAdd(t.ws.nfin, nfw);
    }
}

__global__ void k_init(const InstParams* __restrict__ dP, TickArgs t)
{
    __shared__ BlockShared sh;
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
    const InstParams& P = sh.P;
    float* m = P.state[sh.t.src];
    float* v = m + P.D;
    for (int i = threadIdx.x; i < P.nb * P.nf; i += blockDim.x) init_entry(P, sh.t, i, m[i], v[i]);
    if (threadIdx.x == 0 && P.adaptive) {
        m[P.D - 1] = P.q_init * 0.001f;
        v[P.D - 1] = P.var_f_init;
    }
}

// Item it of a batched launch belongs to the last controller whose first item
// is <= it (records are in item order).  which: 0 tiles, 1 selections, 2 refits.
__device__ __forceinline__ int find_rec(const InstRec* recs, int n, int it, int which)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b =
            which == 0 ? recs[mid].tile_begin : (which == 1 ? recs[mid].select_begin : recs[mid].refit_begin);
        if (b <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int rec_begin(const InstRec& r, int which)
{
    return which == 0 ? r.tile_begin : (which == 1 ? r.select_begin : r.refit_begin);
}

// The same record found by the whole block in at most two rounds of independent
// loads instead of the search's chain of dependent ones.  Record i holds item it
// when begin(i) <= it < begin(i + 1) (begins are non-decreasing from 0, and a
// record with no items has begin(i) = begin(i + 1), so exactly one record
// matches).  With more records than threads, the bucket of ceil(n / T)
// consecutive records that holds it is found first by the same test on the
// bucket boundaries, then the record within it.

__device__ __forceinline__ int find_rec_block(BlockShared& sh, const InstRec* recs, int n, int it, int which)
{
    const int T = blockDim.x;
    int lo = 0, cnt = n;
    if (n > T) {  // first the bucket of ceil(n / T) records that holds the item
        const int w = (n + T - 1) / T;
        const int i = threadIdx.x * w;
        if (i < n) {
            const int b0 = rec_begin(recs[i], which);
            const int b1 = i + w < n ? rec_begin(recs[i + w], which) : 0x7fffffff;
            if (b0 <= it && it < b1) sh.item = i;
        }
        __syncthreads();
        lo = sh.item;
        cnt = min(w, n - lo);
        __syncthreads();
    }
    for (int j = threadIdx.x; j < cnt; j += T) {
        const int i = lo + j;
        const int b0 = rec_begin(recs[i], which);
        const int b1 = i + 1 < n ? rec_begin(recs[i + 1], which) : 0x7fffffff;
        if (b0 <= it && it < b1) sh.item = i;
    }
    __syncthreads();
    return sh.item;
}

// counts = {controllers, end of the tile items, selection items, refit items, first
// tile item of a grid launch}; heads = queue heads.
// Every controller of one launch uses the same policy (NP).
template <int NP, bool EXT>
__global__ void __launch_bounds__(SBS_MAX_TILE) k_batch_rollout(const InstRec* __restrict__ recs,
                                                                const int* __restrict__ counts, int* heads)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int n = counts[0], nitems = counts[1];
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&heads[0], 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= nitems) break;
        const int i = find_rec(recs, n, it, 0);
        load_params(recs[i].dP, sh);
        load_tick(&recs[i].t, sh);
        __syncthreads();
        rollout_tile<NP, EXT>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
        __syncthreads();
    }
}

// One block per item: the hardware block scheduler is the queue (items are
// dispatched in index order, heavy controllers first).  Unused blocks exit.
template <int NP, bool EXT>
__device__ __forceinline__ void rollout_grid_item(const InstRec* __restrict__ recs, const int* __restrict__ counts)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int it = blockIdx.x + counts[4];  // a launch may start past the first tiles
    if (it >= counts[1]) return;
    const int i = find_rec_block(sh, recs, counts[0], it, 0);
    load_params(recs[i].dP, sh);
    load_tick(&recs[i].t, sh);
    __syncthreads();
    rollout_tile<NP, EXT>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
}

template <int NP, bool EXT>
__global__ void __launch_bounds__(SBS_MAX_TILE) k_grid_rollout(const InstRec* __restrict__ recs,
                                                               const int* __restrict__ counts)
{
    rollout_grid_item<NP, EXT>(recs, counts);
}

// The ordinary per-step grid rollout with the register cap of k_rollout_lean.
__global__ void __launch_bounds__(SBS_MAX_TILE, 4) k_grid_rollout_lean(const InstRec* __restrict__ recs,
                                                                       const int* __restrict__ counts)
{
    rollout_grid_item<0, false>(recs, counts);
}

// The same with two samples per thread (T / 2 threads per tile item).
template <bool ADAPT>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2, 4) k_grid_rollout_pair(const InstRec* __restrict__ recs,
                                                                           const int* __restrict__ counts)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int it = blockIdx.x + counts[4];
    if (it >= counts[1]) return;
    const int i = find_rec_block(sh, recs, counts[0], it, 0);
    load_params(recs[i].dP, sh);
    load_tick(&recs[i].t, sh);
    __syncthreads();
    rollout_tile_pair<ADAPT>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
}

// Persistent blocks pulling tile items, two samples per thread.
template <bool ADAPT>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2) k_batch_rollout_pair(const InstRec* __restrict__ recs,
                                                                         const int* __restrict__ counts, int* heads)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int n = counts[0], nitems = counts[1];
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&heads[0], 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= nitems) break;
        const int i = find_rec(recs, n, it, 0);
        load_params(recs[i].dP, sh);
        load_tick(&recs[i].t, sh);
        __syncthreads();
        rollout_tile_pair<ADAPT>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
        __syncthreads();
    }
}

// The spline policy with two samples per thread (T / 2 threads per tile item).
template <int NP>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2, 3) k_grid_rollout_pair_spline(const InstRec* __restrict__ recs,
                                                                                  const int* __restrict__ counts)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int it = blockIdx.x + counts[4];
    if (it >= counts[1]) return;
    const int i = find_rec_block(sh, recs, counts[0], it, 0);
    load_params(recs[i].dP, sh);
    load_tick(&recs[i].t, sh);
    __syncthreads();
    rollout_tile_pair_spline<NP>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
}

template <int NP>
__global__ void __launch_bounds__(SBS_MAX_TILE / 2) k_batch_rollout_pair_spline(const InstRec* __restrict__ recs,
                                                                                const int* __restrict__ counts,
                                                                                int* heads)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int n = counts[0], nitems = counts[1];
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&heads[0], 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= nitems) break;
        const int i = find_rec(recs, n, it, 0);
        load_params(recs[i].dP, sh);
        load_tick(&recs[i].t, sh);
        __syncthreads();
        rollout_tile_pair_spline<NP>(sh, reinterpret_cast<float*>(dyn4), it - recs[i].tile_begin);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSelectThreads) k_grid_select(const InstRec* __restrict__ recs,
                                                               const int* __restrict__ counts)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int it = blockIdx.x;
    if (it >= counts[2]) return;
    const int i = find_rec_block(sh, recs, counts[0], it, 1);
    load_params(recs[i].dP, sh);
    load_tick(&recs[i].t, sh);
    __syncthreads();
    select_block(sh, reinterpret_cast<uint32_t*>(dyn4));
}

template <bool REGEN>
__global__ void __launch_bounds__(kBatchRefitThreads) k_grid_refit(const InstRec* __restrict__ recs,
                                                             const int* __restrict__ counts)
{
    __shared__ BlockShared sh;
    const int it = blockIdx.x;
    if (it >= counts[3]) return;
    const int i = find_rec_block(sh, recs, counts[0], it, 2);
    load_params(recs[i].dP, sh);
    load_tick(&recs[i].t, sh);
    __syncthreads();
    refit_item<REGEN>(sh, it - recs[i].refit_begin);
}

__global__ void __launch_bounds__(kSelectThreads) k_batch_select(const InstRec* __restrict__ recs,
                                                                const int* __restrict__ counts, int* heads)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    const int n = counts[0], nitems = counts[2];
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&heads[1], 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= nitems) break;
        const int i = find_rec(recs, n, it, 1);
        load_params(recs[i].dP, sh);
        load_tick(&recs[i].t, sh);
        __syncthreads();
        select_block(sh, reinterpret_cast<uint32_t*>(dyn4));
        __syncthreads();
    }
}

template <bool REGEN>
__global__ void __launch_bounds__(kBatchRefitThreads) k_batch_refit(const InstRec* __restrict__ recs,
                                                              const int* __restrict__ counts, int* heads)
{
    __shared__ BlockShared sh;
    const int n = counts[0], nitems = counts[3];
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(&heads[2], 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= nitems) break;
        const int i = find_rec(recs, n, it, 2);
        load_params(recs[i].dP, sh);
        load_tick(&recs[i].t, sh);
        __syncthreads();
        refit_item<REGEN>(sh, it - recs[i].refit_begin);
        __syncthreads();
    }
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, uint32_t* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 w = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

__global__ void k_sqrt_hw(const float* __restrict__ x, float* __restrict__ y, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = sqrt_hw(x[i]);
}

// The attitude sine and cosine: out = [sin, cos (one lane) | sin, cos (lane pairs
// (2m, 2m + 1); the last lane of an odd n paired with itself) | the library's
// sincosf | the hardware approximation], n floats each.
__global__ void k_sincos(const float* __restrict__ x, float* __restrict__ out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c;
    sincos_v<float>(x[i], s, c);
    out[i] = s;
    out[n + i] = c;
    const int i0 = i & ~1, i1 = min(i0 + 1, n - 1);
    float2 s2, c2;
    sincos_v<float2>(make_float2(x[i0], x[i1]), s2, c2);
    out[2 * n + i] = (i & 1) ? s2.y : s2.x;
    out[3 * n + i] = (i & 1) ? c2.y : c2.x;
    sincosf(x[i], &s, &c);
    out[4 * n + i] = s;
    out[5 * n + i] = c;
    __sincosf(x[i], &s, &c);
    out[6 * n + i] = s;
    out[7 * n + i] = c;
}

__global__ void k_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nk) return;
    const uint32_t k = (uint32_t)(k0 + i);
    float* o = out + (size_t)i * (nn + 1);
    const uint4 w = philox4x32_10(make_uint4(k, 0u, (uint32_t)iter, (uint32_t)(iter >> 32)), seed, ctrl);
    o[0] = box_muller(w.x, w.y).x;
    // force draws through the per-sample precomputed Philox state the rollout uses
    const PhiloxPre pp = philox_pre(k, iter, seed, ctrl);
    for (int d = 0; 6 * d < nn; ++d) {
        float zz[6];
        normals6(philox_draw(pp, 1u + (uint32_t)d), zz);
        for (int s = 0; s < 6 && 6 * d + s < nn; ++s) o[1 + 6 * d + s] = zz[s];
    }
}

// FP32 FMA chains: 8 independent accumulators per thread, 2 FLOP per FMA.
__global__ void k_fma_peak(float* out, int iters)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
    const float b = 0.999f, c = 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

// ---------------------------------------------------------------------------
// Multi-block elite selection of one large controller (K > kSelectSmemMaxK, plain
// solves): the same threshold key and ordered list as select_block, with the
// passes over all K costs spread over blocks of kSelChunk keys.
//   k_sel_find    1 block: the 16-bit bin holding rank Ke (rollout histograms)
//   k_sel_gather  the bin's keys (low 16 bits) into ws.cand, any order
//   k_sel_thr     1 block: two 8-bit passes over them: thr, need_eq
//   k_sel_count   per block: keys below / equal to thr; best cost, finite count
//   k_sel_write   per block: its offset from the blocks before it, then its
//                 part of the list in index order; block 0 writes the record
// ws.sel holds {b16, rank in bin, bin count, gather counter, thr, need_eq, best
// cost key, finite count}.
// ---------------------------------------------------------------------------
constexpr int kSelChunk = 2048;
constexpr int kSelBlock = 256;

__device__ __forceinline__ void load_block_params(BlockShared& sh, const InstParams* dP, const TickArgs& t)
{
    load_params(dP, sh);
    if (threadIdx.x == 0) sh.t = t;
    __syncthreads();
}

__global__ void __launch_bounds__(kSelectThreads) k_sel_find(const InstParams* __restrict__ dP, TickArgs t)
{
    __shared__ BlockShared sh;
    load_block_params(sh, dP, t);
    uint32_t b16;
    int rank, ncand;
    find_bin16(sh, b16, rank, ncand, false);  // k_sel_gather clears the histograms
    if (threadIdx.x == 0) {
        uint32_t* sc = t.ws.sel;
        sc[0] = b16;
        sc[1] = (uint32_t)rank;
        sc[2] = (uint32_t)ncand;
        sc[3] = 0u;
        sc[6] = 0xffffffffu;
        sc[7] = 0u;
    }
}

__global__ void __launch_bounds__(kSelBlock) k_sel_gather(const InstParams* __restrict__ dP, TickArgs t)
{
    const int K = dP->K;
    const uint32_t b16 = __ldcg(t.ws.sel);
    const int lane = threadIdx.x & 31;
    // clear the rollout's histograms for the next solve (k_sel_find has read them)
    for (int i = blockIdx.x * kSelBlock + threadIdx.x; i < kHistBins + 256; i += gridDim.x * kSelBlock)
        t.ws.hist[i] = 0u;
    const int i0 = blockIdx.x * kSelChunk + 4 * threadIdx.x;
    for (int r = 0; r < kSelChunk / (4 * kSelBlock); ++r) {
        const int i = i0 + r * 4 * kSelBlock;
        float c[4];
        load4(t.ws.J, i, K, c);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t key = cost_key(c[u]);
            const bool m = i + u < K && (key >> 16) == b16;
            const unsigned bal = __ballot_sync(kFull, m);
            if (bal) {
                unsigned at = 0;
                if (lane == __ffs(bal) - 1) at = atomicAdd(t.ws.sel + 3, (unsigned)__popc(bal));
                at = __shfl_sync(kFull, at, __ffs(bal) - 1);
                if (m) t.ws.cand[at + __popc(bal & ((1u << lane) - 1u))] = key & 0xffffu;
            }
        }
    }
}

__global__ void __launch_bounds__(kSelectThreads) k_sel_thr(const InstParams* __restrict__ dP, TickArgs t)
{
    extern __shared__ float4 dyn4[];
    __shared__ BlockShared sh;
    load_block_params(sh, dP, t);
    uint32_t* sc = t.ws.sel;
    const uint32_t b16 = __ldcg(sc);
    int rank = (int)__ldcg(sc + 1);
    const int n = (int)__ldcg(sc + 3);
    uint32_t prefix, mask;
    if (n <= kSelectSmemMaxK) {
        uint32_t* keys = reinterpret_cast<uint32_t*>(dyn4);
        for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = __ldcg(t.ws.cand + i);
        __syncthreads();
        prefix = 0;
        mask = 0;
        radix_pass<true>(sh, keys, nullptr, n, 8, prefix, mask, rank);
        radix_pass<true>(sh, keys, nullptr, n, 0, prefix, mask, rank);
        prefix |= b16 << 16;
    } else {  // the bin does not fit: finish over all keys
        prefix = b16 << 16;
        mask = 0xffff0000u;
        radix_pass<false>(sh, nullptr, t.ws.J, sh.P.K, 8, prefix, mask, rank);
        radix_pass<false>(sh, nullptr, t.ws.J, sh.P.K, 0, prefix, mask, rank);
    }
    if (threadIdx.x == 0) {
        sc[4] = prefix;
        sc[5] = (uint32_t)rank;
    }
}

__global__ void __launch_bounds__(kSelBlock) k_sel_count(const InstParams* __restrict__ dP, TickArgs t)
{
    __shared__ int s_cnt[2][kSelBlock / 32];
    __shared__ float s_min[kSelBlock / 32];
    const int K = dP->K;
    const uint32_t thr = __ldcg(t.ws.sel + 4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = blockIdx.x * kSelChunk + 4 * tid;
    int lt = 0, eq = 0, nf = 0;
    float bmin = kInf;
    for (int r = 0; r < kSelChunk / (4 * kSelBlock); ++r) {
        const int i = i0 + r * 4 * kSelBlock;
        float c[4];
        load4(t.ws.J, i, K, c);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i + u < K) {
                const uint32_t key = cost_key(c[u]);
                lt += key < thr ? 1 : 0;
                eq += key == thr ? 1 : 0;
                bmin = fminf(bmin, c[u]);
                nf += c[u] < kInf ? 1 : 0;
            }
        }
    }
    lt = warp_sum_int(lt);
    eq = warp_sum_int(eq);
    nf = warp_sum_int(nf);
    bmin = warp_min(bmin);
    if (lane == 0) {
        s_cnt[0][warp] = lt;
        s_cnt[1][warp] = eq;
        s_min[warp] = bmin;
        if (nf) atomicAdd(t.ws.sel + 7, (unsigned)nf);
    }
    __syncthreads();
    if (tid == 0) {
        int a = 0, b = 0;
        float m = kInf;
        for (int w = 0; w < kSelBlock / 32; ++w) {
            a += s_cnt[0][w];
            b += s_cnt[1][w];
            m = fminf(m, s_min[w]);
        }
        t.ws.bcnt[2 * blockIdx.x] = a;
        t.ws.bcnt[2 * blockIdx.x + 1] = b;
        atomicMin(t.ws.sel + 6, cost_key(m));
    }
}

__global__ void __launch_bounds__(kSelBlock) k_sel_write(const InstParams* __restrict__ dP, TickArgs t)
{
    __shared__ BlockShared sh;
    load_block_params(sh, dP, t);
    const int K = sh.P.K;
    const uint32_t* sc = t.ws.sel;
    const uint32_t thr = __ldcg(sc + 4);
    const int need_eq = (int)__ldcg(sc + 5);
    if (threadIdx.x < 32) {
        // this block's offset and share of the ties: the blocks before it hold lt keys
        // below thr and eq equal to it, of which the first need_eq are taken
        int lt = 0, eq = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += 32) {
            lt += __ldcg(t.ws.bcnt + 2 * b);
            eq += __ldcg(t.ws.bcnt + 2 * b + 1);
        }
        lt = warp_sum_int(lt);
        eq = warp_sum_int(eq);
        if (threadIdx.x == 0) {
            sh.digit = lt + min(eq, need_eq);
            sh.below = max(0, need_eq - eq);
        }
    }
    __syncthreads();
    const int begin = blockIdx.x * kSelChunk, end = min(K, begin + kSelChunk);
    float bm;
    int nf;
    compact_range<1>(sh, thr, sh.below, begin, end, sh.digit, &bm, &nf);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t mk = __ldcg(sc + 6);
        const int nfin = (int)__ldcg(sc + 7);
        sbs_result* r = t.result;
        r->cost_min = mk == 0xffffffffu ? kInf : key_cost(mk);
        r->ess = (float)sh.P.Ke;
        r->status = nfin > 0 ? SBS_OK : SBS_ERR_DIVERGED;
        r->n_finite = nfin;
        r->iter_lo = (uint32_t)t.iter;
        r->iter_hi = (uint32_t)(t.iter >> 32);
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int status_of(cudaError_t e) { return e == cudaSuccess ? SBS_OK : SBS_ERR_CUDA; }

static int ensure_smem_attr(const void* fn, size_t smem)
{
    // the 48 KB a block may take without opting in include its static BlockShared
    if (smem + sizeof(BlockShared) <= 48 * 1024) return SBS_OK;
    return status_of(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
}

template <int NP, bool S>
static const void* batch_fn(int mode)
{
    if (mode == SBS_BATCH_GRID)
        return NP == 0 && !S ? (const void*)k_grid_rollout_lean : (const void*)k_grid_rollout<NP, S>;
    return (const void*)k_batch_rollout<NP, S>;
}

template <bool S>
static const void* rollout_kernel_s(int P)
{
    switch (P) {
        case 0: return S ? (const void*)k_rollout<0, S> : (const void*)k_rollout_lean;
        case 2: return (const void*)k_rollout<2, S>;
        case 3: return (const void*)k_rollout<3, S>;
        case 4: return (const void*)k_rollout<4, S>;
        case 6: return (const void*)k_rollout<6, S>;
        case 8: return (const void*)k_rollout<8, S>;
        default: return nullptr;
    }
}

template <bool S>
static const void* batch_rollout_fn_s(int P, int mode)
{
    switch (P) {
        case 0: return batch_fn<0, S>(mode);
        case 2: return batch_fn<2, S>(mode);
        case 3: return batch_fn<3, S>(mode);
        case 4: return batch_fn<4, S>(mode);
        case 6: return batch_fn<6, S>(mode);
        case 8: return batch_fn<8, S>(mode);
        default: return nullptr;
    }
}

static const void* pair_spline_fn(int P, int mode)  // mode: -1 plain launch
{
    switch (P) {
#define SBS_PAIR_SPLINE(N)                                                                        \
    case N:                                                                                       \
        return mode < 0 ? (const void*)k_rollout_pair_spline<N>                                   \
                        : mode == SBS_BATCH_GRID ? (const void*)k_grid_rollout_pair_spline<N>     \
                                                 : (const void*)k_batch_rollout_pair_spline<N>;
        SBS_PAIR_SPLINE(2)
        SBS_PAIR_SPLINE(3)
        SBS_PAIR_SPLINE(4)
        SBS_PAIR_SPLINE(6)
        SBS_PAIR_SPLINE(8)
#undef SBS_PAIR_SPLINE
        default: return nullptr;
    }
}

static const void* rollout_kernel(int variant)
{
    if (variant & kPairVariant) {
        const int P = variant & 0xff;
        if (P > 0) return (variant & ~0xff) == kPairVariant ? pair_spline_fn(P, -1) : nullptr;
        if ((variant & ~kAdaptVariant) != kPairVariant) return nullptr;
        return (variant & kAdaptVariant) ? (const void*)k_rollout_pair<true> : (const void*)k_rollout_pair<false>;
    }
    const int P = variant & ~kExtVariant;
    return (variant & kExtVariant) ? rollout_kernel_s<true>(P) : rollout_kernel_s<false>(P);
}

const void* batch_rollout_fn(int variant, int mode)
{
    variant &= ~kRegenVariant;  // the rollouts read the tick's flag
    if (variant & kPairVariant) {
        const int P = variant & 0xff;
        if (P > 0) return (variant & ~0xff) == kPairVariant ? pair_spline_fn(P, mode) : nullptr;
        if ((variant & ~kAdaptVariant) != kPairVariant) return nullptr;
        if (variant & kAdaptVariant)
            return mode == SBS_BATCH_GRID ? (const void*)k_grid_rollout_pair<true> : (const void*)k_batch_rollout_pair<true>;
        return mode == SBS_BATCH_GRID ? (const void*)k_grid_rollout_pair<false> : (const void*)k_batch_rollout_pair<false>;
    }
    const int P = variant & ~kExtVariant;
    return (variant & kExtVariant) ? batch_rollout_fn_s<true>(P, mode) : batch_rollout_fn_s<false>(P, mode);
}

const void* batch_select_fn(int mode)
{
    return mode == SBS_BATCH_GRID ? (const void*)k_grid_select : (const void*)k_batch_select;
}

const void* batch_refit_fn(int mode, bool regen)
{
    if (regen) return mode == SBS_BATCH_GRID ? (const void*)k_grid_refit<true> : (const void*)k_batch_refit<true>;
    return mode == SBS_BATCH_GRID ? (const void*)k_grid_refit<false> : (const void*)k_batch_refit<false>;
}

int launch_init(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream)
{
    (void)hP;
    k_init<<<1, 256, 0, (cudaStream_t)stream>>>(dP, t);
    return status_of(cudaGetLastError());
}

int launch_rollout(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream, int spt, int tiles)
{
    if (tiles < 0) tiles = hP.ntiles;
    if (tiles == 0) return SBS_OK;
    if (spt == SBS_SPT_NOISE_WARPS) {
        const bool ext0 = hP.n_freq > 0 || hP.world_feet || hP.friction_project;
        if (ws_capable(hP.P, ext0, hP.H, hP.T, hP.nb)) {
            const size_t smem = ws_smem_bytes(hP.H, hP.T, hP.nb);
            const void* fn = ext0 ? (const void*)k_rollout_ws<true> : (const void*)k_rollout_ws<false>;
            int st = ensure_smem_attr(fn, smem);
            if (st) return st;
            if (ext0) k_rollout_ws<true><<<tiles, 2 * hP.T, smem, (cudaStream_t)stream>>>(dP, t);
            else k_rollout_ws<false><<<tiles, 2 * hP.T, smem, (cudaStream_t)stream>>>(dP, t);
            return status_of(cudaGetLastError());
        }
        spt = 1;
    }
    const bool ext = hP.n_freq > 0 || hP.world_feet || hP.friction_project;
    const bool pair = spt == 2 && pair_capable(hP.P, ext, hP.T) && pair_fits(hP.H, hP.P, hP.T, hP.nb);
    const size_t smem = rollout_smem_bytes(hP.H, hP.P, hP.T, hP.nb, pair);
    const void* fn = rollout_kernel(rollout_variant(hP.P, ext, pair, false, hP.adaptive != 0));
    if (!fn) return SBS_ERR_INVALID_ARG;
    int st = ensure_smem_attr(fn, smem);
    if (st) return st;
    TickArgs targ = t;
    const InstParams* parg = dP;
    void* args[] = {(void*)&parg, (void*)&targ};
    return status_of(
        cudaLaunchKernel(fn, dim3(tiles), dim3(pair ? hP.T / 2 : hP.T), args, smem, (cudaStream_t)stream));
}

int launch_shard_finish(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream)
{
    const size_t smem = (2 * (size_t)hP.nb * hP.nf + hP.nf + kPartHeader) * sizeof(float);
    int st = ensure_smem_attr((const void*)k_shard_combine, smem);
    if (st) return st;
    k_shard_combine<<<hP.ngroups, 256, smem, (cudaStream_t)stream>>>(dP, t);
    return status_of(cudaGetLastError());
}

int launch_cost_keys(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream)
{
    if (!t.ws.hist && !t.ws.best) return SBS_OK;
    k_cost_keys<<<(hP.K + 255) / 256, 256, 0, (cudaStream_t)stream>>>(dP, t);
    return status_of(cudaGetLastError());
}

int launch_select(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream)
{
    if (hP.method == SBS_ELITE && hP.K > kSelectSmemMaxK && t.ws.hist && t.ws.sel) {
        cudaStream_t s = (cudaStream_t)stream;
        const int G = (hP.K + kSelChunk - 1) / kSelChunk;
        const size_t thr_smem = 4 * (size_t)kSelectSmemMaxK;
        int st = ensure_smem_attr((const void*)k_sel_thr, thr_smem);
        if (st) return st;
        k_sel_find<<<1, kSelectThreads, 0, s>>>(dP, t);
        k_sel_gather<<<G, kSelBlock, 0, s>>>(dP, t);
        k_sel_thr<<<1, kSelectThreads, thr_smem, s>>>(dP, t);
        k_sel_count<<<G, kSelBlock, 0, s>>>(dP, t);
        k_sel_write<<<G, kSelBlock, 0, s>>>(dP, t);
        return status_of(cudaGetLastError());
    }
    const size_t smem = select_smem_bytes(hP.K);
    int st = ensure_smem_attr((const void*)k_select, smem);
    if (st) return st;
    k_select<<<1, kSelectThreads, smem, (cudaStream_t)stream>>>(dP, t);
    return status_of(cudaGetLastError());
}

int launch_refit(const InstParams* dP, const InstParams& hP, const TickArgs& t, void* stream)
{
    const int grid = hP.nt + (hP.adaptive ? 1 : 0);
    const int threads = hP.method == SBS_ELITE ? refit_lanes(hP.Ke) : kRefitThreads;
    if (t.regen) k_refit<true><<<grid, threads, 0, (cudaStream_t)stream>>>(dP, t);
    else k_refit<false><<<grid, threads, 0, (cudaStream_t)stream>>>(dP, t);
    return status_of(cudaGetLastError());
}

// Grid sizes of the three stages.  Persistent mode: as many blocks as fit on the
// GPU at once.  Grid mode: one block per item (at least one).
int batch_grid(int P, int mode, size_t smem, size_t sel_smem, int T, const int counts[4], int grids[3])
{
    const void* fn = batch_rollout_fn(P, mode);
    if (!fn) return SBS_ERR_INVALID_ARG;
    int st = ensure_smem_attr(fn, smem);
    if (st) return st;
    st = ensure_smem_attr(batch_select_fn(mode), sel_smem);
    if (st) return st;
    if (mode == SBS_BATCH_GRID) {
        grids[0] = counts[1] > 0 ? counts[1] : 1;
        grids[1] = counts[2] > 0 ? counts[2] : 1;
        grids[2] = counts[3] > 0 ? counts[3] : 1;
        return SBS_OK;
    }
    int dev, sms, b1 = 0, b2 = 0, b3 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SBS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SBS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, fn, T, smem) != cudaSuccess) return SBS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_batch_select, kSelectThreads, sel_smem) != cudaSuccess)
        return SBS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, batch_refit_fn(mode, (P & kRegenVariant) != 0),
                                                      kBatchRefitThreads, 0) != cudaSuccess)
        return SBS_ERR_CUDA;
    if (b1 < 1 || b2 < 1 || b3 < 1) return SBS_ERR_INVALID_ARG;
    grids[0] = sms * b1;
    grids[1] = sms * b2;
    grids[2] = sms * b3;
    return SBS_OK;
}

// events: null, or four CUDA events recorded before and after each stage.
int launch_batch(int P, int mode, const InstRec* dRecs, const int* dCounts, int* dHeads, size_t smem,
                 size_t sel_smem, int T, const int grids[4], void* stream, void* const* events)
{
    cudaStream_t s = (cudaStream_t)stream;
    const void* fns[3] = {batch_rollout_fn(P, mode), batch_select_fn(mode),
                          batch_refit_fn(mode, (P & kRegenVariant) != 0)};
    if (!fns[0]) return SBS_ERR_INVALID_ARG;
    const dim3 blocks[3] = {dim3(T), dim3(mode == SBS_BATCH_GRID ? kBatchSelectThreads : kSelectThreads),
                            dim3(kBatchRefitThreads)};
    const size_t shm[3] = {smem, sel_smem, 0};
    const InstRec* r = dRecs;
    const int* c = dCounts;
    const int* c2 = dCounts + kBatchCountsB;
    int* hd = dHeads;
    void* args[] = {(void*)&r, (void*)&c, (void*)&hd};
    void* args2[] = {(void*)&r, (void*)&c2, (void*)&hd};
    for (int k = 0; k < 3; ++k) {
        if (events) cudaEventRecord((cudaEvent_t)events[k], s);
        if (cudaLaunchKernel(fns[k], dim3(grids[k]), blocks[k], args, shm[k], s) != cudaSuccess) return SBS_ERR_CUDA;
        if (k == 0 && grids[3] > 0 &&  // the MPPI controllers' tiles (grid mode, split tick)
            cudaLaunchKernel(fns[0], dim3(grids[3]), blocks[0], args2, shm[0], s) != cudaSuccess)
            return SBS_ERR_CUDA;
    }
    if (events) cudaEventRecord((cudaEvent_t)events[3], s);
    return SBS_OK;
}

int launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* stream)
{
    if (n <= 0) return SBS_OK;
    k_philox<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(ctr, key, out, n);
    return status_of(cudaGetLastError());
}

int launch_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out, void* stream)
{
    if (nk <= 0) return SBS_OK;
    k_normals<<<(nk + 127) / 128, 128, 0, (cudaStream_t)stream>>>(seed, ctrl, iter, k0, nk, nn, out);
    return status_of(cudaGetLastError());
}

int launch_sincos(const float* x, float* out, int n, void* stream)
{
    if (n <= 0) return SBS_OK;
    k_sincos<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, out, n);
    return status_of(cudaGetLastError());
}

int launch_sqrt_hw(const float* x, float* y, int n, void* stream)
{
    if (n <= 0) return SBS_OK;
    k_sqrt_hw<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return status_of(cudaGetLastError());
}

int launch_fma_peak(float* out, int iters, int blocks, int threads, void* stream)
{
    k_fma_peak<<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters);
    return status_of(cudaGetLastError());
}

}  // namespace sbs
