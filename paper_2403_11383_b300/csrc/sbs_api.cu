// Host side of the C ABI declared in include/sbs.h: validation, device-state
// layout, the plain per-solve launch sequence, batched graph-captured ticks,
// checkpoints and the FP32 peak microbenchmark.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <numeric>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "sbs_internal.h"

using namespace sbs;

namespace {

constexpr uint32_t kStateMagic = 0x53425331u;  // "SBS1"

bool finite_all(const float* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace sbs {

int validate_config(const sbs_config* c)
{
    if (!c) return SBS_ERR_INVALID_ARG;
    if (c->K < 1 || c->K > SBS_MAX_K) return SBS_ERR_INVALID_ARG;
    if (c->H < 1 || c->H > SBS_MAX_H) return SBS_ERR_INVALID_ARG;
    if (!(c->P == 0 || c->P == 2 || c->P == 3 || c->P == 4 || c->P == 6 || c->P == 8)) return SBS_ERR_INVALID_ARG;
    if (c->P > 0 && c->H < 2) return SBS_ERR_INVALID_ARG;
    if (c->method < SBS_MPPI || c->method > SBS_NAIVE) return SBS_ERR_INVALID_ARG;
    if (c->iterations < 1 || c->iterations > 1000) return SBS_ERR_INVALID_ARG;
    if (c->method == SBS_ELITE && (c->elite_count < 1 || c->elite_count > c->K)) return SBS_ERR_INVALID_ARG;
    if (c->dt_us < 1 || c->dt_us > 1000000) return SBS_ERR_INVALID_ARG;
    if (!(c->lambda > 0.0f) || !std::isfinite(c->lambda)) return SBS_ERR_INVALID_ARG;
    if (!(c->f_min > 0.0f) || !(c->f_max >= c->f_min) || !std::isfinite(c->f_max)) return SBS_ERR_INVALID_ARG;
    // the per-step phase advance q * dt_us must stay below one cycle
    const double qmax = std::max<double>(c->q_init, std::floor(1000.0 * c->f_max + 0.5) + 1.0);
    if (qmax * c->dt_us >= 1e9) return SBS_ERR_INVALID_ARG;
    if (c->q_init < 1) return SBS_ERR_INVALID_ARG;
    if (!(c->sigma_init >= 0.0f) || !(c->sigma_min >= 0.0f) || !(c->sigma_f_init >= 0.0f) || !(c->sigma_f_min >= 0.0f))
        return SBS_ERR_INVALID_ARG;
    if (c->tile != 0 && (c->tile < 64 || c->tile > SBS_MAX_TILE || c->tile % 32 != 0)) return SBS_ERR_INVALID_ARG;
    const sbs_model& m = c->model;
    if (!(m.mass > 0.0f)) return SBS_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(m.inertia[a] > 0.0f)) return SBS_ERR_INVALID_ARG;
    if (!finite_all(&m.foot[0][0], 12) || !finite_all(m.gravity, 3)) return SBS_ERR_INVALID_ARG;
    const sbs_cost& k = c->cost;
    if (!finite_all(k.Q, 12) || !finite_all(k.R, 3)) return SBS_ERR_INVALID_ARG;
    for (int i = 0; i < 12; ++i)
        if (k.Q[i] < 0) return SBS_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (k.R[i] < 0) return SBS_ERR_INVALID_ARG;
    if (!(k.w_fc >= 0) || !(k.mu >= 0) || !(k.rho >= 0) || !std::isfinite(k.f_nominal)) return SBS_ERR_INVALID_ARG;
    if (!(k.w_terminal >= 0) || !std::isfinite(k.w_terminal)) return SBS_ERR_INVALID_ARG;
    if (c->world_feet != 0 && c->world_feet != 1) return SBS_ERR_INVALID_ARG;
    if (c->friction_project != 0 && c->friction_project != 1) return SBS_ERR_INVALID_ARG;
    if (c->world_feet && !(m.gravity[2] < 0.0f)) return SBS_ERR_INVALID_ARG;  // the foothold rule needs g_z < 0
    // discrete step-frequency set (Naive only): distinct values, each advancing the
    // phase by less than one cycle per step
    if (c->n_freq < 0 || c->n_freq > SBS_MAX_FREQ) return SBS_ERR_INVALID_ARG;
    if (c->n_freq > 0) {
        if (c->method != SBS_NAIVE || c->adaptive || c->compare_mppi) return SBS_ERR_INVALID_ARG;
        for (int i = 0; i < c->n_freq; ++i) {
            const uint32_t f = c->freq_set[i];
            if (f < 1 || f > 10000 || (double)f * c->dt_us >= 1e9) return SBS_ERR_INVALID_ARG;
            for (int j = 0; j < i; ++j)
                if (c->freq_set[j] == f) return SBS_ERR_INVALID_ARG;
        }
    }
    // the rollout's shared memory (the distribution of every block, reference,
    // spline tables, per-warp sums) must fit one block
    const int T = c->tile ? c->tile : 128;
    if (rollout_smem_bytes(c->H, c->P, T, c->n_freq > 0 ? c->n_freq : 1) > kMaxDynamicSmem) return SBS_ERR_INVALID_ARG;
    return SBS_OK;
}

int validate_gait(const sbs_gait* g)
{
    if (!g) return SBS_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (g->offset[i] >= kPhaseOne) return SBS_ERR_INVALID_ARG;
    if (g->duty > kPhaseOne || g->phase0 >= kPhaseOne) return SBS_ERR_INVALID_ARG;
    return SBS_OK;
}

// Sizes and constants of a validated configuration (device pointers left null).
void fill_params(const sbs_config* cfg, InstParams* out)
{
    InstParams& P = *out;
    std::memset(&P, 0, sizeof(P));
    P.K = cfg->K;
    P.H = cfg->H;
    P.P = cfg->P;
    P.nt = cfg->P > 0 ? cfg->P : cfg->H;
    P.nf = 12 * P.nt;
    P.adaptive = cfg->adaptive ? 1 : 0;
    P.n_freq = cfg->n_freq;
    P.nb = cfg->n_freq > 0 ? cfg->n_freq : 1;
    for (int i = 0; i < cfg->n_freq; ++i) P.freq[i] = cfg->freq_set[i];
    P.D = P.nb * P.nf + P.adaptive;
    P.world_feet = cfg->world_feet;
    P.inv_g = cfg->world_feet ? 1.0f / -cfg->model.gravity[2] : 0.0f;
    P.friction_project = cfg->friction_project;
    P.inv_1pmu2 = 1.0f / (1.0f + cfg->cost.mu * cfg->cost.mu);
    P.method = cfg->method;
    P.Ke = cfg->method == SBS_ELITE ? cfg->elite_count : 1;
    P.T = cfg->tile ? cfg->tile : 128;
    P.ntiles = (cfg->K + P.T - 1) / P.T;
    P.ngroups = (P.ntiles + kGroup - 1) / kGroup;
    P.compare_mppi = cfg->compare_mppi ? 1 : 0;
    P.part_stride = kPartHeader + P.nf;
    P.dt_us = cfg->dt_us;
    P.q_init = cfg->q_init;
    P.seed = cfg->seed;
    P.ctrl = cfg->controller_id;
    P.dt = (float)(cfg->dt_us * 1e-6);
    P.lambda = cfg->lambda;
    P.inv_lambda = 1.0f / cfg->lambda;
    P.inv_mass = 1.0f / cfg->model.mass;
    P.weight_z = cfg->model.mass * -cfg->model.gravity[2];
    for (int a = 0; a < 3; ++a) {
        const double I0 = cfg->model.inertia[a], I1 = cfg->model.inertia[(a + 1) % 3],
                     I2 = cfg->model.inertia[(a + 2) % 3];
        P.gyro[a] = (float)((I1 - I2) / I0);
        P.inv_inertia[a] = 1.0f / cfg->model.inertia[a];
        P.gravity[a] = cfg->model.gravity[a];
        P.R[a] = cfg->cost.R[a];
    }
    std::memcpy(P.foot, &cfg->model.foot[0][0], sizeof(P.foot));
    std::memcpy(P.Q, cfg->cost.Q, sizeof(P.Q));
    P.w_fc = cfg->cost.w_fc;
    P.mu = cfg->cost.mu;
    P.rho = cfg->cost.rho;
    P.f_nominal = cfg->cost.f_nominal;
    P.w_terminal = cfg->cost.w_terminal;
    P.f_min = cfg->f_min;
    P.f_max = cfg->f_max;
    P.var_init = cfg->sigma_init * cfg->sigma_init;
    P.var_min = cfg->sigma_min * cfg->sigma_min;
    P.var_f_init = cfg->sigma_f_init * cfg->sigma_f_init;
    P.var_f_min = cfg->sigma_f_min * cfg->sigma_f_min;
}

}  // namespace sbs

namespace {

// ---------------------------------------------------------------- natural cubic spline (Sec. IV-B)
// Knots at t_p = p T / (P - 1), T = (H - 1) dt.  The second derivatives M solve
// the natural-spline system; here the system is assembled in full (end rows
// M_0 = M_{P-1} = 0) and solved for the P x P matrix X with M = X y by Gaussian
// elimination with partial pivoting.
struct Spline {
    int P;
    double h;
    std::vector<double> tk, X;  // X: P x P

    Spline(int H, int P_, double dt) : P(P_), tk(P_), X((size_t)P_ * P_, 0.0)
    {
        const double T = (H - 1) * dt;
        h = T / (P - 1);
        for (int p = 0; p < P; ++p) tk[p] = T * p / (P - 1);
        std::vector<double> A((size_t)P * P, 0.0), Rhs((size_t)P * P, 0.0);
        A[0] = 1.0;
        A[(size_t)(P - 1) * P + P - 1] = 1.0;
        for (int i = 1; i < P - 1; ++i) {
            A[(size_t)i * P + i - 1] = h;
            A[(size_t)i * P + i] = 4.0 * h;
            A[(size_t)i * P + i + 1] = h;
            Rhs[(size_t)i * P + i - 1] = 6.0 / h;
            Rhs[(size_t)i * P + i] = -12.0 / h;
            Rhs[(size_t)i * P + i + 1] = 6.0 / h;
        }
        // solve A X = Rhs
        for (int col = 0; col < P; ++col) {
            int piv = col;
            for (int r = col + 1; r < P; ++r)
                if (std::fabs(A[(size_t)r * P + col]) > std::fabs(A[(size_t)piv * P + col])) piv = r;
            if (piv != col)
                for (int c = 0; c < P; ++c) {
                    std::swap(A[(size_t)piv * P + c], A[(size_t)col * P + c]);
                    std::swap(Rhs[(size_t)piv * P + c], Rhs[(size_t)col * P + c]);
                }
            for (int r = 0; r < P; ++r) {
                if (r == col) continue;
                const double f = A[(size_t)r * P + col] / A[(size_t)col * P + col];
                if (f == 0.0) continue;
                for (int c = 0; c < P; ++c) {
                    A[(size_t)r * P + c] -= f * A[(size_t)col * P + c];
                    Rhs[(size_t)r * P + c] -= f * Rhs[(size_t)col * P + c];
                }
            }
        }
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) X[(size_t)r * P + c] = Rhs[(size_t)r * P + c] / A[(size_t)r * P + r];
    }

    // weight of knot value y_p in the spline's value at time t (clamped to [0, T])
    double weight(double t, int p) const
    {
        t = std::min(std::max(t, tk[0]), tk[P - 1]);
        int s = (int)std::floor((t - tk[0]) / h);
        s = std::min(std::max(s, 0), P - 2);
        const double a = tk[s + 1] - t, b = t - tk[s];
        const double Ms = X[(size_t)s * P + p], Ms1 = X[(size_t)(s + 1) * P + p];
        const double ys = (p == s) ? 1.0 : 0.0, ys1 = (p == s + 1) ? 1.0 : 0.0;
        return Ms * a * a * a / (6.0 * h) + Ms1 * b * b * b / (6.0 * h) + (ys / h - Ms * h / 6.0) * a +
               (ys1 / h - Ms1 * h / 6.0) * b;
    }
};

// ---------------------------------------------------------------- allocation
void* dev_alloc(const sbs_allocator* a, bool has, size_t bytes)
{
    if (has) return a->alloc(bytes, a->ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(const sbs_allocator* a, bool has, void* p)
{
    if (!p) return;
    if (has) a->free(p, a->ctx);
    else cudaFree(p);
}

TickArgs make_tick(const sbs_handle* h, const sbs_gait& g)
{
    TickArgs t;
    std::memset(&t, 0, sizeof(t));
    for (int i = 0; i < 4; ++i) t.offset[i] = g.offset[i];
    t.duty = g.duty;
    t.phase0 = g.phase0;
    t.src = h->cur;
    t.iter = h->iter;
    return t;
}

}  // namespace

// =====================================================================================
extern "C" {

const char* sbs_status_str(int s)
{
    switch (s) {
        case SBS_OK: return "ok";
        case SBS_PENDING: return "pending";
        case SBS_ERR_INVALID_ARG: return "invalid argument";
        case SBS_ERR_OOM: return "out of device memory";
        case SBS_ERR_BUDGET: return "over the device-memory budget";
        case SBS_ERR_CUDA: return "CUDA error";
        case SBS_ERR_TIMEOUT: return "timed out";
        case SBS_ERR_DIVERGED: return "no finite cost (diverged)";
        default: return "unknown status";
    }
}

int sbs_create(const sbs_config* cfg, const sbs_allocator* alloc, sbs_handle** out)
{
    if (!out) return SBS_ERR_INVALID_ARG;
    *out = nullptr;
    int st = validate_config(cfg);
    if (st) return st;
    if (alloc && (!alloc->alloc || !alloc->free)) return SBS_ERR_INVALID_ARG;
    static std::atomic<uint64_t> next_uid{1};
    sbs_handle* h = new (std::nothrow) sbs_handle();
    if (!h) return SBS_ERR_OOM;
    h->uid = next_uid.fetch_add(1);
    h->cfg = *cfg;
    h->has_alloc = alloc != nullptr;
    if (alloc) h->alloc = *alloc;
    cudaGetDevice(&h->device);

    InstParams& P = h->hP;
    fill_params(cfg, &P);

    // device layout (256-byte aligned pieces)
    h->wsl = ws_layout(P.K, P.H, P.P, P.T, P.Ke, P.method == SBS_ELITE && P.K > kSelectSmemMaxK,
                       P.method == SBS_NAIVE ? P.nb : 0);
    const size_t D = P.D;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_params = take(sizeof(InstParams));
    const size_t o_state0 = take(2 * D * sizeof(float));
    const size_t o_state1 = take(2 * D * sizeof(float));
    const size_t o_mppi = take(D * sizeof(float));
    const size_t o_B = take(P.P > 0 ? (size_t)P.H * P.P * sizeof(float) : 0);
    const size_t o_S = take(P.P > 0 ? (size_t)P.P * P.P * sizeof(float) : 0);
    const size_t o_res = take(sizeof(sbs_result));
    const size_t in_floats = 24 + 12 * (size_t)P.H;  // x0 | f_ext | pad | feet | xref
    const size_t o_in = take(in_floats * sizeof(float));
    h->dev_bytes = off;
    h->dev_base = (char*)dev_alloc(&h->alloc, h->has_alloc, off);
    if (!h->dev_base) {
        delete h;
        return SBS_ERR_OOM;
    }
    char* b = h->dev_base;
    h->dP = (InstParams*)(b + o_params);
    P.state[0] = (float*)(b + o_state0);
    P.state[1] = (float*)(b + o_state1);
    P.mppi_mean = (float*)(b + o_mppi);
    P.Bsp = P.P > 0 ? (const float*)(b + o_B) : nullptr;
    P.Ssp = P.P > 0 ? (const float*)(b + o_S) : nullptr;
    h->res_dev = (sbs_result*)(b + o_res);
    h->dev_in = (float*)(b + o_in);

    cudaError_t e = cudaMemset(b, 0, off);
    if (e == cudaSuccess && P.P > 0) {
        // spline basis B[j][p] = weight of knot p at t_j, and the one-step shift map
        // S[p][r] = weight of knot r at t_p + dt (held at the horizon end)
        Spline sp(P.H, P.P, cfg->dt_us * 1e-6);
        std::vector<float> B((size_t)P.H * P.P), S((size_t)P.P * P.P);
        const double dt = cfg->dt_us * 1e-6;
        for (int j = 0; j < P.H; ++j)
            for (int p = 0; p < P.P; ++p) B[(size_t)j * P.P + p] = (float)sp.weight(j * dt, p);
        for (int p = 0; p < P.P; ++p)
            for (int r = 0; r < P.P; ++r) S[(size_t)p * P.P + r] = (float)sp.weight(sp.tk[p] + dt, r);
        e = cudaMemcpy((void*)P.Bsp, B.data(), B.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((void*)P.Ssp, S.data(), S.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->dP, &P, sizeof(P), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&h->pin_in, in_floats * sizeof(float), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags((cudaEvent_t*)&h->in_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->pin_in) cudaFreeHost(h->pin_in);
        dev_free(&h->alloc, h->has_alloc, h->dev_base);
        delete h;
        return SBS_ERR_CUDA;
    }
    h->cur = 0;
    h->iter = 0;
    h->initialized = false;
    *out = h;
    return SBS_OK;
}

void sbs_destroy(sbs_handle* h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->in_done) cudaEventDestroy((cudaEvent_t)h->in_done);
    dev_free(&h->alloc, h->has_alloc, h->ws_base);
    if (h->pin_in) cudaFreeHost(h->pin_in);
    dev_free(&h->alloc, h->has_alloc, h->dev_base);
    delete h;
}

int sbs_dim(const sbs_handle* h) { return h ? h->hP.D : SBS_ERR_INVALID_ARG; }

size_t sbs_device_bytes(const sbs_handle* h) { return h ? h->dev_bytes : 0; }

size_t sbs_workspace_bytes(const sbs_handle* h) { return h ? h->wsl.bytes : 0; }

size_t sbs_workspace_bytes_mode(const sbs_handle* h, int theta_mode)
{
    return h ? ws_bytes(h->wsl, theta_mode == SBS_THETA_REGENERATE) : 0;
}

int sbs_reset(sbs_handle* h, const sbs_gait* gait, uint64_t iter, void* stream)
{
    if (!h) return SBS_ERR_INVALID_ARG;
    int st = validate_gait(gait);
    if (st) return st;
    h->iter = iter;
    TickArgs t = make_tick(h, *gait);
    st = launch_init(h->dP, h->hP, t, stream);
    if (st) return st;
    h->initialized = true;
    return SBS_OK;
}

// The handle's own workspace, allocated (zeroed) on its first plain solve.
static int ensure_workspace(sbs_handle* h)
{
    if (h->ws_base) return SBS_OK;
    const size_t cnt = align_up((size_t)h->wsl.counters * sizeof(unsigned), 256);
    char* b = (char*)dev_alloc(&h->alloc, h->has_alloc, cnt + h->wsl.bytes);
    if (!b) return SBS_ERR_OOM;
    if (cudaMemset(b, 0, cnt) != cudaSuccess) {
        dev_free(&h->alloc, h->has_alloc, b);
        return SBS_ERR_CUDA;
    }
    h->ws_base = b;
    h->ws = ws_at(h->wsl, b + cnt, (unsigned*)b);
    h->dev_bytes += cnt + h->wsl.bytes;
    return SBS_OK;
}

int sbs_prepare(sbs_handle* h) { return h ? ensure_workspace(h) : SBS_ERR_INVALID_ARG; }

int sbs_solve(sbs_handle* h, const sbs_problem* prob, sbs_result* result, void* stream)
{
    if (!h || !prob || !result || !prob->x0 || !prob->xref || h->shard_pending) return SBS_ERR_INVALID_ARG;
    if (h->hP.world_feet && !prob->feet) return SBS_ERR_INVALID_ARG;
    int st = validate_gait(&prob->gait);
    if (st) return st;
    const InstParams& P = h->hP;
    if (prob->shift < 0) return SBS_ERR_INVALID_ARG;
    if (P.P > 0 && prob->shift > 1) return SBS_ERR_INVALID_ARG;
    st = ensure_workspace(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const float *x0 = prob->x0, *xref = prob->xref, *fext = prob->f_ext, *feet = prob->feet;
    sbs_result* res = result;
    if (prob->host_memory) {
        if (!finite_all(x0, 12) || !finite_all(xref, 12 * P.H) || (fext && !finite_all(fext, 3)) ||
            (P.world_feet && !finite_all(feet, 8)))
            return SBS_ERR_INVALID_ARG;
        if (h->in_pending && cudaEventSynchronize((cudaEvent_t)h->in_done) != cudaSuccess) return SBS_ERR_CUDA;
        std::memcpy(h->pin_in, x0, 12 * sizeof(float));
        if (fext) std::memcpy(h->pin_in + 12, fext, 3 * sizeof(float));
        else std::memset(h->pin_in + 12, 0, 3 * sizeof(float));
        h->pin_in[15] = 0.0f;
        if (P.world_feet) std::memcpy(h->pin_in + 16, feet, 8 * sizeof(float));
        else std::memset(h->pin_in + 16, 0, 8 * sizeof(float));
        std::memcpy(h->pin_in + 24, xref, 12 * (size_t)P.H * sizeof(float));
        if (cudaMemcpyAsync(h->dev_in, h->pin_in, (24 + 12 * (size_t)P.H) * sizeof(float), cudaMemcpyHostToDevice,
                            s) != cudaSuccess)
            return SBS_ERR_CUDA;
        if (cudaEventRecord((cudaEvent_t)h->in_done, s) != cudaSuccess) return SBS_ERR_CUDA;
        h->in_pending = true;
        x0 = h->dev_in;
        fext = h->dev_in + 12;
        feet = P.world_feet ? h->dev_in + 16 : nullptr;
        xref = h->dev_in + 24;
        res = h->res_dev;
    }
    int shift = prob->shift;
    if (!h->initialized) {
        TickArgs t0 = make_tick(h, prob->gait);
        st = launch_init(h->dP, P, t0, stream);
        if (st) return st;
        h->initialized = true;
        shift = 0;
    }
    for (int it = 0; it < h->cfg.iterations; ++it) {
        TickArgs t = make_tick(h, prob->gait);
        t.x0 = x0;
        t.xref = xref;
        t.fext = fext;
        t.feet = feet;
        t.shift = it == 0 ? shift : 0;
        t.partials = (P.method == SBS_MPPI || (P.compare_mppi && it == 0)) ? 1 : 0;
        t.mppi_to_state = P.method == SBS_MPPI ? 1 : 0;
        t.regen = h->regen;
        t.result = res;
        t.ws = h->ws;
        st = launch_rollout(h->dP, P, t, stream, h->spt > 0 ? h->spt : 1);
        if (st) return st;
        if (P.method != SBS_MPPI) {
            st = launch_select(h->dP, P, t, stream);
            if (st) return st;
            st = launch_refit(h->dP, P, t, stream);
            if (st) return st;
        }
        h->cur ^= 1;
        h->iter += 1;
    }
    if (prob->host_memory) {
        if (cudaMemcpyAsync(result, h->res_dev, sizeof(sbs_result), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SBS_ERR_CUDA;
    }
    return SBS_OK;
}

// ---- sample sharding of one controller over ranks (one GPU each) -----------------
// Exchange buffer, 32-bit words: costs [K] at 0, quantised frequencies [K] at Kp,
// MPPI tile rows [ntiles][part_stride] at 2 Kp (Kp = K rounded up to 64 words).
static size_t shard_costs_stride(const sbs_handle* h) { return align_up((size_t)h->hP.K, 64); }

size_t sbs_shard_exchange_bytes(const sbs_handle* h)
{
    if (!h) return 0;
    return 4 * (2 * shard_costs_stride(h) + (size_t)h->hP.ntiles * h->hP.part_stride);
}

int sbs_shard_range(int ntiles, int rank, int world, int* begin, int* end)
{
    if (ntiles < 0 || world < 1 || rank < 0 || rank >= world || !begin || !end) return SBS_ERR_INVALID_ARG;
    *begin = (int)((int64_t)ntiles * rank / world);
    *end = (int)((int64_t)ntiles * (rank + 1) / world);
    return SBS_OK;
}

int sbs_shard_tiles(const sbs_handle* h) { return h ? h->hP.ntiles : SBS_ERR_INVALID_ARG; }

int sbs_shard_rollout(sbs_handle* h, const sbs_problem* prob, int rank, int world, void* xbuf, void* stream)
{
    if (!h || !prob || !prob->x0 || !prob->xref || !xbuf || prob->host_memory) return SBS_ERR_INVALID_ARG;
    if (((uintptr_t)xbuf & 15) != 0 || h->shard_pending) return SBS_ERR_INVALID_ARG;
    if (h->hP.world_feet && !prob->feet) return SBS_ERR_INVALID_ARG;
    const InstParams& P = h->hP;
    int begin = 0, end = 0;
    int st = sbs_shard_range(P.ntiles, rank, world, &begin, &end);
    if (st) return st;
    st = validate_gait(&prob->gait);
    if (st) return st;
    if (prob->shift < 0 || (P.P > 0 && prob->shift > 1)) return SBS_ERR_INVALID_ARG;
    st = ensure_workspace(h);
    if (st) return st;
    int shift = prob->shift;
    if (!h->initialized) {
        TickArgs t0 = make_tick(h, prob->gait);
        st = launch_init(h->dP, P, t0, stream);
        if (st) return st;
        h->initialized = true;
        shift = 0;
    }
    TickArgs t = make_tick(h, prob->gait);
    t.x0 = prob->x0;
    t.xref = prob->xref;
    t.fext = prob->f_ext;
    t.feet = prob->feet;
    const bool first = h->shard_it == 0;
    t.shift = first ? shift : 0;
    t.partials = (P.method == SBS_MPPI || (P.compare_mppi && first)) ? 2 : 0;
    t.mppi_to_state = P.method == SBS_MPPI ? 1 : 0;
    t.regen = 1;  // no rank holds another rank's deviations: the refit regenerates them
    t.tile_base = begin;
    t.result = nullptr;
    t.ws = h->ws;
    const size_t Kp = shard_costs_stride(h);
    t.ws.J = (float*)xbuf;
    t.ws.q = (int32_t*)xbuf + Kp;
    t.ws.part = (float*)xbuf + 2 * Kp;
    t.ws.hist = nullptr;  // built from the assembled costs by the update
    t.ws.best = nullptr;
    t.ws.nfin = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(xbuf, 0, sbs_shard_exchange_bytes(h), s) != cudaSuccess) return SBS_ERR_CUDA;
    st = launch_rollout(h->dP, P, t, stream, h->spt > 0 ? h->spt : 1, end - begin);
    if (st) return st;
    h->shard_t = t;
    h->shard_pending = true;
    return SBS_OK;
}

int sbs_shard_update(sbs_handle* h, const void* xbuf, sbs_result* result, void* stream)
{
    if (!h || !xbuf || !result || !h->shard_pending) return SBS_ERR_INVALID_ARG;
    const InstParams& P = h->hP;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t Kp = shard_costs_stride(h);
    const float* x = (const float*)xbuf;
    TickArgs t = h->shard_t;
    t.ws = h->ws;
    t.result = result;
    if (cudaMemcpyAsync(t.ws.J, x, (size_t)P.K * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(t.ws.q, x + Kp, (size_t)P.K * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SBS_ERR_CUDA;
    int st;
    if (t.partials) {
        if (cudaMemcpyAsync(t.ws.part, x + 2 * Kp, (size_t)P.ntiles * P.part_stride * 4, cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return SBS_ERR_CUDA;
        st = launch_shard_finish(h->dP, P, t, stream);
        if (st) return st;
    }
    if (P.method != SBS_MPPI) {
        st = launch_cost_keys(h->dP, P, t, stream);
        if (st) return st;
        st = launch_select(h->dP, P, t, stream);
        if (st) return st;
        st = launch_refit(h->dP, P, t, stream);
        if (st) return st;
    }
    h->shard_pending = false;
    h->shard_it = (h->shard_it + 1) % h->cfg.iterations;
    h->cur ^= 1;
    h->iter += 1;
    return SBS_OK;
}

int sbs_read(const sbs_handle* h, int which, void* dst, size_t bytes, int host_dst, void* stream)
{
    if (!h || !dst) return SBS_ERR_INVALID_ARG;
    const InstParams& P = h->hP;
    const void* src = nullptr;
    size_t n = 0;
    switch (which) {
        case SBS_BUF_MEAN: src = P.state[h->cur]; n = P.D * sizeof(float); break;
        case SBS_BUF_VAR: src = P.state[h->cur] + P.D; n = P.D * sizeof(float); break;
        case SBS_BUF_COST: src = h->ws.J; n = (size_t)P.K * sizeof(float); break;
        case SBS_BUF_FREQ: src = h->ws.q; n = (size_t)P.K * sizeof(int32_t); break;
        case SBS_BUF_ELITE:
            src = h->ws.elite;
            n = (size_t)(P.method == SBS_NAIVE ? P.nb + 1 : P.Ke) * sizeof(int32_t);
            break;
        case SBS_BUF_MPPI_MEAN: src = P.mppi_mean; n = P.D * sizeof(float); break;
        default: return SBS_ERR_INVALID_ARG;
    }
    if (bytes != n) return SBS_ERR_INVALID_ARG;
    if ((which == SBS_BUF_COST || which == SBS_BUF_FREQ || which == SBS_BUF_ELITE) && !h->ws_base)
        return SBS_ERR_INVALID_ARG;  // no plain solve yet
    cudaError_t e = cudaMemcpyAsync(dst, src, n, host_dst ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? SBS_OK : SBS_ERR_CUDA;
}

size_t sbs_state_size(const sbs_handle* h)
{
    return h ? 32 + 2 * (size_t)h->hP.D * sizeof(float) : 0;
}

int sbs_get_state(const sbs_handle* h, void* buf, size_t bytes, void* stream)
{
    if (!h || !buf || bytes != sbs_state_size(h)) return SBS_ERR_INVALID_ARG;
    uint32_t* w = (uint32_t*)buf;
    std::memset(buf, 0, 32);
    w[0] = kStateMagic;
    w[1] = (uint32_t)h->hP.D;
    w[2] = (uint32_t)h->iter;
    w[3] = (uint32_t)(h->iter >> 32);
    w[4] = h->initialized ? 1u : 0u;
    if (h->initialized) {
        cudaStream_t s = (cudaStream_t)stream;
        if (cudaMemcpyAsync((char*)buf + 32, h->hP.state[h->cur], 2 * h->hP.D * sizeof(float), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return SBS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SBS_ERR_CUDA;
    }
    return SBS_OK;
}

int sbs_set_state(sbs_handle* h, const void* buf, size_t bytes, void* stream)
{
    if (!h || !buf || bytes != sbs_state_size(h)) return SBS_ERR_INVALID_ARG;
    const uint32_t* w = (const uint32_t*)buf;
    if (w[0] != kStateMagic || w[1] != (uint32_t)h->hP.D) return SBS_ERR_INVALID_ARG;
    const uint64_t iter = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
    const bool init = w[4] != 0;
    if (init) {
        const float* f = (const float*)((const char*)buf + 32);
        if (!finite_all(f, 2 * h->hP.D)) return SBS_ERR_INVALID_ARG;
        cudaStream_t s = (cudaStream_t)stream;
        if (cudaMemcpyAsync(h->hP.state[h->cur], f, 2 * h->hP.D * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return SBS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SBS_ERR_CUDA;
    }
    h->iter = iter;
    h->initialized = init;
    return SBS_OK;
}

int sbs_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return SBS_ERR_INVALID_ARG;
    return launch_philox(ctr, key, out, n, stream);
}

int sbs_normals(uint32_t seed, uint32_t ctrl, uint64_t iter, int k0, int nk, int nn, float* out, void* stream)
{
    if (k0 < 0 || nk < 0 || nn < 0 || (nk > 0 && !out)) return SBS_ERR_INVALID_ARG;
    return launch_normals(seed, ctrl, iter, k0, nk, nn, out, stream);
}

int sbs_sqrt_hw(const float* x, float* y, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return SBS_ERR_INVALID_ARG;
    return launch_sqrt_hw(x, y, n, stream);
}

int sbs_sincos(const float* x, float* out, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !out))) return SBS_ERR_INVALID_ARG;
    return launch_sincos(x, out, n, stream);
}

int sbs_fp32_peak(double* flops, void* stream)
{
    if (!flops) return SBS_ERR_INVALID_ARG;
    int dev, sms;
    if (cudaGetDevice(&dev) != cudaSuccess) return SBS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SBS_ERR_CUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return SBS_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256, blocks = sms * 8, iters = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int st = launch_fma_peak(out, 64, blocks, threads, stream);
    float best = 1e30f;
    for (int rep = 0; rep < 5 && st == SBS_OK; ++rep) {
        cudaEventRecord(a, s);
        st = launch_fma_peak(out, iters, blocks, threads, stream);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (st) return st;
    *flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * blocks / (best * 1e-3);
    return SBS_OK;
}

// =====================================================================================
// Batched ticks
// =====================================================================================
struct sbs_batch_slot {
    char* pin;            // [counts (kBatchHeader bytes) | records]
    char* dev;            // device mirror
    int* heads;           // device queue heads (4)
    char* arena;          // workspace arena of this slot's ticks
    unsigned* counters;   // counter arena (zero while idle)
    cudaEvent_t done;
    cudaEvent_t copied;   // the records are on the device (replayed ticks copy them on the batch's copy stream)
    bool used;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t kernel_node[4];  // rollout, select, refit, MPPI rollout
    cudaKernelNodeParams kparams[4];
    size_t key_smem, key_sel;
    int key_T, key_var, key_mode;
    bool key_split;
    int grids[4];
};

// What a batched tick needs that depends on its controllers alone (not on their
// problems or state): checked and computed when the list of controllers differs
// from the last call's, reused otherwise.
struct sbs_batch_plan {
    std::vector<const sbs_handle*> h;
    std::vector<uint64_t> uid;
    std::vector<int> order;  // heavier tiles first
    size_t smem = 0, smem_pair = 0, sel_smem = 0, arena = 0, arena_regen = 0;
    long long counters = 0;
    bool ext = false;
    bool adapt = false;  // some controller samples its step frequency
};

struct sbs_batch {
    int max_inst;
    size_t arena_bytes;
    int counter_words;
    sbs_allocator alloc;
    bool has_alloc;
    size_t bytes;
    int nslots;
    sbs_batch_slot slot[8];
    int next;
    bool use_graph;
    int mode;
    bool profiling;
    cudaEvent_t ev[4];
    bool ev_valid;
    cudaStream_t cstream;  // records copies of replayed ticks, ahead of the tick before
    sbs_batch_plan plan;
    int spt;               // samples per thread of the rollout: 0 (default: one) , 1 or 2
    int regen;             // 1: the sampled deviations are regenerated by their readers, not stored
    // host-memory ticks (sbs_batch_solve_host): pinned staging of every
    // controller's inputs and results, and their device copies
    char* h_in = nullptr;
    char* d_in = nullptr;
    size_t in_cap = 0;
    sbs_result* h_res = nullptr;
    sbs_result* d_res = nullptr;
    int res_cap = 0;
    std::vector<sbs_problem> dprobs;
};

extern "C" int sbs_batch_create(int max_instances, int inflight, size_t workspace_bytes, const sbs_allocator* alloc,
                                sbs_batch** out)
{
    if (!out || max_instances < 1 || inflight < 1 || inflight > 8 || workspace_bytes < 256 * (size_t)inflight)
        return SBS_ERR_INVALID_ARG;
    *out = nullptr;
    sbs_batch* b = new (std::nothrow) sbs_batch();
    if (!b) return SBS_ERR_OOM;
    b->max_inst = max_instances;
    b->nslots = inflight;
    b->arena_bytes = workspace_bytes / inflight / 256 * 256;
    // zero-when-idle words: per controller its completion counters and, for Naive,
    // its best keys (at most 2 SBS_MAX_FREQ + 2 words); large selections add a histogram
    b->counter_words = 24 * max_instances + (int)std::min<size_t>(b->arena_bytes / 8192, 1 << 24) + 1024;
    b->has_alloc = alloc != nullptr;
    if (alloc) b->alloc = *alloc;
    b->bytes = kBatchHeader + (size_t)max_instances * sizeof(InstRec);
    b->mode = SBS_BATCH_GRID;
    const char* ng = std::getenv("SBS_NO_GRAPH");
    b->use_graph = !(ng && ng[0] == '1');
    if (cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return SBS_ERR_CUDA;
    }
    for (int i = 0; i < b->nslots; ++i) {
        sbs_batch_slot& sl = b->slot[i];
        sl.key_mode = -1;
        const size_t rec_bytes = align_up(b->bytes, 256);
        const size_t cnt_bytes = align_up((size_t)b->counter_words * 4, 256);
        const size_t total = rec_bytes + 256 + cnt_bytes + b->arena_bytes;
        sl.dev = (char*)dev_alloc(&b->alloc, b->has_alloc, total);
        if (!sl.dev || cudaHostAlloc((void**)&sl.pin, b->bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            sbs_batch_destroy(b);
            return SBS_ERR_OOM;
        }
        sl.heads = (int*)(sl.dev + rec_bytes);
        sl.counters = (unsigned*)(sl.dev + rec_bytes + 256);
        sl.arena = sl.dev + rec_bytes + 256 + cnt_bytes;
        if (cudaMemset(sl.dev, 0, rec_bytes + 256 + cnt_bytes) != cudaSuccess) {
            sbs_batch_destroy(b);
            return SBS_ERR_CUDA;
        }
    }
    *out = b;
    return SBS_OK;
}

extern "C" int sbs_batch_set_mode(sbs_batch* b, int mode)
{
    if (!b || (mode != SBS_BATCH_GRID && mode != SBS_BATCH_PERSISTENT)) return SBS_ERR_INVALID_ARG;
    b->mode = mode;
    return SBS_OK;
}

extern "C" int sbs_batch_get_mode(const sbs_batch* b) { return b ? b->mode : SBS_ERR_INVALID_ARG; }

extern "C" int sbs_batch_set_profiling(sbs_batch* b, int on)
{
    if (!b) return SBS_ERR_INVALID_ARG;
    if (on && !b->ev[0]) {
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&b->ev[i]) != cudaSuccess) return SBS_ERR_CUDA;
    }
    b->profiling = on != 0;
    b->ev_valid = false;
    return SBS_OK;
}

extern "C" int sbs_batch_stage_ms(sbs_batch* b, float ms[3])
{
    if (!b || !ms || !b->ev_valid) return SBS_ERR_INVALID_ARG;
    if (cudaEventSynchronize(b->ev[3]) != cudaSuccess) return SBS_ERR_CUDA;
    for (int i = 0; i < 3; ++i)
        if (cudaEventElapsedTime(&ms[i], b->ev[i], b->ev[i + 1]) != cudaSuccess) return SBS_ERR_CUDA;
    return SBS_OK;
}

extern "C" void sbs_batch_destroy(sbs_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (int i = 0; i < 4; ++i)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    for (int i = 0; i < 8; ++i) {
        sbs_batch_slot& sl = b->slot[i];
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.copied) cudaEventDestroy(sl.copied);
        if (sl.pin) cudaFreeHost(sl.pin);
        dev_free(&b->alloc, b->has_alloc, sl.dev);
    }
    if (b->h_in) cudaFreeHost(b->h_in);
    if (b->h_res) cudaFreeHost(b->h_res);
    dev_free(&b->alloc, b->has_alloc, b->d_in);
    dev_free(&b->alloc, b->has_alloc, b->d_res);
    if (b->cstream) cudaStreamDestroy(b->cstream);
    delete b;
}

// The tick graph of a slot: queue-head reset -> rollout -> select -> refit (the records
// reach the device before the launch, on the batch's copy stream).  A split tick (grid mode, elite or Naive controllers and MPPI controllers in
// one batch) rolls out the former first, so their selection and refit run beside a
// second rollout launch over the MPPI controllers' tiles; the update chain takes
// the device's highest stream priority so that its blocks are dispatched first
// (the refit's small blocks overlap best: 0.831 -> 0.819 ms per tick of the batched
// workload, where 512- and 256-thread selection blocks lost to 1024).
static int build_graph(sbs_batch* b, sbs_batch_slot& sl, int P, int mode, size_t smem, size_t sel_smem, int T,
                       bool split)
{
    if (sl.exec) {
        cudaGraphExecDestroy(sl.exec);
        sl.exec = nullptr;
    }
    if (sl.graph) {
        cudaGraphDestroy(sl.graph);
        sl.graph = nullptr;
    }
    cudaGraph_t g;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return SBS_ERR_CUDA;
    cudaGraphNode_t n_ms;
    bool ok = true;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = sl.heads;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 4;
    mp.height = 1;
    ok = ok && cudaGraphAddMemsetNode(&n_ms, g, nullptr, 0, &mp) == cudaSuccess;
    const InstRec* recs = (const InstRec*)(sl.dev + kBatchHeader);
    const int* counts = (const int*)sl.dev;
    const int* counts_b = counts + kBatchCountsB;
    int* heads = sl.heads;
    void* args[] = {(void*)&recs, (void*)&counts, (void*)&heads};
    void* args_b[] = {(void*)&recs, (void*)&counts_b, (void*)&heads};
    const void* fns[4] = {batch_rollout_fn(P, mode), batch_select_fn(mode),
                          batch_refit_fn(mode, (P & kRegenVariant) != 0), batch_rollout_fn(P, mode)};
    const int threads[4] = {T, mode == SBS_BATCH_GRID ? kBatchSelectThreads : kSelectThreads, kBatchRefitThreads, T};
    const size_t shm[4] = {smem, sel_smem, 0, smem};
    int least = 0, greatest = 0;
    if (split && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) ok = false;
    cudaGraphNode_t prev = n_ms;
    for (int k = 0; k < (split ? 4 : 3) && ok; ++k) {
        cudaKernelNodeParams& kp = sl.kparams[k];
        std::memset(&kp, 0, sizeof(kp));
        kp.func = (void*)fns[k];
        kp.gridDim = dim3(sl.grids[k]);
        kp.blockDim = dim3(threads[k]);
        kp.sharedMemBytes = (unsigned)shm[k];
        kp.kernelParams = k == 3 ? args_b : args;
        cudaGraphNode_t dep = k == 3 ? n_ms : prev;
        ok = cudaGraphAddKernelNode(&sl.kernel_node[k], g, &dep, 1, &kp) == cudaSuccess;
        if (ok && split && k < 3) {
            cudaKernelNodeAttrValue pv;
            std::memset(&pv, 0, sizeof(pv));
            pv.priority = greatest;
            ok = cudaGraphKernelNodeSetAttribute(sl.kernel_node[k], cudaKernelNodeAttributePriority, &pv) ==
                 cudaSuccess;
        }
        if (k < 3) prev = sl.kernel_node[k];
    }
    cudaGraphExec_t ex = nullptr;
    // the update chain's priority holds only when the graph runs its nodes' own
    // priorities; otherwise every node takes the launching stream's, and the
    // selection queues behind all of the second rollout launch's blocks
    ok = ok && cudaGraphInstantiateWithFlags(&ex, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return SBS_ERR_CUDA;
    }
    for (int k = 0; k < 4; ++k) sl.kparams[k].kernelParams = nullptr;  // args above go out of scope
    sl.graph = g;
    sl.exec = ex;
    return SBS_OK;
}

// Point a graph's kernel nodes at new grid sizes (grid mode).
static int update_graph_grids(sbs_batch_slot& sl, const int grids[4], bool split)
{
    const InstRec* recs = (const InstRec*)(sl.dev + kBatchHeader);
    const int* counts = (const int*)sl.dev;
    const int* counts_b = counts + kBatchCountsB;
    int* heads = sl.heads;
    void* args[] = {(void*)&recs, (void*)&counts, (void*)&heads};
    void* args_b[] = {(void*)&recs, (void*)&counts_b, (void*)&heads};
    for (int k = 0; k < (split ? 4 : 3); ++k) {
        if (sl.kparams[k].gridDim.x == (unsigned)grids[k]) continue;
        cudaKernelNodeParams kp = sl.kparams[k];
        kp.gridDim = dim3(grids[k]);
        kp.kernelParams = k == 3 ? args_b : args;
        if (cudaGraphExecKernelNodeSetParams(sl.exec, sl.kernel_node[k], &kp) != cudaSuccess) return SBS_ERR_CUDA;
        sl.kparams[k].gridDim = kp.gridDim;
    }
    return SBS_OK;
}

// The controllers' own checks (same tile and policy, one iteration, distinct
// handles) and the launch sizes and tile order that follow from them.
static int plan_batch(sbs_batch_plan& pl, int n, sbs_handle* const* handles)
{
    pl.h.clear();
    pl.uid.clear();
    const int T = handles[0]->hP.T, Pk = handles[0]->hP.P;
    size_t smem = 0, smem_pair = 0, sel_smem = 0, arena = 0, arena_regen = 0;
    long long counters = 0;
    bool ext = false;  // some controller uses an extended model feature
    bool adapt = false;
    for (int i = 0; i < n; ++i) {
        const sbs_handle* h = handles[i];
        if (h->hP.T != T || h->hP.P != Pk || h->cfg.iterations != 1) return SBS_ERR_INVALID_ARG;
        smem = std::max(smem, rollout_smem_bytes(h->hP.H, h->hP.P, T, h->hP.nb));
        smem_pair = std::max(smem_pair, rollout_smem_bytes(h->hP.H, h->hP.P, T, h->hP.nb, true));
        ext = ext || h->hP.n_freq > 0 || h->hP.world_feet || h->hP.friction_project;
        adapt = adapt || h->hP.adaptive;
        if (h->hP.method != SBS_MPPI) sel_smem = std::max(sel_smem, select_smem_bytes(h->hP.K));
        arena += align_up(ws_bytes(h->wsl), 256);
        arena_regen += align_up(ws_bytes(h->wsl, true), 256);
        counters += h->wsl.counters;
    }
    {
        std::vector<const sbs_handle*> u(handles, handles + n);
        std::sort(u.begin(), u.end());
        if (std::adjacent_find(u.begin(), u.end()) != u.end()) return SBS_ERR_INVALID_ARG;
    }
    // controllers with a selection and refit first (a split tick rolls them out in
    // the first launch), then heavier tiles first (longer horizon, then more tiles)
    // so the tail is short
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const InstParams &A = handles[a]->hP, &C = handles[c]->hP;
        const bool ua = A.method != SBS_MPPI, uc = C.method != SBS_MPPI;
        if (ua != uc) return ua;
        if (A.H != C.H) return A.H > C.H;
        return A.ntiles > C.ntiles;
    });
    pl.order = std::move(order);
    pl.smem = smem;
    pl.smem_pair = smem_pair;
    pl.sel_smem = sel_smem;
    pl.arena = arena;
    pl.arena_regen = arena_regen;
    pl.counters = counters;
    pl.ext = ext;
    pl.adapt = adapt;
    pl.h.assign(handles, handles + n);
    for (int i = 0; i < n; ++i) pl.uid.push_back(handles[i]->uid);
    return SBS_OK;
}

extern "C" int sbs_batch_solve(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                               sbs_result* results, void* stream)
{
    if (!b || n < 1 || n > b->max_inst || !handles || !probs || !results) return SBS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i)
        if (!handles[i]) return SBS_ERR_INVALID_ARG;
    sbs_batch_plan& pl = b->plan;
    bool same = (int)pl.h.size() == n;
    for (int i = 0; same && i < n; ++i) same = pl.h[i] == handles[i] && pl.uid[i] == handles[i]->uid;
    if (!same) {
        const int st = plan_batch(pl, n, handles);
        if (st) return st;
    }
    for (int i = 0; i < n; ++i) {
        const sbs_handle* h = handles[i];
        const sbs_problem* p = &probs[i];
        if (!p->x0 || !p->xref || p->host_memory) return SBS_ERR_INVALID_ARG;
        if (h->hP.world_feet && !p->feet) return SBS_ERR_INVALID_ARG;
        if (validate_gait(&p->gait) || p->shift < 0 || (h->hP.P > 0 && p->shift > 1)) return SBS_ERR_INVALID_ARG;
    }
    const bool regen = b->regen != 0;
    if ((regen ? pl.arena_regen : pl.arena) > b->arena_bytes || pl.counters > b->counter_words) return SBS_ERR_BUDGET;
    const int T = handles[0]->hP.T;
    const int Pk = handles[0]->hP.P;
    const std::vector<int>& order = pl.order;
    const bool ext = pl.ext;
    const bool pair = b->spt == 2 && pair_capable(Pk, ext, T) && pl.smem_pair <= kMaxDynamicSmem;
    const size_t smem = pair ? pl.smem_pair : pl.smem;
    const int RT = pair ? T / 2 : T;  // threads of a rollout block
    size_t sel_smem = pl.sel_smem;
    sbs_batch_slot& sl = b->slot[b->next];
    b->next = (b->next + 1) % b->nslots;
    if (sl.used && cudaEventSynchronize(sl.done) != cudaSuccess) return SBS_ERR_CUDA;
    // controllers solved for the first time start from their initial distribution
    for (int i = 0; i < n; ++i) {
        sbs_handle* h = handles[i];
        if (!h->initialized) {
            TickArgs t0 = make_tick(h, probs[i].gait);
            int st = launch_init(h->dP, h->hP, t0, stream);
            if (st) return st;
        }
    }
    int* counts = (int*)sl.pin;
    InstRec* recs = (InstRec*)(sl.pin + kBatchHeader);
    int tile_begin = 0, select_begin = 0, refit_begin = 0, tiles_upd = 0;
    size_t aoff = 0;
    unsigned* cnt = sl.counters;
    for (int r = 0; r < n; ++r) {
        const int i = order[r];
        sbs_handle* h = handles[i];
        const InstParams& P = h->hP;
        InstRec& R = recs[r];
        R.t = make_tick(h, probs[i].gait);  // zeroed there; every other field is written below
        R.t.x0 = probs[i].x0;
        R.t.xref = probs[i].xref;
        R.t.fext = probs[i].f_ext;
        R.t.feet = probs[i].feet;
        R.t.shift = h->initialized ? probs[i].shift : 0;
        R.t.partials = (P.method == SBS_MPPI || P.compare_mppi) ? 1 : 0;
        R.t.mppi_to_state = P.method == SBS_MPPI ? 1 : 0;
        R.t.regen = b->regen;
        R.t.result = results + i;
        R.t.ws = ws_at(h->wsl, sl.arena + aoff, cnt, regen);
        aoff += align_up(ws_bytes(h->wsl, regen), 256);
        cnt += h->wsl.counters;
        R.dP = h->dP;
        R.tile_begin = tile_begin;
        R.select_begin = select_begin;
        R.refit_begin = refit_begin;
        R.pad[0] = R.pad[1] = R.pad[2] = 0;
        tile_begin += P.ntiles;
        if (P.method != SBS_MPPI) {
            select_begin += 1;
            refit_begin += refit_items(P.method, P.Ke, P.nt, P.adaptive);
            tiles_upd = tile_begin;  // these records come first
        }
    }
    const int mode = b->mode;
    // a replayed grid-mode tick with both kinds of controllers: two rollout launches
    // (profiled ticks keep one, so that their stage times are the kernels' own)
    const bool split = mode == SBS_BATCH_GRID && b->use_graph && !b->profiling && tiles_upd > 0 &&
                       tiles_upd < tile_begin;
    counts[0] = n;
    counts[1] = split ? tiles_upd : tile_begin;
    counts[2] = select_begin;
    counts[3] = refit_begin;
    counts[4] = 0;
    counts[5] = counts[6] = counts[7] = 0;
    int* counts_b = counts + kBatchCountsB;
    counts_b[0] = n;
    counts_b[1] = tile_begin;
    counts_b[2] = select_begin;
    counts_b[3] = refit_begin;
    counts_b[4] = split ? tiles_upd : 0;
    counts_b[5] = counts_b[6] = counts_b[7] = 0;
    if (sel_smem == 0) sel_smem = 256;
    const size_t used = kBatchHeader + (size_t)n * sizeof(InstRec);
    int grids[4];
    const int var = rollout_variant(Pk, ext, pair, b->regen != 0, pl.adapt);
    int st = batch_grid(var, mode, smem, sel_smem, RT, counts, grids);
    if (st) return st;
    grids[3] = split ? tile_begin - tiles_upd : 0;
    const bool rekey = sl.key_smem != smem || sl.key_sel != sel_smem || sl.key_T != RT || sl.key_var != var ||
                       sl.key_mode != mode || sl.key_split != split;
    if (b->use_graph && !b->profiling) {
        if (!sl.exec || rekey) {
            std::memcpy(sl.grids, grids, sizeof(grids));
            st = build_graph(b, sl, var, mode, smem, sel_smem, RT, split);
            if (st) return st;
        } else if (mode == SBS_BATCH_GRID) {
            st = update_graph_grids(sl, grids, split);
            if (st) return st;
        }
        // the slot's last tick has finished (synchronised above), so its records may be
        // replaced while the tick before this one still runs
        if (cudaMemcpyAsync(sl.dev, sl.pin, used, cudaMemcpyHostToDevice, b->cstream) != cudaSuccess ||
            cudaEventRecord(sl.copied, b->cstream) != cudaSuccess || cudaStreamWaitEvent(s, sl.copied, 0) != cudaSuccess)
            return SBS_ERR_CUDA;
        if (cudaGraphLaunch(sl.exec, s) != cudaSuccess) return SBS_ERR_CUDA;
    } else {
        if (sl.exec && rekey) {  // the graph's launch shapes no longer match
            cudaGraphExecDestroy(sl.exec);
            sl.exec = nullptr;
        }
        if (cudaMemcpyAsync(sl.dev, sl.pin, used, cudaMemcpyHostToDevice, s) != cudaSuccess) return SBS_ERR_CUDA;
        if (cudaMemsetAsync(sl.heads, 0, 16, s) != cudaSuccess) return SBS_ERR_CUDA;
        st = launch_batch(var, mode, (const InstRec*)(sl.dev + kBatchHeader), (const int*)sl.dev, sl.heads, smem,
                          sel_smem, RT, grids, stream, b->profiling ? (void* const*)b->ev : nullptr);
        if (st) return st;
        b->ev_valid = b->profiling;
    }
    sl.key_smem = smem;
    sl.key_sel = sel_smem;
    sl.key_T = RT;
    sl.key_var = var;
    sl.key_mode = mode;
    sl.key_split = split;
    if (cudaEventRecord(sl.done, s) != cudaSuccess) return SBS_ERR_CUDA;
    sl.used = true;
    for (int i = 0; i < n; ++i) {
        sbs_handle* h = handles[i];
        h->initialized = true;
        h->cur ^= 1;
        h->iter += 1;
    }
    return SBS_OK;
}

// One tick from host memory: every controller's inputs are gathered into one
// pinned buffer and copied to the device in one transfer on the caller's stream,
// the tick runs on the device copies, and the n results come back in one
// transfer; the call returns when they are in `results`.
// Bytes of the host staging of one controller's inputs (16-byte aligned pieces):
// x0 | xref | f_ext (when given) | feet (ground-fixed feet).
static size_t staged_bytes(const sbs_handle* h, bool fext)
{
    return align_up(12 * 4, 16) + align_up((size_t)12 * h->hP.H * 4, 16) + (fext ? 16 : 0) +
           (h->hP.world_feet ? 32 : 0);
}

// Waits for the batch's ticks in flight, then grows the pinned input staging (and
// its device twin) to at least `need` bytes.
static int host_staging(sbs_batch* b, size_t need)
{
    for (int k = 0; k < b->nslots; ++k)
        if (b->slot[k].used && cudaEventSynchronize(b->slot[k].done) != cudaSuccess) return SBS_ERR_CUDA;
    if (need > b->in_cap) {
        if (b->h_in) cudaFreeHost(b->h_in);
        dev_free(&b->alloc, b->has_alloc, b->d_in);
        b->h_in = nullptr;
        b->in_cap = 0;
        const size_t cap = align_up(need + need / 4, 4096);
        b->d_in = (char*)dev_alloc(&b->alloc, b->has_alloc, cap);
        if (!b->d_in || cudaHostAlloc((void**)&b->h_in, cap, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            dev_free(&b->alloc, b->has_alloc, b->d_in);
            b->d_in = nullptr;
            b->h_in = nullptr;
            return SBS_ERR_OOM;
        }
        b->in_cap = cap;
    }
    return SBS_OK;
}

extern "C" int sbs_batch_host_inputs(sbs_batch* b, int n, sbs_handle* const* handles, int with_fext,
                                     sbs_problem* probs)
{
    if (!b || n < 1 || n > b->max_inst || !handles || !probs) return SBS_ERR_INVALID_ARG;
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return SBS_ERR_INVALID_ARG;
        need += staged_bytes(handles[i], with_fext != 0);
    }
    int st = host_staging(b, need);
    if (st) return st;
    size_t off = 0;
    auto take = [&](size_t count) {
        float* p = (float*)(b->h_in + off);
        off += align_up(count * 4, 16);
        return p;
    };
    for (int i = 0; i < n; ++i) {
        sbs_problem& q = probs[i];
        q.host_memory = 1;
        q.x0 = take(12);
        q.xref = take((size_t)12 * handles[i]->hP.H);
        q.f_ext = with_fext ? take(3) : nullptr;
        q.feet = handles[i]->hP.world_feet ? take(8) : nullptr;
    }
    return SBS_OK;
}

extern "C" int sbs_batch_solve_host(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                                    sbs_result* results, void* stream)
{
    if (!b || n < 1 || n > b->max_inst || !handles || !probs || !results) return SBS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        const sbs_handle* h = handles[i];
        const sbs_problem& p = probs[i];
        if (!h || !p.x0 || !p.xref || p.host_memory != 1) return SBS_ERR_INVALID_ARG;
        if (h->hP.world_feet && !p.feet) return SBS_ERR_INVALID_ARG;
        need += staged_bytes(h, p.f_ext != nullptr);
    }
    // wait for any earlier tick of this batch before its staging is rewritten
    int st0 = host_staging(b, need);
    if (st0) return st0;
    if (n > b->res_cap) {
        if (b->h_res) cudaFreeHost(b->h_res);
        dev_free(&b->alloc, b->has_alloc, b->d_res);
        b->h_res = nullptr;
        b->res_cap = 0;
        b->d_res = (sbs_result*)dev_alloc(&b->alloc, b->has_alloc, (size_t)b->max_inst * sizeof(sbs_result));
        if (!b->d_res ||
            cudaHostAlloc((void**)&b->h_res, (size_t)b->max_inst * sizeof(sbs_result), cudaHostAllocDefault) !=
                cudaSuccess) {
            cudaGetLastError();
            dev_free(&b->alloc, b->has_alloc, b->d_res);
            b->d_res = nullptr;
            b->h_res = nullptr;
            return SBS_ERR_OOM;
        }
        b->res_cap = b->max_inst;
    }
    b->dprobs.resize(n);
    size_t off = 0;
    auto stage = [&](const float* src, size_t count) -> const float* {
        float* dst = (float*)(b->h_in + off);
        if (src != dst) std::memcpy(dst, src, count * 4);  // inputs the caller wrote in place stay
        const float* d = (const float*)(b->d_in + off);
        off += align_up(count * 4, 16);
        return d;
    };
    for (int i = 0; i < n; ++i) {
        const sbs_problem& p = probs[i];
        sbs_problem& q = b->dprobs[i];
        q = p;
        q.host_memory = 0;
        q.x0 = stage(p.x0, 12);
        q.xref = stage(p.xref, (size_t)12 * handles[i]->hP.H);
        q.f_ext = p.f_ext ? stage(p.f_ext, 3) : nullptr;
        q.feet = handles[i]->hP.world_feet ? stage(p.feet, 8) : nullptr;
    }
    if (cudaMemcpyAsync(b->d_in, b->h_in, off, cudaMemcpyHostToDevice, s) != cudaSuccess) return SBS_ERR_CUDA;
    int st = sbs_batch_solve(b, n, handles, b->dprobs.data(), b->d_res, stream);
    if (st) {
        cudaStreamSynchronize(s);
        return st;
    }
    if (cudaMemcpyAsync(b->h_res, b->d_res, (size_t)n * sizeof(sbs_result), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SBS_ERR_CUDA;
    std::memcpy(results, b->h_res, (size_t)n * sizeof(sbs_result));
    return SBS_OK;
}

extern "C" int sbs_batch_autotune(sbs_batch* b, int n, sbs_handle* const* handles, const sbs_problem* probs,
                                  sbs_result* results, int ticks, float ms_out[2], void* stream)
{
    if (!b || ticks < 1 || !ms_out || n < 1 || !handles || !handles[0]) return SBS_ERR_INVALID_ARG;
    const bool prof = b->profiling;
    int st = sbs_batch_set_profiling(b, 1);
    if (st) return st;
    // launch modes, and one or two samples per thread where the launch can take two
    bool ext = false, fits = true;
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return SBS_ERR_INVALID_ARG;
        const InstParams& Pi = handles[i]->hP;
        ext = ext || Pi.n_freq > 0 || Pi.world_feet || Pi.friction_project;
        fits = fits && pair_fits(Pi.H, Pi.P, Pi.T, Pi.nb);
    }
    const int nspt = pair_capable(handles[0]->hP.P, ext, handles[0]->hP.T) && fits ? 2 : 1;
    const int modes[2] = {SBS_BATCH_GRID, SBS_BATCH_PERSISTENT};
    float best = 1e30f;
    int best_mode = SBS_BATCH_GRID, best_spt = 1, best_regen = 0;
    for (int m = 0; m < 2 && st == SBS_OK; ++m) {
        b->mode = modes[m];
        ms_out[m] = 1e30f;
        for (int sp = 1; sp <= nspt && st == SBS_OK; ++sp) {
            for (int rg = 0; rg < 2 && st == SBS_OK; ++rg) {
                b->spt = sp;
                b->regen = rg;
                double tot = 0.0;
                bool fits = true;
                for (int k = 0; k <= ticks && st == SBS_OK; ++k) {  // the first tick of a setting is a warm-up
                    st = sbs_batch_solve(b, n, handles, probs, results, stream);
                    if (k == 0 && st == SBS_ERR_BUDGET) {  // refused before any launch: the setting's
                        st = SBS_OK;                       // workspace does not fit the arena
                        fits = false;
                        break;
                    }
                    float ms[3];
                    if (st == SBS_OK) st = sbs_batch_stage_ms(b, ms);
                    if (st == SBS_OK && k > 0) tot += (double)ms[0] + ms[1] + ms[2];
                }
                if (!fits) continue;
                const float avg = (float)(tot / ticks);
                if (st == SBS_OK && avg < ms_out[m]) ms_out[m] = avg;
                if (st == SBS_OK && avg < best) {
                    best = avg;
                    best_mode = modes[m];
                    best_spt = sp;
                    best_regen = rg;
                }
            }
        }
    }
    sbs_batch_set_profiling(b, prof ? 1 : 0);
    if (st) return st;
    if (best >= 1e30f) return SBS_ERR_BUDGET;  // no setting fits the arena
    b->mode = best_mode;
    b->spt = best_spt;
    b->regen = best_regen;
    return SBS_OK;
}

extern "C" int sbs_autotune(sbs_handle* h, const sbs_problem* prob, sbs_result* result, int ticks, float ms_out[6],
                            void* stream)
{
    if (!h || !prob || !result || ticks < 1 || !ms_out) return SBS_ERR_INVALID_ARG;
    const InstParams& P = h->hP;
    const bool ext = P.n_freq > 0 || P.world_feet || P.friction_project;
    const bool pair = pair_capable(P.P, ext, P.T) && pair_fits(P.H, P.P, P.T, P.nb);
    const bool ws = ws_capable(P.P, ext, P.H, P.T, P.nb);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return SBS_ERR_CUDA;
    }
    int st = SBS_OK, best_spt = 1, best_regen = 0;
    float best = 1e30f;
    for (int i = 0; i < 6; ++i) ms_out[i] = -1.0f;
    for (int sp = 1; sp <= 3 && st == SBS_OK; ++sp) {
        if ((sp == 2 && !pair) || (sp == SBS_SPT_NOISE_WARPS && !ws)) continue;
        for (int rg = 0; rg < 2 && st == SBS_OK; ++rg) {
            h->spt = sp;
            h->regen = rg;
            st = sbs_solve(h, prob, result, stream);  // warm-up of this setting
            if (st) break;
            if (cudaEventRecord(a, s) != cudaSuccess) st = SBS_ERR_CUDA;
            for (int k = 0; k < ticks && st == SBS_OK; ++k) st = sbs_solve(h, prob, result, stream);
            if (st == SBS_OK && (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess))
                st = SBS_ERR_CUDA;
            float ms = 0.0f;
            if (st == SBS_OK && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) st = SBS_ERR_CUDA;
            if (st) break;
            ms /= (float)ticks;
            ms_out[2 * (sp - 1) + rg] = ms;
            if (ms < best) {
                best = ms;
                best_spt = sp;
                best_regen = rg;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) {
        cudaGetLastError();
        return st;
    }
    h->spt = best_spt;
    h->regen = best_regen;
    return SBS_OK;
}

extern "C" int sbs_get_samples_per_thread(const sbs_handle* h) { return h ? (h->spt > 0 ? h->spt : 1) : SBS_ERR_INVALID_ARG; }

extern "C" int sbs_get_theta_mode(const sbs_handle* h)
{
    return h ? (h->regen ? SBS_THETA_REGENERATE : SBS_THETA_STORE) : SBS_ERR_INVALID_ARG;
}

extern "C" int sbs_batch_set_theta_mode(sbs_batch* b, int mode)
{
    if (!b || (mode != SBS_THETA_STORE && mode != SBS_THETA_REGENERATE)) return SBS_ERR_INVALID_ARG;
    b->regen = mode == SBS_THETA_REGENERATE ? 1 : 0;
    return SBS_OK;
}

extern "C" int sbs_batch_get_theta_mode(const sbs_batch* b)
{
    return b ? (b->regen ? SBS_THETA_REGENERATE : SBS_THETA_STORE) : SBS_ERR_INVALID_ARG;
}

extern "C" int sbs_set_theta_mode(sbs_handle* h, int mode)
{
    if (!h || (mode != SBS_THETA_STORE && mode != SBS_THETA_REGENERATE)) return SBS_ERR_INVALID_ARG;
    h->regen = mode == SBS_THETA_REGENERATE ? 1 : 0;
    return SBS_OK;
}

extern "C" int sbs_batch_set_samples_per_thread(sbs_batch* b, int spt)
{
    if (!b || spt < 0 || spt > 2) return SBS_ERR_INVALID_ARG;
    b->spt = spt;
    return SBS_OK;
}

extern "C" int sbs_batch_get_samples_per_thread(const sbs_batch* b) { return b ? b->spt : SBS_ERR_INVALID_ARG; }

extern "C" int sbs_set_samples_per_thread(sbs_handle* h, int spt)
{
    if (!h || spt < 0 || spt > SBS_SPT_NOISE_WARPS) return SBS_ERR_INVALID_ARG;
    h->spt = spt;
    return SBS_OK;
}

}  // extern "C"
