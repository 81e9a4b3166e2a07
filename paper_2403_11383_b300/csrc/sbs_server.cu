// Request loop with continuous batching (include/sbs.h, "serving").
//
// Callers submit solves as they arrive.  A dispatcher thread owns S tick slots,
// each with its own stream, batch context (workspace = budget / S), pinned input
// staging and result buffers.  Whenever a slot is free it admits waiting
// requests - oldest first, one per controller, while their workspaces fit the
// slot's budget share - packs their inputs into one host-to-device copy, issues
// one batched launch and copies the results back, all on the slot's stream, so
// consecutive ticks overlap on the GPU.  Finished slots are harvested by
// polling their completion events; latency runs from submission to the moment
// the dispatcher sees the tick complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "sbs_internal.h"

using namespace sbs;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kInFloats = 24 + 12 * SBS_MAX_H;  // x0 | f_ext | pad | feet | xref, per request

struct Request {
    uint64_t ticket;
    sbs_handle* h;
    sbs_gait gait;
    int32_t shift;
    bool has_fext;
    bool has_feet;
    int H;
    size_t ws;
    Clock::time_point t_submit;
    std::vector<float> in;  // 24 + 12 H floats
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    sbs_batch* batch = nullptr;
    float* pin_in = nullptr;
    float* dev_in = nullptr;
    sbs_result* pin_res = nullptr;
    sbs_result* dev_res = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
};

}  // namespace

struct sbs_server {
    sbs_server_config cfg;
    int device = 0;
    sbs_allocator alloc;
    bool has_alloc = false;
    size_t slot_budget = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, sbs_result> finished;
    std::unordered_set<uint64_t> open;  // pending or in flight
    std::unordered_set<sbs_handle*> busy_handles;
    uint64_t next_ticket = 1;
    std::thread worker;
    bool stop = false;
    int error = SBS_OK;
    // statistics
    std::vector<double> lat_us;
    uint64_t ticks = 0, completed = 0, admission_waits = 0, max_inflight = 0;
    double batch_sum = 0.0;
};

namespace {

void* srv_alloc(sbs_server* s, size_t bytes)
{
    if (s->has_alloc) return s->alloc.alloc(bytes, s->alloc.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void srv_free(sbs_server* s, void* p)
{
    if (!p) return;
    if (s->has_alloc) s->alloc.free(p, s->alloc.ctx);
    else cudaFree(p);
}

// Move the finished requests of a completed slot to the result table.
void harvest(sbs_server* s, Slot& sl)
{
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const Request& r = sl.reqs[i];
        s->finished[r.ticket] = sl.pin_res[i];
        s->open.erase(r.ticket);
        s->busy_handles.erase(r.h);
        s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
        s->completed += 1;
    }
    sl.reqs.clear();
    sl.busy = false;
}

// Admit waiting requests into a free slot.  Returns the number admitted.
size_t admit(sbs_server* s, Slot& sl)
{
    std::lock_guard<std::mutex> lock(s->mu);
    const size_t cap = s->cfg.plain ? 1 : (size_t)s->cfg.max_batch;
    size_t used = 0;
    int T = -1, P = -1;
    std::unordered_set<sbs_handle*> taken;
    for (auto it = s->pending.begin(); it != s->pending.end() && sl.reqs.size() < cap;) {
        sbs_handle* h = it->h;
        if (s->busy_handles.count(h) || taken.count(h)) {  // one solve per controller at a time, in order
            taken.insert(h);
            ++it;
            continue;
        }
        const size_t need = (it->ws + 255) / 256 * 256;
        const bool fits = s->cfg.plain || (used + need <= s->slot_budget && (T < 0 || (h->hP.T == T && h->hP.P == P)));
        if (!fits) {
            s->admission_waits += 1;
            taken.insert(h);
            ++it;
            continue;
        }
        used += need;
        T = h->hP.T;
        P = h->hP.P;
        taken.insert(h);
        s->busy_handles.insert(h);
        sl.reqs.push_back(std::move(*it));
        it = s->pending.erase(it);
    }
    return sl.reqs.size();
}

// Issue one tick of a slot: inputs in, solve, results out, completion event.
int issue(sbs_server* s, Slot& sl)
{
    const size_t n = sl.reqs.size();
    size_t off = 0;
    std::vector<size_t> offs(n);
    for (size_t i = 0; i < n; ++i) {
        const Request& r = sl.reqs[i];
        offs[i] = off;
        std::memcpy(sl.pin_in + off, r.in.data(), r.in.size() * sizeof(float));
        off += (r.in.size() + 3) / 4 * 4;  // keep each request's inputs 16-byte aligned
    }
    if (cudaMemcpyAsync(sl.dev_in, sl.pin_in, off * sizeof(float), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return SBS_ERR_CUDA;
    std::vector<sbs_handle*> hs(n);
    std::vector<sbs_problem> ps(n);
    for (size_t i = 0; i < n; ++i) {
        const Request& r = sl.reqs[i];
        const float* base = sl.dev_in + offs[i];
        sbs_problem& p = ps[i];
        std::memset(&p, 0, sizeof(p));
        p.x0 = base;
        p.f_ext = r.has_fext ? base + 12 : nullptr;
        p.feet = r.has_feet ? base + 16 : nullptr;
        p.xref = base + 24;
        p.gait = r.gait;
        p.shift = r.shift;
        p.host_memory = 0;
        hs[i] = r.h;
    }
    int st = SBS_OK;
    if (s->cfg.plain) {
        st = sbs_solve(hs[0], &ps[0], sl.dev_res, sl.stream);
    } else {
        st = sbs_batch_solve(sl.batch, (int)n, hs.data(), ps.data(), sl.dev_res, sl.stream);
    }
    if (st) return st;
    if (cudaMemcpyAsync(sl.pin_res, sl.dev_res, n * sizeof(sbs_result), cudaMemcpyDeviceToHost, sl.stream) !=
        cudaSuccess)
        return SBS_ERR_CUDA;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return SBS_ERR_CUDA;
    sl.busy = true;
    uint64_t inflight = 0;
    for (const Slot& o : s->slots) inflight += o.busy ? 1 : 0;
    std::lock_guard<std::mutex> lock(s->mu);
    s->ticks += 1;
    s->batch_sum += (double)n;
    s->max_inflight = std::max(s->max_inflight, inflight);
    return SBS_OK;
}

void dispatch_loop(sbs_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progressed = false;
        for (Slot& sl : s->slots) {
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
                harvest(s, sl);
                progressed = true;
            }
        }
        for (Slot& sl : s->slots) {
            if (sl.busy) continue;
            if (admit(s, sl) == 0) break;
            const int st = issue(s, sl);
            if (st) {
                std::lock_guard<std::mutex> lock(s->mu);
                s->error = st;
                // the admitted requests fail: report them finished with the error status
                for (Request& r : sl.reqs) {
                    sbs_result res;
                    std::memset(&res, 0, sizeof(res));
                    res.status = st;
                    s->finished[r.ticket] = res;
                    s->open.erase(r.ticket);
                    s->busy_handles.erase(r.h);
                }
                sl.reqs.clear();
                sl.busy = false;
            }
            progressed = true;
        }
        std::unique_lock<std::mutex> lock(s->mu);
        if (s->stop) break;
        if (!progressed) {
            bool any_busy = false;
            for (const Slot& sl : s->slots) any_busy = any_busy || sl.busy;
            // wake on a submission, or soon to poll the GPU for finished ticks
            s->cv.wait_for(lock, std::chrono::microseconds(any_busy ? 10 : 200));
        }
    }
    for (Slot& sl : s->slots)
        if (sl.busy) {
            cudaEventSynchronize(sl.done);
            harvest(s, sl);
        }
}

}  // namespace

extern "C" int sbs_server_create(const sbs_server_config* cfg, const sbs_allocator* alloc, sbs_server** out)
{
    if (!out || !cfg) return SBS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 8 || cfg->max_batch < 1 || cfg->max_pending < 1) return SBS_ERR_INVALID_ARG;
    if (!cfg->plain && cfg->budget_bytes < 4096) return SBS_ERR_INVALID_ARG;
    if (cfg->samples_per_thread < 0 || cfg->samples_per_thread > 2 ||
        (cfg->theta_mode != SBS_THETA_STORE && cfg->theta_mode != SBS_THETA_REGENERATE))
        return SBS_ERR_INVALID_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return SBS_ERR_INVALID_ARG;
    sbs_server* s = new (std::nothrow) sbs_server();
    if (!s) return SBS_ERR_OOM;
    s->cfg = *cfg;
    if (s->cfg.plain) s->cfg.max_batch = 1;
    s->has_alloc = alloc != nullptr;
    if (alloc) s->alloc = *alloc;
    cudaGetDevice(&s->device);
    s->slot_budget = cfg->plain ? 0 : cfg->budget_bytes / cfg->slots;
    s->slots.resize(cfg->slots);
    const int mb = s->cfg.max_batch;
    int st = SBS_OK;
    for (Slot& sl : s->slots) {
        const size_t in_bytes = (size_t)mb * kInFloats * sizeof(float);
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.pin_in, in_bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void**)&sl.pin_res, (size_t)mb * sizeof(sbs_result), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            st = SBS_ERR_CUDA;
            break;
        }
        sl.dev_in = (float*)srv_alloc(s, in_bytes);
        sl.dev_res = (sbs_result*)srv_alloc(s, (size_t)mb * sizeof(sbs_result));
        if (!sl.dev_in || !sl.dev_res) {
            st = SBS_ERR_OOM;
            break;
        }
        if (!cfg->plain) {
            st = sbs_batch_create(mb, 1, s->slot_budget, alloc, &sl.batch);
            if (st) break;
            st = sbs_batch_set_samples_per_thread(sl.batch, cfg->samples_per_thread);
            if (!st) st = sbs_batch_set_theta_mode(sl.batch, cfg->theta_mode);
            if (st) break;
        }
    }
    if (st) {
        sbs_server_destroy(s);
        return st;
    }
    s->worker = std::thread(dispatch_loop, s);
    *out = s;
    return SBS_OK;
}

extern "C" void sbs_server_destroy(sbs_server* s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();
    }
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.batch) sbs_batch_destroy(sl.batch);
        srv_free(s, sl.dev_in);
        srv_free(s, sl.dev_res);
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_res) cudaFreeHost(sl.pin_res);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete s;
}

static bool finite_n(const float* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!(p[i] - p[i] == 0.0f)) return false;
    return true;
}

extern "C" int sbs_server_submit(sbs_server* s, int n, sbs_handle* const* handles, const sbs_problem* probs,
                                 uint64_t* tickets)
{
    if (!s || n < 1 || !handles || !probs || !tickets) return SBS_ERR_INVALID_ARG;
    std::vector<Request> reqs(n);
    for (int i = 0; i < n; ++i) {
        sbs_handle* h = handles[i];
        const sbs_problem* p = &probs[i];
        if (!h || !p->x0 || !p->xref || !p->host_memory) return SBS_ERR_INVALID_ARG;
        if (validate_gait(&p->gait) || p->shift < 0 || (h->hP.P > 0 && p->shift > 1)) return SBS_ERR_INVALID_ARG;
        if (h->cfg.iterations != 1) return SBS_ERR_INVALID_ARG;
        const int H = h->hP.H;
        if (!finite_n(p->x0, 12) || !finite_n(p->xref, 12 * H) || (p->f_ext && !finite_n(p->f_ext, 3)))
            return SBS_ERR_INVALID_ARG;
        if (h->hP.world_feet && (!p->feet || !finite_n(p->feet, 8))) return SBS_ERR_INVALID_ARG;
        const size_t ws = ws_bytes(h->wsl, !s->cfg.plain && s->cfg.theta_mode == SBS_THETA_REGENERATE);
        if (!s->cfg.plain && ws + 256 > s->slot_budget) return SBS_ERR_BUDGET;
        Request& r = reqs[i];
        r.h = h;
        r.gait = p->gait;
        r.shift = p->shift;
        r.has_fext = p->f_ext != nullptr;
        r.has_feet = h->hP.world_feet != 0;
        r.H = H;
        r.ws = ws;
        r.in.assign(24 + 12 * (size_t)H, 0.0f);
        std::memcpy(r.in.data(), p->x0, 12 * sizeof(float));
        if (p->f_ext) std::memcpy(r.in.data() + 12, p->f_ext, 3 * sizeof(float));
        if (r.has_feet) std::memcpy(r.in.data() + 16, p->feet, 8 * sizeof(float));
        std::memcpy(r.in.data() + 24, p->xref, 12 * (size_t)H * sizeof(float));
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->open.size() + (size_t)n > (size_t)s->cfg.max_pending) return SBS_PENDING;
        const auto now = Clock::now();
        for (int i = 0; i < n; ++i) {
            reqs[i].ticket = s->next_ticket++;
            reqs[i].t_submit = now;
            tickets[i] = reqs[i].ticket;
            s->open.insert(reqs[i].ticket);
            s->pending.push_back(std::move(reqs[i]));
        }
    }
    s->cv.notify_one();
    return SBS_OK;
}

extern "C" int sbs_server_poll(sbs_server* s, int n, const uint64_t* tickets, sbs_result* results, int32_t* status)
{
    if (!s || n < 0 || (n > 0 && (!tickets || !results || !status))) return SBS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    for (int i = 0; i < n; ++i) {
        auto it = s->finished.find(tickets[i]);
        if (it != s->finished.end()) {
            results[i] = it->second;
            status[i] = SBS_OK;
            s->finished.erase(it);
        } else {
            status[i] = s->open.count(tickets[i]) ? SBS_PENDING : SBS_ERR_INVALID_ARG;
        }
    }
    return s->error;
}

extern "C" int sbs_server_stats_get(sbs_server* s, sbs_server_stats* out, int reset)
{
    if (!s || !out) return SBS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->ticks = s->ticks;
    out->admission_waits = s->admission_waits;
    out->max_inflight = s->max_inflight;
    out->mean_batch = s->ticks ? s->batch_sum / (double)s->ticks : 0.0;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        const size_t m = v.size();
        out->p50_us = v[m / 2];
        out->p99_us = v[std::min(m - 1, (size_t)(0.99 * (double)m))];
        out->max_us = v.back();
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_us = sum / (double)m;
    }
    if (reset) {
        s->lat_us.clear();
        s->completed = s->ticks = s->admission_waits = s->max_inflight = 0;
        s->batch_sum = 0.0;
    }
    return SBS_OK;
}
