// Continuous-batching request loop for ESDG solves (the library's served form).
//
// A worker thread owns the GPU work.  Requests arrive as built (not yet
// attached) contexts with host initial data; they wait in a FIFO queue and are
// admitted when their device footprint fits the HBM budget.  Every iteration
// advances every active request by up to kMaxChunk steps: FP32 requests that
// need at least a whole chunk go together in one ensemble launch per RK stage
// (one ensemble per volume rule), an FP32 request with fewer steps left runs
// just those on its own stage kernels in the same iteration, and FP64 requests
// run on their own streams, so their (often small) grids overlap on the GPU.
// No request waits for another to finish and none runs past its step count.
// Finished requests are retired between iterations (state copied to the
// caller's host buffer, device memory returned), which lets queued requests
// in.  All host work of a request (esdg_prepare) runs in the submitting
// thread, so admission is one host-to-device copy.  Built only on the public C
// ABI of esdg.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "esdg.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxChunk = 20;  // steps per iteration at most
// Working set: admission stops while the active requests of a precision hold
// this many unknowns per field (K Np) -- enough to keep the device busy, few
// enough that an overloaded server finishes requests in arrival order instead
// of advancing all of them slowly.  A request is always admitted when nothing
// of its precision is active.
constexpr long long kWorkingSetFP32 = 1LL << 23;
constexpr long long kWorkingSetFP64 = 1LL << 21;

struct Request {
    int ticket = 0;
    esdg_ctx* ctx = nullptr;
    int precision = ESDG_FP32;
    int rule = ESDG_RULE_COLLAPSED;
    long long dofs = 0;  // K Np: unknowns per field
    int nsteps = 0, remaining = 0;
    double dt = 0, t = 0;      // step size and the request's simulated time (forcing terms depend on it)
    double* result = nullptr;  // caller's host buffer [3][K][Np] ([3][K][Nq] for the DG-SBP method)
    size_t bytes = 0;
    void* dmem = nullptr;
    cudaStream_t stream = nullptr;  // FP64 requests: their own stream (FP32 ones share the server's)
    int state = 0;  // 0 queued, 1 active, 2 done, < 0 failed (status code)
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::string err;
};

}  // namespace

struct esdg_server {
    size_t budget = 0, in_use = 0;
    int max_active = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<int, Request*> all;
    int next_ticket = 1;
    int admitting = 0;  // popped from the queue, not yet running (lock released)
    bool stop = false;
    std::thread worker;
    esdg_ensemble* ens[2] = {nullptr, nullptr};  // FP32 ensembles, per volume rule
    std::vector<Request*> ens_members[2];
    long long iterations = 0, steps_run = 0;
    int max_active_seen = 0;  // the most requests any one iteration advanced
    // where the worker's time goes (seconds): admission (allocation and the
    // copy of each prepared image), ensemble rebuilds, enqueueing the
    // iteration's work, waiting for the GPU, retiring results
    double t_admit = 0, t_rebuild = 0, t_launch = 0, t_wait = 0, t_retire = 0;
    std::string err;
};

static double now_s(const esdg_server* s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

static void finish(esdg_server* s, Request* r, int state, const std::string& why) {
    if (r->ctx) {
        esdg_destroy(r->ctx);
        r->ctx = nullptr;
    }
    if (r->dmem) {
        cudaFreeAsync(r->dmem, r->stream ? r->stream : s->stream);
        r->dmem = nullptr;
        s->in_use -= r->bytes;
    }
    if (r->stream) {
        cudaStreamDestroy(r->stream);  // released once its work is done
        r->stream = nullptr;
    }
    r->state = state;
    r->err = why;
    r->t_done = now_s(s);
}

// Admit queued requests in FIFO order while their footprint fits.
static void admit(esdg_server* s, std::unique_lock<std::mutex>& lk) {
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
        Request* r = s->queue.front();
        if (s->in_use + r->bytes > s->budget) break;
        long long held = 0;
        for (Request* a : s->active)
            if (a->precision == r->precision) held += a->dofs;
        const long long cap = r->precision == ESDG_FP64 ? kWorkingSetFP64 : kWorkingSetFP32;
        if (held > 0 && held + r->dofs > cap) break;
        s->queue.pop_front();
        s->in_use += r->bytes;
        s->admitting += 1;
        lk.unlock();
        int rc = ESDG_OK;
        std::string why;
        cudaStream_t st = s->stream;
        if (r->precision == ESDG_FP64) {
            cudaError_t se = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking);
            if (se == cudaSuccess) st = r->stream;
            else r->stream = nullptr;
        }
        cudaError_t ce = cudaMallocAsync(&r->dmem, r->bytes + 256, st);
        if (ce != cudaSuccess) {
            rc = ESDG_ENOMEM;
            why = std::string("cudaMallocAsync: ") + cudaGetErrorString(ce);
            r->dmem = nullptr;
        }
        if (!rc) {
            char* p = static_cast<char*>(r->dmem);
            p += (256 - (reinterpret_cast<uintptr_t>(p) & 255)) & 255;
            rc = esdg_attach_device(r->ctx, p, r->bytes, st);  // one copy of the prepared image
            if (rc) why = esdg_last_error(r->ctx);
        }
        lk.lock();
        s->admitting -= 1;
        if (rc) {
            finish(s, r, rc, why);
            s->cv.notify_all();
            continue;
        }
        r->state = 1;
        r->t_admit = now_s(s);
        s->active.push_back(r);
    }
}

// Rebuild an FP32 ensemble when the set of its members changed: the active
// FP32 requests of the rule with at least `chunk` steps left.
static int refresh_ensemble(esdg_server* s, const std::vector<Request*>& act, int rule, int chunk) {
    std::vector<Request*> fp32;
    for (Request* r : act)
        if (r->precision == ESDG_FP32 && r->rule == rule && r->remaining >= chunk) fp32.push_back(r);
    if (fp32 == s->ens_members[rule] && (s->ens[rule] || fp32.empty())) return ESDG_OK;
    if (s->ens[rule]) {
        esdg_ensemble_destroy(s->ens[rule]);
        s->ens[rule] = nullptr;
    }
    s->ens_members[rule] = fp32;
    if (fp32.empty()) return ESDG_OK;
    std::vector<esdg_ctx*> ctxs;
    for (Request* r : fp32) ctxs.push_back(r->ctx);
    int rc = esdg_ensemble_create(ctxs.data(), int(ctxs.size()), &s->ens[rule]);
    if (rc) s->err = esdg_ensemble_error(nullptr);
    return rc;
}

static void run(esdg_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        {
            const Clock::time_point a0 = Clock::now();
            admit(s, lk);
            s->t_admit += std::chrono::duration<double>(Clock::now() - a0).count();
        }
        if (s->stop) {
            // esdg_server_destroy: running requests end after their last iteration
            for (Request* r : s->active) finish(s, r, ESDG_ESTATE, "server destroyed while the request ran");
            s->active.clear();
            s->cv.notify_all();
            break;
        }
        if (s->active.empty()) {
            s->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        const int chunk = kMaxChunk;
        std::vector<Request*> act = s->active;
        lk.unlock();
        // steps each request advances in this iteration
        std::vector<int> adv(act.size());
        for (size_t i = 0; i < act.size(); ++i) adv[i] = std::min(chunk, act[i]->remaining);
        int rc = ESDG_OK;
        double t_rb = 0;
        const Clock::time_point l0 = Clock::now();
        for (int rule = 0; rule < 2 && !rc; ++rule) {
            const Clock::time_point r0 = Clock::now();
            rc = refresh_ensemble(s, act, rule, chunk);
            t_rb += std::chrono::duration<double>(Clock::now() - r0).count();
            if (!rc && s->ens[rule]) rc = esdg_ensemble_step_async(s->ens[rule], chunk);
        }
        for (size_t i = 0; i < act.size() && !rc; ++i) {
            Request* r = act[i];
            if (r->precision == ESDG_FP64 || r->remaining < chunk) rc = esdg_step_async(r->ctx, adv[i], r->dt, r->t);
        }
        const Clock::time_point w0 = Clock::now();
        cudaStreamSynchronize(s->stream);
        for (Request* r : act)
            if (r->stream) cudaStreamSynchronize(r->stream);
        const Clock::time_point w1 = Clock::now();
        std::vector<std::pair<Request*, int>> outcome;
        for (Request* r : act) {
            int st = rc ? rc : esdg_check(r->ctx);
            outcome.emplace_back(r, st);
        }
        long long stepped = 0;
        for (size_t i = 0; i < outcome.size(); ++i) {
            Request* r = outcome[i].first;
            if (outcome[i].second) continue;
            r->remaining -= adv[i];
            r->t += adv[i] * r->dt;
            stepped = std::max<long long>(stepped, adv[i]);
            if (r->remaining == 0) outcome[i].second = esdg_copy_state(r->ctx, r->result, 0);
        }
        lk.lock();
        s->t_rebuild += t_rb;
        s->t_launch += std::chrono::duration<double>(w0 - l0).count() - t_rb;
        s->t_wait += std::chrono::duration<double>(w1 - w0).count();
        s->t_retire += std::chrono::duration<double>(Clock::now() - w1).count();
        s->iterations += 1;
        s->steps_run += stepped;
        s->max_active_seen = std::max(s->max_active_seen, (int)act.size());
        std::vector<Request*> keep;
        for (auto& o : outcome) {
            Request* r = o.first;
            if (o.second) {
                finish(s, r, o.second, r->ctx ? esdg_last_error(r->ctx) : "failed");
            } else if (r->remaining == 0) {
                finish(s, r, 2, "");
            } else {
                keep.push_back(r);
            }
        }
        s->active = keep;
        s->cv.notify_all();
    }
    for (int rule = 0; rule < 2; ++rule)
        if (s->ens[rule]) {
            esdg_ensemble_destroy(s->ens[rule]);
            s->ens[rule] = nullptr;
        }
}

extern "C" {

int esdg_server_create(size_t hbm_budget_bytes, int max_active, void* stream, esdg_server** out) {
    if (!out || hbm_budget_bytes == 0 || max_active < 1) return ESDG_EINVAL;
    esdg_server* s = new (std::nothrow) esdg_server();
    if (!s) return ESDG_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    s->t0 = Clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return ESDG_ECUDA;
    }
    s->worker = std::thread(run, s);
    *out = s;
    return ESDG_OK;
}

int esdg_server_submit(esdg_server* s, esdg_ctx* ctx, const double* b_nodal, const double* q_volq, int mode,
                       int nsteps, double* result_host, int* ticket) {
    if (!s || !ctx || !b_nodal || !q_volq || !result_host || !ticket || nsteps < 1) return ESDG_EINVAL;
    size_t bytes = 0;
    int rc = esdg_sizes(ctx, nullptr, nullptr, nullptr, nullptr, &bytes);
    if (rc) return rc;
    Request* r = new (std::nothrow) Request();
    if (!r) return ESDG_ENOMEM;
    r->ctx = ctx;
    r->nsteps = r->remaining = nsteps;
    r->result = result_host;
    r->bytes = (bytes + 255) & ~size_t(255);
    int nghost = 0;
    rc = esdg_partition_info(ctx, nullptr, &nghost, nullptr, nullptr, nullptr, nullptr);
    if (rc || nghost > 0) return rc ? rc : ESDG_EINVAL;  // a block of a partition needs its halo exchange
    esdg_config cfg;
    rc = esdg_get_config(ctx, &cfg);
    // FP32 requests run inside an ensemble launch, which carries neither
    // forcing terms, the weight-adjusted inverse nor the DG-SBP method; FP64
    // requests run through their own contexts and take any configuration
    if (rc || (cfg.precision == ESDG_FP32 && (cfg.forcing != ESDG_FORCING_NONE || cfg.mass != ESDG_MASS_EXACT ||
                                              cfg.method != ESDG_METHOD_MODAL))) {
        delete r;
        return rc ? rc : ESDG_EINVAL;
    }
    r->precision = cfg.precision;
    {
        int K = 0, Np = 0, Nq = 0;
        esdg_sizes(ctx, &K, &Np, &Nq, nullptr, nullptr);
        r->dofs = (long long)K * (cfg.method == ESDG_METHOD_SBP ? Nq : Np);
    }
    esdg_dt(ctx, &r->dt);
    r->rule = cfg.volume_rule == ESDG_RULE_SYMMETRIC ? 1 : 0;
    // all host work of the request (bathymetry, initial projection, operator
    // and geometry packing) runs here, in the submitting thread
    rc = esdg_prepare(ctx, b_nodal, q_volq, mode);
    if (rc) {
        delete r;
        return rc;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->bytes + 256 > s->budget) {
        delete r;
        return ESDG_EBUSY;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_s(s);
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv.notify_all();
    return ESDG_OK;
}

int esdg_server_query(esdg_server* s, int ticket, int* state, double* t_submit, double* t_admit, double* t_done) {
    if (!s) return ESDG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return ESDG_EINVAL;
    Request* r = it->second;
    if (state) *state = r->state;
    if (t_submit) *t_submit = r->t_submit;
    if (t_admit) *t_admit = r->t_admit;
    if (t_done) *t_done = r->t_done;
    return ESDG_OK;
}

int esdg_server_drain(esdg_server* s, double timeout_s) {
    if (!s) return ESDG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!s->queue.empty() || !s->active.empty() || s->admitting > 0) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return ESDG_ETIMEOUT;
    }
    return ESDG_OK;
}

int esdg_server_stats(esdg_server* s, long long* iterations, long long* steps, size_t* bytes_in_use,
                      int* max_active_seen) {
    if (!s) return ESDG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (max_active_seen) *max_active_seen = s->max_active_seen;
    if (iterations) *iterations = s->iterations;
    if (steps) *steps = s->steps_run;
    if (bytes_in_use) *bytes_in_use = s->in_use;
    return ESDG_OK;
}

int esdg_server_timing(esdg_server* s, double* seconds) {
    if (!s || !seconds) return ESDG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    seconds[0] = s->t_admit;
    seconds[1] = s->t_rebuild;
    seconds[2] = s->t_launch;
    seconds[3] = s->t_wait;
    seconds[4] = s->t_retire;
    return ESDG_OK;
}

int esdg_server_destroy(esdg_server* s) {
    if (!s) return ESDG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests are dropped
        for (Request* r : s->queue) finish(s, r, ESDG_ESTATE, "server destroyed");
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (auto& kv : s->all) delete kv.second;
    delete s;
    return ESDG_OK;
}

}  // extern "C"
