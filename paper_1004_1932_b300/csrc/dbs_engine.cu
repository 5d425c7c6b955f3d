// Serving engine (include/dbs.h, dbs_engine_*): a queue of simulation
// requests admitted by a device-memory budget and advanced together.
//
// Each tick: (1) admit queued requests in arrival order while the budget and
// the slot limit allow (a request becomes a suspension handle with its own
// stream); (2) give every resident request min(block_steps, remaining) Heun
// steps -- those that fit the cluster path as one ensemble (rebuilt when the
// resident set changes), the others on the grid path, all concurrently;
// (3) wait, then copy out and free the finished ones.  Requests that arrive
// while others run join at the next tick: continuous batching.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "dbs.h"
#include "dbs_internal.cuh"

namespace {

thread_local char g_eng_error[256] = "";

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    dbs_params p{};
    std::vector<double> x0, lam, phi, result;
    int64_t steps = 0, remaining = 0;
    int32_t state = DBS_REQ_PENDING;
    dbs_suspension *h = nullptr;
    size_t bytes = 0;
    double t_submit = 0, t_done = 0;
    bool cluster = false;
};

size_t request_bytes(int64_t S, int32_t precision)
{
    const int64_t N = 2 * S;
    const size_t rec = precision == DBS_FP64 ? 96 : 48;
    const int64_t C = std::min<int64_t>(std::max<int64_t>(1, S / 16), 64);
    return (size_t)(120 * N + 48 * S + 3 * rec * S + C * 12 * 8 * S) + 65536 + 16384;
}

}  // namespace

struct dbs_engine {
    dbs_engine_params P{};
    int device = 0;
    int status = DBS_OK;
    char msg[256] = "";
    std::deque<int64_t> queue;
    std::vector<int64_t> active;
    std::unordered_map<int64_t, Request> req;
    size_t used = 0;
    int64_t next_id = 1;
    dbs_ensemble *ens = nullptr;
    std::vector<int64_t> ens_ids;  // members of ens, in order
};

static int engfail(dbs_engine *e, int st, const char *fmt, ...)
{
    char *buf = e ? e->msg : g_eng_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    if (e) e->status = st;
    return st;
}

static void release(dbs_engine *e, Request &r)
{
    if (r.h) {
        dbs_destroy(r.h);
        r.h = nullptr;
        e->used -= r.bytes;
    }
}

static void drop_ensemble(dbs_engine *e)
{
    if (e->ens) {
        ens_destroy(e->ens);
        e->ens = nullptr;
    }
    e->ens_ids.clear();
}

extern "C" {

const char *dbs_engine_last_error(const dbs_engine *e) { return e ? e->msg : g_eng_error; }

int dbs_engine_request_bytes(int64_t S, int32_t precision, size_t *bytes)
{
    if (S < 1 || !bytes) return DBS_E_ARG;
    *bytes = request_bytes(S, precision);
    return DBS_OK;
}

int dbs_engine_create(const dbs_engine_params *p, dbs_engine **out)
{
    if (!out) return DBS_E_ARG;
    *out = nullptr;
    if (!p || p->block_steps < 1 || p->max_active < 0 || p->reserved != 0)
        return engfail(nullptr, DBS_E_ARG, "block_steps >= 1, max_active >= 0, reserved = 0");
    dbs_engine *e = new (std::nothrow) dbs_engine();
    if (!e) return engfail(nullptr, DBS_E_NOMEM, "host allocation");
    e->P = *p;
    int dev = p->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    e->device = dev;
    *out = e;
    return DBS_OK;
}

int dbs_engine_destroy(dbs_engine *e)
{
    if (!e) return DBS_OK;
    cudaSetDevice(e->device);
    drop_ensemble(e);
    for (auto &kv : e->req) release(e, kv.second);
    delete e;
    return DBS_OK;
}

int dbs_engine_submit(dbs_engine *e, const dbs_params *p, const double *x0, const double *lambda,
                      const double *phase, int64_t steps, int64_t *id)
{
    if (!e || !p || !x0 || !id || steps < 0) return DBS_E_ARG;
    if (e->status != DBS_OK) return e->status;
    if (p->S < 1 || p->stream != nullptr) return engfail(e, DBS_E_ARG, "S >= 1 and stream NULL");
    Request r;
    r.id = e->next_id++;
    r.p = *p;
    r.p.device = e->device;
    r.x0.assign(x0, x0 + 6 * p->S);
    r.lam.assign(p->S, 0.0);
    r.phi.assign(p->S, 0.0);
    if (lambda) r.lam.assign(lambda, lambda + p->S);
    if (phase) r.phi.assign(phase, phase + p->S);
    r.steps = r.remaining = steps;
    r.bytes = request_bytes(p->S, p->precision);
    r.t_submit = now_s();
    *id = r.id;
    e->queue.push_back(r.id);
    e->req.emplace(r.id, std::move(r));
    e->status = DBS_OK;
    return DBS_OK;
}

static void finish(dbs_engine *e, Request &r)
{
    r.result.resize(6 * r.p.S);
    if (dbs_positions(r.h, r.result.data()) != DBS_OK) {
        r.state = DBS_REQ_FAILED;
    } else {
        r.state = DBS_REQ_DONE;
    }
    r.t_done = now_s();
    release(e, r);
}

int dbs_engine_tick(dbs_engine *e, int32_t *active, int32_t *pending)
{
    if (!e) return DBS_E_ARG;
    if (cudaSetDevice(e->device) != cudaSuccess) return engfail(e, DBS_E_CUDA, "cudaSetDevice");
    bool changed = false;
    // (1) admission, arrival order
    while (!e->queue.empty()) {
        Request &r = e->req[e->queue.front()];
        if (r.state == DBS_REQ_CANCELLED) {
            e->queue.pop_front();
            continue;
        }
        if (e->P.max_active > 0 && (int32_t)e->active.size() >= e->P.max_active) break;
        if (e->P.hbm_budget_bytes > 0 && e->used + r.bytes > e->P.hbm_budget_bytes) break;
        e->queue.pop_front();
        int rc = dbs_create_suspension(&r.p, r.x0.data(), &r.h);
        if (rc == DBS_OK) rc = dbs_set_stroke(r.h, r.lam.data(), r.phi.data());
        if (rc != DBS_OK) {
            if (r.h) dbs_destroy(r.h);
            r.h = nullptr;
            r.state = DBS_REQ_FAILED;
            r.t_done = now_s();
            continue;
        }
        e->used += r.bytes;
        r.state = DBS_REQ_RUNNING;
        r.cluster = ens_member_ok(r.h);
        e->active.push_back(r.id);
        changed = true;
        if (r.remaining == 0) {  // nothing to do: done at once
            finish(e, r);
            e->active.pop_back();
        }
    }
    // (2) advance: cluster members as one ensemble, the rest on the grid path
    std::vector<int64_t> cl, gr;
    for (int64_t id : e->active) (e->req[id].cluster ? cl : gr).push_back(id);
    if (changed || cl != e->ens_ids) {
        drop_ensemble(e);
        if (!cl.empty()) {
            std::vector<dbs_suspension *> hs;
            for (int64_t id : cl) hs.push_back(e->req[id].h);
            int rc = ens_create((int32_t)hs.size(), hs.data(), nullptr, &e->ens);
            if (rc != DBS_OK) return engfail(e, rc, "ensemble: %s", ens_error(nullptr));
            e->ens_ids = cl;
        }
    }
    std::vector<int64_t> ksteps;
    for (int64_t id : cl) ksteps.push_back(std::min<int64_t>(e->req[id].remaining, e->P.block_steps));
    if (e->ens) {
        int rc = ens_step_v(e->ens, ksteps.data());
        if (rc != DBS_OK) return engfail(e, rc, "ensemble step: %s", ens_error(e->ens));
    }
    for (int64_t id : gr) {
        Request &r = e->req[id];
        const int64_t k = std::min<int64_t>(r.remaining, e->P.block_steps);
        if (dbs_step(r.h, k) != DBS_OK) {
            r.state = DBS_REQ_FAILED;
            r.t_done = now_s();
        }
    }
    // (3) wait, account, retire
    std::vector<int64_t> still;
    for (size_t i = 0; i < cl.size(); ++i) {
        Request &r = e->req[cl[i]];
        r.remaining -= ksteps[i];
    }
    for (int64_t id : gr) {
        Request &r = e->req[id];
        if (r.state == DBS_REQ_RUNNING) r.remaining -= std::min<int64_t>(r.remaining, e->P.block_steps);
    }
    for (int64_t id : e->active) {
        Request &r = e->req[id];
        if (r.state == DBS_REQ_FAILED) {
            release(e, r);
            continue;
        }
        if (dbs_sync(r.h) != DBS_OK) {
            r.state = DBS_REQ_FAILED;
            r.t_done = now_s();
            release(e, r);
            continue;
        }
        if (r.remaining == 0) {
            finish(e, r);
        } else {
            still.push_back(id);
        }
    }
    e->active.swap(still);
    if (active) *active = (int32_t)e->active.size();
    if (pending) *pending = (int32_t)e->queue.size();
    return DBS_OK;
}

int dbs_engine_poll(dbs_engine *e, int64_t id, int32_t *state, double *x_out, double *latency_s)
{
    if (!e) return DBS_E_ARG;
    auto it = e->req.find(id);
    if (it == e->req.end()) return DBS_E_ARG;
    Request &r = it->second;
    if (state) *state = r.state;
    if (r.state == DBS_REQ_DONE) {
        if (x_out) std::copy(r.result.begin(), r.result.end(), x_out);
        if (latency_s) *latency_s = r.t_done - r.t_submit;
    }
    return DBS_OK;
}

int dbs_engine_cancel(dbs_engine *e, int64_t id)
{
    if (!e) return DBS_E_ARG;
    auto it = e->req.find(id);
    if (it == e->req.end()) return DBS_E_ARG;
    Request &r = it->second;
    if (r.state == DBS_REQ_PENDING) {
        r.state = DBS_REQ_CANCELLED;
        return DBS_OK;
    }
    if (r.state == DBS_REQ_RUNNING) {
        cudaSetDevice(e->device);
        drop_ensemble(e);
        if (r.h) dbs_sync(r.h);
        release(e, r);
        r.state = DBS_REQ_CANCELLED;
        e->active.erase(std::remove(e->active.begin(), e->active.end(), id), e->active.end());
        return DBS_OK;
    }
    return DBS_E_STATE;
}

}  // extern "C"
