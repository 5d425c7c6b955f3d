// Serving engine (include/dbs.h, dbs_engine_*): a queue of simulation
// requests admitted by a device-memory budget and advanced together.
//
// Each tick: (1) admit queued requests in arrival order while the budget and
// the slot limit allow (a request becomes a suspension handle with its own
// stream); (2) wait until some block in flight completes -- the one ensemble
// of all cluster-path requests, or one grid-path request's block on its own
// stream -- and count its steps; (3) copy out and free the finished requests;
// (4) launch the next min(block_steps, remaining) Heun steps of everything
// idle: the cluster-path requests as one ensemble (rebuilt when the resident
// set changes), each other request on its own stream, all concurrently.
// Blocks complete independently, so a small request does not wait for a large
// one's block.  Requests that arrive while others run join at the next tick:
// continuous batching.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dbs.h"
#include "dbs_internal.cuh"

namespace {

thread_local char g_eng_error[256] = "";

#ifndef DBS_ENGINE_GRID_INFLIGHT
#define DBS_ENGINE_GRID_INFLIGHT 2
#endif
constexpr int kGridInflight = DBS_ENGINE_GRID_INFLIGHT;   // grid-path blocks in flight at once

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
    int64_t inflight = 0;          // grid path: steps launched, not yet accounted
    cudaEvent_t ev = nullptr;      // grid path: recorded after the last launch
    cudaStream_t stream = nullptr; // the request's stream (least priority), owned by the engine
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
    std::vector<int64_t> ens_k;    // steps of the ensemble block in flight, per member
    bool ens_busy = false;
    cudaEvent_t ens_ev = nullptr;  // recorded after the block in flight
    // host-side accounting (dbs_engine_stats)
    int64_t ticks = 0, rebuilds = 0;
    double tick_s = 0.0, rebuild_s = 0.0, wait_s = 0.0;
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
    if (r.ev) {
        cudaEventDestroy(r.ev);
        r.ev = nullptr;
    }
    if (r.stream) {
        cudaStreamDestroy(r.stream);
        r.stream = nullptr;
    }
    r.inflight = 0;
}

// The ensemble block in flight has completed: its members' steps count.
static void ens_settle(dbs_engine *e)
{
    if (!e->ens_busy) return;
    for (size_t i = 0; i < e->ens_ids.size(); ++i) {
        auto it = e->req.find(e->ens_ids[i]);
        if (it != e->req.end()) it->second.remaining -= e->ens_k[i];
    }
    e->ens_busy = false;
}

// Wait for the ensemble block in flight (if any), count it, and drop the ensemble.
static void drop_ensemble(dbs_engine *e)
{
    if (e->ens_busy) {
        cudaEventSynchronize(e->ens_ev);
        ens_settle(e);
    }
    if (e->ens) {
        ens_destroy(e->ens);
        e->ens = nullptr;
    }
    e->ens_ids.clear();
    e->ens_k.clear();
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
    if (e->ens_ev) cudaEventDestroy(e->ens_ev);
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
    const double t_tick = now_s();
    struct TickClock {   // adds this tick's host time to the engine's total on every return
        dbs_engine *e;
        double t0;
        ~TickClock() { e->tick_s += now_s() - t0; ++e->ticks; }
    } tick_clock{e, t_tick};
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
        // each request on a stream of the least priority: the ensemble of the
        // small ones (greatest priority) is scheduled ahead of large single systems
        int rc = DBS_OK, least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&r.stream, cudaStreamNonBlocking, least) != cudaSuccess)
            rc = DBS_E_CUDA;
        r.p.stream = r.stream;
        if (rc == DBS_OK) rc = dbs_create_suspension(&r.p, r.x0.data(), &r.h);
        if (rc == DBS_OK) rc = dbs_set_stroke(r.h, r.lam.data(), r.phi.data());
        if (rc == DBS_OK && cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
            rc = DBS_E_CUDA;
        if (rc != DBS_OK) {
            release(e, r);
            r.state = DBS_REQ_FAILED;
            r.t_done = now_s();
            continue;
        }
        e->used += r.bytes;
        r.state = DBS_REQ_RUNNING;
        r.cluster = ens_member_ok(r.h);
        e->active.push_back(r.id);
        if (r.remaining == 0) {  // nothing to do: done at once
            finish(e, r);
            e->active.pop_back();
        }
    }
    // (2) wait until some work in flight completes (the ensemble's block, or one
    // grid-path request's block), polling without blocking the others
    bool inflight = e->ens_busy;
    for (int64_t id : e->active) inflight |= e->req[id].inflight > 0;
    const double t_wait = now_s();
    while (inflight) {
        bool progress = false;
        if (e->ens_busy) {
            const cudaError_t q = cudaEventQuery(e->ens_ev);
            if (q == cudaSuccess) {
                ens_settle(e);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                return engfail(e, DBS_E_CUDA, "ensemble: %s", cudaGetErrorString(q));
            }
        }
        for (int64_t id : e->active) {
            Request &r = e->req[id];
            if (r.inflight == 0) continue;
            const cudaError_t q = cudaEventQuery(r.ev);
            if (q == cudaSuccess) {
                r.remaining -= r.inflight;
                r.inflight = 0;
                progress = true;
            } else if (q != cudaErrorNotReady) {
                r.state = DBS_REQ_FAILED;
                r.t_done = now_s();
                r.inflight = 0;
                progress = true;
            }
        }
        if (progress) break;
        if (now_s() - t_wait > 600.0) return engfail(e, DBS_E_TIMEOUT, "no block completed in 600 s");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    e->wait_s += now_s() - t_wait;
    // (3) retire: failed requests, and finished ones that nothing still runs
    std::vector<int64_t> still;
    for (int64_t id : e->active) {
        Request &r = e->req[id];
        const bool in_ens = e->ens_busy && std::find(e->ens_ids.begin(), e->ens_ids.end(), id) != e->ens_ids.end();
        if (r.state == DBS_REQ_FAILED && !in_ens) {
            if (r.inflight == 0) release(e, r);
            else still.push_back(id);
            continue;
        }
        if (r.remaining == 0 && r.inflight == 0 && !in_ens) finish(e, r);
        else still.push_back(id);
    }
    e->active.swap(still);
    // (4) launch the next block of everything idle: the cluster-path requests as
    // one ensemble (rebuilt when its membership changes), the others each on its
    // own stream; all run concurrently
    if (!e->ens_busy) {
        std::vector<int64_t> cl;
        for (int64_t id : e->active) {
            const Request &r = e->req[id];
            if (r.cluster && r.state == DBS_REQ_RUNNING && r.remaining > 0) cl.push_back(id);
        }
        if (cl != e->ens_ids) {
            const double t_rb = now_s();
            drop_ensemble(e);
            if (!cl.empty()) {
                std::vector<dbs_suspension *> hs;
                for (int64_t id : cl) hs.push_back(e->req[id].h);
                int rc = ens_create((int32_t)hs.size(), hs.data(), nullptr, &e->ens);
                if (rc != DBS_OK) return engfail(e, rc, "ensemble: %s", ens_error(nullptr));
                e->ens_ids = cl;
            }
            ++e->rebuilds;
            e->rebuild_s += now_s() - t_rb;
        }
        if (e->ens) {
            e->ens_k.clear();
            for (int64_t id : cl) e->ens_k.push_back(std::min<int64_t>(e->req[id].remaining, e->P.block_steps));
            int rc = ens_step_v(e->ens, e->ens_k.data());
            if (rc != DBS_OK) return engfail(e, rc, "ensemble step: %s", ens_error(e->ens));
            if (!e->ens_ev && cudaEventCreateWithFlags(&e->ens_ev, cudaEventDisableTiming) != cudaSuccess)
                return engfail(e, DBS_E_CUDA, "event");
            // the members' streams wait for the ensemble's block: an event on one of them
            if (cudaEventRecord(e->ens_ev, e->req[cl[0]].h->stream) != cudaSuccess)
                return engfail(e, DBS_E_CUDA, "event record");
            e->ens_busy = true;
        }
    }
    // grid-path requests (each fills the device on its own): at most kGridInflight
    // of them have a block in flight, the ones with the least remaining work first
    std::vector<int64_t> idle;
    int busy = 0;
    for (int64_t id : e->active) {
        const Request &r = e->req[id];
        if (r.cluster || r.state != DBS_REQ_RUNNING) continue;
        if (r.inflight > 0) ++busy;
        else if (r.remaining > 0) idle.push_back(id);
    }
    auto work = [&](int64_t id) {
        const Request &r = e->req[id];
        return (double)r.remaining * (double)r.p.S * (double)r.p.S;
    };
    std::stable_sort(idle.begin(), idle.end(), [&](int64_t a, int64_t b) { return work(a) < work(b); });
    for (int64_t id : idle) {
        if (busy >= kGridInflight) break;
        Request &r = e->req[id];
        const int64_t k = std::min<int64_t>(r.remaining, e->P.block_steps);
        if (dbs_step(r.h, k) != DBS_OK || cudaEventRecord(r.ev, r.h->stream) != cudaSuccess) {
            r.state = DBS_REQ_FAILED;
            r.t_done = now_s();
            continue;
        }
        r.inflight = k;
        ++busy;
    }
    if (active) *active = (int32_t)e->active.size();
    if (pending) *pending = (int32_t)e->queue.size();
    return DBS_OK;
}

int dbs_engine_stats(const dbs_engine *e, dbs_engine_stats_t *out)
{
    if (!e || !out) return DBS_E_ARG;
    out->ticks = e->ticks;
    out->ensemble_rebuilds = e->rebuilds;
    out->tick_s = e->tick_s;
    out->rebuild_s = e->rebuild_s;
    out->wait_s = e->wait_s;
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
    if (r.state == DBS_REQ_RUNNING || r.state == DBS_REQ_FAILED) {
        cudaSetDevice(e->device);
        drop_ensemble(e);   // waits for an ensemble block in flight
        if (r.h) dbs_sync(r.h);
        release(e, r);
        r.state = DBS_REQ_CANCELLED;
        e->active.erase(std::remove(e->active.begin(), e->active.end(), id), e->active.end());
        return DBS_OK;
    }
    return DBS_E_STATE;
}

}  // extern "C"
