// Ensembles of independent suspensions advanced together by the
// cluster-resident kernel (resident_kernel.cuh), and the single-system
// cluster path of dbs_step (a private one-member ensemble).
//
// Every member gets a thread-block cluster of G CTAs (G in {1, 2, 4, 8, 16})
// that holds its whole state for a block of up to K_BLOCK Heun steps.  Members
// are grouped by (mobility, threads per CTA, G) into launch classes; the
// classes of one block run concurrently on their own streams (fork/join with
// events on the ensemble stream).  Cluster sizes come from a balance rule
// (work S^2 / G close to the mean per-CTA work) or from the caller (autotuner).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "dbs.h"
#include "dbs_internal.cuh"
#include "resident_kernel.cuh"

using namespace dbs;

#ifndef DBS_ENS_HEAVY_FIRST
#define DBS_ENS_HEAVY_FIRST 1
#endif

namespace {

constexpr int K_BLOCK = 1024;     // Heun steps per resident launch (< clock ring / 2)
constexpr int NT_BIG = 512;       // threads per CTA for S > SMALL_RES_S
constexpr int NT_SMALL = 128;     // threads per CTA for small members
constexpr int SMALL_RES_S = 64;
constexpr size_t SMEM_LIMIT = 227 * 1024;

thread_local char g_ens_error[256] = "";

struct ClassKey {
    int mob, nt, G;
    bool operator<(const ClassKey &o) const { return std::tie(mob, nt, G) < std::tie(o.mob, o.nt, o.G); }
};

struct Class {
    std::vector<int> members;  // member indices, cluster order
    int *csys = nullptr;       // device copy of members
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    size_t smem = 0;
};

template <int MOB, int NT>
const void *kernel_ptr() { return (const void *)resident_kernel<MOB, NT>; }

const void *pick_kernel(int mob, int nt)
{
    if (mob == DBS_OSEEN) return nt == NT_BIG ? kernel_ptr<0, NT_BIG>() : kernel_ptr<0, NT_SMALL>();
    return nt == NT_BIG ? kernel_ptr<1, NT_BIG>() : kernel_ptr<1, NT_SMALL>();
}

int nt_for(int64_t S) { return S <= SMALL_RES_S ? NT_SMALL : NT_BIG; }

int min_cluster(int64_t S, int nt)
{
    int G = 1;
    while (G < 16 && (S + G - 1) / G > nt) G *= 2;
    return G;
}

}  // namespace

struct dbs_ensemble {
    int test_g_scale = 1;          // diagnostic: the kernels expect G x this (1 = the true shape)
    std::vector<dbs_suspension *> m;
    std::vector<int> G;            // cluster size per member
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int status = DBS_OK;
    char msg[256] = "";
    ResSys *d_sys = nullptr;
    std::map<ClassKey, Class> classes;
    cudaEvent_t fork = nullptr, joined = nullptr;
    bool classes_ready = false;
    cudaGraphExec_t launches = nullptr;   // captured fork / class launches / join of one block
};

static int efail(dbs_ensemble *e, int st, const char *fmt, ...)
{
    char *buf = e ? e->msg : g_ens_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    if (e) e->status = st;
    return st;
}

#define ECK(e, call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return efail((e), e_ == cudaErrorMemoryAllocation ? DBS_E_NOMEM : DBS_E_CUDA,      \
                         "%s: %s", #call, cudaGetErrorString(e_));                             \
    } while (0)

static bool member_ok(const dbs_suspension *h)
{
    return h && h->status == DBS_OK && h->p.precision == DBS_FP32C && h->S >= 1 &&
           h->dyn == DBS_DYN_SPRING &&
           resident_smem_bytes((int)h->S, min_cluster(h->S, nt_for(h->S)), nt_for(h->S)) <= SMEM_LIMIT;
}

// Balance rule: per-CTA work S^2 / G near the mean over all CTA slots.
static void auto_clusters(dbs_ensemble *e)
{
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
    double total = 0;
    for (auto *h : e->m) total += (double)h->S * (double)h->S;
    const double per_slot = total / (double)sms;
    e->G.resize(e->m.size());
    for (size_t i = 0; i < e->m.size(); ++i) {
        const int64_t S = e->m[i]->S;
        int G = min_cluster(S, nt_for(S));
        const double w = (double)S * (double)S;
        while (G < 16 && w / G > per_slot && (S + 2 * G - 1) / (2 * G) >= 8) G *= 2;
        e->G[i] = G;
    }
}

static void free_classes(dbs_ensemble *e)
{
    for (auto &kv : e->classes) {
        if (kv.second.csys) cudaFree(kv.second.csys);
        if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
        if (kv.second.done) cudaEventDestroy(kv.second.done);
    }
    e->classes.clear();
    e->classes_ready = false;
    if (e->launches) cudaGraphExecDestroy(e->launches);
    e->launches = nullptr;
}

static int build_classes(dbs_ensemble *e)
{
    free_classes(e);
    for (size_t i = 0; i < e->m.size(); ++i) {
        const dbs_suspension *h = e->m[i];
        const int nt = nt_for(h->S);
        if (e->G[i] < min_cluster(h->S, nt) || e->G[i] > 16)
            return efail(e, DBS_E_ARG, "cluster size %d invalid for member %zu (S=%lld)", e->G[i], i,
                         (long long)h->S);
        const size_t smem = resident_smem_bytes((int)h->S, e->G[i], nt);
        if (smem > SMEM_LIMIT) return efail(e, DBS_E_ARG, "member %zu too large for the cluster path", i);
        Class &c = e->classes[ClassKey{h->p.mobility, nt, e->G[i]}];
        c.members.push_back((int)i);
        c.smem = std::max(c.smem, smem);
    }
    for (auto &kv : e->classes) {
        Class &c = kv.second;
        if (DBS_ENS_HEAVY_FIRST) {
            // heaviest members (pair work ~ S^2) first: their clusters get the lowest
            // block indices and are dispatched first
            std::stable_sort(c.members.begin(), c.members.end(),
                             [&](int a, int b) { return e->m[a]->S > e->m[b]->S; });
        }
        ECK(e, cudaMalloc(&c.csys, sizeof(int) * c.members.size()));
        ECK(e, cudaMemcpy(c.csys, c.members.data(), sizeof(int) * c.members.size(), cudaMemcpyHostToDevice));
        // the greatest priority: where an ensemble shares the device with large
        // single systems (the serving engine), its blocks are scheduled first
        int least = 0, greatest = 0;
        ECK(e, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        ECK(e, cudaStreamCreateWithPriority(&c.stream, cudaStreamNonBlocking, greatest));
        ECK(e, cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
        const void *k = pick_kernel(kv.first.mob, kv.first.nt);
        ECK(e, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT));
        ECK(e, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    e->classes_ready = true;
    return DBS_OK;
}

static ResSys make_sys(const dbs_suspension *h, int G)
{
    const EvalArgs A = base_args(h);
    ResSys P{};
    P.S = (int)h->S;
    P.G = G;
    P.inv6pimua = A.inv6pimua;
    P.k0 = A.k0;
    P.ell = A.ell;
    P.dt = A.dt;
    P.c2 = A.c2;
    P.c3 = A.c3;
    P.overlap_r2 = A.overlap_r2;
    P.x = h->x;
    P.v0 = h->v0;
    P.Fd = h->Fd;
    P.Fext = h->Fext;
    P.lam = h->lam;
    P.sinphi = h->sinphi;
    P.cosphi = h->cosphi;
    P.pack = h->packA;
    P.trig = h->trig;
    P.trig_mask = A.trig_mask;
    P.step = h->step;
    P.flags = h->flags;
    P.Racc = h->Racc;
    P.Rbar = h->Rbar;
    P.avg_n0 = h->avg_n0;
    P.avg_m = h->avg_m;
    P.avg_maxk = h->avg_maxk;
    P.noise_sigma = h->noise_sigma;
    P.noise_seed = h->noise_seed;
    P.pack_args = A;
    return P;
}

// Advance member i by steps[i] Heun steps (all members by n when steps is
// null); all work is ordered after the members' pending work and before their
// later work.  Blocks of at most K_BLOCK steps; a member whose count is used up
// sits out the remaining blocks (K = 0 launches nothing for it).
// One block of resident launches on the ensemble stream: fork to the class
// streams, one launch per class (members read their K and state from d_sys),
// join.  Captured once per class layout into a CUDA graph and replayed for every
// block; what changes from block to block (step counts, buffers) is data in
// d_sys, uploaded before each replay.
static int enqueue_launches(dbs_ensemble *e)
{
    ECK(e, cudaEventRecord(e->fork, e->stream));
    // classes in decreasing order of pair work (sum of S^2), so that the heaviest,
    // which set the batch's time, are dispatched first
    std::vector<std::pair<const ClassKey, Class> *> order;
    for (auto &kv : e->classes) order.push_back(&kv);
    auto work = [&](const Class &c) {
        double w = 0;
        for (int i : c.members) w += (double)e->m[i]->S * (double)e->m[i]->S;
        return w;
    };
    if (DBS_ENS_HEAVY_FIRST)
        std::stable_sort(order.begin(), order.end(),
                         [&](auto *a, auto *b) { return work(a->second) > work(b->second); });
    for (auto *kvp : order) {
        auto &kv = *kvp;
        Class &c = kv.second;
        ECK(e, cudaStreamWaitEvent(c.stream, e->fork, 0));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(kv.first.G * c.members.size()));
        cfg.blockDim = dim3((unsigned)kv.first.nt);
        cfg.dynamicSmemBytes = c.smem;
        cfg.stream = c.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kv.first.G;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const ResSys *ds = e->d_sys;
        const int *cs = c.csys;
        const int nc = (int)c.members.size(), Gc = kv.first.G * e->test_g_scale;   // the shape the kernel checks
        cudaError_t err;
        if (kv.first.mob == DBS_OSEEN)
            err = kv.first.nt == NT_BIG ? cudaLaunchKernelEx(&cfg, resident_kernel<0, NT_BIG>, ds, cs, nc, Gc)
                                        : cudaLaunchKernelEx(&cfg, resident_kernel<0, NT_SMALL>, ds, cs, nc, Gc);
        else
            err = kv.first.nt == NT_BIG ? cudaLaunchKernelEx(&cfg, resident_kernel<1, NT_BIG>, ds, cs, nc, Gc)
                                        : cudaLaunchKernelEx(&cfg, resident_kernel<1, NT_SMALL>, ds, cs, nc, Gc);
        if (err != cudaSuccess)
            return efail(e, DBS_E_CUDA, "resident launch (G=%d, %zu members): %s", kv.first.G,
                         c.members.size(), cudaGetErrorString(err));
        ECK(e, cudaEventRecord(c.done, c.stream));
        ECK(e, cudaStreamWaitEvent(e->stream, c.done, 0));
    }
    return DBS_OK;
}

static int capture_launches(dbs_ensemble *e)
{
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_launches(e);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return efail(e, DBS_E_CUDA, "ensemble capture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&e->launches, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return efail(e, DBS_E_CUDA, "ensemble graph: %s", cudaGetErrorString(ie));
    return DBS_OK;
}

static int ensemble_step_v(dbs_ensemble *e, int64_t n, const int64_t *steps)
{
    if (e->status != DBS_OK) return e->status;
    ECK(e, cudaSetDevice(e->device));
    if (!e->classes_ready) {
        int rc = build_classes(e);
        if (rc) return rc;
    }
    const size_t M = e->m.size();
    std::vector<int64_t> left(M);
    for (size_t i = 0; i < M; ++i) left[i] = steps ? steps[i] : n;
    // the ensemble stream waits for each member's stream
    for (auto *h : e->m) {
        ECK(e, cudaEventRecord(e->joined, h->stream));
        ECK(e, cudaStreamWaitEvent(e->stream, e->joined, 0));
    }
    std::vector<ResSys> sys(M);
    for (;;) {
        int64_t kmax = 0;
        for (size_t i = 0; i < M; ++i) kmax = std::max(kmax, std::min<int64_t>(left[i], K_BLOCK));
        if (kmax == 0) break;
        for (size_t i = 0; i < M; ++i) {
            dbs_suspension *h = e->m[i];
            if (h->status != DBS_OK) return efail(e, h->status, "member %zu is in an error state", i);
            const int K = (int)std::min<int64_t>(left[i], K_BLOCK);
            int rc = ensure_trig(h, h->n_host + K + 1, e->stream);
            if (rc) return efail(e, rc, "member %zu: %s", i, h->msg);
            sys[i] = make_sys(h, e->G[i]);
            sys[i].K = K;
        }
        if (!e->d_sys) ECK(e, cudaMalloc(&e->d_sys, sizeof(ResSys) * M));
        ECK(e, cudaMemcpyAsync(e->d_sys, sys.data(), sizeof(ResSys) * M, cudaMemcpyHostToDevice,
                               e->stream));
        if (!e->launches) {
            int rc = capture_launches(e);
            if (rc) return rc;
        }
        ECK(e, cudaGraphLaunch(e->launches, e->stream));
        for (size_t i = 0; i < M; ++i) {
            const int K = (int)std::min<int64_t>(left[i], K_BLOCK);
            e->m[i]->n_host += K;
            left[i] -= K;
        }
    }
    // members' later work waits for the ensemble
    ECK(e, cudaEventRecord(e->joined, e->stream));
    for (auto *h : e->m) ECK(e, cudaStreamWaitEvent(h->stream, e->joined, 0));
    return DBS_OK;
}

static int ensemble_step(dbs_ensemble *e, int64_t n) { return ensemble_step_v(e, n, nullptr); }

static int ensemble_create(int32_t count, dbs_suspension *const *members, void *stream,
                           dbs_ensemble **out)
{
    *out = nullptr;
    dbs_ensemble *e = new (std::nothrow) dbs_ensemble();
    if (!e) return efail(nullptr, DBS_E_NOMEM, "host allocation");
    e->device = members[0]->device;
    for (int32_t i = 0; i < count; ++i) {
        if (!member_ok(members[i]) || members[i]->device != e->device) {
            delete e;
            return efail(nullptr, DBS_E_ARG,
                         "member %d: needs an FP32C suspension on one device, S within the cluster path", i);
        }
        for (int32_t j = 0; j < i; ++j)
            if (members[j] == members[i]) {
                delete e;
                return efail(nullptr, DBS_E_ARG, "member %d listed twice", i);
            }
        e->m.push_back(members[i]);
    }
    auto bail = [&](int rc) {
        snprintf(g_ens_error, sizeof(g_ens_error), "%s", e->msg);
        free_classes(e);
        if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
        delete e;
        return rc;
    };
    if (cudaSetDevice(e->device) != cudaSuccess) return bail(efail(e, DBS_E_CUDA, "cudaSetDevice"));
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(efail(e, DBS_E_CUDA, "stream creation"));
        e->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->joined, cudaEventDisableTiming) != cudaSuccess)
        return bail(efail(e, DBS_E_CUDA, "event creation"));
    auto_clusters(e);
    *out = e;
    return DBS_OK;
}

static void ensemble_destroy(dbs_ensemble *e)
{
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    free_classes(e);
    if (e->d_sys) cudaFree(e->d_sys);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->joined) cudaEventDestroy(e->joined);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

// ---- internal entry points (serving engine) ------------------------------------
bool ens_member_ok(const dbs_suspension *h) { return member_ok(h); }
int ens_create(int32_t count, dbs_suspension *const *members, void *stream, dbs_ensemble **out)
{
    return ensemble_create(count, members, stream, out);
}
int ens_step_v(dbs_ensemble *e, const int64_t *steps) { return ensemble_step_v(e, 0, steps); }
void ens_destroy(dbs_ensemble *e) { ensemble_destroy(e); }
const char *ens_error(const dbs_ensemble *e) { return e ? e->msg : g_ens_error; }

// ---- single-system cluster path -------------------------------------------------
int solo_step(dbs_suspension *h, int64_t n)
{
    int rc = ensemble_step(h->solo, n);
    if (rc) return fail(h, rc, "cluster path: %s", h->solo->msg);
    return DBS_OK;
}

void solo_destroy(dbs_suspension *h)
{
    ensemble_destroy(h->solo);
    h->solo = nullptr;
}

extern "C" {

const char *dbs_ensemble_last_error(const dbs_ensemble *e) { return e ? e->msg : g_ens_error; }

int dbs_ensemble_create(int32_t count, dbs_suspension *const *members, void *stream,
                        dbs_ensemble **out)
{
    if (!out) return DBS_E_ARG;
    *out = nullptr;
    if (count < 1 || !members) return efail(nullptr, DBS_E_ARG, "empty ensemble");
    for (int32_t i = 0; i < count; ++i)
        if (!members[i]) return efail(nullptr, DBS_E_ARG, "member %d is NULL", i);
    return ensemble_create(count, members, stream, out);
}

int dbs_ensemble_destroy(dbs_ensemble *e)
{
    ensemble_destroy(e);
    return DBS_OK;
}

int dbs_ensemble_set_clusters(dbs_ensemble *e, const int32_t *G)
{
    if (!e) return DBS_E_ARG;
    if (e->status != DBS_OK) return e->status;
    if (!G) {
        auto_clusters(e);
    } else {
        for (size_t i = 0; i < e->m.size(); ++i) {
            const int nt = nt_for(e->m[i]->S);
            if (G[i] != 1 && G[i] != 2 && G[i] != 4 && G[i] != 8 && G[i] != 16) return DBS_E_ARG;
            if (G[i] < min_cluster(e->m[i]->S, nt)) return DBS_E_ARG;
        }
        for (size_t i = 0; i < e->m.size(); ++i) e->G[i] = G[i];
    }
    if (e->stream) cudaStreamSynchronize(e->stream);
    free_classes(e);
    return DBS_OK;
}

int dbs_ensemble_get_clusters(dbs_ensemble *e, int32_t *G)
{
    if (!e || !G) return DBS_E_ARG;
    for (size_t i = 0; i < e->m.size(); ++i) G[i] = e->G[i];
    return DBS_OK;
}

int dbs_ensemble_step(dbs_ensemble *e, int64_t n)
{
    if (!e || n < 0) return DBS_E_ARG;
    return ensemble_step(e, n);
}

int dbs_ensemble_sync(dbs_ensemble *e)
{
    if (!e) return DBS_E_ARG;
    if (e->status != DBS_OK) return e->status;
    ECK(e, cudaStreamSynchronize(e->stream));
    for (auto *h : e->m) {
        int rc = check_flags(h);
        if (rc) return efail(e, rc, "member fault: %s", h->msg);
    }
    return DBS_OK;
}

int dbs_test_ensemble_misshape(dbs_ensemble *e)
{
    if (!e) return DBS_E_ARG;
    if (e->status != DBS_OK) return e->status;
    ECK(e, cudaSetDevice(e->device));
    // one step recaptured with kernels told to expect twice their cluster size,
    // then the true shape again for any later capture
    if (e->launches) cudaGraphExecDestroy(e->launches);
    e->launches = nullptr;
    e->test_g_scale = 2;
    const int rc = ensemble_step(e, 1);
    e->test_g_scale = 1;
    if (e->launches) cudaGraphExecDestroy(e->launches);
    e->launches = nullptr;
    if (rc) return rc;
    return dbs_ensemble_sync(e);
}

int dbs_set_path(dbs_suspension *h, int32_t path, int32_t cluster_size)
{
    if (!h) return DBS_E_ARG;
    if (h->status != DBS_OK) return h->status;
    cudaSetDevice(h->device);
    if (h->solo) {
        cudaStreamSynchronize(h->stream);
        solo_destroy(h);
    }
    if (h->dyn != DBS_DYN_SPRING && !(path == DBS_PATH_GRID || (path == DBS_PATH_COOP && h->p.precision != DBS_FP64)))
        return refuse(h, DBS_E_STATE, "shape-driven dynamics run on the grid path, or the cooperative one in FP32C");
    h->path = DBS_PATH_GRID;
    if (path == DBS_PATH_GRID) return DBS_OK;
    if (path == DBS_PATH_COOP) {
        int rc = coop_setup(h);   // a size the path cannot hold is refused, the handle stays usable
        if (rc) return rc;
        h->path = DBS_PATH_COOP;
        return DBS_OK;
    }
    if (path != DBS_PATH_CLUSTER) return DBS_E_ARG;
    if (!member_ok(h)) return refuse(h, DBS_E_ARG, "cluster path needs FP32C and S small enough");
    if (h->solo) solo_destroy(h);
    dbs_suspension *one[1] = {h};
    dbs_ensemble *e = nullptr;
    int rc = ensemble_create(1, one, h->stream, &e);
    if (rc) return fail(h, rc, "cluster path: %s", g_ens_error);
    // a lone system takes the largest cluster (every SM of it works on the one system)
    const int nt = nt_for(h->S);
    int G = cluster_size;
    if (G == 0) {
        G = 16;
        while (G > min_cluster(h->S, nt) && (h->S + G - 1) / G < 8) G /= 2;
    }
    int32_t g32 = G;
    rc = dbs_ensemble_set_clusters(e, &g32);
    if (rc) {
        ensemble_destroy(e);
        return fail(h, rc, "cluster size %d not valid for S=%lld", G, (long long)h->S);
    }
    h->solo = e;
    h->path = DBS_PATH_CLUSTER;
    return DBS_OK;
}

int dbs_get_path(dbs_suspension *h, int32_t *path, int32_t *cluster_size)
{
    if (!h) return DBS_E_ARG;
    if (path) *path = h->path;
    if (cluster_size) *cluster_size = h->solo ? h->solo->G[0] : 0;
    return DBS_OK;
}

}  // extern "C"
