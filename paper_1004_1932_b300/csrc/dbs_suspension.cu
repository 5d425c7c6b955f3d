// C-ABI of the microscopic suspension (include/dbs.h): handle management,
// validation, launches of the fused pair-sum/Heun kernels, checkpointing and
// stroke averages.  All device work runs on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dbs.h"
#include "dbs_common.cuh"
#include "eval_kernel.cuh"
#include "flow_kernel.cuh"
#include "sd_flow_kernel.cuh"
#include "flow64_kernel.cuh"
#include "dbs_internal.cuh"

using namespace dbs;

namespace {

#ifndef DBS_BT_LARGE
#define DBS_BT_LARGE 512
#endif
#ifndef DBS_TILE_LARGE
#define DBS_TILE_LARGE 512
#endif
constexpr int BT32 = DBS_BT_LARGE;      // dumbbells per CTA (FP32C, large systems)
constexpr int TILE32 = DBS_TILE_LARGE;  // dumbbell records per shared-memory tile (FP32C)
constexpr int BT32S = 32;    // dumbbells per CTA (FP32C, S <= SMALL_S): more CTAs, spread epilogue
constexpr int TILE32S = 64;
constexpr int BT64 = 128;    // dumbbells per CTA (FP64)
constexpr int TILE64 = 64;   // dumbbell records per tile (FP64, 6 KB)
constexpr int BT64S = 32;
constexpr int TILE64S = 32;
constexpr int64_t SMALL_S = 2048;
constexpr int BT32M = 256;    // dumbbells per CTA (FP32C, SMALL_S < S <= MID_S)
constexpr int TILE32M = 256;
constexpr int64_t MID_S = 8192;
constexpr int TRIG_RING = kTrigRing;  // entries of the (sin, cos)(omega t_k) ring (power of two)
constexpr int GRAPH_STEPS = 32;  // Heun steps per captured CUDA graph

thread_local char g_create_error[256] = "";

const double PI = 3.14159265358979323846;

}  // namespace

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
int fail(dbs_suspension *h, int status, const char *fmt, ...)
{
    char *buf = h ? h->msg : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    if (h) h->status = status;
    return status;
}

// An argument or state error: the message is kept, the handle stays usable.
int refuse(dbs_suspension *h, int status, const char *msg)
{
    snprintf(h->msg, sizeof(h->msg), "%s", msg);
    return status;
}

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), e_ == cudaErrorMemoryAllocation ? DBS_E_NOMEM : DBS_E_CUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define GUARD(h)                                                  \
    do {                                                          \
        if (!(h)) return DBS_E_ARG;                               \
        if ((h)->status != DBS_OK) return (h)->status;            \
        cudaError_t e0_ = cudaSetDevice((h)->device);             \
        if (e0_ != cudaSuccess)                                   \
            return fail((h), DBS_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e0_)); \
    } while (0)

static bool all_finite(const double *a, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

static void drop_flow(dbs_suspension *h);

static bool is_f64(const dbs_suspension *h) { return h->p.precision == DBS_FP64; }

static size_t pack_bytes(const dbs_suspension *h)
{
    return (size_t)h->S * (is_f64(h) ? sizeof(DbF64) : sizeof(DbF32));
}

EvalArgs base_args(const dbs_suspension *h)
{
    EvalArgs A{};
    A.S = h->S;
    A.N = h->N;
    A.x = h->x;
    A.v0 = h->v0;
    A.Fd = h->Fd;
    A.Fext = h->Fext;
    A.lam = h->lam;
    A.sinphi = h->sinphi;
    A.cosphi = h->cosphi;
    A.trig = h->trig;
    A.trig_df = h->trig_df;
    A.trig_mask = TRIG_RING - 1;
    A.vout = h->vout;
    A.part = h->part;
    A.tickets = h->tickets;
    A.done = h->done;
    A.step = h->step;
    A.Racc = h->Racc;
    A.Rbar = h->Rbar;
    A.avg_n0 = h->avg_n0;
    A.avg_m = h->avg_m;
    A.avg_maxk = h->avg_maxk;
    A.flags = h->flags;
    A.cx = h->cx;
    A.cy = h->cy;
    A.cz = h->cz;
    A.a = h->p.a;
    A.inv6pimua = 1.0 / (6.0 * PI * h->p.mu * h->p.a);
    A.inv8pimu = 1.0 / (8.0 * PI * h->p.mu);
    A.inv8pimu_f = (float)A.inv8pimu;
    A.k0 = h->p.k0;
    A.ell = h->p.ell;
    A.omega = h->p.omega;
    A.dt = h->p.dt;
    A.c2 = (float)(2.0 * h->p.a * h->p.a / 3.0);
    A.c3 = (float)(-2.0 * h->p.a * h->p.a);
    A.overlap_r2 = (float)(4.0 * h->p.a * h->p.a);
    A.chunks = h->chunks;
    A.ib0 = 0;
    A.nib = (int)((h->S + h->bt - 1) / h->bt);
    A.apply_self = 1;
    A.noise_sigma = h->noise_sigma;
    A.noise_seed = h->noise_seed;
    return A;
}

// Launch with programmatic stream serialisation (PDL): the grid may be scheduled
// while the previous kernel on the stream is still running; the kernel waits
// for it with griddepcontrol.wait before reading its results.
template <typename K>
static void launch_pdl(K kern, int grid, int bt, size_t smem, cudaStream_t st, const EvalArgs &A)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(bt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, A);
}

// FP32C launch configuration by size: dumbbells per CTA and records per tile
// (measured on B300: 32 for small systems, where latency rules; 256 up to
// S = 8192; 512, one CTA per SM, for the largest)
static int fp32_bt(int64_t S) { return S <= SMALL_S ? BT32S : (S <= MID_S ? BT32M : BT32); }
static int fp32_tile(int bt) { return bt == BT32S ? TILE32S : (bt == BT32M ? TILE32M : TILE32); }
static const void *fp32_occ_kernel(int bt)
{
    if (bt == BT32S) return (const void *)eval_kernel<float, 1, PHASE_CORRECT, BT32S, TILE32S>;
    if (bt == BT32M) return (const void *)eval_kernel<float, 1, PHASE_CORRECT, BT32M, TILE32M>;
    return (const void *)eval_kernel<float, 1, PHASE_CORRECT, BT32, TILE32>;
}

template <typename Real, int MOB, int PHASE>
static void launch_eval_t(const EvalArgs &A, int grid, int bt, cudaStream_t st)
{
    if constexpr (sizeof(Real) == 4) {
        if (bt == BT32S)
            launch_pdl(eval_kernel<float, MOB, PHASE, BT32S, TILE32S>, grid, BT32S,
                       eval_smem_bytes<float>(BT32S, TILE32S, A.chunks), st, A);
        else if (bt == BT32M)
            launch_pdl(eval_kernel<float, MOB, PHASE, BT32M, TILE32M>, grid, BT32M,
                       eval_smem_bytes<float>(BT32M, TILE32M, A.chunks), st, A);
        else
            launch_pdl(eval_kernel<float, MOB, PHASE, BT32, TILE32>, grid, BT32,
                       eval_smem_bytes<float>(BT32, TILE32, A.chunks), st, A);
    } else {
        if (bt == BT64S)
            launch_pdl(eval_kernel<double, MOB, PHASE, BT64S, TILE64S>, grid, BT64S,
                       eval_smem_bytes<double>(BT64S, TILE64S, A.chunks), st, A);
        else
            launch_pdl(eval_kernel<double, MOB, PHASE, BT64, TILE64>, grid, BT64,
                       eval_smem_bytes<double>(BT64, TILE64, A.chunks), st, A);
    }
}

template <typename Real>
static void launch_eval_r(int mob, int phase, const EvalArgs &A, int grid, int bt, cudaStream_t st)
{
    if (mob == DBS_OSEEN) {
        if (phase == PHASE_PREDICT) launch_eval_t<Real, 0, PHASE_PREDICT>(A, grid, bt, st);
        else if (phase == PHASE_CORRECT) launch_eval_t<Real, 0, PHASE_CORRECT>(A, grid, bt, st);
        else launch_eval_t<Real, 0, PHASE_APPLY>(A, grid, bt, st);
    } else {
        if (phase == PHASE_PREDICT) launch_eval_t<Real, 1, PHASE_PREDICT>(A, grid, bt, st);
        else if (phase == PHASE_CORRECT) launch_eval_t<Real, 1, PHASE_CORRECT>(A, grid, bt, st);
        else launch_eval_t<Real, 1, PHASE_APPLY>(A, grid, bt, st);
    }
}

static void launch_eval(const dbs_suspension *h, int phase, const EvalArgs &A)
{
    if (is_f64(h)) launch_eval_r<double>(h->p.mobility, phase, A, h->grid, h->bt, h->stream);
    else launch_eval_r<float>(h->p.mobility, phase, A, h->grid, h->bt, h->stream);
}

void launch_apply(const dbs_suspension *h, const EvalArgs &A) { launch_eval(h, PHASE_APPLY, A); }

// Pack the current positions with spring (+ external) forces at t_n, or with a
// given force Fgiven, into `out`; optionally record the FP64 force in Fd.
template <typename Real>
__global__ void pack_kernel(EvalArgs A, const double *Fgiven, double *Fd_out, void *out)
{
    using Rec = typename RecOf<Real>::type;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    double xq[6];
    for (int k = 0; k < 6; ++k) xq[k] = A.x[6 * s + k];
    double F[6];
    if (Fgiven) {
        for (int k = 0; k < 6; ++k) F[k] = Fgiven[6 * s + k];
    } else {
        const double2 sc = A.trig[(*A.step) & A.trig_mask];
        const double L = rest_length(A.ell, A.lam[s], sc.x, sc.y, A.sinphi[s], A.cosphi[s]);
        spring_force(xq, xq + 3, L, A.k0, F, F + 3);
        if (A.Fext)
            for (int k = 0; k < 6; ++k) F[k] += A.Fext[6 * s + k];
    }
    if (Fd_out)
        for (int k = 0; k < 6; ++k) Fd_out[6 * s + k] = F[k];
    store_rec((Rec *)out, s, xq, F, A);
}

// ring[k & mask] = (sin, cos)(omega t_k), t_k = k dt, for k in [k0, k0 + count);
// ring_df holds the same values split into FP32 (hi, lo) pairs.
__global__ void trig_fill_kernel(double2 *ring, float4 *ring_df, int mask, int64_t k0, int count,
                                 double omega, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t k = k0 + i;
    double sw, cw;
    sincos(omega * ((double)k * dt), &sw, &cw);
    ring[k & mask] = make_double2(sw, cw);
    const float sh = (float)sw, ch = (float)cw;
    ring_df[k & mask] = make_float4(sh, (float)(sw - (double)sh), ch, (float)(cw - (double)ch));
}

__global__ void avg_start_kernel(EvalArgs A)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    for (int k = 0; k < 3; ++k) A.Racc[3 * s + k] = 0.5 * 0.5 * (A.x[6 * s + k] + A.x[6 * s + 3 + k]);
}

__global__ void set_step_kernel(int64_t *step, int64_t n) { *step = n; }

// Make the trig ring cover step indices up to k_hi.  Fills are stream-ordered
// before the launches that read them and cover TRIG_RING/2 steps at a time, so
// a fill never overwrites an entry that later-enqueued work still needs.
int ensure_trig(dbs_suspension *h, int64_t k_hi, cudaStream_t st)
{
    if (!st) st = h->stream;
    while (h->trig_hi < k_hi) {
        const int count = TRIG_RING / 2;
        trig_fill_kernel<<<(count + 127) / 128, 128, 0, st>>>(
            h->trig, h->trig_df, TRIG_RING - 1, h->trig_hi + 1, count, h->p.omega, h->p.dt);
        CK(h, cudaGetLastError());
        h->trig_hi += count;
    }
    return DBS_OK;
}

static int reset_trig(dbs_suspension *h, int64_t n)
{
    h->trig_hi = n - 1;
    return ensure_trig(h, n + 1);
}

static int repack(dbs_suspension *h);
int spring_repack(dbs_suspension *h) { return repack(h); }

static int repack(dbs_suspension *h)
{
    EvalArgs A = base_args(h);
    const int thr = 128;
    const int blocks = (int)((h->S + thr - 1) / thr);
    if (is_f64(h)) pack_kernel<double><<<blocks, thr, 0, h->stream>>>(A, nullptr, h->Fd, h->packA);
    else pack_kernel<float><<<blocks, thr, 0, h->stream>>>(A, nullptr, h->Fd, h->packA);
    CK(h, cudaGetLastError());
    return DBS_OK;
}

void drop_graph(dbs_suspension *h)
{
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

template <typename K>
static int occupancy(K kern, int bt)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bt, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return occ;
}

// Choose the j-split C and the persistent grid.  With U = iblocks * C equal
// work units over G = SMs * occupancy resident CTAs, the kernel takes
// ceil(U / G) unit-times of which U / G do work; C minimises that waste
// (ties within 1% go to the smaller C, which writes fewer partial sums).
static void choose_launch(dbs_suspension *h)
{
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const bool small = h->S <= SMALL_S;
    const bool f64 = is_f64(h);
    const int bt = f64 ? (small ? BT64S : BT64) : fp32_bt(h->S);
    const int tdb = f64 ? (small ? TILE64S : TILE64) : fp32_tile(bt);
    h->bt = bt;
    auto occ_for = [&](int64_t c) {
        int occ = 0;
        const size_t smem = f64 ? eval_smem_bytes<double>(bt, tdb, (int)c)
                                : eval_smem_bytes<float>(bt, tdb, (int)c);
        cudaError_t e;
        if (f64)
            e = small ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &occ, eval_kernel<double, 1, PHASE_CORRECT, BT64S, TILE64S>, bt, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &occ, eval_kernel<double, 1, PHASE_CORRECT, BT64, TILE64>, bt, smem);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp32_occ_kernel(bt), bt, smem);
        return (e == cudaSuccess && occ > 0) ? occ : 1;
    };
    const int64_t iblocks = (h->S + bt - 1) / bt;
    // chunks of at least 16 (small systems) / 32 dumbbell records; small FP32C
    // systems also keep C x BT within the shared-memory staging of the partials.
    // Small FP64 systems go down to one record per chunk: an FP64 instruction
    // holds its SM sub-partition for 64 cycles on this part, so a tiny system's
    // sums must be spread over many SMs (S = 16: one CTA took ~50 us per
    // evaluation, measured)
    const int64_t max_chunks = std::max<int64_t>(
        1, small ? (f64 ? h->S : std::min<int64_t>(h->S / 16, STAGE_MAX / bt)) : h->S / 32);
    // Single pass when it leaves at least 4 chunks: every CTA takes at most one
    // unit, and the fixup of each i-block reads few partials.  Otherwise (large
    // systems) many equal units over the persistent grid, C minimising
    // waves / C (the unit time scales as 1/C; ties within 1% to the smaller C).
    int64_t C = std::min<int64_t>(max_chunks, ((int64_t)sms * occ_for(max_chunks)) / iblocks);
    if (C < 4) {
        double best = 1e300;
        C = 1;
        for (int64_t c = 1; c <= max_chunks; ++c) {
            const int64_t gfull = (int64_t)sms * occ_for(c);
            const int64_t u = iblocks * c;
            const int64_t waves = (u + gfull - 1) / gfull;
            const double t = (double)waves / (double)c;
            if (t < best * 0.99) {
                best = t;
                C = c;
            }
        }
    }
    C = std::max<int64_t>(1, C);
    h->chunks = (int)C;
    h->grid = (int)std::min<int64_t>((int64_t)sms * occ_for(C), iblocks * C);
    h->sms = sms;
}

// grid for a given chunk count (same occupancy rule as choose_launch)
static int grid_for(dbs_suspension *h, int C)
{
    const bool f64 = is_f64(h);
    const bool small = h->S <= SMALL_S;
    const int bt = h->bt;
    const int tdb = f64 ? (small ? TILE64S : TILE64) : fp32_tile(bt);
    const size_t smem = f64 ? eval_smem_bytes<double>(bt, tdb, C) : eval_smem_bytes<float>(bt, tdb, C);
    int occ = 0;
    if (f64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, small ? (const void *)eval_kernel<double, 1, PHASE_CORRECT, BT64S, TILE64S>
                        : (const void *)eval_kernel<double, 1, PHASE_CORRECT, BT64, TILE64>, bt, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp32_occ_kernel(bt), bt, smem);
    occ = std::max(1, occ);
    const int64_t iblocks = (h->S + bt - 1) / bt;
    return (int)std::min<int64_t>((int64_t)h->sms * occ, iblocks * C);
}

static int alloc_all(dbs_suspension *h)
{
    const size_t v3 = sizeof(double) * 3 * h->N;
    CK(h, cudaMalloc(&h->x, v3));
    CK(h, cudaMalloc(&h->v0, v3));
    CK(h, cudaMalloc(&h->Fd, v3));
    CK(h, cudaMalloc(&h->vout, v3));
    CK(h, cudaMalloc(&h->Ftmp, v3));
    CK(h, cudaMalloc(&h->lam, sizeof(double) * h->S));
    CK(h, cudaMalloc(&h->sinphi, sizeof(double) * h->S));
    CK(h, cudaMalloc(&h->cosphi, sizeof(double) * h->S));
    CK(h, cudaMalloc(&h->packA, pack_bytes(h)));
    CK(h, cudaMalloc(&h->packB, pack_bytes(h)));
    CK(h, cudaMalloc(&h->packT, pack_bytes(h)));
    CK(h, cudaMalloc(&h->trig, sizeof(double2) * TRIG_RING));
    CK(h, cudaMalloc(&h->trig_df, sizeof(float4) * TRIG_RING));
    const int64_t iblocks = (h->S + h->bt - 1) / h->bt;
    if (h->chunks > 1) {
        const size_t pb = (size_t)h->chunks * h->S * (is_f64(h) ? 6 * sizeof(double) : 12 * sizeof(float));
        CK(h, cudaMalloc(&h->part, pb));
    }
    CK(h, cudaMalloc(&h->tickets, sizeof(unsigned) * iblocks));
    CK(h, cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * iblocks, h->stream));
    CK(h, cudaMalloc(&h->done, sizeof(unsigned)));
    CK(h, cudaMemsetAsync(h->done, 0, sizeof(unsigned), h->stream));
    CK(h, cudaMalloc(&h->step, sizeof(int64_t)));
    CK(h, cudaMemsetAsync(h->step, 0, sizeof(int64_t), h->stream));
    CK(h, cudaMalloc(&h->flags, sizeof(int)));
    CK(h, cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
    CK(h, cudaMalloc(&h->Racc, sizeof(double) * 3 * h->S));
    // passive start: lambda = 0, phi = 0 (sin 0 = 0, cos 0 = 1)
    std::vector<double> zeros(h->S, 0.0), ones(h->S, 1.0);
    CK(h, cudaMemcpy(h->lam, zeros.data(), sizeof(double) * h->S, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->sinphi, zeros.data(), sizeof(double) * h->S, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->cosphi, ones.data(), sizeof(double) * h->S, cudaMemcpyHostToDevice));
    return DBS_OK;
}

static void free_all(dbs_suspension *h)
{
    drop_graph(h);
    drop_flow(h);
    shape_free(h);
    void *bufs[] = {h->x, h->v0, h->Fd, h->Fext, h->lam, h->sinphi, h->cosphi, h->vout, h->Ftmp, h->packA,
                    h->packB, h->packT, h->trig, h->trig_df, h->part, h->tickets, h->done, h->step, h->flags,
                    h->Racc, h->Rbar};
    for (void *b : bufs)
        if (b) cudaFree(b);
}

static void set_centre(dbs_suspension *h, const double *x)
{
    double lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
    for (int64_t i = 0; i < h->N; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], x[3 * i + k]);
            hi[k] = std::max(hi[k], x[3 * i + k]);
        }
    h->cx = 0.5 * (lo[0] + hi[0]);
    h->cy = 0.5 * (lo[1] + hi[1]);
    h->cz = 0.5 * (lo[2] + hi[2]);
}

int check_flags(dbs_suspension *h)
{
    CK(h, cudaStreamSynchronize(h->stream));
    int f = 0;
    CK(h, cudaMemcpy(&f, h->flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & FLAG_OVERLAP)
        return fail(h, DBS_E_OVERLAP, "two spheres closer than 2a (RPY) or coincident");
    if (f & FLAG_NONFINITE) return fail(h, DBS_E_NONFINITE, "non-finite velocity or position");
    if (f & FLAG_TIMEOUT) return fail(h, DBS_E_TIMEOUT, "device-side wait timed out");
    if (f & FLAG_LAUNCH) return fail(h, DBS_E_CUDA, "kernel launched in a grid or cluster shape it cannot run");
    return DBS_OK;
}

// one Heun step: predictor packA -> packB, corrector packB -> packA
static void enqueue_heun(dbs_suspension *h)
{
    EvalArgs A = base_args(h);
    A.pack_in = h->packA;
    A.pack_out = h->packB;
    launch_eval(h, PHASE_PREDICT, A);
    A.pack_in = h->packB;
    A.pack_out = h->packA;
    launch_eval(h, PHASE_CORRECT, A);
}

static int build_graph(dbs_suspension *h)
{
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < GRAPH_STEPS; ++k) enqueue_heun(h);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(h, DBS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, DBS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return DBS_OK;
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *dbs_version(void) { return "dbs 0.1 (sm_103a)"; }

const char *dbs_status_string(int s)
{
    switch (s) {
    case DBS_OK: return "DBS_OK";
    case DBS_E_ARG: return "DBS_E_ARG";
    case DBS_E_NOMEM: return "DBS_E_NOMEM";
    case DBS_E_CUDA: return "DBS_E_CUDA";
    case DBS_E_OVERLAP: return "DBS_E_OVERLAP";
    case DBS_E_NONFINITE: return "DBS_E_NONFINITE";
    case DBS_E_TIMEOUT: return "DBS_E_TIMEOUT";
    case DBS_E_STATE: return "DBS_E_STATE";
    default: return "DBS_E_UNKNOWN";
    }
}

const char *dbs_last_error(const dbs_suspension *h) { return h ? h->msg : g_create_error; }

int dbs_create_suspension(const dbs_params *p, const double *x0, dbs_suspension **out)
{
    if (!out) return fail(nullptr, DBS_E_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !x0) return fail(nullptr, DBS_E_ARG, "params or x0 is NULL");
    if (p->S < 1 || p->S > (int64_t(1) << 29)) return fail(nullptr, DBS_E_ARG, "S out of range (1 .. 2^29)");
    const double vals[] = {p->a, p->mu, p->k0, p->ell, p->omega, p->dt};
    if (!all_finite(vals, 6)) return fail(nullptr, DBS_E_ARG, "non-finite parameter");
    if (!(p->a > 0 && p->mu > 0 && p->omega > 0 && p->dt > 0 && p->k0 >= 0))
        return fail(nullptr, DBS_E_ARG, "a, mu, omega, dt must be > 0 and k0 >= 0");
    if (!(p->ell > 2 * p->a)) return fail(nullptr, DBS_E_ARG, "ell must exceed 2a (Sec. II)");
    if (p->mobility != DBS_OSEEN && p->mobility != DBS_RPY)
        return fail(nullptr, DBS_E_ARG, "mobility must be DBS_OSEEN or DBS_RPY");
    if (p->precision != DBS_FP32C && p->precision != DBS_FP64)
        return fail(nullptr, DBS_E_ARG, "precision must be DBS_FP32C or DBS_FP64");
    if (p->flags != 0) return fail(nullptr, DBS_E_ARG, "flags must be 0");
    if (!all_finite(x0, 6 * p->S)) return fail(nullptr, DBS_E_ARG, "non-finite x0");

    dbs_suspension *h = new (std::nothrow) dbs_suspension();
    if (!h) return fail(nullptr, DBS_E_NOMEM, "host allocation failed");
    h->p = *p;
    h->S = p->S;
    h->N = 2 * p->S;
    int dev = p->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    h->device = dev;
    int rc = DBS_OK;
    auto bail = [&](int r) {
        snprintf(g_create_error, sizeof(g_create_error), "%s", h->msg);
        free_all(h);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return r;
    };
    if (cudaSetDevice(dev) != cudaSuccess) {
        fail(h, DBS_E_CUDA, "cudaSetDevice(%d) failed", dev);
        return bail(DBS_E_CUDA);
    }
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(h, DBS_E_CUDA, "stream creation failed");
            return bail(DBS_E_CUDA);
        }
        h->own_stream = true;
    }
    choose_launch(h);
    if ((rc = alloc_all(h)) != DBS_OK) return bail(rc);
    set_centre(h, x0);
    if ((rc = reset_trig(h, 0)) != DBS_OK) return bail(rc);
    if (cudaMemcpyAsync(h->x, x0, sizeof(double) * 3 * h->N, cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess) {
        fail(h, DBS_E_CUDA, "upload of x0 failed");
        return bail(DBS_E_CUDA);
    }
    if ((rc = repack(h)) != DBS_OK) return bail(rc);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        fail(h, DBS_E_CUDA, "create: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(DBS_E_CUDA);
    }
    *out = h;
    return DBS_OK;
}

int dbs_destroy(dbs_suspension *h)
{
    if (!h) return DBS_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->solo) solo_destroy(h);
    free_all(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return DBS_OK;
}

int dbs_set_stroke(dbs_suspension *h, const double *lambda, const double *phase)
{
    GUARD(h);
    if (!lambda || !phase) return DBS_E_ARG;
    if (!all_finite(lambda, h->S) || !all_finite(phase, h->S)) return DBS_E_ARG;
    double lmax = 0;
    for (int64_t s = 0; s < h->S; ++s) lmax = std::max(lmax, std::fabs(lambda[s]));
    if (!(h->p.ell > 2 * h->p.a + lmax)) return DBS_E_ARG;  // Sec. II: ell > 2a + lambda
    h->lam_max = lmax;
    std::vector<double> sp(h->S), cp(h->S);
    for (int64_t s = 0; s < h->S; ++s) {
        sp[s] = std::sin(phase[s]);
        cp[s] = std::cos(phase[s]);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->lam, lambda, sizeof(double) * h->S, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->sinphi, sp.data(), sizeof(double) * h->S, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->cosphi, cp.data(), sizeof(double) * h->S, cudaMemcpyHostToDevice));
    int rc = repack(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return DBS_OK;
}

int dbs_set_noise(dbs_suspension *h, double kT, uint64_t seed)
{
    GUARD(h);
    if (!(kT >= 0.0) || !std::isfinite(kT)) return DBS_E_ARG;
    if (h->dyn == DBS_DYN_SHAPE && kT > 0.0) return refuse(h, DBS_E_STATE, "no noise with shape-driven dynamics");
    if (h->path == DBS_PATH_COOP && is_f64(h) && kT > 0.0)
        return refuse(h, DBS_E_STATE, "cooperative FP64 path: no additive noise (use the grid path)");
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);
    h->noise_sigma = std::sqrt(2.0 * kT * h->p.dt / (6.0 * PI * h->p.mu * h->p.a));
    h->noise_seed = seed;
    // the cooperative path runs a separate kernel instantiation with noise: re-derive its split
    if (h->path == DBS_PATH_COOP) return coop_setup(h);
    return DBS_OK;
}

int dbs_set_external_force(dbs_suspension *h, const double *F)
{
    GUARD(h);
    if (h->dyn == DBS_DYN_SHAPE && F) return refuse(h, DBS_E_STATE, "no external force with shape-driven dynamics");
    if (F && !all_finite(F, 3 * h->N)) return DBS_E_ARG;
    drop_graph(h);
    if (!F) {
        if (h->Fext) {
            CK(h, cudaStreamSynchronize(h->stream));
            cudaFree(h->Fext);
            h->Fext = nullptr;
        }
    } else {
        if (!h->Fext) CK(h, cudaMalloc(&h->Fext, sizeof(double) * 3 * h->N));
        CK(h, cudaMemcpyAsync(h->Fext, F, sizeof(double) * 3 * h->N, cudaMemcpyHostToDevice, h->stream));
    }
    int rc = repack(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return DBS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// cooperative dataflow path (flow_kernel)
// ---------------------------------------------------------------------------
constexpr int FLOW_MAX_T = 32;        // dumbbells per CTA at most (FP32C)
constexpr int FLOW64_MAX_T = 4;       // dumbbells per CTA at most (FP64)
constexpr int64_t FLOW_MAX_S = 4096;  // all records of a suspension in one CTA's shared memory
constexpr int FLOW_MAX_STEPS = 1024;  // Heun steps per launch

// FP32C: flow_kernel, 256 threads, 3 record words per dumbbell; FP64:
// flow64_kernel, 128 threads, 6 record words per dumbbell
static int flow_threads(const dbs_suspension *h) { return is_f64(h) ? FLOW64_NT : FLOW_NT; }
static size_t flow_words(const dbs_suspension *h)
{
    return 2 * (size_t)h->flow_G * h->flow_T * (is_f64(h) ? 6 : 3);
}

static void drop_flow(dbs_suspension *h)
{
    cudaFree(h->ll_rec);
    h->ll_rec = nullptr;
}

template <int MOB, bool NOISE>
static const void *flow_pick(int T)
{
    switch (T) {
    case 1: return (const void *)flow_kernel<MOB, 1, NOISE>;
    case 2: return (const void *)flow_kernel<MOB, 2, NOISE>;
    case 4: return (const void *)flow_kernel<MOB, 4, NOISE>;
    case 8: return (const void *)flow_kernel<MOB, 8, NOISE>;
    case 16: return (const void *)flow_kernel<MOB, 16, NOISE>;
    case 32: return (const void *)flow_kernel<MOB, 32, NOISE>;
    default: return nullptr;
    }
}

template <int MOB>
static const void *flow64_pick(int T)
{
    switch (T) {
    case 1: return (const void *)flow64_kernel<MOB, 1>;
    case 2: return (const void *)flow64_kernel<MOB, 2>;
    case 4: return (const void *)flow64_kernel<MOB, 4>;
    default: return nullptr;
    }
}

template <int MOB>
static const void *sd_pick(int T)
{
    switch (T) {
    case 1: return (const void *)sd_flow_kernel<MOB, 1>;
    case 2: return (const void *)sd_flow_kernel<MOB, 2>;
    case 4: return (const void *)sd_flow_kernel<MOB, 4>;
    case 8: return (const void *)sd_flow_kernel<MOB, 8>;
    case 16: return (const void *)sd_flow_kernel<MOB, 16>;
    case 32: return (const void *)sd_flow_kernel<MOB, 32>;
    default: return nullptr;
    }
}

static const void *flow_fn(const dbs_suspension *h, int T)
{
    if (h->dyn == DBS_DYN_SHAPE && !is_f64(h)) return h->p.mobility == DBS_OSEEN ? sd_pick<0>(T) : sd_pick<1>(T);
    if (is_f64(h)) return h->p.mobility == DBS_OSEEN ? flow64_pick<0>(T) : flow64_pick<1>(T);
    const bool noise = h->noise_sigma > 0.0;
    if (h->p.mobility == DBS_OSEEN) return noise ? flow_pick<0, true>(T) : flow_pick<0, false>(T);
    return noise ? flow_pick<1, true>(T) : flow_pick<1, false>(T);
}

// dynamic shared memory of the cooperative kernel: every record of the suspension
static size_t flow_smem(const dbs_suspension *h, int G, int T)
{
    return (size_t)G * T * (is_f64(h) ? sizeof(DbF64) : sizeof(DbF32));
}

static cudaLaunchConfig_t flow_config(const dbs_suspension *h, int G, int T, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(flow_threads(h));
    cfg.dynamicSmemBytes = flow_smem(h, G, T);
    cfg.stream = h->stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Split: T dumbbells per CTA, the smallest power of two (at least the largest
// one not above a dbs_set_chunks request; FP32C: 16 for S <= 16, so that one CTA
// holds a tiny system, else at least 2; FP64 spreads even a tiny system over the
// SMs, whose FP64 pipes are the bound) for which all ceil(S / T) CTAs fit the
// SMs, one CTA each.
int coop_setup(dbs_suspension *h)
{
    const bool f64 = is_f64(h);
    if (h->S > FLOW_MAX_S) return refuse(h, DBS_E_ARG, "cooperative path needs S <= 4096");
    if (h->dyn == DBS_DYN_SHAPE && f64)
        return refuse(h, DBS_E_ARG, "cooperative shape-driven dynamics: FP32C only (FP64 runs on the grid path)");
    if (f64 && h->noise_sigma > 0.0)
        return refuse(h, DBS_E_ARG, "cooperative FP64 path: no additive noise (use the grid path)");
    const int max_t = f64 ? FLOW64_MAX_T : FLOW_MAX_T;
    int coop = 0, sms = 0, optin = 0;
    CK(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    CK(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (!coop) return refuse(h, DBS_E_ARG, "device without cooperative launch");
    // tiny FP32C systems: one CTA holds all dumbbells and no record leaves it
    // FP32C: at least two dumbbells per CTA (S = 64 / 128 / 148: 3.51 / 3.80 / 4.39
    // us per Heun step with one, 3.30 / 3.47 / 3.70 with two, measured)
    int T = f64 ? 1 : (h->S <= 16 ? 16 : 2);
    if (h->flow_creq > 0) {
        T = 1;
        while (2 * T <= std::min(h->flow_creq, max_t)) T *= 2;
    }
    int G = 0;
    for (;; T *= 2) {
        if (T > max_t) return refuse(h, DBS_E_ARG, "cooperative path: grid does not fit the device");
        G = (int)((h->S + T - 1) / T);
        if (G > sms) continue;
        const void *k = flow_fn(h, T);
        // the limit is a property of the kernel, shared by every handle that launches
        // it: set it to all the device allows (never to this handle's need, which
        // would shrink it under a larger suspension set up earlier)
        cudaFuncAttributes fa{};
        CK(h, cudaFuncGetAttributes(&fa, k));
        if (flow_smem(h, G, T) + fa.sharedSizeBytes > (size_t)optin) continue;
        CK(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   optin - (int)fa.sharedSizeBytes));
        int occ = 0;
        CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, flow_threads(h), flow_smem(h, G, T)));
        if ((int64_t)occ * sms >= G) break;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    drop_flow(h);
    h->flow_T = T;
    h->flow_G = G;
    const size_t words = flow_words(h);
    CK(h, cudaMalloc(&h->ll_rec, words * sizeof(ulonglong2)));
    // a cleared buffer carries parity bit 0 everywhere: the evaluation counter
    // starts at a multiple of 4, whose first two evaluations expect bit 1
    CK(h, cudaMemsetAsync(h->ll_rec, 0, words * sizeof(ulonglong2), h->stream));
    h->flow_base = 0;
    return DBS_OK;
}

static int coop_step(dbs_suspension *h, int64_t n)
{
    int64_t left = n;
    while (left > 0) {
        const int K = (int)std::min<int64_t>(left, FLOW_MAX_STEPS);
        int rc = ensure_trig(h, h->n_host + K + 1);
        if (rc) return rc;
        const EvalArgs A = base_args(h);
        FlowArgs P{};
        P.rec = h->ll_rec;
        P.pack = (DbF32 *)h->packA;
        P.n0 = h->n_host;
        P.G = h->flow_G + h->flow_test_dG;
        P.K = K;
        P.base = h->flow_base;
        P.timeout_ns = 1000000000ull;
        Flow64Args P64{};
        P64.rec = P.rec;
        P64.pack = (DbF64 *)h->packA;
        P64.n0 = P.n0;
        P64.G = P.G;
        P64.K = P.K;
        P64.base = P.base;
        P64.timeout_ns = P.timeout_ns;
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = flow_config(h, h->flow_G, h->flow_T, attr);
        const bool sd = h->dyn == DBS_DYN_SHAPE;
        const int M = h->sd_iters;   // shape-driven: pair sums per evaluation point
        void *args[] = {(void *)&A, is_f64(h) ? (void *)&P64 : (void *)&P, (void *)&M};
        cudaError_t e = cudaLaunchKernelExC(&cfg, flow_fn(h, h->flow_T), args);
        if (e != cudaSuccess) return fail(h, DBS_E_CUDA, "cooperative launch: %s", cudaGetErrorString(e));
        // the evaluation counter runs on from launch to launch (2K evaluations per
        // launch, 2MK for the shape-driven kernel, so it stays even; modulo 2^32 it
        // keeps its residue mod 4, which is all the parity bits depend on)
        h->flow_base += (unsigned)(2 * K * (sd ? M : 1));
        h->n_host += K;
        left -= K;
    }
    // shape-driven: the one-launch records and FP64 forces of the current state
    if (h->dyn == DBS_DYN_SHAPE && n > 0) return shape_finish(h);
    return DBS_OK;
}


extern "C" {

int dbs_step(dbs_suspension *h, int64_t n)
{
    GUARD(h);
    if (n < 0) return DBS_E_ARG;
    if (h->shard_nib > 0) return refuse(h, DBS_E_STATE, "a row-sharded handle steps with dbs_shard_eval");
    if (h->solo) return solo_step(h, n);
    if (h->path == DBS_PATH_COOP) return coop_step(h, n);
    if (h->dyn == DBS_DYN_SHAPE) return shape_step(h, n);
    int64_t left = n, k = h->n_host;
    int rc;
    if (left >= GRAPH_STEPS) {
        if (!h->graph && (rc = build_graph(h)) != DBS_OK) return rc;
        while (left >= GRAPH_STEPS) {
            if ((rc = ensure_trig(h, k + GRAPH_STEPS)) != DBS_OK) return rc;
            CK(h, cudaGraphLaunch(h->graph, h->stream));
            left -= GRAPH_STEPS;
            k += GRAPH_STEPS;
        }
    }
    for (; left > 0; --left, ++k) {
        if ((rc = ensure_trig(h, k + 1)) != DBS_OK) return rc;
        enqueue_heun(h);
    }
    CK(h, cudaGetLastError());
    h->n_host += n;
    return DBS_OK;
}

int dbs_sync(dbs_suspension *h)
{
    GUARD(h);
    return check_flags(h);
}

static int apply_to_host(dbs_suspension *h, const void *pack, double *Fd, int self, double *out)
{
    EvalArgs A = base_args(h);
    A.pack_in = pack;
    A.Fd = Fd;
    A.apply_self = self;
    launch_eval(h, PHASE_APPLY, A);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(out, h->vout, sizeof(double) * 3 * h->N, cudaMemcpyDeviceToHost, h->stream));
    return check_flags(h);
}

int dbs_velocities(dbs_suspension *h, double *v)
{
    GUARD(h);
    if (!v) return DBS_E_ARG;
    return apply_to_host(h, h->packA, h->Fd, 1, v);
}

int dbs_interaction(dbs_suspension *h, double *u)
{
    GUARD(h);
    if (!u) return DBS_E_ARG;
    return apply_to_host(h, h->packA, h->Fd, 0, u);
}

int dbs_mobility_apply(dbs_suspension *h, const double *F, double *v)
{
    GUARD(h);
    if (!F || !v) return DBS_E_ARG;
    if (!all_finite(F, 3 * h->N)) return DBS_E_ARG;
    CK(h, cudaMemcpyAsync(h->Ftmp, F, sizeof(double) * 3 * h->N, cudaMemcpyHostToDevice, h->stream));
    EvalArgs A = base_args(h);
    const int thr = 128, blocks = (int)((h->S + thr - 1) / thr);
    if (is_f64(h)) pack_kernel<double><<<blocks, thr, 0, h->stream>>>(A, h->Ftmp, nullptr, h->packT);
    else pack_kernel<float><<<blocks, thr, 0, h->stream>>>(A, h->Ftmp, nullptr, h->packT);
    CK(h, cudaGetLastError());
    return apply_to_host(h, h->packT, h->Ftmp, 1, v);
}

int dbs_set_chunks(dbs_suspension *h, int32_t chunks)
{
    GUARD(h);
    // grid path: at least 8 dumbbell records per chunk; cooperative path: the
    // split request (j-chunks, or dumbbells per CTA) is at most 16
    const int64_t cmax = h->path == DBS_PATH_COOP ? 16 : std::max<int64_t>(1, h->S / 8);
    if (chunks < 0 || chunks > cmax) return DBS_E_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);
    if (chunks == 0) {
        choose_launch(h);
    } else {
        h->chunks = chunks;
        h->grid = grid_for(h, chunks);
    }
    if (h->part) {
        cudaFree(h->part);
        h->part = nullptr;
    }
    if (h->chunks > 1) {
        const size_t pb = (size_t)h->chunks * h->S * (is_f64(h) ? 6 * sizeof(double) : 12 * sizeof(float));
        CK(h, cudaMalloc(&h->part, pb));
    }
    if (h->path == DBS_PATH_COOP) {
        h->flow_creq = chunks;
        return coop_setup(h);
    }
    return DBS_OK;
}

int dbs_get_launch(dbs_suspension *h, int32_t *bt, int32_t *chunks, int32_t *grid)
{
    GUARD(h);
    const bool coop = h->path == DBS_PATH_COOP;
    if (bt) *bt = coop ? h->flow_T : h->bt;
    if (chunks) *chunks = coop ? 1 : h->chunks;
    if (grid) *grid = coop ? h->flow_G : h->grid;
    return DBS_OK;
}

// ---- one suspension split by target rows (several processes) ------------------
int dbs_shard_rows(int64_t S, int32_t rows_per_block, int32_t nranks, int32_t rank, int64_t *row0,
                   int64_t *row1)
{
    if (S < 1 || rows_per_block < 1 || nranks < 1 || rank < 0 || rank >= nranks || !row0 || !row1)
        return DBS_E_ARG;
    const int64_t nb = (S + rows_per_block - 1) / rows_per_block;   // i-blocks
    if (nranks > nb) return DBS_E_ARG;                               // every rank needs a block
    const int64_t b0 = nb * rank / nranks, b1 = nb * (rank + 1) / nranks;   // sizes differ by <= 1
    *row0 = b0 * rows_per_block;
    *row1 = std::min<int64_t>(S, b1 * rows_per_block);
    return DBS_OK;
}

int dbs_shard_set(dbs_suspension *h, int32_t nranks, int32_t rank, int64_t *row0, int64_t *row1)
{
    GUARD(h);
    if (h->path != DBS_PATH_GRID || h->dyn != DBS_DYN_SPRING || h->solo)
        return refuse(h, DBS_E_STATE, "row sharding needs the grid path and spring dynamics");
    int64_t r0 = 0, r1 = 0;
    int rc = dbs_shard_rows(h->S, h->bt, nranks, rank, &r0, &r1);
    if (rc) return refuse(h, rc, "no row block for this rank (more ranks than i-blocks?)");
    h->shard_ib0 = (int)(r0 / h->bt);
    h->shard_nib = (int)((r1 - r0 + h->bt - 1) / h->bt);
    h->shard_grid = (int)std::min<int64_t>(h->grid, (int64_t)h->shard_nib * h->chunks);
    if (row0) *row0 = r0;
    if (row1) *row1 = r1;
    return DBS_OK;
}

int dbs_shard_eval(dbs_suspension *h, int32_t phase)
{
    GUARD(h);
    if (h->shard_nib < 1) return refuse(h, DBS_E_STATE, "dbs_shard_set first");
    if (phase != 0 && phase != 1) return DBS_E_ARG;
    int rc = ensure_trig(h, h->n_host + 1);
    if (rc) return rc;
    EvalArgs A = base_args(h);
    A.ib0 = h->shard_ib0;
    A.nib = h->shard_nib;
    A.pack_in = phase == 0 ? h->packA : h->packB;    // predictor: x_n -> records of x~
    A.pack_out = phase == 0 ? h->packB : h->packA;   // corrector: x~ -> records of x_{n+1}
    const int ph = phase == 0 ? PHASE_PREDICT : PHASE_CORRECT;
    if (is_f64(h)) launch_eval_r<double>(h->p.mobility, ph, A, h->shard_grid, h->bt, h->stream);
    else launch_eval_r<float>(h->p.mobility, ph, A, h->shard_grid, h->bt, h->stream);
    CK(h, cudaGetLastError());
    if (phase == 1) h->n_host += 1;
    return DBS_OK;
}

int dbs_shard_buffers(dbs_suspension *h, void **records_a, void **records_b, int64_t *record_bytes)
{
    GUARD(h);
    if (records_a) *records_a = h->packA;
    if (records_b) *records_b = h->packB;
    if (record_bytes) *record_bytes = (int64_t)(is_f64(h) ? sizeof(DbF64) : sizeof(DbF32));
    return DBS_OK;
}

int dbs_test_set_flow_tag(dbs_suspension *h, uint32_t tag)
{
    GUARD(h);
    if (h->path != DBS_PATH_COOP || !h->ll_rec) return DBS_E_STATE;
    // a cleared buffer and a counter at a multiple of 4, as after the path's set-up
    CK(h, cudaMemsetAsync(h->ll_rec, 0, flow_words(h) * sizeof(ulonglong2), h->stream));
    h->flow_base = tag & ~3u;
    return DBS_OK;
}

int dbs_test_flow_misshape(dbs_suspension *h)
{
    GUARD(h);
    if (h->path != DBS_PATH_COOP) return DBS_E_STATE;
    // one Heun step whose kernel is told it has one CTA more than it was launched with
    h->flow_test_dG = 1;
    const int rc = coop_step(h, 1);
    h->flow_test_dG = 0;
    if (rc) return rc;
    return check_flags(h);
}

int dbs_test_wait_timeout(int32_t timeout_ms, int32_t *status)
{
    if (!status || timeout_ms < 1 || timeout_ms > 10000) return DBS_E_ARG;
    void *w = nullptr;
    if (cudaMalloc(&w, 32) != cudaSuccess) return DBS_E_NOMEM;
    cudaError_t e = cudaMemset(w, 0, 32);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 32>>>((const ulonglong2 *)w, (int *)((char *)w + 16),
                                       (unsigned long long)timeout_ms * 1000000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flags, (char *)w + 16, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(w);
    if (e != cudaSuccess) return DBS_E_CUDA;
    *status = (flags & FLAG_TIMEOUT) ? DBS_E_TIMEOUT : DBS_OK;
    return DBS_OK;
}

int dbs_velocities_device(dbs_suspension *h, double *v_dev)
{
    GUARD(h);
    if (!v_dev) return DBS_E_ARG;
    EvalArgs A = base_args(h);
    A.pack_in = h->packA;
    A.vout = v_dev;
    launch_eval(h, PHASE_APPLY, A);
    CK(h, cudaGetLastError());
    return DBS_OK;
}

int dbs_step_timed(dbs_suspension *h, int64_t n, double *mean_ms)
{
    GUARD(h);
    if (h->dyn == DBS_DYN_SHAPE) return refuse(h, DBS_E_STATE, "dbs_step_timed times the spring model");
    if (n < 1 || !mean_ms) return DBS_E_ARG;
    cudaEvent_t ev[4];
    for (auto &e : ev) CK(h, cudaEventCreate(&e));
    double total = 0;
    for (int64_t k = 0; k < n; ++k) {
        int rc = ensure_trig(h, h->n_host + k + 1);
        if (rc) return rc;
        EvalArgs A = base_args(h);
        A.pack_in = h->packA;
        A.pack_out = h->packB;
        CK(h, cudaEventRecord(ev[0], h->stream));
        launch_eval(h, PHASE_PREDICT, A);
        CK(h, cudaGetLastError());
        CK(h, cudaEventRecord(ev[1], h->stream));
        A.pack_in = h->packB;
        A.pack_out = h->packA;
        CK(h, cudaEventRecord(ev[2], h->stream));
        launch_eval(h, PHASE_CORRECT, A);
        CK(h, cudaGetLastError());
        CK(h, cudaEventRecord(ev[3], h->stream));
        CK(h, cudaEventSynchronize(ev[3]));
        float a = 0, b = 0;
        CK(h, cudaEventElapsedTime(&a, ev[0], ev[1]));
        CK(h, cudaEventElapsedTime(&b, ev[2], ev[3]));
        total += a + b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    h->n_host += n;
    *mean_ms = total / (2.0 * n);
    return check_flags(h);
}

int dbs_positions(dbs_suspension *h, double *x)
{
    GUARD(h);
    if (!x) return DBS_E_ARG;
    CK(h, cudaMemcpyAsync(x, h->x, sizeof(double) * 3 * h->N, cudaMemcpyDeviceToHost, h->stream));
    return check_flags(h);
}

int dbs_positions_device(dbs_suspension *h, double *x_dev)
{
    GUARD(h);
    if (!x_dev) return DBS_E_ARG;
    CK(h, cudaMemcpyAsync(x_dev, h->x, sizeof(double) * 3 * h->N, cudaMemcpyDeviceToDevice, h->stream));
    return DBS_OK;
}

int dbs_get_time(dbs_suspension *h, int64_t *n, double *t)
{
    GUARD(h);
    if (n) *n = h->n_host;
    if (t) *t = (double)h->n_host * h->p.dt;
    return DBS_OK;
}

int dbs_get_state(dbs_suspension *h, double *x, int64_t *n)
{
    GUARD(h);
    if (n) *n = h->n_host;
    if (x) return dbs_positions(h, x);
    return DBS_OK;
}

int dbs_set_state(dbs_suspension *h, const double *x, int64_t n)
{
    GUARD(h);
    if (!x || n < 0 || !all_finite(x, 3 * h->N)) return DBS_E_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpyAsync(h->x, x, sizeof(double) * 3 * h->N, cudaMemcpyHostToDevice, h->stream));
    set_step_kernel<<<1, 1, 0, h->stream>>>(h->step, n);
    CK(h, cudaGetLastError());
    h->n_host = n;
    int rc = reset_trig(h, n);
    if (rc) return rc;
    rc = h->dyn == DBS_DYN_SHAPE ? shape_reset(h) : repack(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return DBS_OK;
}

int dbs_enable_period_average(dbs_suspension *h, int64_t m, int64_t max_periods)
{
    GUARD(h);
    if (m < 0 || (m > 0 && max_periods < 1)) return DBS_E_ARG;
    drop_graph(h);
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->Rbar) {
        cudaFree(h->Rbar);
        h->Rbar = nullptr;
    }
    h->avg_m = m;
    h->avg_maxk = m > 0 ? max_periods : 0;
    h->avg_n0 = h->n_host;
    if (m > 0) {
        CK(h, cudaMalloc(&h->Rbar, sizeof(double) * 3 * h->S * max_periods));
        EvalArgs A = base_args(h);
        const int thr = 128, blocks = (int)((h->S + thr - 1) / thr);
        avg_start_kernel<<<blocks, thr, 0, h->stream>>>(A);
        CK(h, cudaGetLastError());
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return DBS_OK;
}

int dbs_period_count(dbs_suspension *h, int64_t *count)
{
    GUARD(h);
    if (!count) return DBS_E_ARG;
    *count = h->avg_m > 0 ? std::min(h->avg_maxk, (h->n_host - h->avg_n0) / h->avg_m) : 0;
    return DBS_OK;
}

int dbs_period_averages(dbs_suspension *h, int64_t k0, int64_t count, double *Rbar)
{
    GUARD(h);
    int64_t have = 0;
    dbs_period_count(h, &have);
    if (!Rbar || k0 < 0 || count < 0 || k0 + count > have) return DBS_E_ARG;
    CK(h, cudaMemcpyAsync(Rbar, h->Rbar + 3 * h->S * k0, sizeof(double) * 3 * h->S * count,
                          cudaMemcpyDeviceToHost, h->stream));
    return check_flags(h);
}

int dbs_period_average_device(dbs_suspension *h, int64_t k, const double **Rbar_dev)
{
    GUARD(h);
    int64_t have = 0;
    dbs_period_count(h, &have);
    if (!Rbar_dev || k < 0 || k >= have) return DBS_E_ARG;
    *Rbar_dev = h->Rbar + 3 * h->S * k;
    return DBS_OK;
}

}  // extern "C"
