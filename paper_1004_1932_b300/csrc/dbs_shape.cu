// Shape-driven dumbbells (Appendix A.2, "Three-dimensional case"), the
// infinitely stiff limit of the spring model: the length of dumbbell s is the
// prescribed L^s(t) of Eq. (4), and internal forces F^{s1} = f^s N^s,
// F^{s2} = -f^s N^s along the axis keep it so,
//   dL^s/dt = N^s . (dX^{s2}/dt - dX^{s1}/dt).
// The forces come from the paper's iteration
//   f^s_(n) = [dL^s/dt - sum_{r != s} b^{sr} f^r_(n-1)] / b^{ss},  f_(0) = 0,
// with the exact tensors of Eq. (3) (no far-field expansion).  One iteration
// is one pair sum: sum_{r != s} b^{sr} f^r = N^s . (u^{s2} - u^{s1}) - 2 f^s h_c,
// where u = sum_{j != i} H_ij F_j is the interaction part of Eq. (3) for the
// forces of iterate n-1 (the grid path's pair-sum kernel in its APPLY phase)
// and 2 f^s h_c, h_c = N^s . H(L N^s) . N^s, removes the dumbbell's coupling to
// itself; b^{ss} = 2 h_c - 2/(6 pi mu a).  Then v = H F (Eq. (3)) gives
//   dR^s/dt = (v^{s1} + v^{s2})/2,  dN^s/dt = (I - N N^T)(v^{s2} - v^{s1}) / L^s,
// integrated by Heun on (R, N) with N renormalised and the spheres placed at
// R -/+ N L(t)/2.  Grid path here (FP32C or FP64); the cooperative path (FP32C)
// runs the same iteration in sd_flow_kernel.  No external force or noise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "dbs.h"
#include "dbs_common.cuh"
#include "dbs_internal.cuh"

using namespace dbs;

namespace {

// Programmatic dependent launch: the step's small kernels may be scheduled
// while the previous kernel on the stream finishes; each waits for it (and its
// memory) before reading anything, then lets the next one be scheduled.  Both
// are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_sync()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t sd_launch(void (*kern)(KArgs...), int blocks, int thr, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(thr);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

__global__ void sd_set_step_kernel(int64_t *step, int64_t n)
{
    pdl_sync();
    *step = n;
}

// Work arrays of one handle, carved from h->sd_buf (doubles).
struct SdBuf {
    double *f, *bss, *hc, *L, *Ld;  // [S] each
    double *N;                      // [S][3] axis at the current evaluation point
    double *R0, *N0;                // [S][3] centre and axis at x_n
    double *rate0;                  // [S][6] predictor (dR/dt, dN/dt)
    double *xt;                     // [N][3] predictor point
};

size_t sd_doubles(int64_t S) { return (size_t)S * (5 + 3 + 6 + 6 + 12); }

SdBuf sd_view(const dbs_suspension *h)
{
    const int64_t S = h->S;
    double *b = h->sd_buf;
    SdBuf B;
    B.f = b;
    B.bss = b + S;
    B.hc = b + 2 * S;
    B.L = b + 3 * S;
    B.Ld = b + 4 * S;
    B.N = b + 5 * S;
    B.R0 = b + 8 * S;
    B.N0 = b + 11 * S;
    B.rate0 = b + 14 * S;
    B.xt = b + 20 * S;
    return B;
}

__device__ __forceinline__ double2 rest_and_rate(const EvalArgs &A, int64_t s, int64_t k)
{
    // L and dL/dt at t_k: ell + lam sin(wt + phi), lam w cos(wt + phi)
    const double2 sc = A.trig[k & A.trig_mask];
    const double sp = A.sinphi[s], cp = A.cosphi[s];
    const double L = rest_length(A.ell, A.lam[s], sc.x, sc.y, sp, cp);
    const double Ld = A.lam[s] * A.omega * fma(sc.y, cp, -sc.x * sp);
    return make_double2(L, Ld);
}

// The axis, h_c, b^{ss}, L, dL/dt at the point P (time index k), the first
// iterate f_(1) = dL/dt / b^{ss}, and the records / FP64 forces of f_(1).
template <typename Real>
__global__ void sd_begin_kernel(EvalArgs A, const double *P, int64_t k, SdBuf B, int rpy, void *pack)
{
    pdl_sync();
    using Rec = typename RecOf<Real>::type;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    double xq[6];
    for (int j = 0; j < 6; ++j) xq[j] = P[6 * s + j];
    const double e[3] = {xq[3] - xq[0], xq[4] - xq[1], xq[5] - xq[2]};
    const double d = sqrt(fma(e[2], e[2], fma(e[1], e[1], e[0] * e[0])));
    // h_c = N.H(d N).N of Eq. (3b): 1/(4 pi mu d), minus a^2/(6 pi mu d^3) under RPY
    double hc = 2.0 * A.inv8pimu / d;
    if (rpy) hc -= A.a * A.a * A.a * A.inv6pimua / (d * d * d);
    const double bss = 2.0 * hc - 2.0 * A.inv6pimua;
    const double2 LLd = rest_and_rate(A, s, k);
    const double f = LLd.y / bss;
    double F[6];
    for (int j = 0; j < 3; ++j) {
        const double n = e[j] / d;
        B.N[3 * s + j] = n;
        F[j] = f * n;
        F[3 + j] = -f * n;
    }
    B.f[s] = f;
    B.bss[s] = bss;
    B.hc[s] = hc;
    B.L[s] = LLd.x;
    B.Ld[s] = LLd.y;
    for (int j = 0; j < 6; ++j) A.Fd[6 * s + j] = F[j];
    store_rec((Rec *)pack, s, xq, F, A);
}

// One iteration from the interaction u of the previous iterate's forces.
template <typename Real>
__global__ void sd_iter_kernel(EvalArgs A, const double *P, SdBuf B, const double *u, void *pack)
{
    pdl_sync();
    using Rec = typename RecOf<Real>::type;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    const double *u1 = u + 6 * s, *u2 = u1 + 3, *n = B.N + 3 * s;
    double nu = 0.0;
    for (int j = 0; j < 3; ++j) nu = fma(n[j], u2[j] - u1[j], nu);
    const double others = nu - 2.0 * B.f[s] * B.hc[s];   // sum_{r != s} b^{sr} f^r
    const double f = (B.Ld[s] - others) / B.bss[s];
    B.f[s] = f;
    double xq[6], F[6];
    for (int j = 0; j < 6; ++j) xq[j] = P[6 * s + j];
    for (int j = 0; j < 3; ++j) {
        F[j] = f * n[j];
        F[3 + j] = -f * n[j];
    }
    for (int j = 0; j < 6; ++j) A.Fd[6 * s + j] = F[j];
    store_rec((Rec *)pack, s, xq, F, A);
}

__device__ __forceinline__ void unit3(double *v)
{
    const double r = rsqrt(fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0])));
    for (int j = 0; j < 3; ++j) v[j] *= r;
}

// Rates from the full velocities v, then the Heun stage: predictor (phase 0)
// writes the predictor point, corrector (phase 1) the new positions and the
// stroke average of the centre.
__global__ void sd_heun_kernel(EvalArgs A, SdBuf B, const double *v, int phase, int64_t n)
{
    pdl_sync();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    const double *v1 = v + 6 * s, *v2 = v1 + 3, *nv = B.N + 3 * s;
    double Rd[3], w[3], nw = 0.0;
    for (int j = 0; j < 3; ++j) {
        Rd[j] = 0.5 * (v1[j] + v2[j]);
        w[j] = (v2[j] - v1[j]) / B.L[s];
        nw = fma(nv[j], w[j], nw);
    }
    double Nd[3];
    for (int j = 0; j < 3; ++j) Nd[j] = w[j] - nv[j] * nw;
    const double L1 = rest_and_rate(A, s, n + 1).x;   // placement at t_{n+1}
    double R[3], Nn[3];
    if (phase == 0) {
        const double *x = A.x + 6 * s;
        for (int j = 0; j < 3; ++j) {
            const double r0 = 0.5 * (x[j] + x[3 + j]);
            B.R0[3 * s + j] = r0;
            B.N0[3 * s + j] = nv[j];
            B.rate0[6 * s + j] = Rd[j];
            B.rate0[6 * s + 3 + j] = Nd[j];
            R[j] = fma(A.dt, Rd[j], r0);
            Nn[j] = fma(A.dt, Nd[j], nv[j]);
        }
    } else {
        for (int j = 0; j < 3; ++j) {
            R[j] = fma(0.5 * A.dt, B.rate0[6 * s + j] + Rd[j], B.R0[3 * s + j]);
            Nn[j] = fma(0.5 * A.dt, B.rate0[6 * s + 3 + j] + Nd[j], B.N0[3 * s + j]);
        }
    }
    unit3(Nn);
    double *out = (phase == 0 ? B.xt : A.x) + 6 * s;
    bool fin = true;
    for (int j = 0; j < 3; ++j) {
        out[j] = fma(-0.5 * L1, Nn[j], R[j]);
        out[3 + j] = fma(0.5 * L1, Nn[j], R[j]);
        fin &= finite1(out[j]) && finite1(out[3 + j]);
    }
    if (!fin) atomicOr(A.flags, FLAG_NONFINITE);
    // stroke average of the centre (corrector), trapezoid rule as in the spring model
    if (phase == 1 && A.avg_m > 0) {
        const int64_t k_local = n + 1 - A.avg_n0;
        if (k_local > 0) {
            const int64_t r = 3 * s;
            const bool end = (k_local % A.avg_m) == 0;
            const int64_t kidx = k_local / A.avg_m - 1;
            for (int j = 0; j < 3; ++j) {
                double acc = A.Racc[r + j];
                if (end) {
                    acc += 0.5 * R[j];
                    if (kidx < A.avg_maxk) A.Rbar[kidx * 3 * A.S + r + j] = acc / (double)A.avg_m;
                    acc = 0.5 * R[j];
                } else {
                    acc += R[j];
                }
                A.Racc[r + j] = acc;
            }
        }
    }
}

#define SCK(h, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), e_ == cudaErrorMemoryAllocation ? DBS_E_NOMEM : DBS_E_CUDA,     \
                        "%s: %s", #call, cudaGetErrorString(e_));                            \
    } while (0)

// Constraint forces at the point P (time index k) into packT / Fd, then the
// full velocities into vout.
int shape_eval(dbs_suspension *h, const double *P, int64_t k)
{
    const bool f64 = h->p.precision == DBS_FP64;
    const int rpy = h->p.mobility == DBS_RPY;
    const int thr = 128, blocks = (int)((h->S + thr - 1) / thr);
    EvalArgs A = base_args(h);
    const SdBuf B = sd_view(h);
    if (f64) sd_launch(sd_begin_kernel<double>, blocks, thr, h->stream, A, P, k, B, rpy, h->packT);
    else sd_launch(sd_begin_kernel<float>, blocks, thr, h->stream, A, P, k, B, rpy, h->packT);
    SCK(h, cudaGetLastError());
    EvalArgs Ap = A;
    Ap.pack_in = h->packT;
    for (int it = 1; it < h->sd_iters; ++it) {
        Ap.apply_self = 0;   // interaction only
        launch_apply(h, Ap);
        if (f64) sd_launch(sd_iter_kernel<double>, blocks, thr, h->stream, A, P, B, (const double *)h->vout, h->packT);
        else sd_launch(sd_iter_kernel<float>, blocks, thr, h->stream, A, P, B, (const double *)h->vout, h->packT);
        SCK(h, cudaGetLastError());
    }
    Ap.apply_self = 1;       // v = H F, Eq. (3)
    launch_apply(h, Ap);
    SCK(h, cudaGetLastError());
    return DBS_OK;
}

}  // namespace

// Place the spheres of every dumbbell on the prescribed length at t_n:
// x = R -/+ N L(t_n)/2 with R, N from the current positions.
__global__ void sd_project_kernel(EvalArgs A, int64_t n)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    double *x = A.x + 6 * s;
    double R[3], e[3];
    for (int j = 0; j < 3; ++j) {
        R[j] = 0.5 * (x[j] + x[3 + j]);
        e[j] = x[3 + j] - x[j];
    }
    unit3(e);
    const double L = rest_and_rate(A, s, n).x;
    for (int j = 0; j < 3; ++j) {
        x[j] = fma(-0.5 * L, e[j], R[j]);
        x[3 + j] = fma(0.5 * L, e[j], R[j]);
    }
}

int shape_step(dbs_suspension *h, int64_t n)
{
    const int thr = 128, blocks = (int)((h->S + thr - 1) / thr);
    const SdBuf B = sd_view(h);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = h->n_host;
        int rc = ensure_trig(h, k + 1);
        if (rc) return rc;
        EvalArgs A = base_args(h);
        if ((rc = shape_eval(h, h->x, k))) return rc;
        sd_launch(sd_heun_kernel, blocks, thr, h->stream, A, B, (const double *)h->vout, 0, k);
        SCK(h, cudaGetLastError());
        if ((rc = shape_eval(h, B.xt, k + 1))) return rc;
        sd_launch(sd_heun_kernel, blocks, thr, h->stream, A, B, (const double *)h->vout, 1, k);
        SCK(h, cudaGetLastError());
        h->n_host = k + 1;
    }
    sd_launch(sd_set_step_kernel, 1, 1, h->stream, h->step, h->n_host);
    SCK(h, cudaGetLastError());
    return shape_finish(h);
}

// Leave packA / Fd describing the current state (constraint forces and records
// at x_n), for dbs_velocities and friends.
int shape_finish(dbs_suspension *h)
{
    int rc = ensure_trig(h, h->n_host + 1);
    if (rc) return rc;
    rc = shape_eval(h, h->x, h->n_host);
    if (rc) return rc;
    SCK(h, cudaMemcpyAsync(h->packA, h->packT, (size_t)h->S * (h->p.precision == DBS_FP64 ? sizeof(DbF64) : sizeof(DbF32)),
                           cudaMemcpyDeviceToDevice, h->stream));
    return DBS_OK;
}

// Project the current positions onto the prescribed lengths at t_n and leave
// packA / Fd describing that state.
int shape_reset(dbs_suspension *h)
{
    int rc = ensure_trig(h, h->n_host + 1);
    if (rc) return rc;
    const int thr = 128, blocks = (int)((h->S + thr - 1) / thr);
    sd_project_kernel<<<blocks, thr, 0, h->stream>>>(base_args(h), h->n_host);
    SCK(h, cudaGetLastError());
    rc = shape_eval(h, h->x, h->n_host);
    if (rc) return rc;
    SCK(h, cudaMemcpyAsync(h->packA, h->packT, (size_t)h->S * (h->p.precision == DBS_FP64 ? sizeof(DbF64) : sizeof(DbF32)),
                           cudaMemcpyDeviceToDevice, h->stream));
    return DBS_OK;
}

void shape_free(dbs_suspension *h)
{
    if (h->sd_buf) cudaFree(h->sd_buf);
    h->sd_buf = nullptr;
}

extern "C" {

int dbs_set_dynamics(dbs_suspension *h, int32_t model, int32_t iterations)
{
    if (!h) return DBS_E_ARG;
    if (h->status != DBS_OK) return h->status;
    if (model != DBS_DYN_SPRING && model != DBS_DYN_SHAPE) return DBS_E_ARG;
    if (model == DBS_DYN_SHAPE && (iterations < 1 || iterations > 1000)) return DBS_E_ARG;
    SCK(h, cudaSetDevice(h->device));
    SCK(h, cudaStreamSynchronize(h->stream));
    if (model == DBS_DYN_SPRING) {
        if (h->dyn == DBS_DYN_SHAPE) {
            shape_free(h);
            h->dyn = DBS_DYN_SPRING;
            int rc = spring_repack(h);   // the spring's records and forces at the current state
            if (rc) return rc;
            if (h->path == DBS_PATH_COOP && (rc = coop_setup(h)) != DBS_OK) return rc;   // the spring's kernel
            SCK(h, cudaStreamSynchronize(h->stream));
        }
        return DBS_OK;
    }
    const bool coop_ok = h->path == DBS_PATH_COOP && h->p.precision != DBS_FP64;
    if ((h->path != DBS_PATH_GRID && !coop_ok) || h->Fext || h->noise_sigma > 0.0)
        return refuse(h, DBS_E_STATE,
                      "shape-driven dynamics: grid path (or cooperative, FP32C), no external force, no noise");
    if (!h->sd_buf) SCK(h, cudaMalloc(&h->sd_buf, sizeof(double) * sd_doubles(h->S)));
    drop_graph(h);
    const int prev_dyn = h->dyn;
    h->dyn = DBS_DYN_SHAPE;
    h->sd_iters = iterations;
    int rc = shape_reset(h);
    if (rc) return rc;
    if (h->path == DBS_PATH_COOP && prev_dyn != DBS_DYN_SHAPE && (rc = coop_setup(h)) != DBS_OK) {
        h->dyn = prev_dyn;       // the cooperative shape-driven kernel cannot hold it
        shape_free(h);
        if (spring_repack(h) == DBS_OK) cudaStreamSynchronize(h->stream);
        return rc;
    }
    SCK(h, cudaStreamSynchronize(h->stream));
    return DBS_OK;
}

}  // extern "C"
