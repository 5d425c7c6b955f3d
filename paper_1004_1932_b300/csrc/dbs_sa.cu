// Stroke-averaged far-field model, Eqs. (9a)-(9e) (Sec. III.B), and the
// pair-distance comparison of the averaged model against the microscopic one.
//
// A CTA owns TL dumbbells s (TL a power of two, about 128 CTAs in all); its
// threads split, per target, every shared-memory tile of packed source records r
// (centre relative to the system centre, amplitude, orientation, sin/cos of
// the phase), and their partial sums are folded in a fixed order.  Per pair, with D = R^s - R^r,
// Dh = D/|D|, s = Dh.N^s, r = Dh.N^r, q = N^s.N^r and
// sin(phi^s - phi^r) = sin phi^s cos phi^r - cos phi^s sin phi^r:
//   J = (9/64) a w ell^2 lam^s lam^r sin(dphi) |D|^-4
//         [N^s (2s + 4qr - 10 s r^2) + Dh (1 + 2q^2 - 5s^2 - 5r^2 - 20qsr + 35 s^2 r^2)]
//   K = kpref w a ell^2 lam^s lam^r sin(dphi) |D|^-5
//         Dh (3s + 6rq + 6sq^2 - 7s^3 - 21sr^2 - 42qs^2r + 63 s^3 r^2)
// ((lambda/ell)^2 (ell/D)^4 = lam^s lam^r ell^2 / D^4 for equal amplitudes),
// then dR/dt = sum J, dN/dt = -(I - N N^T) sum K, Heun in time, N renormalised.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <new>
#include <vector>

#include "dbs.h"
#include "dbs_common.cuh"

using namespace dbs;

namespace {

constexpr int SA_NT = 256;    // threads per CTA
constexpr int SA_TILE = 256;
thread_local char g_sa_create_error[256] = "";

struct __align__(16) SaRecF32 {
    float4 R;   // centre - c, amplitude lambda
    float4 N;   // orientation, 0
    float4 sc;  // sin phi, cos phi, 0, 0
};
struct __align__(16) SaRecF64 {
    double Rx, Ry, Rz, lam;
    double Nx, Ny, Nz, pad;
    double sn, cs, pad2, pad3;
};

struct SaArgs {
    int64_t S;
    const void *rec_in;
    void *rec_out;
    double *R, *N;        // state [S][3]
    double *rate0;        // predictor rates [S][6]
    double *rate_out;     // rates output (RATES phase) [S][6]
    const double *lam, *sinp, *cosp;
    double cx, cy, cz;
    double CJ, CK;        // (9/64) a w ell^2, kpref w a ell^2
    double dt;
    int phase;            // 0 predict, 1 correct, 2 rates only
};

template <typename T> struct SaRecOf;
template <> struct SaRecOf<float> { using type = SaRecF32; };
template <> struct SaRecOf<double> { using type = SaRecF64; };

__device__ __forceinline__ void store_rec(SaRecF32 *o, int64_t s, const double R[3], const double N[3],
                                          const SaArgs &A)
{
    SaRecF32 r;
    r.R = make_float4((float)(R[0] - A.cx), (float)(R[1] - A.cy), (float)(R[2] - A.cz), (float)A.lam[s]);
    r.N = make_float4((float)N[0], (float)N[1], (float)N[2], 0.f);
    r.sc = make_float4((float)A.sinp[s], (float)A.cosp[s], 0.f, 0.f);
    o[s] = r;
}
__device__ __forceinline__ void store_rec(SaRecF64 *o, int64_t s, const double R[3], const double N[3],
                                          const SaArgs &A)
{
    SaRecF64 r;
    r.Rx = R[0] - A.cx; r.Ry = R[1] - A.cy; r.Rz = R[2] - A.cz; r.lam = A.lam[s];
    r.Nx = N[0]; r.Ny = N[1]; r.Nz = N[2]; r.pad = 0;
    r.sn = A.sinp[s]; r.cs = A.cosp[s]; r.pad2 = 0; r.pad3 = 0;
    o[s] = r;
}

template <typename T, typename Rec>
__device__ __forceinline__ void sa_pair(bool self, T Rx, T Ry, T Rz, T lam_s, T Nx, T Ny, T Nz,
                                        T sn_s, T cs_s, const Rec &q, T J[3], T K[3])
{
    T qRx, qRy, qRz, qlam, qNx, qNy, qNz, qsn, qcs;
    if constexpr (sizeof(T) == 4) {
        qRx = q.R.x; qRy = q.R.y; qRz = q.R.z; qlam = q.R.w;
        qNx = q.N.x; qNy = q.N.y; qNz = q.N.z; qsn = q.sc.x; qcs = q.sc.y;
    } else {
        qRx = q.Rx; qRy = q.Ry; qRz = q.Rz; qlam = q.lam;
        qNx = q.Nx; qNy = q.Ny; qNz = q.Nz; qsn = q.sn; qcs = q.cs;
    }
    T Dx = Rx - qRx, Dy = Ry - qRy, Dz = Rz - qRz;
    T D2 = Dx * Dx + Dy * Dy + Dz * Dz;
    T w;
    if constexpr (sizeof(T) == 4) w = self ? 0.f : rsqrtf(D2);
    else w = self ? 0.0 : rsqrt(D2);
    T hx = Dx * w, hy = Dy * w, hz = Dz * w;
    T s = hx * Nx + hy * Ny + hz * Nz;
    T r = hx * qNx + hy * qNy + hz * qNz;
    T qq = Nx * qNx + Ny * qNy + Nz * qNz;
    T sd = sn_s * qcs - cs_s * qsn;          // sin(phi^s - phi^r)
    T amp = lam_s * qlam * sd;
    T w2 = w * w;
    T w4 = w2 * w2;
    T s2 = s * s, r2 = r * r;
    T pN = 2 * s + 4 * qq * r - 10 * s * r2;
    T pD = 1 + 2 * qq * qq - 5 * s2 - 5 * r2 - 20 * qq * s * r + 35 * s2 * r2;
    T pK = 3 * s + 6 * r * qq + 6 * s * qq * qq - 7 * s2 * s - 21 * s * r2 - 42 * qq * s2 * r
           + 63 * s2 * s * r2;
    T cj = amp * w4;        // times CJ in the epilogue
    T ck = amp * w4 * w * pK;  // times CK in the epilogue
    J[0] += cj * (Nx * pN + hx * pD);
    J[1] += cj * (Ny * pN + hy * pD);
    J[2] += cj * (Nz * pN + hz * pD);
    K[0] += ck * hx;
    K[1] += ck * hy;
    K[2] += ck * hz;
}

// (s, c) += (s2, c2): FP32 with Knuth's two-sum on the sums, FP64 plain sums.
template <typename T>
__device__ __forceinline__ void sa_merge(T &s, T &c, T s2, T c2)
{
    if constexpr (sizeof(T) == 4) {
        const T u = s + s2;
        const T z = u - s;
        c += c2 + ((s - (u - z)) + (s2 - z));
        s = u;
    } else {
        s += s2;
        c += c2;
    }
}

// TL target dumbbells per CTA; thread tid takes target tid / NSL and, of every
// tile, the records k = (tid mod NSL) + NSL i.  The slice sums of a target are
// folded across the lanes of a warp (shuffles) and then across its warps in
// warp order; thread t < TL runs the epilogue of target t.
template <typename T, int TL>
__global__ void __launch_bounds__(SA_NT) sa_eval_kernel(SaArgs A)
{
    using Rec = typename SaRecOf<T>::type;
    constexpr int NSL = SA_NT / TL;               // slices (threads) per target
    constexpr int LW = NSL < 32 ? NSL : 32;       // lanes of a target within a warp
    constexpr int WPT = NSL > 32 ? NSL / 32 : 1;  // warps per target
    __shared__ Rec tile[SA_TILE];
    __shared__ T red[WPT == 1 ? TL : SA_NT / 32][12];   // J sum, J comp., K sum, K comp. (x, y, z)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = tid / NSL, sl = tid - t * NSL;
    const int64_t st = (int64_t)blockIdx.x * TL + t;
    const bool act = st < A.S;
    const Rec *in = (const Rec *)A.rec_in;
    Rec me{};
    if (act) me = in[st];
    T Rx, Ry, Rz, lam, Nx, Ny, Nz, sn, cs;
    if constexpr (sizeof(T) == 4) {
        Rx = me.R.x; Ry = me.R.y; Rz = me.R.z; lam = me.R.w;
        Nx = me.N.x; Ny = me.N.y; Nz = me.N.z; sn = me.sc.x; cs = me.sc.y;
    } else {
        Rx = me.Rx; Ry = me.Ry; Rz = me.Rz; lam = me.lam;
        Nx = me.Nx; Ny = me.Ny; Nz = me.Nz; sn = me.sn; cs = me.cs;
    }
    // FP32: per-tile FP32 sums folded into (sum, compensation); FP64: plain sums
    T Js[3] = {0, 0, 0}, Jc[3] = {0, 0, 0}, Ks[3] = {0, 0, 0}, Kc[3] = {0, 0, 0};
    for (int64_t t0 = 0; t0 < A.S; t0 += SA_TILE) {
        const int len = (int)min((int64_t)SA_TILE, A.S - t0);
        __syncthreads();
        for (int k = tid; k < len; k += SA_NT) tile[k] = in[t0 + k];
        __syncthreads();
        T J[3] = {0, 0, 0}, K[3] = {0, 0, 0};
        if (act)
            for (int k = sl; k < len; k += NSL)
                sa_pair<T, Rec>(t0 + k == st, Rx, Ry, Rz, lam, Nx, Ny, Nz, sn, cs, tile[k], J, K);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sa_merge(Js[k], Jc[k], J[k], T(0));
            sa_merge(Ks[k], Kc[k], K[k], T(0));
        }
    }
#pragma unroll
    for (int off = LW / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T js = __shfl_xor_sync(0xffffffffu, Js[k], off), jc = __shfl_xor_sync(0xffffffffu, Jc[k], off);
            const T ks = __shfl_xor_sync(0xffffffffu, Ks[k], off), kc = __shfl_xor_sync(0xffffffffu, Kc[k], off);
            sa_merge(Js[k], Jc[k], js, jc);
            sa_merge(Ks[k], Kc[k], ks, kc);
        }
    }
    if (WPT == 1 ? sl == 0 : lane == 0) {
        const int row = WPT == 1 ? t : warp;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            red[row][k] = Js[k];
            red[row][3 + k] = Jc[k];
            red[row][6 + k] = Ks[k];
            red[row][9 + k] = Kc[k];
        }
    }
    __syncthreads();
    if (tid >= TL) return;
    const int64_t sg = (int64_t)blockIdx.x * TL + tid;
    if (sg >= A.S) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Js[k] = red[tid * WPT][k];
        Jc[k] = red[tid * WPT][3 + k];
        Ks[k] = red[tid * WPT][6 + k];
        Kc[k] = red[tid * WPT][9 + k];
    }
    for (int w = 1; w < WPT; ++w) {   // the target's warps, in warp order
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sa_merge(Js[k], Jc[k], red[tid * WPT + w][k], red[tid * WPT + w][3 + k]);
            sa_merge(Ks[k], Kc[k], red[tid * WPT + w][6 + k], red[tid * WPT + w][9 + k]);
        }
    }
    double Jd[3], Kd[3];
    for (int k = 0; k < 3; ++k) {
        Jd[k] = A.CJ * ((double)Js[k] + (double)Jc[k]);
        Kd[k] = A.CK * ((double)Ks[k] + (double)Kc[k]);
    }
    double Nn[3] = {A.N[3 * sg], A.N[3 * sg + 1], A.N[3 * sg + 2]};
    double Rn[3] = {A.R[3 * sg], A.R[3 * sg + 1], A.R[3 * sg + 2]};
    double rate[6];
    if (A.phase == 1) {
        // corrector: the rates at the predicted point use the predicted N for the projector
        double Nt[3], Rt[3];
        for (int k = 0; k < 3; ++k) {
            Rt[k] = Rn[k] + A.dt * A.rate0[6 * sg + k];
            Nt[k] = Nn[k] + A.dt * A.rate0[6 * sg + 3 + k];
        }
        (void)Rt;
        const double NK = Nt[0] * Kd[0] + Nt[1] * Kd[1] + Nt[2] * Kd[2];
        for (int k = 0; k < 3; ++k) {
            rate[k] = Jd[k];
            rate[3 + k] = -(Kd[k] - Nt[k] * NK);
        }
    } else {
        const double NK = Nn[0] * Kd[0] + Nn[1] * Kd[1] + Nn[2] * Kd[2];
        for (int k = 0; k < 3; ++k) {
            rate[k] = Jd[k];
            rate[3 + k] = -(Kd[k] - Nn[k] * NK);
        }
    }
    if (A.phase == 2) {
        for (int k = 0; k < 6; ++k) A.rate_out[6 * sg + k] = rate[k];
        return;
    }
    Rec *out = (Rec *)A.rec_out;
    if (A.phase == 0) {
        double Rt[3], Nt[3];
        for (int k = 0; k < 3; ++k) {
            A.rate0[6 * sg + k] = rate[k];
            A.rate0[6 * sg + 3 + k] = rate[3 + k];
            Rt[k] = Rn[k] + A.dt * rate[k];
            Nt[k] = Nn[k] + A.dt * rate[3 + k];
        }
        store_rec(out, sg, Rt, Nt, A);
    } else {
        double R1[3], N1[3];
        for (int k = 0; k < 3; ++k) {
            R1[k] = Rn[k] + 0.5 * A.dt * (A.rate0[6 * sg + k] + rate[k]);
            N1[k] = Nn[k] + 0.5 * A.dt * (A.rate0[6 * sg + 3 + k] + rate[3 + k]);
        }
        const double nn = sqrt(N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2]);
        for (int k = 0; k < 3; ++k) {
            N1[k] /= nn;
            A.R[3 * sg + k] = R1[k];
            A.N[3 * sg + k] = N1[k];
        }
        store_rec(out, sg, R1, N1, A);
    }
}

template <typename T>
__global__ void sa_pack_kernel(SaArgs A)
{
    using Rec = typename SaRecOf<T>::type;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    double R[3] = {A.R[3 * s], A.R[3 * s + 1], A.R[3 * s + 2]};
    double N[3] = {A.N[3 * s], A.N[3 * s + 1], A.N[3 * s + 2]};
    store_rec((Rec *)A.rec_out, s, R, N, A);
}

// ---- pair-distance comparison (FP64) ----------------------------------------
// The upper triangle of pairs (s < r) is cut into 32 x 32 tiles; CTAs take
// tiles in a grid-stride loop, reduce their pairs in a fixed tree order into a
// per-CTA partial, and the last CTA to finish (arrival ticket) combines the
// partials in CTA order, so the result does not depend on CTA timing.  The
// partials live in a file-scope device array: calls are serialised on the host.
constexpr int PD_T = 32;
constexpr int PD_BT = 256;
constexpr int PD_MAX_BLOCKS = 1184;
__device__ double g_pd_part[PD_MAX_BLOCKS * 3];
__device__ double g_pd_out[3];
__device__ unsigned g_pd_ticket;

// tile t of the upper triangle (row-major) -> block row bi, block column bj >= bi
__device__ __forceinline__ void pd_tile(int64_t t, int64_t nb, int64_t &bi, int64_t &bj)
{
    const double b = 2.0 * (double)nb + 1.0;
    int64_t i = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
    auto start = [nb](int64_t r) { return r * nb - r * (r - 1) / 2; };  // first tile of row r
    if (i < 0) i = 0;
    while (i > 0 && start(i) > t) --i;
    while (i + 1 < nb && start(i + 1) <= t) ++i;
    bi = i;
    bj = i + (t - start(i));
}

__device__ __forceinline__ double pd_dist(const double *a, const double *b)
{
    const double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
    return sqrt(fma(z, z, fma(y, y, x * x)));
}

__global__ void __launch_bounds__(PD_BT) pair_dist_kernel(int64_t S, const double *A0, const double *A1,
                                                           const double *B0, const double *B1)
{
    __shared__ double rows[4][PD_T][3], cols[4][PD_T][3];
    __shared__ double smax[PD_BT], ssq[PD_BT], sref[PD_BT];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const double *src[4] = {A0, A1, B0, B1};
    const int64_t nb = (S + PD_T - 1) / PD_T, ntiles = nb * (nb + 1) / 2;
    double mx = 0, sq = 0, rf = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int64_t bi, bj;
        pd_tile(t, nb, bi, bj);
        __syncthreads();
        for (int q = tid; q < 4 * PD_T * 3; q += PD_BT) {
            const int a = q / (PD_T * 3), e = (q / 3) % PD_T, k = q % 3;
            const int64_t s = bi * PD_T + e, r = bj * PD_T + e;
            rows[a][e][k] = s < S ? src[a][3 * s + k] : 0.0;
            cols[a][e][k] = r < S ? src[a][3 * r + k] : 0.0;
        }
        __syncthreads();
        const int e = tid & (PD_T - 1);
        const int64_t s = bi * PD_T + e;
        for (int f = tid / PD_T; f < PD_T; f += PD_BT / PD_T) {
            const int64_t r = bj * PD_T + f;
            if (s >= S || r >= S || r <= s) continue;
            const double dA = pd_dist(rows[1][e], cols[1][f]) - pd_dist(rows[0][e], cols[0][f]);
            const double dB = pd_dist(rows[3][e], cols[3][f]) - pd_dist(rows[2][e], cols[2][f]);
            const double err = dA - dB;
            mx = fmax(mx, fabs(err));
            sq = fma(err, err, sq);
            rf = fma(dB, dB, rf);
        }
    }
    smax[tid] = mx;
    ssq[tid] = sq;
    sref[tid] = rf;
    __syncthreads();
    for (int w = PD_BT / 2; w > 0; w >>= 1) {
        if (tid < w) {
            smax[tid] = fmax(smax[tid], smax[tid + w]);
            ssq[tid] += ssq[tid + w];
            sref[tid] += sref[tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) {
        g_pd_part[3 * blockIdx.x] = smax[0];
        g_pd_part[3 * blockIdx.x + 1] = ssq[0];
        g_pd_part[3 * blockIdx.x + 2] = sref[0];
        __threadfence();
        s_last = atomicAdd(&g_pd_ticket, 1u) == gridDim.x - 1u;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    // last CTA: thread t folds partials t, t + PD_BT, ... in order, then the tree
    mx = 0;
    sq = 0;
    rf = 0;
    for (unsigned b = tid; b < gridDim.x; b += PD_BT) {
        mx = fmax(mx, __ldcg(&g_pd_part[3 * b]));
        sq += __ldcg(&g_pd_part[3 * b + 1]);
        rf += __ldcg(&g_pd_part[3 * b + 2]);
    }
    smax[tid] = mx;
    ssq[tid] = sq;
    sref[tid] = rf;
    __syncthreads();
    for (int w = PD_BT / 2; w > 0; w >>= 1) {
        if (tid < w) {
            smax[tid] = fmax(smax[tid], smax[tid + w]);
            ssq[tid] += ssq[tid + w];
            sref[tid] += sref[tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) {
        g_pd_out[0] = smax[0];
        g_pd_out[1] = ssq[0];
        g_pd_out[2] = sref[0];
        g_pd_ticket = 0u;
    }
}

}  // namespace

struct dbs_sa {
    dbs_sa_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int status = DBS_OK;
    char msg[256] = "";
    double *R = nullptr, *N = nullptr, *rate0 = nullptr, *rate_out = nullptr, *lam = nullptr,
           *sinp = nullptr, *cosp = nullptr;
    void *recA = nullptr, *recB = nullptr;
    double cx = 0, cy = 0, cz = 0;
};

static int sa_fail(dbs_sa *h, int st, const char *fmt, ...)
{
    char *buf = h ? h->msg : g_sa_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
    if (h) h->status = st;
    return st;
}

#define SCK(h, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return sa_fail((h), e_ == cudaErrorMemoryAllocation ? DBS_E_NOMEM : DBS_E_CUDA, \
                           "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

#define SGUARD(h)                                               \
    do {                                                        \
        if (!(h)) return DBS_E_ARG;                             \
        if ((h)->status != DBS_OK) return (h)->status;          \
        if (cudaSetDevice((h)->device) != cudaSuccess)          \
            return sa_fail((h), DBS_E_CUDA, "cudaSetDevice");   \
    } while (0)

static bool sa_f64(const dbs_sa *h) { return h->p.precision == DBS_FP64; }

static SaArgs sa_args(const dbs_sa *h)
{
    SaArgs A{};
    A.S = h->p.S;
    A.R = h->R;
    A.N = h->N;
    A.rate0 = h->rate0;
    A.rate_out = h->rate_out;
    A.lam = h->lam;
    A.sinp = h->sinp;
    A.cosp = h->cosp;
    A.cx = h->cx;
    A.cy = h->cy;
    A.cz = h->cz;
    const double a = h->p.a, w = h->p.omega, l = h->p.ell;
    A.CJ = (9.0 / 64.0) * a * w * l * l;
    A.CK = h->p.kpref * w * a * l * l;
    A.dt = h->p.dt;
    return A;
}

template <typename T, int TL>
static void sa_launch_t(const dbs_sa *h, const SaArgs &A)
{
    const int blocks = (int)((h->p.S + TL - 1) / TL);
    sa_eval_kernel<T, TL><<<blocks, SA_NT, 0, h->stream>>>(A);
}

// Targets per CTA: the smallest power of two that keeps the grid within about
// 128 CTAs (one wave on the SMs), at most 32.
template <typename T>
static void sa_launch_p(const dbs_sa *h, const SaArgs &A)
{
    const int64_t S = h->p.S;
    if (S <= 128) sa_launch_t<T, 1>(h, A);
    else if (S <= 256) sa_launch_t<T, 2>(h, A);
    else if (S <= 512) sa_launch_t<T, 4>(h, A);
    else if (S <= 1024) sa_launch_t<T, 8>(h, A);
    else if (S <= 2048) sa_launch_t<T, 16>(h, A);
    else sa_launch_t<T, 32>(h, A);
}

static void sa_launch(const dbs_sa *h, const SaArgs &A)
{
    if (sa_f64(h)) sa_launch_p<double>(h, A);
    else sa_launch_p<float>(h, A);
}

static int sa_repack(dbs_sa *h)
{
    SaArgs A = sa_args(h);
    A.rec_out = h->recA;
    const int blocks = (int)((h->p.S + 127) / 128);
    if (sa_f64(h)) sa_pack_kernel<double><<<blocks, 128, 0, h->stream>>>(A);
    else sa_pack_kernel<float><<<blocks, 128, 0, h->stream>>>(A);
    SCK(h, cudaGetLastError());
    return DBS_OK;
}

static void sa_free(dbs_sa *h)
{
    void *b[] = {h->R, h->N, h->rate0, h->rate_out, h->lam, h->sinp, h->cosp, h->recA, h->recB};
    for (void *p : b)
        if (p) cudaFree(p);
}

extern "C" {

const char *dbs_sa_last_error(const dbs_sa *h) { return h ? h->msg : g_sa_create_error; }

int dbs_sa_create(const dbs_sa_params *p, const double *R, const double *N, const double *phi,
                  const double *lambda, dbs_sa **out)
{
    if (!out) return sa_fail(nullptr, DBS_E_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !R || !N || !phi || !lambda) return sa_fail(nullptr, DBS_E_ARG, "NULL argument");
    if (p->S < 2) return sa_fail(nullptr, DBS_E_ARG, "S must be >= 2");
    if (!(p->a > 0 && p->ell > 0 && p->omega > 0 && p->dt > 0 && std::isfinite(p->kpref)))
        return sa_fail(nullptr, DBS_E_ARG, "a, ell, omega, dt must be > 0");
    if (p->precision != DBS_FP32C && p->precision != DBS_FP64)
        return sa_fail(nullptr, DBS_E_ARG, "bad precision");
    const int64_t S = p->S;
    for (int64_t i = 0; i < 3 * S; ++i)
        if (!std::isfinite(R[i]) || !std::isfinite(N[i])) return sa_fail(nullptr, DBS_E_ARG, "non-finite R/N");
    for (int64_t s = 0; s < S; ++s) {
        if (!std::isfinite(phi[s]) || !std::isfinite(lambda[s])) return sa_fail(nullptr, DBS_E_ARG, "non-finite phi/lambda");
        const double nn = std::sqrt(N[3 * s] * N[3 * s] + N[3 * s + 1] * N[3 * s + 1] + N[3 * s + 2] * N[3 * s + 2]);
        if (std::fabs(nn - 1.0) > 1e-6) return sa_fail(nullptr, DBS_E_ARG, "N must be unit vectors");
    }
    dbs_sa *h = new (std::nothrow) dbs_sa();
    if (!h) return sa_fail(nullptr, DBS_E_NOMEM, "host allocation");
    h->p = *p;
    int dev = p->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    h->device = dev;
    auto bail = [&](int r) {
        snprintf(g_sa_create_error, sizeof(g_sa_create_error), "%s", h->msg);
        sa_free(h);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return r;
    };
    int rc;
#define SCREATE(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            sa_fail(h, DBS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
            return bail(e_ == cudaErrorMemoryAllocation ? DBS_E_NOMEM : DBS_E_CUDA); \
        }                                                                           \
    } while (0)
    SCREATE(cudaSetDevice(dev));
    if (p->stream) h->stream = (cudaStream_t)p->stream;
    else {
        SCREATE(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    const size_t v3 = sizeof(double) * 3 * S;
    SCREATE(cudaMalloc(&h->R, v3));
    SCREATE(cudaMalloc(&h->N, v3));
    SCREATE(cudaMalloc(&h->rate0, 2 * v3));
    SCREATE(cudaMalloc(&h->rate_out, 2 * v3));
    SCREATE(cudaMalloc(&h->lam, sizeof(double) * S));
    SCREATE(cudaMalloc(&h->sinp, sizeof(double) * S));
    SCREATE(cudaMalloc(&h->cosp, sizeof(double) * S));
    const size_t rb = (size_t)S * (sa_f64(h) ? sizeof(SaRecF64) : sizeof(SaRecF32));
    SCREATE(cudaMalloc(&h->recA, rb));
    SCREATE(cudaMalloc(&h->recB, rb));
    std::vector<double> sn(S), cs(S);
    for (int64_t s = 0; s < S; ++s) {
        sn[s] = std::sin(phi[s]);
        cs[s] = std::cos(phi[s]);
    }
    double lo[3] = {R[0], R[1], R[2]}, hi[3] = {R[0], R[1], R[2]};
    for (int64_t s = 0; s < S; ++s)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], R[3 * s + k]);
            hi[k] = std::max(hi[k], R[3 * s + k]);
        }
    h->cx = 0.5 * (lo[0] + hi[0]);
    h->cy = 0.5 * (lo[1] + hi[1]);
    h->cz = 0.5 * (lo[2] + hi[2]);
    SCREATE(cudaMemcpyAsync(h->R, R, v3, cudaMemcpyHostToDevice, h->stream));
    SCREATE(cudaMemcpyAsync(h->N, N, v3, cudaMemcpyHostToDevice, h->stream));
    SCREATE(cudaMemcpyAsync(h->lam, lambda, sizeof(double) * S, cudaMemcpyHostToDevice, h->stream));
    SCREATE(cudaMemcpyAsync(h->sinp, sn.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->stream));
    SCREATE(cudaMemcpyAsync(h->cosp, cs.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->stream));
    if ((rc = sa_repack(h)) != DBS_OK) return bail(rc);
    SCREATE(cudaStreamSynchronize(h->stream));
#undef SCREATE
    *out = h;
    return DBS_OK;
}

int dbs_sa_destroy(dbs_sa *h)
{
    if (!h) return DBS_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    sa_free(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return DBS_OK;
}

int dbs_sa_step(dbs_sa *h, int64_t n)
{
    SGUARD(h);
    if (n < 0) return DBS_E_ARG;
    SaArgs A = sa_args(h);
    for (int64_t k = 0; k < n; ++k) {
        A.phase = 0;
        A.rec_in = h->recA;
        A.rec_out = h->recB;
        sa_launch(h, A);
        A.phase = 1;
        A.rec_in = h->recB;
        A.rec_out = h->recA;
        sa_launch(h, A);
    }
    SCK(h, cudaGetLastError());
    return DBS_OK;
}

int dbs_sa_rates(dbs_sa *h, double *Rdot, double *Ndot)
{
    SGUARD(h);
    if (!Rdot || !Ndot) return DBS_E_ARG;
    SaArgs A = sa_args(h);
    A.phase = 2;
    A.rec_in = h->recA;
    sa_launch(h, A);
    SCK(h, cudaGetLastError());
    std::vector<double> r(6 * h->p.S);
    SCK(h, cudaMemcpyAsync(r.data(), h->rate_out, sizeof(double) * 6 * h->p.S, cudaMemcpyDeviceToHost, h->stream));
    SCK(h, cudaStreamSynchronize(h->stream));
    for (int64_t s = 0; s < h->p.S; ++s)
        for (int k = 0; k < 3; ++k) {
            Rdot[3 * s + k] = r[6 * s + k];
            Ndot[3 * s + k] = r[6 * s + 3 + k];
        }
    return DBS_OK;
}

int dbs_sa_state(dbs_sa *h, double *R, double *N)
{
    SGUARD(h);
    if (!R || !N) return DBS_E_ARG;
    const size_t v3 = sizeof(double) * 3 * h->p.S;
    SCK(h, cudaMemcpyAsync(R, h->R, v3, cudaMemcpyDeviceToHost, h->stream));
    SCK(h, cudaMemcpyAsync(N, h->N, v3, cudaMemcpyDeviceToHost, h->stream));
    SCK(h, cudaStreamSynchronize(h->stream));
    return DBS_OK;
}

int dbs_sa_centres_device(dbs_sa *h, const double **R_dev)
{
    SGUARD(h);
    if (!R_dev) return DBS_E_ARG;
    *R_dev = h->R;
    return DBS_OK;
}

int dbs_sa_copy_centres(dbs_sa *h, double *R_dev)
{
    SGUARD(h);
    if (!R_dev) return DBS_E_ARG;
    SCK(h, cudaMemcpyAsync(R_dev, h->R, sizeof(double) * 3 * h->p.S, cudaMemcpyDeviceToDevice, h->stream));
    return DBS_OK;
}

int dbs_pair_distance_error(int64_t S, const double *A0, const double *A1, const double *B0,
                            const double *B1, double *out, void *stream)
{
    if (S < 2 || S > (int64_t)1 << 31 || !A0 || !A1 || !B0 || !B1 || !out) return DBS_E_ARG;
    static std::mutex mu;  // the partials and the ticket are one file-scope array per device
    std::lock_guard<std::mutex> lock(mu);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nb = (S + PD_T - 1) / PD_T, ntiles = nb * (nb + 1) / 2;
    const int blocks = (int)std::min<int64_t>(PD_MAX_BLOCKS, ntiles);
    pair_dist_kernel<<<blocks, PD_BT, 0, st>>>(S, A0, A1, B0, B1);
    double hb[3];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(hb, g_pd_out, sizeof(hb), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DBS_E_CUDA;
    out[0] = hb[0];
    out[1] = hb[1];
    out[2] = hb[2];
    out[3] = (double)S * (double)(S - 1) / 2.0;
    return DBS_OK;
}

}  // extern "C"
