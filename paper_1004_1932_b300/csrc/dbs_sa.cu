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
// N^s is the target's own orientation, so the pair code accumulates
// sum_r cj pN (one scalar) and sum_r cj pD Dh apart, and the epilogue forms
// sum J = N^s sum(cj pN) + sum(cj pD Dh); the polynomials are evaluated as
//   pN = s (2 - 10 r^2) + 4 q r,
//   pK = s (3 + 6 q^2 - 7 s^2 - 21 r^2 + 63 s^2 r^2) + q r (6 - 42 s^2).
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
// source records per shared-memory tile: 16 KB either way (one tile holds a
// 512-dumbbell suspension in FP32)
template <typename T> __host__ __device__ constexpr int sa_tile() { return sizeof(T) == 4 ? 512 : 256; }
thread_local char g_sa_create_error[256] = "";

// Amplitude and phase enter the pair term only through lam^s lam^r sin(phi^s -
// phi^r) = (lam sin phi)^s (lam cos phi)^r - (lam cos phi)^s (lam sin phi)^r, so a
// record carries the two products (formed in FP64, then rounded).
struct __align__(16) SaRecF32 {
    float4 R;   // centre - c, lam sin phi
    float4 N;   // orientation, lam cos phi
};
struct __align__(16) SaRecF64 {
    double Rx, Ry, Rz, ls;   // centre - c, lam sin phi
    double Nx, Ny, Nz, lc;   // orientation, lam cos phi
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
    // source chunks per target group (sa_eval_kernel): with chunks > 1 CTA
    // c * groups + g sums group g over the sources [S c / chunks, S (c + 1) / chunks)
    // into part[c][s][14], and the last of the group's CTAs to arrive (tickets[g])
    // merges the chunks in chunk order and runs the epilogue
    int chunks;
    void *part;
    unsigned *tickets;
};

template <typename T> struct SaRecOf;
template <> struct SaRecOf<float> { using type = SaRecF32; };
template <> struct SaRecOf<double> { using type = SaRecF64; };

__device__ __forceinline__ void store_rec(SaRecF32 *o, int64_t s, const double R[3], const double N[3],
                                          const SaArgs &A)
{
    SaRecF32 r;
    r.R = make_float4((float)(R[0] - A.cx), (float)(R[1] - A.cy), (float)(R[2] - A.cz),
                      (float)(A.lam[s] * A.sinp[s]));
    r.N = make_float4((float)N[0], (float)N[1], (float)N[2], (float)(A.lam[s] * A.cosp[s]));
    o[s] = r;
}
__device__ __forceinline__ void store_rec(SaRecF64 *o, int64_t s, const double R[3], const double N[3],
                                          const SaArgs &A)
{
    SaRecF64 r;
    r.Rx = R[0] - A.cx; r.Ry = R[1] - A.cy; r.Rz = R[2] - A.cz; r.ls = A.lam[s] * A.sinp[s];
    r.Nx = N[0]; r.Ny = N[1]; r.Nz = N[2]; r.lc = A.lam[s] * A.cosp[s];
    o[s] = r;
}

// Target s: centre R, orientation N, ls_s = lam sin phi, mlc_s = -lam cos phi.
template <typename T, typename Rec>
__device__ __forceinline__ void sa_pair(bool self, T Rx, T Ry, T Rz, T ls_s, T Nx, T Ny, T Nz,
                                        T mlc_s, const Rec &q, T J[4], T K[3])
{
    T qRx, qRy, qRz, qls, qNx, qNy, qNz, qlc;
    if constexpr (sizeof(T) == 4) {
        qRx = q.R.x; qRy = q.R.y; qRz = q.R.z; qls = q.R.w;
        qNx = q.N.x; qNy = q.N.y; qNz = q.N.z; qlc = q.N.w;
    } else {
        qRx = q.Rx; qRy = q.Ry; qRz = q.Rz; qls = q.ls;
        qNx = q.Nx; qNy = q.Ny; qNz = q.Nz; qlc = q.lc;
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
    T amp = ls_s * qlc + mlc_s * qls;        // lam^s lam^r sin(phi^s - phi^r)
    T w2 = w * w;
    T w4 = w2 * w2;
    T s2 = s * s, r2 = r * r, qr = qq * r, s2r2 = s2 * r2;
    T pN = s * (2 - 10 * r2) + 4 * qr;
    T pD = 1 + 2 * qq * qq - 5 * s2 - 5 * r2 - 20 * qr * s + 35 * s2r2;
    T pK = s * (3 + 6 * qq * qq - 7 * s2 - 21 * r2 + 63 * s2r2) + qr * (6 - 42 * s2);
    T cj = amp * w4;        // times CJ in the epilogue
    T ck = cj * w * pK;     // times CK in the epilogue
    T cjD = cj * pD;
    J[0] += cjD * hx;       // the pD part of J; J[3]: sum of cj pN (times N^s in the epilogue)
    J[1] += cjD * hy;
    J[2] += cjD * hz;
    J[3] += cj * pN;
    K[0] += ck * hx;
    K[1] += ck * hy;
    K[2] += ck * hz;
}

// FP32: the same pair term for two source records at once with paired f32x2
// instructions (FFMA2/FMUL2: two IEEE single-precision lanes per instruction),
// half the issue slots of two scalar calls; lane .x is record q0, .y record q1.
// The target's fields come duplicated in both lanes.  self0 / self1 mask the
// target's own record (w = 0 makes its term exactly zero).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

__device__ __forceinline__ void sa_pair2f(bool self0, bool self1, float2 Rx, float2 Ry, float2 Rz, float2 ls_s,
                                          float2 Nx, float2 Ny, float2 Nz, float2 mlc_s, float2 qRx,
                                          float2 qRy, float2 qRz, float2 qls, float2 qNx, float2 qNy,
                                          float2 qNz, float2 qlc, float2 J[4], float2 K[3])
{
    const float2 m1 = f2s(-1.f);
    const float2 Dx = __ffma2_rn(qRx, m1, Rx);
    const float2 Dy = __ffma2_rn(qRy, m1, Ry);
    const float2 Dz = __ffma2_rn(qRz, m1, Rz);
    float2 D2 = __fmul2_rn(Dx, Dx);
    D2 = __ffma2_rn(Dy, Dy, D2);
    D2 = __ffma2_rn(Dz, Dz, D2);
    const float2 w = f2(self0 ? 0.f : rsqrtf(D2.x), self1 ? 0.f : rsqrtf(D2.y));
    const float2 hx = __fmul2_rn(Dx, w), hy = __fmul2_rn(Dy, w), hz = __fmul2_rn(Dz, w);
    float2 s = __fmul2_rn(hx, Nx);
    s = __ffma2_rn(hy, Ny, s);
    s = __ffma2_rn(hz, Nz, s);
    float2 r = __fmul2_rn(hx, qNx);
    r = __ffma2_rn(hy, qNy, r);
    r = __ffma2_rn(hz, qNz, r);
    float2 qq = __fmul2_rn(Nx, qNx);
    qq = __ffma2_rn(Ny, qNy, qq);
    qq = __ffma2_rn(Nz, qNz, qq);
    // lam^s lam^r sin(phi^s - phi^r)
    const float2 amp = __ffma2_rn(ls_s, qlc, __fmul2_rn(mlc_s, qls));
    const float2 w2 = __fmul2_rn(w, w);
    const float2 w4 = __fmul2_rn(w2, w2);
    const float2 s2 = __fmul2_rn(s, s), r2 = __fmul2_rn(r, r);
    const float2 qr = __fmul2_rn(qq, r), qq2 = __fmul2_rn(qq, qq), s2r2 = __fmul2_rn(s2, r2);
    // pN = s (2 - 10 r^2) + 4 q r
    const float2 pN = __ffma2_rn(f2s(4.f), qr, __fmul2_rn(s, __ffma2_rn(f2s(-10.f), r2, f2s(2.f))));
    // pD = 1 + 2 q^2 - 5 s^2 - 5 r^2 - 20 q s r + 35 s^2 r^2
    float2 pD = __ffma2_rn(f2s(2.f), qq2, f2s(1.f));
    pD = __ffma2_rn(f2s(-5.f), s2, pD);
    pD = __ffma2_rn(f2s(-5.f), r2, pD);
    pD = __ffma2_rn(f2s(-20.f), __fmul2_rn(qr, s), pD);
    pD = __ffma2_rn(f2s(35.f), s2r2, pD);
    // pK = s (3 + 6 q^2 - 7 s^2 - 21 r^2 + 63 s^2 r^2) + q r (6 - 42 s^2)
    float2 pA = __ffma2_rn(f2s(6.f), qq2, f2s(3.f));
    pA = __ffma2_rn(f2s(-7.f), s2, pA);
    pA = __ffma2_rn(f2s(-21.f), r2, pA);
    pA = __ffma2_rn(f2s(63.f), s2r2, pA);
    const float2 pK = __ffma2_rn(qr, __ffma2_rn(f2s(-42.f), s2, f2s(6.f)), __fmul2_rn(s, pA));
    const float2 cj = __fmul2_rn(amp, w4);          // times CJ in the epilogue
    const float2 ck = __fmul2_rn(__fmul2_rn(cj, w), pK);  // times CK in the epilogue
    const float2 cjD = __fmul2_rn(cj, pD);
    // the pD part of J; J[3]: sum of cj pN (times the target's N in the epilogue)
    J[0] = __ffma2_rn(cjD, hx, J[0]);
    J[1] = __ffma2_rn(cjD, hy, J[1]);
    J[2] = __ffma2_rn(cjD, hz, J[2]);
    J[3] = __ffma2_rn(cj, pN, J[3]);
    K[0] = __ffma2_rn(ck, hx, K[0]);
    K[1] = __ffma2_rn(ck, hy, K[1]);
    K[2] = __ffma2_rn(ck, hz, K[2]);
}

// Two source records stored pair-interleaved (record k in lanes .x, record
// k + NSL in .y of every field), so that the paired operands load as they are:
// a = (Rx, Ry), b = (Rz, lam sin phi), c = (Nx, Ny), d = (Nz, lam cos phi); in
// sa_eval_kernel's shared memory each of a, b, c, d is a plane of its own.
struct __align__(16) SaPairF32 {
    float4 a, b, c, d;
};
__device__ __forceinline__ void sa_pair2(bool self0, bool self1, float2 Rx, float2 Ry, float2 Rz, float2 ls_s,
                                         float2 Nx, float2 Ny, float2 Nz, float2 mlc_s, const SaPairF32 &q,
                                         float2 J[4], float2 K[3])
{
    const float4 a = q.a, b = q.b, c = q.c, d = q.d;
    sa_pair2f(self0, self1, Rx, Ry, Rz, ls_s, Nx, Ny, Nz, mlc_s, f2(a.x, a.y), f2(a.z, a.w), f2(b.x, b.y),
              f2(b.z, b.w), f2(c.x, c.y), f2(c.z, c.w), f2(d.x, d.y), f2(d.z, d.w), J, K);
}

// Records in shared memory as planes of 16-byte fields (FP32: R[k], N[k]; FP64:
// (Rx, Ry), (Rz, ls), (Nx, Ny), (Nz, lc)), so that the 16-byte loads of
// consecutive records by consecutive lanes hit distinct banks (a 32- or 64-byte
// record stride puts two or four lanes of each quarter-warp on the same banks).
// NP: records per plane.
template <int NP>
__device__ __forceinline__ void sa_tile_put(float4 *tb, int k, const SaRecF32 &q)
{
    tb[k] = q.R;
    tb[NP + k] = q.N;
}
template <int NP>
__device__ __forceinline__ void sa_tile_put(float4 *tb, int k, const SaRecF64 &q)
{
    double2 *d = reinterpret_cast<double2 *>(tb);
    d[k] = make_double2(q.Rx, q.Ry);
    d[NP + k] = make_double2(q.Rz, q.ls);
    d[2 * NP + k] = make_double2(q.Nx, q.Ny);
    d[3 * NP + k] = make_double2(q.Nz, q.lc);
}
template <typename Rec, int NP>
__device__ __forceinline__ Rec sa_tile_get(const float4 *tb, int k)
{
    if constexpr (sizeof(Rec) == sizeof(SaRecF32)) {
        return Rec{tb[k], tb[NP + k]};
    } else {
        const double2 *d = reinterpret_cast<const double2 *>(tb);
        const double2 a = d[k], b = d[NP + k], c = d[2 * NP + k], e = d[3 * NP + k];
        return Rec{a.x, a.y, b.x, b.y, c.x, c.y, e.x, e.y};
    }
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

// Fold six (sum, compensation) components over the LW lanes of a target by
// transposition: they sit in eight slots, each of the first three shuffle
// levels halves the slots a lane carries (the lane whose level bit is clear
// keeps the lower half and merges its partner's copy into its own), and the
// remaining levels are a butterfly on the one slot left, which is slot `ci` of
// this lane.  About a third of the shuffles of a butterfly on all six.
template <typename T, int LW>
__device__ __forceinline__ void sa_fold_lanes(T fs[8], T fc[8], int lane, int &ci)
{
    static_assert(LW >= 8, "the transposing fold needs 8 lanes per target");
    ci = 0;
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) {
        const int off = LW / (8 / h);
        const bool hi = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const T ss = hi ? fs[k] : fs[k + h], sc = hi ? fc[k] : fc[k + h];
            const T ks = hi ? fs[k + h] : fs[k], kc = hi ? fc[k + h] : fc[k];
            const T rs = __shfl_xor_sync(0xffffffffu, ss, off);
            const T rc = __shfl_xor_sync(0xffffffffu, sc, off);
            fs[k] = ks;
            fc[k] = kc;
            sa_merge(fs[k], fc[k], rs, rc);
        }
        ci += hi ? h : 0;
    }
#pragma unroll
    for (int off = LW / 16; off >= 1; off >>= 1) {
        const T rs = __shfl_xor_sync(0xffffffffu, fs[0], off);
        const T rc = __shfl_xor_sync(0xffffffffu, fc[0], off);
        sa_merge(fs[0], fc[0], rs, rc);
    }
}

// 1/sqrt(x) for x near 1 (the squared norm of an orientation after one Heun
// step): an FP32 seed refined by two Newton steps on f(y) = 1/y^2 - x,
// y <- y (3 - x y^2) / 2, each of which squares the relative error (2^-22 ->
// 1e-13 -> FP64 rounding), in 9 FP64 instructions instead of a square root and
// three divisions (an FP64 instruction holds its SM sub-partition 64 cycles).
__device__ __forceinline__ double sa_inv_norm(double x)
{
    const double h = 0.5 * x;
    double y = (double)rsqrtf((float)x);
    y *= fma(-h, y * y, 1.5);
    y *= fma(-h, y * y, 1.5);
    return y;
}

// Record components along axis a (and, for a = 0, amplitude and phase) of
// dumbbell s: the epilogue's three axis warps each write their own.
__device__ __forceinline__ void store_rec_axis(SaRecF32 *o, int64_t s, int a, double R, double N,
                                               const SaArgs &A)
{
    float *f = (float *)(o + s);
    f[a] = (float)(R - (a == 0 ? A.cx : (a == 1 ? A.cy : A.cz)));
    f[4 + a] = (float)N;
    if (a == 0) {
        f[3] = (float)(A.lam[s] * A.sinp[s]);
        f[7] = (float)(A.lam[s] * A.cosp[s]);
    }
}
__device__ __forceinline__ void store_rec_axis(SaRecF64 *o, int64_t s, int a, double R, double N,
                                               const SaArgs &A)
{
    double *f = (double *)(o + s);
    f[a] = R - (a == 0 ? A.cx : (a == 1 ? A.cy : A.cz));
    f[4 + a] = N;
    if (a == 0) {
        f[3] = A.lam[s] * A.sinp[s];
        f[7] = A.lam[s] * A.cosp[s];
    }
}

// TL target dumbbells per CTA; thread tid takes target tid / NSL and, of every
// tile, the records k = (tid mod NSL) + NSL i.  The slice sums of a target are
// folded across the lanes of a warp (shuffles) and then across its warps in
// warp order.  The epilogue runs on three axis warps: lane t of warp a takes
// component a of target t, each warp forming the dot products and the norm it
// needs from all three components (FP64 instructions are slow on this part, so
// the FP64 Heun update is spread over three sub-partitions).
// CH: the source-chunked form (A.chunks > 1; the one-chunk form is compiled
// without its index arithmetic and merge).  FP32 at TL >= 16 (the grids of more
// than one wave) keeps three CTAs per SM: at most 80 registers per thread.
template <typename T, int TL, bool CH>
__global__ void __launch_bounds__(SA_NT, sizeof(T) == 4 && TL >= 16 ? 3 : 1) sa_eval_kernel(SaArgs A)
{
    using Rec = typename SaRecOf<T>::type;
    constexpr int NSL = SA_NT / TL;               // slices (threads) per target
    constexpr int LW = NSL < 32 ? NSL : 32;       // lanes of a target within a warp
    constexpr int WPT = NSL > 32 ? NSL / 32 : 1;  // warps per target
    constexpr int TILE = sa_tile<T>();
    __shared__ float4 tile[TILE * sizeof(Rec) / sizeof(float4)];   // planes, see sa_tile_put
    // per row: the pD part of J (sums 0-2, compensations 3-5), K (6-8, 9-11) and
    // the sum of cj pN (12, 13)
    __shared__ T red[WPT == 1 ? TL : SA_NT / 32][14];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = tid / NSL, sl = tid - t * NSL;
    // chunk-major: every group's last chunk falls in the last wave, so the merges
    // run side by side at the end of the launch
    const int groups = CH ? (int)((A.S + TL - 1) / TL) : (int)gridDim.x;
    const int c = CH ? (int)blockIdx.x / groups : 0, g = (int)blockIdx.x - c * groups;
    const int64_t db = CH ? A.S * c / A.chunks : 0, de = CH ? A.S * (c + 1) / A.chunks : A.S;   // sources
    const int64_t st = (int64_t)g * TL + t;
    const bool act = st < A.S;
    // Programmatic dependent launch: this grid may have been scheduled before the
    // previous step's launch finished; wait for it (and its memory) before reading
    // anything, then let the next launch be scheduled.  No-ops for an ordinary launch.
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    // the epilogue's state (lane ta of axis warp a), loaded now so that its
    // latency overlaps the sweep where the kernel is latency-bound (few targets
    // per CTA); for the larger splits the registers held across the sweep would
    // cost a CTA per SM (S = 8192: 464 -> 662 us per step, measured), so those
    // load it in the epilogue
    constexpr bool EARLY = TL <= 8;
    const int ea = warp, ta = lane;
    const int64_t sg = (int64_t)g * TL + ta;
    const bool on = warp < 3 && ta < TL && sg < A.S;
    double Nn[3] = {0.0, 0.0, 0.0}, Ra = 0.0, r0a = 0.0, n0[3] = {0.0, 0.0, 0.0};
    auto load_state = [&]() {
        if (!on) return;
#pragma unroll
        for (int k = 0; k < 3; ++k) Nn[k] = A.N[3 * sg + k];
        Ra = A.R[3 * sg + ea];
        if (A.phase == 1) {
            r0a = A.rate0[6 * sg + ea];
#pragma unroll
            for (int k = 0; k < 3; ++k) n0[k] = A.rate0[6 * sg + 3 + k];
        }
    };
    if (EARLY) load_state();
    const Rec *in = (const Rec *)A.rec_in;
    Rec me{};
    if (act) me = in[st];
    T Rx, Ry, Rz, ls, Nx, Ny, Nz, mlc;
    if constexpr (sizeof(T) == 4) {
        Rx = me.R.x; Ry = me.R.y; Rz = me.R.z; ls = me.R.w;
        Nx = me.N.x; Ny = me.N.y; Nz = me.N.z; mlc = -me.N.w;
    } else {
        Rx = me.Rx; Ry = me.Ry; Rz = me.Rz; ls = me.ls;
        Nx = me.Nx; Ny = me.Ny; Nz = me.Nz; mlc = -me.lc;
    }
    // FP32: per-tile FP32 sums folded into (sum, compensation); FP64: plain sums.
    // Slots 0-2: the pD part of J, 3-5: K, 6: sum of cj pN, 7: empty (for the
    // transposing fold).
    T fs[8] = {0, 0, 0, 0, 0, 0, 0, 0}, fc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // FP32 with TL >= 4: two records per paired call (with TL <= 2 a thread holds at
    // most two records of a tile, and the paired code would only cost registers),
    // the tile stored pair-interleaved (TILE / 2 pairs: four planes a, b, c, d of
    // TILE / 2 float4) so that the paired operands load as they are
    constexpr bool PAIRED = sizeof(T) == 4 && TL >= 4;
    constexpr int PH = TILE / 2;
    for (int64_t t0 = db; t0 < de; t0 += TILE) {
        const int len = (int)min((int64_t)TILE, de - t0);
        // records k and k + NSL (k mod 2 NSL < NSL) share pair (k div 2 NSL) NSL + k mod NSL;
        // the records past the tile's end up to a whole group of 2 NSL are zero-amplitude
        // stand-ins far away, whose terms are exactly zero
        const int kmax = PAIRED ? (len + 2 * NSL - 1) / (2 * NSL) * (2 * NSL) : len;
        __syncthreads();
        if constexpr (PAIRED) {
            for (int k = tid; k < kmax; k += SA_NT) {
                const int i = k / (2 * NSL), r = k - i * 2 * NSL, h = r / NSL;
                const int p = i * NSL + (r - h * NSL);
                float *fa = (float *)(tile + p), *fb = (float *)(tile + PH + p);
                float *fc = (float *)(tile + 2 * PH + p), *fd = (float *)(tile + 3 * PH + p);
                if (k < len) {
                    const Rec q = in[t0 + k];
                    fa[h] = q.R.x; fa[2 + h] = q.R.y; fb[h] = q.R.z; fb[2 + h] = q.R.w;
                    fc[h] = q.N.x; fc[2 + h] = q.N.y; fd[h] = q.N.z; fd[2 + h] = q.N.w;
                } else {
                    fa[h] = 1.0e18f; fa[2 + h] = 1.0e18f; fb[h] = 1.0e18f; fb[2 + h] = 0.f;
                    fc[h] = 1.f; fc[2 + h] = 0.f; fd[h] = 0.f; fd[2 + h] = 0.f;
                }
            }
        } else {
            for (int k = tid; k < len; k += SA_NT) sa_tile_put<TILE>(tile, k, in[t0 + k]);
        }
        __syncthreads();
        T J[4] = {0, 0, 0, 0}, K[3] = {0, 0, 0};
        if (act) {
            int k = sl;
            if constexpr (PAIRED) {
                float2 J2[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                float2 K2[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                for (; k < kmax; k += 2 * NSL) {
                    const int p = (k / (2 * NSL)) * NSL + sl;
                    const SaPairF32 q{tile[p], tile[PH + p], tile[2 * PH + p], tile[3 * PH + p]};
                    sa_pair2(t0 + k == st, t0 + k + NSL == st, f2s(Rx), f2s(Ry), f2s(Rz), f2s(ls), f2s(Nx),
                             f2s(Ny), f2s(Nz), f2s(mlc), q, J2, K2);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    sa_merge(fs[c], fc[c], J2[c].x, T(0));
                    sa_merge(fs[c], fc[c], J2[c].y, T(0));
                    sa_merge(fs[3 + c], fc[3 + c], K2[c].x, T(0));
                    sa_merge(fs[3 + c], fc[3 + c], K2[c].y, T(0));
                }
                sa_merge(fs[6], fc[6], J2[3].x, T(0));
                sa_merge(fs[6], fc[6], J2[3].y, T(0));
            }
            for (; k < len; k += NSL)
                sa_pair<T, Rec>(t0 + k == st, Rx, Ry, Rz, ls, Nx, Ny, Nz, mlc, sa_tile_get<Rec, TILE>(tile, k),
                                J, K);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sa_merge(fs[k], fc[k], J[k], T(0));
            sa_merge(fs[3 + k], fc[3 + k], K[k], T(0));
        }
        sa_merge(fs[6], fc[6], J[3], T(0));
    }
    int ci;
    sa_fold_lanes<T, LW>(fs, fc, lane, ci);
    if ((lane & (LW / 8 - 1)) == 0 && ci < 7) {
        const int row = WPT == 1 ? t : warp;
        // pD part of J: sum ci, comp. 3 + ci; K: sum 6 + k, comp. 9 + k; cj pN: 12, 13
        const int col = ci < 3 ? ci : (ci < 6 ? 3 + ci : 12);
        red[row][col] = fs[0];
        red[row][col + (ci < 6 ? 3 : 1)] = fc[0];
    }
    __syncthreads();
    if (warp >= 3) return;
    // ---- epilogue: lane ta of axis warp a --------------------------------------
    const int a = ea;
    // (issued before the sums are read, so that its latency overlaps theirs; with
    // chunks only the last CTA of the group loads it)
    if (!EARLY && !CH) load_state();
    // the target's sums: pD part of J along a, cj pN, K (sum, compensation)
    T js = 0, jc = 0, ns = 0, nc = 0, ks[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    if (on) {
        const int r0w = ta * WPT;
        js = red[r0w][a]; jc = red[r0w][3 + a]; ns = red[r0w][12]; nc = red[r0w][13];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ks[k] = red[r0w][6 + k];
            kc[k] = red[r0w][9 + k];
        }
        for (int w = 1; w < WPT; ++w) {   // the target's warps, in warp order
            sa_merge(js, jc, red[r0w + w][a], red[r0w + w][3 + a]);
            sa_merge(ns, nc, red[r0w + w][12], red[r0w + w][13]);
#pragma unroll
            for (int k = 0; k < 3; ++k) sa_merge(ks[k], kc[k], red[r0w + w][6 + k], red[r0w + w][9 + k]);
        }
    }
    if constexpr (CH) {
        // this chunk's sums of the target, laid out as a row of red (axis lane a
        // writes its components of J and K, lane 0 also the cj pN sum)
        if (on) {
            T *p = (T *)A.part + ((int64_t)c * A.S + sg) * 14;
            p[a] = js;
            p[3 + a] = jc;
            p[6 + a] = a == 0 ? ks[0] : (a == 1 ? ks[1] : ks[2]);
            p[9 + a] = a == 0 ? kc[0] : (a == 1 ? kc[1] : kc[2]);
            if (a == 0) {
                p[12] = ns;
                p[13] = nc;
            }
        }
        // the named barrier orders the three axis warps' partial writes before
        // thread 0, whose fence makes them visible device-wide before its arrival
        // ticket; the last arriver fences again before its warps read the others'
        asm volatile("bar.sync 2, 96;" ::: "memory");
        if (tid == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&A.tickets[g], 1u);
            s_last = prev == (unsigned)A.chunks - 1u;
            if (s_last) {
                A.tickets[g] = 0u;
                __threadfence();
            }
        }
        asm volatile("bar.sync 2, 96;" ::: "memory");
        if (!s_last) return;
        if (!EARLY) load_state();
        if (on) {
            // all chunks of the target, in chunk order (read from L2: other SMs wrote them)
            const T *p = (const T *)A.part + sg * 14;
            js = __ldcg(p + a); jc = __ldcg(p + 3 + a); ns = __ldcg(p + 12); nc = __ldcg(p + 13);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ks[k] = __ldcg(p + 6 + k);
                kc[k] = __ldcg(p + 9 + k);
            }
            for (int cc = 1; cc < A.chunks; ++cc) {
                const T *q = p + (int64_t)cc * A.S * 14;
                sa_merge(js, jc, __ldcg(q + a), __ldcg(q + 3 + a));
                sa_merge(ns, nc, __ldcg(q + 12), __ldcg(q + 13));
#pragma unroll
                for (int k = 0; k < 3; ++k) sa_merge(ks[k], kc[k], __ldcg(q + 6 + k), __ldcg(q + 9 + k));
            }
        }
    }
    double JD = (double)js + (double)jc, JN = (double)ns + (double)nc, Kd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Kd[k] = A.CK * ((double)ks[k] + (double)kc[k]);
    // every axis warp has read the state components that the others rewrite below
    asm volatile("bar.sync 1, 96;" ::: "memory");
    if (!on) return;
    // dN/dt = -(I - N N^T) K, with N the orientation at the evaluation point (the
    // predicted one in the corrector)
    double Nb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Nb[k] = A.phase == 1 ? fma(A.dt, n0[k], Nn[k]) : Nn[k];
    // J along a: the target's orientation at the evaluation point times the cj pN sum
    const double Ja = A.CJ * fma(a == 0 ? Nb[0] : (a == 1 ? Nb[1] : Nb[2]), JN, JD);
    const double NK = fma(Nb[0], Kd[0], fma(Nb[1], Kd[1], Nb[2] * Kd[2]));
    double rK[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) rK[k] = -(Kd[k] - Nb[k] * NK);
    const double rKa = a == 0 ? rK[0] : (a == 1 ? rK[1] : rK[2]);
    if (A.phase == 2) {
        A.rate_out[6 * sg + a] = Ja;
        A.rate_out[6 * sg + 3 + a] = rKa;
        return;
    }
    Rec *out = (Rec *)A.rec_out;
    if (A.phase == 0) {
        A.rate0[6 * sg + a] = Ja;
        A.rate0[6 * sg + 3 + a] = rKa;
        const double Nna = a == 0 ? Nn[0] : (a == 1 ? Nn[1] : Nn[2]);
        store_rec_axis(out, sg, a, fma(A.dt, Ja, Ra), fma(A.dt, rKa, Nna), A);
    } else {
        const double R1 = fma(0.5 * A.dt, r0a + Ja, Ra);
        double N1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) N1[k] = fma(0.5 * A.dt, n0[k] + rK[k], Nn[k]);
        const double inv = sa_inv_norm(fma(N1[0], N1[0], fma(N1[1], N1[1], N1[2] * N1[2])));
        const double N1a = (a == 0 ? N1[0] : (a == 1 ? N1[1] : N1[2])) * inv;
        A.R[3 * sg + a] = R1;
        A.N[3 * sg + a] = N1a;
        store_rec_axis(out, sg, a, R1, N1a, A);
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

// ---- cooperative form of the averaged model (FP32C, S <= 4096) ---------------
// One cooperative launch of G <= SMs CTAs advances K averaged Heun steps.  CTA
// g owns the TL dumbbells [g TL, g TL + TL) and keeps every record of the
// suspension in shared memory; amplitude and phase do not change, so they are
// loaded once per launch, and per evaluation only (R, N) travel: one 64-bit
// word per dumbbell and axis a, (R_a - c_a) in its low half and N_a in its high
// half, whose lowest bit carries the evaluation's parity bit (bit 1 of the
// evaluation counter, inverted), so a reader that sees the expected bit has
// that evaluation's pair of values: no fence, flag or barrier.  Buffers
// alternate by evaluation parity; a slot is rewritten (evaluation e + 2) only
// after its owner has finished e + 1, which needed every CTA's words of e + 1,
// which each CTA publishes only after it has copied all words of e into shared
// memory.  Every wait is bounded (1 s of %globaltimer, and at once when another
// CTA has raised SAF_TIMEOUT).
//
// Precision.  The pair sums are FP32 with two-sum compensation, as in
// sa_eval_kernel, and so are the rates formed from them (their accuracy is the
// pair terms' FP32 accuracy either way).  Within a launch the state (R - c and
// N) is carried as double-single pairs hi + lo (48-bit significands; FP64
// instructions, each of which holds its sub-partition's FP64 pipe 64 cycles on
// this part, would set the pace of the step): the Heun step of Sec. III.B
// advances them, and N is renormalised with an FP32 reciprocal square root and
// one Newton step in double-single (|N| = 1 to about 1e-14).  The state is read
// from and written back to the FP64 arrays once per launch, N renormalised in
// FP64 there.  The critical path forms each next record from those pairs in
// FP32 (the corrector's N normalised in FP32 for its record); the
// double-single update runs in the next poll's gap.
constexpr int SAF_TIMEOUT = 4, SAF_LAUNCH = 8;
#ifndef DBS_SA_COOP_UNROLL
#define DBS_SA_COOP_UNROLL 4
#endif
constexpr int kSaCoopUnroll = DBS_SA_COOP_UNROLL;   // paired calls in flight per thread in the sweep
constexpr int SAC_CHUNK = 512;     // records per compensated partial sum (as sa_eval_kernel's tile)
constexpr int SAC_POLL = 8;        // words per thread and round of a poll
// Records of the cooperative kernel's shared-memory tile: Spad rounded up to a
// whole group of 2 (256 / TL) records (the paired sweep's stand-ins), 48 bytes
// each (R with lam sin phi, N with lam cos phi, 16 bytes unused).  Measured
// against a pair-interleaved tile of four 16-byte planes (as sa_eval_kernel's)
// and records as two 16-byte planes R[s], N[s]: S = 512 4.95 / 5.44 / 5.53,
// S = 1024 10.0 / 10.9 / 11.1, S = 4096 84.9 / 85.1 / 89.7 us per averaged step.
constexpr int SAC_REC = 48;
__host__ __device__ constexpr int sac_records(int Spad, int TL)
{
    return (Spad + 512 / TL - 1) / (512 / TL) * (512 / TL);
}

struct SaFlowArgs {
    unsigned long long *words;     // [2][Spad][3]
    int *flags;
    int G, K;                      // CTAs, averaged Heun steps
    unsigned base;                 // evaluation counter at evaluation 0 of the launch (even)
    unsigned long long timeout_ns;
};

template <int TL>
struct SaOwn {
    float Rh[3][TL], Rl[3][TL];    // R - c as double-single
    float Nh[3][TL], Nl[3][TL];    // N as double-single
    float r0f[3][TL], n0f[3][TL];  // predictor rates (J, projected K)
};

__device__ __forceinline__ unsigned long long sac_ld(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void sac_st(unsigned long long *p, float R, float N, unsigned bit)
{
    const unsigned long long v =
        (unsigned long long)((__float_as_uint(N) & ~1u) | bit) << 32 | __float_as_uint(R);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long sac_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned sac_bit(unsigned e) { return ((e >> 1) & 1u) ^ 1u; }
__device__ __forceinline__ float sac_nclear(float n) { return __uint_as_float(__float_as_uint(n) & ~1u); }
// FP32 of (hi + (lo + d)) for a small increment d
__device__ __forceinline__ float sac_add(float h, float l, float d) { return h + (l + d); }

// double-single (hi, lo), |lo| <= ulp(hi) / 2: Knuth's two-sum and the FMA
// two-product (Dekker)
struct sads { float h, l; };
__device__ __forceinline__ sads sads_fast(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ sads sads_add(sads a, sads b)
{
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
    return sads_fast(s, e);
}
__device__ __forceinline__ sads sads_mul(sads a, sads b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + fmaf(a.h, b.l, a.l * b.h);
    return sads_fast(p, e);
}
__device__ __forceinline__ void sads_split(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

template <int TL>
__global__ void __launch_bounds__(SA_NT, 1) sa_flow_kernel(const SaArgs A, const SaFlowArgs P)
{
    constexpr int NSL = SA_NT / TL;
    constexpr int LW = NSL < 32 ? NSL : 32;
    constexpr int WPT = NSL > 32 ? NSL / 32 : 1;
    extern __shared__ float4 sac_smem[];          // all records, 3 float4 each (SAC_REC)
    __shared__ SaOwn<TL> own;
    __shared__ float red[WPT == 1 ? TL : SA_NT / 32][14];   // as in sa_eval_kernel
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    const int S = (int)A.S;
    const int Spad = P.G * TL;
    const int st0 = g * TL, nown = min(TL, S - st0);
    // field f of record s: 0-2 R - c, 3 lam sin phi, 4-6 N, 7 lam cos phi
    float4 *const tile = sac_smem;
    auto sac_slot = [&](int s, int f) -> float * { return (float *)tile + 12 * s + f; };
    if (gridDim.x != (unsigned)P.G || blockDim.x != (unsigned)SA_NT) {
        if (tid == 0) atomicOr(P.flags, SAF_LAUNCH);
        return;
    }
    const float CJf = (float)A.CJ, CKf = (float)A.CK, dtf = (float)A.dt, hdtf = (float)(0.5 * A.dt);
    const double cen_a = warp == 0 ? A.cx : (warp == 1 ? A.cy : A.cz);   // axis warps

    // ---- static record fields of every dumbbell; the owned state; evaluation 0
    for (int s = tid; s < sac_records(Spad, TL); s += SA_NT) {
        if (s < S) {
            *sac_slot(s, 3) = (float)(A.lam[s] * A.sinp[s]);
            *sac_slot(s, 7) = (float)(A.lam[s] * A.cosp[s]);
        } else {
#pragma unroll
            for (int f = 0; f < 8; ++f) *sac_slot(s, f) = f < 3 ? 1.0e18f : (f == 4 ? 1.f : 0.f);
        }
    }
    if (warp < 3 && lane < nown) {
        const int a = warp, d = lane, s = st0 + d;
        const double R = A.R[3 * (int64_t)s + a] - cen_a, N = A.N[3 * (int64_t)s + a];
        sads_split(R, own.Rh[a][d], own.Rl[a][d]);
        sads_split(N, own.Nh[a][d], own.Nl[a][d]);
        const float Rf = (float)R, Nf = sac_nclear((float)N);
        *sac_slot(s, a) = Rf;
        *sac_slot(s, 4 + a) = Nf;
        sac_st(P.words + (size_t)s * 3 + a, Rf, Nf, sac_bit(P.base));
    }
    __syncthreads();

    const int t = tid / NSL, sl = tid - t * NSL;
    const int st = st0 + t;
    const bool act = t < nown;
    const int nwords = 3 * S, own_w0 = 3 * st0, own_w1 = 3 * (st0 + nown);
    const bool ax = warp < 3 && lane < nown;      // epilogue lane: axis warp, dumbbell lane
    // The corrector's increments dt/2 (rate0 + rate) of R along this warp's axis
    // and of all three components of N; the next poll's gap adds them to the
    // double-single state and renormalises N.  `pend` is the same in all lanes of
    // an axis warp (the update meets the other axis warps at a barrier).
    float incR = 0.f, incN[3] = {0.f, 0.f, 0.f};
    bool pend = false;
    auto state_update = [&]() {
        if (warp >= 3 || !pend) return;
        const int a = warp, d = lane;
        const bool on = d < nown;
        sads N1[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (on) {
#pragma unroll
            for (int k = 0; k < 3; ++k) N1[k] = sads_add({own.Nh[k][d], own.Nl[k][d]}, {incN[k], 0.f});
            const sads R1 = sads_add({own.Rh[a][d], own.Rl[a][d]}, {incR, 0.f});
            own.Rh[a][d] = R1.h;
            own.Rl[a][d] = R1.l;
        }
        // every axis warp has read the components of N that the others rewrite
        // below (whole warps, converged, meet at the barrier)
        __syncwarp();
        asm volatile("bar.sync 1, 96;" ::: "memory");
        if (on) {
            const sads q = sads_add(sads_add(sads_mul(N1[0], N1[0]), sads_mul(N1[1], N1[1])), sads_mul(N1[2], N1[2]));
            // y = 1/sqrt(q): FP32 seed, one Newton step y + y (1 - q y^2) / 2
            const float y0 = rsqrtf(q.h);
            const sads qy2 = sads_mul(q, sads_mul({y0, 0.f}, {y0, 0.f}));
            const float e = (1.f - qy2.h) - qy2.l;
            const sads y = sads_fast(y0, 0.5f * y0 * e);
            const sads Na = sads_mul(a == 0 ? N1[0] : (a == 1 ? N1[1] : N1[2]), y);
            own.Nh[a][d] = Na.h;
            own.Nl[a][d] = Na.l;
        }
        pend = false;
    };

    bool dead = false;
    for (int ev = 0; ev < 2 * P.K && !dead; ++ev) {
        const unsigned bit = sac_bit(P.base + (unsigned)ev);
        const bool corr = (ev & 1) != 0;
        const unsigned long long *W = P.words + (size_t)(ev & 1) * Spad * 3;
        // 1. poll the words of the records this CTA does not own, two staggered
        // rounds of SAC_POLL loads per thread, into shared memory
        bool ok = true;
        for (int b0 = 0; b0 < nwords && ok; b0 += SAC_POLL * SA_NT) {
            unsigned pending = 0;
#pragma unroll
            for (int j = 0; j < SAC_POLL; ++j) {
                const int idx = b0 + j * SA_NT + tid;
                if (idx < nwords && (idx < own_w0 || idx >= own_w1)) pending |= 1u << j;
            }
            auto has = [&](unsigned long long v) { return ((unsigned)(v >> 32) & 1u) == bit; };
            auto store = [&](int j, unsigned long long v) {
                const int idx = b0 + j * SA_NT + tid, s = idx / 3, a = idx - 3 * s;
                *sac_slot(s, a) = __uint_as_float((unsigned)v);
                *sac_slot(s, 4 + a) = __uint_as_float((unsigned)(v >> 32) & ~1u);
            };
            unsigned long long va[SAC_POLL], vb[SAC_POLL];
            const unsigned long long *base = W + b0 + tid;
#pragma unroll
            for (int j = 0; j < SAC_POLL; ++j)
                if ((pending >> j) & 1u) va[j] = sac_ld(base + j * SA_NT);
            {
                const long long c0 = clock64();
                state_update();
                while (clock64() - c0 < 300) {
                }
            }
            unsigned long long t0 = 0;
            for (unsigned it = 0; pending; ++it) {
                const unsigned pb = pending;
#pragma unroll
                for (int j = 0; j < SAC_POLL; ++j)
                    if ((pb >> j) & 1u) vb[j] = sac_ld(base + j * SA_NT);
#pragma unroll
                for (int j = 0; j < SAC_POLL; ++j)
                    if (((pending >> j) & 1u) && has(va[j])) {
                        store(j, va[j]);
                        pending &= ~(1u << j);
                    }
                if (!pending) break;
                const unsigned pa = pending;
#pragma unroll
                for (int j = 0; j < SAC_POLL; ++j)
                    if ((pa >> j) & 1u) va[j] = sac_ld(base + j * SA_NT);
#pragma unroll
                for (int j = 0; j < SAC_POLL; ++j)   // pending is within pb: vb[j] was loaded
                    if (((pending >> j) & 1u) && has(vb[j])) {
                        store(j, vb[j]);
                        pending &= ~(1u << j);
                    }
                if (!pending) break;
                if (it == 0) t0 = sac_ns();
                if ((it & 7u) == 7u) {
                    if (*(volatile int *)P.flags & SAF_TIMEOUT) { ok = false; break; }
                    if (sac_ns() - t0 > P.timeout_ns) {
                        atomicOr(P.flags, SAF_TIMEOUT);
                        ok = false;
                        break;
                    }
                }
            }
        }
        state_update();   // done in the first gap: ends the live range of its inputs
        dead = __syncthreads_or(!ok);
        if (dead) break;

        // 2. sweep: target t against records sl, sl + NSL, ... in compensated chunks
        float fs[8] = {0, 0, 0, 0, 0, 0, 0, 0}, fc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (act) {
            const float4 mR = tile[3 * st], mN = tile[3 * st + 1];
            for (int t0 = 0; t0 < S; t0 += SAC_CHUNK) {
                const int len = min(SAC_CHUNK, S - t0);
                if constexpr (TL >= 4) {
                    // two records per paired call (the partners missing at the end of
                    // the last chunk are stand-ins)
                    const int kmax = (len + 2 * NSL - 1) / (2 * NSL) * (2 * NSL);
                    float2 J2[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                    float2 K2[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll kSaCoopUnroll
                    for (int k = sl; k < kmax; k += 2 * NSL) {
                        const float4 R0 = tile[3 * (t0 + k)], N0 = tile[3 * (t0 + k) + 1];
                        const float4 R1 = tile[3 * (t0 + k + NSL)], N1 = tile[3 * (t0 + k + NSL) + 1];
                        const SaPairF32 q{make_float4(R0.x, R1.x, R0.y, R1.y), make_float4(R0.z, R1.z, R0.w, R1.w),
                                          make_float4(N0.x, N1.x, N0.y, N1.y), make_float4(N0.z, N1.z, N0.w, N1.w)};
                        sa_pair2(t0 + k == st, t0 + k + NSL == st, f2s(mR.x), f2s(mR.y), f2s(mR.z), f2s(mR.w),
                                 f2s(mN.x), f2s(mN.y), f2s(mN.z), f2s(-mN.w), q, J2, K2);
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sa_merge(fs[c], fc[c], J2[c].x, 0.f);
                        sa_merge(fs[c], fc[c], J2[c].y, 0.f);
                        sa_merge(fs[3 + c], fc[3 + c], K2[c].x, 0.f);
                        sa_merge(fs[3 + c], fc[3 + c], K2[c].y, 0.f);
                    }
                    sa_merge(fs[6], fc[6], J2[3].x, 0.f);
                    sa_merge(fs[6], fc[6], J2[3].y, 0.f);
                } else {
                    // TL = 2: a thread holds at most two records of a chunk; the paired
                    // form with a stand-in was slower (S = 64: 4.0 against 3.68 us per
                    // averaged step, measured)
                    float J[4] = {0, 0, 0, 0}, K[3] = {0, 0, 0};
                    for (int k = sl; k < len; k += NSL)
                        sa_pair<float, SaRecF32>(t0 + k == st, mR.x, mR.y, mR.z, mR.w, mN.x, mN.y, mN.z, -mN.w,
                                                 SaRecF32{tile[3 * (t0 + k)], tile[3 * (t0 + k) + 1]}, J, K);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        sa_merge(fs[c], fc[c], J[c], 0.f);
                        sa_merge(fs[3 + c], fc[3 + c], K[c], 0.f);
                    }
                    sa_merge(fs[6], fc[6], J[3], 0.f);
                }
            }
        }
        // 3. fold: lanes by transposition, then the target's warps in warp order
        {
            int ci;
            sa_fold_lanes<float, LW>(fs, fc, lane, ci);
            if ((lane & (LW / 8 - 1)) == 0 && ci < 7) {
                const int row = WPT == 1 ? t : warp;
                const int col = ci < 3 ? ci : (ci < 6 ? 3 + ci : 12);
                red[row][col] = fs[0];
                red[row][col + (ci < 6 ? 3 : 1)] = fc[0];
            }
        }
        __syncthreads();

        // 4. epilogue: lane d of axis warp a forms its record component of the next
        // evaluation point from the double-single state and publishes it
        if (warp < 3) {
            const int a = warp, d = lane, s = st0 + d;
            float Rn = 0.f, Nn = 0.f;
            if (ax) {
                const int r0w = d * WPT;
                float js = red[r0w][a], jc = red[r0w][3 + a], ns = red[r0w][12], nc = red[r0w][13];
                float ks[3], kc[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ks[k] = red[r0w][6 + k];
                    kc[k] = red[r0w][9 + k];
                }
                for (int w = 1; w < WPT; ++w) {
                    sa_merge(js, jc, red[r0w + w][a], red[r0w + w][3 + a]);
                    sa_merge(ns, nc, red[r0w + w][12], red[r0w + w][13]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) sa_merge(ks[k], kc[k], red[r0w + w][6 + k], red[r0w + w][9 + k]);
                }
                // the target's orientation in the record the sums were taken at
                const float mN[3] = {*sac_slot(s, 4), *sac_slot(s, 5), *sac_slot(s, 6)};
                const float Nrec = mN[a];
                const float Jf = CJf * fmaf(Nrec, ns + nc, js + jc);
                float Kf[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) Kf[k] = CKf * (ks[k] + kc[k]);
                const float Kfa = a == 0 ? Kf[0] : (a == 1 ? Kf[1] : Kf[2]);
                if (!corr) {   // x~ = x_n + dt (J, -(I - N N^T) K) at (R_n, N_n)
                    const float NK = fmaf(own.Nh[0][d], Kf[0], fmaf(own.Nh[1][d], Kf[1], own.Nh[2][d] * Kf[2]));
                    const float rK = -(Kfa - own.Nh[a][d] * NK);
                    own.r0f[a][d] = Jf;
                    own.n0f[a][d] = rK;
                    Rn = sac_add(own.Rh[a][d], own.Rl[a][d], dtf * Jf);
                    Nn = sac_add(own.Nh[a][d], own.Nl[a][d], dtf * rK);
                } else {       // x_{n+1} = x_n + dt/2 (rate0 + rate(x~)), N renormalised
                    const float *Nb = mN;   // the predicted point's orientation
                    const float NK = fmaf(Nb[0], Kf[0], fmaf(Nb[1], Kf[1], Nb[2] * Kf[2]));
                    float N1[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        incN[k] = hdtf * (own.n0f[k][d] - (Kf[k] - Nb[k] * NK));
                        N1[k] = sac_add(own.Nh[k][d], own.Nl[k][d], incN[k]);
                    }
                    const float inv = rsqrtf(fmaf(N1[0], N1[0], fmaf(N1[1], N1[1], N1[2] * N1[2])));
                    incR = hdtf * (own.r0f[a][d] + Jf);
                    Rn = sac_add(own.Rh[a][d], own.Rl[a][d], incR);
                    Nn = (a == 0 ? N1[0] : (a == 1 ? N1[1] : N1[2])) * inv;
                }
                Nn = sac_nclear(Nn);
            }
            if (corr) {   // all three axis warps have read the predicted record before it changes
                pend = true;
                __syncwarp();
                asm volatile("bar.sync 2, 96;" ::: "memory");
            }
            if (ax) {
                *sac_slot(s, a) = Rn;
                *sac_slot(s, 4 + a) = Nn;
                if (ev + 1 < 2 * P.K)
                    sac_st(P.words + ((size_t)((ev + 1) & 1) * Spad + s) * 3 + a, Rn, Nn,
                           sac_bit(P.base + (unsigned)ev + 1u));
            }
        }
        // The other warps wait here for the axis warps' epilogue: started at once,
        // their polls ran ahead of this CTA's own publish and every evaluation took
        // longer (S = 128 / 512 / 1024: 4.6-4.8 / 7.7 / 13.0 us per averaged step
        // without this barrier, 3.8-3.9 / 5.3-5.4 / 11.2 with it, measured).  The
        // next poll writes only records this CTA does not own.
        __syncthreads();
    }
    state_update();
    __syncthreads();
    // the FP64 state: R - c and N from their double-single pairs, N renormalised
    if (warp < 3 && lane < nown) {
        const int a = warp, d = lane, s = st0 + d;
        double N[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) N[k] = (double)own.Nh[k][d] + (double)own.Nl[k][d];
        const double inv = sa_inv_norm(fma(N[0], N[0], fma(N[1], N[1], N[2] * N[2])));
        A.R[3 * (int64_t)s + a] = cen_a + ((double)own.Rh[a][d] + (double)own.Rl[a][d]);
        A.N[3 * (int64_t)s + a] = (a == 0 ? N[0] : (a == 1 ? N[1] : N[2])) * inv;
    }
}

// ---- pair-distance comparison (FP64) ----------------------------------------
// The upper triangle of pairs (s < r) is cut into 32 x 32 tiles; CTAs take
// tiles in a grid-stride loop, reduce their pairs in a fixed tree order into a
// per-CTA partial, and the last CTA to finish (arrival ticket) combines the
// partials in CTA order, so the result does not depend on CTA timing.  The
// partials live in a file-scope device array: calls are serialised on the host,
// and enqueued calls (dbs_pair_distance_error_async) must not overlap on
// different streams.
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

// out: when not null, also the final {max, RMS of the error, RMS of dB, pairs}
__global__ void __launch_bounds__(PD_BT) pair_dist_kernel(int64_t S, const double *A0, const double *A1,
                                                           const double *B0, const double *B1, double *out)
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
        if (out) {
            const double pairs = (double)S * (double)(S - 1) / 2.0;
            out[0] = smax[0];
            out[1] = sqrt(ssq[0] / pairs);
            out[2] = sqrt(sref[0] / pairs);
            out[3] = pairs;
        }
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
    int sms = 0;   // SMs of the device
    // cooperative path (sa_flow_kernel): split, exchange words, evaluation counter
    int path = DBS_PATH_GRID;
    int coop_T = 0, coop_G = 0;
    unsigned coop_base = 0;
    unsigned long long *words = nullptr;
    int *flags = nullptr;       // SAF_* raised by the cooperative kernel
    bool recs_stale = false;    // recA behind the state after cooperative steps
    int test_dG = 0;            // diagnostic: CTAs the kernel is told beyond those launched
    // one launch per evaluation: source chunks per target group (SaArgs::chunks),
    // the requested count (0: built-in), partial sums and arrival tickets
    int chunks = 1, chunks_req = 0;
    void *part = nullptr;
    unsigned *tickets = nullptr;
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

// a refusal that leaves the handle usable (no sticky status)
static int sa_refuse(dbs_sa *h, int st, const char *msg)
{
    snprintf(h->msg, sizeof(h->msg), "%s", msg);
    return st;
}

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
    A.chunks = h->chunks;
    A.part = h->part;
    A.tickets = h->tickets;
    return A;
}

template <typename T, int TL>
static void sa_launch_t(const dbs_sa *h, const SaArgs &A)
{
    const int blocks = (int)((h->p.S + TL - 1) / TL) * h->chunks;
    // Programmatic stream serialisation where the grid has at most one CTA per SM
    // (the latency-bound sizes): scheduled while the previous launch on the stream
    // finishes, the kernel waiting for it before reading anything.  A larger grid
    // launched that way is placed around the previous grid's CTAs, up to three of
    // its CTAs on some SMs and one on others (S = 8192 in FP64: 22.4 -> 33.6 ms per
    // step, measured), so it is launched in plain stream order.
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(SA_NT);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = blocks <= h->sms ? 1 : 0;
    if (h->chunks > 1) cudaLaunchKernelEx(&cfg, sa_eval_kernel<T, TL, true>, A);
    else cudaLaunchKernelEx(&cfg, sa_eval_kernel<T, TL, false>, A);
}

// Targets per CTA: the smallest power of two that keeps the grid within about
// 128 CTAs (one wave on the SMs), at most 16; 32 for FP32 once groups of 32
// outnumber the SMs, where the source chunks spread them over the SMs and each
// source tile then serves twice the targets (S = 6000 / 8192 / 12000 / 16384:
// 196 / 334 / 693 / 1195 -> 180 / 302 / 638 / 1123 us per averaged step,
// measured; at S = 2500 - 4096 and in FP64 up to 4096 it was 3-45 % slower, at
// FP64 8192 equal).
static int sa_tl(int64_t S, bool f64, int sms)
{
    const int tl_max = (!f64 && S > 32 * (int64_t)sms) ? 32 : 16;
    int tl = 1;
    while (tl < tl_max && S > 128 * (int64_t)tl) tl *= 2;
    return tl;
}
template <typename T>
static void sa_launch_p(const dbs_sa *h, const SaArgs &A)
{
    switch (sa_tl(h->p.S, sa_f64(h), h->sms)) {
    case 1: sa_launch_t<T, 1>(h, A); break;
    case 2: sa_launch_t<T, 2>(h, A); break;
    case 4: sa_launch_t<T, 4>(h, A); break;
    case 8: sa_launch_t<T, 8>(h, A); break;
    case 16: sa_launch_t<T, 16>(h, A); break;
    default: sa_launch_t<T, 32>(h, A); break;
    }
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

// ---- cooperative path ---------------------------------------------------------
constexpr int64_t SAC_MAX_S = 4096;   // every CTA holds all records in shared memory
constexpr int SAC_MAX_T = 32;
constexpr int SAC_MAX_STEPS = 1024;   // averaged Heun steps per launch

static const void *sa_flow_fn(int T)
{
    switch (T) {
    case 1: return (const void *)sa_flow_kernel<1>;
    case 2: return (const void *)sa_flow_kernel<2>;
    case 4: return (const void *)sa_flow_kernel<4>;
    case 8: return (const void *)sa_flow_kernel<8>;
    case 16: return (const void *)sa_flow_kernel<16>;
    case 32: return (const void *)sa_flow_kernel<32>;
    default: return nullptr;
    }
}

// Split: T dumbbells per CTA, the smallest power of two from 2 up for which
// ceil(S / T) CTAs fit the SMs one each with all records in shared memory.
static int sa_coop_setup(dbs_sa *h)
{
    if (sa_f64(h)) return sa_refuse(h, DBS_E_ARG, "cooperative averaged model: FP32C only");
    if (h->p.S > SAC_MAX_S) return sa_refuse(h, DBS_E_ARG, "cooperative averaged model needs S <= 4096");
    int coop = 0, optin = 0;
    SCK(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
    SCK(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (!coop) return sa_refuse(h, DBS_E_ARG, "device without cooperative launch");
    // at least two dumbbells per CTA: with one, the step took 1.7-2.2x as long
    // (S = 64 / 128: 7.0 / 10.2 us against 4.1 / 4.6 us with two, measured)
    int T = 2, G = 0;
    for (;; T *= 2) {
        if (T > SAC_MAX_T) return sa_refuse(h, DBS_E_ARG, "cooperative averaged model: grid does not fit the device");
        G = (int)((h->p.S + T - 1) / T);
        if (G > h->sms) continue;
        const void *k = sa_flow_fn(T);
        cudaFuncAttributes fa{};
        SCK(h, cudaFuncGetAttributes(&fa, k));
        const size_t smem = (size_t)sac_records(G * T, T) * SAC_REC;
        if (smem + fa.sharedSizeBytes > (size_t)optin) continue;
        // a property of the kernel, shared by every handle: all the device allows
        SCK(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
        int occ = 0;
        SCK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, SA_NT, smem));
        if ((int64_t)occ * h->sms >= G) break;
    }
    SCK(h, cudaStreamSynchronize(h->stream));
    if (h->words) cudaFree(h->words);
    h->words = nullptr;
    const size_t nw = 2 * (size_t)G * T * 3;
    SCK(h, cudaMalloc(&h->words, nw * sizeof(unsigned long long)));
    // a cleared buffer carries parity bit 0: the counter starts at a multiple of 4,
    // whose first two evaluations expect bit 1
    SCK(h, cudaMemsetAsync(h->words, 0, nw * sizeof(unsigned long long), h->stream));
    h->coop_T = T;
    h->coop_G = G;
    h->coop_base = 0;
    h->path = DBS_PATH_COOP;
    return DBS_OK;
}

static int sa_coop_step(dbs_sa *h, int64_t n)
{
    for (int64_t left = n; left > 0;) {
        const int K = (int)std::min<int64_t>(left, SAC_MAX_STEPS);
        const SaArgs A = sa_args(h);
        SaFlowArgs P{};
        P.words = h->words;
        P.flags = h->flags;
        P.G = h->coop_G + h->test_dG;
        P.K = K;
        P.base = h->coop_base;
        P.timeout_ns = 1000000000ull;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(h->coop_G);
        cfg.blockDim = dim3(SA_NT);
        cfg.dynamicSmemBytes = (size_t)sac_records(h->coop_G * h->coop_T, h->coop_T) * SAC_REC;
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {(void *)&A, (void *)&P};
        SCK(h, cudaLaunchKernelExC(&cfg, sa_flow_fn(h->coop_T), args));
        // 2K evaluations per launch: the counter stays even and keeps its residue mod 4
        h->coop_base += (unsigned)(2 * K);
        left -= K;
    }
    h->recs_stale = true;
    return DBS_OK;
}

// after a synchronisation: a fault the cooperative kernel raised becomes the
// handle's sticky status
static int sa_check_flags(dbs_sa *h)
{
    int f = 0;
    SCK(h, cudaMemcpy(&f, h->flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & SAF_TIMEOUT) return sa_fail(h, DBS_E_TIMEOUT, "cooperative averaged model: a bounded wait ran out");
    if (f & SAF_LAUNCH) return sa_fail(h, DBS_E_CUDA, "kernel launched in a grid or cluster shape it cannot run");
    return DBS_OK;
}

// Source chunks of the one-launch kernel: the requested count, else the
// built-in choice (sa_chunks_builtin); the partial sums and tickets it needs.
// Built-in: one chunk while the groups fit one CTA per SM (the latency-bound
// sizes); above, the count in 1..8 whose CTAs spread most evenly over the SMs:
// u = groups x C / SMs CTAs per SM on average, u / ceil(u) of the busiest SM's
// work done by the average SM, less 0.015 per extra chunk.  Measured (µs per
// averaged step, FP32C; best count in brackets, C = 1 first): S = 3000 89 / 74
// (3), 4096 115 / 114 (4), 6000 238 / 221 (3), 8192 402 / 368 (2), 12000 820
// / 735 (4), 16384 1286 (1); FP64 4096 4460 / 3920 (4), 8192 17730 / 15520 (2):
// the rule picks each best count.
constexpr int SA_MAX_CHUNKS = 64;
static int sa_chunks_builtin(const dbs_sa *h, int groups)
{
    if (groups <= h->sms) return 1;
    int best = 1;
    double best_e = -1.0;
    for (int C = 1; C <= 8; ++C) {
        const double u = (double)groups * C / h->sms;
        const double e = u / std::ceil(u) - 0.015 * (C - 1);
        if (e > best_e + 1e-12) {
            best_e = e;
            best = C;
        }
    }
    return best;
}
static int sa_chunks_setup(dbs_sa *h)
{
    const int64_t S = h->p.S;
    const int tl = sa_tl(S, sa_f64(h), h->sms);
    const int groups = (int)((S + tl - 1) / tl);
    int C = h->chunks_req > 0 ? h->chunks_req : sa_chunks_builtin(h, groups);
    C = (int)std::min<int64_t>(std::min(C, SA_MAX_CHUNKS), S);
    if (C == h->chunks && (C == 1 || h->part)) return DBS_OK;
    SCK(h, cudaStreamSynchronize(h->stream));
    if (h->part) cudaFree(h->part);
    if (h->tickets) cudaFree(h->tickets);
    h->part = nullptr;
    h->tickets = nullptr;
    h->chunks = 1;
    if (C > 1) {
        const size_t pb = (size_t)C * S * 14 * (sa_f64(h) ? sizeof(double) : sizeof(float));
        SCK(h, cudaMalloc(&h->part, pb));
        SCK(h, cudaMalloc(&h->tickets, sizeof(unsigned) * groups));
        SCK(h, cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * groups, h->stream));
    }
    h->chunks = C;
    return DBS_OK;
}

static void sa_free(dbs_sa *h)
{
    if (h->part) cudaFree(h->part);
    if (h->tickets) cudaFree(h->tickets);
    if (h->words) cudaFree(h->words);
    if (h->flags) cudaFree(h->flags);
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
    SCREATE(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
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
    SCREATE(cudaMalloc(&h->flags, sizeof(int)));
    SCREATE(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
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
    if ((rc = sa_chunks_setup(h)) != DBS_OK) return bail(rc);
    if ((rc = sa_repack(h)) != DBS_OK) return bail(rc);
    // FP32C systems that fit take the cooperative path; the others (and a device
    // that cannot hold it) keep one launch per evaluation
    if (!sa_f64(h) && S <= SAC_MAX_S) {
        if ((rc = sa_coop_setup(h)) == DBS_E_NOMEM || rc == DBS_E_CUDA) return bail(rc);
        h->msg[0] = '\0';
    }
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
    if (h->path == DBS_PATH_COOP) return sa_coop_step(h, n);
    if (h->recs_stale) {
        const int rc = sa_repack(h);
        if (rc) return rc;
        h->recs_stale = false;
    }
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
    if (h->recs_stale) {
        const int rc = sa_repack(h);
        if (rc) return rc;
        h->recs_stale = false;
    }
    SaArgs A = sa_args(h);
    A.phase = 2;
    A.rec_in = h->recA;
    sa_launch(h, A);
    SCK(h, cudaGetLastError());
    std::vector<double> r(6 * h->p.S);
    SCK(h, cudaMemcpyAsync(r.data(), h->rate_out, sizeof(double) * 6 * h->p.S, cudaMemcpyDeviceToHost, h->stream));
    SCK(h, cudaStreamSynchronize(h->stream));
    if (const int rc = sa_check_flags(h)) return rc;
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
    return sa_check_flags(h);
}

int dbs_sa_set_path(dbs_sa *h, int32_t path)
{
    SGUARD(h);
    if (path == DBS_PATH_GRID) {
        h->path = DBS_PATH_GRID;
        return DBS_OK;
    }
    if (path != DBS_PATH_COOP) return sa_refuse(h, DBS_E_ARG, "path must be DBS_PATH_GRID or DBS_PATH_COOP");
    if (h->path == DBS_PATH_COOP) return DBS_OK;
    return sa_coop_setup(h);
}

int dbs_test_sa_flow_misshape(dbs_sa *h)
{
    SGUARD(h);
    if (h->path != DBS_PATH_COOP) return sa_refuse(h, DBS_E_STATE, "not on the cooperative path");
    // one averaged step whose kernel is told it has one CTA more than it was launched with
    h->test_dG = 1;
    const int rc = sa_coop_step(h, 1);
    h->test_dG = 0;
    if (rc) return rc;
    SCK(h, cudaStreamSynchronize(h->stream));
    return sa_check_flags(h);
}

int dbs_sa_set_chunks(dbs_sa *h, int32_t chunks)
{
    SGUARD(h);
    if (chunks < 0) return sa_refuse(h, DBS_E_ARG, "chunks must be >= 0");
    h->chunks_req = chunks;
    return sa_chunks_setup(h);
}

int dbs_sa_get_chunks(dbs_sa *h, int32_t *chunks)
{
    if (!h || !chunks) return DBS_E_ARG;
    *chunks = h->chunks;
    return DBS_OK;
}

int dbs_sa_get_path(dbs_sa *h, int32_t *path, int32_t *targets_per_cta)
{
    if (!h || !path) return DBS_E_ARG;
    *path = h->path;
    if (targets_per_cta) *targets_per_cta = h->path == DBS_PATH_COOP ? h->coop_T : 0;
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
    pair_dist_kernel<<<blocks, PD_BT, 0, st>>>(S, A0, A1, B0, B1, nullptr);
    double hb[3];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(hb, g_pd_out, sizeof(hb), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DBS_E_CUDA;
    const double pairs = (double)S * (double)(S - 1) / 2.0;
    out[0] = hb[0];
    out[1] = std::sqrt(hb[1] / pairs);
    out[2] = std::sqrt(hb[2] / pairs);
    out[3] = pairs;
    return DBS_OK;
}

int dbs_pair_distance_error_async(int64_t S, const double *A0, const double *A1, const double *B0,
                                  const double *B1, double *out_dev, void *stream)
{
    if (S < 2 || S > (int64_t)1 << 31 || !A0 || !A1 || !B0 || !B1 || !out_dev) return DBS_E_ARG;
    const int64_t nb = (S + PD_T - 1) / PD_T, ntiles = nb * (nb + 1) / 2;
    const int blocks = (int)std::min<int64_t>(PD_MAX_BLOCKS, ntiles);
    pair_dist_kernel<<<blocks, PD_BT, 0, (cudaStream_t)stream>>>(S, A0, A1, B0, B1, out_dev);
    return cudaGetLastError() == cudaSuccess ? DBS_OK : DBS_E_CUDA;
}

}  // extern "C"
