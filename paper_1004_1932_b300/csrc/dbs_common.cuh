// Shared device-side definitions of libdbs (B300, sm_103a).
//
// Physics (Putz, Dunkel & Yeomans, "CUDA simulations of active dumbbell
// suspensions"):
//   Eq. (4):  L^s(t) = ell + lambda^s sin(omega t + phi^s),
//             F_{2s+1} = -k0 (d - L) e,  F_{2s} = +k0 (d - L) e,  e = (X_{2s+1} - X_{2s}) / d
//   Eq. (3a): self mobility 1 / (6 pi mu a)
//   Eq. (3b): pair mobility; with G = F / (8 pi mu) folded into the packed force,
//             H_ab F_b = (G + rh (rh.G)) / r + (2a^2/3) (G - 3 rh (rh.G)) / r^3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dbs {

// device fault flags (bitwise OR into one int per handle)
enum : int {
    FLAG_OVERLAP = 1,    // r < 2a under RPY, or coincident spheres
    FLAG_NONFINITE = 2,  // a velocity or position is NaN/Inf
    FLAG_TIMEOUT = 4,    // a bounded wait ran out
    FLAG_LAUNCH = 8,     // a kernel found itself launched in a shape it cannot run
};

enum Phase : int {
    PHASE_PREDICT = 0,   // eval at (x_n, t_n): v0, x~ = x_n + dt v0, repack at (x~, t_{n+1})
    PHASE_CORRECT = 1,   // eval at (x~, t_{n+1}): x_{n+1} = x_n + dt/2 (v0 + v1), repack
    PHASE_APPLY = 2,     // eval only: v = F/(6 pi mu a) + u (or u alone)
};

// Packed j-records, one per dumbbell (its two spheres side by side, so that a
// pair of j-spheres feeds one paired f32x2 instruction):
//   a = (x_2r, x_2r+1, y_2r, y_2r+1), b = (z_2r, z_2r+1, Gx_2r, Gx_2r+1),
//   c = (Gy_2r, Gy_2r+1, Gz_2r, Gz_2r+1),
// positions relative to the system centre, G = F / (8 pi mu).
struct __align__(16) DbF32 {
    float4 a, b, c;
};

// FP64 record: x[2], y[2], z[2] then Gx[2], Gy[2], Gz[2] of the two spheres.
struct __align__(16) DbF64 {
    double x[2], y[2], z[2];
    double gx[2], gy[2], gz[2];
};

template <typename R> struct RecOf;
template <> struct RecOf<float> { using type = DbF32; };
template <> struct RecOf<double> { using type = DbF64; };

// Everything an evaluation kernel needs, passed by value.
struct EvalArgs {
    int64_t S;            // dumbbells
    int64_t N;            // spheres = 2S
    const void *pack_in;  // packed dumbbell records read by the pair sum [S]
    void *pack_out;       // packed dumbbell records written by the epilogue [S]
    double *x;            // positions x_n [N][3]
    double *v0;           // predictor velocity [N][3]
    double *Fd;           // FP64 force at the point of pack_in [N][3] (self term); updated in place
    const double *Fext;   // external force [N][3] or nullptr
    const double *lam;    // [S]
    const double *sinphi; // [S] sin(phi^s)
    const double *cosphi; // [S] cos(phi^s)
    const double2 *trig;  // ring of (sin, cos)(omega t_k) at index k & trig_mask
    const float4 *trig_df;  // the same ring as FP32 pairs (sin_hi, sin_lo, cos_hi, cos_lo)
    int trig_mask;
    double *vout;         // APPLY output [N][3]
    float *part;          // j-split partial sums [C][N][6] (FP32C) or [C][N][3] doubles (FP64)
    unsigned *tickets;    // per i-block arrival counters (zero between launches)
    unsigned *done;       // per-launch CTA counter (zero between launches)
    int64_t *step;        // device step counter n (advanced by the corrector)
    double *Racc;         // period-average running sum [S][3] or nullptr
    double *Rbar;         // period-average snapshots [maxK][S][3]
    int64_t avg_n0;       // step counter at which averaging started
    int64_t avg_m;        // steps per period (0 = off)
    int64_t avg_maxk;     // snapshot capacity
    int *flags;           // fault flags
    double cx, cy, cz;    // packing centre
    double a, inv6pimua, inv8pimu, k0, ell, omega, dt;
    float inv8pimu_f;     // 1 / (8 pi mu) in FP32
    float c2;             // 2 a^2 / 3 (RPY)
    float c3;             // -2 a^2     (RPY: -3 * c2)
    float overlap_r2;     // (2a)^2 in FP32 (RPY overlap threshold)
    int chunks;           // C, number of j-chunks per i-block
    int ib0, nib;         // i-blocks (of BT dumbbells) this launch computes: [ib0, ib0 + nib)
    int apply_self;       // APPLY: 1 = add self term, 0 = interaction only
    double noise_sigma;   // additive noise per step, sqrt(2 kT dt / (6 pi mu a)); 0 = off
    unsigned long long noise_seed;  // key of the noise generator
};

// Knuth two-sum: s + c accumulates p with the rounding error of every addition kept in c.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float p)
{
    float t = s + p;
    float z = t - s;
    c += (s - (t - z)) + (p - z);
    s = t;
}

// Eq. (4) rest length at time t.  sin(omega t + phi) is expanded as
// sin(omega t) cos(phi) + cos(omega t) sin(phi): sin/cos(omega t) are computed
// once per CTA (double-precision sincos, called not reimplemented) and
// sin/cos(phi) once per stroke setting, so the per-dumbbell cost is three FMAs.
__device__ __forceinline__ double rest_length(double ell, double lam, double sin_wt, double cos_wt,
                                              double sin_phi, double cos_phi)
{
    return fma(lam, fma(sin_wt, cos_phi, cos_wt * sin_phi), ell);
}

// Eq. (4) spring force on the two spheres of one dumbbell:
// F_b = -k0 (d - L) e/d, F_a = -F_b, with 1/d from one double rsqrt.
__device__ __forceinline__ void spring_force(const double xa[3], const double xb[3], double L,
                                             double k0, double Fa[3], double Fb[3])
{
    double e0 = xb[0] - xa[0], e1 = xb[1] - xa[1], e2 = xb[2] - xa[2];
    double dd = fma(e2, e2, fma(e1, e1, e0 * e0));
    double inv_d = rsqrt(dd);
    double f = k0 * fma(dd, inv_d, -L) * inv_d;
    Fa[0] = f * e0; Fa[1] = f * e1; Fa[2] = f * e2;
    Fb[0] = -Fa[0]; Fb[1] = -Fa[1]; Fb[2] = -Fa[2];
}

// Write dumbbell s's record from its FP64 positions xq[6] and forces F[6]
// (sphere 2s first).  FP32: positions are reduced by the centre in FP64 and
// rounded once; forces are rounded to FP32 and scaled there.
__device__ __forceinline__ void store_rec(DbF32 *out, int64_t s, const double xq[6],
                                          const double F[6], const EvalArgs &A)
{
    const float k = A.inv8pimu_f;
    DbF32 r;
    r.a = make_float4((float)(xq[0] - A.cx), (float)(xq[3] - A.cx), (float)(xq[1] - A.cy),
                      (float)(xq[4] - A.cy));
    r.b = make_float4((float)(xq[2] - A.cz), (float)(xq[5] - A.cz), (float)F[0] * k,
                      (float)F[3] * k);
    r.c = make_float4((float)F[1] * k, (float)F[4] * k, (float)F[2] * k, (float)F[5] * k);
    out[s] = r;
}

__device__ __forceinline__ void store_rec(DbF64 *out, int64_t s, const double xq[6],
                                          const double F[6], const EvalArgs &A)
{
    DbF64 r;
    r.x[0] = xq[0] - A.cx; r.x[1] = xq[3] - A.cx;
    r.y[0] = xq[1] - A.cy; r.y[1] = xq[4] - A.cy;
    r.z[0] = xq[2] - A.cz; r.z[1] = xq[5] - A.cz;
    r.gx[0] = F[0] * A.inv8pimu; r.gx[1] = F[3] * A.inv8pimu;
    r.gy[0] = F[1] * A.inv8pimu; r.gy[1] = F[4] * A.inv8pimu;
    r.gz[0] = F[2] * A.inv8pimu; r.gz[1] = F[5] * A.inv8pimu;
    out[s] = r;
}

// Finite test on the exponent bits (integer pipe, not the FP64 pipe).
__device__ __forceinline__ bool finite1(double v)
{
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ bool finite6(const double v[6])
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) ok &= finite1(v[k]);
    return ok;
}

}  // namespace dbs
