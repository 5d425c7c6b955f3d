// The all-pairs mobility evaluation with its fused Heun epilogue.
//
// One thread owns one dumbbell s, i.e. the two target spheres 2s and 2s+1,
// so that the spring force of Eq. (4), the Heun update of Sec. IV and the
// stroke-average accumulation of Eqs. (6b)/(7b) all stay in the thread's
// registers.  A CTA of BT threads owns BT dumbbells (2 BT targets) and sweeps
// one j-chunk of packed dumbbell records through shared-memory tiles; every
// record of a tile is read by all threads as a broadcast.
//
// Pair term (Eq. (3b), G = F / (8 pi mu) already folded into the record),
// r = x_i - x_j, w = 1/|r|, t = (r.G) w^2:
//   Oseen: u += w (G + r t)
//   RPY:   u += w (1 + c2 w^2) G + t w (1 + c3 w^2) r,  c2 = 2a^2/3, c3 = -2a^2
// FP32C evaluates the two spheres of a j-record together with paired f32x2
// instructions (FFMA2/FADD2/FMUL2: two IEEE single-precision lanes per
// instruction, half the issue slots of scalar code), accumulates each tile
// in FP32 and folds the tile sum into a per-target (sum, compensation) pair
// with Knuth's two-sum.
//
// With C > 1 j-chunks per i-block, each CTA writes its per-target partials and
// the last CTA of the i-block (arrival ticket) combines the C partials in chunk
// order (FP32 two-sum) and runs the epilogue, so results do not depend on CTA
// timing.
#pragma once
#include "dbs_common.cuh"
#include "noise.cuh"

// Tuning macros (defaults measured on B300 at N = 65536):
//   DBS_RPY_W35           RPY coefficients as A = w + c2 w^3, B = (r.G)(w^3 + c3 w^5)
//   DBS_UNROLL            unroll of the fast j-loop for CTAs of fewer than 256 threads
//   DBS_UNROLL_LARGE      the same for CTAs of 256 threads or more (large systems)
//   DBS_FP32_WARPS_PER_SM resident warps the FP32 kernels are register-capped for
//   DBS_W2_RCP            w^2 from rcp.approx instead of w*w (slower on B300; off)
//   DBS_UNIT_ORDER        1: work units of large CTAs in chunk-major order, 0: i-block-major
#ifndef DBS_RPY_W35
#define DBS_RPY_W35 1
#endif
#ifndef DBS_UNROLL
#define DBS_UNROLL 2
#endif
#ifndef DBS_UNROLL_LARGE
#define DBS_UNROLL_LARGE 8
#endif
#ifndef DBS_FP32_WARPS_PER_SM
#define DBS_FP32_WARPS_PER_SM 20
#endif
#ifndef DBS_W2_RCP
#define DBS_W2_RCP 0
#endif
#ifndef DBS_UNIT_ORDER
#define DBS_UNIT_ORDER 1
#endif

namespace dbs {
constexpr int kPairUnroll = DBS_UNROLL;  // unroll of the fast j-loop
}

namespace dbs {

// ---- FP32 pair terms, two j-spheres per call ----------------------------------
// Target sphere (px, py, pz), duplicated in both halves, against the two
// spheres of one j-record (half .x = sphere 2r, half .y = sphere 2r + 1).
// GUARD masks the self pair: w = 0 makes its term exactly zero.  IMIN3 selects
// how the overlap minimum of r^2 is kept: one three-input integer min on the
// bit patterns (fewer issue slots: faster in the throughput-bound large-system
// sweep) or two float mins (shorter latency: faster in the latency-bound
// cooperative and cluster-resident kernels, measured on B300).
template <int MOB, bool GUARD, bool IMIN3 = true>
__device__ __forceinline__ void pair2(const float2 px, const float2 py, const float2 pz,
                                      const float2 jx, const float2 jy, const float2 jz,
                                      const float2 gx, const float2 gy, const float2 gz,
                                      const float2 c2, const float2 c3, float2 &ux, float2 &uy,
                                      float2 &uz, float &r2min, bool skip_x, bool skip_y)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 rx = __ffma2_rn(jx, m1, px);   // px - jx, exact product by -1
    const float2 ry = __ffma2_rn(jy, m1, py);
    const float2 rz = __ffma2_rn(jz, m1, pz);
    float2 r2 = __fmul2_rn(rx, rx);
    r2 = __ffma2_rn(ry, ry, r2);
    r2 = __ffma2_rn(rz, rz, r2);
    float2 w = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    if (GUARD) {
        if (skip_x) w.x = 0.f;
        if (skip_y) w.y = 0.f;
    }
#if DBS_W2_RCP
    // w^2 = 1/r^2 from the special-function unit (approximate reciprocal, like the
    // approximate rsqrt): moves one paired multiply off the FP32 pipe
    float2 w2;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(w2.x) : "f"(r2.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(w2.y) : "f"(r2.y));
    if (GUARD) {
        if (skip_x) w2.x = 0.f;
        if (skip_y) w2.y = 0.f;
    }
#else
    const float2 w2 = __fmul2_rn(w, w);
#endif
    float2 dot = __fmul2_rn(rx, gx);
    dot = __ffma2_rn(ry, gy, dot);
    dot = __ffma2_rn(rz, gz, dot);
    const float2 t = __fmul2_rn(dot, w2);
    if (MOB == 0) {
        ux = __ffma2_rn(w, __ffma2_rn(rx, t, gx), ux);
        uy = __ffma2_rn(w, __ffma2_rn(ry, t, gy), uy);
        uz = __ffma2_rn(w, __ffma2_rn(rz, t, gz), uz);
    } else {
#if DBS_RPY_W35
        // A = w + c2 w^3, B = (r.G)(w^3 + c3 w^5): one paired op fewer than via t
        const float2 w3 = __fmul2_rn(w, w2);
        const float2 Af = __ffma2_rn(c2, w3, w);
        const float2 Bf = __fmul2_rn(dot, __ffma2_rn(c3, __fmul2_rn(w3, w2), w3));
#else
        const float2 Af = __ffma2_rn(w, __fmul2_rn(c2, w2), w);
        const float2 Bf = __fmul2_rn(t, __ffma2_rn(w, __fmul2_rn(c3, w2), w));
#endif
        ux = __ffma2_rn(Bf, rx, __ffma2_rn(Af, gx, ux));
        uy = __ffma2_rn(Bf, ry, __ffma2_rn(Af, gy, uy));
        uz = __ffma2_rn(Bf, rz, __ffma2_rn(Af, gz, uz));
        if (GUARD) {
            r2min = fminf(r2min, skip_x ? 3.0e38f : r2.x);
            r2min = fminf(r2min, skip_y ? 3.0e38f : r2.y);
        } else if (!IMIN3) {
            r2min = fminf(r2min, fminf(r2.x, r2.y));
        } else {
            // r2 >= 0, and non-negative floats order like their bit patterns read as
            // unsigned integers: one three-input integer min instead of two float
            // mins (a NaN pattern lies above every finite value, so it is ignored
            // as fminf ignores it)
            r2min = __uint_as_float(__vimin3_u32(__float_as_uint(r2min), __float_as_uint(r2.x),
                                                 __float_as_uint(r2.y)));
        }
    }
}

// ---- FP64 pair term (one j-sphere) --------------------------------------------
template <int MOB>
__device__ __forceinline__ void pair_f64(bool self, double px, double py, double pz, double jx,
                                         double jy, double jz, double gx, double gy, double gz,
                                         double c2, double c3, double &ux, double &uy, double &uz,
                                         double &r2min)
{
    double rx = px - jx, ry = py - jy, rz = pz - jz;
    double r2 = fma(rz, rz, fma(ry, ry, rx * rx));
    double w = self ? 0.0 : rsqrt(r2);
    double w2 = w * w;
    double dot = fma(rz, gz, fma(ry, gy, rx * gx));
    double t = dot * w2;
    if (MOB == 0) {
        ux = fma(w, fma(rx, t, gx), ux);
        uy = fma(w, fma(ry, t, gy), uy);
        uz = fma(w, fma(rz, t, gz), uz);
    } else {
        double Af = fma(w, c2 * w2, w);
        double Bf = t * fma(w, c3 * w2, w);
        ux = fma(Bf, rx, fma(Af, gx, ux));
        uy = fma(Bf, ry, fma(Af, gy, uy));
        uz = fma(Bf, rz, fma(Af, gz, uz));
        if (!self) r2min = fmin(r2min, r2);
    }
}

// ---- epilogue: self term, Heun, spring force, repack, period average --------
template <typename Real, int PHASE>
__device__ __forceinline__ void epilogue(const EvalArgs &A, void *pack_out, int s, const double u[6],
                                         int64_t n)
{
    using Rec = typename RecOf<Real>::type;
    const int64_t o = 6 * (int64_t)s;
    if constexpr (PHASE == PHASE_APPLY) {
        double v[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            v[k] = A.apply_self ? fma(A.Fd[o + k], A.inv6pimua, u[k]) : u[k];
        if (!finite6(v)) atomicOr(A.flags, FLAG_NONFINITE);
#pragma unroll
        for (int k = 0; k < 6; ++k) A.vout[o + k] = v[k];
    } else {
        double xq[6];  // point of the next evaluation
        double w[6] = {0, 0, 0, 0, 0, 0};  // additive noise of step n, the same in both phases
        if (A.noise_sigma > 0.0) {
            Real z[6];
            sphere_normals(A.noise_seed, n, 2 * (int64_t)s, z);
            sphere_normals(A.noise_seed, n, 2 * (int64_t)s + 1, z + 3);
#pragma unroll
            for (int k = 0; k < 6; ++k) w[k] = A.noise_sigma * (double)z[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double v = fma(A.Fd[o + k], A.inv6pimua, u[k]);  // Eq. (3a) + pair sum
            if (PHASE == PHASE_PREDICT) {
                A.v0[o + k] = v;
                xq[k] = fma(A.dt, v, A.x[o + k]) + w[k];             // x~ = x_n + dt v0 (+ noise)
            } else {
                xq[k] = fma(0.5 * A.dt, A.v0[o + k] + v, A.x[o + k]) + w[k];
                A.x[o + k] = xq[k];                                  // x_n + dt/2 (v0 + v1) (+ noise)
            }
        }
        if (!finite6(xq)) atomicOr(A.flags, FLAG_NONFINITE);
        // Eq. (4) at t_{n+1} for the point just produced
        const double2 sc = A.trig[(n + 1) & A.trig_mask];
        const double L = rest_length(A.ell, A.lam[s], sc.x, sc.y, A.sinphi[s], A.cosphi[s]);
        double Fn[6];
        spring_force(xq, xq + 3, L, A.k0, Fn, Fn + 3);
        if (A.Fext) {
#pragma unroll
            for (int k = 0; k < 6; ++k) Fn[k] += A.Fext[o + k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) A.Fd[o + k] = Fn[k];
        store_rec((Rec *)pack_out, s, xq, Fn, A);
        // stroke average of the geometric centre (corrector only), trapezoid rule
        if (PHASE == PHASE_CORRECT && A.avg_m > 0) {
            const int64_t k_local = n + 1 - A.avg_n0;
            if (k_local > 0) {
                const int64_t r = 3 * (int64_t)s;
                const bool end = (k_local % A.avg_m) == 0;
                const int64_t kidx = k_local / A.avg_m - 1;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double Rt = 0.5 * (xq[k] + xq[3 + k]);
                    double acc = A.Racc[r + k];
                    if (end) {
                        acc += 0.5 * Rt;
                        if (kidx < A.avg_maxk) A.Rbar[kidx * 3 * A.S + r + k] = acc / (double)A.avg_m;
                        acc = 0.5 * Rt;
                    } else {
                        acc += Rt;
                    }
                    A.Racc[r + k] = acc;
                }
            }
        }
    }
}

// ---- j-sweeps -------------------------------------------------------------------
// Dumbbell-record range [db, de) through tiles of TDB records.  The CTA's own
// dumbbells are [blk_lo, blk_hi); tiles that overlap them take the guarded path.
template <int MOB, int BT, int TDB>
__device__ __forceinline__ void sweep_f32(const DbF32 *__restrict__ pin, DbF32 *tile, int db,
                                          int de, int s, int blk_lo, int blk_hi, bool active,
                                          float c2s, float c3s, float s_[6], float c_[6],
                                          float &r2min)
{
    // large CTAs (the throughput-bound large-system configuration): unroll by 8
    // and the three-input integer min; small ones keep the latency-friendly forms
    constexpr int kUnroll = BT >= 256 ? DBS_UNROLL_LARGE : kPairUnroll;
    constexpr bool kImin3 = BT >= 256;
    const int tid = threadIdx.x;
    float2 pax = make_float2(0.f, 0.f), pay = pax, paz = pax, pbx = pax, pby = pax, pbz = pax;
    if (active) {
        const DbF32 me = pin[s];
        pax = make_float2(me.a.x, me.a.x);
        pay = make_float2(me.a.z, me.a.z);
        paz = make_float2(me.b.x, me.b.x);
        pbx = make_float2(me.a.y, me.a.y);
        pby = make_float2(me.a.w, me.a.w);
        pbz = make_float2(me.b.y, me.b.y);
    }
    const float2 c2 = make_float2(c2s, c2s), c3 = make_float2(c3s, c3s);
    for (int t0 = db; t0 < de; t0 += TDB) {
        const int len = min(TDB, de - t0);
        __syncthreads();
        for (int k = tid; k < len; k += BT) tile[k] = pin[t0 + k];
        __syncthreads();
        const bool diag = (t0 < blk_hi) && (t0 + len > blk_lo);
        float2 qa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float2 qb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (!diag) {
#pragma unroll kUnroll
            for (int k = 0; k < len; ++k) {
                const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                pair2<MOB, false, kImin3>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                  qa[2], r2min, false, false);
                pair2<MOB, false, kImin3>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
                                  qb[2], r2min, false, false);
            }
        } else {
            for (int k = 0; k < len; ++k) {
                const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                const bool self = (t0 + k == s);
                pair2<MOB, true>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                 qa[2], r2min, self, false);
                pair2<MOB, true>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
                                 qb[2], r2min, false, self);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            two_sum_acc(s_[k], c_[k], qa[k].x + qa[k].y);
            two_sum_acc(s_[3 + k], c_[3 + k], qb[k].x + qb[k].y);
        }
    }
}

template <int MOB, int BT, int TDB>
__device__ __forceinline__ void sweep_f64(const DbF64 *__restrict__ pin, DbF64 *tile, int db,
                                          int de, int s, bool active, double c2, double c3,
                                          double acc[6], double &r2min)
{
    const int tid = threadIdx.x;
    double ax = 0, ay = 0, az = 0, bx = 0, by = 0, bz = 0;
    if (active) {
        const DbF64 &me = pin[s];
        ax = me.x[0]; ay = me.y[0]; az = me.z[0];
        bx = me.x[1]; by = me.y[1]; bz = me.z[1];
    }
    for (int t0 = db; t0 < de; t0 += TDB) {
        const int len = min(TDB, de - t0);
        __syncthreads();
        for (int k = tid; k < len; k += BT) tile[k] = pin[t0 + k];
        __syncthreads();
        for (int k = 0; k < len; ++k) {
            const DbF64 &q = tile[k];
            const bool self = (t0 + k == s);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                pair_f64<MOB>(self && h == 0, ax, ay, az, q.x[h], q.y[h], q.z[h], q.gx[h], q.gy[h],
                              q.gz[h], c2, c3, acc[0], acc[1], acc[2], r2min);
                pair_f64<MOB>(self && h == 1, bx, by, bz, q.x[h], q.y[h], q.z[h], q.gx[h], q.gy[h],
                              q.gz[h], c2, c3, acc[3], acc[4], acc[5], r2min);
            }
        }
    }
}

// ---- the kernel ---------------------------------------------------------------
// Persistent over work units: unit u = (i-block u / C, j-chunk u % C); CTA b
// takes units b, b + gridDim.x, ...  The host picks C (see choose_launch) so
// that the units fill whole waves of the resident grid.  Indices are 32-bit
// (the host limits S to 2^29).
//
// FP32: registers capped so that DBS_FP32_WARPS_PER_SM warps stay resident
// (20 warps: at most 102 registers) for CTAs of up to 640 threads; a 512-thread
// CTA (the large-system configuration, one CTA per SM) may use up to 128.  FP64
// keeps the compiler's choice.  Dynamic shared memory:
// eval_smem_bytes(BT, TDB, C).
template <typename Real, int BT>
struct MinBlocks { static constexpr int value = sizeof(Real) == 4 ? 32 * DBS_FP32_WARPS_PER_SM / BT : 1; };

// FP32C partials are staged through shared memory when C x BT <= STAGE_MAX
// (24 KB); larger splits (large systems, where the fixup is a negligible part
// of the launch) read them from L2 directly.
constexpr int STAGE_MAX = 512;
__host__ __device__ inline bool staged_fixup(int bt, int chunks)
{
    return chunks > 1 && chunks * bt <= STAGE_MAX;
}

template <typename Real>
inline size_t eval_smem_bytes(int bt, int tdb, int chunks)
{
    const size_t t = (size_t)tdb * sizeof(typename RecOf<Real>::type);
    const size_t st = (sizeof(Real) == 4 && staged_fixup(bt, chunks))
                          ? (size_t)chunks * bt * 3 * sizeof(float4) : 0;
    return t > st ? t : st;
}

// All work units of one evaluation assigned to this CTA (the body of
// eval_kernel).
template <typename Real, int MOB, int PHASE, int BT, int TDB>
__device__ __forceinline__ void eval_units(const EvalArgs &A, const void *pack_in, void *pack_out,
                                           int64_t n, float4 *smem_dyn, int &s_last)
{
    using Rec = typename RecOf<Real>::type;
    Rec *tile = (Rec *)smem_dyn;
    float4 *stage = smem_dyn;
    const int tid = threadIdx.x;
    const Rec *pin = (const Rec *)pack_in;
    const int S = (int)A.S, C = A.chunks;
    const int iblocks = A.nib;   // all ceil(S / BT) i-blocks, or one row block of a sharded system
    const int units = iblocks * C;

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        // Large CTAs (one per SM): chunk-major, so that every i-block's last chunk
        // falls in the last wave and the i-blocks' fixups run side by side at the
        // end of the launch instead of piling onto one CTA (a CTA that did a fixup
        // lags and would arrive last, and do the fixup, in each of its following
        // i-blocks).  Smaller CTAs, several per SM, keep i-block-major order (the
        // other order costs the FP64 kernel 8 registers and one CTA per SM).
        constexpr bool kChunkMajor = DBS_UNIT_ORDER && BT >= 256;
        const int c = kChunkMajor ? unit / iblocks : unit % C;
        const int ib_ = A.ib0 + (kChunkMajor ? unit - c * iblocks : unit / C);
        const int s = ib_ * BT + tid;
        const bool active = s < S;
        const int db = (int)(((int64_t)S * c) / C);
        const int de = (int)(((int64_t)S * (c + 1)) / C);
        const int blk_lo = ib_ * BT;
        const int blk_hi = min(blk_lo + BT, S);

        if (PHASE != PHASE_APPLY && active) {
            // warm L1 with what the epilogue of this dumbbell will read, in case this
            // CTA turns out to be the last of its i-block
            const int64_t o = 6 * (int64_t)s;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.x + o));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.Fd + o));
            if (PHASE == PHASE_CORRECT) asm volatile("prefetch.global.L1 [%0];" ::"l"(A.v0 + o));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.lam + s));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.sinphi + s));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.cosphi + s));
        }
        double u[6];
        if constexpr (sizeof(Real) == 4) {
            float s_[6] = {0, 0, 0, 0, 0, 0}, c_[6] = {0, 0, 0, 0, 0, 0};
            float r2min = 3.0e38f;
            sweep_f32<MOB, BT, TDB>((const DbF32 *)pin, (DbF32 *)tile, db, de, s, blk_lo,
                                          blk_hi, active, A.c2, A.c3, s_, c_, r2min);
            if (MOB == 1 && active && r2min < A.overlap_r2) atomicOr(A.flags, FLAG_OVERLAP);
            if (C > 1) {
                if (active) {
                    float4 *dst = (float4 *)(A.part + ((int64_t)c * S + s) * 12);
                    dst[0] = make_float4(s_[0], s_[1], s_[2], c_[0]);
                    dst[1] = make_float4(c_[1], c_[2], s_[3], s_[4]);
                    dst[2] = make_float4(s_[5], c_[3], c_[4], c_[5]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) u[k] = (double)s_[k] + (double)c_[k];
            }
        } else {
            double acc[6] = {0, 0, 0, 0, 0, 0};
            double r2min = 1.0e300;
            sweep_f64<MOB, BT, TDB>((const DbF64 *)pin, (DbF64 *)tile, db, de, s, active,
                                    2.0 * A.a * A.a / 3.0, -2.0 * A.a * A.a, acc, r2min);
            if (MOB == 1 && active && r2min < 4.0 * A.a * A.a) atomicOr(A.flags, FLAG_OVERLAP);
            if (C > 1) {
                if (active) {
                    double *dst = (double *)A.part + ((int64_t)c * S + s) * 6;
#pragma unroll
                    for (int k = 0; k < 6; ++k) dst[k] = acc[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) u[k] = acc[k];
            }
        }

        bool do_epi = true;
        if (C > 1) {
            // block-level release/acquire: the barrier orders every thread's partial
            // writes before thread 0, whose fence makes them visible device-wide
            // before its arrival ticket; the last arriver fences again before the
            // CTA reads the other chunks' partials
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const unsigned prev = atomicAdd(&A.tickets[ib_], 1u);
                s_last = (prev == (unsigned)C - 1u);
                if (s_last) {
                    A.tickets[ib_] = 0u;
                    __threadfence();
                }
            }
            __syncthreads();
            do_epi = s_last;
            if (do_epi) {
                const bool staged = staged_fixup(BT, C);
                if (sizeof(Real) == 4 && staged) {
                    // stage the i-block's C x BT partial records (48 B each) into shared
                    // memory with asynchronous 16-byte copies, all in flight together
                    const int nb = blk_hi - blk_lo;      // dumbbells in this i-block
                    const int per_chunk = 3 * nb;        // float4 per chunk
                    const float4 *g = (const float4 *)A.part + (int64_t)blk_lo * 3;
                    for (int f = tid; f < C * per_chunk; f += BT) {
                        const int cc = f / per_chunk, rem = f - cc * per_chunk;
                        const unsigned sa = (unsigned)__cvta_generic_to_shared(stage + cc * 3 * BT + rem);
                        const float4 *ga = g + (int64_t)cc * S * 3 + rem;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(ga));
                    }
                    asm volatile("cp.async.commit_group;\n" ::);
                    asm volatile("cp.async.wait_group 0;\n" ::);
                    __syncthreads();
                }
                if (active) {
                    if constexpr (sizeof(Real) == 4) {
                        // the C partials combined in chunk order with FP32 two-sum, from
                        // shared memory (staged above) or, for large splits, from L2 with
                        // the next chunk's loads issued before the current one is added
                        float S_[6], C_[6];
                        const float4 *src = staged ? stage + tid * 3
                                                   : (const float4 *)(A.part + (int64_t)s * 12);
                        const int64_t stride = staged ? 3 * BT : (int64_t)S * 3;
                        float4 w0 = staged ? src[0] : __ldcg(src);
                        float4 w1 = staged ? src[1] : __ldcg(src + 1);
                        float4 w2 = staged ? src[2] : __ldcg(src + 2);
                        for (int cc = 0; cc < C; ++cc) {
                            float4 n0 = w0, n1 = w1, n2 = w2;
                            if (cc + 1 < C) {
                                const float4 *nx = src + (cc + 1) * stride;
                                n0 = staged ? nx[0] : __ldcg(nx);
                                n1 = staged ? nx[1] : __ldcg(nx + 1);
                                n2 = staged ? nx[2] : __ldcg(nx + 2);
                            }
                            // layout: a: s0 s1 s2 c0 c1 c2, b: s0 s1 s2 c0 c1 c2
                            const float ps[6] = {w0.x, w0.y, w0.z, w1.z, w1.w, w2.x};
                            const float pc[6] = {w0.w, w1.x, w1.y, w2.y, w2.z, w2.w};
                            if (cc == 0) {
#pragma unroll
                                for (int k = 0; k < 6; ++k) {
                                    S_[k] = ps[k];
                                    C_[k] = pc[k];
                                }
                            } else {
#pragma unroll
                                for (int k = 0; k < 6; ++k) {
                                    two_sum_acc(S_[k], C_[k], ps[k]);
                                    C_[k] += pc[k];
                                }
                            }
                            w0 = n0;
                            w1 = n1;
                            w2 = n2;
                        }
#pragma unroll
                        for (int k = 0; k < 6; ++k) u[k] = (double)S_[k] + (double)C_[k];
                    } else {
#pragma unroll
                        for (int k = 0; k < 6; ++k) u[k] = 0.0;
                        for (int cc = 0; cc < C; ++cc) {
                            const double *src = (const double *)A.part + ((int64_t)cc * S + s) * 6;
#pragma unroll
                            for (int k = 0; k < 6; ++k) u[k] += __ldcg(src + k);
                        }
                    }
                }
            }
        }
        if (do_epi && active) epilogue<Real, PHASE>(A, pack_out, s, u, n);
    }
}

template <typename Real, int MOB, int PHASE, int BT, int TDB>
__global__ void __launch_bounds__(BT, (MinBlocks<Real, BT>::value)) eval_kernel(const EvalArgs A)
{
    // dynamic shared memory, max(TDB records, C x BT x 48 B): the j-tile during
    // the sweep, then (FP32C, last CTA of an i-block) the staged chunk partials
    extern __shared__ float4 smem_dyn[];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    // Programmatic dependent launch: this grid may have been scheduled before the
    // previous evaluation finished; wait for it (and its memory) before reading
    // anything it wrote, then allow the next evaluation to be scheduled.  Both
    // are no-ops for an ordinary launch.
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int64_t n = *A.step;
    eval_units<Real, MOB, PHASE, BT, TDB>(A, A.pack_in, A.pack_out, n, smem_dyn, s_last);

    if (PHASE == PHASE_CORRECT) {
        // the last CTA of the launch advances the device step counter; every CTA
        // has read *A.step before it arrives here
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(A.done, 1u);
            if (prev == gridDim.x - 1u) {
                *A.done = 0u;
                *A.step = n + 1;
                __threadfence();
            }
        }
    }
}

}  // namespace dbs
