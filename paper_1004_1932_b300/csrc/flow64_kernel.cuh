// Cooperative dataflow kernel in double precision: K Heun steps (Sec. IV) of a
// small all-FP64 suspension in one launch, the design of flow_kernel with every
// value in FP64.
//
// On this part an FP64 instruction holds its SM sub-partition for 64 cycles,
// whatever the number of active lanes, so the split is chosen for FP64
// parallelism rather than for FP32 issue: 128 threads per CTA (one warp per
// sub-partition), T <= 4 dumbbells per CTA (at most 4 x 148 = 592 dumbbells),
// and the pair terms of the CTA's 2T target spheres dealt to the warps
// round-robin, so that the four FP64 pipes share them.
//
// Work of one evaluation, CTA g owning dumbbells [gT, gT + T):
//   1. poll the other CTAs' records of this evaluation into shared memory (two
//      staggered rounds of relaxed loads, as flow_kernel);
//   2. thread (warp w, lane l) takes target sphere t = l mod 2T and the source
//      spheres j = sl, sl + 64/T, ... with slice sl = (l div 2T) 4 + w, and sums
//      the pair terms of Eq. (3b) in FP64 (the self pair masked);
//   3. fold the slices of a target across the lanes of each warp (a transposing
//      fold: the three components and a zero sit in four slots, the first two
//      shuffle levels halve the slots a lane carries, the rest is a butterfly),
//      then across the four warps in warp order;
//   4. warp 0, lane (axis a, dumbbell d): self term of Eq. (3a), Heun step of
//      both spheres, e = x_b - x_a; the lanes of one dumbbell exchange their
//      axis components by shuffles (no barrier) and form the spring force of
//      Eq. (4) at t_{n+1} (its rest length formed by warp 1 during the poll),
//      write the next records and publish them.
//
// Exchange.  A record is the grid path's DbF64 (positions relative to the
// centre, G = F / (8 pi mu)) sent as six 16-byte words: word k holds component
// k (x, y, z, Gx, Gy, Gz) of sphere 2s and of sphere 2s + 1.  The lowest
// significand bit of every double carries the evaluation's parity bit
// (flow_bit), and the writer and every reader use the value with that bit
// cleared (a relative change below 2^-52, the same on all sides), so the pair
// sum of a dumbbell's spheres does not depend on the CTA that computes it.  Each
// 64-bit half is single-copy atomic; buffers alternate by evaluation parity, with
// the ordering argument of flow_kernel.  The FP64 state itself (positions,
// forces, stroke-average sums) is never rounded.
#pragma once
#include "flow_kernel.cuh"

namespace dbs {

constexpr int FLOW64_NT = 128;            // threads per CTA (4 warps)
constexpr int FLOW64_NW = FLOW64_NT / 32;
constexpr int FLOW64_POLL = 8;            // words per thread and round of a poll

struct Flow64Args {
    ulonglong2 *rec;   // tagged records [2][Spad][6]: word k = component k of both spheres
    DbF64 *pack;       // plain records of the final state (the grid path's input)
    int64_t n0;        // step number at launch
    int G, K;          // CTAs (owners of T dumbbells each), Heun steps
    unsigned base;     // evaluation counter at evaluation 0 of the launch (even)
    unsigned long long timeout_ns;
};

__device__ __forceinline__ double d_clear(double v)
{
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) & ~1ull));
}

__device__ __forceinline__ unsigned long long d_tag(double v, unsigned bit)
{
    return ((unsigned long long)__double_as_longlong(v) & ~1ull) | bit;
}

__device__ __forceinline__ void st_word64(ulonglong2 *p, double a, double b, unsigned bit)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(d_tag(a, bit)),
                 "l"(d_tag(b, bit))
                 : "memory");
}

__device__ __forceinline__ bool word64_has(const ulonglong2 &v, unsigned bit)
{
    return (((v.x ^ bit) | (v.y ^ bit)) & 1ull) == 0ull;
}

// State of the T owned dumbbells, component-major (lane d reads column d).
template <int T>
struct Flow64Owner {
    double x[6][T];      // x - centre, spheres 2s (0..2) and 2s+1 (3..5)
    double F[6][T];      // force at the current evaluation point
    double v0[6][T];     // Heun predictor velocity
    double fext[6][T];
    double R[3][T];      // stroke-average sums (trapezoid rule)
    double lam[T], sph[T], cph[T];
    double L[2][T];      // rest length L(t_{n+1}), by evaluation parity
};

template <int MOB, int T>
__global__ void __launch_bounds__(FLOW64_NT, 1) flow64_kernel(const EvalArgs A, const Flow64Args P)
{
    constexpr int NT = FLOW64_NT, NW = FLOW64_NW;
    constexpr int NTG = 2 * T;            // target spheres per CTA
    constexpr int NSL = NT / NTG;         // slices per target sphere
    constexpr int SPW = 32 / NTG;         // slices of one target within a warp
    static_assert(T == 1 || T == 2 || T == 4, "FP64 cooperative split: 1, 2 or 4 dumbbells per CTA");
    static_assert(SPW >= 4, "the transposing fold needs 4 lanes per target in a warp");
    extern __shared__ double2 flow64_smem[];   // all S records (Spad x DbF64)
    __shared__ Flow64Owner<T> own;
    __shared__ double red[NW][NTG][3];         // folded sums per (warp, target, component)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    const int S = (int)A.S;
    const int Spad = P.G * T;
    const int st0 = g * T;
    const int nown = min(T, S - st0);
    DbF64 *tile = (DbF64 *)flow64_smem;
    auto cen = [&](int k) { return k == 0 ? A.cx : (k == 1 ? A.cy : A.cz); };   // packing centre
    if (gridDim.x != (unsigned)P.G || blockDim.x != (unsigned)NT) {   // not the shape the host made
        if (tid == 0) atomicOr(A.flags, FLAG_LAUNCH);
        return;
    }

    // ---- load the owned state, publish the records of evaluation 0 -----------
    if (warp == 0 && lane < nown) {
        const int d = lane, s = st0 + d;
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            own.x[k][d] = A.x[o + k] - cen(k % 3);
            own.F[k][d] = A.Fd[o + k];
            own.fext[k][d] = A.Fext ? A.Fext[o + k] : 0.0;
        }
        own.lam[d] = A.lam[s];
        own.sph[d] = A.sinphi[s];
        own.cph[d] = A.cosphi[s];
        if (A.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) own.R[k][d] = A.Racc[3 * (int64_t)s + k];
        }
        const unsigned bit = flow_bit(P.base);
        double2 *q = (double2 *)(tile + s);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double pa = d_clear(own.x[a][d]), pb = d_clear(own.x[a + 3][d]);
            const double ga = d_clear(own.F[a][d] * A.inv8pimu), gb = d_clear(own.F[a + 3][d] * A.inv8pimu);
            q[a] = make_double2(pa, pb);
            q[3 + a] = make_double2(ga, gb);
            st_word64(P.rec + (size_t)s * 6 + a, pa, pb, bit);
            st_word64(P.rec + (size_t)s * 6 + 3 + a, ga, gb, bit);
        }
    }
    __syncthreads();   // warp 1 reads the stroke parameters in the first poll

    const double c2 = 2.0 * A.a * A.a / 3.0, c3 = -2.0 * A.a * A.a;
    const int nwords = 6 * S;
    const int own_w0 = 6 * st0, own_w1 = 6 * (st0 + nown);   // words not polled (own records)
    // sweep: target sphere ti (dumbbell ti / 2, sphere ti & 1) and slice sl
    const int ti = lane % NTG;
    const int sl = (lane / NTG) * NW + warp;
    const int i_me = 2 * st0 + ti;                            // global target sphere
    const bool act = (ti >> 1) < nown;
    // epilogue: warp 0, lane (axis ea, dumbbell ed)
    const int ea = lane / T, ed = lane - (lane / T) * T;
    const bool eax = warp == 0 && ea < 3 && ed < nown;

    int64_t hn = -1;   // stroke average of step hn pending (warp 0, axis lanes), -1: none
    auto flush_avg = [&]() {
        if (hn < 0) return;
        const int a = ea, d = ed;
        const int64_t k_local = hn + 1 - A.avg_n0;
        if (A.avg_m > 0 && k_local > 0) {
            const double Rt = 0.5 * (own.x[a][d] + own.x[a + 3][d]) + cen(a);
            double acc = own.R[a][d];
            if ((k_local % A.avg_m) == 0) {
                acc += 0.5 * Rt;
                const int64_t kidx = k_local / A.avg_m - 1;
                if (kidx < A.avg_maxk) A.Rbar[kidx * 3 * A.S + 3 * (int64_t)(st0 + d) + a] = acc / (double)A.avg_m;
                acc = 0.5 * Rt;
            } else {
                acc += Rt;
            }
            own.R[a][d] = acc;
        }
        hn = -1;
    };

    bool dead = false;
    for (int ev = 0; ev < 2 * P.K && !dead; ++ev) {
        const unsigned bit = flow_bit(P.base + (unsigned)ev);
        const int par = ev & 1;
        const bool corr = (ev & 1) != 0;
        const int64_t n = P.n0 + (ev >> 1);
        const ulonglong2 *R = P.rec + (size_t)par * Spad * 6;

        // work for the poll's gap: the rest length L(t_{n+1}) of Eq. (4) (warp 1, lane
        // d), the pending stroke average (warp 0)
        bool gap_done = false;
        auto gap = [&]() {
            if (gap_done) return;
            gap_done = true;
            if (warp == 1 && lane < nown) {
                const double2 sc = A.trig[(n + 1) & A.trig_mask];
                own.L[par][lane] = rest_length(A.ell, own.lam[lane], sc.x, sc.y, own.sph[lane], own.cph[lane]);
            }
            if (eax) flush_avg();
        };

        // 1. poll the records this CTA does not own into shared memory
        bool ok = true;
        auto has = [&](const ulonglong2 &v) { return word64_has(v, bit); };
        for (int b0 = 0; b0 < nwords && ok; b0 += FLOW64_POLL * NT) {
            unsigned pend = 0;
#pragma unroll
            for (int j = 0; j < FLOW64_POLL; ++j) {
                const int idx = b0 + j * NT + tid;
                if (idx < nwords && (idx < own_w0 || idx >= own_w1)) pend |= 1u << j;
            }
            // word idx: component idx mod 6 of record idx / 6, both spheres, bit cleared
            auto store = [&](int j, const ulonglong2 &v) {
                const int idx = b0 + tid + j * NT;
                ((double2 *)flow64_smem)[idx] =
                    make_double2(__longlong_as_double((long long)(v.x & ~1ull)),
                                 __longlong_as_double((long long)(v.y & ~1ull)));
            };
            ulonglong2 va[FLOW64_POLL], vb[FLOW64_POLL];
            ok = poll_words<FLOW64_POLL, NT>(R + b0 + tid, pend, A.flags, P.timeout_ns, DBS_FLOW_STAGGER, gap,
                                             has, store, va, vb);
        }
        gap();   // a thread with no batch to poll still takes its share of the gap's work
        dead = __syncthreads_or(!ok);
        if (dead) break;

        // 2. sweep: target sphere i_me against sources sl, sl + NSL, ... (self pair masked)
        double ux = 0.0, uy = 0.0, uz = 0.0, r2min = 1.0e300;
        if (act) {
            const DbF64 &me = tile[st0 + (ti >> 1)];
            const int hh = ti & 1;
            const double px = me.x[hh], py = me.y[hh], pz = me.z[hh];
            for (int j = sl; j < 2 * S; j += NSL) {
                const DbF64 &q = tile[j >> 1];
                const int h = j & 1;
                pair_f64<MOB>(j == i_me, px, py, pz, q.x[h], q.y[h], q.z[h], q.gx[h], q.gy[h], q.gz[h], c2,
                              c3, ux, uy, uz, r2min);
            }
            if (MOB == 1 && r2min < 4.0 * A.a * A.a) atomicOr(A.flags, FLAG_OVERLAP);
        }

        // 3. fold: slots (ux, uy, uz, 0); lanes of target ti differ in lane bits
        // NTG, 2 NTG, ... 16.  Level NTG: a lane keeps slots {0, 1} (bit clear) or
        // {2, 3} and adds its partner's copy; level 2 NTG: one slot; then a butterfly.
        {
            const bool hi1 = (lane & NTG) != 0, hi2 = (lane & (2 * NTG)) != 0;
            const double k0 = hi1 ? uz : ux, k1 = hi1 ? 0.0 : uy;        // kept
            const double s0 = hi1 ? ux : uz, s1 = hi1 ? uy : 0.0;        // sent
            const double m0 = k0 + __shfl_xor_sync(0xffffffffu, s0, NTG);
            const double m1 = k1 + __shfl_xor_sync(0xffffffffu, s1, NTG);
            double v = (hi2 ? m1 : m0) + __shfl_xor_sync(0xffffffffu, hi2 ? m0 : m1, 2 * NTG);
#pragma unroll
            for (int off = 4 * NTG; off < 32; off *= 2) v += __shfl_xor_sync(0xffffffffu, v, off);
            const int slot = (hi1 ? 2 : 0) + (hi2 ? 1 : 0);
            if (lane < 4 * NTG && slot < 3) red[warp][ti][slot] = v;
        }
        __syncthreads();

        // 4. epilogue (warp 0): lane (a, d) forms the axis-a velocity of both spheres
        // of dumbbell d (the four warps' sums in warp order plus the self term of
        // Eq. (3a)), their Heun update, and e_a = x_b - x_a; the dumbbell's lanes then
        // share e and each forms the spring force of Eq. (4) along its axis
        if (warp == 0) {
            const int a = ea, d = ed;
            double qa = 0.0, qb = 0.0, e = 0.0;
            if (eax) {
                double ua = red[0][2 * d][a], ub = red[0][2 * d + 1][a];
#pragma unroll
                for (int w = 1; w < NW; ++w) {
                    ua += red[w][2 * d][a];
                    ub += red[w][2 * d + 1][a];
                }
                const double va = fma(own.F[a][d], A.inv6pimua, ua);       // Eq. (3a) + pair sum
                const double vb = fma(own.F[a + 3][d], A.inv6pimua, ub);
                if (!corr) {
                    own.v0[a][d] = va;
                    own.v0[a + 3][d] = vb;
                    qa = fma(A.dt, va, own.x[a][d]);                          // x~ = x_n + dt v0
                    qb = fma(A.dt, vb, own.x[a + 3][d]);
                } else {
                    qa = fma(0.5 * A.dt, own.v0[a][d] + va, own.x[a][d]);     // x_n + dt/2 (v0 + v1)
                    qb = fma(0.5 * A.dt, own.v0[a + 3][d] + vb, own.x[a + 3][d]);
                    own.x[a][d] = qa;
                    own.x[a + 3][d] = qb;
                }
                e = qb - qa;
                if (!(finite1(qa) && finite1(qb))) atomicOr(A.flags, FLAG_NONFINITE);
            }
            const double ex = __shfl_sync(0xffffffffu, e, d);
            const double ey = __shfl_sync(0xffffffffu, e, T + d);
            const double ez = __shfl_sync(0xffffffffu, e, 2 * T + d);
            if (eax) {
                // Eq. (4): F_b = -k0 (|e| - L) e/|e|, F_a = -F_b (as the grid path's spring_force)
                const double dd = fma(ez, ez, fma(ey, ey, ex * ex));
                const double inv_d = rsqrt(dd);
                const double f = A.k0 * fma(dd, inv_d, -own.L[par][d]) * inv_d;
                double Fa = f * e, Fb = -Fa;
                if (A.Fext) {
                    Fa += own.fext[a][d];
                    Fb += own.fext[a + 3][d];
                }
                own.F[a][d] = Fa;
                own.F[a + 3][d] = Fb;
                const double Ga = Fa * A.inv8pimu, Gb = Fb * A.inv8pimu;
                const int s = st0 + d;
                double2 *tq = (double2 *)(tile + s);
                const double pa = d_clear(qa), pb = d_clear(qb), ga = d_clear(Ga), gb = d_clear(Gb);
                tq[a] = make_double2(pa, pb);           // components a and 3 + a of the next record
                tq[3 + a] = make_double2(ga, gb);
                if (ev + 1 < 2 * P.K) {
                    const unsigned nb = flow_bit(P.base + (unsigned)ev + 1u);
                    ulonglong2 *dst = P.rec + ((size_t)(par ^ 1) * Spad + s) * 6;
                    st_word64(dst + a, pa, pb, nb);
                    st_word64(dst + 3 + a, ga, gb, nb);
                } else {
                    double2 *pk = (double2 *)(P.pack + s);   // the final state's records, unrounded
                    pk[a] = make_double2(qa, qb);
                    pk[3 + a] = make_double2(Ga, Gb);
                }
                if (corr) hn = n;   // its stroke average runs in the next poll's gap
            }
        }
        // The other warps wait here for warp 0's epilogue: started at once, their
        // polls ran ahead of this CTA's own publish and every evaluation took longer
        // (S = 16 / 64 / 148: 7.3-7.7 / 9.6-10.5 / 15.7-16.2 us per Heun step without
        // this barrier, 6.8 / 8.5 / 13.6 with it, measured).  The next poll writes
        // only records this CTA does not own.
        __syncthreads();
    }

    // ---- write the owned state back ----------------------------------------------
    if (eax) flush_avg();
    __syncthreads();
    if (warp == 0 && lane < nown) {
        const int d = lane, s = st0 + d;
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A.x[o + k] = own.x[k][d] + cen(k % 3);
            A.Fd[o + k] = own.F[k][d];
        }
        if (A.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) A.Racc[3 * (int64_t)s + k] = own.R[k][d];
        }
    }
    if (g == 0 && tid == 0) *A.step = P.n0 + P.K;
}

}  // namespace dbs
