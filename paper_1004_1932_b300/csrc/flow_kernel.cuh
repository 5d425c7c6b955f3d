// Cooperative dataflow kernel: K Heun steps of one small suspension in one
// launch over up to one CTA per SM, one exchange per evaluation and no
// grid-wide barrier.
//
// Work split.  CTA g owns the T consecutive dumbbells [gT, gT + T) and, for
// each evaluation, sums the pair terms of Eq. (3b) for its own 2T target
// spheres over ALL S records: each target dumbbell has P = 256 / T slices, and
// slice p takes the records r = p + P k.  With TPW targets interleaved per warp
// (lane mod TPW; TPW = 2 for T = 2, 4 and 16), the TPW lanes that read one record
// share its 16-byte shared-memory load: 32 / TPW different records per load,
// half the shared-memory wavefronts of one target per warp (consecutive 48-byte
// records are free of bank conflicts for 16-byte loads).  The slice sums are
// folded with FP32 two-sum, first across the lanes of a warp (shuffles), then
// across the warps of a target in warp order, so no partial sum leaves the
// CTA: the CTA then runs the epilogue of its dumbbells (self term of Eq. (3a),
// Heun step of Sec. IV, spring force of Eq. (4), stroke average) and
// publishes their next records.
//
// Exchange.  Records travel through global memory as three 16-byte words, one
// per axis, each made of two single-copy-atomic 64-bit halves (a position and
// its sphere's G, whose lowest bit carries the evaluation's parity bit),
// double-buffered by evaluation parity.  A slot is rewritten (evaluation e + 2)
// only after its owner has finished evaluation e + 1, which needed every CTA's
// records of e + 1, which each CTA publishes only after it has copied all
// records of evaluation e into shared memory: a slot read for e holds e or
// e - 2, and the parity bit tells them apart.  Every wait is bounded (global
// timer and the shared abort flag); a CTA whose wait runs out raises
// FLAG_TIMEOUT and stops, the others then give up too.  No CTA touches another
// CTA's shared memory, so a CTA may leave early.
//
// Precision (FP32C).  Pair sums in FP32 with two-sum folding, as in
// eval_kernel.  Positions (relative to the suspension's centre), their Heun
// update and the stroke-average sums are FP64; an FP64 instruction holds its SM
// sub-partition for 64 cycles on this part, so that work is kept off the
// critical path: the corrector leaves its inputs in registers of the three axis
// warps, and the next poll runs it while its first round of loads is in flight.
// The critical path takes the Heun step on a double-single copy of the
// positions (refreshed from the FP64 state at every launch); the rest length L
// and d^2 = |x_b - x_a|^2 are double-single pairs hi + lo (Dekker's two-sum and
// the FMA two-product), so the small stretch d - L = (d^2 - L^2)/(d + L) keeps
// FP32 relative accuracy; the force and the velocity are FP32, as in the records.
#pragma once
#include "dbs_common.cuh"
#include "eval_kernel.cuh"

#ifndef DBS_FLOW_STAGGER
#define DBS_FLOW_STAGGER 300   // cycles between the two rounds of a poll
#endif
#ifndef DBS_FLOW_UNROLL
#define DBS_FLOW_UNROLL 8
#endif
// targets interleaved per warp (1, 2 or 4) at T = 2, 4, 8 and 16 dumbbells per CTA
#ifndef DBS_FLOW_TPW2
#define DBS_FLOW_TPW2 2
#endif
#ifndef DBS_FLOW_TPW4
#define DBS_FLOW_TPW4 2
#endif
#ifndef DBS_FLOW_TPW8
#define DBS_FLOW_TPW8 1
#endif
#ifndef DBS_FLOW_TPW16
#define DBS_FLOW_TPW16 2
#endif

namespace dbs {

constexpr int kFlowUnroll = DBS_FLOW_UNROLL;   // unroll of the sweep over a thread's records

// Tagged words are read and written with relaxed accesses at GPU scope (the
// exchange is between CTAs of one grid): each 64-bit half is single-copy atomic.
__device__ __forceinline__ ulonglong2 ld_tagged(const ulonglong2 *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool tagged(const ulonglong2 &v, unsigned tag)
{
    return (unsigned)(v.x >> 32) == tag && (unsigned)(v.y >> 32) == tag;
}

__device__ __forceinline__ unsigned long long flow_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Poll *p until both words carry `tag` and return them.  Gives up after
// timeout_ns (raising FLAG_TIMEOUT), or at once when another CTA has already
// given up; the caller sees the failure as a word without `tag`.
__device__ __noinline__ ulonglong2 wait_tagged(const ulonglong2 *p, unsigned tag, int *flags,
                                               unsigned long long timeout_ns)
{
    const unsigned long long t0 = flow_ns();
    for (unsigned it = 1;; ++it) {
        const ulonglong2 v = ld_tagged(p);
        if (tagged(v, tag)) return v;
        if ((it & 31u) == 0u) {
            if (*(volatile int *)flags & FLAG_TIMEOUT) return v;
            if (flow_ns() - t0 > timeout_ns) {
                atomicOr(flags, FLAG_TIMEOUT);
                return v;
            }
        }
    }
}

__device__ __forceinline__ float lo_float(unsigned long long w) { return __uint_as_float((unsigned)w); }

// ---- double-single (hi + lo) arithmetic, |lo| <= ulp(hi)/2 -------------------
struct ds { float h, l; };

__device__ __forceinline__ ds ds_fast(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ ds ds_add(ds a, ds b)
{
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
    return ds_fast(s, e);
}

__device__ __forceinline__ ds ds_mul(ds a, ds b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + fmaf(a.h, b.l, a.l * b.h);
    return ds_fast(p, e);
}

__device__ __forceinline__ ds ds_mul_f(ds a, float b)
{
    const float p = a.h * b;
    return ds_fast(p, fmaf(a.h, b, -p) + a.l * b);
}

__device__ __forceinline__ ds ds_of(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double ds_to_double(ds a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ds ds_neg(ds a) { return {-a.h, -a.l}; }

// ---- compact tagged record words ------------------------------------------------
// The record of dumbbell s travels as three 16-byte words, one per axis a:
// {p_a(2s), G_a(2s), p_a(2s+1), G_a(2s+1)}.  Each 64-bit half (a position and its
// sphere's G) is written and read as one single-copy-atomic access, and the lowest
// significand bit of its G carries the evaluation's parity bit, so a reader that
// sees the expected bit in a half has that evaluation's pair of values.  G is
// rounded once to FP32 and its lowest bit cleared before use, on the writer's and
// on every reader's side alike (a relative change below 2^-23).
//
// Buffers alternate by evaluation parity, so a slot read for evaluation e holds
// evaluation e or e - 2: the parity bit of e is bit 1 of e, inverted, which
// differs between the two (evaluations 0 and 1 of a zero-cleared buffer expect 1).
__device__ __forceinline__ unsigned flow_bit(unsigned e) { return ((e >> 1) & 1u) ^ 1u; }

__device__ __forceinline__ float g_clear(float g) { return __uint_as_float(__float_as_uint(g) & ~1u); }

__device__ __forceinline__ void st_word(ulonglong2 *p, float pa, float ga, float pb, float gb, unsigned bit)
{
    const unsigned long long x = (unsigned long long)((__float_as_uint(ga) & ~1u) | bit) << 32 | __float_as_uint(pa);
    const unsigned long long y = (unsigned long long)((__float_as_uint(gb) & ~1u) | bit) << 32 | __float_as_uint(pb);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
}

__device__ __forceinline__ bool word_has(const ulonglong2 &v, unsigned bit)
{
    return ((((unsigned)(v.x >> 32) ^ bit) | ((unsigned)(v.y >> 32) ^ bit)) & 1u) == 0u;
}

// Store word a of a record into its shared-memory copy (the DbF32 layout, whose
// pairs (sphere 2s, sphere 2s+1) feed the paired f32x2 instructions directly):
// positions along a into pair a, G along a (parity bit cleared) into pair 3 + a.
__device__ __forceinline__ void put_word(DbF32 *rec, int a, const ulonglong2 &v)
{
    float2 *q = (float2 *)rec;
    q[a] = make_float2(__uint_as_float((unsigned)v.x), __uint_as_float((unsigned)v.y));
    q[3 + a] = make_float2(__uint_as_float((unsigned)(v.x >> 32) & ~1u),
                           __uint_as_float((unsigned)(v.y >> 32) & ~1u));
}

__device__ __forceinline__ void put_axis(DbF32 *rec, int a, float pa, float ga, float pb, float gb)
{
    float2 *q = (float2 *)rec;
    q[a] = make_float2(pa, pb);
    q[3 + a] = make_float2(ga, gb);
}

__device__ __forceinline__ bool finite_f(float v) { return ((__float_as_uint(v) >> 23) & 0xffu) != 0xffu; }

constexpr int FLOW_NT = 256;      // threads per CTA (8 warps)
constexpr int FLOW_NW = FLOW_NT / 32;

struct FlowArgs {
    ulonglong2 *rec;   // tagged records [2][Spad][3]: word a = axis a of the dumbbell
    DbF32 *pack;       // plain records of the final state (the grid path's input)
    int64_t n0;        // step number at launch
    int G, K;          // CTAs (owners of T dumbbells each), Heun steps
    unsigned base;     // evaluation counter at evaluation 0 of the launch (even)
    unsigned long long timeout_ns;
};

// State of the T owned dumbbells, component-major (lane d reads column d).
template <int T>
struct FlowOwner {
    double x[6][T];                   // x - centre, spheres 2s (0..2) and 2s+1 (3..5)
    float2 Q[3][T];                   // stroke-average sums (trapezoid rule) of x_a + x_b - 2 c,
                                      // double-single (see flush_fp64)
    float2 xs[6][T];                  // x as double-single (hi, lo): the critical path's copy,
                                      // set from x at launch, then advanced with x
    float lamh[T], laml[T], sph[T], spl[T], cph[T], cpl[T];
    float F[6][T];                    // force at the current evaluation point
    float v0[6][T];                   // Heun predictor velocity
    float fext[6][T];
    float z[6][T];                    // additive-noise normals of the current step
    float2 ee[3][T];                  // (x_b - x_a)^2 per axis (double-single)
    float2 L[2][T], L2[2][T];         // rest length at t_{n+1} and its square, by evaluation parity
};

// (s, c) += (s2, c2) with Knuth's two-sum on the sums (exact error, any order).
__device__ __forceinline__ void ts_merge(float &s, float &c, float s2, float c2)
{
    const float t = s + s2;
    const float z = t - s;
    c += c2 + ((s - (t - z)) + (s2 - z));
    s = t;
}

// The three normals of one sphere at step n into z[0], z[stride], z[2 stride]
// (out of line: the per-evaluation code stays short).
__device__ __noinline__ void draw_sphere_normals(unsigned long long seed, int64_t n, int64_t sphere,
                                                 float *z, int stride)
{
    float w[3];
    sphere_normals(seed, n, sphere, w);
    z[0] = w[0];
    z[stride] = w[1];
    z[2 * stride] = w[2];
}

// Fold the (sum, compensation) pairs of 8 slots (the six components of one target
// dumbbell and two empty ones) across the LS consecutive lanes that hold partial
// sums of the same target, by transposition: while a lane carries more than one
// slot, each level halves them (the lane whose level bit is clear keeps the lower
// half and merges its partner's copy of it, the other lane the upper half); the
// levels left are a butterfly on the one slot.  On return the lane carries the
// M = max(1, 8 / LS) slots [base, base + M) in fs[0 .. M), fc[0 .. M).  ZERO_C:
// the compensations start at zero, so the first level moves the sums only.
// STRIDE: the target's lanes are STRIDE apart (lane bits log2(STRIDE) and up).
template <int LS, bool ZERO_C = false, int STRIDE = 1>
__device__ __forceinline__ int lane_fold(float (&fs)[8], float (&fc)[8], int lane)
{
    int base = 0;
#pragma unroll
    for (int off = (LS / 2) * STRIDE, m = 8; off >= STRIDE; off >>= 1) {
        if (m > 1) {
            const int h = m / 2;
            const bool hi = (lane & off) != 0;
            const bool first = ZERO_C && m == 8;
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const float ss = hi ? fs[k] : fs[k + h], sc = hi ? fc[k] : fc[k + h];
                const float ks = hi ? fs[k + h] : fs[k], kc = hi ? fc[k + h] : fc[k];
                const float rs = __shfl_xor_sync(0xffffffffu, ss, off);
                const float rc = first ? 0.f : __shfl_xor_sync(0xffffffffu, sc, off);
                fs[k] = ks;
                fc[k] = first ? 0.f : kc;
                ts_merge(fs[k], fc[k], rs, rc);
            }
            base += hi ? h : 0;
            m = h;
        } else {
            const float rs = __shfl_xor_sync(0xffffffffu, fs[0], off);
            const float rc = __shfl_xor_sync(0xffffffffu, fc[0], off);
            ts_merge(fs[0], fc[0], rs, rc);
        }
    }
    return base;
}

// Poll the tagged words base[j NT] (bit j of `pending`) until has(word) holds for
// each, and hand each to store(j, word) (which writes its values into the
// shared-memory copy of the records).  Two rounds of loads are kept in flight, va
// and vb, the second issued `stagger` cycles after the first, so every word is
// read twice per memory round trip: a word that becomes visible just after one
// round passed it is seen by the other about half a round trip later.  `gap()`
// runs between the two rounds, while the first is in flight.  On return one
// round may still be in flight; the caller owns va and vb, so it decides whether
// their registers stay reserved until that round has landed.  False on timeout
// or abort.
template <int NB, int NT, class Gap, class Has, class Store>
__device__ __forceinline__ bool poll_words(const ulonglong2 *base, unsigned pending, int *flags,
                                           unsigned long long timeout_ns, int stagger, Gap &&gap,
                                           Has &&has, Store &&store, ulonglong2 (&va)[NB],
                                           ulonglong2 (&vb)[NB])
{
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if ((pending >> j) & 1u) va[j] = ld_tagged(base + j * NT);
    const long long c0 = clock64();
    gap();
    while (clock64() - c0 < stagger) {
    }
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        const unsigned pb = pending;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if ((pb >> j) & 1u) vb[j] = ld_tagged(base + j * NT);
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (((pending >> j) & 1u) && has(va[j])) {
                store(j, va[j]);
                pending &= ~(1u << j);
            }
        if (!pending) return true;
        const unsigned pa = pending;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if ((pa >> j) & 1u) va[j] = ld_tagged(base + j * NT);
#pragma unroll
        for (int j = 0; j < NB; ++j)   // pending is within pb: vb[j] was loaded
            if (((pending >> j) & 1u) && has(vb[j])) {
                store(j, vb[j]);
                pending &= ~(1u << j);
            }
        if (!pending) return true;
        if (it == 0) t0 = flow_ns();
        if ((it & 7u) == 7u) {
            if (*(volatile int *)flags & FLAG_TIMEOUT) return false;
            if (flow_ns() - t0 > timeout_ns) {
                atomicOr(flags, FLAG_TIMEOUT);
                return false;
            }
        }
    }
}

// NOISE: additive Brownian noise on (a separate instantiation).
template <int MOB, int T, bool NOISE>
__global__ void __launch_bounds__(FLOW_NT, 1) flow_kernel(const EvalArgs A, const FlowArgs P)
{
    constexpr int NT = FLOW_NT;
    constexpr int PS = NT / T;                 // slices (threads) per target dumbbell
    // TPW > 1: TPW targets interleaved in each warp (lane mod TPW), so that the
    // lanes reading one record share its shared-memory load (a 16-byte load of 32
    // different records takes 4 shared-memory wavefronts, of 16 records 2)
    constexpr int TPW = T == 2    ? DBS_FLOW_TPW2
                        : T == 4  ? DBS_FLOW_TPW4
                        : T == 8  ? DBS_FLOW_TPW8
                        : T == 16 ? DBS_FLOW_TPW16
                                  : 1;
    // lanes of one target within a warp, and warps per target
    constexpr int LW = TPW == 1 ? (PS < 32 ? PS : 32) : 32 / TPW;
    constexpr int WPT = TPW == 1 ? (PS > 32 ? PS / 32 : 1) : PS / LW;
    static_assert(TPW == 1 || PS >= LW, "interleaved targets need LW slices per target");
    // words per thread and round: up to 6 words (S <= 512 in one round) the poll's
    // registers stay reserved across the evaluation, so that the round still in
    // flight when the last word arrives is never waited for; above that (larger
    // systems, whose sweep dominates) 12 words per round and the registers are
    // released after the poll
    constexpr bool KEEP = T <= 4;
    constexpr int POLL = KEEP ? 6 : 12;
    static_assert(LW >= 8, "the transposing fold needs 8 lanes per target");
    extern __shared__ float4 flow_smem[];     // all S records (Spad x DbF32)
    __shared__ FlowOwner<T> own;
    __shared__ float2 red[WPT == 1 ? T : T * WPT][6];   // folded sums per (target, warp of it)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    const int S = (int)A.S;
    const int Spad = P.G * T;
    const int st0 = g * T;                     // first owned dumbbell
    const int nown = min(T, S - st0);          // owned dumbbells (the last CTA may hold fewer)
    DbF32 *tile = (DbF32 *)flow_smem;
    const float k8 = A.inv8pimu_f;
    const float inv6 = (float)A.inv6pimua, k0f = (float)A.k0;
    const double cen[3] = {A.cx, A.cy, A.cz};
    const ds ell = ds_of(A.ell);
    const ds dt_ds = ds_of(A.dt), hdt_ds = ds_of(0.5 * A.dt), sig_ds = ds_of(A.noise_sigma);
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
            own.x[k][d] = A.x[o + k] - cen[k % 3];
            const ds xk = ds_of(own.x[k][d]);
            own.xs[k][d] = make_float2(xk.h, xk.l);
            own.F[k][d] = (float)A.Fd[o + k];
            own.fext[k][d] = A.Fext ? (float)A.Fext[o + k] : 0.f;
        }
        ds t = ds_of(A.lam[s]);
        own.lamh[d] = t.h; own.laml[d] = t.l;
        t = ds_of(A.sinphi[s]);
        own.sph[d] = t.h; own.spl[d] = t.l;
        t = ds_of(A.cosphi[s]);
        own.cph[d] = t.h; own.cpl[d] = t.l;
        if (A.avg_m > 0) {
            // the FP64 sum carried between launches, sum of w_i R_i with R the
            // geometric centre and the weights w summing to 1/2 + (k mod m) after
            // sample k, as Q = sum of w_i (x_a + x_b - 2 c)_i = 2 (sum - c sum w)
            const int64_t kl = P.n0 - A.avg_n0;
            const double sw = 0.5 + (double)(kl > 0 ? kl % A.avg_m : 0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ds q = ds_of(2.0 * (A.Racc[3 * (int64_t)s + k] - cen[k] * sw));
                own.Q[k][d] = make_float2(q.h, q.l);
            }
        }
        const unsigned bit = flow_bit(P.base);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float pa = (float)own.x[a][d], pb = (float)own.x[a + 3][d];
            const float ga = g_clear(own.F[a][d] * k8), gb = g_clear(own.F[a + 3][d] * k8);
            put_axis(tile + s, a, pa, ga, pb, gb);
            st_word(P.rec + (size_t)s * 3 + a, pa, ga, pb, gb, bit);
        }
    }
    __syncthreads();   // the owned state is read by warp 3 (rest length) in the first poll
    const float2 c2 = make_float2(A.c2, A.c2), c3 = make_float2(A.c3, A.c3);
    const int nwords = 3 * S;
    const int own_w0 = 3 * st0, own_w1 = 3 * (st0 + nown);   // words not polled (own records)
    // sweep: target and slice (TPW = 1: consecutive threads; else interleaved)
    const int t_me = TPW == 1 ? tid / PS : (warp / WPT) * TPW + lane % TPW;
    const int sl = TPW == 1 ? tid - t_me * PS : (warp % WPT) * (32 / TPW) + lane / TPW;
    const int s_me = st0 + t_me;
    const bool act = t_me < nown;
    ulonglong2 kva[KEEP ? POLL : 1], kvb[KEEP ? POLL : 1];   // the kept poll registers

    // The FP64 Heun update x_{n+1} = x_n + dt/2 (v0 + v1) (+ noise) of the state
    // and the stroke average of the geometric centre (trapezoid rule) stay off the
    // critical path: a corrector evaluation leaves their inputs in registers (hn =
    // its step n), and the next poll runs them while its first round of loads is in
    // flight (the end of the launch runs the last one).
    float hsa = 0.f, hsb = 0.f, hza = 0.f, hzb = 0.f;   // v0 + v1 and the normals along a
    int64_t hn = -1;                                    // -1: nothing pending
    // the stroke average's sample index k = n + 1 - avg_n0 of the next flush and its
    // residue mod avg_m, advanced by one per flush (the flushes take consecutive
    // steps): no 64-bit division per step.  (A 32-bit residue computed from n, and
    // advancing only with averaging on, measured slower: the gap's code is
    // sensitive to its schedule.)
    int64_t k_next = P.n0 + 1 - A.avg_n0;
    int64_t k_mod = A.avg_m > 0 ? ((k_next % A.avg_m) + A.avg_m) % A.avg_m : 0;
    auto flush_fp64 = [&]() {
        if (hn < 0) return;
        const int a = warp, d = lane;
        double xa = fma(0.5 * A.dt, (double)hsa, own.x[a][d]);
        double xb = fma(0.5 * A.dt, (double)hsb, own.x[a + 3][d]);
        if (NOISE) {
            xa = fma(A.noise_sigma, (double)hza, xa);
            xb = fma(A.noise_sigma, (double)hzb, xb);
        }
        own.x[a][d] = xa;
        own.x[a + 3][d] = xb;
        if (!(finite1(xa) && finite1(xb))) atomicOr(A.flags, FLAG_NONFINITE);
        const int64_t k_local = k_next;   // hn + 1 - avg_n0
        if (A.avg_m > 0 && k_local > 0) {
            // the sample x_a + x_b of step n + 1 from the double-single copy (FP32
            // instructions; three FP64 ones per step here cost 1-2 % of the step)
            const ds xs = ds_add({own.xs[a][d].x, own.xs[a][d].y}, {own.xs[a + 3][d].x, own.xs[a + 3][d].y});
            ds q = {own.Q[a][d].x, own.Q[a][d].y};
            if (k_mod == 0) {   // the period's last sample (weight 1/2), the next one's first
                const ds half = {0.5f * xs.h, 0.5f * xs.l};
                q = ds_add(q, half);
                const int64_t kidx = k_local / A.avg_m - 1;
                if (kidx < A.avg_maxk)
                    A.Rbar[kidx * 3 * A.S + 3 * (int64_t)(st0 + d) + a] =
                        (a == 0 ? A.cx : (a == 1 ? A.cy : A.cz)) + 0.5 * ds_to_double(q) / (double)A.avg_m;
                q = half;
            } else {
                q = ds_add(q, xs);
            }
            own.Q[a][d] = make_float2(q.h, q.l);
        }
        ++k_next;
        if (++k_mod == A.avg_m) k_mod = 0;
        hn = -1;
    };

    bool dead = false;
    for (int ev = 0; ev < 2 * P.K && !dead; ++ev) {
        const unsigned bit = flow_bit(P.base + (unsigned)ev);
        const int par = ev & 1;
        const bool corr = (ev & 1) != 0;
        const int64_t n = P.n0 + (ev >> 1);
        const ulonglong2 *R = P.rec + (size_t)par * Spad * 3;
        float4 trig = make_float4(0.f, 0.f, 1.f, 0.f);
        if (warp == 3) trig = A.trig_df[(n + 1) & A.trig_mask];   // rest length (warp 3, in the poll)
        // Eq. (4) rest length L(t_{n+1}) and its square, double-single, formed by
        // warp 3 while the records are on their way (it needs no sum); buffered by
        // evaluation parity, so the previous evaluation's spring may still read
        // the other copy
        auto rest_length_ds = [&]() {
            if (warp != 3 || lane >= nown) return;
            const int d = lane;
            const ds sarg = ds_add(ds_mul({trig.x, trig.y}, {own.cph[d], own.cpl[d]}),
                                   ds_mul({trig.z, trig.w}, {own.sph[d], own.spl[d]}));
            const ds L = ds_add(ell, ds_mul({own.lamh[d], own.laml[d]}, sarg));
            const ds L2 = ds_mul(L, L);
            own.L[par][d] = make_float2(L.h, L.l);
            own.L2[par][d] = make_float2(L2.h, L2.l);
        };
        auto gap = [&]() {
            flush_fp64();
            rest_length_ds();
        };

        // the normals of step n, drawn once (predictor) by the last 2T threads while
        // the other CTAs' records are on their way
        if (NOISE && !corr) {
            const int q = tid - (NT - 2 * T);
            if (q >= 0) {
                const int d = q >> 1, h = q & 1;
                if (d < nown)
                    draw_sphere_normals(A.noise_seed, n, 2 * ((int64_t)st0 + d) + h, &own.z[3 * h][d], T);
            }
        }

        // 1. poll the S - T records this CTA does not own, POLL words per thread
        // in two staggered rounds of loads, into shared memory
        bool ok = true;
        auto has = [&](const ulonglong2 &v) { return word_has(v, bit); };
        for (int b0 = 0; b0 < nwords && ok; b0 += POLL * NT) {
            unsigned pend = 0;
#pragma unroll
            for (int j = 0; j < POLL; ++j) {
                const int idx = b0 + j * NT + tid;
                if (idx < nwords && (idx < own_w0 || idx >= own_w1)) pend |= 1u << j;
            }
            // word idx: axis idx mod 3 of record idx / 3
            auto store = [&](int j, const ulonglong2 &v) {
                const int idx = b0 + tid + j * NT;
                put_word(tile + idx / 3, idx - 3 * (idx / 3), v);
            };
            if constexpr (KEEP) {
                ok = poll_words<POLL, NT>(R + b0 + tid, pend, A.flags, P.timeout_ns, DBS_FLOW_STAGGER, gap,
                                          has, store, kva, kvb);
            } else {
                ulonglong2 va[POLL], vb[POLL];
                ok = poll_words<POLL, NT>(R + b0 + tid, pend, A.flags, P.timeout_ns, DBS_FLOW_STAGGER, gap,
                                          has, store, va, vb);
            }
        }
        flush_fp64();   // done in the first gap: ends the live range of its inputs
        dead = __syncthreads_or(!ok);
        if (dead) break;

        // 2. sweep: target t_me against records sl, sl + PS, ... (self pair masked)
        float2 qa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float2 qb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (act) {
            const float4 a4 = tile[s_me].a, b4 = tile[s_me].b;
            const float2 pax = make_float2(a4.x, a4.x), pay = make_float2(a4.z, a4.z);
            const float2 paz = make_float2(b4.x, b4.x), pbx = make_float2(a4.y, a4.y);
            const float2 pby = make_float2(a4.w, a4.w), pbz = make_float2(b4.y, b4.y);
            // overlap minimum of r^2: one chain per target sphere at T = 2 (two
            // short dependence chains interleave better with the pair arithmetic
            // there: S = 256 4.03 -> 3.84 us per Heun step; at T = 4 they cost
            // 0.5 %, at T = 1 and 8 they change nothing), one chain otherwise
            float r2min = 3.0e38f, r2mb = 3.0e38f;
            float &r2b = T == 2 ? r2mb : r2min;
#pragma unroll kFlowUnroll
            for (int k = sl; k < S; k += PS) {
                const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                const bool self = (k == s_me);
                pair2<MOB, true>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1], qa[2],
                                 r2min, self, false);
                pair2<MOB, true>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1], qb[2],
                                 r2b, false, self);
            }
            r2min = fminf(r2min, r2mb);
            if (MOB == 1 && r2min < A.overlap_r2) atomicOr(A.flags, FLAG_OVERLAP);
        }

        // 3. fold the slices of each target: FP32 two-sum across the LW lanes of a
        // warp by transposition (lane_fold: the six components sit in eight slots,
        // each of the first three levels halves the slots a lane carries, the rest
        // is a butterfly on the one slot left: 14 shuffle pairs at LW = 32 instead
        // of 30 for a butterfly on all six), then across the WPT warps of a target
        // in warp order in the epilogue
        {
            float fs[8], fc[8];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fs[k] = qa[k].x + qa[k].y;
                fs[3 + k] = qb[k].x + qb[k].y;
            }
            fs[6] = fs[7] = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) fc[k] = 0.f;
            const int sb = lane_fold<LW, true, TPW>(fs, fc, lane);
            if (((lane / TPW) & (LW / 8 - 1)) == 0 && sb < 6)
                red[WPT == 1 ? t_me : t_me * WPT + warp % WPT][sb] = make_float2(fs[0], fc[0]);
        }
        __syncthreads();

        // 4. epilogue.  Warps 0-2 take axis a = warp of the owned dumbbells (lane d):
        // self term of Eq. (3a), Heun update of both spheres (Sec. IV) on the
        // double-single copy of the positions, the axis component of
        // e = x_b - x_a (the rest length L(t_{n+1}) of Eq. (4) was formed during
        // the poll).  Then each axis warp forms the spring magnitude (the same
        // value in the three warps, which saves a barrier), its force component,
        // writes and publishes its record words, and only then updates the FP64
        // state.
        const int a = warp, d = lane;
        const bool eax = warp < 3 && d < nown;
        float pa = 0.f, pb = 0.f, eh = 0.f;
        if (eax) {
            // the target's pair sums along a: its warps' pairs folded in warp order
            float2 ua = red[d * WPT][a], ub = red[d * WPT][a + 3];
#pragma unroll
            for (int w = 1; w < WPT; ++w) {
                ts_merge(ua.x, ua.y, red[d * WPT + w][a].x, red[d * WPT + w][a].y);
                ts_merge(ub.x, ub.y, red[d * WPT + w][a + 3].x, red[d * WPT + w][a + 3].y);
            }
            const float va = fmaf(own.F[a][d], inv6, ua.x + ua.y);           // Eq. (3a)
            const float vb = fmaf(own.F[a + 3][d], inv6, ub.x + ub.y);
            // the new positions of both spheres along a in double-single (the
            // records and the spring need FP32 accuracy; the FP64 state takes the
            // same Heun update once the records are out)
            ds na = {own.xs[a][d].x, own.xs[a][d].y}, nb = {own.xs[a + 3][d].x, own.xs[a + 3][d].y};
            // the normals are read before the barrier below: the next predictor
            // draws the next step's into the same place after it
            const float za = NOISE ? own.z[a][d] : 0.f, zb = NOISE ? own.z[a + 3][d] : 0.f;
            if (!corr) {
                own.v0[a][d] = va;
                own.v0[a + 3][d] = vb;
                na = ds_add(na, ds_mul_f(dt_ds, va));                             // x~ = x_n + dt v0
                nb = ds_add(nb, ds_mul_f(dt_ds, vb));
            } else {
                hsa = own.v0[a][d] + va;
                hsb = own.v0[a + 3][d] + vb;
                hza = za;
                hzb = zb;
                na = ds_add(na, ds_mul_f(hdt_ds, hsa));                           // x_n + dt/2 (v0 + v1)
                nb = ds_add(nb, ds_mul_f(hdt_ds, hsb));
            }
            if (NOISE) {
                na = ds_add(na, ds_mul_f(sig_ds, za));
                nb = ds_add(nb, ds_mul_f(sig_ds, zb));
            }
            const ds e = ds_add(nb, ds_neg(na));
            const ds e2 = ds_mul(e, e);
            own.ee[a][d] = make_float2(e2.h, e2.l);
            eh = e.h;
            pa = na.h + na.l;
            pb = nb.h + nb.l;
            if (corr) {   // x_{n+1}; the copy is refreshed from the FP64 state at every launch
                own.xs[a][d] = make_float2(na.h, na.l);
                own.xs[a + 3][d] = make_float2(nb.h, nb.l);
            }
            if (!(finite_f(pa) && finite_f(pb))) atomicOr(A.flags, FLAG_NONFINITE);
        }
        __syncthreads();
        if (eax) {
            // Eq. (4): F_a = k0 (d - L) e/d with d - L = (d^2 - L^2)/(d + L)
            const ds dd = ds_add(ds_add({own.ee[0][d].x, own.ee[0][d].y}, {own.ee[1][d].x, own.ee[1][d].y}),
                                 {own.ee[2][d].x, own.ee[2][d].y});
            const ds st2 = ds_add(dd, ds_neg({own.L2[par][d].x, own.L2[par][d].y}));
            const float rd = rsqrtf(dd.h);
            const float f = k0f * __fdividef((st2.h + st2.l) * rd, dd.h * rd + own.L[par][d].x);
            const float Fa = fmaf(f, eh, own.fext[a][d]), Fb = fmaf(-f, eh, own.fext[a + 3][d]);
            own.F[a][d] = Fa;
            own.F[a + 3][d] = Fb;
            const float ga = g_clear(Fa * k8), gb = g_clear(Fb * k8);
            const int s = st0 + d;
            put_axis(tile + s, a, pa, ga, pb, gb);   // record word a of the next evaluation
            if (ev + 1 < 2 * P.K) {
                st_word(P.rec + ((size_t)(par ^ 1) * Spad + s) * 3 + a, pa, ga, pb, gb,
                        flow_bit(P.base + (unsigned)ev + 1u));
            } else {
                float2 *pk = (float2 *)(P.pack + s);   // the final state's records, for the grid path
                pk[a] = make_float2(pa, pb);
                pk[3 + a] = make_float2(ga, gb);
            }
            if (corr) hn = n;   // the FP64 update of step n runs in the next poll
        }
        // no barrier here: the next poll writes only records this CTA does not own,
        // and the next sweep reads the own records after the poll's barrier
    }

    // ---- write the owned state back ----------------------------------------------
    flush_fp64();
    __syncthreads();
    if (warp == 0 && lane < nown) {
        const int d = lane, s = st0 + d;
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A.x[o + k] = own.x[k][d] + cen[k % 3];
            A.Fd[o + k] = (double)own.F[k][d];
        }
        if (A.avg_m > 0) {
            const int64_t kl = P.n0 + P.K - A.avg_n0;   // the last sample taken
            const double sw = 0.5 + (double)(kl % A.avg_m);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                A.Racc[3 * (int64_t)s + k] = cen[k] * sw + 0.5 * ds_to_double({own.Q[k][d].x, own.Q[k][d].y});
        }
    }
    if (g == 0 && tid == 0) *A.step = P.n0 + P.K;
}

// Test of the bounded wait: polls a word that nothing writes.
__global__ void wait_timeout_kernel(const ulonglong2 *word, int *flags, unsigned long long timeout_ns)
{
    wait_tagged(word, 1u, flags, timeout_ns);
}

}  // namespace dbs
