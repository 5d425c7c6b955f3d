// Cooperative dataflow kernel: K Heun steps of one small suspension in one
// launch over all SMs, with no grid-wide barrier.
//
// Work split.  Dumbbells form i-blocks of 32 (one per lane); q consecutive
// i-blocks form a j-chunk; CTA (ib, c) sums, for the 32 targets of i-block ib,
// the pair terms of Eq. (3b) over the records of chunk c.  Its W warps split
// the chunk's records, and their sums are folded with FP32 two-sum.  The CTA
// whose chunk holds its own i-block is the i-block's owner: it keeps the
// dumbbells' state (FP64 positions, forces, Heun velocity, stroke-average
// accumulators) in shared memory for the whole launch and runs the epilogue
// (self term of Eq. (3a), Heun step of Sec. IV, spring force of Eq. (4),
// record repack, stroke average).
//
// Exchange.  Records and partial sums travel through global memory as
// flag-tagged 64-bit words (low half: the FP32 value, high half: the number of
// the evaluation they belong to).  A naturally aligned 64-bit access is
// single-copy atomic, so a reader that sees the expected tag in every word it
// reads has the value of that evaluation: no fence, ticket or barrier sits on
// the critical path.  Each evaluation:
//   1. every CTA polls the records of its chunk (and, off the owner, the
//      positions of its targets) for tag e, into shared memory;
//   2. sweeps them (W warps, one record range each) and folds the W sums;
//   3. the C CTAs of an i-block form one thread-block cluster: a non-owner
//      writes its (sum, compensation) pairs, tagged the same way, straight
//      into the owner's shared memory (DSMEM); the owner polls its own shared
//      memory for the C-1 tags, folds all C pairs in chunk order, runs the
//      epilogue and publishes the next records with tag e + 1.
// Records and partials are double-buffered by the parity of e; the dependence
// chain of the algorithm guarantees that a slot is rewritten only after every
// reader of its previous contents is done (the owner's table of pairs needs
// no second buffer: a non-owner can only start the next sweep once the owner
// has published records it folded from this table).  Every wait is bounded
// (global timer); a wait that runs out raises FLAG_TIMEOUT, the CTA stops
// working but keeps to the protocol (no early exit, so no CTA leaves while a
// cluster peer may still write its shared memory), and the others then give up
// too: a launch always ends.
//
// Precision (FP32C).  Pair sums as in eval_kernel (FP32 pair math, two-sum
// across ranges).  Positions (relative to the suspension's centre) and the
// stroke-average sums are FP64 and the Heun update is FP64.  An FP64
// instruction holds its sub-partition for 64 cycles on this part, so the
// owner spreads that work over three warps, one per axis, each on its own
// sub-partition.  The rest length L and d^2 = |x_b - x_a|^2 (from the FP64
// difference) are formed as unevaluated FP32 pairs hi + lo (double-single:
// Dekker's two-sum and the FMA two-product), so the small stretch
// d - L = (d^2 - L^2)/(d + L) keeps FP32 relative accuracy; the force and the
// velocity are FP32, as in the records.
#pragma once
#include <cooperative_groups.h>

#include "dbs_common.cuh"
#include "eval_kernel.cuh"

namespace dbs {

constexpr int FLOW_IB = 32;  // dumbbells per i-block (one per lane)

struct FlowArgs {
    ulonglong2 *rec;   // tagged records [2][Spad][6]: word w holds record floats 2w, 2w+1
    DbF32 *pack;       // plain records of the final state (the grid path's input)
    int64_t n0;        // step number at launch
    int I, q, C, K;    // i-blocks, i-blocks per chunk, chunks, Heun steps
    unsigned base;     // tag of evaluation 0
    unsigned long long timeout_ns;
};

// Owner state of one i-block, in shared memory (component-major: lane d reads
// column d).  Positions are relative to the centre; all pairs are double-single.
struct FlowOwner {
    double x[6][FLOW_IB];                   // x - centre, spheres 2s (0..2) and 2s+1 (3..5)
    double R[3][FLOW_IB];                   // stroke-average sums (trapezoid rule)
    float lamh[FLOW_IB], laml[FLOW_IB], sph[FLOW_IB], spl[FLOW_IB], cph[FLOW_IB], cpl[FLOW_IB];
    float F[6][FLOW_IB];                    // force at the current evaluation point
    float v0[6][FLOW_IB];                   // Heun predictor velocity
    float fext[6][FLOW_IB];
    float z[6][FLOW_IB];                    // additive-noise normals of the current step
    float2 e[3][FLOW_IB];                   // x_b - x_a per axis (double-single)
    float2 ee[3][FLOW_IB];                  // its square (double-single)
    float2 L[FLOW_IB], L2[FLOW_IB];         // rest length at t_{n+1} and its square
    float f[FLOW_IB];                       // k0 (d - L) / d
};

__device__ __forceinline__ ulonglong2 ld_tagged(const ulonglong2 *p)
{
    ulonglong2 v;
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_tagged(ulonglong2 *p, float a, float b, unsigned tag)
{
    const unsigned long long hi = (unsigned long long)tag << 32;
    const unsigned long long x = hi | __float_as_uint(a), y = hi | __float_as_uint(b);
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y) : "memory");
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

// Poll the tagged words p[j] (bit j of `pending`) until all carry `tag`; every round issues the
// loads of all words still missing, so a round costs one memory round trip
// however many words it waits for.  False on timeout or abort (see wait_tagged).
template <int NB>
__device__ __forceinline__ bool wait_batch(const ulonglong2 *const (&p)[NB], unsigned pending,
                                           unsigned tag, ulonglong2 (&v)[NB], int *flags,
                                           unsigned long long timeout_ns)
{
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if ((pending >> j) & 1u) v[j] = ld_tagged(p[j]);
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (((pending >> j) & 1u) && tagged(v[j], tag)) pending &= ~(1u << j);
        if (!pending) return true;
        if (it == 0) t0 = flow_ns();
        if ((it & 15u) == 15u) {
            if (*(volatile int *)flags & FLAG_TIMEOUT) return false;
            if (flow_ns() - t0 > timeout_ns) {
                atomicOr(flags, FLAG_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void put_record(DbF32 *t, const float r[12])
{
    float4 *q = (float4 *)t;
    q[0] = make_float4(r[0], r[1], r[2], r[3]);
    q[1] = make_float4(r[4], r[5], r[6], r[7]);
    q[2] = make_float4(r[8], r[9], r[10], r[11]);
}

__device__ __forceinline__ void publish_record(ulonglong2 *dst, const float r[12], unsigned tag)
{
#pragma unroll
    for (int w = 0; w < 6; ++w) st_tagged(dst + w, r[2 * w], r[2 * w + 1], tag);
}

// A tagged pair into the shared memory of cluster rank `rank` (the local
// address `local` mapped there).
__device__ __forceinline__ void st_tagged_peer(const void *local, unsigned rank, float a, float b,
                                               unsigned tag)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(local)), "r"(rank));
    const unsigned long long hi = (unsigned long long)tag << 32;
    asm volatile("st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(r),
                 "l"(hi | __float_as_uint(a)), "l"(hi | __float_as_uint(b))
                 : "memory");
}

__device__ __forceinline__ ulonglong2 ld_tagged_local(const ulonglong2 *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.cluster.shared::cta.v2.u64 {%0, %1}, [%2];"
                 : "=l"(v.x), "=l"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}

// The three normals of one sphere at step n into z[0], z[32], z[64] (kept out of
// line: the kernel's per-evaluation code stays short).
__device__ __noinline__ void draw_sphere_normals(unsigned long long seed, int64_t n, int64_t sphere,
                                                 float *z)
{
    float w[3];
    sphere_normals(seed, n, sphere, w);
    z[0] = w[0];
    z[FLOW_IB] = w[1];
    z[2 * FLOW_IB] = w[2];
}

__device__ __forceinline__ bool finite_f(float v) { return ((__float_as_uint(v) >> 23) & 0xffu) != 0xffu; }

template <int W>
struct FlowMinBlocks { static constexpr int value = W <= 4 ? 4 : (W <= 8 ? 2 : 1); };

// NOISE: additive Brownian noise on (a separate instantiation, so that the
// deterministic kernel carries none of its code).
template <int MOB, int W, bool NOISE>
__global__ void __launch_bounds__(32 * W, FlowMinBlocks<W>::value)
flow_kernel(const EvalArgs A, const FlowArgs P)
{
    constexpr int NT = 32 * W;
    namespace cg = cooperative_groups;
    // dynamic: the chunk's records (q x 32 DbF32), then the owner's table of
    // tagged chunk pairs [C][6][32]
    extern __shared__ float4 flow_smem[];
    __shared__ FlowOwner own;
    __shared__ float red[W][6][FLOW_IB];
    __shared__ float2 pairs[6][FLOW_IB];    // owner: the C pairs folded
    __shared__ float tgt[FLOW_IB][6];       // non-owner: target positions (x0 x1 y0 y1 z0 z1)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ib = blockIdx.x / P.C, c = blockIdx.x - ib * P.C;
    const int c_own = ib / P.q;
    const bool owner = (c == c_own);
    const int S = (int)A.S;
    const int Spad = P.I * FLOW_IB;
    const int s = ib * FLOW_IB + lane;
    const bool active = s < S;
    const int g_ib0 = ib * FLOW_IB;   // first dumbbell of the i-block
    const int db = c * P.q * FLOW_IB;
    const int m = min(db + P.q * FLOW_IB, S) - db;    // records in the chunk
    const int own_off = ib * FLOW_IB - db;           // owner: own i-block's place in the tile
    const int n_ib = min(FLOW_IB, S - ib * FLOW_IB);  // dumbbells of i-block ib
    DbF32 *tile = (DbF32 *)flow_smem;
    ulonglong2 *ptab = (ulonglong2 *)(tile + P.q * FLOW_IB);
    const float k8 = A.inv8pimu_f;
    const float inv6 = (float)A.inv6pimua, k0f = (float)A.k0;
    const double cen[3] = {A.cx, A.cy, A.cz};
    const ds ell = ds_of(A.ell);
    cg::cluster_group cluster = cg::this_cluster();   // the C CTAs of i-block ib, rank c
    // The exchange addresses cluster ranks 0..C-1: a launch without that shape
    // (one the host did not make) must not touch a peer's shared memory.  The
    // shape is the same for every CTA, so all of them leave here together.
    if (cluster.num_blocks() != (unsigned)P.C || cluster.block_rank() != (unsigned)c ||
        gridDim.x != (unsigned)(P.I * P.C)) {
        if (tid == 0) atomicOr(A.flags, FLAG_LAUNCH);
        return;
    }
    for (int i = tid; i < P.C * 6 * FLOW_IB; i += NT) ptab[i] = make_ulonglong2(0ull, 0ull);  // no tag is 0
    cluster.sync();   // every CTA of the cluster runs, and its table is clear, before a peer writes it

    // ---- owner: load the state, publish the records of evaluation 0 ----------
    if (owner && warp == 0 && active) {
        const int64_t o = 6 * (int64_t)s;
        float r[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            own.x[k][lane] = A.x[o + k] - cen[k % 3];
            own.F[k][lane] = (float)A.Fd[o + k];
            own.fext[k][lane] = A.Fext ? (float)A.Fext[o + k] : 0.f;
        }
        ds t = ds_of(A.lam[s]);
        own.lamh[lane] = t.h; own.laml[lane] = t.l;
        t = ds_of(A.sinphi[s]);
        own.sph[lane] = t.h; own.spl[lane] = t.l;
        t = ds_of(A.cosphi[s]);
        own.cph[lane] = t.h; own.cpl[lane] = t.l;
        if (A.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) own.R[k][lane] = A.Racc[3 * (int64_t)s + k];
        }
        r[0] = (float)own.x[0][lane]; r[1] = (float)own.x[3][lane]; r[2] = (float)own.x[1][lane];
        r[3] = (float)own.x[4][lane]; r[4] = (float)own.x[2][lane]; r[5] = (float)own.x[5][lane];
        r[6] = own.F[0][lane] * k8; r[7] = own.F[3][lane] * k8; r[8] = own.F[1][lane] * k8;
        r[9] = own.F[4][lane] * k8; r[10] = own.F[2][lane] * k8; r[11] = own.F[5][lane] * k8;
        put_record(tile + own_off + lane, r);
        publish_record(P.rec + (size_t)s * 6, r, P.base);
    }

    // words polled in step 1: the chunk's records (own i-block excepted on the
    // owner), then, off the owner, the targets' positions (3 words each)
    const int n_chunk = (m - (owner ? n_ib : 0)) * 6;
    const int n_words = n_chunk + (owner ? 0 : 3 * n_ib);
    const float2 c2 = make_float2(A.c2, A.c2), c3 = make_float2(A.c3, A.c3);

    bool dead = false;   // a wait ran out: stop working, keep the protocol
    for (int ev = 0; ev < 2 * P.K; ++ev) {
        const unsigned tag = P.base + (unsigned)ev;
        const int par = ev & 1;
        const bool corr = (ev & 1) != 0;
        const int64_t n = P.n0 + (ev >> 1);
        const ulonglong2 *R = P.rec + (size_t)par * Spad * 6;
        float4 trig = make_float4(0.f, 0.f, 1.f, 0.f);
        if (owner && warp == 3) trig = A.trig_df[(n + 1) & A.trig_mask];   // rest length, epilogue warp 3

        // 1. poll the words of this evaluation, up to 8 per thread in flight
        bool ok = !dead;
        for (int b0 = 0; b0 < n_words && ok; b0 += 8 * NT) {
            const ulonglong2 *pp[8];
            unsigned pend = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int idx = b0 + j * NT + tid;
                pp[j] = R;
                if (idx < n_chunk) {
                    const int jj = idx / 6, w = idx - jj * 6;
                    const int jr = (owner && jj >= own_off) ? jj + n_ib : jj;
                    pp[j] = R + (size_t)(db + jr) * 6 + w;
                    pend |= 1u << j;
                } else if (idx < n_words) {
                    const int t = idx - n_chunk, d = t / 3, w = t - d * 3;
                    pp[j] = R + (size_t)(ib * FLOW_IB + d) * 6 + w;
                    pend |= 1u << j;
                }
            }
            ulonglong2 v[8];
            ok = wait_batch<8>(pp, pend, tag, v, A.flags, P.timeout_ns);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!((pend >> j) & 1u)) continue;
                const int idx = b0 + j * NT + tid;
                float *dst;
                if (idx < n_chunk) {
                    const int jj = idx / 6, w = idx - jj * 6;
                    const int jr = (owner && jj >= own_off) ? jj + n_ib : jj;
                    dst = (float *)(tile + jr) + 2 * w;
                } else {
                    const int t = idx - n_chunk, d = t / 3, w = t - d * 3;
                    dst = &tgt[d][2 * w];
                }
                dst[0] = lo_float(v[j].x);
                dst[1] = lo_float(v[j].y);
            }
        }
        dead = __syncthreads_or(!ok);

        // 2. sweep: warp `warp` takes records [j0, j1) of the chunk
        float2 qa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float2 qb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (active && !dead) {
            float p[6];
            if (owner) {
                const float4 a4 = tile[own_off + lane].a, b4 = tile[own_off + lane].b;
                p[0] = a4.x; p[1] = a4.y; p[2] = a4.z; p[3] = a4.w; p[4] = b4.x; p[5] = b4.y;
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) p[k] = tgt[lane][k];
            }
            const float2 pax = make_float2(p[0], p[0]), pay = make_float2(p[2], p[2]);
            const float2 paz = make_float2(p[4], p[4]), pbx = make_float2(p[1], p[1]);
            const float2 pby = make_float2(p[3], p[3]), pbz = make_float2(p[5], p[5]);
            const int j0 = (m * warp) / W, j1 = (m * (warp + 1)) / W;
            float r2min = 3.0e38f;
            if (!owner) {
#pragma unroll 2
                for (int k = j0; k < j1; ++k) {
                    const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                    const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                    const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                    const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                    pair2<MOB, false, false>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                      qa[2], r2min, false, false);
                    pair2<MOB, false, false>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
                                      qb[2], r2min, false, false);
                }
            } else {
                // the owner's chunk holds its own dumbbells: mask the self pairs
                for (int k = j0; k < j1; ++k) {
                    const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                    const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                    const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                    const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                    const bool self = (db + k == s);
                    pair2<MOB, true>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                     qa[2], r2min, self, false);
                    pair2<MOB, true>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
                                     qb[2], r2min, false, self);
                }
            }
            if (MOB == 1 && r2min < A.overlap_r2) atomicOr(A.flags, FLAG_OVERLAP);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            red[warp][k][lane] = qa[k].x + qa[k].y;
            red[warp][3 + k][lane] = qb[k].x + qb[k].y;
        }
        __syncthreads();

        // 3a. fold the W warp sums into this chunk's pair; a non-owner writes
        // it, tagged, into the owner's table through DSMEM and is done
        float2 mine0 = {0.f, 0.f}, mine1 = {0.f, 0.f};   // owner: its own pairs (items tid, tid + NT)
        for (int it = tid, j = 0; it < 6 * FLOW_IB; it += NT, ++j) {
            const int k = it >> 5, d = it & 31;
            if (d >= n_ib || dead) continue;
            float sum = red[0][k][d], cmp = 0.f;
#pragma unroll
            for (int w = 1; w < W; ++w) two_sum_acc(sum, cmp, red[w][k][d]);
            if (owner) (j == 0 ? mine0 : mine1) = make_float2(sum, cmp);
            else st_tagged_peer(&ptab[(c * 6 + k) * FLOW_IB + d], (unsigned)c_own, sum, cmp, tag);
        }
        if (!owner) continue;

        // the normals of step n, drawn once (predictor) by the threads that have
        // no pair to poll, for the 2 x 32 spheres of the i-block
        if (NOISE && !corr) {
            for (int q = tid - (NT >= 256 ? 6 * FLOW_IB : 0); q >= 0 && q < 2 * FLOW_IB;
                 q += (NT >= 256 ? 2 * FLOW_IB : NT)) {
                const int d = q >> 1, h = q & 1;
                if (d < n_ib)
                    draw_sphere_normals(A.noise_seed, n, 2 * ((int64_t)g_ib0 + d) + h, &own.z[3 * h][d]);
            }
        }

        // 3b. owner: the other chunks' pairs, polled in its own shared memory
        // (all loads of a round in flight together), folded in chunk order
        ok = !dead;
        for (int it = tid, j = 0; it < 6 * FLOW_IB && ok; it += NT, ++j) {
            const int k = it >> 5, d = it & 31;
            if (d >= n_ib) continue;
            float sum = 0.f, cmp = 0.f;
            for (int cb = 0; cb < P.C && ok; cb += 8) {
                ulonglong2 v[8];
                unsigned pend = 0;
#pragma unroll
                for (int q8 = 0; q8 < 8; ++q8)
                    if (cb + q8 < P.C && cb + q8 != c) pend |= 1u << q8;
                unsigned long long t0 = 0;   // read the global timer only once a wait begins
                for (unsigned round = 0; pend; ++round) {
#pragma unroll
                    for (int q8 = 0; q8 < 8; ++q8)
                        if ((pend >> q8) & 1u) v[q8] = ld_tagged_local(&ptab[((cb + q8) * 6 + k) * FLOW_IB + d]);
#pragma unroll
                    for (int q8 = 0; q8 < 8; ++q8)
                        if (((pend >> q8) & 1u) && tagged(v[q8], tag)) pend &= ~(1u << q8);
                    if (pend && round == 0) t0 = flow_ns();
                    if (pend && (round & 63u) == 63u) {
                        if ((*(volatile int *)A.flags & FLAG_TIMEOUT) || flow_ns() - t0 > P.timeout_ns) {
                            atomicOr(A.flags, FLAG_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
#pragma unroll
                for (int q8 = 0; q8 < 8; ++q8) {
                    const int cc = cb + q8;
                    if (cc < P.C) {
                        const float2 mp = j == 0 ? mine0 : mine1;
                        const float ps = cc == c ? mp.x : lo_float(v[q8].x);
                        const float pc = cc == c ? mp.y : lo_float(v[q8].y);
                        if (cc == 0) {
                            sum = ps;
                            cmp = pc;
                        } else {
                            two_sum_acc(sum, cmp, ps);
                            cmp += pc;
                        }
                    }
                }
            }
            pairs[k][d] = make_float2(sum, cmp);
        }
        dead = __syncthreads_or(!ok);

        // 3c. owner epilogue.  Warps 0-2 take axis a = warp of the i-block's
        // dumbbells (lane d): self term of Eq. (3a), FP64 Heun update of both
        // spheres (Sec. IV), the axis component of e = x_b - x_a; warp 3 the rest
        // length L(t_{n+1}) of Eq. (4).  Then warp 0 the spring magnitude, and
        // warps 0-2 the forces, records and their publication.
        const int a = warp, d = lane;
        const bool eax = warp < 3 && active && !dead;
        float pa = 0.f, pb = 0.f;   // record positions along a (FP32, centre-relative)
        float eh = 0.f;
        if (eax) {
            const float va = fmaf(own.F[a][d], inv6, pairs[a][d].x + pairs[a][d].y);           // Eq. (3a)
            const float vb = fmaf(own.F[a + 3][d], inv6, pairs[a + 3][d].x + pairs[a + 3][d].y);
            double xa = own.x[a][d], xb = own.x[a + 3][d];
            if (!corr) {
                own.v0[a][d] = va;
                own.v0[a + 3][d] = vb;
                xa = fma(A.dt, (double)va, xa);                                   // x~ = x_n + dt v0
                xb = fma(A.dt, (double)vb, xb);
            } else {
                xa = fma(0.5 * A.dt, (double)(own.v0[a][d] + va), xa);           // x_n + dt/2 (v0 + v1)
                xb = fma(0.5 * A.dt, (double)(own.v0[a + 3][d] + vb), xb);
            }
            if (NOISE) {
                xa = fma(A.noise_sigma, (double)own.z[a][d], xa);
                xb = fma(A.noise_sigma, (double)own.z[a + 3][d], xb);
            }
            if (corr) {
                own.x[a][d] = xa;
                own.x[a + 3][d] = xb;
            }
            if (!(finite1(xa) && finite1(xb))) atomicOr(A.flags, FLAG_NONFINITE);
            const ds e = ds_of(xb - xa);
            const ds e2 = ds_mul(e, e);
            own.e[a][d] = make_float2(e.h, e.l);
            own.ee[a][d] = make_float2(e2.h, e2.l);
            eh = e.h;
            pa = (float)xa;
            pb = (float)xb;
            // stroke average of the geometric centre along a (corrector), trapezoid rule
            if (corr && A.avg_m > 0) {
                const int64_t k_local = n + 1 - A.avg_n0;
                if (k_local > 0) {
                    const double Rt = 0.5 * (xa + xb) + (a == 0 ? A.cx : (a == 1 ? A.cy : A.cz));
                    double acc = own.R[a][d];
                    if ((k_local % A.avg_m) == 0) {
                        acc += 0.5 * Rt;
                        const int64_t kidx = k_local / A.avg_m - 1;
                        if (kidx < A.avg_maxk) A.Rbar[kidx * 3 * A.S + 3 * (int64_t)s + a] = acc / (double)A.avg_m;
                        acc = 0.5 * Rt;
                    } else {
                        acc += Rt;
                    }
                    own.R[a][d] = acc;
                }
            }
        } else if (warp == 3 && active && !dead) {
            const ds sarg = ds_add(ds_mul({trig.x, trig.y}, {own.cph[d], own.cpl[d]}),
                                   ds_mul({trig.z, trig.w}, {own.sph[d], own.spl[d]}));
            const ds L = ds_add(ell, ds_mul({own.lamh[d], own.laml[d]}, sarg));
            const ds L2 = ds_mul(L, L);
            own.L[d] = make_float2(L.h, L.l);
            own.L2[d] = make_float2(L2.h, L2.l);
        }
        __syncthreads();
        if (warp == 0 && active && !dead) {
            // Eq. (4): F_a = k0 (d - L) e/d with d - L = (d^2 - L^2)/(d + L)
            const ds dd = ds_add(ds_add({own.ee[0][d].x, own.ee[0][d].y}, {own.ee[1][d].x, own.ee[1][d].y}),
                                 {own.ee[2][d].x, own.ee[2][d].y});
            const ds st2 = ds_add(dd, ds_neg({own.L2[d].x, own.L2[d].y}));
            const float rd = rsqrtf(dd.h);
            own.f[d] = k0f * __fdividef((st2.h + st2.l) * rd, dd.h * rd + own.L[d].x);
        }
        __syncthreads();
        if (eax) {
            const float f = own.f[d];
            const float Fa = fmaf(f, eh, own.fext[a][d]), Fb = fmaf(-f, eh, own.fext[a + 3][d]);
            own.F[a][d] = Fa;
            own.F[a + 3][d] = Fb;
            const float2 wp = make_float2(pa, pb), wg = make_float2(Fa * k8, Fb * k8);
            float2 *tr = (float2 *)(tile + own_off + d);
            tr[a] = wp;            // record word a: positions along a
            tr[3 + a] = wg;        // record word 3 + a: G along a
            if (ev + 1 < 2 * P.K) {
                ulonglong2 *dst = P.rec + ((size_t)(par ^ 1) * Spad + s) * 6;
                st_tagged(dst + a, wp.x, wp.y, tag + 1);
                st_tagged(dst + 3 + a, wg.x, wg.y, tag + 1);
            } else {
                float2 *pk = (float2 *)(P.pack + s);   // the final state's records, for the grid path
                pk[a] = wp;
                pk[3 + a] = wg;
            }
        }
        __syncthreads();  // the tile's own records are complete before the next sweep
    }
    cluster.sync();   // no CTA leaves while a peer may still write its shared memory

    // ---- owner: write the state back ------------------------------------------
    if (owner && warp == 0 && active) {
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A.x[o + k] = own.x[k][lane] + cen[k % 3];
            A.Fd[o + k] = (double)own.F[k][lane];
        }
        if (A.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) A.Racc[3 * (int64_t)s + k] = own.R[k][lane];
        }
    }
    if (blockIdx.x == 0 && tid == 0) *A.step = P.n0 + P.K;
}

// Test of the bounded wait: polls a word that nothing writes.
__global__ void wait_timeout_kernel(const ulonglong2 *word, int *flags, unsigned long long timeout_ns)
{
    wait_tagged(word, 1u, flags, timeout_ns);
}

}  // namespace dbs
