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
//   3. a non-owner stores its (sum, compensation) pairs with tag e;
//      the owner polls the other C-1 chunks' pairs, folds all C in chunk order,
//      runs the epilogue and publishes the next records with tag e + 1.
// Records and partials are double-buffered by the parity of e; the dependence
// chain of the algorithm guarantees that a slot is rewritten only after every
// reader of its previous contents is done.  Every wait is bounded (global
// timer); a wait that runs out raises FLAG_TIMEOUT and the CTA returns, and the
// others then run out too, so a launch always ends.
//
// Precision (FP32C).  Pair sums as in eval_kernel (FP32 pair math, two-sum
// across ranges).  Positions stay FP64 (relative to the suspension's centre).
// The spring force is formed from d^2 - L^2 computed in FP64, so that the
// small stretch d - L = (d^2 - L^2)/(d + L) keeps FP32 relative accuracy; the
// force itself, the velocity and the Heun average are FP32, as in the records.
#pragma once
#include "dbs_common.cuh"
#include "eval_kernel.cuh"

namespace dbs {

constexpr int FLOW_IB = 32;  // dumbbells per i-block (one per lane)

struct FlowArgs {
    ulonglong2 *rec;   // tagged records [2][Spad][6]: word w holds record floats 2w, 2w+1
    ulonglong2 *part;  // tagged partials [2][C][Spad][6]: word k holds (sum, compensation) of component k
    DbF32 *pack;       // plain records of the final state (the grid path's input)
    int64_t n0;        // step number at launch
    int I, q, C, K;    // i-blocks, i-blocks per chunk, chunks, Heun steps
    unsigned base;     // tag of evaluation 0
    unsigned long long timeout_ns;
};

// Owner state of one i-block, in shared memory (component-major: lane d reads
// column d).
struct FlowOwner {
    double xr[6][FLOW_IB];   // x - centre, spheres 2s (0..2) and 2s+1 (3..5)
    double R[3][FLOW_IB];    // stroke-average accumulator (trapezoid sum)
    double lam[FLOW_IB], sphi[FLOW_IB], cphi[FLOW_IB];
    float F[6][FLOW_IB];     // force at the current evaluation point
    float v0[6][FLOW_IB];    // Heun predictor velocity
    float fext[6][FLOW_IB];
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

// Record floats of dumbbell d from the owner state: positions relative to the
// centre (rounded once), G = F / (8 pi mu).
__device__ __forceinline__ void owner_record(const FlowOwner &o, int d, float k8, float r[12])
{
    r[0] = (float)o.xr[0][d]; r[1] = (float)o.xr[3][d];
    r[2] = (float)o.xr[1][d]; r[3] = (float)o.xr[4][d];
    r[4] = (float)o.xr[2][d]; r[5] = (float)o.xr[5][d];
    r[6] = o.F[0][d] * k8;  r[7] = o.F[3][d] * k8;
    r[8] = o.F[1][d] * k8;  r[9] = o.F[4][d] * k8;
    r[10] = o.F[2][d] * k8; r[11] = o.F[5][d] * k8;
}

template <int W>
struct FlowMinBlocks { static constexpr int value = W <= 4 ? 4 : 2; };

template <int MOB, int W>
__global__ void __launch_bounds__(32 * W, FlowMinBlocks<W>::value)
flow_kernel(const EvalArgs A, const FlowArgs P)
{
    extern __shared__ float4 flow_smem[];  // the chunk's records, q * 32 DbF32
    __shared__ FlowOwner own;
    __shared__ float red[W][6][FLOW_IB];
    __shared__ float2 pairs[6][FLOW_IB];   // owner: own chunk's pair, then the folded total
    __shared__ float tgt[6][FLOW_IB];      // non-owner: target positions (x0 x1 y0 y1 z0 z1)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ib = blockIdx.x / P.C, c = blockIdx.x - ib * P.C;
    const int c_own = ib / P.q;
    const bool owner = (c == c_own);
    const int S = (int)A.S;
    const int Spad = P.I * FLOW_IB;
    const int s = ib * FLOW_IB + lane;
    const bool active = s < S;
    const int db = c * P.q * FLOW_IB;
    const int m = min(db + P.q * FLOW_IB, S) - db;   // records in the chunk
    const int own_off = ib * FLOW_IB - db;          // owner: own i-block's place in the tile
    DbF32 *tile = (DbF32 *)flow_smem;
    const float k8 = A.inv8pimu_f;
    const double cen[3] = {A.cx, A.cy, A.cz};

    // ---- owner: load the state, publish the records of evaluation 0 ----------
    if (owner && warp == 0 && active) {
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            own.xr[k][lane] = A.x[o + k] - cen[k % 3];
            own.F[k][lane] = (float)A.Fd[o + k];
            own.fext[k][lane] = A.Fext ? (float)A.Fext[o + k] : 0.f;
        }
        own.lam[lane] = A.lam[s];
        own.sphi[lane] = A.sinphi[s];
        own.cphi[lane] = A.cosphi[s];
        if (A.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) own.R[k][lane] = A.Racc[3 * (int64_t)s + k];
        }
        float r[12];
        owner_record(own, lane, k8, r);
        float4 *t = (float4 *)(tile + own_off + lane);
        t[0] = make_float4(r[0], r[1], r[2], r[3]);
        t[1] = make_float4(r[4], r[5], r[6], r[7]);
        t[2] = make_float4(r[8], r[9], r[10], r[11]);
        ulonglong2 *dst = P.rec + (size_t)s * 6;
#pragma unroll
        for (int w = 0; w < 6; ++w) st_tagged(dst + w, r[2 * w], r[2 * w + 1], P.base);
    }

    const float2 c2 = make_float2(A.c2, A.c2), c3 = make_float2(A.c3, A.c3);
    for (int e = 0; e < 2 * P.K; ++e) {
        const unsigned tag = P.base + (unsigned)e;
        const int par = e & 1;
        const bool corr = (e & 1) != 0;
        const int64_t n = P.n0 + (e >> 1);
        const ulonglong2 *R = P.rec + (size_t)par * Spad * 6;

        // 1. the chunk's records (own i-block excepted on the owner) and the targets
        bool ok = true;
        for (int idx = tid; idx < m * 6; idx += 32 * W) {
            const int jr = idx / 6, w = idx - jr * 6;
            if (owner && jr >= own_off && jr < own_off + FLOW_IB) continue;
            const ulonglong2 v = wait_tagged(R + (size_t)(db + jr) * 6 + w, tag, A.flags, P.timeout_ns);
            if (!tagged(v, tag)) {
                ok = false;
                break;
            }
            float *t = (float *)(tile + jr) + 2 * w;
            t[0] = lo_float(v.x);
            t[1] = lo_float(v.y);
        }
        if (!owner && ok) {
            for (int idx = tid; idx < FLOW_IB * 3; idx += 32 * W) {
                const int d = idx / 3, w = idx - d * 3;
                if (ib * FLOW_IB + d >= S) continue;
                const ulonglong2 v =
                    wait_tagged(R + (size_t)(ib * FLOW_IB + d) * 6 + w, tag, A.flags, P.timeout_ns);
                if (!tagged(v, tag)) {
                    ok = false;
                    break;
                }
                tgt[2 * w][d] = lo_float(v.x);
                tgt[2 * w + 1][d] = lo_float(v.y);
            }
        }
        if (__syncthreads_or(!ok)) return;

        // 2. sweep: warp `warp` takes records [j0, j1) of the chunk
        float2 qa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float2 qb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float r2min = 3.0e38f;
        if (active) {
            float p[6];
            if (owner) {
                const float4 a = tile[own_off + lane].a, b = tile[own_off + lane].b;
                p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w; p[4] = b.x; p[5] = b.y;
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) p[k] = tgt[k][lane];
            }
            const float2 pax = make_float2(p[0], p[0]), pay = make_float2(p[2], p[2]);
            const float2 paz = make_float2(p[4], p[4]), pbx = make_float2(p[1], p[1]);
            const float2 pby = make_float2(p[3], p[3]), pbz = make_float2(p[5], p[5]);
            const int j0 = (m * warp) / W, j1 = (m * (warp + 1)) / W;
            if (!owner) {
#pragma unroll 2
                for (int k = j0; k < j1; ++k) {
                    const float4 ra = tile[k].a, rb = tile[k].b, rc = tile[k].c;
                    const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                    const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                    const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                    pair2<MOB, false>(pax, pay, paz, jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                      qa[2], r2min, false, false);
                    pair2<MOB, false>(pbx, pby, pbz, jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
                                      qb[2], r2min, false, false);
                }
            } else {
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

        // 3a. fold the W warp sums; a non-owner publishes its pair and is done
        ulonglong2 *Pp = P.part + (size_t)par * P.C * Spad * 6;
        for (int it = tid; it < 6 * FLOW_IB; it += 32 * W) {
            const int k = it >> 5, d = it & 31;
            if (ib * FLOW_IB + d >= S) continue;
            float sum = red[0][k][d], cmp = 0.f;
#pragma unroll
            for (int w = 1; w < W; ++w) two_sum_acc(sum, cmp, red[w][k][d]);
            if (owner) pairs[k][d] = make_float2(sum, cmp);
            else st_tagged(Pp + ((size_t)c * Spad + ib * FLOW_IB + d) * 6 + k, sum, cmp, tag);
        }
        if (!owner) continue;
        __syncthreads();

        // 3b. owner: all C pairs in chunk order
        for (int it = tid; it < 6 * FLOW_IB; it += 32 * W) {
            const int k = it >> 5, d = it & 31;
            const int sd = ib * FLOW_IB + d;
            if (sd >= S) continue;
            float sum = 0.f, cmp = 0.f;
            for (int cb = 0; cb < P.C; cb += 8) {
                // up to 8 chunks' words in flight at once, then the stragglers one by one
                ulonglong2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int cc = cb + j;
                    v[j] = (cc < P.C && cc != c) ? ld_tagged(Pp + ((size_t)cc * Spad + sd) * 6 + k)
                                                 : make_ulonglong2(0ull, 0ull);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int cc = cb + j;
                    if (cc < P.C) {
                        float ps, pc;
                        if (cc == c) {
                            ps = pairs[k][d].x;
                            pc = pairs[k][d].y;
                        } else {
                            if (!tagged(v[j], tag)) {
                                v[j] = wait_tagged(Pp + ((size_t)cc * Spad + sd) * 6 + k, tag, A.flags,
                                                   P.timeout_ns);
                                ok &= tagged(v[j], tag);
                            }
                            ps = lo_float(v[j].x);
                            pc = lo_float(v[j].y);
                        }
                        if (cc == 0) {
                            sum = ps;
                            cmp = pc;
                        } else {
                            two_sum_acc(sum, cmp, ps);
                            cmp += pc;
                        }
                    }
                }
                if (!ok) break;
            }
            // every thread has read pairs[k][d] of its own items before rewriting them
            pairs[k][d] = make_float2(sum, cmp);
        }
        if (__syncthreads_or(!ok)) return;

        // 3c. owner epilogue: one lane per dumbbell
        if (warp == 0 && active) {
            const int d = lane;
            float v[6];
#pragma unroll
            for (int k = 0; k < 6; ++k)
                v[k] = fmaf(own.F[k][d], (float)A.inv6pimua, pairs[k][d].x + pairs[k][d].y);  // Eq. (3a)
            double xq[6];
            if (!corr) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    own.v0[k][d] = v[k];
                    xq[k] = fma(A.dt, (double)v[k], own.xr[k][d]);             // x~ = x_n + dt v0
                }
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    xq[k] = fma(A.dt, (double)(0.5f * (own.v0[k][d] + v[k])), own.xr[k][d]);
                    own.xr[k][d] = xq[k];                                       // x_n + dt/2 (v0 + v1)
                }
            }
            if (!finite6(xq)) atomicOr(A.flags, FLAG_NONFINITE);
            // Eq. (4) at t_{n+1}: F_a = k0 (d - L) e/d with d - L = (d^2 - L^2)/(d + L)
            const double2 sc = A.trig[(n + 1) & A.trig_mask];
            const double L = rest_length(A.ell, own.lam[d], sc.x, sc.y, own.sphi[d], own.cphi[d]);
            const double ex = xq[3] - xq[0], ey = xq[4] - xq[1], ez = xq[5] - xq[2];
            const double dd = fma(ez, ez, fma(ey, ey, ex * ex));
            const float stretch2 = (float)fma(-L, L, dd);
            const float dist = sqrtf((float)dd);
            const float f = (float)A.k0 * (stretch2 / (dist + (float)L)) / dist;
            const float fe[3] = {f * (float)ex, f * (float)ey, f * (float)ez};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                own.F[k][d] = fe[k] + own.fext[k][d];
                own.F[3 + k][d] = -fe[k] + own.fext[3 + k][d];
            }
            if (!corr) {
                // the predictor point's record (positions of x~), kept apart from x_n
                float r[12];
                r[0] = (float)xq[0]; r[1] = (float)xq[3]; r[2] = (float)xq[1];
                r[3] = (float)xq[4]; r[4] = (float)xq[2]; r[5] = (float)xq[5];
                r[6] = own.F[0][d] * k8; r[7] = own.F[3][d] * k8; r[8] = own.F[1][d] * k8;
                r[9] = own.F[4][d] * k8; r[10] = own.F[2][d] * k8; r[11] = own.F[5][d] * k8;
                float4 *t = (float4 *)(tile + own_off + d);
                t[0] = make_float4(r[0], r[1], r[2], r[3]);
                t[1] = make_float4(r[4], r[5], r[6], r[7]);
                t[2] = make_float4(r[8], r[9], r[10], r[11]);
                ulonglong2 *dst = P.rec + ((size_t)(par ^ 1) * Spad + s) * 6;
#pragma unroll
                for (int w = 0; w < 6; ++w) st_tagged(dst + w, r[2 * w], r[2 * w + 1], tag + 1);
            } else {
                float r[12];
                owner_record(own, d, k8, r);
                float4 *t = (float4 *)(tile + own_off + d);
                t[0] = make_float4(r[0], r[1], r[2], r[3]);
                t[1] = make_float4(r[4], r[5], r[6], r[7]);
                t[2] = make_float4(r[8], r[9], r[10], r[11]);
                if (e + 1 < 2 * P.K) {
                    ulonglong2 *dst = P.rec + ((size_t)(par ^ 1) * Spad + s) * 6;
#pragma unroll
                    for (int w = 0; w < 6; ++w) st_tagged(dst + w, r[2 * w], r[2 * w + 1], tag + 1);
                } else {
                    DbF32 pr;
                    pr.a = t[0];
                    pr.b = t[1];
                    pr.c = t[2];
                    P.pack[s] = pr;
                }
                // stroke average of the geometric centre, trapezoid rule
                if (A.avg_m > 0) {
                    const int64_t k_local = n + 1 - A.avg_n0;
                    if (k_local > 0) {
                        const bool end = (k_local % A.avg_m) == 0;
                        const int64_t kidx = k_local / A.avg_m - 1;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const double Rt = 0.5 * (xq[k] + xq[3 + k]) + cen[k];
                            double acc = own.R[k][d];
                            if (end) {
                                acc += 0.5 * Rt;
                                if (kidx < A.avg_maxk)
                                    A.Rbar[kidx * 3 * A.S + 3 * (int64_t)s + k] = acc / (double)A.avg_m;
                                acc = 0.5 * Rt;
                            } else {
                                acc += Rt;
                            }
                            own.R[k][d] = acc;
                        }
                    }
                }
            }
        }
        __syncthreads();  // the tile's own records are complete before the next sweep
    }

    // ---- owner: write the state back ------------------------------------------
    if (owner && warp == 0 && active) {
        const int64_t o = 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A.x[o + k] = own.xr[k][lane] + cen[k % 3];
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
