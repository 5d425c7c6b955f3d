// Cluster-resident multi-step kernel: a thread-block cluster of G CTAs holds
// one whole suspension and advances it K Heun steps (Sec. IV) in one launch.
//
// Layout per CTA (dynamic shared memory):
//   rec[2][S]         packed j-records of all S dumbbells, double-buffered
//                     (evaluation e reads rec[e & 1], writes rec[(e + 1) & 1])
//   part[JS][TP][12]  per-j-split partial sums of the CTA's TP target dumbbells
// CTA rank r of the cluster owns target dumbbells [r S / G, (r + 1) S / G).
// Thread t works on target lt = t % TP over j-split js = t / TP of the
// j-range; the JS partials of a target are combined in js order with FP32
// two-sum, then the js == 0 thread runs the FP64 epilogue (self term, Heun,
// spring force, period average) on state it keeps in registers for the
// whole launch, and stores the new record of its dumbbell into the next
// buffer of every CTA of the cluster (distributed shared memory).  One
// hardware cluster barrier per evaluation separates the writes of the next
// buffer from its reads; no global memory is touched between evaluations.
#pragma once
#include <cooperative_groups.h>

#include "dbs_common.cuh"
#include "eval_kernel.cuh"

namespace dbs {

namespace cg = cooperative_groups;

// One member suspension of a resident launch (global memory, read-only in
// the kernel except for the state it advances).
struct ResSys {
    int S;            // dumbbells
    int G;            // cluster size of this member
    int K;            // Heun steps of this member in this launch (<= the launch's K)
    double inv6pimua, k0, ell, dt;
    float c2, c3, overlap_r2;
    double *x, *v0, *Fd;        // [2S][3] FP64 state (read at start, written at end)
    const double *Fext;         // [2S][3] or nullptr
    const double *lam, *sinphi, *cosphi;
    void *pack;                 // DbF32 [S] records of the current state (read, written)
    const double2 *trig;        // (sin, cos)(omega t_k) ring
    int trig_mask;
    int64_t *step;              // device step counter
    int *flags;                 // fault flags
    double *Racc, *Rbar;        // stroke-average accumulator / snapshots
    int64_t avg_n0, avg_m, avg_maxk;
    double noise_sigma;         // additive noise per step (0 = off)
    unsigned long long noise_seed;
    EvalArgs pack_args;         // centre and scaling used by store_rec
};

__host__ __device__ inline size_t resident_smem_bytes(int S, int G, int nt)
{
    const int tp = (S + G - 1) / G;
    const int js = (tp > 0) ? (nt / tp > S ? S : nt / tp) : 1;
    return (size_t)2 * S * sizeof(DbF32) + (size_t)(js < 1 ? 1 : js) * tp * 12 * sizeof(float);
}

// One target dumbbell (spheres a, b) against records [db, de): FP32 sums of
// 64 records at a time folded into (sum, compensation) with two-sum.
template <int MOB>
__device__ __forceinline__ void res_sweep(const DbF32 *rec, int db, int de, int s, float c2s,
                                          float c3s, const float2 pa[3], const float2 pb[3],
                                          float s_[6], float c_[6], float &r2min)
{
    const float2 c2 = make_float2(c2s, c2s), c3 = make_float2(c3s, c3s);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s_[k] = 0.f;
        c_[k] = 0.f;
    }
    for (int k0 = db; k0 < de; k0 += 64) {
        const int k1 = min(k0 + 64, de);
        float2 qa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float2 qb[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (!(s >= k0 && s < k1)) {
#pragma unroll 2
            for (int k = k0; k < k1; ++k) {
                const float4 ra = rec[k].a, rb = rec[k].b, rc = rec[k].c;
                const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                pair2<MOB, false, false>(pa[0], pa[1], pa[2], jx, jy, jz, gx, gy, gz, c2, c3, qa[0],
                                  qa[1], qa[2], r2min, false, false);
                pair2<MOB, false, false>(pb[0], pb[1], pb[2], jx, jy, jz, gx, gy, gz, c2, c3, qb[0],
                                  qb[1], qb[2], r2min, false, false);
            }
        } else {
            for (int k = k0; k < k1; ++k) {
                const float4 ra = rec[k].a, rb = rec[k].b, rc = rec[k].c;
                const float2 jx = make_float2(ra.x, ra.y), jy = make_float2(ra.z, ra.w);
                const float2 jz = make_float2(rb.x, rb.y), gx = make_float2(rb.z, rb.w);
                const float2 gy = make_float2(rc.x, rc.y), gz = make_float2(rc.z, rc.w);
                const bool self = (k == s);
                pair2<MOB, true>(pa[0], pa[1], pa[2], jx, jy, jz, gx, gy, gz, c2, c3, qa[0], qa[1],
                                 qa[2], r2min, self, false);
                pair2<MOB, true>(pb[0], pb[1], pb[2], jx, jy, jz, gx, gy, gz, c2, c3, qb[0], qb[1],
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

// P.K Heun steps of the cluster's suspension (members of one launch may take
// different step counts).  Grid = nclust clusters of Gl CTAs (all members of a
// launch share the cluster size); csys[cluster] is the member index.  NT
// threads per CTA.  A launch in any other shape (a tool that drops the cluster
// dimension, say) would index csys past its end: every CTA checks the shape
// first, and on a mismatch all of them (the test is grid-uniform) raise
// FLAG_LAUNCH on the first member and return before any cluster barrier.
template <int MOB, int NT>
__global__ void __launch_bounds__(NT, 1)
resident_kernel(const ResSys *__restrict__ systems, const int *__restrict__ csys, int nclust, int Gl)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int G = (int)cluster.num_blocks();
    if (G != Gl || gridDim.x != (unsigned)(Gl * nclust) || blockDim.x != (unsigned)NT) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(systems[csys[0]].flags, FLAG_LAUNCH);
        return;
    }
    const int r = (int)cluster.block_rank();
    const int cid = blockIdx.x / G;
    const ResSys &P = systems[csys[cid]];
    const int S = P.S;
    const int K = P.K;
    if (K <= 0) return;  // the whole cluster sits out this launch
    const int t0 = (int)(((int64_t)S * r) / G), t1 = (int)(((int64_t)S * (r + 1)) / G);
    const int TP = t1 - t0;
    const int tp_max = (S + G - 1) / G;
    const int JS = max(1, min(NT / tp_max, S));

    extern __shared__ float4 smem_res[];
    DbF32 *rec0 = (DbF32 *)smem_res;
    DbF32 *rec1 = rec0 + S;
    float4 *part = (float4 *)(rec1 + S);  // [JS][tp_max][3] float4

    const int tid = threadIdx.x;
    const int lt = tid % tp_max, js = tid / tp_max;
    const bool worker = (js < JS) && (lt < TP);
    const int s = t0 + lt;                 // own dumbbell
    const int db = (int)(((int64_t)S * js) / JS), de = (int)(((int64_t)S * (js + 1)) / JS);
    const bool owner = worker && js == 0;  // runs the FP64 epilogue of dumbbell s

    // load the current records of all S dumbbells
    const DbF32 *gpack = (const DbF32 *)P.pack;
    for (int k = tid; k < S; k += NT) rec0[k] = gpack[k];
    const int64_t n0 = *P.step;
    // FP64 state of the owned dumbbell, kept in registers for the launch
    double x[6], v0[6], F[6], Racc[3] = {0, 0, 0};
    if (owner) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            x[k] = P.x[6 * (int64_t)s + k];
            v0[k] = P.v0[6 * (int64_t)s + k];
            F[k] = P.Fd[6 * (int64_t)s + k];
        }
        if (P.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) Racc[k] = P.Racc[3 * (int64_t)s + k];
        }
    }
    float r2min = 3.0e38f;
    cluster.sync();  // every CTA of the cluster is running and has its records

    for (int e = 0; e < 2 * K; ++e) {
        const DbF32 *cur = (e & 1) ? rec1 : rec0;
        DbF32 *nxt = (e & 1) ? rec0 : rec1;
        const int64_t n = n0 + (e >> 1);
        if (worker) {
            const DbF32 me = cur[s];
            float2 pa[3] = {make_float2(me.a.x, me.a.x), make_float2(me.a.z, me.a.z),
                            make_float2(me.b.x, me.b.x)};
            float2 pb[3] = {make_float2(me.a.y, me.a.y), make_float2(me.a.w, me.a.w),
                            make_float2(me.b.y, me.b.y)};
            float s_[6], c_[6];
            res_sweep<MOB>(cur, db, de, s, P.c2, P.c3, pa, pb, s_, c_, r2min);
            float4 *dst = part + (js * tp_max + lt) * 3;
            dst[0] = make_float4(s_[0], s_[1], s_[2], c_[0]);
            dst[1] = make_float4(c_[1], c_[2], s_[3], s_[4]);
            dst[2] = make_float4(s_[5], c_[3], c_[4], c_[5]);
        }
        __syncthreads();
        if (owner) {
            // combine the JS partials in js order (FP32 two-sum), then FP64
            float S_[6], C_[6];
            for (int q = 0; q < JS; ++q) {
                const float4 *src = part + (q * tp_max + lt) * 3;
                const float4 w0 = src[0], w1 = src[1], w2 = src[2];
                const float ps[6] = {w0.x, w0.y, w0.z, w1.z, w1.w, w2.x};
                const float pc[6] = {w0.w, w1.x, w1.y, w2.y, w2.z, w2.w};
                if (q == 0) {
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
            }
            double xq[6];
            double w[6] = {0, 0, 0, 0, 0, 0};   // additive noise of step n
            if (P.noise_sigma > 0.0) {
                float z[6];
                sphere_normals(P.noise_seed, n, 2 * (int64_t)s, z);
                sphere_normals(P.noise_seed, n, 2 * (int64_t)s + 1, z + 3);
#pragma unroll
                for (int k = 0; k < 6; ++k) w[k] = P.noise_sigma * (double)z[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const double u = (double)S_[k] + (double)C_[k];
                const double v = fma(F[k], P.inv6pimua, u);          // Eq. (3a) + pair sum
                if ((e & 1) == 0) {
                    v0[k] = v;
                    xq[k] = fma(P.dt, v, x[k]) + w[k];               // predictor
                } else {
                    x[k] = fma(0.5 * P.dt, v0[k] + v, x[k]) + w[k];  // corrector
                    xq[k] = x[k];
                }
            }
            if (!finite6(xq)) atomicOr(P.flags, FLAG_NONFINITE);
            const double2 sc = P.trig[(n + 1) & P.trig_mask];
            const double L = rest_length(P.ell, P.lam[s], sc.x, sc.y, P.sinphi[s], P.cosphi[s]);
            spring_force(xq, xq + 3, L, P.k0, F, F + 3);
            if (P.Fext) {
#pragma unroll
                for (int k = 0; k < 6; ++k) F[k] += P.Fext[6 * (int64_t)s + k];
            }
            // the new record goes to the next buffer of every CTA of the cluster
            DbF32 nr;
            {
                DbF32 tmp[1];
                store_rec(tmp, 0, xq, F, P.pack_args);
                nr = tmp[0];
            }
            for (int q = 0; q < G; ++q) {
                DbF32 *peer = cluster.map_shared_rank(nxt, q);
                peer[s] = nr;
            }
            if ((e & 1) == 1 && P.avg_m > 0) {
                const int64_t k_local = n + 1 - P.avg_n0;
                if (k_local > 0) {
                    const bool end = (k_local % P.avg_m) == 0;
                    const int64_t kidx = k_local / P.avg_m - 1;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const double Rt = 0.5 * (xq[k] + xq[3 + k]);
                        if (end) {
                            Racc[k] += 0.5 * Rt;
                            if (kidx < P.avg_maxk)
                                P.Rbar[kidx * 3 * (int64_t)S + 3 * (int64_t)s + k] =
                                    Racc[k] / (double)P.avg_m;
                            Racc[k] = 0.5 * Rt;
                        } else {
                            Racc[k] += Rt;
                        }
                    }
                }
            }
        }
        cluster.sync();  // next buffer complete in every CTA; current buffer free
    }

    if (MOB == 1 && worker && r2min < P.overlap_r2) atomicOr(P.flags, FLAG_OVERLAP);
    // write back: the owned state, and this CTA's range of the final records
    if (owner) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            P.x[6 * (int64_t)s + k] = x[k];
            P.v0[6 * (int64_t)s + k] = v0[k];
            P.Fd[6 * (int64_t)s + k] = F[k];
        }
        if (P.avg_m > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) P.Racc[3 * (int64_t)s + k] = Racc[k];
        }
    }
    const DbF32 *fin = ((2 * K) & 1) ? rec1 : rec0;
    DbF32 *gout = (DbF32 *)P.pack;
    for (int k = t0 + tid; k < t1; k += NT) gout[k] = fin[k];
    if (r == 0 && tid == 0) *P.step = n0 + K;
}

}  // namespace dbs
