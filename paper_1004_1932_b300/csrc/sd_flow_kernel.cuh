// Cooperative form of the shape-driven dynamics (Appendix A.2): K Heun steps of
// one FP32C suspension in one launch over up to one CTA per SM, one exchange per
// pair sum and no grid-wide barrier, on the machinery of flow_kernel (tagged
// 16-byte record words, bounded polls, FP32 pair sums with two-sum folding).
//
// A Heun step of the shape-driven model is 2M pair sums, M constraint
// iterations at each of the two evaluation points.  CTA g owns the T dumbbells
// [gT, gT + T) and, after every pair sum u_i = sum_{j != i} H(r_ij) F_j (the
// interaction part of Eq. (3), the partner sphere included), warp 0 runs one
// of two epilogues for its dumbbells (lane d: dumbbell d, all three axes):
//  * a constraint iteration (not the last of the point):
//      f <- [dL/dt - (N . (u2 - u1) - 2 f h_c)] / b^ss,
//    the records keep their positions and take the new G = +/- f N / (8 pi mu);
//  * the last iteration of the point: v = u + F / (6 pi mu a) (Eq. (3a)),
//    dR/dt = (v1 + v2)/2, dN/dt = (I - N N^T)(v2 - v1)/L, the Heun stage of
//    Sec. IV on (R, N) with N renormalised, the spheres placed at
//    R -/+ N L(t_{n+1})/2, and the first iterate of the next point,
//    h_c = N . H(L N) . N, b^ss = 2 h_c - 2/(6 pi mu a), f = (dL/dt) / b^ss.
//
// Precision: the records and the rates are FP32 (FP32 pair sums); within a
// launch the state (R - c and N at the start of the step) is carried as
// double-single pairs, advanced by the corrector's increments and renormalised
// (FP32 seed and one Newton step in double-single) in the next poll's gap; the
// FP64 positions are read at the start of a launch and written at its end,
// placed at L(t) in FP64.  The stroke averages of the centre (trapezoid rule)
// accumulate in FP64 in the same gap.
#pragma once
#include "flow_kernel.cuh"

namespace dbs {

template <int T>
struct SdOwn {
    float Rh[3][T], Rl[3][T];    // centre - c at the start of the step (double-single)
    float Nh[3][T], Nl[3][T];    // unit axis at the start of the step (double-single)
    float Np[3][T];              // axis at the current evaluation point
    float Lp[T], Ldp[T];         // rest length L and dL/dt at the point
    float hc[T], bss[T], f[T];   // h_c, b^ss and the current iterate f at the point
    float r0[6][T];              // predictor rates dR/dt, dN/dt
    float lam[T], sph[T], cph[T];
    float2 Q[3][T];              // stroke-average running sums of R - c, double-single
};

// the first iterate of a point with axis N and rest length L: h_c, b^ss, f_(1)
__device__ __forceinline__ void sd_point(int mob, float L, float Ld, float inv8, float inv6, float a3inv6,
                                         float &hc, float &bss, float &f)
{
    hc = 2.f * inv8 / L;
    if (mob == 1) hc -= a3inv6 / (L * L * L);
    bss = 2.f * hc - 2.f * inv6;
    f = Ld / bss;
}

template <int MOB, int T>
__global__ void __launch_bounds__(FLOW_NT, 1) sd_flow_kernel(const EvalArgs A, const FlowArgs P, const int M)
{
    constexpr int NT = FLOW_NT;
    constexpr int PS = NT / T;                   // slices (threads) per target dumbbell
    constexpr int LW = PS < 32 ? PS : 32;        // lanes of a target within a warp
    constexpr int WPT = PS > 32 ? PS / 32 : 1;   // warps per target
    constexpr bool KEEP = T <= 4;                // as in flow_kernel
    constexpr int POLL = KEEP ? 6 : 12;
    static_assert(LW >= 8, "the transposing fold needs 8 lanes per target");
    extern __shared__ float4 flow_smem[];        // all S records (Spad x DbF32)
    __shared__ SdOwn<T> own;
    __shared__ float2 red[WPT == 1 ? T : T * WPT][6];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    const int S = (int)A.S;
    const int Spad = P.G * T;
    const int st0 = g * T;
    const int nown = min(T, S - st0);
    DbF32 *tile = (DbF32 *)flow_smem;
    if (gridDim.x != (unsigned)P.G || blockDim.x != (unsigned)NT || M < 1) {   // not the shape the host made
        if (tid == 0) atomicOr(A.flags, FLAG_LAUNCH);
        return;
    }
    const float k8 = A.inv8pimu_f, inv6 = (float)A.inv6pimua;
    const float a3inv6 = (float)(A.a * A.a * A.a * A.inv6pimua);
    const float ellf = (float)A.ell, omf = (float)A.omega, dtf = (float)A.dt, hdtf = (float)(0.5 * A.dt);
    const double cen[3] = {A.cx, A.cy, A.cz};
    const bool ep = warp == 0 && lane < nown;    // epilogue lane: dumbbell lane of warp 0

    // ---- the owned state from the FP64 positions, the first point, evaluation 0
    if (ep) {
        const int d = lane, s = st0 + d;
        const double *x = A.x + 6 * (int64_t)s;
        double e[3], dd = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            e[k] = x[3 + k] - x[k];
            dd = fma(e[k], e[k], dd);
        }
        const double inv = 1.0 / sqrt(dd);
        const float lam = (float)A.lam[s], sp = (float)A.sinphi[s], cp = (float)A.cosphi[s];
        own.lam[d] = lam;
        own.sph[d] = sp;
        own.cph[d] = cp;
        const float4 tr = A.trig_df[P.n0 & A.trig_mask];   // (sin, cos)(w t_n0), hi parts .x, .z
        const float L = ellf + lam * fmaf(tr.x, cp, tr.z * sp);
        const float Ld = lam * omf * fmaf(tr.z, cp, -tr.x * sp);
        float hc, bss, f;
        sd_point(MOB, L, Ld, k8, inv6, a3inv6, hc, bss, f);
        own.Lp[d] = L;
        own.Ldp[d] = Ld;
        own.hc[d] = hc;
        own.bss[d] = bss;
        own.f[d] = f;
        const unsigned bit = flow_bit(P.base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ds Rk = ds_of(0.5 * (x[k] + x[3 + k]) - cen[k]);
            const ds Nk = ds_of(e[k] * inv);
            own.Rh[k][d] = Rk.h;
            own.Rl[k][d] = Rk.l;
            own.Nh[k][d] = Nk.h;
            own.Nl[k][d] = Nk.l;
            own.Np[k][d] = Nk.h;
            if (A.avg_m > 0) {
                // the FP64 sum carried between launches, sum of w_i R_i with weights
                // summing to 1/2 + (k mod m) after sample k, as sum of w_i (R_i - c)
                const int64_t kl = P.n0 - A.avg_n0;
                const double sw = 0.5 + (double)(kl > 0 ? kl % A.avg_m : 0);
                const ds q = ds_of(A.Racc[3 * (int64_t)s + k] - cen[k] * sw);
                own.Q[k][d] = make_float2(q.h, q.l);
            }
            const float pa = (float)(x[k] - cen[k]), pb = (float)(x[3 + k] - cen[k]);
            const float ga = g_clear(f * Nk.h * k8), gb = g_clear(-f * Nk.h * k8);
            put_axis(tile + s, k, pa, ga, pb, gb);
            st_word(P.rec + (size_t)s * 3 + k, pa, ga, pb, gb, bit);
        }
    }
    __syncthreads();

    const float2 c2 = make_float2(A.c2, A.c2), c3 = make_float2(A.c3, A.c3);
    const int nwords = 3 * S;
    const int own_w0 = 3 * st0, own_w1 = 3 * (st0 + nown);
    const int t_me = tid / PS, sl = tid - t_me * PS;   // sweep: target and slice
    const int s_me = st0 + t_me;
    const bool act = t_me < nown;
    ulonglong2 kva[KEEP ? POLL : 1], kvb[KEEP ? POLL : 1];

    // The corrector's increments dt/2 (rate0 + rate) of R and N (lane d of warp
    // 0, all three axes) and its step n; the next poll's gap adds them to the
    // double-single state, renormalises N and accumulates the stroke average.
    float incR[3] = {0.f, 0.f, 0.f}, incN[3] = {0.f, 0.f, 0.f};
    int64_t hn = -1;
    // the stroke average's sample index k = n + 1 - avg_n0 of the next update and
    // its residue mod avg_m, advanced by one per update (consecutive steps)
    int64_t k_next = P.n0 + 1 - A.avg_n0;
    int64_t k_mod = A.avg_m > 0 ? ((k_next % A.avg_m) + A.avg_m) % A.avg_m : 0;
    auto state_update = [&]() {
        if (hn < 0) return;
        const int d = lane;
        ds N1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ds R1 = ds_add({own.Rh[k][d], own.Rl[k][d]}, {incR[k], 0.f});
            own.Rh[k][d] = R1.h;
            own.Rl[k][d] = R1.l;
            N1[k] = ds_add({own.Nh[k][d], own.Nl[k][d]}, {incN[k], 0.f});
        }
        // 1/|N1|: FP32 seed, one Newton step y + y (1 - q y^2) / 2 in double-single
        const ds q = ds_add(ds_add(ds_mul(N1[0], N1[0]), ds_mul(N1[1], N1[1])), ds_mul(N1[2], N1[2]));
        const float y0 = rsqrtf(q.h);
        const ds qy2 = ds_mul(q, ds_mul({y0, 0.f}, {y0, 0.f}));
        const ds y = ds_fast(y0, 0.5f * y0 * ((1.f - qy2.h) - qy2.l));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ds Nk = ds_mul(N1[k], y);
            own.Nh[k][d] = Nk.h;
            own.Nl[k][d] = Nk.l;
        }
        const int64_t k_local = k_next;   // hn + 1 - avg_n0
        if (A.avg_m > 0 && k_local > 0) {   // trapezoid rule, as the spring model's, in double-single
            const bool end = k_mod == 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ds Rk = {own.Rh[k][d], own.Rl[k][d]};
                ds q = {own.Q[k][d].x, own.Q[k][d].y};
                if (end) {
                    const ds half = {0.5f * Rk.h, 0.5f * Rk.l};
                    q = ds_add(q, half);
                    const int64_t kidx = k_local / A.avg_m - 1;
                    if (kidx < A.avg_maxk)
                        A.Rbar[kidx * 3 * A.S + 3 * (int64_t)(st0 + d) + k] = cen[k] + ds_to_double(q) / (double)A.avg_m;
                    q = half;
                } else {
                    q = ds_add(q, Rk);
                }
                own.Q[k][d] = make_float2(q.h, q.l);
            }
        }
        ++k_next;
        if (++k_mod == A.avg_m) k_mod = 0;
        hn = -1;
    };
    auto gap = [&]() {
        if (ep) state_update();
    };

    const int nev = 2 * M * P.K;
    bool dead = false;
    for (int ev = 0; ev < nev && !dead; ++ev) {
        const unsigned bit = flow_bit(P.base + (unsigned)ev);
        const int par = ev & 1;
        const int e = ev % (2 * M);
        const bool corr = e >= M;                  // second point of the step
        const bool last = (e % M) == M - 1;        // last iteration at this point
        const int64_t n = P.n0 + ev / (2 * M);
        const ulonglong2 *R = P.rec + (size_t)par * Spad * 3;
        // (sin, cos)(w t_{n+1}) for the last iteration's placement, loaded while the
        // records are on their way
        float4 tr1 = make_float4(0.f, 0.f, 1.f, 0.f);
        if (ep && last) tr1 = A.trig_df[(n + 1) & A.trig_mask];

        // 1. poll the records this CTA does not own (as flow_kernel)
        bool ok = true;
        auto has = [&](const ulonglong2 &v) { return word_has(v, bit); };
        for (int b0 = 0; b0 < nwords && ok; b0 += POLL * NT) {
            unsigned pend = 0;
#pragma unroll
            for (int j = 0; j < POLL; ++j) {
                const int idx = b0 + j * NT + tid;
                if (idx < nwords && (idx < own_w0 || idx >= own_w1)) pend |= 1u << j;
            }
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
        gap();
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
            float r2min = 3.0e38f;
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
                                 r2min, false, self);
            }
            if (MOB == 1 && r2min < A.overlap_r2) atomicOr(A.flags, FLAG_OVERLAP);
        }

        // 3. fold the slices of each target (FP32 two-sum, lanes by transposition,
        // then the target's warps in warp order in the epilogue)
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
            const int sb = lane_fold<LW, true, 1>(fs, fc, lane);
            if ((lane & (LW / 8 - 1)) == 0 && sb < 6)
                red[WPT == 1 ? t_me : t_me * WPT + warp % WPT][sb] = make_float2(fs[0], fc[0]);
        }
        __syncthreads();

        // 4. epilogue, lane d of warp 0: dumbbell d, all three axes
        if (ep) {
            const int d = lane, s = st0 + d;
            float u1[3], u2[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float2 ua = red[d * WPT][k], ub = red[d * WPT][3 + k];
#pragma unroll
                for (int w = 1; w < WPT; ++w) {
                    ts_merge(ua.x, ua.y, red[d * WPT + w][k].x, red[d * WPT + w][k].y);
                    ts_merge(ub.x, ub.y, red[d * WPT + w][3 + k].x, red[d * WPT + w][3 + k].y);
                }
                u1[k] = ua.x + ua.y;
                u2[k] = ub.x + ub.y;
            }
            const float N[3] = {own.Np[0][d], own.Np[1][d], own.Np[2][d]};
            float pa[3], pb[3], Nn[3], fnew;
            if (!last) {
                // a constraint iteration: sum_{r != s} b^sr f^r = N . (u2 - u1) - 2 f h_c
                const float nu = fmaf(N[0], u2[0] - u1[0], fmaf(N[1], u2[1] - u1[1], N[2] * (u2[2] - u1[2])));
                fnew = (own.Ldp[d] - (nu - 2.f * own.f[d] * own.hc[d])) / own.bss[d];
                own.f[d] = fnew;
                const float4 a4 = tile[s].a, b4 = tile[s].b;   // positions unchanged
                pa[0] = a4.x; pb[0] = a4.y; pa[1] = a4.z; pb[1] = a4.w; pa[2] = b4.x; pb[2] = b4.y;
#pragma unroll
                for (int k = 0; k < 3; ++k) Nn[k] = N[k];
            } else {
                // v = u + F/(6 pi mu a), F = +/- f N; rates; Heun stage; placement at t_{n+1}
                const float fN = own.f[d], L = own.Lp[d];
                float Rd[3], w[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float v1 = fmaf(fN * N[k], inv6, u1[k]);
                    const float v2 = fmaf(-fN * N[k], inv6, u2[k]);
                    Rd[k] = 0.5f * (v1 + v2);
                    w[k] = (v2 - v1) / L;
                }
                const float nw = fmaf(N[0], w[0], fmaf(N[1], w[1], N[2] * w[2]));
                float Rn[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float Nd = w[k] - N[k] * nw;
                    if (!corr) {
                        own.r0[k][d] = Rd[k];
                        own.r0[3 + k][d] = Nd;
                        Rn[k] = own.Rh[k][d] + (own.Rl[k][d] + dtf * Rd[k]);
                        Nn[k] = own.Nh[k][d] + (own.Nl[k][d] + dtf * Nd);
                    } else {
                        incR[k] = hdtf * (own.r0[k][d] + Rd[k]);
                        incN[k] = hdtf * (own.r0[3 + k][d] + Nd);
                        Rn[k] = own.Rh[k][d] + (own.Rl[k][d] + incR[k]);
                        Nn[k] = own.Nh[k][d] + (own.Nl[k][d] + incN[k]);
                    }
                }
                if (corr) hn = n;   // the double-single update of step n runs in the next poll
                const float inv = rsqrtf(fmaf(Nn[0], Nn[0], fmaf(Nn[1], Nn[1], Nn[2] * Nn[2])));
                const float4 tr = tr1;
                const float lam = own.lam[d], sp = own.sph[d], cp = own.cph[d];
                const float L1 = ellf + lam * fmaf(tr.x, cp, tr.z * sp);
                const float Ld1 = lam * omf * fmaf(tr.z, cp, -tr.x * sp);
                float hc, bss;
                sd_point(MOB, L1, Ld1, k8, inv6, a3inv6, hc, bss, fnew);
                own.Lp[d] = L1;
                own.Ldp[d] = Ld1;
                own.hc[d] = hc;
                own.bss[d] = bss;
                own.f[d] = fnew;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Nn[k] *= inv;
                    own.Np[k][d] = Nn[k];
                    pa[k] = fmaf(-0.5f * L1, Nn[k], Rn[k]);
                    pb[k] = fmaf(0.5f * L1, Nn[k], Rn[k]);
                }
                if (!(finite_f(pa[0]) && finite_f(pa[1]) && finite_f(pa[2]) && finite_f(pb[0]) &&
                      finite_f(pb[1]) && finite_f(pb[2]) && finite_f(fnew)))
                    atomicOr(A.flags, FLAG_NONFINITE);
            }
            // the records of the next pair sum: G = +/- f N / (8 pi mu)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float ga = g_clear(fnew * Nn[k] * k8), gb = g_clear(-fnew * Nn[k] * k8);
                put_axis(tile + s, k, pa[k], ga, pb[k], gb);
                if (ev + 1 < nev)
                    st_word(P.rec + ((size_t)(par ^ 1) * Spad + s) * 3 + k, pa[k], ga, pb[k], gb,
                            flow_bit(P.base + (unsigned)ev + 1u));
            }
        }
        // The other warps wait here for warp 0's epilogue: started at once, their
        // polls ran ahead of this CTA's own publish, and every pair sum took longer
        // (S = 128 / 512, 2 iterations: 12.7 / 17.2 us per Heun step without this
        // barrier, 7.6 / 14.1 with it; with the clock prefetched above as well 7.0 /
        // 10.7, measured).  The next poll writes only records this CTA does not own.
        __syncthreads();
    }

    // ---- the FP64 state: R and N from their pairs (N renormalised in FP64), the
    // spheres placed at R -/+ N L(t)/2 at the launch's last time ---------------------
    gap();
    __syncthreads();
    if (ep) {
        const int d = lane, s = st0 + d;
        const int64_t nend = P.n0 + P.K;
        double R[3], N[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R[k] = ((double)own.Rh[k][d] + (double)own.Rl[k][d]) + cen[k];
            N[k] = (double)own.Nh[k][d] + (double)own.Nl[k][d];
        }
        const double inv = 1.0 / sqrt(fma(N[0], N[0], fma(N[1], N[1], N[2] * N[2])));
        const double2 sc = A.trig[nend & A.trig_mask];
        const double L = rest_length(A.ell, A.lam[s], sc.x, sc.y, A.sinphi[s], A.cosphi[s]);
        double *x = A.x + 6 * (int64_t)s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = fma(-0.5 * L, N[k] * inv, R[k]);
            x[3 + k] = fma(0.5 * L, N[k] * inv, R[k]);
            if (A.avg_m > 0) {
                const int64_t kl = P.n0 + P.K - A.avg_n0;   // the last sample taken
                A.Racc[3 * (int64_t)s + k] =
                    cen[k] * (0.5 + (double)(kl % A.avg_m)) + ds_to_double({own.Q[k][d].x, own.Q[k][d].y});
            }
        }
    }
    if (g == 0 && tid == 0) *A.step = P.n0 + P.K;
}

}  // namespace dbs
