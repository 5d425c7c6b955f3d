/*
 * FP64 CPU oracle for active spring-dumbbell suspensions
 * (Putz, Dunkel, Yeomans, "CUDA simulations of active dumbbell suspensions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library; both sides read only the seeded inputs.
 *
 * Every routine is the plain definition written out in double precision,
 * one loop per sum of the paper, with no blocking, fusion or reordering:
 *
 *   orc_rest_length       Eq. (4), Sec. II: L^s(t) = ell + lambda^s sin(omega t + phi^s)
 *   orc_spring_forces     Eq. (4), Sec. II: F = -dU/dX, U^s = k0/2 (d^s - L^s)^2
 *   orc_mobility_apply    Eq. (1a) at T = 0 with Eq. (3): v_a = sum_b H_ab F_b
 *                         (Eq. (3a) self term + Eq. (3b) pair term; Oseen drops
 *                         the a^2 line of Eq. (3b), Sec. II)
 *   orc_mobility_matrix   the paper's own "full tensor" method, Sec. IV: the
 *                         dense 3N x 3N matrix of Eq. (3)
 *   orc_velocities        spring forces at time t, plus an optional external
 *                         force, pushed through Eq. (3)
 *   orc_heun              Heun predictor-corrector, Sec. IV
 *   orc_heun_period_avg   Heun plus the stroke-averaged centres of Eqs. (6b),
 *                         (7b) over consecutive stroke periods (trapezoid rule
 *                         on the discrete trajectory)
 *   orc_sa_rates          stroke-averaged far-field EOM, Eqs. (9a)-(9e), Sec. III
 *   orc_sa_heun           Heun on (R, N) for Eqs. (9a)-(9b), N renormalised
 *                         after each step
 *   orc_pair_distance_change  |R^s - R^r|(k) - |R^s - R^r|(k0) for all pairs
 *   orc_philox4x32_10     the counter-based generator Philox4x32-10 (Salmon et
 *                         al., SC'11), written from its published definition
 *   orc_sphere_normals    standard normals of one sphere at one step (Box-Muller)
 *   orc_sd_rates          shape-driven dumbbells (Appendix A.2): constraint
 *                         forces by the iteration f_(n), then dR/dt, dN/dt
 *   orc_sd_heun           Heun on (R, N) of the shape-driven model, lengths
 *                         prescribed by Eq. (4)
 *   orc_heun_noise        Heun with the additive noise of a constant matrix
 *                         C = sqrt(2 kT / (6 pi mu a)) I, the dilute-limit
 *                         approximation of the closing remarks of Sec. IV
 *
 * Conventions: spheres are 0-based; dumbbell s owns spheres 2s and 2s+1
 * (the paper's 2s-1 and 2s).  Positions, forces and velocities are [N][3]
 * row-major doubles.  The orientation N^s points from sphere 2s to 2s+1.
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *  - Heun: predictor with F(x_n, t_n), corrector with F(x~, t_{n+1}),
 *    t_n = n dt computed from the step counter.
 *  - The RPY form is only defined for r > 2a; this oracle evaluates the
 *    printed formula for any r > 0 and the caller checks the geometry.
 *  - Unequal stroke amplitudes in the stroke-averaged law: (lambda/ell)^2 is
 *    read as lambda^s lambda^r / ell^2 (the stroke average that produces the
 *    amplitude factor multiplies one amplitude of each dumbbell).
 *  - K prefactor: the printed 15/64 of Eq. (9d) is used by default and is
 *    passed in as an argument; an exact stroke average of the shape-driven
 *    pair (a test of this oracle) confirms it.
 *  - Additive noise (the paper names the constant matrix C but not its value
 *    or the integrator): C = sqrt(2 kT / (6 pi mu a)) I, the square root of the
 *    self part of Eq. (3) times 2 kT; each Heun step adds C dW with
 *    dW = sqrt(dt) z, the same z in predictor and corrector.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OSEEN 0
#define ORC_RPY 1

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* Eq. (4): time-dependent rest length of dumbbell s. */
double orc_rest_length(double ell, double lambda, double omega, double phi, double t)
{
    return ell + lambda * sin(omega * t + phi);
}

/*
 * Eq. (4): F_(b i) = -d U / d X_(b i) with U^s = (k0/2) (d^s - L^s(t))^2 and
 * d^s = |X_{2s+1} - X_{2s}|.  With e = (X_{2s+1} - X_{2s}) / d^s:
 *   d d^s / d X_{2s+1} = +e,  d d^s / d X_{2s} = -e,
 * so F_{2s+1} = -k0 (d^s - L^s) e and F_{2s} = +k0 (d^s - L^s) e.
 */
void orc_spring_forces(int64_t S, const double *x, double ell, const double *lambda,
                       double omega, const double *phi, double k0, double t, double *F)
{
    for (int64_t s = 0; s < S; ++s) {
        const double *xa = x + 3 * (2 * s);
        const double *xb = x + 3 * (2 * s + 1);
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = xb[k] - xa[k];
        double d = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        double L = orc_rest_length(ell, lambda[s], omega, phi[s], t);
        double dUdd = k0 * (d - L);
        for (int k = 0; k < 3; ++k) {
            F[3 * (2 * s + 1) + k] = -dUdd * e[k] / d;
            F[3 * (2 * s) + k] = +dUdd * e[k] / d;
        }
    }
}

/*
 * Eq. (3b) for one pair: acc += H(x_a - x_b) F_b with
 *   H_ij = 1/(8 pi mu r) (delta_ij + r_i r_j / r^2)
 *        + 2 a^2 / (24 pi mu r^3) (delta_ij - 3 r_i r_j / r^2),
 * r_i = x_(a i) - x_(b i), r = |x_a - x_b|.  The Oseen approximation keeps
 * only the first line.
 */
static void add_pair_term(const double *xa, const double *xb, const double *Fb, double a,
                          double mu, int mobility, double *acc)
{
    double rv[3];
    for (int i = 0; i < 3; ++i) rv[i] = xa[i] - xb[i];
    double r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    double r = sqrt(r2);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double dij = (i == j) ? 1.0 : 0.0;
            double h = (dij + rv[i] * rv[j] / r2) / (8.0 * ORC_PI * mu * r);
            if (mobility == ORC_RPY)
                h += 2.0 * a * a / (24.0 * ORC_PI * mu * r * r2) * (dij - 3.0 * rv[i] * rv[j] / r2);
            acc[i] += h * Fb[j];
        }
    }
}

/*
 * Eq. (3) applied to a force vector:
 *   v_a = F_a / (6 pi mu a)  [Eq. (3a)]  +  sum_{b != a} H_ab F_b  [Eq. (3b)],
 * the sum over b in index order.
 */
void orc_mobility_apply(int64_t N, const double *x, const double *F, double a, double mu,
                        int mobility, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t al = 0; al < N; ++al) {
        double acc[3];
        for (int i = 0; i < 3; ++i) acc[i] = F[3 * al + i] / (6.0 * ORC_PI * mu * a);
        for (int64_t be = 0; be < N; ++be)
            if (be != al) add_pair_term(x + 3 * al, x + 3 * be, F + 3 * be, a, mu, mobility, acc);
        for (int i = 0; i < 3; ++i) v[3 * al + i] = acc[i];
    }
}

/* The interaction part alone: u_a = sum_{b != a} H_ab F_b (Eq. (3b) only). */
void orc_interaction(int64_t N, const double *x, const double *F, double a, double mu,
                     int mobility, double *u)
{
#pragma omp parallel for schedule(static)
    for (int64_t al = 0; al < N; ++al) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t be = 0; be < N; ++be)
            if (be != al) add_pair_term(x + 3 * al, x + 3 * be, F + 3 * be, a, mu, mobility, acc);
        for (int i = 0; i < 3; ++i) u[3 * al + i] = acc[i];
    }
}

/*
 * The paper's own method (Sec. IV): assemble the full 3N x 3N tensor of
 * Eq. (3).  H is row-major, H[(3a+i)*3N + (3b+j)] = H_(a i)(b j).
 */
void orc_mobility_matrix(int64_t N, const double *x, double a, double mu, int mobility, double *H)
{
    int64_t M = 3 * N;
    for (int64_t al = 0; al < N; ++al) {
        for (int64_t be = 0; be < N; ++be) {
            double rv[3] = {0, 0, 0}, r2 = 0, r = 0;
            if (be != al) {
                for (int i = 0; i < 3; ++i) rv[i] = x[3 * al + i] - x[3 * be + i];
                r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
                r = sqrt(r2);
            }
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) {
                    double dij = (i == j) ? 1.0 : 0.0;
                    double h;
                    if (be == al) {
                        h = dij / (6.0 * ORC_PI * mu * a);
                    } else {
                        h = (dij + rv[i] * rv[j] / r2) / (8.0 * ORC_PI * mu * r);
                        if (mobility == ORC_RPY)
                            h += 2.0 * a * a / (24.0 * ORC_PI * mu * r * r2) * (dij - 3.0 * rv[i] * rv[j] / r2);
                    }
                    H[(3 * al + i) * M + (3 * be + j)] = h;
                }
            }
        }
    }
}

/* Parameters of one suspension, as the oracle's entry points take them. */
typedef struct {
    int64_t S;          /* number of dumbbells; N = 2S spheres */
    double a;           /* sphere radius */
    double mu;          /* viscosity */
    double k0;          /* spring constant */
    double ell;         /* mean rest length */
    double omega;       /* stroke angular frequency, T = 2 pi / omega */
    double dt;          /* time step */
    int mobility;       /* ORC_OSEEN or ORC_RPY */
} orc_params;

/*
 * Velocities at (x, t): F = spring forces of Eq. (4) at time t plus the
 * optional constant external force Fext (NULL for none), then Eq. (3).
 */
void orc_velocities(const orc_params *p, const double *lambda, const double *phi,
                    const double *Fext, const double *x, double t, double *v)
{
    int64_t N = 2 * p->S;
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    orc_spring_forces(p->S, x, p->ell, lambda, p->omega, phi, p->k0, t, F);
    if (Fext)
        for (int64_t k = 0; k < 3 * N; ++k) F[k] += Fext[k];
    orc_mobility_apply(N, x, F, p->a, p->mu, p->mobility, v);
    free(F);
}

/*
 * Heun predictor-corrector (Sec. IV), nsteps steps from step counter n0:
 *   t_n = n dt,  v0 = v(x_n, t_n),  x~ = x_n + dt v0,
 *   v1 = v(x~, t_{n+1}),  x_{n+1} = x_n + dt/2 (v0 + v1).
 * x is updated in place.
 */
void orc_heun(const orc_params *p, const double *lambda, const double *phi, const double *Fext,
              double *x, int64_t n0, int64_t nsteps)
{
    int64_t N3 = 6 * p->S;
    double *v0 = (double *)malloc(sizeof(double) * N3);
    double *v1 = (double *)malloc(sizeof(double) * N3);
    double *xt = (double *)malloc(sizeof(double) * N3);
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        double t0 = (double)n * p->dt;
        double t1 = (double)(n + 1) * p->dt;
        orc_velocities(p, lambda, phi, Fext, x, t0, v0);
        for (int64_t k = 0; k < N3; ++k) xt[k] = x[k] + p->dt * v0[k];
        orc_velocities(p, lambda, phi, Fext, xt, t1, v1);
        for (int64_t k = 0; k < N3; ++k) x[k] = x[k] + 0.5 * p->dt * (v0[k] + v1[k]);
    }
    free(v0);
    free(v1);
    free(xt);
}

/*
 * Heun (as orc_heun, optional external force Fext) over nper consecutive
 * stroke periods of m steps each,
 * starting at step counter n0, recording for every period k the stroke
 * average of the geometric centre, Eqs. (6b) and (7b):
 *   Rbar^s_k = (1/T) int_{t_k}^{t_k + T} (X_{2s} + X_{2s+1})/2 du,  T = m dt,
 * with t_k = (n0 + k m) dt, evaluated by the trapezoid rule on the discrete
 * trajectory.  Rbar is [nper][S][3].
 */
void orc_heun_period_avg(const orc_params *p, const double *lambda, const double *phi,
                         const double *Fext, double *x, int64_t n0, int64_t m, int64_t nper,
                         double *Rbar)
{
    int64_t S = p->S;
    for (int64_t k = 0; k < nper; ++k) {
        double *Rk = Rbar + 3 * S * k;
        for (int64_t s = 0; s < 3 * S; ++s) Rk[s] = 0.0;
        for (int64_t n = 0; n <= m; ++n) {
            if (n > 0) orc_heun(p, lambda, phi, Fext, x, n0 + k * m + n - 1, 1);
            double w = (n == 0 || n == m) ? 0.5 : 1.0;
            for (int64_t s = 0; s < S; ++s)
                for (int i = 0; i < 3; ++i)
                    Rk[3 * s + i] += w * 0.5 * (x[3 * (2 * s) + i] + x[3 * (2 * s + 1) + i]);
        }
        for (int64_t s = 0; s < 3 * S; ++s) Rk[s] /= (double)m;
    }
}

/*
 * Stroke-averaged far-field equations of motion, Eqs. (9a)-(9e):
 *   dR^s/dt = sum_{r != s} J^{sr},
 *   dN^s/dt = -(I - N^s N^s^T) sum_{r != s} K^{sr},
 *   J^{sr}_i = a w sin(phi^s - phi^r) (9/64) (lambda/ell)^2 (ell/D)^4
 *              { N^s_i (2s + 4qr - 10 s r^2)
 *                + Dh_i (1 + 2q^2 - 5s^2 - 5r^2 - 20 q s r + 35 s^2 r^2) },
 *   K^{sr}_k = w sin(phi^s - phi^r) kpref (a/ell) (lambda/ell)^2 (ell/D)^5
 *              Dh_k (3s + 6rq + 6 s q^2 - 7 s^3 - 21 s r^2 - 42 q s^2 r + 63 s^3 r^2),
 * with D = R^s - R^r, Dh = D/|D|, s = Dh.N^s, r = Dh.N^r, q = N^s.N^r and the
 * printed kpref = 15/64.  (lambda/ell)^2 -> lambda^s lambda^r / ell^2.
 */
void orc_sa_rates(int64_t S, const double *R, const double *Nv, const double *phi,
                  const double *lambda, double a, double ell, double omega, double kpref,
                  double *Rdot, double *Ndot)
{
#pragma omp parallel for schedule(static)
    for (int64_t sg = 0; sg < S; ++sg) {
        double Jsum[3] = {0, 0, 0}, Ksum[3] = {0, 0, 0};
        const double *Ns = Nv + 3 * sg;
        for (int64_t rh = 0; rh < S; ++rh) {
            if (rh == sg) continue;
            const double *Nr = Nv + 3 * rh;
            double D[3];
            for (int i = 0; i < 3; ++i) D[i] = R[3 * sg + i] - R[3 * rh + i];
            double Dn = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            double Dh[3] = {D[0] / Dn, D[1] / Dn, D[2] / Dn};
            double s = Dh[0] * Ns[0] + Dh[1] * Ns[1] + Dh[2] * Ns[2];
            double r = Dh[0] * Nr[0] + Dh[1] * Nr[1] + Dh[2] * Nr[2];
            double q = Ns[0] * Nr[0] + Ns[1] * Nr[1] + Ns[2] * Nr[2];
            double sphi = sin(phi[sg] - phi[rh]);
            double lam2 = lambda[sg] * lambda[rh] / (ell * ell);
            double cJ = a * omega * sphi * (9.0 / 64.0) * lam2 * pow(ell / Dn, 4);
            double pN = 2 * s + 4 * q * r - 10 * s * r * r;
            double pD = 1 + 2 * q * q - 5 * s * s - 5 * r * r - 20 * q * s * r + 35 * s * s * r * r;
            double cK = omega * sphi * kpref * (a / ell) * lam2 * pow(ell / Dn, 5);
            double pK = 3 * s + 6 * r * q + 6 * s * q * q - 7 * s * s * s - 21 * s * r * r
                        - 42 * q * s * s * r + 63 * s * s * s * r * r;
            for (int i = 0; i < 3; ++i) {
                Jsum[i] += cJ * (Ns[i] * pN + Dh[i] * pD);
                Ksum[i] += cK * Dh[i] * pK;
            }
        }
        double NK = Ns[0] * Ksum[0] + Ns[1] * Ksum[1] + Ns[2] * Ksum[2];
        for (int i = 0; i < 3; ++i) {
            Rdot[3 * sg + i] = Jsum[i];
            Ndot[3 * sg + i] = -(Ksum[i] - Ns[i] * NK);
        }
    }
}

/*
 * Heun on the stroke-averaged state (R, N) of Eqs. (9a)-(9b), nsteps steps of
 * size dt; N is renormalised to unit length after every full step.
 */
void orc_sa_heun(int64_t S, double *R, double *Nv, const double *phi, const double *lambda,
                 double a, double ell, double omega, double kpref, double dt, int64_t nsteps)
{
    int64_t M = 3 * S;
    double *R0 = (double *)malloc(sizeof(double) * M), *N0 = (double *)malloc(sizeof(double) * M);
    double *R1 = (double *)malloc(sizeof(double) * M), *N1 = (double *)malloc(sizeof(double) * M);
    double *Rt = (double *)malloc(sizeof(double) * M), *Nt = (double *)malloc(sizeof(double) * M);
    for (int64_t n = 0; n < nsteps; ++n) {
        orc_sa_rates(S, R, Nv, phi, lambda, a, ell, omega, kpref, R0, N0);
        for (int64_t k = 0; k < M; ++k) {
            Rt[k] = R[k] + dt * R0[k];
            Nt[k] = Nv[k] + dt * N0[k];
        }
        orc_sa_rates(S, Rt, Nt, phi, lambda, a, ell, omega, kpref, R1, N1);
        for (int64_t k = 0; k < M; ++k) {
            R[k] = R[k] + 0.5 * dt * (R0[k] + R1[k]);
            Nv[k] = Nv[k] + 0.5 * dt * (N0[k] + N1[k]);
        }
        for (int64_t s = 0; s < S; ++s) {
            double *v = Nv + 3 * s;
            double nn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            for (int i = 0; i < 3; ++i) v[i] /= nn;
        }
    }
    free(R0); free(N0); free(R1); free(N1); free(Rt); free(Nt);
}

/*
 * Change of every pairwise centre distance between two snapshots:
 *   dD[s][r] = |R1^s - R1^r| - |R0^s - R0^r|   (dD is [S][S], zero diagonal).
 */
void orc_pair_distance_change(int64_t S, const double *R0, const double *R1, double *dD)
{
    for (int64_t s = 0; s < S; ++s) {
        for (int64_t r = 0; r < S; ++r) {
            double d0 = 0, d1 = 0;
            for (int i = 0; i < 3; ++i) {
                double e0 = R0[3 * s + i] - R0[3 * r + i];
                double e1 = R1[3 * s + i] - R1[3 * r + i];
                d0 += e0 * e0;
                d1 += e1 * e1;
            }
            dD[s * S + r] = (s == r) ? 0.0 : sqrt(d1) - sqrt(d0);
        }
    }
}

/*
 * Eq. (3) for a subset of target spheres: v[k] = H F restricted to rows[k]
 * (same sum, same order as orc_mobility_apply), for parity checks of large
 * systems on sampled targets.
 */
void orc_mobility_rows(int64_t N, const double *x, const double *F, double a, double mu,
                       int mobility, const int64_t *rows, int64_t nrows, double *v)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t al = rows[k];
        double acc[3];
        for (int i = 0; i < 3; ++i) acc[i] = F[3 * al + i] / (6.0 * ORC_PI * mu * a);
        for (int64_t be = 0; be < N; ++be)
            if (be != al) add_pair_term(x + 3 * al, x + 3 * be, F + 3 * be, a, mu, mobility, acc);
        for (int i = 0; i < 3; ++i) v[3 * k + i] = acc[i];
    }
}

/*
 * Philox4x32-10: ten rounds on the 128-bit counter c with the 64-bit key k,
 *   c -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * M0 = 0xD2511F53, M1 = 0xCD9E8D57, where hi/lo are the halves of the 64-bit
 * product; before every round but the first the key advances by the Weyl
 * constants W0 = 0x9E3779B9, W1 = 0xBB67AE85 (mod 2^32).
 */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Standard normals of sphere i at step n: Philox4x32-10 on the counter
 * (n mod 2^32, n / 2^32, i, 0) with key (seed mod 2^32, seed / 2^32), the four
 * words r mapped to u = (r + 1/2) 2^-32 in (0, 1), then Box-Muller:
 *   z0 = sqrt(-2 ln u0) cos(2 pi u1),  z1 = sqrt(-2 ln u0) sin(2 pi u1),
 *   z2 = sqrt(-2 ln u2) cos(2 pi u3).
 */
void orc_sphere_normals(uint64_t seed, int64_t n, int64_t i, double z[3])
{
    uint64_t un = (uint64_t)n;
    uint32_t ctr[4] = {(uint32_t)un, (uint32_t)(un >> 32), (uint32_t)i, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)r[k] + 0.5) / 4294967296.0;
    double ra = sqrt(-2.0 * log(u[0])), rb = sqrt(-2.0 * log(u[2]));
    z[0] = ra * cos(2.0 * ORC_PI * u[1]);
    z[1] = ra * sin(2.0 * ORC_PI * u[1]);
    z[2] = rb * cos(2.0 * ORC_PI * u[3]);
}

/*
 * Heun with additive noise, nsteps steps from step counter n0:
 *   w = sigma z_n (z_n: orc_sphere_normals per sphere), sigma = sqrt(2 kT dt / (6 pi mu a)),
 *   x~ = x_n + dt v(x_n, t_n) + w,
 *   x_{n+1} = x_n + dt/2 [v(x_n, t_n) + v(x~, t_{n+1})] + w.
 * With kT = 0 this is orc_heun.
 */
void orc_heun_noise(const orc_params *p, const double *lambda, const double *phi, const double *Fext,
                    double *x, int64_t n0, int64_t nsteps, double kT, uint64_t seed)
{
    int64_t N = 2 * p->S, N3 = 3 * N;
    double sigma = sqrt(2.0 * kT * p->dt / (6.0 * ORC_PI * p->mu * p->a));
    double *v0 = (double *)malloc(sizeof(double) * N3);
    double *v1 = (double *)malloc(sizeof(double) * N3);
    double *xt = (double *)malloc(sizeof(double) * N3);
    double *w = (double *)malloc(sizeof(double) * N3);
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        double t0 = (double)n * p->dt;
        double t1 = (double)(n + 1) * p->dt;
        for (int64_t i = 0; i < N; ++i) {
            double z[3];
            orc_sphere_normals(seed, n, i, z);
            for (int k = 0; k < 3; ++k) w[3 * i + k] = sigma * z[k];
        }
        orc_velocities(p, lambda, phi, Fext, x, t0, v0);
        for (int64_t k = 0; k < N3; ++k) xt[k] = x[k] + p->dt * v0[k] + w[k];
        orc_velocities(p, lambda, phi, Fext, xt, t1, v1);
        for (int64_t k = 0; k < N3; ++k) x[k] = x[k] + 0.5 * p->dt * (v0[k] + v1[k]) + w[k];
    }
    free(v0);
    free(v1);
    free(xt);
    free(w);
}

/*
 * Shape-driven dumbbells (Appendix A.2, "Three-dimensional case"): the length
 * of dumbbell s is prescribed, L^s(t) of Eq. (4), dL^s/dt = lambda^s omega
 * cos(omega t + phi^s); sphere 2s is X^{s1}, sphere 2s+1 is X^{s2}, and
 * N^s = (X^{s2} - X^{s1}) / |X^{s2} - X^{s1}|.  The internal forces
 * F^{s1} = f^s N^s, F^{s2} = -f^s N^s (force- and torque-free) keep the shape:
 *   dL^s/dt = N^s . (dX^{s2}/dt - dX^{s1}/dt).
 * The paper solves this by the iteration
 *   f^s_(n) = [dL^s/dt - sum_{r != s} b^{sr} f^r_(n-1)] / b^{ss},  f_(0) = 0,
 *   b^{sr} = N^s . [h^{(s2)(r1)} + h^{(s1)(r2)} - h^{(s2)(r2)} - h^{(s1)(r1)}] . N^r,
 * h^{(sb)(rc)} the mobility block of Eq. (3) between spheres (s,b) and (r,c)
 * (self block (6 pi mu a)^{-1} I); here every b^{sr} is taken with the exact
 * tensor, not its far-field expansion.  niter >= 1 iterations are made
 * (niter = 1: the isolated dumbbell f_(1) = dL/dt / b^{ss}; niter = 2: the
 * pair correction of the paper).  Then, with v = H F (Eq. (3)),
 *   dR^s/dt = (v^{s1} + v^{s2}) / 2,
 *   dN^s/dt = (I - N^s N^s^T) (v^{s2} - v^{s1}) / L^s.
 * x must satisfy |X^{s2} - X^{s1}| = L^s(t).  f_out (optional) receives f.
 */
void orc_sd_rates(const orc_params *p, const double *lambda, const double *phi, const double *x,
                  double t, int niter, double *Rdot, double *Ndot, double *f_out)
{
    int64_t S = p->S, N = 2 * S;
    double self = 1.0 / (6.0 * ORC_PI * p->mu * p->a);
    double *Nv = (double *)malloc(sizeof(double) * 3 * S);
    double *L = (double *)malloc(sizeof(double) * S);
    double *Ld = (double *)malloc(sizeof(double) * S);
    double *bss = (double *)malloc(sizeof(double) * S);
    double *f = (double *)calloc(S, sizeof(double));
    double *fn = (double *)malloc(sizeof(double) * S);
    for (int64_t s = 0; s < S; ++s) {
        const double *x1 = x + 3 * (2 * s), *x2 = x + 3 * (2 * s + 1);
        double e[3] = {x2[0] - x1[0], x2[1] - x1[1], x2[2] - x1[2]};
        double d = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        for (int k = 0; k < 3; ++k) Nv[3 * s + k] = e[k] / d;
        L[s] = orc_rest_length(p->ell, lambda[s], p->omega, phi[s], t);
        Ld[s] = lambda[s] * p->omega * cos(p->omega * t + phi[s]);
        /* b^{ss}: h^{(s2)(s1)} and h^{(s1)(s2)} are the pair tensor at +-L N, h^{(sb)(sb)} the self block */
        double u[3] = {0, 0, 0};
        add_pair_term(x2, x1, Nv + 3 * s, p->a, p->mu, p->mobility, u);
        double hc = u[0] * Nv[3 * s] + u[1] * Nv[3 * s + 1] + u[2] * Nv[3 * s + 2];
        bss[s] = 2.0 * hc - 2.0 * self;
    }
    for (int it = 0; it < niter; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < S; ++s) {
            const double *xs1 = x + 3 * (2 * s), *xs2 = x + 3 * (2 * s + 1);
            double sum = 0.0;
            for (int64_t r = 0; r < S; ++r) {
                if (r == s) continue;
                const double *xr1 = x + 3 * (2 * r), *xr2 = x + 3 * (2 * r + 1);
                double u[3] = {0, 0, 0}, w[3] = {0, 0, 0};
                /* [h^{(s2)(r1)} - h^{(s2)(r2)}] N^r and [h^{(s1)(r2)} - h^{(s1)(r1)}] N^r */
                add_pair_term(xs2, xr1, Nv + 3 * r, p->a, p->mu, p->mobility, u);
                add_pair_term(xs1, xr2, Nv + 3 * r, p->a, p->mu, p->mobility, u);
                add_pair_term(xs2, xr2, Nv + 3 * r, p->a, p->mu, p->mobility, w);
                add_pair_term(xs1, xr1, Nv + 3 * r, p->a, p->mu, p->mobility, w);
                double bsr = 0.0;
                for (int k = 0; k < 3; ++k) bsr += Nv[3 * s + k] * (u[k] - w[k]);
                sum += bsr * f[r];
            }
            fn[s] = (Ld[s] - sum) / bss[s];
        }
        for (int64_t s = 0; s < S; ++s) f[s] = fn[s];
    }
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    double *v = (double *)malloc(sizeof(double) * 3 * N);
    for (int64_t s = 0; s < S; ++s)
        for (int k = 0; k < 3; ++k) {
            F[3 * (2 * s) + k] = f[s] * Nv[3 * s + k];
            F[3 * (2 * s + 1) + k] = -f[s] * Nv[3 * s + k];
        }
    orc_mobility_apply(N, x, F, p->a, p->mu, p->mobility, v);
    for (int64_t s = 0; s < S; ++s) {
        const double *v1 = v + 3 * (2 * s), *v2 = v + 3 * (2 * s + 1);
        double w[3], nw = 0.0;
        for (int k = 0; k < 3; ++k) {
            Rdot[3 * s + k] = 0.5 * (v1[k] + v2[k]);
            w[k] = (v2[k] - v1[k]) / L[s];
            nw += Nv[3 * s + k] * w[k];
        }
        for (int k = 0; k < 3; ++k) Ndot[3 * s + k] = w[k] - Nv[3 * s + k] * nw;
        if (f_out) f_out[s] = f[s];
    }
    free(Nv); free(L); free(Ld); free(bss); free(f); free(fn); free(F); free(v);
}

/*
 * Heun on (R, N) of the shape-driven model, nsteps steps from step n0, x
 * (spheres) updated in place:
 *   R = (X^{s1} + X^{s2})/2, N = (X^{s2} - X^{s1})/|.|,
 *   (R0', N0') = orc_sd_rates(x_n, t_n),  R~ = R + dt R0',  N~ = unit(N + dt N0'),
 *   x~ = R~ -/+ N~ L(t_{n+1})/2,  (R1', N1') = orc_sd_rates(x~, t_{n+1}),
 *   R_{n+1} = R + dt/2 (R0' + R1'),  N_{n+1} = unit(N + dt/2 (N0' + N1')),
 *   x_{n+1} = R_{n+1} -/+ N_{n+1} L(t_{n+1})/2.
 */
static void sd_place(int64_t S, const double *R, const double *Nv, const orc_params *p,
                     const double *lambda, const double *phi, double t, double *x)
{
    for (int64_t s = 0; s < S; ++s) {
        double L = orc_rest_length(p->ell, lambda[s], p->omega, phi[s], t);
        for (int k = 0; k < 3; ++k) {
            x[3 * (2 * s) + k] = R[3 * s + k] - 0.5 * L * Nv[3 * s + k];
            x[3 * (2 * s + 1) + k] = R[3 * s + k] + 0.5 * L * Nv[3 * s + k];
        }
    }
}

static void unit3(double *v)
{
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) v[k] /= n;
}

void orc_sd_heun(const orc_params *p, const double *lambda, const double *phi, double *x, int64_t n0,
                 int64_t nsteps, int niter)
{
    int64_t S = p->S;
    double *R = (double *)malloc(sizeof(double) * 3 * S), *Nv = (double *)malloc(sizeof(double) * 3 * S);
    double *R0 = (double *)malloc(sizeof(double) * 3 * S), *N0 = (double *)malloc(sizeof(double) * 3 * S);
    double *R1 = (double *)malloc(sizeof(double) * 3 * S), *N1 = (double *)malloc(sizeof(double) * 3 * S);
    double *Rt = (double *)malloc(sizeof(double) * 3 * S), *Nt = (double *)malloc(sizeof(double) * 3 * S);
    double *xt = (double *)malloc(sizeof(double) * 6 * S);
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        double t0 = (double)n * p->dt, t1 = (double)(n + 1) * p->dt;
        for (int64_t s = 0; s < S; ++s) {
            const double *x1 = x + 3 * (2 * s), *x2 = x + 3 * (2 * s + 1);
            for (int k = 0; k < 3; ++k) {
                R[3 * s + k] = 0.5 * (x1[k] + x2[k]);
                Nv[3 * s + k] = x2[k] - x1[k];
            }
            unit3(Nv + 3 * s);
        }
        orc_sd_rates(p, lambda, phi, x, t0, niter, R0, N0, NULL);
        for (int64_t s = 0; s < S; ++s) {
            for (int k = 0; k < 3; ++k) {
                Rt[3 * s + k] = R[3 * s + k] + p->dt * R0[3 * s + k];
                Nt[3 * s + k] = Nv[3 * s + k] + p->dt * N0[3 * s + k];
            }
            unit3(Nt + 3 * s);
        }
        sd_place(S, Rt, Nt, p, lambda, phi, t1, xt);
        orc_sd_rates(p, lambda, phi, xt, t1, niter, R1, N1, NULL);
        for (int64_t s = 0; s < S; ++s) {
            for (int k = 0; k < 3; ++k) {
                Rt[3 * s + k] = R[3 * s + k] + 0.5 * p->dt * (R0[3 * s + k] + R1[3 * s + k]);
                Nt[3 * s + k] = Nv[3 * s + k] + 0.5 * p->dt * (N0[3 * s + k] + N1[3 * s + k]);
            }
            unit3(Nt + 3 * s);
        }
        sd_place(S, Rt, Nt, p, lambda, phi, t1, x);
    }
    free(R); free(Nv); free(R0); free(N0); free(R1); free(N1); free(Rt); free(Nt); free(xt);
}
