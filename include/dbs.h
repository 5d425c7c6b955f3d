/*
 * dbs.h -- C-ABI of the B300-native active-dumbbell suspension library (libdbs.so).
 *
 * The library advances S actively driven spring dumbbells (N = 2S spheres)
 * in unbounded Stokes flow, the microscopic model of Putz, Dunkel & Yeomans,
 * "CUDA simulations of active dumbbell suspensions":
 *
 *   dX_a/dt = sum_b H_ab F_b                       Eq. (1a) at zero temperature
 *   H_aa = I / (6 pi mu a)                         Eq. (3a)
 *   H_ab = (I + r r^T/r^2) / (8 pi mu r)
 *        + 2 a^2 (I - 3 r r^T/r^2) / (24 pi mu r^3)   Eq. (3b) (RPY-Mazur);
 *                                                  the Oseen form drops the a^2 line
 *   F = -dU/dX,  U = sum_s k0/2 (d^s - L^s(t))^2,
 *   L^s(t) = ell + lambda^s sin(omega t + phi^s)   Eq. (4)
 *   Heun predictor-corrector in time               Sec. IV
 *
 * and the stroke-averaged far-field model of Eqs. (9a)-(9e) (Sec. III.B).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Spheres are 0-based.  Dumbbell s owns spheres 2s and 2s+1 (the paper's
 *    2s-1 and 2s); its orientation points from sphere 2s to sphere 2s+1.
 *  - Host arrays are row-major doubles, sphere-major [N][3] (positions,
 *    forces, velocities) or [S] (amplitudes, phases).  They are owned by the
 *    caller, read or written during the call only, and never retained.
 *  - Arguments named *_dev are device pointers on the handle's device; the
 *    library reads or writes them in stream order on the handle's stream and
 *    returns without synchronising.
 *  - Handles are opaque and own their device memory (cudaMalloc at create,
 *    cudaFree at destroy).  A handle must not be used from two host threads
 *    at once.
 *  - Every call returns DBS_OK (0) or a negative DBS_E_* status.  Errors found
 *    while computing (device faults, CUDA failures) are sticky: once a handle
 *    has failed, every later call on it returns the same status until it is
 *    destroyed; dbs_last_error() describes it.  Refused arguments (DBS_E_ARG)
 *    and calls not valid in the handle's mode (DBS_E_STATE) leave it usable.
 *  - Time is t_n = n dt, computed in double precision from the step counter n.
 *
 * Arithmetic: FP32C evaluates the pair sum of Eq. (3b) in single precision
 * with per-target compensated (two-sum) accumulation across j-tiles, and
 * keeps positions, the clock and the Heun update in double precision.  The
 * spring force and the self term are double precision on the grid and
 * cluster paths; the cooperative path forms them in single precision from a
 * double-single d^2 - L^2 (the stretch d - L keeps single-precision relative
 * accuracy).  FP64 does everything in double precision (on the cooperative
 * path the pair sum reads positions and G with their lowest bit cleared).
 */
#ifndef DBS_H
#define DBS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DBS_API __attribute__((visibility("default")))
#else
#define DBS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DBS_OK 0
#define DBS_E_ARG (-1)       /* invalid argument (sizes, non-finite values, NULL) */
#define DBS_E_NOMEM (-2)     /* device allocation failed */
#define DBS_E_CUDA (-3)      /* a CUDA runtime call failed */
#define DBS_E_OVERLAP (-4)   /* two distinct spheres coincide, or r < 2a under RPY */
#define DBS_E_NONFINITE (-5) /* a velocity or position became NaN or Inf */
#define DBS_E_TIMEOUT (-6)   /* a bounded device-side wait ran out */
#define DBS_E_STATE (-7)     /* call not valid in the handle's current state */

/* ---- enums --------------------------------------------------------------- */
#define DBS_OSEEN 0 /* Eq. (3b) without its a^2 line (Sec. II) */
#define DBS_RPY 1   /* full Eq. (3b), Rotne-Prager-Yamakawa-Mazur */

#define DBS_FP32C 0 /* FP32 pair math, compensated accumulation, FP64 state */
#define DBS_FP64 1  /* FP64 everywhere */

/* Physical and numerical parameters of one suspension (Secs. II and IV). */
typedef struct {
    int64_t S;        /* number of dumbbells, >= 1; N = 2S spheres */
    double a;         /* sphere radius, > 0 */
    double mu;        /* viscosity, > 0 */
    double k0;        /* spring constant, >= 0 */
    double ell;       /* mean rest length, > 2a + max|lambda| (Sec. II) */
    double omega;     /* stroke angular frequency, T = 2 pi / omega, > 0 */
    double dt;        /* time step, > 0 */
    int32_t mobility; /* DBS_OSEEN or DBS_RPY */
    int32_t precision;/* DBS_FP32C or DBS_FP64 */
    void *stream;     /* cudaStream_t for all device work, NULL = a stream the handle creates */
    int32_t device;   /* CUDA device ordinal, -1 = the calling thread's current device */
    int32_t flags;    /* reserved, must be 0 */
} dbs_params;

typedef struct dbs_suspension dbs_suspension;

/*
 * Create a suspension with initial sphere positions x0 [2S][3] (host).
 * Stroke amplitudes start at 0 and phases at 0 (passive dumbbells); call
 * dbs_set_stroke to make them active.  The step counter starts at n = 0.
 * Errors: DBS_E_ARG (bad parameters, non-finite x0), DBS_E_NOMEM, DBS_E_CUDA.
 * On failure *out is NULL.
 */
DBS_API int dbs_create_suspension(const dbs_params *p, const double *x0, dbs_suspension **out);

/* Release the handle and its device memory (waits for its stream).  NULL is a no-op. */
DBS_API int dbs_destroy(dbs_suspension *h);

/*
 * Stroke amplitudes lambda [S] and phases phi [S] (host) of Eq. (4).
 * Requires ell > 2a + |lambda^s| for every s (Sec. II); else DBS_E_ARG.
 */
DBS_API int dbs_set_stroke(dbs_suspension *h, const double *lambda, const double *phase);

/*
 * Constant external force [2S][3] (host) added to the spring force of every
 * sphere (Sec. II: F may include external fields).  NULL removes it.
 */
DBS_API int dbs_set_external_force(dbs_suspension *h, const double *F);

/*
 * Additive Brownian noise (closing remarks of Sec. IV: a constant matrix C
 * in place of a Cholesky factor of the hydrodynamic tensor, adequate for
 * dilute suspensions).  Every sphere is displaced by sigma z per Heun step,
 * sigma = sqrt(2 kT dt / (6 pi mu a)), z ~ N(0, I_3) the same in predictor and
 * corrector.  z is drawn from Philox4x32-10 (Salmon et al., SC'11) on the
 * counter (n mod 2^32, n / 2^32, sphere index, 0) with `seed` as the key,
 * then Box-Muller: z0, z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1),
 * z2 = sqrt(-2 ln u2) cos(2 pi u3), u = (r + 1/2) 2^-32.  kT = 0 turns it
 * off (the default).  kT must be finite and >= 0, else DBS_E_ARG.  All paths
 * but the FP64 cooperative one (kT > 0 there: DBS_E_STATE).
 */
DBS_API int dbs_set_noise(dbs_suspension *h, double kT, uint64_t seed);

/*
 * Dynamics model.  DBS_DYN_SPRING (default): the spring of Eq. (4).
 * DBS_DYN_SHAPE: shape-driven dumbbells (Appendix A.2), the infinitely stiff
 * limit: lengths held at L(t) of Eq. (4) by axial internal forces
 * F^{s1} = f^s N^s, F^{s2} = -f^s N^s from `iterations` >= 1 steps of the
 * paper's iteration f_(n) (1: isolated dumbbells; 2: the pair correction;
 * more approach the exact constraint solution), each one pair sum of Eq. (3)
 * with the exact tensors; then Heun on centre R and axis N (N renormalised),
 * spheres placed at R -/+ N L(t)/2.  Entering it projects the current
 * positions onto L(t_n) (R and N kept).  Grid path, or in FP32C the
 * cooperative path (DBS_PATH_COOP: one launch per <= 1024 steps, one exchange
 * per pair sum; the state double-single within a launch, FP64 between
 * launches); no external force, no noise (DBS_E_STATE otherwise); k0 is
 * ignored.  dbs_velocities then reports the shape-driven velocities.
 */
#define DBS_DYN_SPRING 0
#define DBS_DYN_SHAPE 1
DBS_API int dbs_set_dynamics(dbs_suspension *h, int32_t model, int32_t iterations);

/*
 * Advance n >= 0 Heun steps (Sec. IV) on the device.  Asynchronous: returns
 * after enqueuing; geometry faults found on the device (DBS_E_OVERLAP,
 * DBS_E_NONFINITE) are reported by the next synchronising call
 * (dbs_sync, dbs_positions, dbs_velocities, ...).
 */
DBS_API int dbs_step(dbs_suspension *h, int64_t n);

/* Wait for the handle's stream and report any device-side fault flag. */
DBS_API int dbs_sync(dbs_suspension *h);

/*
 * Velocities v [2S][3] (host) at the current state (x_n, t_n): spring (+
 * external) forces pushed through Eq. (3).  Synchronising.
 */
DBS_API int dbs_velocities(dbs_suspension *h, double *v);

/*
 * Interaction part only, u_a = sum_{b != a} H_ab F_b (Eq. (3b)), for the
 * current forces, into u [2S][3] (host).  Diagnostic.  Synchronising.
 */
DBS_API int dbs_interaction(dbs_suspension *h, double *u);

/*
 * Raw mobility product v = H F (Eq. (3), self term included) at the current
 * positions for an arbitrary force F [2S][3] (host) into v [2S][3] (host).
 * Does not touch the simulation state.  Synchronising.
 */
DBS_API int dbs_mobility_apply(dbs_suspension *h, const double *F, double *v);

/*
 * Velocities at the current state into a device buffer v_dev [2S][3] doubles.
 * Asynchronous (stream-ordered on the handle's stream); faults are reported by
 * the next synchronising call.
 */
DBS_API int dbs_velocities_device(dbs_suspension *h, double *v_dev);

/*
 * Profiling form of dbs_step: n Heun steps launched one kernel at a time (no
 * graph), with a CUDA event pair recorded on the handle's stream around every
 * pair-sum launch; *mean_ms receives the mean device time of one launch.
 * Results are identical to dbs_step.  Synchronising.
 */
DBS_API int dbs_step_timed(dbs_suspension *h, int64_t n, double *mean_ms);

/*
 * Launch tuning of the pair-sum kernel (used by the autotuner): split the
 * j-range into `chunks` pieces (1 <= chunks <= max(1, S/8); 0 restores the
 * built-in choice; on the cooperative path the request is dumbbells per CTA,
 * see DBS_PATH_COOP).  Results change only in the rounding of the j-sum order.
 * dbs_get_launch reports dumbbells per CTA, chunks and grid size (on the
 * cooperative path: dumbbells per CTA, 1, CTAs).
 */
DBS_API int dbs_set_chunks(dbs_suspension *h, int32_t chunks);
DBS_API int dbs_get_launch(dbs_suspension *h, int32_t *bt, int32_t *chunks, int32_t *grid);

/* Current positions x [2S][3] (host).  Synchronising. */
DBS_API int dbs_positions(dbs_suspension *h, double *x);

/* Copy current positions to a device buffer x_dev [2S][3] doubles, stream-ordered. */
DBS_API int dbs_positions_device(dbs_suspension *h, double *x_dev);

/* Step counter n and time t = n dt. */
DBS_API int dbs_get_time(dbs_suspension *h, int64_t *n, double *t);

/* Checkpoint: positions x [2S][3] (host) and step counter n (restart is bit-exact). */
DBS_API int dbs_get_state(dbs_suspension *h, double *x, int64_t *n);
DBS_API int dbs_set_state(dbs_suspension *h, const double *x, int64_t n);

/*
 * Stroke averages of the geometric centre, Eqs. (6b) and (7b): after this
 * call, every complete block of m steps (a stroke period T = m dt) starting
 * at the current step counter yields one snapshot
 *   Rbar^s_k = (1/T) int_{t_k}^{t_k+T} (X_{2s} + X_{2s+1})/2 du
 * (trapezoid rule on the discrete trajectory), accumulated on the device in
 * the integrator's epilogue.  At most max_periods snapshots are kept.
 * m = 0 switches the accumulation off.
 */
DBS_API int dbs_enable_period_average(dbs_suspension *h, int64_t m, int64_t max_periods);

/* Number of complete snapshots so far. */
DBS_API int dbs_period_count(dbs_suspension *h, int64_t *count);

/* Snapshots k0 .. k0+count-1 into Rbar [count][S][3] (host).  Synchronising. */
DBS_API int dbs_period_averages(dbs_suspension *h, int64_t k0, int64_t count, double *Rbar);

/* Device pointer of snapshot k ([S][3] doubles) for device-side comparisons. */
DBS_API int dbs_period_average_device(dbs_suspension *h, int64_t k, const double **Rbar_dev);

/* Static description of the last error on h (or of the last failed create if h is NULL). */
DBS_API const char *dbs_last_error(const dbs_suspension *h);

/* Static name of a status code. */
DBS_API const char *dbs_status_string(int status);

/* ======================================================================== */
/* Stroke-averaged far-field model, Eqs. (9a)-(9e), Sec. III.B              */
/* ======================================================================== */

typedef struct {
    int64_t S;        /* number of dumbbells, >= 2 */
    double a;         /* sphere radius */
    double ell;       /* mean dumbbell length */
    double omega;     /* stroke angular frequency */
    double dt;        /* Heun time step of the averaged dynamics */
    double kpref;     /* K prefactor; Eq. (9d) prints 15/64 */
    int32_t precision;/* DBS_FP32C or DBS_FP64 */
    int32_t device;   /* -1 = current */
    void *stream;     /* cudaStream_t, NULL = own stream */
} dbs_sa_params;

typedef struct dbs_sa dbs_sa;

/*
 * Create the averaged model with centres R [S][3], unit orientations N [S][3],
 * phases phi [S] and amplitudes lambda [S] (host).  Unequal amplitudes enter
 * as lambda^s lambda^r / ell^2 in place of (lambda/ell)^2.
 */
DBS_API int dbs_sa_create(const dbs_sa_params *p, const double *R, const double *N, const double *phi,
                  const double *lambda, dbs_sa **out);
DBS_API int dbs_sa_destroy(dbs_sa *h);

/*
 * n Heun steps of
 *   dR^s/dt = sum_{r != s} J^{sr},  dN^s/dt = -(I - N^s N^s^T) sum_{r != s} K^{sr},
 * N renormalised to unit length after every step.  Asynchronous.
 */
DBS_API int dbs_sa_step(dbs_sa *h, int64_t n);

/* Rates (dR/dt, dN/dt) at the current state into Rdot, Ndot [S][3] (host). */
DBS_API int dbs_sa_rates(dbs_sa *h, double *Rdot, double *Ndot);

/* Current state R, N [S][3] (host).  Synchronising; reports DBS_E_TIMEOUT /
 * DBS_E_CUDA raised by the cooperative path (sticky). */
DBS_API int dbs_sa_state(dbs_sa *h, double *R, double *N);

/*
 * Execution path of dbs_sa_step (Sec. III.B's Heun step either way):
 *  DBS_PATH_GRID  one launch per evaluation of Eqs. (9a)-(9e) (any size and
 *                 precision).
 *  DBS_PATH_COOP  one cooperative launch of up to one CTA per SM advances up to
 *                 1024 averaged steps; each CTA owns T dumbbells (T the
 *                 smallest power of two from 2 to 32 for which ceil(S / T) CTAs
 *                 fit the SMs), holds every record in shared memory and sums its
 *                 targets over all of them; CTAs exchange only (R, N), one
 *                 64-bit word per dumbbell and axis with a parity bit in the
 *                 lowest significand bit of N's component (cleared on use),
 *                 point to point, with no grid-wide barrier.  The next record is
 *                 formed in FP32 from double-single copies of the state, the FP64
 *                 state update (N renormalised) off the critical path from the
 *                 same pair sums.  Every wait is bounded (about one second): a
 *                 launch whose exchange cannot complete ends with DBS_E_TIMEOUT
 *                 (reported by dbs_sa_state / dbs_sa_rates).  FP32C and
 *                 S <= 4096 only (DBS_E_ARG otherwise, the handle stays usable);
 *                 the default wherever it applies.
 * Results of the two paths differ only in the rounding of the pair sums.
 */
DBS_API int dbs_sa_set_path(dbs_sa *h, int32_t path);
/* The path in use and, on DBS_PATH_COOP, the dumbbells per CTA (else 0). */
DBS_API int dbs_sa_get_path(dbs_sa *h, int32_t *path, int32_t *targets_per_cta);

/*
 * Source chunks of DBS_PATH_GRID's launch (Eqs. (9a)-(9e) summed over the
 * sources in `chunks` contiguous ranges by separate CTAs; the last CTA of a
 * target group to finish merges the ranges' compensated partial sums in range
 * order, so results do not depend on which CTA finishes last).  0 restores the
 * built-in choice (more chunks where the grid of target groups would leave
 * part of the SMs idle in its last wave); at most 64 and at most S.  Results
 * for different counts differ only in the rounding of the pair sums.  The
 * partial sums take chunks x S x 14 floats (doubles in FP64) of device memory.
 * DBS_E_ARG for chunks < 0.
 */
DBS_API int dbs_sa_set_chunks(dbs_sa *h, int32_t chunks);
/* The chunk count in use. */
DBS_API int dbs_sa_get_chunks(dbs_sa *h, int32_t *chunks);

/* Device pointer of the current centres R ([S][3] doubles). */
DBS_API int dbs_sa_centres_device(dbs_sa *h, const double **R_dev);

/* Stream-ordered copy of the current centres into R_dev [S][3] doubles (device). */
DBS_API int dbs_sa_copy_centres(dbs_sa *h, double *R_dev);

DBS_API const char *dbs_sa_last_error(const dbs_sa *h);

/* ======================================================================== */
/* Comparison of the two models (pair-distance error)                       */
/* ======================================================================== */

/*
 * For S centres in four device arrays [S][3] (doubles), with
 *   dA^{sr} = |A1^s - A1^r| - |A0^s - A0^r|,  dB^{sr} likewise,
 * computes over all P = S (S - 1) / 2 pairs s < r:
 *   out[0] = max |dA - dB|,  out[1] = sqrt(sum (dA - dB)^2 / P)  (RMS error),
 *   out[2] = sqrt(sum dB^2 / P)  (RMS of the reference change),  out[3] = P,
 * into out (host, 4 doubles).  Stream-ordered on `stream`, then synchronises.
 */
DBS_API int dbs_pair_distance_error(int64_t S, const double *A0_dev, const double *A1_dev,
                            const double *B0_dev, const double *B1_dev, double *out,
                            void *stream);

/*
 * The same four values into out_dev (device, 4 doubles), enqueued on `stream`
 * without synchronising (one kernel launch; the caller reads out_dev after the
 * stream has reached it).  Calls share one device array of partial sums: calls
 * on one stream are ordered; calls on different streams must not overlap.
 * DBS_E_ARG for S < 2 or null pointers, DBS_E_CUDA if the launch fails.
 */
DBS_API int dbs_pair_distance_error_async(int64_t S, const double *A0_dev, const double *A1_dev,
                                          const double *B0_dev, const double *B1_dev, double *out_dev,
                                          void *stream);

/* ======================================================================== */
/* Cluster-resident execution: one system or an ensemble of independent ones */
/* ======================================================================== */

/*
 * Execution path of dbs_step for one FP32C suspension.
 *  DBS_PATH_GRID     every evaluation of Eq. (3) is one launch over all SMs
 *                    (default; any size).
 *  DBS_PATH_CLUSTER  a thread-block cluster of cluster_size CTAs (1, 2, 4, 8 or
 *                    16; 0 = largest useful) holds the whole suspension in
 *                    shared memory and advances up to 1024 Heun steps per
 *                    launch, exchanging j-data through distributed shared
 *                    memory with hardware cluster barriers.  Needs
 *                    2 S x 48 B + partial sums <= 227 KB per CTA (S <= ~2200)
 *                    and S / cluster_size <= 512.
 * Both paths compute the same quantities (Secs. II and IV); the rounding of
 * the j-sums differs.  Errors: DBS_E_ARG for FP64 handles or sizes the path
 * cannot hold.
 */
#define DBS_PATH_GRID 0
#define DBS_PATH_CLUSTER 1
/*
 *  DBS_PATH_COOP     one cooperative launch of up to one CTA per SM advances up
 *                    to 1024 Heun steps.  Each CTA owns T dumbbells and sums
 *                    their pair terms over all records itself; CTAs exchange
 *                    only the records, through flag-tagged words in device
 *                    memory, point to point, with no grid-wide barrier.  Every
 *                    wait is bounded (about one second): a launch whose
 *                    exchange cannot complete ends with DBS_E_TIMEOUT instead
 *                    of hanging.  FP32C: S <= 4096 (every CTA holds all
 *                    records in shared memory), T <= 32.  FP64 (every value
 *                    double precision; a record's doubles carry the exchange's
 *                    parity bit in their lowest significand bit, cleared on
 *                    use, so the pair sum sees positions and G within one unit
 *                    in the last place of the state's): T <= 4, so S <= 4 x the
 *                    SM count (592 on B300), and no additive noise (DBS_E_ARG
 *                    here, DBS_E_STATE from dbs_set_noise on this path).
 *                    dbs_set_chunks(c) on this path (1 <= c <= 16) asks for T =
 *                    the largest power of two not above min(c, the T limit),
 *                    raised until ceil(S / T) CTAs fit the SMs; 0 restores the
 *                    built-in choice (the smallest T that fits; FP32C: 16 for
 *                    S <= 16, at least 2 above).
 */
#define DBS_PATH_COOP 2
DBS_API int dbs_set_path(dbs_suspension *h, int32_t path, int32_t cluster_size);
DBS_API int dbs_get_path(dbs_suspension *h, int32_t *path, int32_t *cluster_size);

typedef struct dbs_ensemble dbs_ensemble;

/*
 * Group `count` independent FP32C suspensions (existing handles on one device,
 * each listed once) so that dbs_ensemble_step advances all of them together:
 * every member runs on its own thread-block cluster, members of equal cluster
 * size and mobility share one launch, and the launches of one block of steps
 * run concurrently.  The members stay valid handles: their state advances in
 * place, and work issued on a member's own stream is ordered before and after
 * the ensemble's.  stream: cudaStream_t of the ensemble, NULL = its own.
 */
DBS_API int dbs_ensemble_create(int32_t count, dbs_suspension *const *members, void *stream,
                                dbs_ensemble **out);
DBS_API int dbs_ensemble_destroy(dbs_ensemble *e);

/* n Heun steps of every member (asynchronous). */
DBS_API int dbs_ensemble_step(dbs_ensemble *e, int64_t n);

/* Wait for the ensemble's work and report member faults. */
DBS_API int dbs_ensemble_sync(dbs_ensemble *e);

/*
 * Cluster size of every member (1, 2, 4, 8 or 16, at least S/512 rounded up
 * to a power of two).  G = NULL restores the built-in balance rule, which
 * gives each member a cluster in proportion to its pair work S^2.  Used by the
 * autotuner.
 */
DBS_API int dbs_ensemble_set_clusters(dbs_ensemble *e, const int32_t *G);
DBS_API int dbs_ensemble_get_clusters(dbs_ensemble *e, int32_t *G);
DBS_API const char *dbs_ensemble_last_error(const dbs_ensemble *e);

/* ======================================================================== */
/* Serving engine: requests admitted by device-memory budget, batched        */
/* ======================================================================== */

/*
 * A request is one simulation: parameters, initial positions, stroke and a
 * number of Heun steps; its result is the positions after those steps.  The
 * engine keeps requests resident on the device as independent suspensions and
 * advances them concurrently, block by block, through dbs_engine_tick
 * (continuous batching): requests that arrive while others run are admitted
 * at the next tick as soon as the device-memory budget and the slot limit
 * allow, members that fit the cluster path run as one ensemble and the others
 * on the grid path, each on its own stream, and finished requests are copied
 * out and freed.
 */
typedef struct {
    size_t hbm_budget_bytes; /* admission budget for resident request state, 0 = unlimited */
    int32_t max_active;      /* resident requests at most, 0 = unlimited */
    int32_t block_steps;     /* Heun steps per request per tick, >= 1 */
    int32_t device;          /* -1 = current device */
    int32_t reserved;        /* must be 0 */
} dbs_engine_params;

#define DBS_REQ_PENDING 0
#define DBS_REQ_RUNNING 1
#define DBS_REQ_DONE 2
#define DBS_REQ_CANCELLED 3
#define DBS_REQ_FAILED 4

typedef struct dbs_engine dbs_engine;

DBS_API int dbs_engine_create(const dbs_engine_params *p, dbs_engine **out);
DBS_API int dbs_engine_destroy(dbs_engine *e);

/*
 * Queue a request (host arrays are copied): p->stream must be NULL, x0 [2S][3],
 * lambda [S], phase [S] (NULL = passive), steps >= 0.  *id identifies it.
 * Parameters are validated when the request is admitted (invalid ones end in
 * DBS_REQ_FAILED).
 */
DBS_API int dbs_engine_submit(dbs_engine *e, const dbs_params *p, const double *x0,
                              const double *lambda, const double *phase, int64_t steps,
                              int64_t *id);

/* Admit queued requests; wait until some block in flight completes (the one
 * ensemble of all cluster-path requests, or one grid-path request's block)
 * and count its steps; retire finished requests; launch the next block of up
 * to block_steps Heun steps of every idle resident request (of the requests on
 * the grid path, each of which fills the device, at most two have a block in
 * flight at a time, the least remaining work -- steps x S^2 -- first).  Blocks
 * complete independently, so a small request never waits for a large one's
 * block.
 * Reports the numbers of resident and queued requests afterwards.
 * DBS_E_TIMEOUT if no block completes within 600 s. */
DBS_API int dbs_engine_tick(dbs_engine *e, int32_t *active, int32_t *pending);

/*
 * State of a request; for DBS_REQ_DONE, x_out [2S][3] (host, may be NULL)
 * receives the final positions and *latency_s (may be NULL) the time from
 * submission to completion on the host clock.
 */
/*
 * Host-side accounting of the engine since creation: ticks, their total host
 * time, the part spent waiting for a block to complete, and how often (and for
 * how long in total) the ensemble of cluster-path requests was rebuilt because
 * its membership changed.  The paper has no counterpart (serving machinery).
 */
typedef struct {
    int64_t ticks, ensemble_rebuilds;
    double tick_s, rebuild_s, wait_s;
} dbs_engine_stats_t;
DBS_API int dbs_engine_stats(const dbs_engine *e, dbs_engine_stats_t *out);

DBS_API int dbs_engine_poll(dbs_engine *e, int64_t id, int32_t *state, double *x_out,
                            double *latency_s);

/* Cancel a queued or resident request (its device memory is freed). */
DBS_API int dbs_engine_cancel(dbs_engine *e, int64_t id);

/* Device bytes the engine charges against the budget for a request of S dumbbells. */
DBS_API int dbs_engine_request_bytes(int64_t S, int32_t precision, size_t *bytes);

DBS_API const char *dbs_engine_last_error(const dbs_engine *e);

/* ======================================================================== */
/* One suspension split by target rows over several processes              */
/* ======================================================================== */

/*
 * The pair sum of Eq. (3b) splits by target rows: the velocity of a sphere
 * needs every record, but only its own dumbbell's state.  Each of nranks
 * processes (one GPU each) holds a full copy of the suspension and computes the
 * Heun evaluations (Sec. IV) of one contiguous block of dumbbells; after every
 * evaluation the ranks exchange the packed records of their blocks (an
 * all-gather, done by the caller, e.g. with NCCL), so that each rank's record
 * buffer again holds all S records before the next evaluation.  The j-order of
 * every sum, the j-split and the i-blocks are those of the unsharded grid path,
 * so each rank's rows are bit-identical to an unsharded run of the same
 * handle configuration (same S, precision, mobility and dbs_set_chunks).
 *
 * dbs_shard_rows: the block [*row0, *row1) of dumbbells that rank `rank` of
 * nranks owns, for i-blocks of rows_per_block dumbbells (the `bt` of
 * dbs_get_launch): rank r takes i-blocks [r nb / nranks, (r + 1) nb / nranks)
 * of the nb = ceil(S / rows_per_block) (block counts differ by at most one).
 * Host only, no device needed.  DBS_E_ARG if nranks exceeds nb.
 */
DBS_API int dbs_shard_rows(int64_t S, int32_t rows_per_block, int32_t nranks, int32_t rank,
                           int64_t *row0, int64_t *row1);

/*
 * Make h (grid path, spring dynamics) compute only rank `rank`'s row block in
 * dbs_shard_eval; *row0, *row1 (may be NULL) receive it.  Call it after any
 * dbs_set_chunks.  A sharded handle refuses dbs_step (DBS_E_STATE).
 */
DBS_API int dbs_shard_set(dbs_suspension *h, int32_t nranks, int32_t rank, int64_t *row0,
                          int64_t *row1);

/*
 * One evaluation for the handle's row block, stream-ordered on its stream:
 * phase 0 = predictor (reads record buffer A, the state x_n; writes the
 * records of x~ for its rows into buffer B), phase 1 = corrector (reads B,
 * writes the records of x_{n+1} into A and advances the step).  Before the
 * next evaluation the caller must fill the other rows of the buffer just
 * written with the other ranks' records (all-gather on the same stream, or
 * after a device synchronisation).
 */
DBS_API int dbs_shard_eval(dbs_suspension *h, int32_t phase);

/*
 * Device pointers of the two record buffers A and B (S records each, owned by
 * the handle) and the bytes of one record (48 for FP32C, 96 for FP64): record
 * s of dumbbell s at byte offset s * record_bytes.
 */
DBS_API int dbs_shard_buffers(dbs_suspension *h, void **records_a, void **records_b,
                              int64_t *record_bytes);

/* ======================================================================== */
/* Allocation-free mobility product                                         */
/* ======================================================================== */

/*
 * Largest number of dumbbells dbs_mobility_apply_noalloc accepts (N = 2S
 * spheres).  Its scratch memory, about 3.3 MB, is a fixed array inside the
 * library, held on every GPU that loads the library until the process exits.
 */
#define DBS_NOALLOC_MAX_S 4096

/*
 * v = H F, the self term plus the FP32 compensated pair sum, for S
 * dumbbells whose positions x_dev [2S][3], forces F_dev [2S][3] and output
 * v_dev [2S][3] are caller-owned device buffers (doubles) on the current
 * device; mobility is DBS_OSEEN or DBS_RPY.  Positions are packed relative to
 * the first sphere before their FP32 rounding, so the result does not depend
 * on where the suspension sits.  Work is enqueued on `stream` (NULL = legacy
 * default stream); the call then waits for it and reads a status word back to
 * the host before it returns, reporting DBS_E_OVERLAP / DBS_E_NONFINITE for
 * geometry faults.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run -- code inside a framework that
 * owns all device memory through its own capped pool, or a latency-critical
 * loop where cudaMalloc/cudaFree would stall the device.  It needs no handle
 * and calls no allocator: its scratch (packed j-data, chunk partial sums,
 * arrival counters) lives in one static device array that every call shares.
 *  - S > DBS_NOALLOC_MAX_S (or S < 1) is rejected with DBS_E_ARG.
 *  - The array keeps the last call's contents; the counters that must start
 *    at zero are cleared at the start of every call.
 *  - Calls that overlap on the GPU (two streams, two host threads) race on
 *    the array: serialise them.
 *  - The first call on each device performs a one-time set-up (it looks up
 *    the array's device address); make that first call before any stream
 *    capture.
 */
DBS_API int dbs_mobility_apply_noalloc(int64_t S, const double *x_dev, const double *F_dev,
                                       double a, double mu, int32_t mobility, double *v_dev,
                                       void *stream);

/*
 * Diagnostic of the bounded device-side wait used by the cooperative path:
 * one warp polls a word that nothing writes, so that its wait must run out
 * after timeout_ms (1..10000); *status receives the outcome (DBS_E_TIMEOUT
 * expected) and the call returns DBS_OK if the device stayed usable.
 */
DBS_API int dbs_test_wait_timeout(int32_t timeout_ms, int32_t *status);

/*
 * Diagnostic: set the evaluation counter of the cooperative path (rounded down
 * to a multiple of 4; the exchange buffers are cleared), so that a test can run
 * the counter through its wrap-around at 2^32: the records' parity bits depend
 * only on the counter modulo 4, which the wrap keeps.  DBS_E_STATE if the
 * handle is not on the cooperative path.
 */
DBS_API int dbs_test_set_flow_tag(dbs_suspension *h, uint32_t tag);

/*
 * Diagnostic of the cooperative kernel's launch-shape check: one Heun step on
 * the cooperative path whose kernel is told it has one CTA more than it was
 * launched with.  Every CTA must refuse before touching the state or the
 * exchange buffers and raise the launch flag; returns what the flag check then
 * returns (DBS_E_CUDA expected; the handle keeps that error).  DBS_E_STATE if
 * the handle is not on the cooperative path.
 */
DBS_API int dbs_test_flow_misshape(dbs_suspension *h);

/*
 * Diagnostic of the cluster-resident kernel's launch-shape check: one Heun step
 * of the ensemble whose kernels are told to expect twice their true cluster
 * size.  Every CTA must refuse before touching member state and raise the
 * launch flag; returns what dbs_ensemble_sync then returns (DBS_E_CUDA,
 * "kernel launched in a grid or cluster shape it cannot run", expected).  The
 * members are left in that error state (sticky): destroy them afterwards.
 */
DBS_API int dbs_test_ensemble_misshape(dbs_ensemble *e);

/*
 * Diagnostic of the averaged model's cooperative kernel's launch-shape check:
 * one averaged step whose kernel is told it has one CTA more than it was
 * launched with.  Every CTA must refuse before touching the state or the
 * exchange words; returns what the flag check then returns (DBS_E_CUDA
 * expected; the handle keeps that error).  DBS_E_STATE if the handle is not on
 * the cooperative path.
 */
DBS_API int dbs_test_sa_flow_misshape(dbs_sa *h);

/* Library version string. */
DBS_API const char *dbs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DBS_H */
