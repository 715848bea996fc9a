/*
 * qym.h -- C ABI of libqym, a GB300 (sm_103a) implementation of the
 * democratic-heliocentric (DH) hybrid symplectic step of Moore & Quillen,
 * "QYMSYM: A GPU-accelerated hybrid symplectic integrator that permits close
 * encounters" (New Astronomy).
 *
 * One step (Sec. 2, Eq. 5) is E_Dft(tau/2) E_Int(tau/2) E_Kep(tau) E_Int(tau/2)
 * E_Dft(tau/2), with close encounters found during the step and handed to a
 * Hermite sub-integrator (Sec. 2.1-2.4).
 *
 * Conventions shared by every call:
 *  - Plain C types only. No exception crosses this boundary; every call returns
 *    a qym_status (0 = QYM_OK). qym_last_error() gives a message for the last
 *    failing call on a context (or on the thread, for context-free calls).
 *  - Units: G, masses, lengths and times are the caller's; the paper uses
 *    G m0 = 1 and lengths in units of a planet's semi-major axis.
 *  - A "system" is one star plus its bodies; rows of a batch are concatenated
 *    and offsets[s] is the row of system s's star (offsets[nsys] = rows). The
 *    star row of each system is held at Q = P = 0 (Sec. 2: the star is kept
 *    at index 0 and its mass is zeroed in H_Int).
 *  - HOST arrays (the qym_ctx calls) are caller owned, row-major [rows][3]
 *    float64, read or written during the call only, never retained.
 *  - DEVICE arrays (the *_dev calls) are caller-owned CUDA device pointers in
 *    the current device's memory, structure-of-arrays [3][n] float64 (all x,
 *    then all y, then all z); work is enqueued on `stream` (a cudaStream_t
 *    passed as void*, NULL = legacy default stream) and the call returns
 *    without waiting unless stated. Device status words are int32 in device
 *    memory; the library only ever sets bits in them (OR), so zero them first.
 *  - Nothing here traps or spins without bound on the GPU: every device-side
 *    iteration has a cap and reports through a status word instead.
 */
#ifndef QYM_H
#define QYM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qym_status {
    QYM_OK = 0,
    QYM_EINVAL = 1,     /* bad argument (sizes, offsets, tau, parameters) */
    QYM_ENOMEM = 2,     /* device or host allocation failed */
    QYM_ECUDA = 3,      /* a CUDA runtime call failed (message has the name) */
    QYM_ENAN = 4,       /* a non-finite position or velocity appeared */
    QYM_ENOCONV = 5,    /* Kepler iteration or Hermite step cap reached */
    QYM_EOVERFLOW = 6,  /* a candidate / encounter / set capacity was exceeded */
    QYM_ENODEV = 7      /* no CUDA device, or the device is not sm_103 class */
} qym_status;

/* Bits of the device status word (per step, OR-ed). */
#define QYM_ST_KEPLER_NOCONV   0x01  /* a Kepler solve hit max_kepler_iter */
#define QYM_ST_HERMITE_CAP     0x02  /* an encounter set hit max_hermite_steps */
#define QYM_ST_CAND_OVERFLOW   0x04  /* more crude candidates than max_candidates, or
                                        more flagged (row, chunk) records of the mixed
                                        search kick than max_candidates + rows */
#define QYM_ST_ENC_OVERFLOW    0x08  /* more encounter pairs than max_encounters */
#define QYM_ST_SET_OVERFLOW    0x10  /* a set larger than the set capacity (or than
                                        the 320 members the Hermite holds on chip) */
#define QYM_ST_NAN             0x20  /* non-finite state after the Kepler drift */
#define QYM_ST_UF_CAP          0x40  /* set-building iteration cap reached */
#define QYM_ST_LOG_OVERFLOW    0x80  /* encounter log of this qym_step call is full */

/* Kick arithmetic (Sec. 2, footnote on precision; Gaburov-style corrector). */
#define QYM_KICK_FP64   0   /* plain FP64 pair forces */
#define QYM_KICK_MIXED  1   /* FP32 pair forces on double-single separations,
                               compensated (two-sum) accumulation into FP64 */

/* Kepler solver and starting guess (Appendix). */
#define QYM_SOLVER_LAGUERRE 0   /* Laguerre, n = 5 */
#define QYM_SOLVER_NEWTON   1
#define QYM_SOLVER_NEWTON32 2   /* Newton steps in FP32 from the starting guess until a step
                                   falls below 1e-5 |x|, then Laguerre in FP64 under the same
                                   residual test and bracket: the same root, fewer FP64
                                   evaluations; the iteration count adds both kinds */
#define QYM_GUESS_STANDARD  0   /* x0 = sqrt(mu) dt / r0 */
#define QYM_GUESS_R0        1   /* x0 = r0, as the Appendix does */
#define QYM_GUESS_MLP       2   /* learned guess (qym_set_mlp); falls back to
                                   Laguerre from the standard guess */

typedef struct qym_params {
    double G;            /* gravitational constant */
    double a_E;          /* encounter factor: flag d_min < a_E (r_H,i + r_H,j) (Sec. 2.4) */
    double a_H;          /* transition factor: r_crit = a_H max r_H over a set (Eq. 9) */
    double eps_H;        /* Hermite smoothing length (Sec. 2.2: small but not zero, so
                            that a near-collision cannot drive the step to zero) */
    double eta, eta_s;   /* Hermite step accuracy and start-up factors (Sec. 2.2) */
    int32_t kick_prec;   /* QYM_KICK_* */
    int32_t solver;      /* QYM_SOLVER_* */
    int32_t guess;       /* QYM_GUESS_* */
    int32_t encounters;  /* 0: plain DH step; 1: hybrid step with encounters (Sec. 2.3) */
    int32_t coords;      /* 0: q, v given/returned heliocentric; 1: DH (heliocentric q,
                            barycentric v = P/m) */
    int32_t hill_fixed;  /* 0: Hill radii from the orbit entering each Kepler step;
                            1: Hill radii computed once at init and held */
    int32_t max_kepler_iter;
    int32_t device;      /* CUDA device ordinal */
    int64_t max_hermite_steps;  /* per set per step */
    int64_t max_candidates;     /* crude candidate pairs per step (0: automatic) */
    int64_t max_encounters;     /* rigorous encounter pairs per step (0: automatic) */
    int64_t max_log;            /* encounter records kept per qym_step call (0: automatic) */
    int64_t l2_flush_bytes;     /* > 0: write a scratch buffer of this size at the start of
                                   every step (benchmarks that must not reuse L2 between
                                   steps); 0: off */
    double heavy_mass;          /* mixed kick only: bodies with m >= heavy_mass * m0 (at most
                                   QYM_HEAVY_CAP per system) pull on every body in FP64; the
                                   N^2 part among the others stays FP32. <= 0: off */
    int32_t merge_kicks;        /* 1: inside one qym_step call, the closing kick of a step
                                   and the opening kick of the next are one kick of tau
                                   (exact: E_Dft is a uniform shift and E_Int conserves the
                                   total momentum, so Int(tau/2) Dft(tau) Int(tau/2) =
                                   Dft(tau) Int(tau)); one all-pairs pass per step instead
                                   of two. 0: the paper's two kicks per step */
    int32_t hermite_cluster;    /* CTAs of a thread-block cluster that share one large
                                   encounter set in the Hermite: 2, 4 or 8; 0: automatic
                                   (8 for a single system, 2 for a batch of systems) */
    int32_t search;             /* how the close-encounter candidates are found (Sec. 2.4):
                                   QYM_SEARCH_AUTO (default), _FUSED, _BINNED or _ESCAPE */
    int32_t whole_hermite;      /* 1: Sec. 2.3, last paragraph: when a step's encounter sets
                                   put two planets in one set, that system's step is redone
                                   by the Hermite for every body: from the positions after the
                                   opening drift and the velocities entering the first kick,
                                   all bodies over tau under H_Kep + H_Int (star fixed at the
                                   origin, every pair with its full force, smoothed with
                                   eps_H), no K corrections and no second kick, then the
                                   closing drift. qym_step then reads the sets back once per
                                   step (no step graph); not with merge_kicks or a split
                                   step. 0 (default): off */
    double planet_mass;         /* planets for whole_hermite: m >= planet_mass * m0
                                   (default 1e-7) */
} qym_params;

/* Close-encounter search: which pairs the rigorous test (Sec. 2.4) examines.
 * FUSED: a crude reach per body from the state before the first kick, tested
 *   inside that kick over all pairs (the paper's crude sweep riding on the
 *   kick); rows whose kick or Hill radius exceeds what the reach assumed are
 *   re-searched exactly.
 * BINNED: after the Kepler drift, per body a box that holds its cubic
 *   Hermite path over the step widened by a_E r_H and a bound on how far the
 *   test's cubic can fall below the paths' distance; tiles of bodies (the
 *   kick's Morton order for one system) and pairs of overlapping tiles; within
 *   them pairs of overlapping boxes, filtered by the test's cubic in FP32 with
 *   an error allowance. Every pair the test can flag is examined, by
 *   construction; the kicks carry no search. A split context (qym_split_init)
 *   always uses FUSED. */
#define QYM_SEARCH_FUSED  0
#define QYM_SEARCH_BINNED 1
#define QYM_SEARCH_AUTO   2   /* BINNED for one system of at least 65536 bodies (there
                                 binning costs less than the all-pairs reach test in the
                                 kick), FUSED otherwise */
/* ESCAPE: the paper's own crude sweep (Sec. 2.4), fused into the first kick like
 *   FUSED: a pair is a candidate when its separation at the start of the step is
 *   below a_E times the Hill radii plus the distance a body covers at its escape
 *   velocity sqrt(2 G m0 / |Q|) over tau, each body contributing its own term
 *   (rho_i = a_E r_H,i + |tau| v_esc,i; tested as r^2 < 2 rho_i^2 + 2 rho_j^2). No
 *   |a| allowance and no re-search: as the paper notes, a body moving faster than
 *   escape can be missed (the other modes' lists equal the all-pairs test). A
 *   split context uses FUSED. */
#define QYM_SEARCH_ESCAPE 3

#define QYM_HEAVY_CAP 256

typedef struct qym_stats {
    int64_t steps;              /* steps taken by the last qym_step call */
    int64_t candidates;         /* crude candidate pairs, summed over those steps */
    int64_t encounters;         /* rigorous encounter pairs, summed */
    int64_t sets;               /* encounter sets, summed */
    int64_t max_set;            /* largest set seen */
    int64_t kepler_iters;       /* Kepler solver iterations, summed over bodies and steps */
    int64_t hermite_steps;      /* Hermite steps, summed over sets and steps */
    int64_t rescans;            /* bodies re-searched because a crude bound was exceeded */
    int64_t launches;           /* kernel launches enqueued by the last qym_step call */
    int64_t hermite_steps_max;  /* most Hermite steps one set took within one step */
    int32_t status_bits;        /* OR of QYM_ST_* seen */
    int32_t kick_tile_i, kick_tile_splits;  /* launch shape in use */
    int32_t whole_steps;        /* steps integrated whole by the Hermite (whole_hermite) */
} qym_stats;

typedef struct qym_ctx qym_ctx;   /* opaque; owned by the library */

/* ------------------------------------------------------------------------ */
/* Context API: state resident on the device between calls (Sec. 2:         */
/* positions and velocities stay on the GPU; host copies only on request).  */
/* ------------------------------------------------------------------------ */

/* Fill *p with defaults: G = 1, a_E = 3, a_H = 1, eps_H = 1e-6, eta = 0.02,
 * eta_s = 0.01, mixed kick, Laguerre, standard guess, encounters on,
 * heliocentric coordinates, per-step Hill radii, 50 Kepler iterations,
 * 1e5 Hermite steps, automatic capacities. Returns QYM_EINVAL if p is NULL. */
qym_status qym_default_params(qym_params *p);

/* Create a context on params->device and upload a batch of systems.
 *  nsys      number of systems (>= 1)
 *  offsets   host int64[nsys+1], offsets[0] = 0, strictly increasing; each
 *            system has its star at row offsets[s] and at least one body
 *  m         host float64[rows] masses (m > 0 for stars, m >= 0 for bodies)
 *  q, v      host float64[rows][3]: positions relative to the system's star
 *            and velocities (heliocentric or DH per params->coords); star rows
 *            are ignored and set to zero
 * Heliocentric velocities are converted to barycentric ones on the device
 * (Sec. 2). Device memory is sized here for the capacities in params.
 * On error *out is NULL and nothing is leaked. */
qym_status qym_init(const qym_params *params, int32_t nsys, const int64_t *offsets,
                    const double *m, const double *q, const double *v, qym_ctx **out);

/* Advance every system by nsteps steps of size tau (tau may be negative for a
 * reversed integration; tau = 0 or nsteps < 0 is QYM_EINVAL). Returns after the
 * device has finished. Encounter records of this call replace the previous
 * call's. On QYM_ENOCONV / QYM_EOVERFLOW / QYM_ENAN the steps already taken are
 * kept, qym_stats tells which, and the context stays usable. */
qym_status qym_step(qym_ctx *ctx, double tau, int64_t nsteps);

/* Copy the state to host float64[rows][3] arrays (coordinates per
 * params->coords; star rows are zero). Either pointer may be NULL. */
qym_status qym_get_state(qym_ctx *ctx, double *q, double *v);

/* Replace the state (same layout and coordinates as qym_init). Used to resume
 * from a checkpoint; Hill radii are recomputed if params.hill_fixed. */
qym_status qym_set_state(qym_ctx *ctx, const double *q, const double *v);

/* Copy the encounter records of the last qym_step call to host int64
 * recs[cap][3] = (step, i, j): step counted from 0 within that call, i < j
 * global row indices, sorted by (step, i, j). *count receives the total number
 * found (which may exceed cap; only cap records are written). */
qym_status qym_get_encounters(qym_ctx *ctx, int64_t *recs, int64_t cap, int64_t *count);

/* Copy the order in which the kick holds the bodies' operand packs to host
 * int32 order[rows]: position p holds row order[p]. A single system of at
 * least 2048 bodies with the mixed kick is held along a Morton curve of its
 * positions (ordered by (code, row); taken at qym_set_state, at the start of
 * every qym_step call and every 32 steps within one; the star row stays at
 * 0); otherwise the order is the identity. Results depend on it only through
 * the grouping of the FP32 sums of the single-precision interaction step
 * (Sec. 2). */
qym_status qym_get_order(qym_ctx *ctx, int32_t *order);

/* Total energy H_Dft + H_Kep + H_Int of each system (Sec. 2, Eqs. 2-4, star
 * mass restored for the pair sum), FP64, into host double E[nsys]. */
qym_status qym_energy(qym_ctx *ctx, double *E);

/* Counters of the last qym_step call. */
qym_status qym_get_stats(qym_ctx *ctx, qym_stats *st);

/* The parameters ctx runs with: those given to qym_init, with the choices
 * the library made filled in (search: QYM_SEARCH_FUSED or _BINNED, never
 * _AUTO; a split context reports FUSED). */
qym_status qym_get_params(const qym_ctx *ctx, qym_params *p);

/* Learned Kepler starting guess (the Appendix's universal Kepler equation
 * solved from a predicted start instead of x_std = sqrt(mu) dt / r0). A
 * 4 -> 64 -> 64 -> 1 perceptron with GELU (tanh form) maps the features
 *   u1 = q.v / sqrt(mu r0), u2 = r0 |v|^2 / mu, u3 = ln s,
 *   u4 = dt / P (dt sqrt(mu alpha^3) / 2 pi for bound orbits, else 0),
 * s = |dt| sqrt(mu / r0^3), each normalised as (u - mean) / std, to
 * t = om + osd * y; the guess is x_std (1 + sigma t) with sigma = s / (1 + s).
 * Weights: one float32 vector of QYM_MLP_NW entries, in the order W1[64][4],
 * b1[64], W2[64][64], b2[64], W3[64], b3, mean[4], std[4], om, osd. The matrices
 * are rounded to bf16 where they are used (tensor cores, FP32 accumulation).
 * The network is used for bodies on bound orbits (alpha = 2/r0 - |v|^2/mu > 0,
 * where |u1| < sqrt 2 and u2 < 2); the others keep x_std. If the iteration
 * from the learned guess does not converge, Laguerre from the standard guess
 * is run. */
#define QYM_MLP_NW 4555

/* Set the network used by qym_step with params.guess == QYM_GUESS_MLP
 * (host float32 weights[n], n == QYM_MLP_NW, std entries > 0). Returns
 * QYM_EINVAL for a wrong n or non-finite weights. qym_step with
 * QYM_GUESS_MLP fails with QYM_EINVAL until a network is set. */
qym_status qym_set_mlp(qym_ctx *ctx, const float *weights, int64_t n);

/* Log every Kepler solve of the following qym_step calls as a training row
 * (u1, u2, u3, u4, t) with t = (x / x_std - 1) / sigma at the converged root
 * x: device float32 rows[cap][5] (caller owned, kept until replaced). The
 * solve of row k in the s-th step after this call goes to row s * R + k (R
 * = total rows of ctx) while that is below cap; only solves on bound orbits
 * are written (star rows and unbound bodies leave their rows untouched).
 * cap = 0 (rows NULL) stops logging. */
qym_status qym_set_kepler_log(qym_ctx *ctx, float *rows, int64_t cap);

/* Record the inputs of the rigorous encounter test (Sec. 2.3 item 4, Sec.
 * 2.4) of the last step of every following qym_step call: the state entering
 * the Kepler drift (positions q0 after the opening drift, velocities v0 after
 * the first kick), the Kepler drift's result (q1, v1, before the Hermite
 * replaces the encounter sets' rows) and the Hill radii rH the test used.
 * q0, v0, q1, v1: device float64[3][rows] (all x, then y, then z); rH:
 * device float64[rows]; caller owned, written by device-to-device copies on
 * the context's stream inside qym_step, kept until replaced. Positions are
 * heliocentric, velocities barycentric (the DH coordinates the test works
 * in), star rows zero. With these arrays the encounter records of that step
 * (qym_get_encounters) can be recomputed exactly by anyone: they are the
 * pairs i < j of one system with d_min^2 < (a_E (rH_i + rH_j))^2. All five
 * NULL stops recording; a mix of NULL and non-NULL is QYM_EINVAL. */
qym_status qym_set_encounter_snapshot(qym_ctx *ctx, double *q0, double *v0, double *q1,
                                      double *v1, double *rH);

/* Message for the last error on ctx (ctx may be NULL: last context-free error
 * of the calling thread). The string lives until the next call on ctx. */
const char *qym_last_error(const qym_ctx *ctx);

/* Free every device and host resource of ctx (NULL is accepted). */
void qym_destroy(qym_ctx *ctx);

/* Number of rows and systems of ctx. */
qym_status qym_shape(const qym_ctx *ctx, int64_t *rows, int32_t *nsys);

/* The CUDA stream (cudaStream_t as void*) on which ctx enqueues all of its
 * work, for callers that record events or order their own work after it. */
qym_status qym_get_stream(const qym_ctx *ctx, void **stream);

/* Time the all-pairs kick kernel of ctx alone: `reps` launches on the ctx
 * stream over the current state, bracketed by CUDA events, without changing
 * the state (velocities are not updated). with_search = 1 times the variant
 * with the fused crude encounter search. *ms_per_launch gets the mean launch
 * duration in milliseconds; *pairs the ordered interacting pairs per launch
 * (sum over systems of N_b (N_b - 1)). */
qym_status qym_time_kick(qym_ctx *ctx, int32_t with_search, int32_t reps, double *ms_per_launch,
                         int64_t *pairs);

/* Time E_Dft (Sec. 2, Eq. 2) of ctx alone: `reps` launches each of the
 * barycentric-momentum reduction (S = sum m v per system) and of the drift
 * (Q += (tau/2) S / m0 twice, the closing and the next opening half-drift,
 * then the kick's float packs) on the ctx stream, bracketed by CUDA events;
 * the drift reads a copy of the state and the state is put back afterwards.
 * *ms_momentum and *ms_drift get the mean launch times in milliseconds.
 * QYM_EINVAL for reps < 1, tau zero or not finite, or a NULL pointer. */
qym_status qym_time_drift(qym_ctx *ctx, double tau, int32_t reps, double *ms_momentum,
                          double *ms_drift);

/* Set the kick launch shape: threads per CTA (128 or 256), i rows per thread
 * (1, 2, or 4 for the mixed kick) and j splits per system (1 .. the largest
 * the context's buffers hold, at least 4); QYM_EINVAL otherwise. For
 * reproducing a shape the tuner chose (qym_stats kick_tile_i, _splits). */
qym_status qym_set_kick_shape(qym_ctx *ctx, int32_t threads, int32_t ipt, int32_t splits);

/* Pick the kick launch shape (threads per CTA, rows per thread, j splits)
 * by timing candidate shapes with qym_time_kick on the current state, and
 * keep the fastest. The state is unchanged; results can differ from the
 * default shape in the last bits (summation grouping). */
qym_status qym_autotune(qym_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Device-level calls: one operator of the step on caller-owned device      */
/* buffers, enqueued on `stream`. These are the same kernels qym_step runs. */
/* ------------------------------------------------------------------------ */

/* E_Kep (Sec. 2, Appendix): advance n bodies on Kepler orbits about a star of
 * gravitational parameter mu for dt with universal-variable f and g functions.
 *  q0, v0    device float64[3][n] input state (not modified)
 *  q1, v1    device float64[3][n] output state (must not alias q0, v0)
 *  solver    QYM_SOLVER_*; guess QYM_GUESS_STANDARD, QYM_GUESS_R0, or
 *            QYM_GUESS_MLP with mlp_w != NULL
 *  mlp_w     device float32[QYM_MLP_NW] guess network (16-byte aligned), or NULL
 *  x_out     device float64[n] universal variable x, or NULL
 *  x0_out    device float64[n] starting value of x, or NULL
 *  iters     device int32[n] iterations used, or NULL
 *  log_rows  device float32[n][5] training row (u1..u4, t) of each body on a
 *            bound orbit with r0 > 0 and dt != 0 (others untouched), or NULL
 *  status    device int32 word, QYM_ST_KEPLER_NOCONV / QYM_ST_NAN OR-ed in, or NULL
 * n = 0 is a no-op. Returns QYM_EINVAL for n < 0, mu <= 0, max_iter < 1, an
 * unknown solver or guess, or QYM_GUESS_MLP without mlp_w. */
qym_status qym_kepler_drift_dev(int64_t n, const double *q0, const double *v0, double *q1,
                                double *v1, double mu, double dt, int32_t solver, int32_t guess,
                                const float *mlp_w, int32_t max_iter, double *x_out,
                                double *x0_out, int32_t *iters, float *log_rows, int32_t *status,
                                void *stream);

/* The transition function of the hybrid split (Sec. 2.1) as the Hermite
 * sub-integrator evaluates it: K(y) = sin(pi y / 2) for 0 < y < 1 (0 below,
 * 1 above), y = 1.1 s / r_crit - 0.1, with its first and second derivatives
 * with respect to s, for n distances s (device float64[n]) into device
 * float64 K[n], Kp[n], Kpp[n]. Returns QYM_EINVAL for n < 0 or r_crit <= 0. */
qym_status qym_transition_dev(int64_t n, const double *s, double r_crit, double *K, double *Kp,
                              double *Kpp, void *stream);

/* The guess network's normalised output y for raw features u (device
 * float32[n][4], 16-byte aligned) into device float32 y[n]; w as in
 * qym_set_mlp (device, 16-byte aligned). n = 0 is a no-op. */
qym_status qym_mlp_forward_dev(int64_t n, const float *w, const float *u, float *y, void *stream);

/* Training of the guess network on rows (u1, u2, u3, u4, t), device
 * float32[n][5]: the loss is the mean over the rows of (y - (t - om)/osd)^2.
 * work: device scratch of qym_mlp_workspace_bytes() bytes (caller owned).
 *
 * qym_mlp_grad_dev: dL/dw of all n rows into device float32 grad[QYM_MLP_NW]
 *   (zero for the ten normalisation entries) and, if loss != NULL, L into
 *   device float32 *loss.
 * qym_mlp_adam_dev: one Adam step (Kingma & Ba) number t >= 1 with gradient
 *   grad on w, first and second moments m, v (device float32[QYM_MLP_NW]):
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); the normalisation
 *   entries are left unchanged.
 * qym_mlp_train_dev: `epochs` passes over the rows in minibatches of `batch`
 *   consecutive rows (the last one ragged), a gradient and an Adam step per
 *   minibatch (betas 0.9, 0.999, eps 1e-8, step numbers t0 + 1, ...) with the
 *   learning rate following a cosine from lr down to lr_final over all steps;
 *   losses: device float32[steps] minibatch losses, or NULL. */
size_t qym_mlp_workspace_bytes(void);
qym_status qym_mlp_grad_dev(int64_t n, const float *w, const float *rows, float *grad, float *loss,
                            void *work, size_t work_bytes, void *stream);
qym_status qym_mlp_adam_dev(float *w, float *m, float *v, const float *grad, int64_t t, float lr,
                            float beta1, float beta2, float eps, void *stream);
qym_status qym_mlp_train_dev(float *w, float *m, float *v, int64_t t0, const float *rows, int64_t n,
                             int64_t batch, int32_t epochs, float lr, float lr_final, float *losses,
                             void *work, size_t work_bytes, void *stream);

/* E_Int acceleration (Sec. 2, Eq. 4) of one system: for rows i >= 1
 *   a_i = -sum_{j >= 1, j != i} G m_j (Q_i - Q_j) / |Q_i - Q_j|^3,
 * star row excluded (a_0 = 0).
 *  m           device float64[rows]
 *  q           device float64[3][rows]
 *  a           device float64[3][rows] output
 *  prec        QYM_KICK_FP64 or QYM_KICK_MIXED
 *  heavy_mass  QYM_KICK_MIXED: bodies with m >= heavy_mass * m[0] (the first
 *              QYM_HEAVY_CAP of them) are summed in FP64; <= 0: none
 *  work        device scratch of qym_accel_workspace_bytes(rows, prec) bytes
 *              (caller owned, contents irrelevant on entry)
 * Returns QYM_EINVAL for rows < 2 or a NULL / short workspace. */
size_t qym_accel_workspace_bytes(int64_t rows, int32_t prec);
qym_status qym_accel_dev(int64_t rows, const double *m, const double *q, double *a, double G,
                         int32_t prec, double heavy_mass, void *work, size_t work_bytes,
                         void *stream);

/* The same accelerations as qym_accel_dev, for callers that cannot allocate
 * device memory: code running where the host application owns every device
 * allocation, or loops that must not call the allocator (and its implicit
 * synchronisation) once they are running. The scratch lives in one fixed
 * array inside the library (qym_static_scratch_bytes() bytes, 8 MiB),
 * which every GPU that loads the library holds until the process exits.
 * The paper has no counterpart; this is a deployment convenience.
 *  rows     2 .. QYM_STATIC_MAX_ROWS; larger systems return QYM_EINVAL with a
 *           clear message (use qym_accel_dev then)
 *  m, q, a, G, prec, heavy_mass, stream: as qym_accel_dev (caller-owned)
 * Error messages go where every context-free call's go (qym_last_error(NULL));
 * qym_static_last_error() returns the same text.
 * The call allocates nothing (no cudaMalloc or allocating library routine).
 * The array's device address is looked up, with the current device, on every
 * call that is not being captured into a CUDA graph (so a device reset between
 * calls is harmless); a call made during a capture uses the address its last
 * call on that device found, so make one call on a device before capturing
 * it (a capture without one fails with QYM_ECUDA). All calls
 * share the one array and every call rewrites all of the scratch it reads,
 * so nothing carries over between calls; calls that overlap on the GPU (on
 * different streams, or from several threads) race on it and must be
 * serialised by the caller. */
#define QYM_STATIC_MAX_ROWS 32768
size_t qym_static_scratch_bytes(void);
qym_status qym_accel_dev_static(int64_t rows, const double *m, const double *q, double *a,
                                double G, int32_t prec, double heavy_mass, void *stream);
const char *qym_static_last_error(void);

/* Rigorous encounter test (Sec. 2.4): for each of npairs candidate pairs
 * (pairs[2k], pairs[2k+1]) of rows, the minimum over [0, tau] of the cubic that
 * interpolates |dQ(t)|^2 from its values and slopes at t = 0 (q0, v0) and
 * t = tau (q1, v1), clamped at 0, into d2[k]; flag[k] = d2[k] <
 * (a_E (rH_i + rH_j))^2. All arrays are device arrays ([3][rows] for states). */
qym_status qym_encounter_test_dev(int64_t rows, const double *q0, const double *v0,
                                  const double *q1, const double *v1, const double *rH,
                                  double tau, double a_E, int64_t npairs, const int32_t *pairs,
                                  double *d2, int32_t *flag, void *stream);

/* Total energy of one system (Sec. 2, Eqs. 2-4), star at row 0, into device
 * double E[1]. `work` is caller-owned device scratch of
 * qym_energy_workspace_bytes(rows) bytes. Small work tables are staged from
 * the host, so this call waits for `stream` before returning. */
size_t qym_energy_workspace_bytes(int64_t rows);
qym_status qym_energy_dev(int64_t rows, const double *m, const double *q, const double *v,
                          double G, double *E, void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* One system's step split over several GPUs (one process and one context  */
/* per GPU). Every context holds the whole state. Context `rank` of `world`  */
/* owns the contiguous block of bodies qym_split_rows gives (equal blocks,   */
/* the last one shorter): it computes the kick of those rows against every  */
/* row (Sec. 2, Eq. 4) with the crude encounter search of those rows (Sec.  */
/* 2.4), their Kepler drift (Appendix), the rigorous test of their           */
/* candidates, and the Hermite sub-integration (Sec. 2.2-2.3) of the         */
/* encounter sets whose lowest row it owns. The momentum sum, the drifts     */
/* (Sec. 2, Eq. 2), the kick operand packs and the encounter sets are        */
/* computed on every context from identical data in a fixed order, so they   */
/* agree to the bit without an exchange. The caller runs the phases of each  */
/* step in order and moves data between the contexts after some of them:     */
/*                                                                           */
/*   OPEN      first step of a run only: momentum, opening drift, packs      */
/*   KICK1     step begin, first kick of the own rows (with the search       */
/*             unless this is the run's first step after init / set_state),   */
/*             finish of the own rows;                                       */
/*             then allgather v, amag and rH of the own rows                 */
/*   SEARCH    (first step of a run only) reaches of every row from the      */
/*             kicked state, search of the own rows                          */
/*   KEPLER    Kepler drift of the own rows; then allgather q1, v1           */
/*   REFINE    rigorous test of the own candidates; then gather every        */
/*             context's pairs (enc[0 .. qym_split_encounter_count)) and     */
/*             give the concatenation to qym_split_import_encounters on      */
/*             every context (the order of the pairs does not matter)        */
/*   HERMITE   encounter sets of all pairs, Hermite of the own sets; then    */
/*             every context sends the rows set_mem[first .. first + count)  */
/*             (qym_split_owned_members) with their q1, v1 and hcost to all  */
/*             the others, which write them over their own copies            */
/*   KICK2     pack from (q1, v1), second kick and finish of the own rows;   */
/*             then allgather v and amag of the own rows                     */
/*   CLOSE     momentum, closing drift (and, unless last, the next step's    */
/*             opening drift and packs), step end; with last = 1 it waits    */
/*             for the device and returns the run's status as qym_step does   */
/* A run is OPEN, then for each step KICK1, SEARCH, KEPLER, REFINE, HERMITE,  */
/* KICK2, CLOSE (last = 1 on its last step). With encounters off the         */
/* SEARCH, REFINE and HERMITE phases do nothing. Arrays of the state are     */
/* structure-of-arrays [3][rows] (v: barycentric), per-row arrays [rows];    */
/* qym_split_arrays gives their device addresses (valid until               */
/* qym_destroy) and the context's stream, on which every phase enqueues its  */
/* work: exchanges must be ordered after it. The Kepler solve log            */
/* (qym_set_kepler_log) is not available on a split context. Results equal   */
/* those of qym_step on one GPU to rounding: the kick of a row sums the same  */
/* partial slots in the same order, and only which sets take thread-block     */
/* clusters in the Hermite (hence a set's summation order) can differ.       */
/* ------------------------------------------------------------------------ */
#define QYM_PHASE_OPEN    0
#define QYM_PHASE_KICK1   1
#define QYM_PHASE_SEARCH  2
#define QYM_PHASE_KEPLER  3
#define QYM_PHASE_REFINE  4
#define QYM_PHASE_HERMITE 5
#define QYM_PHASE_KICK2   6
#define QYM_PHASE_CLOSE   7

typedef struct qym_split_view {
    int64_t rows, own_lo, own_hi;  /* all rows; the own rows [own_lo, own_hi) */
    double *q, *v;                 /* [3][rows] state (v after the first kick in REFINE) */
    double *q1, *v1;               /* [3][rows] Kepler result / Hermite result */
    double *rH;                    /* [rows] Hill radii of the step */
    float *amag;                   /* [rows] |a| of the last kick (sizes the next search) */
    int32_t *hcost;                /* [rows] Hermite block steps of each row's set */
    int32_t *enc;                  /* [max_enc][2] encounter pairs (i < j) */
    int64_t max_enc;
    int32_t *set_mem;              /* members of the encounter sets, set by set */
    void *stream;                  /* the context's cudaStream_t */
} qym_split_view;

/* The block of bodies of context `rank` of `world` over a system of `rows`
 * rows (star at row 0): rows [*lo, *hi), possibly empty. */
void qym_split_rows(int64_t rows, int32_t rank, int32_t world, int64_t *lo, int64_t *hi);

/* Make ctx (one system; no Kepler solve log) context `rank` of `world`. The
 * kick items are rebuilt for the own rows; the next phase OPEN starts a run. */
qym_status qym_split_init(qym_ctx *ctx, int32_t rank, int32_t world);

/* Enqueue one phase (QYM_PHASE_*) of a step of size tau; last marks the run's
 * last step (CLOSE). QYM_EINVAL for an unknown phase or a context that is
 * not split; CLOSE with last = 1 returns the run's status. */
qym_status qym_split_phase(qym_ctx *ctx, int32_t phase, double tau, int32_t last);

qym_status qym_split_arrays(qym_ctx *ctx, qym_split_view *view);

/* Pairs the own rigorous test found this step (waits for the device). */
qym_status qym_split_encounter_count(qym_ctx *ctx, int64_t *n);

/* This step's encounter pairs from every context (device int32[n][2], i < j):
 * they replace the list and become the step's records (qym_get_encounters). */
qym_status qym_split_import_encounters(qym_ctx *ctx, const int32_t *pairs, int64_t n);

/* After HERMITE: the members of the own sets are set_mem[*first .. *first +
 * *count) (waits for the device). */
qym_status qym_split_owned_members(qym_ctx *ctx, int64_t *first, int64_t *count);

/* ------------------------------------------------------------------------ */
/* Measurement                                                              */
/* ------------------------------------------------------------------------ */

/* Arithmetic peak of the current device, measured: blocks_per_sm x SMs CTAs
 * of 256 threads each run 8 independent chains of `iters` fused
 * multiply-adds (kind 0: FP32 FFMA, 1: packed FP32x2 FFMA2, counted as two
 * lanes each, 2: FP64 DFMA), timed by CUDA events on `stream`. *tflops gets
 * 2 flops per lane-FMA over the elapsed time, *ms (if not NULL) that time.
 * Waits for the launch. These are the denominators of the roofline fractions
 * of the FP32 kick (Sec. 2, Eq. 4: 20 flops per pair by convention) and the
 * FP64 Kepler drift (Appendix); the paper has no such call. QYM_EINVAL for
 * kind outside 0..2, iters < 1 or blocks_per_sm outside 1..8. */
qym_status qym_probe_fma(int32_t kind, int64_t iters, int32_t blocks_per_sm, double *tflops,
                         double *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QYM_H */
