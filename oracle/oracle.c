/*
 * oracle.c -- plain, slow, FP64 CPU reference of the democratic-heliocentric
 * (DH) hybrid symplectic step of Moore & Quillen, "QYMSYM: A GPU-accelerated
 * hybrid symplectic integrator that permits close encounters".
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The CUDA product path never calls it
 * and shares no code, header or table with it.
 *
 * Everything is written for readability: explicit loops, one body at a time,
 * array-of-structures [rows][3] float64, star at row 0 with Q0 = P0 = 0.
 * Compile with -O2 -ffp-contract=off and no fast-math.
 *
 * Paper passages followed (section / equation numbers of the paper):
 *   Sec. 2, Eqs. 1-4   H = H_Dft + H_Kep + H_Int in heliocentric Q, barycentric P
 *   Sec. 2, Eq. 5      step E_Dft(tau/2) E_Int(tau/2) E_Kep(tau) E_Int(tau/2) E_Dft(tau/2)
 *   Sec. 2             star kept at index 0, its mass zeroed in H_Int, restored for energy
 *   Sec. 2.1, Eqs. 6-8 transition function K(y), y = 1.1 q / r_crit - 0.1
 *   Sec. 2.2           Hermite accelerations and jerks with [1 - K + s K'], r_crit (Eq. 9)
 *   Sec. 2.3           the 10-item per-step procedure (hybrid integration)
 *   Sec. 2.4           rigorous encounter test: third-order interpolation of the
 *                      minimum separation vs a_E times the sum of Hill radii
 *   Appendix           universal-variable f and g functions, Stumpff C and S,
 *                      F, F', F'' and the Laguerre iteration (n = 5)
 *
 * Readings of passages that are silent or garbled (each is also listed in the
 * design notes of the repository):
 *   R1 Laguerre update: x <- x - n F / (F' + sgn(F') sqrt|(n-1)^2 F'^2 - n(n-1) F F''|),
 *      evaluated as n (F/F') / (1 + sqrt|(n-1)^2 - n(n-1) (F/F')(F''/F')|).
 *   R2 mu = G m0 (the Kepler term uses the star mass only); sqrt(mu) where the
 *      appendix writes sqrt(mu).
 *   R3 fdot = sqrt(mu) x (alpha x^2 S(alpha x^2) - 1) / (r r0), r = F'(x).
 *   R4 Hermite force and jerk carry an overall minus sign (attraction); the
 *      star jerk term uses s_i0^3.
 *   R5 K, K', K'' are taken with respect to the separation s (chain factor
 *      1.1 / r_crit included); the kick corrections use the unsmoothed q.
 *   R6 Hill radius r_H,i = |Q_i| (m_i / (3 m0))^(1/3), the Hill radius at the
 *      body's heliocentric distance in the state entering the Kepler step
 *      (equal to the semi-major-axis form on circular orbits; the osculating
 *      semi-major axis diverges on near-parabolic orbits).
 *   R7 rigorous test: cubic Hermite interpolant of d^2(t) = |dQ(t)|^2 on
 *      [0, tau] from values and slopes at both ends; the minimum over [0, tau]
 *      (clamped at 0) is compared with (a_E (r_H,i + r_H,j))^2.
 *   R9 Hermite: 4th-order predictor / evaluate / corrector (PEC) of Makino &
 *      Aarseth (1992) with individual block time steps: Aarseth criterion with
 *      eta, start-up step eta_s |a| / |adot|, each rounded down to tau / 2^k;
 *      a step may double only on a commensurate block time.
 *   R10 the Hermite integration starts from (q0, v0) after the first kick and
 *      the K correction.
 *   R12 Stumpff series used for |y| < 0.1, summed to the y^8 term.
 *   R13 Kepler iteration stops when |F| <= 1e-14 times the sum of the
 *      magnitudes of F's terms at an evaluated x. A step below 2^-50 |x| (or
 *      a bracket that narrow) is followed by one more evaluation at the new
 *      x; if that still misses 1e-14, the iteration stops there anyway, at
 *      whichever of the last two points has the smaller residual: the root
 *      is then known to rounding, and on orbits with r1 >> r0 no double
 *      need meet 1e-14 (F moves by F' = r1 per unit of x).
 *   R14 standard starting guess x0 = sqrt(mu) dt / r0; the paper's x0 = r0 is
 *      kept as a separate guess mode.
 *   R15 the iteration is kept inside the bracket [0, sqrt(mu) dt / r_p]
 *      (r_p the periapsis distance; F' = r >= r_p; for unbound orbits also
 *      sqrt(-alpha) |x| <= 700, beyond which C and S overflow), falling back to bisection
 *      when a step leaves it, does not halve the previous step, or F
 *      overflows; the residual test of R13 is taken against the sum of the
 *      magnitudes of F's terms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads for the loops over bodies (the all-pairs kick, the Kepler drift of
 * each body, the all-pairs encounter test), 1 by default. Every body's result
 * is computed by one thread in the same order whatever the count, and the
 * encounter list is assembled in row order, so results are bit-identical for
 * any count. Only the all-core CPU baseline sets it; built without OpenMP the
 * pragmas are ignored and the loops run on one thread. */
static int g_threads = 1;
void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return g_threads; }

#define OR_PI 3.14159265358979323846

typedef struct {
    double G, a_E, a_H, eps_H, eta, eta_s;
    int32_t solver;            /* 0 Laguerre n=5 (Appendix), 1 Newton */
    int32_t guess;             /* 0 sqrt(mu) dt / r0, 1 x0 = r0 (Appendix) */
    int32_t encounters;        /* 0 plain DH step, 1 hybrid step with encounters */
    int32_t max_kepler_iter;
    int64_t max_hermite_steps;
    int32_t whole_hermite;     /* 1: Sec. 2.3, last paragraph (see or_step) */
    double planet_mass;        /* planets: m >= planet_mass * m0 */
} or_params;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* Appendix: Stumpff functions C(y), S(y) (Eqs. 2.40 of Prussing)      */
/* ------------------------------------------------------------------ */
void or_stumpff(double y, double *C, double *S)
{
    if (fabs(y) < 0.1) {
        /* C = 1/2! - y/4! + y^2/6! - ...,  S = 1/3! - y/5! + y^2/7! - ... */
        double c = 0.0, s = 0.0, term_c = 0.5, term_s = 1.0 / 6.0;
        for (int k = 0; k <= 8; ++k) {
            c += term_c;
            s += term_s;
            term_c *= -y / ((2.0 * k + 3.0) * (2.0 * k + 4.0));
            term_s *= -y / ((2.0 * k + 4.0) * (2.0 * k + 5.0));
        }
        *C = c;
        *S = s;
    } else if (y > 0.0) {
        double sy = sqrt(y);
        *C = (1.0 - cos(sy)) / y;
        *S = (sy - sin(sy)) / (sy * sy * sy);
    } else {
        double sy = sqrt(-y);
        *C = (cosh(sy) - 1.0) / (-y);
        *S = (sinh(sy) - sy) / (sy * sy * sy);
    }
}

/* ------------------------------------------------------------------ */
/* Appendix: F(x), F'(x), F''(x) of the universal Kepler equation       */
/*   sig = (r0 . v0) / sqrt(mu)                                        */
/* ------------------------------------------------------------------ */
void or_kepler_F(double x, double sqmu, double dt, double r0, double sig, double alpha,
                 double *F, double *Fp, double *Fpp)
{
    double y = alpha * x * x, C, S;
    or_stumpff(y, &C, &S);
    double b = 1.0 - r0 * alpha;
    *F = -sqmu * dt + sig * x * x * C + b * x * x * x * S + r0 * x;
    *Fp = sig * x * (1.0 - y * S) + b * x * x * C + r0;
    *Fpp = sig * (1.0 - y * C) + b * x * (1.0 - y * S);
}

int or_kepler_solve_br(double sqmu, double dt, double r0, double sig, double alpha, int solver,
                       int max_iter, double lo, double hi, double *x_io, int32_t *iters);

/* Solve F(x) = 0 from x (in/out). solver 0: Laguerre n = 5 (R1); 1: Newton.
 * F is increasing (F' = r > 0), so the root is unique and lies in the
 * bracket [lo, hi] passed in (R15); a step that leaves the bracket or lands
 * where F is not finite (C, S overflow on strongly hyperbolic orbits) is
 * replaced by bisection, and the bracket shrinks with every evaluation.
 * Returns 0 on convergence (R13), 1 when max_iter evaluations did not. */
int or_kepler_solve(double sqmu, double dt, double r0, double sig, double alpha,
                    int solver, int max_iter, double *x_io, int32_t *iters)
{
    return or_kepler_solve_br(sqmu, dt, r0, sig, alpha, solver, max_iter, -INFINITY, INFINITY,
                              x_io, iters);
}

int or_kepler_solve_br(double sqmu, double dt, double r0, double sig, double alpha, int solver,
                       int max_iter, double lo, double hi, double *x_io, int32_t *iters)
{
    const double n = 5.0;
    double x = *x_io;
    if (!(x >= lo && x <= hi)) x = (isfinite(lo) && isfinite(hi)) ? 0.5 * (lo + hi) : x;
    double dx_old = INFINITY;
    /* after a step at the rounding level: the point it started from and its
     * relative residual */
    int settle = 0;
    double x_prev = x, res_prev = INFINITY;
    int it;
    for (it = 0; it < max_iter; ++it) {
        double F, Fp, Fpp;
        or_kepler_F(x, sqmu, dt, r0, sig, alpha, &F, &Fp, &Fpp);
        if (!isfinite(F) || !isfinite(Fp) || !isfinite(Fpp)) {
            /* beyond the representable range: the root is below |x| */
            if (x > 0.0) hi = x; else lo = x;
            x = 0.5 * (lo + hi);
            continue;
        }
        if (F < 0.0) lo = x; else hi = x;
        /* residual against the rounding floor of F: the sum of its terms */
        double y = alpha * x * x, C, S;
        or_stumpff(y, &C, &S);
        double scale = fabs(sqmu * dt) + fabs(sig * x * x * C) +
                       fabs((1.0 - r0 * alpha) * x * x * x * S) + r0 * fabs(x);
        if (fabs(F) <= 1e-14 * scale) {
            *x_io = x;
            *iters = it;
            return 0;
        }
        if (settle) {
            /* evaluated after a rounding-level step and still above 1e-14:
             * keep the better of the last two points (R13) */
            *x_io = fabs(F) / scale <= res_prev ? x : x_prev;
            *iters = it;
            return 0;
        }
        double dx;
        if (solver == 0) {
            /* R1 with F' factored out of the square root (the same value; F'^2
             * itself overflows near the top of an unbound orbit's bracket) */
            double rf = F / Fp, rpp = Fpp / Fp;
            double sq = sqrt(fabs((n - 1.0) * (n - 1.0) - n * (n - 1.0) * rf * rpp));
            dx = n * rf / (1.0 + sq);
        } else {
            dx = F / Fp;
        }
        double xn = x - dx;
        int bracketed = isfinite(lo) && isfinite(hi);
        /* bisect when the step is not finite, leaves the bracket, or does not
         * at least halve the previous step (slow approach along the
         * exponential flank of F on unbound orbits) */
        if (bracketed && (!isfinite(dx) || !(xn >= lo && xn <= hi) || fabs(dx) > 0.5 * fabs(dx_old))) {
            xn = 0.5 * (lo + hi);
            dx = x - xn;
        }
        dx_old = dx;
        if (fabs(dx) <= 0x1p-50 * fabs(xn) || (isfinite(lo) && isfinite(hi) && hi - lo <= 0x1p-50 * fabs(xn))) {
            settle = 1;
            x_prev = x;
            res_prev = fabs(F) / scale;
        }
        x = xn;
    }
    *x_io = x;
    *iters = it;
    return 1;
}

/* Appendix: advance one body on its Kepler orbit about the star for dt with
 * universal-variable f and g functions. x_guess is used when guess == 2.
 * Returns the solver status; writes x and the iteration count. */
int or_kepler_body(const double *q0, const double *v0, double *q1, double *v1, double mu,
                   double dt, int solver, int guess, double x_guess, int max_iter,
                   double *x_out, int32_t *iters_out)
{
    double sqmu = sqrt(mu);
    double r0 = sqrt(dot3(q0, q0));
    double v2 = dot3(v0, v0);
    double alpha = 2.0 / r0 - v2 / mu;
    double sig = dot3(q0, v0) / sqmu;
    double x;
    if (guess == 0)
        x = sqmu * dt / r0;
    else if (guess == 1)
        x = r0;
    else
        x = x_guess;
    /* bracket (R15): F(0) = -sqrt(mu) dt and F' = r >= r_p (periapsis
     * distance), so the root lies between 0 and sqrt(mu) dt / r_p */
    double hv[3] = {q0[1] * v0[2] - q0[2] * v0[1], q0[2] * v0[0] - q0[0] * v0[2],
                    q0[0] * v0[1] - q0[1] * v0[0]};
    double p = dot3(hv, hv) / mu;
    double ecc = sqrt(fmax(0.0, 1.0 - p * alpha));
    double rp = p / (1.0 + ecc);
    double lo = -INFINITY, hi = INFINITY;
    if (rp > 0.0) {
        /* widened by 1e-12: r_p itself carries rounding */
        double xb = sqmu * dt / rp * (1.0 + 1e-12);
        if (dt >= 0.0) { lo = 0.0; hi = xb; } else { lo = xb; hi = 0.0; }
    }
    if (alpha < 0.0) {
        /* unbound: beyond sqrt(-alpha) |x| = 700 the position would be
         * ~e^700 from the star (C, S overflow first) */
        double xm = 700.0 / sqrt(-alpha);
        if (dt >= 0.0) { lo = fmax(lo, 0.0); hi = fmin(hi, xm); }
        else { lo = fmax(lo, -xm); hi = fmin(hi, 0.0); }
    }
    int32_t it = 0;
    int st = or_kepler_solve_br(sqmu, dt, r0, sig, alpha, solver, max_iter, lo, hi, &x, &it);
    if (st != 0 && guess == 2) {
        /* fallback: Laguerre from the standard guess */
        int32_t it2 = 0;
        x = sqmu * dt / r0;
        st = or_kepler_solve_br(sqmu, dt, r0, sig, alpha, 0, max_iter, lo, hi, &x, &it2);
        it += it2;
    }
    double y = alpha * x * x, C, S;
    or_stumpff(y, &C, &S);
    double f = 1.0 - x * x / r0 * C;
    double g = dt - x * x * x / sqmu * S;
    for (int k = 0; k < 3; ++k) q1[k] = f * q0[k] + g * v0[k];
    double r = sqrt(dot3(q1, q1));
    double fdot = sqmu * x * (y * S - 1.0) / (r * r0);
    double gdot = 1.0 - x * x / r * C;
    for (int k = 0; k < 3; ++k) v1[k] = fdot * q0[k] + gdot * v0[k];
    if (x_out) *x_out = x;
    if (iters_out) *iters_out = it;
    return st;
}

/* E_Kep for bodies [0, n) (no star row). Returns the number of bodies whose
 * iteration did not converge. */
int64_t or_kepler_drift(int64_t n, const double *q0, const double *v0, double *q1, double *v1,
                        double mu, double dt, int32_t solver, int32_t guess,
                        const double *x_guess, int32_t max_iter, double *x_out, int32_t *iters_out)
{
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : bad) num_threads(g_threads) if (g_threads > 1)
    for (int64_t i = 0; i < n; ++i) {
        double x;
        int32_t it;
        int st = or_kepler_body(q0 + 3 * i, v0 + 3 * i, q1 + 3 * i, v1 + 3 * i, mu, dt, solver,
                                guess, x_guess ? x_guess[i] : 0.0, max_iter, &x, &it);
        if (x_out) x_out[i] = x;
        if (iters_out) iters_out[i] = it;
        if (st) ++bad;
    }
    return bad;
}

/* Relative residual |F(x)| / (sum of the absolute values of the terms of F)
 * of x as a root of the universal Kepler equation (Appendix) for bodies
 * [0, n) with states q0, v0 ([n][3]) about a star of parameter mu. */
void or_kepler_residuals(int64_t n, const double *q0, const double *v0, double mu, double dt,
                         const double *x, double *res)
{
    double sqmu = sqrt(mu);
    for (int64_t i = 0; i < n; ++i) {
        const double *q = q0 + 3 * i, *v = v0 + 3 * i;
        double r0 = sqrt(dot3(q, q));
        double alpha = 2.0 / r0 - dot3(v, v) / mu;
        double sig = dot3(q, v) / sqmu;
        double F, Fp, Fpp, C, S;
        or_kepler_F(x[i], sqmu, dt, r0, sig, alpha, &F, &Fp, &Fpp);
        or_stumpff(alpha * x[i] * x[i], &C, &S);
        double xx = x[i];
        double scale = fabs(sqmu * dt) + fabs(sig * xx * xx * C) +
                       fabs((1.0 - r0 * alpha) * xx * xx * xx * S) + r0 * fabs(xx);
        res[i] = fabs(F) / scale;
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 2: E_Dft -- sum of barycentric momenta, uniform shift of Q      */
/* ------------------------------------------------------------------ */
void or_momentum(int64_t rows, const double *m, const double *v, double *S)
{
    S[0] = S[1] = S[2] = 0.0;
    for (int64_t i = 1; i < rows; ++i)
        for (int k = 0; k < 3; ++k) S[k] += m[i] * v[3 * i + k];
}

void or_drift(int64_t rows, const double *m, double *q, const double *v, double dt)
{
    double S[3];
    or_momentum(rows, m, v, S);
    for (int64_t i = 1; i < rows; ++i)
        for (int k = 0; k < 3; ++k) q[3 * i + k] += dt * S[k] / m[0];
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eq. 4: E_Int acceleration, star excluded (its mass zeroed)   */
/*   a_i = - sum_{j>=1, j!=i} G m_j (Q_i - Q_j) / |Q_i - Q_j|^3         */
/* ------------------------------------------------------------------ */
void or_accel_row(int64_t rows, const double *m, const double *q, double G, int64_t i, double *a)
{
    a[0] = a[1] = a[2] = 0.0;
    for (int64_t j = 1; j < rows; ++j) {
        if (j == i) continue;
        double d[3] = {q[3 * i] - q[3 * j], q[3 * i + 1] - q[3 * j + 1], q[3 * i + 2] - q[3 * j + 2]};
        double r2 = dot3(d, d);
        double r = sqrt(r2);
        double w = G * m[j] / (r2 * r);
        for (int k = 0; k < 3; ++k) a[k] -= w * d[k];
    }
}

void or_accel_int(int64_t rows, const double *m, const double *q, double G, double *a)
{
    a[0] = a[1] = a[2] = 0.0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) if (g_threads > 1)
    for (int64_t i = 1; i < rows; ++i) or_accel_row(rows, m, q, G, i, a + 3 * i);
}

/* accelerations of selected rows only (sampled parity at large sizes) */
void or_accel_rows(int64_t rows, const double *m, const double *q, double G, int64_t nsel,
                   const int64_t *sel, double *a)
{
    for (int64_t k = 0; k < nsel; ++k) or_accel_row(rows, m, q, G, sel[k], a + 3 * k);
}

void or_kick(int64_t rows, const double *m, const double *q, double *v, double G, double dt)
{
    double *a = (double *)malloc(sizeof(double) * 3 * rows);
    or_accel_int(rows, m, q, G, a);
    for (int64_t i = 1; i < rows; ++i)
        for (int k = 0; k < 3; ++k) v[3 * i + k] += dt * a[3 * i + k];
    free(a);
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eqs. 2-4: total energy H_Dft + H_Kep + H_Int (per unit of    */
/* the DH variables: P_i = m_i v_i), star mass restored for the sum     */
/* ------------------------------------------------------------------ */
double or_energy(int64_t rows, const double *m, const double *q, const double *v, double G)
{
    double S[3];
    or_momentum(rows, m, v, S);
    double E = dot3(S, S) / (2.0 * m[0]);
    for (int64_t i = 1; i < rows; ++i) {
        E += 0.5 * m[i] * dot3(v + 3 * i, v + 3 * i);
        E -= G * m[0] * m[i] / sqrt(dot3(q + 3 * i, q + 3 * i));
    }
    /* pair terms summed per row first: added one by one to E, terms of
     * light pairs (m_i m_j / r ~ 1e-21) fall below half an ulp of E and vanish */
    for (int64_t i = 1; i < rows; ++i) {
        double row = 0.0;
        for (int64_t j = i + 1; j < rows; ++j) {
            double d[3] = {q[3 * i] - q[3 * j], q[3 * i + 1] - q[3 * j + 1], q[3 * i + 2] - q[3 * j + 2]};
            row += m[j] / sqrt(dot3(d, d));
        }
        E -= G * m[i] * row;
    }
    return E;
}

/* ------------------------------------------------------------------ */
/* Sec. 2: heliocentric velocities <-> barycentric velocities (P/m)     */
/* ------------------------------------------------------------------ */
void or_helio_to_dh(int64_t rows, const double *m, double *v)
{
    double mt = m[0], s[3] = {0, 0, 0};
    for (int64_t i = 1; i < rows; ++i) {
        mt += m[i];
        for (int k = 0; k < 3; ++k) s[k] += m[i] * v[3 * i + k];
    }
    for (int64_t i = 1; i < rows; ++i)
        for (int k = 0; k < 3; ++k) v[3 * i + k] -= s[k] / mt;
    v[0] = v[1] = v[2] = 0.0;
}

void or_dh_to_helio(int64_t rows, const double *m, double *v)
{
    double S[3];
    or_momentum(rows, m, v, S);
    /* star barycentric velocity V0 = -S / m0; heliocentric v_i = V_i - V0 */
    for (int64_t i = 1; i < rows; ++i)
        for (int k = 0; k < 3; ++k) v[3 * i + k] += S[k] / m[0];
    v[0] = v[1] = v[2] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2 (Eq. 9) and reading R6: Hill radii at the current distance  */
/* ------------------------------------------------------------------ */
void or_hill_radii(int64_t rows, const double *m, const double *q, const double *v, double G,
                   double *rH)
{
    (void)v;
    (void)G;
    rH[0] = 0.0;
    for (int64_t i = 1; i < rows; ++i) {
        double r = sqrt(dot3(q + 3 * i, q + 3 * i));
        rH[i] = r * cbrt(m[i] / (3.0 * m[0]));
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 2.4, reading R7: minimum over [0, tau] of the cubic that         */
/* interpolates d^2(t) = |dQ(t)|^2 from its values and slopes at 0, tau */
/* ------------------------------------------------------------------ */
double or_pair_dmin2(const double *dq0, const double *dv0, const double *dq1, const double *dv1,
                     double tau)
{
    double d0 = dot3(dq0, dq0);
    double d1 = dot3(dq1, dq1);
    double s0 = 2.0 * dot3(dq0, dv0) * tau;   /* d(d^2)/du at u = 0, u = t / tau */
    double s1 = 2.0 * dot3(dq1, dv1) * tau;   /* d(d^2)/du at u = 1 */
    /* p(u) = c0 + c1 u + c2 u^2 + c3 u^3 (cubic Hermite basis expanded) */
    double c0 = d0;
    double c1 = s0;
    double c2 = 3.0 * (d1 - d0) - 2.0 * s0 - s1;
    double c3 = 2.0 * (d0 - d1) + s0 + s1;
    double best = d0 < d1 ? d0 : d1;
    /* stationary points: 3 c3 u^2 + 2 c2 u + c1 = 0, roots from the
     * cancellation-free form w = -(B + sgn(B) sqrt(disc)) / 2, u = w/A, Cc/w
     * (c3 is ~0 whenever the relative motion is nearly straight) */
    double A = 3.0 * c3, B = 2.0 * c2, Cc = c1;
    double u[2];
    int nu = 0;
    double disc = B * B - 4.0 * A * Cc;
    if (disc >= 0.0) {
        double w = -0.5 * (B + (B >= 0.0 ? 1.0 : -1.0) * sqrt(disc));
        if (A != 0.0) u[nu++] = w / A;
        if (w != 0.0) u[nu++] = Cc / w;
    }
    for (int k = 0; k < nu; ++k) {
        if (u[k] > 0.0 && u[k] < 1.0) {
            double p = c0 + u[k] * (c1 + u[k] * (c2 + u[k] * c3));
            if (p < best) best = p;
        }
    }
    return best > 0.0 ? best : 0.0;
}

static void pair_diffs(const double *q0, const double *v0, const double *q1, const double *v1,
                       int64_t i, int64_t j, double *dq0, double *dv0, double *dq1, double *dv1)
{
    for (int k = 0; k < 3; ++k) {
        dq0[k] = q0[3 * i + k] - q0[3 * j + k];
        dv0[k] = v0[3 * i + k] - v0[3 * j + k];
        dq1[k] = q1[3 * i + k] - q1[3 * j + k];
        dv1[k] = v1[3 * i + k] - v1[3 * j + k];
    }
}

/* Sec. 2.4 over ALL pairs 1 <= i < j (brute force; no crude pre-filter).
 * Writes up to cap pairs (i, j), i < j, in ascending (i, j) order, with their
 * d_min^2 and threshold^2; returns the number found. */
int64_t or_encounters_near(int64_t rows, const double *q0, const double *v0, const double *q1,
                           const double *v1, const double *rH, double tau, double a_E,
                           int64_t *pairs, double *d2, double *thr2, int64_t cap, double band,
                           int64_t *near, double *near_d2, int64_t near_cap, int64_t *near_count);

int64_t or_encounters(int64_t rows, const double *q0, const double *v0, const double *q1,
                      const double *v1, const double *rH, double tau, double a_E, int64_t *pairs,
                      double *d2, double *thr2, int64_t cap)
{
    return or_encounters_near(rows, q0, v0, q1, v1, rH, tau, a_E, pairs, d2, thr2, cap, 0.0, NULL,
                              NULL, 0, NULL);
}

/* as or_encounters; in addition, unflagged pairs with threshold^2 <= d^2 <
 * threshold^2 (1 + band) ("near misses", for tests) go to near[] with their
 * (d^2, threshold^2) */
/* flagged pairs and near misses of a range of rows, in (i, j) order */
typedef struct {
    int64_t *pairs, *near;
    double *d2, *thr2, *near_d2;
    int64_t cap, cnt, near_cap, near_cnt;
    int want_near;
} enc_out;

static void enc_push(int64_t **p, double **x, int64_t *cap, int64_t n)
{
    if (n < *cap) return;
    *cap = 2 * *cap + 64;
    *p = (int64_t *)realloc(*p, sizeof(int64_t) * 2 * *cap);
    *x = (double *)realloc(*x, sizeof(double) * 2 * *cap);
}

/* row i against every j > i: flagged pairs into o (all of them counted,
 * the first o->cap written), near misses likewise */
static void enc_row(int64_t rows, const double *q0, const double *v0, const double *q1,
                    const double *v1, const double *rH, double tau, double a_E, double band,
                    int64_t i, enc_out *o)
{
    for (int64_t j = i + 1; j < rows; ++j) {
        double dq0[3], dv0[3], dq1[3], dv1[3];
        pair_diffs(q0, v0, q1, v1, i, j, dq0, dv0, dq1, dv1);
        double R = a_E * (rH[i] + rH[j]);
        double dm = or_pair_dmin2(dq0, dv0, dq1, dv1, tau);
        if (dm < R * R) {
            if (o->cnt < o->cap) {
                o->pairs[2 * o->cnt] = i;
                o->pairs[2 * o->cnt + 1] = j;
                if (o->d2) o->d2[o->cnt] = dm;
                if (o->thr2) o->thr2[o->cnt] = R * R;
            }
            ++o->cnt;
        } else if (o->want_near && dm < R * R * (1.0 + band)) {
            if (o->near_cnt < o->near_cap) {
                o->near[2 * o->near_cnt] = i;
                o->near[2 * o->near_cnt + 1] = j;
                o->near_d2[2 * o->near_cnt] = dm;
                o->near_d2[2 * o->near_cnt + 1] = R * R;
            }
            ++o->near_cnt;
        }
    }
}

int64_t or_encounters_near(int64_t rows, const double *q0, const double *v0, const double *q1,
                           const double *v1, const double *rH, double tau, double a_E,
                           int64_t *pairs, double *d2, double *thr2, int64_t cap, double band,
                           int64_t *near, double *near_d2, int64_t near_cap, int64_t *near_count)
{
    enc_out o = {pairs, near, d2, thr2, near_d2, cap, 0, near_cap,
                 near_count ? *near_count : 0, near_count != NULL};
    if (g_threads <= 1) {
        for (int64_t i = 1; i < rows; ++i) enc_row(rows, q0, v0, q1, v1, rH, tau, a_E, band, i, &o);
        if (near_count) *near_count = o.near_cnt;
        return o.cnt;
    }
    /* several threads: chunks of rows with equal pair counts, each into
     * buffers of its own, then appended in row order */
    enum { NCH = 256 };
    int64_t bound[NCH + 1];
    double tot = 0.5 * (double)(rows - 1) * (double)(rows - 2);
    bound[0] = 1;
    for (int c = 1; c < NCH; ++c) {
        /* rows [1, b) hold about c / NCH of the pairs */
        double f = (double)c / NCH, n1 = (double)(rows - 1);
        double b = 1.0 + n1 - sqrt(n1 * n1 - 2.0 * f * tot);
        int64_t bi = (int64_t)b;
        if (bi < bound[c - 1]) bi = bound[c - 1];
        if (bi > rows) bi = rows;
        bound[c] = bi;
    }
    bound[NCH] = rows;
    enc_out part[NCH];
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int c = 0; c < NCH; ++c) {
        int64_t pc = 64, nc = 64;
        enc_out *w = &part[c];
        w->pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * pc);
        w->d2 = (double *)malloc(sizeof(double) * 2 * pc);
        w->thr2 = NULL;
        w->near = (int64_t *)malloc(sizeof(int64_t) * 2 * nc);
        w->near_d2 = (double *)malloc(sizeof(double) * 2 * nc);
        w->cnt = w->near_cnt = 0;
        w->want_near = near_count != NULL;
        for (int64_t i = bound[c]; i < bound[c + 1]; ++i) {
            /* room for the row's every pair is not known in advance: grow
             * the chunk's buffers between rows (d2 holds d^2 and thr^2) */
            enc_out r = {NULL, NULL, NULL, NULL, NULL, 0, 0, 0, 0, w->want_near};
            int64_t rp = 16, rn = 16;
            r.pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * rp);
            r.d2 = (double *)malloc(sizeof(double) * rp);
            r.thr2 = (double *)malloc(sizeof(double) * rp);
            r.near = (int64_t *)malloc(sizeof(int64_t) * 2 * rn);
            r.near_d2 = (double *)malloc(sizeof(double) * 2 * rn);
            r.cap = rp;
            r.near_cap = rn;
            enc_row(rows, q0, v0, q1, v1, rH, tau, a_E, band, i, &r);
            if (r.cnt > rp || r.near_cnt > rn) {
                /* more than fit: the row once more with room for all */
                rp = r.cnt > rp ? r.cnt : rp;
                rn = r.near_cnt > rn ? r.near_cnt : rn;
                r.pairs = (int64_t *)realloc(r.pairs, sizeof(int64_t) * 2 * rp);
                r.d2 = (double *)realloc(r.d2, sizeof(double) * rp);
                r.thr2 = (double *)realloc(r.thr2, sizeof(double) * rp);
                r.near = (int64_t *)realloc(r.near, sizeof(int64_t) * 2 * rn);
                r.near_d2 = (double *)realloc(r.near_d2, sizeof(double) * 2 * rn);
                r.cap = rp;
                r.near_cap = rn;
                r.cnt = r.near_cnt = 0;
                enc_row(rows, q0, v0, q1, v1, rH, tau, a_E, band, i, &r);
            }
            for (int64_t k = 0; k < r.cnt; ++k) {
                enc_push(&w->pairs, &w->d2, &pc, w->cnt);
                w->pairs[2 * w->cnt] = r.pairs[2 * k];
                w->pairs[2 * w->cnt + 1] = r.pairs[2 * k + 1];
                w->d2[2 * w->cnt] = r.d2[k];
                w->d2[2 * w->cnt + 1] = r.thr2[k];
                ++w->cnt;
            }
            for (int64_t k = 0; k < r.near_cnt; ++k) {
                enc_push(&w->near, &w->near_d2, &nc, w->near_cnt);
                w->near[2 * w->near_cnt] = r.near[2 * k];
                w->near[2 * w->near_cnt + 1] = r.near[2 * k + 1];
                w->near_d2[2 * w->near_cnt] = r.near_d2[2 * k];
                w->near_d2[2 * w->near_cnt + 1] = r.near_d2[2 * k + 1];
                ++w->near_cnt;
            }
            free(r.pairs); free(r.d2); free(r.thr2); free(r.near); free(r.near_d2);
        }
    }
    for (int c = 0; c < NCH; ++c) {
        enc_out *w = &part[c];
        for (int64_t k = 0; k < w->cnt; ++k, ++o.cnt)
            if (o.cnt < o.cap) {
                o.pairs[2 * o.cnt] = w->pairs[2 * k];
                o.pairs[2 * o.cnt + 1] = w->pairs[2 * k + 1];
                if (o.d2) o.d2[o.cnt] = w->d2[2 * k];
                if (o.thr2) o.thr2[o.cnt] = w->d2[2 * k + 1];
            }
        for (int64_t k = 0; k < w->near_cnt; ++k, ++o.near_cnt)
            if (o.want_near && o.near_cnt < o.near_cap) {
                o.near[2 * o.near_cnt] = w->near[2 * k];
                o.near[2 * o.near_cnt + 1] = w->near[2 * k + 1];
                o.near_d2[2 * o.near_cnt] = w->near_d2[2 * k];
                o.near_d2[2 * o.near_cnt + 1] = w->near_d2[2 * k + 1];
            }
        free(w->pairs); free(w->d2); free(w->near); free(w->near_d2);
    }
    if (near_count) *near_count = o.near_cnt;
    return o.cnt;
}

/* rigorous test of selected rows i against all j != i (sampled parity) */
static int64_t enc_rows_serial(int64_t rows, const double *q0, const double *v0, const double *q1,
                               const double *v1, const double *rH, double tau, double a_E,
                               int64_t nsel, const int64_t *sel, int64_t *pairs, double *d2,
                               double *thr2, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t s = 0; s < nsel; ++s) {
        int64_t i = sel[s];
        for (int64_t j = 1; j < rows; ++j) {
            if (j == i) continue;
            double dq0[3], dv0[3], dq1[3], dv1[3];
            int64_t a = i < j ? i : j, b = i < j ? j : i;
            pair_diffs(q0, v0, q1, v1, a, b, dq0, dv0, dq1, dv1);
            double R = a_E * (rH[a] + rH[b]);
            double dm = or_pair_dmin2(dq0, dv0, dq1, dv1, tau);
            if (dm < R * R) {
                if (cnt < cap) {
                    pairs[2 * cnt] = a;
                    pairs[2 * cnt + 1] = b;
                    if (d2) d2[cnt] = dm;
                    if (thr2) thr2[cnt] = R * R;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

int64_t or_encounters_rows(int64_t rows, const double *q0, const double *v0, const double *q1,
                           const double *v1, const double *rH, double tau, double a_E, int64_t nsel,
                           const int64_t *sel, int64_t *pairs, double *d2, double *thr2, int64_t cap)
{
    if (g_threads <= 1 || nsel < 2)
        return enc_rows_serial(rows, q0, v0, q1, v1, rH, tau, a_E, nsel, sel, pairs, d2, thr2, cap);
    /* several threads: each selected row counted, then written at its offset
     * (the same pairs in the same order as one thread) */
    int64_t *off = (int64_t *)calloc(nsel + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int64_t s = 0; s < nsel; ++s)
        off[s + 1] = enc_rows_serial(rows, q0, v0, q1, v1, rH, tau, a_E, 1, sel + s, NULL, NULL,
                                     NULL, 0);
    for (int64_t s = 0; s < nsel; ++s) off[s + 1] += off[s];
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
    for (int64_t s = 0; s < nsel; ++s) {
        int64_t room = cap - off[s];
        if (room <= 0) continue;
        enc_rows_serial(rows, q0, v0, q1, v1, rH, tau, a_E, 1, sel + s, pairs + 2 * off[s],
                        d2 ? d2 + off[s] : NULL, thr2 ? thr2 + off[s] : NULL, room);
    }
    int64_t total = off[nsel];
    free(off);
    return total;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3 item 4: non-intersecting encounter sets (connected          */
/* components of the pair graph) and r_crit (Eq. 9) per set             */
/* ------------------------------------------------------------------ */
static int64_t uf_find(int64_t *parent, int64_t x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/* set_of[rows]: set id or -1. Sets are numbered by ascending smallest
 * member; members ascending within a set. Returns the number of sets. */
int64_t or_sets(int64_t rows, int64_t npairs, const int64_t *pairs, const double *rH, double a_H,
                int64_t *set_of, int64_t *set_start, int64_t *members, double *rcrit)
{
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * rows);
    for (int64_t i = 0; i < rows; ++i) parent[i] = i;
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t a = uf_find(parent, pairs[2 * p]), b = uf_find(parent, pairs[2 * p + 1]);
        if (a == b) continue;
        if (a < b) parent[b] = a; else parent[a] = b;   /* root = smallest index */
    }
    char *inv = (char *)calloc(rows, 1);
    for (int64_t p = 0; p < 2 * npairs; ++p) inv[pairs[p]] = 1;
    int64_t nsets = 0;
    for (int64_t i = 0; i < rows; ++i) set_of[i] = -1;
    for (int64_t i = 0; i < rows; ++i)
        if (inv[i] && uf_find(parent, i) == i) set_of[i] = nsets++;
    for (int64_t i = 0; i < rows; ++i)
        if (inv[i]) set_of[i] = set_of[uf_find(parent, i)];
    /* counting sort by set id, stable in particle index */
    for (int64_t s = 0; s <= nsets; ++s) set_start[s] = 0;
    for (int64_t i = 0; i < rows; ++i)
        if (set_of[i] >= 0) set_start[set_of[i] + 1]++;
    for (int64_t s = 0; s < nsets; ++s) set_start[s + 1] += set_start[s];
    int64_t *fill = (int64_t *)calloc(nsets + 1, sizeof(int64_t));
    for (int64_t i = 0; i < rows; ++i)
        if (set_of[i] >= 0) {
            int64_t s = set_of[i];
            members[set_start[s] + fill[s]++] = i;
        }
    for (int64_t s = 0; s < nsets; ++s) {
        double mx = 0.0;
        for (int64_t k = set_start[s]; k < set_start[s + 1]; ++k)
            if (rH[members[k]] > mx) mx = rH[members[k]];
        rcrit[s] = a_H * mx;
    }
    free(fill);
    free(inv);
    free(parent);
    return nsets;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1 and reading R5: K(s), dK/ds, d2K/ds2                       */
/* ------------------------------------------------------------------ */
void or_transition(double s, double rcrit, double *K, double *Kp, double *Kpp)
{
    double y = 1.1 * s / rcrit - 0.1;
    double c = 1.1 / rcrit;
    if (y <= 0.0) {
        *K = 0.0; *Kp = 0.0; *Kpp = 0.0;
    } else if (y >= 1.0) {
        *K = 1.0; *Kp = 0.0; *Kpp = 0.0;
    } else {
        double ph = 0.5 * OR_PI * y;
        *K = sin(ph);
        *Kp = 0.5 * OR_PI * c * cos(ph);
        *Kpp = -(0.5 * OR_PI * c) * (0.5 * OR_PI * c) * sin(ph);
    }
}

/* Sec. 2.2 and Sec. 2.3 items 5 and 7: v_i -= dt * a^(1-K)_i summed over
 * the other members of the set, with
 *   a^(1-K)_ij = -G m_j q_ij / q^3 [1 - K(q) + q K'(q)]                 */
void or_kcorr(int64_t nmem, const int64_t *mem, const double *m, const double *q, double *v,
              double G, double rcrit, double dt)
{
    double *dv = (double *)calloc(3 * nmem, sizeof(double));
    for (int64_t a = 0; a < nmem; ++a) {
        int64_t i = mem[a];
        for (int64_t b = 0; b < nmem; ++b) {
            if (b == a) continue;
            int64_t j = mem[b];
            double d[3] = {q[3 * i] - q[3 * j], q[3 * i + 1] - q[3 * j + 1], q[3 * i + 2] - q[3 * j + 2]};
            double r = sqrt(dot3(d, d));
            double K, Kp, Kpp;
            or_transition(r, rcrit, &K, &Kp, &Kpp);
            double w = -G * m[j] / (r * r * r) * (1.0 - K + r * Kp);
            for (int k = 0; k < 3; ++k) dv[3 * a + k] += w * d[k];
        }
    }
    for (int64_t a = 0; a < nmem; ++a)
        for (int k = 0; k < 3; ++k) v[3 * mem[a] + k] -= dt * dv[3 * a + k];
    free(dv);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: Hermite accelerations and jerks of the set members, star   */
/* fixed at the origin, pair terms weighted by the transition function  */
/* ------------------------------------------------------------------ */
void or_hermite_force(int64_t k, const double *mm, const double *x, const double *u, double G,
                      double m0, double rcrit, double eps, double *a, double *jk)
{
    for (int64_t i = 0; i < k; ++i) {
        double ai[3] = {0, 0, 0}, ji[3] = {0, 0, 0};
        /* star term */
        {
            double s2 = dot3(x + 3 * i, x + 3 * i) + eps * eps;
            double s = sqrt(s2);
            double rv = dot3(x + 3 * i, u + 3 * i);
            double w = -G * m0 / (s2 * s);
            for (int c = 0; c < 3; ++c) {
                ai[c] += w * x[3 * i + c];
                ji[c] += w * (u[3 * i + c] - 3.0 * rv * x[3 * i + c] / s2);
            }
        }
        for (int64_t j = 0; j < k; ++j) {
            if (j == i) continue;
            double d[3], dv[3];
            for (int c = 0; c < 3; ++c) {
                d[c] = x[3 * i + c] - x[3 * j + c];
                dv[c] = u[3 * i + c] - u[3 * j + c];
            }
            double s2 = dot3(d, d) + eps * eps;
            double s = sqrt(s2);
            double K, Kp, Kpp;
            or_transition(s, rcrit, &K, &Kp, &Kpp);
            double br = 1.0 - K + s * Kp;
            double rv = dot3(d, dv);
            double w = -G * mm[j] / (s2 * s);
            for (int c = 0; c < 3; ++c) {
                ai[c] += w * br * d[c];
                ji[c] += w * (rv * d[c] * Kpp + (dv[c] - 3.0 * rv * d[c] / s2) * br);
            }
        }
        for (int c = 0; c < 3; ++c) {
            a[3 * i + c] = ai[c];
            jk[3 * i + c] = ji[c];
        }
    }
}

static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Sec. 2.2 and reading R9: integrate the members of one set over tau with
 * the 4th-order Hermite scheme of Makino & Aarseth (1992), individual block
 * time steps (no Ahmad-Cohen neighbour scheme). Time runs in integer ticks of
 * |tau| / 2^48; member i steps with dt_i = |tau| 2^-k_i, k_i from the
 * Aarseth criterion (eta; eta_s at start-up) rounded down to a power of two.
 * At each block time all members are predicted, the members whose step ends
 * there are evaluated and corrected, and their new level may drop by one (a
 * doubled step) only when the block time is a multiple of the doubled step.
 * q, v are full-system arrays; members are read and written in place.
 * Returns 0, or 1 when max_steps block steps were taken before tau. */
#define OR_KMAX 48

static int or_level(double dt_c, double T)
{
    /* smallest k with T 2^-k <= dt_c, in [0, OR_KMAX] */
    if (!(dt_c > 0.0)) return OR_KMAX;
    int k = 0;
    double d = T;
    while (d > dt_c && k < OR_KMAX) {
        d *= 0.5;
        ++k;
    }
    return k;
}

static double or_aarseth(const double *a, const double *j, const double *a2, const double *a3,
                         double eta, double cap)
{
    double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    double den = nj * n3 + n2 * n2;
    if (!(den > 0.0)) return cap;
    return sqrt(eta * (na * n2 + nj * nj) / den);
}

int or_hermite_set(int64_t k, const int64_t *mem, const double *m, double m0, double *q, double *v,
                   double G, double rcrit, double eps, double eta, double eta_s, double tau,
                   int64_t max_steps, int64_t *steps_out)
{
    size_t b3 = sizeof(double) * 3 * k;
    double *mm = (double *)malloc(sizeof(double) * k);
    double *x = (double *)malloc(b3), *u = (double *)malloc(b3);
    double *xp = (double *)malloc(b3), *up = (double *)malloc(b3);
    double *a0 = (double *)malloc(b3), *j0 = (double *)malloc(b3);
    double *a1 = (double *)malloc(b3), *j1 = (double *)malloc(b3);
    int64_t *ti = (int64_t *)malloc(sizeof(int64_t) * k);
    int *lev = (int *)malloc(sizeof(int) * k);
    for (int64_t i = 0; i < k; ++i) {
        mm[i] = m[mem[i]];
        for (int c = 0; c < 3; ++c) {
            x[3 * i + c] = q[3 * mem[i] + c];
            u[3 * i + c] = v[3 * mem[i] + c];
        }
    }
    const double T = fabs(tau), sg = tau >= 0.0 ? 1.0 : -1.0;
    const int64_t TT = (int64_t)1 << OR_KMAX;      /* tau in ticks */
    const double tick = T / (double)TT;
    or_hermite_force(k, mm, x, u, G, m0, rcrit, eps, a0, j0);
    /* start-up levels from eta_s |a| / |adot| */
    for (int64_t i = 0; i < k; ++i) {
        double jn = norm3(j0 + 3 * i);
        double dt_c = jn > 0.0 ? eta_s * norm3(a0 + 3 * i) / jn : T;
        lev[i] = or_level(dt_c, T);
        ti[i] = 0;
    }
    int64_t steps = 0;
    int status = 0;
    for (;;) {
        /* next block time: the earliest end of a member's step */
        int64_t tn = TT;
        for (int64_t i = 0; i < k; ++i) {
            int64_t e = ti[i] + ((int64_t)1 << (OR_KMAX - lev[i]));
            if (e < tn) tn = e;
        }
        int done = 1;
        for (int64_t i = 0; i < k; ++i)
            if (ti[i] < TT) done = 0;
        if (done) break;
        if (steps >= max_steps) { status = 1; break; }
        /* predict every member to tn (each from its own time) */
        for (int64_t i = 0; i < k; ++i) {
            double h = sg * (double)(tn - ti[i]) * tick;
            for (int c = 0; c < 3; ++c) {
                int id = 3 * i + c;
                xp[id] = x[id] + h * (u[id] + h * (0.5 * a0[id] + h * j0[id] / 6.0));
                up[id] = u[id] + h * (a0[id] + 0.5 * h * j0[id]);
            }
        }
        or_hermite_force(k, mm, xp, up, G, m0, rcrit, eps, a1, j1);
        /* correct the members whose step ends at tn */
        for (int64_t i = 0; i < k; ++i) {
            int64_t dti = (int64_t)1 << (OR_KMAX - lev[i]);
            if (ti[i] + dti != tn) continue;
            double h = sg * (double)dti * tick;
            double a2[3], a3[3];
            for (int c = 0; c < 3; ++c) {
                int id = 3 * i + c;
                a2[c] = (-6.0 * (a0[id] - a1[id]) - h * (4.0 * j0[id] + 2.0 * j1[id])) / (h * h);
                a3[c] = (12.0 * (a0[id] - a1[id]) + 6.0 * h * (j0[id] + j1[id])) / (h * h * h);
                x[id] = xp[id] + h * h * h * h * (a2[c] / 24.0 + h * a3[c] / 120.0);
                u[id] = up[id] + h * h * h * (a2[c] / 6.0 + h * a3[c] / 24.0);
                a2[c] += h * a3[c];
                a0[id] = a1[id];
                j0[id] = j1[id];
            }
            ti[i] = tn;
            int kn = or_level(or_aarseth(a1 + 3 * i, j1 + 3 * i, a2, a3, eta, T), T);
            if (kn < lev[i]) {
                /* a larger step: one level at a time, on a commensurate time */
                int up1 = lev[i] - 1;
                kn = (tn % ((int64_t)1 << (OR_KMAX - up1)) == 0) ? up1 : lev[i];
            }
            lev[i] = kn;
        }
        ++steps;
    }
    for (int64_t i = 0; i < k; ++i)
        for (int c = 0; c < 3; ++c) {
            q[3 * mem[i] + c] = x[3 * i + c];
            v[3 * mem[i] + c] = u[3 * i + c];
        }
    if (steps_out) *steps_out = steps;
    free(mm); free(x); free(u); free(xp); free(up); free(a0); free(j0); free(a1); free(j1);
    free(ti); free(lev);
    return status;
}

/* Sec. 2.3, last paragraph: does some encounter set hold two or more
 * planets (bodies with m >= mp)?                                      */
static int or_planets_meet(int64_t nsets, const int64_t *set_start, const int64_t *members,
                           const double *m, double mp)
{
    for (int64_t st = 0; st < nsets; ++st) {
        int np = 0;
        for (int64_t a = set_start[st]; a < set_start[st + 1]; ++a)
            if (m[members[a]] >= mp) ++np;
        if (np >= 2) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2, Eq. 5 and Sec. 2.3: one system, nsteps hybrid DH steps.      */
/* q, v: DH state (heliocentric Q, barycentric v), star row zero.       */
/* enc: (step, i, j) records up to enc_cap, enc_d2 (optional) their     */
/* (d_min^2, threshold^2); *enc_count gets the total.                   */
/* stats[0..6]: encounter pairs, sets, largest set, Kepler iterations,  */
/* Hermite steps, Kepler non-convergences (summed over steps), steps    */
/* integrated whole by the Hermite.                                     */
/* With p->whole_hermite (Sec. 2.3, last paragraph, reading R11): when   */
/* a step's encounter sets put two planets in one set, that step is     */
/* redone for the whole system by the Hermite: from the positions after */
/* the opening drift and the velocities entering the first kick, every  */
/* body is integrated over tau under H_Kep + H_Int (star fixed at the   */
/* origin, K = 0 for every pair: r_crit infinite), no K corrections and */
/* no second kick; the closing drift follows as usual.                  */
/* rH_fixed: NULL -> Hill radii from the orbit entering each Kepler step  */
/* (reading R6); else per-body radii held fixed for the whole run.       */
/* Returns 0, or a nonzero status (1 Kepler, 2 Hermite cap).            */
/* ------------------------------------------------------------------ */
int or_step(int64_t rows, const double *m, double *q, double *v, const or_params *p, double tau,
            int64_t nsteps, int64_t step0, const double *rH_fixed, int64_t *enc, double *enc_d2,
            int64_t enc_cap, int64_t *enc_count, int64_t *stats, int64_t *near, double *near_d2,
            int64_t near_cap, int64_t *near_count)
{
    const double G = p->G, m0 = m[0], mu = G * m0;
    int64_t nb = rows - 1;
    size_t b3 = sizeof(double) * 3 * rows;
    double *q0 = (double *)malloc(b3), *v0 = (double *)malloc(b3);
    double *rH = (double *)malloc(sizeof(double) * rows);
    int32_t *its = (int32_t *)malloc(sizeof(int32_t) * (nb > 0 ? nb : 1));
    int64_t pcap = 1024, *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * pcap);
    double *pd2 = (double *)malloc(sizeof(double) * pcap), *pt2 = (double *)malloc(sizeof(double) * pcap);
    int64_t *set_of = (int64_t *)malloc(sizeof(int64_t) * rows);
    int64_t *set_start = (int64_t *)malloc(sizeof(int64_t) * (rows + 1));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * rows);
    double *rcrit = (double *)malloc(sizeof(double) * rows);
    double *vpre = p->whole_hermite ? (double *)malloc(b3) : NULL;
    int64_t *allmem = p->whole_hermite ? (int64_t *)malloc(sizeof(int64_t) * (nb > 0 ? nb : 1)) : NULL;
    for (int64_t i = 0; allmem && i < nb; ++i) allmem[i] = i + 1;
    int status = 0;
    int64_t ne_total = enc_count ? *enc_count : 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        int whole = 0;
        /* item 1: drift tau/2 */
        or_drift(rows, m, q, v, 0.5 * tau);
        if (vpre) memcpy(vpre, v, b3);  /* the velocities entering the first kick */
        /* item 2: interaction tau/2, all pairs, no transition function */
        or_kick(rows, m, q, v, G, 0.5 * tau);
        /* item 3: Kepler tau from (q0, v0) to (q, v); star row stays zero */
        memcpy(q0, q, b3);
        memcpy(v0, v, b3);
        int64_t bad = or_kepler_drift(nb, q0 + 3, v0 + 3, q + 3, v + 3, mu, tau, p->solver, p->guess,
                                      NULL, p->max_kepler_iter, NULL, its);
        if (stats) {
            for (int64_t i = 0; i < nb; ++i) stats[3] += its[i];
            stats[5] += bad;
        }
        if (bad) status = 1;
        if (p->encounters) {
            /* item 4: rigorous test over all pairs; sets; r_crit */
            if (rH_fixed)
                memcpy(rH, rH_fixed, sizeof(double) * rows);
            else
                or_hill_radii(rows, m, q0, v0, G, rH);
            int64_t npairs;
            for (;;) {
                int64_t nn0 = near_count ? *near_count : 0, nn = nn0;
                int64_t *nbuf = near_count ? (int64_t *)malloc(sizeof(int64_t) * 2 * 4096) : NULL;
                double *nd2 = near_count ? (double *)malloc(sizeof(double) * 2 * 4096) : NULL;
                int64_t nloc = 0;
                npairs = or_encounters_near(rows, q0, v0, q, v, rH, tau, p->a_E, pairs, pd2, pt2, pcap,
                                            2e-6, nbuf, nd2, 4096, near_count ? &nloc : NULL);
                if (near_count && npairs <= pcap) {
                    for (int64_t k = 0; k < nloc && k < 4096; ++k, ++nn) {
                        if (nn < near_cap) {
                            near[3 * nn] = step0 + s;
                            near[3 * nn + 1] = nbuf[2 * k];
                            near[3 * nn + 2] = nbuf[2 * k + 1];
                            near_d2[2 * nn] = nd2[2 * k];
                            near_d2[2 * nn + 1] = nd2[2 * k + 1];
                        }
                    }
                    *near_count = nn;
                }
                (void)nn0;
                free(nbuf);
                free(nd2);
                if (npairs <= pcap) break;
                pcap = 2 * npairs;
                pairs = (int64_t *)realloc(pairs, sizeof(int64_t) * 2 * pcap);
                pd2 = (double *)realloc(pd2, sizeof(double) * pcap);
                pt2 = (double *)realloc(pt2, sizeof(double) * pcap);
            }
            for (int64_t k = 0; k < npairs; ++k) {
                if (enc && ne_total < enc_cap) {
                    enc[3 * ne_total] = step0 + s;
                    enc[3 * ne_total + 1] = pairs[2 * k];
                    enc[3 * ne_total + 2] = pairs[2 * k + 1];
                    if (enc_d2) {
                        enc_d2[2 * ne_total] = pd2[k];
                        enc_d2[2 * ne_total + 1] = pt2[k];
                    }
                }
                ++ne_total;
            }
            if (npairs > 0) {
                int64_t nsets = or_sets(rows, npairs, pairs, rH, p->a_H, set_of, set_start, members, rcrit);
                if (stats) {
                    stats[0] += npairs;
                    stats[1] += nsets;
                }
                if (p->whole_hermite)
                    whole = or_planets_meet(nsets, set_start, members, m, p->planet_mass * m0);
                if (whole) {
                    for (int64_t st = 0; st < nsets; ++st) {
                        int64_t k = set_start[st + 1] - set_start[st];
                        if (stats && k > stats[2]) stats[2] = k;
                    }
                    /* the whole system from (q0, velocities entering the first kick) */
                    memcpy(q, q0, b3);
                    memcpy(v, vpre, b3);
                    int64_t hs = 0;
                    if (or_hermite_set(nb, allmem, m, m0, q, v, G, INFINITY, p->eps_H, p->eta,
                                       p->eta_s, tau, p->max_hermite_steps, &hs))
                        status = 2;
                    if (stats) {
                        stats[4] += hs;
                        stats[6] += 1;
                    }
                }
                for (int64_t st = 0; !whole && st < nsets; ++st) {
                    int64_t k0 = set_start[st], k = set_start[st + 1] - k0;
                    if (stats && k > stats[2]) stats[2] = k;
                    /* item 5: remove the (1-K) part of the first kick at q0 */
                    or_kcorr(k, members + k0, m, q0, v0, G, rcrit[st], 0.5 * tau);
                    /* item 6: Hermite over tau from (q0, v0); result into (q, v) */
                    for (int64_t a = 0; a < k; ++a) {
                        int64_t i = members[k0 + a];
                        for (int c = 0; c < 3; ++c) {
                            q[3 * i + c] = q0[3 * i + c];
                            v[3 * i + c] = v0[3 * i + c];
                        }
                    }
                    int64_t hs = 0;
                    if (or_hermite_set(k, members + k0, m, m0, q, v, G, rcrit[st], p->eps_H, p->eta,
                                       p->eta_s, tau, p->max_hermite_steps, &hs))
                        status = 2;
                    if (stats) stats[4] += hs;
                    /* item 7: pre-remove the (1-K) part of the coming kick at q1 */
                    or_kcorr(k, members + k0, m, q, v, G, rcrit[st], 0.5 * tau);
                }
            }
        }
        /* item 9: interaction tau/2 (not after a whole-system Hermite) */
        if (!whole) or_kick(rows, m, q, v, G, 0.5 * tau);
        /* item 10: drift tau/2 */
        or_drift(rows, m, q, v, 0.5 * tau);
    }
    if (enc_count) *enc_count = ne_total;
    free(q0); free(v0); free(rH); free(its); free(pairs); free(pd2); free(pt2);
    free(set_of); free(set_start); free(members); free(rcrit); free(vpre); free(allmem);
    return status;
}
