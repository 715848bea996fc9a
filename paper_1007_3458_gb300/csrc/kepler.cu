// kepler.cu -- E_Kep: universal-variable Kepler drift of every body about its
// star (Sec. 2 and the Appendix: f and g functions, Stumpff C and S, the
// universal Kepler equation F(x) = 0 solved by Laguerre's method, n = 5).
//
// One thread per body, FP64 throughout. Structure-of-arrays loads are
// coalesced; q0, v0 are kept and the result goes to separate buffers because
// the encounter test needs both ends of the step (Sec. 2.3 item 4).
//
// With the learned guess (MLP = true) each warp first evaluates the guess
// network for its 32 bodies on the tensor cores (mlp.cuh); the iteration then
// starts from x_std (1 + sigma t) instead of x_std = sqrt(mu) dt / r0 for the
// bodies on bound orbits (the network's domain). With a log buffer every
// solve on a bound orbit also writes its training row (u1..u4, t) with
// t = (x / x_std - 1) / sigma at the converged root x.
#include "mlp.cuh"

namespace qym {

// Stumpff functions C = c2(y), S = c3(y) (Appendix, Eqs. 2.40) by quartering
// the argument: y is scaled by 4^-k into |y| < 1 (exactly, a power of two),
// where the series C = sum_n (-y)^n / (2n+2)!, S = sum_n (-y)^n / (2n+3)! to
// the y^8 term is exact to rounding (the first omitted term is below 1e-18),
// and k doublings of s = sqrt(y) then follow from the double-angle formulas
// of sin and cos:  c2(4y) = c1(y)^2 / 2,  c3(4y) = (c3(y) + c1(y) c2(y)) / 4,
// with c1(y) = 1 - y c3(y) = sin(s) / s formed afresh at each level. Only
// multiply-adds, no division, square root or transcendental call, and the
// same instructions for bound and unbound orbits. Past 4^64 (s > 2^64) C and
// S are NaN, which the iteration treats as a point beyond the root.
__device__ __forceinline__ void stumpff(double y, double &C, double &S) {
    int k = 0;
    if (!(fabs(y) < 1.0)) {
        // |y| in [2^e, 2^(e+1)): k = floor(e/2) + 1 puts y / 4^k in [1/4, 1)
        const int e = ((__double2hiint(y) >> 20) & 0x7ff) - 1023;
        k = e / 2 + 1;
        if (k > 64) {
            C = S = __longlong_as_double(0x7ff8000000000000ll);
            return;
        }
        y *= __hiloint2double((1023 - 2 * k) << 20, 0);
    }
    // 1/(2n+2)! and 1/(2n+3)! for n = 0..8, alternating signs
    C = 1.0 / 2.0 + y * (-1.0 / 24.0 + y * (1.0 / 720.0 + y * (-1.0 / 40320.0 +
        y * (1.0 / 3628800.0 + y * (-1.0 / 479001600.0 + y * (1.0 / 87178291200.0 +
        y * (-1.0 / 20922789888000.0 + y * (1.0 / 6402373705728000.0))))))));
    S = 1.0 / 6.0 + y * (-1.0 / 120.0 + y * (1.0 / 5040.0 + y * (-1.0 / 362880.0 +
        y * (1.0 / 39916800.0 + y * (-1.0 / 6227020800.0 + y * (1.0 / 1307674368000.0 +
        y * (-1.0 / 355687428096000.0 + y * (1.0 / 121645100408832000.0))))))));
    for (int i = 0; i < k; ++i) {
        const double c1 = fma(-y, S, 1.0);
        S = 0.25 * fma(c1, C, S);
        C = 0.5 * c1 * c1;
        y *= 4.0;
    }
}

// F, F', F'' of the universal Kepler equation (Appendix), sig = r0.v0/sqrt(mu)
struct KepEq {
    double sqmu_dt, r0, sig, alpha, b;  // b = 1 - r0 alpha
    __device__ __forceinline__ void eval(double x, double &F, double &Fp, double &Fpp,
                                         double &C, double &S) const {
        double x2 = x * x;
        double y = alpha * x2;
        stumpff(y, C, S);
        double oyS = 1.0 - y * S;
        F = sig * x2 * C + b * x2 * x * S + r0 * x - sqmu_dt;
        Fp = sig * x * oyS + b * x2 * C + r0;
        Fpp = sig * (1.0 - y * C) + b * x * oyS;
    }
};

// Stumpff functions in FP32 for the first iterations of QYM_SOLVER_NEWTON32:
// the series to the y^6 term for |y| < 1 (its truncation below 1e-11, so
// only FP32 rounding remains), the closed forms beyond (s - sin s and
// sinh s - s lose at most about three bits there)
__device__ __forceinline__ void stumpff_f32(float y, float &C, float &S) {
    if (fabsf(y) < 1.0f) {
        C = 0.5f + y * (-1.0f / 24.0f + y * (1.0f / 720.0f + y * (-1.0f / 40320.0f +
            y * (1.0f / 3628800.0f + y * (-1.0f / 479001600.0f + y * (1.0f / 87178291200.0f))))));
        S = 1.0f / 6.0f + y * (-1.0f / 120.0f + y * (1.0f / 5040.0f + y * (-1.0f / 362880.0f +
            y * (1.0f / 39916800.0f + y * (-1.0f / 6227020800.0f + y * (1.0f / 1307674368000.0f))))));
    } else if (y > 0.0f) {
        const float s = sqrtf(y);
        float sh, ch;
        sincosf(0.5f * s, &sh, &ch);
        C = 2.0f * sh * sh / y;
        S = (s - 2.0f * sh * ch) / (y * s);
    } else {
        const float s = sqrtf(-y);
        C = (coshf(s) - 1.0f) / (-y);
        S = (sinhf(s) - s) / ((-y) * s);
    }
}

// QYM_SOLVER_NEWTON32: Newton's method on F in FP32 from x while it stays in
// the bracket [lo, hi] (at most 12 steps), until a step falls below 1e-5 |x|;
// x then holds the FP32 root (relative error about 1e-7, more where F's terms
// cancel) and the FP64 iteration finishes from there under the unchanged
// residual test. Returns
// the FP32 steps taken, and leaves x unchanged (0 steps counted) when the FP32
// form fails (a step leaves the bracket, F or F' is not finite).
__device__ __forceinline__ int newton_f32(const KepEq &eq, double lo, double hi, double &x) {
    const float sq = (float)eq.sqmu_dt, r0 = (float)eq.r0, sig = (float)eq.sig;
    const float al = (float)eq.alpha, b = (float)eq.b;
    const float lof = (float)lo, hif = (float)hi;
    float xf = (float)x;
    for (int it = 0; it < 12; ++it) {
        const float x2 = xf * xf, y = al * x2;
        float C, S;
        stumpff_f32(y, C, S);
        const float F = sig * x2 * C + b * x2 * xf * S + r0 * xf - sq;
        const float Fp = sig * xf * (1.0f - y * S) + b * x2 * C + r0;
        if (!isfinite(F) || !(Fp > 0.0f) || !isfinite(Fp)) return 0;
        const float dx = F / Fp;
        const float xn = xf - dx;
        if (!(xn >= lof && xn <= hif)) return 0;
        xf = xn;
        if (fabsf(dx) <= 1e-5f * fabsf(xf)) {
            x = (double)xf;
            return it + 1;
        }
    }
    return 0;
}

template <bool MLP>
__global__ void __launch_bounds__(256) k_kepler(KeplerArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int iters = 0;
    const bool act = k < a.n;
    const int64_t r = act ? (a.rows ? a.rows[k] : a.row0 + k) : 0;
    const int64_t ld = a.ld;
    double qx = 0.0, qy = 0.0, qz = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    // mu = G m0 with sqrt(mu) and 1/mu, formed once per system on the host
    // (correctly rounded, as sqrt and the division here would give them)
    double mu = 1.0, sqmu = 1.0, imu = 1.0;
    if (act) {
        qx = a.q0[r]; qy = a.q0[ld + r]; qz = a.q0[2 * ld + r];
        vx = a.v0[r]; vy = a.v0[ld + r]; vz = a.v0[2 * ld + r];
        if (a.kmu) {
            const double *km = a.kmu + 3 * (int64_t)a.sys_of[r];
            mu = km[0]; sqmu = km[1]; imu = km[2];
        } else {
            mu = a.mu; sqmu = a.sqmu; imu = a.imu;
        }
    }
    const double dt = a.dt;
    const double r0 = sqrt(qx * qx + qy * qy + qz * qz);
    const bool feat = act && r0 > 0.0 && dt != 0.0;
    float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    double sigma = 0.0;
    bool bound = false;  // in the learned guess's domain
    if (feat && (MLP || a.log)) bound = mlp::features(qx, qy, qz, vx, vy, vz, r0, mu, dt, u, sigma);
    double x_mlp = 0.0;
    bool have_mlp = false;
    if (MLP) {
        // every lane of the warp takes part, active or not
        float fn[4];
        mlp::normalise(a.mlp_w, u, fn);
        const float y = mlp::warp_forward(a.mlp_w, fn);
        const float tn = a.mlp_w[mlp::OM] + a.mlp_w[mlp::OSD] * y;
        x_mlp = sqmu * dt / r0 * (1.0 + sigma * (double)tn);
        have_mlp = bound && isfinite(x_mlp);
    }
    if (act) {
        if (r0 == 0.0) {
            // a star row (held at Q = v = 0): stays at the origin
            a.q1[r] = 0.0; a.q1[ld + r] = 0.0; a.q1[2 * ld + r] = 0.0;
            a.v1[r] = 0.0; a.v1[ld + r] = 0.0; a.v1[2 * ld + r] = 0.0;
            if (a.x_out) a.x_out[k] = 0.0;
            if (a.x0_out) a.x0_out[k] = 0.0;
            if (a.iters) a.iters[k] = 0;
            goto done;
        }
        {
        double vv = vx * vx + vy * vy + vz * vz;
        // the FP64 pipe bounds this kernel: divisions by mu, sqrt(mu) and r0
        // become products with reciprocals formed once (within an ulp of the
        // quotients)
        const double ir0 = 1.0 / r0, isqmu = sqmu * imu;
        KepEq eq;
        eq.sqmu_dt = sqmu * dt;
        eq.r0 = r0;
        eq.alpha = 2.0 * ir0 - vv * imu;
        eq.sig = (qx * vx + qy * vy + qz * vz) * isqmu;
        eq.b = 1.0 - r0 * eq.alpha;
        double x;
        if (a.guess == QYM_GUESS_R0)
            x = r0;
        else if (MLP && have_mlp)
            x = x_mlp;
        else
            x = eq.sqmu_dt * ir0;
        if (a.x0_out) a.x0_out[k] = x;
        int solver = a.solver;
        bool conv = false;
        bool cs_at_x = false;  // C, S hold the Stumpff values at the final x
        double C = 0.5, S = 1.0 / 6.0;
        // Root bracket: F(0) = -sqrt(mu) dt and F' = r >= r_p (periapsis
        // distance), so the root lies between 0 and sqrt(mu) dt / r_p; for an
        // unbound orbit also |x| <= 700 / sqrt(-alpha), past which C and S
        // overflow. Widened by 1e-12 for the rounding of r_p = p / (1 + e).
        double lo = -INFINITY, hi = INFINITY;
        {
            double hx = qy * vz - qz * vy, hy = qz * vx - qx * vz, hz = qx * vy - qy * vx;
            double p = (hx * hx + hy * hy + hz * hz) * imu;
            double ecc = sqrt(fmax(0.0, 1.0 - p * eq.alpha));
            if (p > 0.0) {
                double xb = eq.sqmu_dt * (1.0 + ecc) / p * (1.0 + 1e-12);
                if (dt >= 0.0) { lo = 0.0; hi = xb; } else { lo = xb; hi = 0.0; }
            }
            if (eq.alpha < 0.0) {
                // rsqrt within 2 ulp: the bound is widened by 1e-12
                double xm = 700.0 * (1.0 + 1e-12) * rsqrt(-eq.alpha);
                if (dt >= 0.0) { lo = fmax(lo, 0.0); hi = fmin(hi, xm); }
                else { lo = fmax(lo, -xm); hi = fmin(hi, 0.0); }
            }
        }
        const double lo0 = lo, hi0 = hi;
        if (solver == QYM_SOLVER_NEWTON32) {
            // FP32 Newton steps first, then the FP64 iteration in Laguerre's
            // form: from the FP32 root (about 1e-7) one cubic step reaches
            // the rounding level, so the evaluation after it meets the
            // residual test
            iters += newton_f32(eq, lo, hi, x);
            solver = QYM_SOLVER_LAGUERRE;
        }
        // two passes at most: the requested start, then (learned guess only)
        // Laguerre from the standard guess if the first did not converge
        for (int pass = 0; pass < 2 && !conv; ++pass) {
            if (pass == 1) {
                if (!MLP) break;
                x = eq.sqmu_dt * ir0;
                solver = QYM_SOLVER_LAGUERRE;
                lo = lo0;
                hi = hi0;
            }
            const bool have_br = isfinite(lo) && isfinite(hi);
            if (!(x >= lo && x <= hi) && have_br) x = 0.5 * (lo + hi);
            double dx_old = INFINITY;
            // after a step at the rounding level: the point it started from
            // and its relative residual
            bool settle = false;
            double x_prev = x, res_prev = INFINITY;
            for (int it = 0; it < a.max_iter; ++it) {
                double F, Fp, Fpp;
                eq.eval(x, F, Fp, Fpp, C, S);
                ++iters;
                if (!isfinite(F) || !isfinite(Fp) || !isfinite(Fpp)) {
                    if (x > 0.0) hi = x; else lo = x;
                    x = 0.5 * (lo + hi);
                    continue;
                }
                if (F < 0.0) lo = x; else hi = x;
                // residual against the rounding floor of F: the sum of |terms|
                double x2 = x * x;
                double scale = fabs(eq.sqmu_dt) + fabs(eq.sig * x2 * C) +
                               fabs(eq.b * x2 * x * S) + r0 * fabs(x);
                if (fabs(F) <= 1e-14 * scale) { --iters; conv = true; cs_at_x = true; break; }
                if (settle) {
                    // evaluated after a rounding-level step and still above
                    // 1e-14: the better of the last two points is the root
                    --iters;
                    conv = true;
                    if (fabs(F) / scale <= res_prev) cs_at_x = true; else x = x_prev;
                    break;
                }
                double dx;
                if (solver == QYM_SOLVER_LAGUERRE) {
                    // Laguerre, n = 5: dx = n F / (F' + sgn(F') sqrt|(n-1)^2 F'^2 - n(n-1) F F''|),
                    // with F' taken out of the root so that F'^2 never overflows:
                    // dx = rf 5 / (1 + sqrt|16 - 20 z|), rf = F / F', z = rf F'' / F'.
                    // Near the root (|z| < 1e-6) the factor is its series
                    // 1 + z / 2 + 13 z^2 / 32 (next term 0.38 z^3 < 4e-19): the same
                    // step to rounding without the square root and the division
                    const double iFp = 1.0 / Fp, rf = F * iFp, z = rf * (Fpp * iFp);
                    if (fabs(z) < 1e-6)
                        dx = rf * fma(z, fma(13.0 / 32.0, z, 0.5), 1.0);
                    else
                        dx = 5.0 * rf / (1.0 + sqrt(fabs(16.0 - 20.0 * z)));
                } else {
                    dx = F / Fp;
                }
                double xn = x - dx;
                // bisect when the step is not finite, leaves the bracket, or fails
                // to halve the previous step (slow approach along exp(sqrt(-alpha) x))
                if (isfinite(lo) && isfinite(hi) &&
                    (!isfinite(dx) || !(xn >= lo && xn <= hi) || fabs(dx) > 0.5 * fabs(dx_old))) {
                    xn = 0.5 * (lo + hi);
                    dx = x - xn;
                }
                dx_old = dx;
                if (fabs(dx) <= 0x1p-50 * fabs(xn) ||
                    (isfinite(lo) && isfinite(hi) && hi - lo <= 0x1p-50 * fabs(xn))) {
                    settle = true;
                    x_prev = x;
                    res_prev = fabs(F) / scale;
                }
                x = xn;
            }
        }
        // f and g functions at the root (Appendix); r before fdot, gdot. The
        // last evaluation left C, S at this x unless the iteration kept the
        // point before it, or ran out of iterations after a step
        double x2 = x * x;
        double y = eq.alpha * x2;
        if (!cs_at_x) stumpff(y, C, S);
        double f = 1.0 - x2 * C * ir0;
        double g = dt - x2 * x * S * isqmu;
        double nx = f * qx + g * vx, ny = f * qy + g * vy, nz = f * qz + g * vz;
        double irr = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
        double fd = sqmu * x * (y * S - 1.0) * irr * ir0;
        double gd = 1.0 - x2 * C * irr;
        double ux = fd * qx + gd * vx, uy = fd * qy + gd * vy, uz = fd * qz + gd * vz;
        a.q1[r] = nx; a.q1[ld + r] = ny; a.q1[2 * ld + r] = nz;
        a.v1[r] = ux; a.v1[ld + r] = uy; a.v1[2 * ld + r] = uz;
        if (a.x_out) a.x_out[k] = x;
        if (a.iters) a.iters[k] = iters;
        if (a.log && bound) {
            // training row of this solve: slot (steps logged so far) * n + k
            const int64_t base = a.log_step ? (int64_t)(*a.log_base + *a.log_step) * a.n : 0;
            const int64_t slot = base + k;
            if (slot < a.log_cap) {
                const double t = (x * r0 / eq.sqmu_dt - 1.0) / sigma;
                float *row = a.log + 5 * slot;
                row[0] = u[0]; row[1] = u[1]; row[2] = u[2]; row[3] = u[3];
                row[4] = (float)t;
            }
        }
        if (a.status) {
            int bits = 0;
            if (!conv) bits |= QYM_ST_KEPLER_NOCONV;
            if (!(isfinite(nx) && isfinite(ny) && isfinite(nz) && isfinite(ux) && isfinite(uy) &&
                  isfinite(uz)))
                bits |= QYM_ST_NAN;
            if (bits) atomicOr(a.status, bits);
        }
        }
    }
done:
    if (a.iter_sum) {
        unsigned long long s = (unsigned long long)iters;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(a.iter_sum, s);
    }
}

cudaError_t launch_kepler(const KeplerArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    int threads = 256;
    int64_t blocks = (a.n + threads - 1) / threads;
    if (a.guess == QYM_GUESS_MLP && a.mlp_w)
        k_kepler<true><<<(unsigned)blocks, threads, 0, st>>>(a);
    else
        k_kepler<false><<<(unsigned)blocks, threads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace qym
