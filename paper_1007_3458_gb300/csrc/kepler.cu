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

// Stumpff functions (Appendix, Eqs. 2.40). Near y = 0 the alternating series
// C = sum_k (-y)^k / (2k+2)!, S = sum_k (-y)^k / (2k+3)! in Horner form to
// the y^8 term; elsewhere the closed forms, C through 2 sin^2(s/2) / y to
// avoid the cancellation of 1 - cos s.
__device__ __forceinline__ void stumpff(double y, double &C, double &S) {
    if (fabs(y) < 0.1) {
        // 1/(2k+2)! and 1/(2k+3)! for k = 0..8, alternating signs
        C = 1.0 / 2.0 + y * (-1.0 / 24.0 + y * (1.0 / 720.0 + y * (-1.0 / 40320.0 +
            y * (1.0 / 3628800.0 + y * (-1.0 / 479001600.0 + y * (1.0 / 87178291200.0 +
            y * (-1.0 / 20922789888000.0 + y * (1.0 / 6402373705728000.0))))))));
        S = 1.0 / 6.0 + y * (-1.0 / 120.0 + y * (1.0 / 5040.0 + y * (-1.0 / 362880.0 +
            y * (1.0 / 39916800.0 + y * (-1.0 / 6227020800.0 + y * (1.0 / 1307674368000.0 +
            y * (-1.0 / 355687428096000.0 + y * (1.0 / 121645100408832000.0))))))));
    } else if (y > 0.0) {
        double s = sqrt(y);
        double sh, ch;
        sincos(0.5 * s, &sh, &ch);
        C = 2.0 * sh * sh / y;
        S = (s - 2.0 * sh * ch) / (y * s);
    } else {
        double s = sqrt(-y);
        C = (cosh(s) - 1.0) / (-y);
        S = (sinh(s) - s) / ((-y) * s);
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

template <bool MLP>
__global__ void __launch_bounds__(256) k_kepler(KeplerArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int iters = 0;
    const bool act = k < a.n;
    const int64_t r = act ? (a.rows ? a.rows[k] : a.row0 + k) : 0;
    const int64_t ld = a.ld;
    double qx = 0.0, qy = 0.0, qz = 0.0, vx = 0.0, vy = 0.0, vz = 0.0, mu = 1.0;
    if (act) {
        qx = a.q0[r]; qy = a.q0[ld + r]; qz = a.q0[2 * ld + r];
        vx = a.v0[r]; vy = a.v0[ld + r]; vz = a.v0[2 * ld + r];
        mu = a.sys_of ? a.G * a.m[a.offsets[a.sys_of[r]]] : a.mu;
    }
    const double dt = a.dt;
    const double sqmu = sqrt(mu);
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
        KepEq eq;
        eq.sqmu_dt = sqmu * dt;
        eq.r0 = r0;
        eq.alpha = 2.0 / r0 - vv / mu;
        eq.sig = (qx * vx + qy * vy + qz * vz) / sqmu;
        eq.b = 1.0 - r0 * eq.alpha;
        double x;
        if (a.guess == QYM_GUESS_R0)
            x = r0;
        else if (MLP && have_mlp)
            x = x_mlp;
        else
            x = eq.sqmu_dt / r0;
        if (a.x0_out) a.x0_out[k] = x;
        int solver = a.solver;
        bool conv = false;
        bool cs_at_x = false;  // C, S hold the Stumpff values at the final x
        double C = 0.5, S = 1.0 / 6.0;
        // Root bracket: F(0) = -sqrt(mu) dt and F' = r >= r_p (periapsis
        // distance), so the root lies between 0 and sqrt(mu) dt / r_p; for an
        // unbound orbit also |x| <= 700 / sqrt(-alpha), past which C and S
        // overflow. Widened by 1e-12 for the rounding of r_p.
        double lo = -INFINITY, hi = INFINITY;
        {
            double hx = qy * vz - qz * vy, hy = qz * vx - qx * vz, hz = qx * vy - qy * vx;
            double p = (hx * hx + hy * hy + hz * hz) / mu;
            double ecc = sqrt(fmax(0.0, 1.0 - p * eq.alpha));
            double rp = p / (1.0 + ecc);
            if (rp > 0.0) {
                double xb = eq.sqmu_dt / rp * (1.0 + 1e-12);
                if (dt >= 0.0) { lo = 0.0; hi = xb; } else { lo = xb; hi = 0.0; }
            }
            if (eq.alpha < 0.0) {
                double xm = 700.0 / sqrt(-eq.alpha);
                if (dt >= 0.0) { lo = fmax(lo, 0.0); hi = fmin(hi, xm); }
                else { lo = fmax(lo, -xm); hi = fmin(hi, 0.0); }
            }
        }
        const double lo0 = lo, hi0 = hi;
        // two passes at most: the requested start, then (learned guess only)
        // Laguerre from the standard guess if the first did not converge
        for (int pass = 0; pass < 2 && !conv; ++pass) {
            if (pass == 1) {
                if (!MLP) break;
                x = eq.sqmu_dt / r0;
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
                    // with F' taken out of the root so that F'^2 never overflows
                    const double rf = F / Fp, rpp = Fpp / Fp;
                    dx = 5.0 * rf / (1.0 + sqrt(fabs(16.0 - 20.0 * rf * rpp)));
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
        double f = 1.0 - x2 / r0 * C;
        double g = dt - x2 * x / sqmu * S;
        double nx = f * qx + g * vx, ny = f * qy + g * vy, nz = f * qz + g * vz;
        double rr = sqrt(nx * nx + ny * ny + nz * nz);
        double fd = sqmu * x * (y * S - 1.0) / (rr * r0);
        double gd = 1.0 - x2 / rr * C;
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
