// hermite.cu -- the close-encounter branch of the hybrid step (Sec. 2.2 and
// Sec. 2.3 items 5-8), one CTA per encounter set:
//   1. remove the (1-K) part of the first kick at q0 (item 5),
//   2. integrate the set for tau with a 4th-order Hermite predictor /
//      evaluate / corrector (Makino & Aarseth, no Ahmad-Cohen) under H'_Kep:
//      the star, fixed at the origin, plus the members' pair forces weighted
//      by [1 - K(s) + s K'(s)], jerks with the K'' term (item 6),
//   3. pre-remove the (1-K) part of the coming kick at q1 (item 7),
//   4. write the members' q1, v1 over their Kepler result (item 8).
// Members carry individual block time steps (Makino & Aarseth): time runs in
// integer ticks of |tau| / 2^48, member i steps with |tau| 2^-k_i from the
// Aarseth criterion (eta; eta_s at start-up) rounded down to a power of two,
// and a step doubles only on a commensurate block time. At each block time
// every member is predicted and the members whose step ends there are
// evaluated and corrected. Every loop has a cap and reports through the
// status word.
#include <climits>

#include "qym_internal.cuh"

namespace qym {

constexpr int HCAP = 512;       // members per set held in shared memory
constexpr int HTHREADS = 256;

// sin and cos of (pi/2) y for y in [0, 1]: y > 1/2 is folded onto 1 - y
// (sin and cos swap), so the argument w = (pi/2) y' stays in [0, pi/4], where
// the Taylor series of sin to w^15 and of cos to w^16 leave truncation errors
// below 7e-17 and 3e-18 (the next terms, w^17/17! and w^18/18!, at pi/4).
__device__ __forceinline__ void sincos_half_pi(double y, double &sn, double &cs) {
    const bool fold = y > 0.5;
    const double w = 1.5707963267948966 * (fold ? 1.0 - y : y);
    const double w2 = w * w;
    double ps = -1.0 / 1307674368000.0;        // -1/15!
    ps = fma(ps, w2, 1.0 / 6227020800.0);      // +1/13!
    ps = fma(ps, w2, -1.0 / 39916800.0);       // -1/11!
    ps = fma(ps, w2, 1.0 / 362880.0);          // +1/9!
    ps = fma(ps, w2, -1.0 / 5040.0);           // -1/7!
    ps = fma(ps, w2, 1.0 / 120.0);             // +1/5!
    ps = fma(ps, w2, -1.0 / 6.0);              // -1/3!
    ps = fma(ps, w2, 1.0);
    const double sw = w * ps;
    double pc = 1.0 / 20922789888000.0;        // +1/16!
    pc = fma(pc, w2, -1.0 / 87178291200.0);    // -1/14!
    pc = fma(pc, w2, 1.0 / 479001600.0);       // +1/12!
    pc = fma(pc, w2, -1.0 / 3628800.0);        // -1/10!
    pc = fma(pc, w2, 1.0 / 40320.0);           // +1/8!
    pc = fma(pc, w2, -1.0 / 720.0);            // -1/6!
    pc = fma(pc, w2, 1.0 / 24.0);              // +1/4!
    pc = fma(pc, w2, -0.5);                    // -1/2!
    pc = fma(pc, w2, 1.0);
    sn = fold ? pc : sw;
    cs = fold ? sw : pc;
}

// Constants of the transition function of one set: K(y) = sin(pi y / 2) with
// y = 1.1 s / r_crit - 0.1 (Sec. 2.1), so y = a s - 0.1 and dy/ds = a.
struct TransC {
    double rc2;  // r_crit^2: K = 1 (and K' = K'' = 0) beyond
    double a;    // 1.1 / r_crit
    double c;    // (pi / 2) a: K' = c cos, K'' = -c^2 sin
    __device__ __forceinline__ explicit TransC(double rc)
        : rc2(rc * rc), a(1.1 / rc), c(0.5 * kPi * (1.1 / rc)) {}
};

// K and its first and second derivatives with respect to s
__device__ __forceinline__ void transition(double s, const TransC &tc, double &K, double &Kp,
                                           double &Kpp) {
    const double y = tc.a * s - 0.1;
    if (y <= 0.0) {
        K = 0.0; Kp = 0.0; Kpp = 0.0;
    } else if (y >= 1.0) {
        K = 1.0; Kp = 0.0; Kpp = 0.0;
    } else {
        double sn, cs;
        sincos_half_pi(y, sn, cs);
        K = sn;
        Kp = tc.c * cs;
        Kpp = -tc.c * tc.c * sn;
    }
}

__global__ void k_transition(int64_t n, const double *s, double rc, double *K, double *Kp,
                             double *Kpp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TransC tc(rc);
    double k0, k1, k2;
    transition(s[i], tc, k0, k1, k2);
    K[i] = k0;
    Kp[i] = k1;
    Kpp[i] = k2;
}

cudaError_t launch_transition(int64_t n, const double *s, double rc, double *K, double *Kp,
                              double *Kpp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_transition<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s, rc, K, Kp, Kpp);
    return cudaGetLastError();
}

struct HermSmem {
    double *ex, *ey, *ez, *eu, *ev, *ew, *m;  // evaluation point of every member
    double *x, *y, *z, *u, *v, *w;            // state at the member's own time
    double *ax, *ay, *az, *jx, *jy, *jz;      // a, adot at the member's own time
    long long *ti;                            // member time in ticks
    int32_t *lev;                             // member level: step = tau 2^-lev
    int32_t *act;                             // members whose step ends now
    int32_t *ids;
};

__device__ __forceinline__ HermSmem carve(void *base) {
    double *p = (double *)base;
    HermSmem s;
    s.ex = p; p += HCAP; s.ey = p; p += HCAP; s.ez = p; p += HCAP;
    s.eu = p; p += HCAP; s.ev = p; p += HCAP; s.ew = p; p += HCAP;
    s.m = p; p += HCAP;
    s.x = p; p += HCAP; s.y = p; p += HCAP; s.z = p; p += HCAP;
    s.u = p; p += HCAP; s.v = p; p += HCAP; s.w = p; p += HCAP;
    s.ax = p; p += HCAP; s.ay = p; p += HCAP; s.az = p; p += HCAP;
    s.jx = p; p += HCAP; s.jy = p; p += HCAP; s.jz = p; p += HCAP;
    s.ti = (long long *)p; p += HCAP;
    int32_t *ip = (int32_t *)p;
    s.lev = ip; ip += HCAP;
    s.act = ip; ip += HCAP;
    s.ids = ip;
    return s;
}
constexpr size_t kHermSmem = sizeof(double) * HCAP * 20 + sizeof(int32_t) * HCAP * 3;
constexpr int KMAX = 48;

// smallest k with T 2^-k <= dt_c, in [0, KMAX]: with T = fT 2^eT and
// dt_c = fd 2^ed (fT, fd in [1/2, 1)), T 2^-k <= dt_c exactly when
// k >= eT - ed + (fT > fd)
__device__ __forceinline__ int level_of(double dt_c, double T) {
    if (!(dt_c > 0.0)) return KMAX;
    if (dt_c >= T) return 0;
    int eT, ed;
    const double fT = frexp(T, &eT), fd = frexp(dt_c, &ed);
    const int k = eT - ed + (fT > fd ? 1 : 0);
    return k < 0 ? 0 : (k > KMAX ? KMAX : k);
}

// Work split of a set of n members over the CTA: each member is handled by
// P consecutive lanes (P a power of two, P * n <= HTHREADS when possible),
// lane l of a member's group takes the partners l, l + P, ...; the group's
// partial sums are combined with warp shuffles in a fixed tree order.
__device__ __forceinline__ int lanes_per_member(int n) {
    int p = 32;
    while (p > 1 && p * n > HTHREADS) p >>= 1;
    return p;
}

__device__ __forceinline__ void group_sum(double *v, int cnt, int P) {
    for (int off = P >> 1; off > 0; off >>= 1)
        for (int c = 0; c < cnt; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
}

// partial (1-K)-weighted pair acceleration of member k at the evaluation
// point, unsmoothed (the kick used the bare separation):
// sum_l -G m_l q_kl / q^3 [1 - K + q K'] over the partners of this lane
__device__ void kcorr_part(const HermSmem &S, int n, int k, int l0, int P, double G,
                           const TransC &tc, double *c) {
    c[0] = c[1] = c[2] = 0.0;
    for (int l = l0; l < n; l += P) {
        if (l == k) continue;
        double qx = S.ex[k] - S.ex[l], qy = S.ey[k] - S.ey[l], qz = S.ez[k] - S.ez[l];
        double q2 = qx * qx + qy * qy + qz * qz;
        if (q2 >= tc.rc2) continue;  // K = 1 beyond r_crit: no (1-K) part
        const double qi = rsqrt(q2);
        const double q = q2 * qi;
        double K, Kp, Kpp;
        transition(q, tc, K, Kp, Kpp);
        double wgt = -G * S.m[l] * (qi * qi * qi) * (1.0 - K + q * Kp);
        c[0] += wgt * qx;
        c[1] += wgt * qy;
        c[2] += wgt * qz;
    }
}

// partial Hermite acceleration and jerk of member k at the evaluation point
// (Sec. 2.2): the star term on lane 0 of the group, the pair terms with the
// transition bracket over this lane's partners
// (one reciprocal square root per pair: q = q2 / sqrt(q2), 1/q^3, 1/q^2)
__device__ void herm_part(const HermSmem &S, int n, int k, int l0, int P, double G, double m0,
                          const TransC &tc, double eps2, double *aj) {
    const double xk = S.ex[k], yk = S.ey[k], zk = S.ez[k];
    const double uk = S.eu[k], vk = S.ev[k], wk = S.ew[k];
    for (int c = 0; c < 6; ++c) aj[c] = 0.0;
    if (l0 == 0) {  // star, fixed at the origin
        double s2 = xk * xk + yk * yk + zk * zk + eps2;
        double si = rsqrt(s2);
        double si2 = si * si;
        double rv = xk * uk + yk * vk + zk * wk;
        double c = -G * m0 * (si2 * si);
        double t = 3.0 * rv * si2;
        aj[0] = c * xk; aj[1] = c * yk; aj[2] = c * zk;
        aj[3] = c * (uk - t * xk); aj[4] = c * (vk - t * yk); aj[5] = c * (wk - t * zk);
    }
    for (int l = l0; l < n; l += P) {
        if (l == k) continue;
        double qx = xk - S.ex[l], qy = yk - S.ey[l], qz = zk - S.ez[l];
        double q2 = qx * qx + qy * qy + qz * qz + eps2;
        if (q2 >= tc.rc2) continue;  // K = 1, K' = K'' = 0: no force, no jerk
        double px = uk - S.eu[l], py = vk - S.ev[l], pz = wk - S.ew[l];
        const double qi = rsqrt(q2);
        const double qi2 = qi * qi;
        const double sq = q2 * qi;
        double K, Kp, Kpp;
        transition(sq, tc, K, Kp, Kpp);
        double br = 1.0 - K + sq * Kp;
        double rvl = qx * px + qy * py + qz * pz;
        double cl = -G * S.m[l] * (qi2 * qi);
        double tl = 3.0 * rvl * qi2;
        aj[0] += cl * br * qx; aj[1] += cl * br * qy; aj[2] += cl * br * qz;
        aj[3] += cl * (rvl * qx * Kpp + (px - tl * qx) * br);
        aj[4] += cl * (rvl * qy * Kpp + (py - tl * qy) * br);
        aj[5] += cl * (rvl * qz * Kpp + (pz - tl * qz) * br);
    }
}

__device__ __forceinline__ long long block_min_ll(long long x, long long *red) {
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    long long r = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = min(r, red[k]);
    return r;
}

__device__ __forceinline__ double block_min(double x, double *red) {
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
    int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double r = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmin(r, red[k]);
    return r;
}

struct HermArgs {
    double G, eps2, eta, eta_s, tau;
    int64_t max_steps;
};

__global__ void __launch_bounds__(HTHREADS) k_hermite(Dev d, HermArgs h) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    HermSmem S = carve(smem);
    const int64_t R = d.rows;
    const int tid = threadIdx.x;
    int nsets = (int)min((unsigned long long)d.max_sets, d.ctr[C_NSETS]);
    for (int set = blockIdx.x; set < nsets; set += gridDim.x) {
        const int st = d.set_start[set];
        const int n = d.set_start[set + 1] - st;
        if (n < 1) continue;
        if (n > HCAP || st + n > d.max_members) {
            if (tid == 0) atomicOr(d.status, QYM_ST_SET_OVERFLOW);
            for (int k = tid; k < n && st + k < d.max_members; k += blockDim.x)
                d.uf[d.set_mem[st + k]] = -1;
            continue;
        }
        const int P = lanes_per_member(n);
        const int NG = HTHREADS / P;             // member groups in the CTA
        const int grp = tid / P, lane = tid % P;
        // members in ascending row order (rank sort)
        __syncthreads();
        for (int k = tid; k < n; k += blockDim.x) S.ids[k] = d.set_mem[st + k];
        __syncthreads();
        int myid[HCAP / HTHREADS], myrank[HCAP / HTHREADS];
        for (int c = 0; c < HCAP / HTHREADS; ++c) {
            int k = tid + c * blockDim.x;
            myid[c] = k < n ? S.ids[k] : 0;
            int rk = 0;
            if (k < n)
                for (int l = 0; l < n; ++l) rk += S.ids[l] < myid[c];
            myrank[c] = rk;
        }
        __syncthreads();
        for (int c = 0; c < HCAP / HTHREADS; ++c) {
            int k = tid + c * blockDim.x;
            if (k < n) S.ids[myrank[c]] = myid[c];
        }
        __syncthreads();
        const int64_t star = d.offsets[d.sys_of[S.ids[0]]];
        const double m0 = d.m[star];
        const TransC tc(d.rcrit[set]);
        const double G = h.G, tau = h.tau;
        // state entering the Kepler drift (after the first kick)
        for (int k = tid; k < n; k += blockDim.x) {
            int64_t r = S.ids[k];
            S.ex[k] = S.x[k] = d.q[r];
            S.ey[k] = S.y[k] = d.q[R + r];
            S.ez[k] = S.z[k] = d.q[2 * R + r];
            S.u[k] = d.v[r];
            S.v[k] = d.v[R + r];
            S.w[k] = d.v[2 * R + r];
            S.m[k] = d.m[r];
        }
        __syncthreads();
        // item 5: remove the (1-K) part of the first kick
        for (int k0 = 0; k0 < n; k0 += NG) {
            int k = k0 + grp;
            double c[3] = {0.0, 0.0, 0.0};
            if (k < n) kcorr_part(S, n, k, lane, P, G, tc, c);
            group_sum(c, 3, P);
            if (k < n && lane == 0) {
                S.u[k] -= 0.5 * tau * c[0];
                S.v[k] -= 0.5 * tau * c[1];
                S.w[k] -= 0.5 * tau * c[2];
            }
        }
        __syncthreads();
        for (int k = tid; k < n; k += blockDim.x) {
            S.eu[k] = S.u[k]; S.ev[k] = S.v[k]; S.ew[k] = S.w[k];
        }
        __syncthreads();
        // start-up: a, adot at t = 0 and the levels from eta_s |a| / |adot|
        const double sgn = tau >= 0.0 ? 1.0 : -1.0;
        const double T = fabs(tau);
        const long long TT = 1ll << KMAX;
        const double tick = T / (double)TT;
        for (int k0 = 0; k0 < n; k0 += NG) {
            int k = k0 + grp;
            double aj[6] = {0, 0, 0, 0, 0, 0};
            if (k < n) herm_part(S, n, k, lane, P, G, m0, tc, h.eps2, aj);
            group_sum(aj, 6, P);
            if (k < n && lane == 0) {
                S.ax[k] = aj[0]; S.ay[k] = aj[1]; S.az[k] = aj[2];
                S.jx[k] = aj[3]; S.jy[k] = aj[4]; S.jz[k] = aj[5];
                double jn = sqrt(aj[3] * aj[3] + aj[4] * aj[4] + aj[5] * aj[5]);
                double dt_c = jn > 0.0 ? h.eta_s * sqrt(aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]) / jn : T;
                S.lev[k] = level_of(dt_c, T);
                S.ti[k] = 0;
            }
        }
        __shared__ long long redl[32];
        __shared__ int n_act;
        int64_t steps = 0;
        bool capped = false;
        for (;;) {
            __syncthreads();
            // next block time: the earliest end of a member's step
            long long tn_l = LLONG_MAX;
            for (int k = tid; k < n; k += blockDim.x)
                tn_l = min(tn_l, S.ti[k] + (1ll << (KMAX - S.lev[k])));
            const long long tn = block_min_ll(tn_l, redl);
            if (tn > TT) break;  // every member has reached tau
            if (steps >= h.max_steps) { capped = true; break; }
            if (tid == 0) n_act = 0;
            // predict every member to tn from its own time; list the active
            for (int k = tid; k < n; k += blockDim.x) {
                const double hs = sgn * (double)(tn - S.ti[k]) * tick;
                const double h6 = hs * (1.0 / 6.0);
                S.ex[k] = S.x[k] + hs * (S.u[k] + hs * (0.5 * S.ax[k] + h6 * S.jx[k]));
                S.ey[k] = S.y[k] + hs * (S.v[k] + hs * (0.5 * S.ay[k] + h6 * S.jy[k]));
                S.ez[k] = S.z[k] + hs * (S.w[k] + hs * (0.5 * S.az[k] + h6 * S.jz[k]));
                S.eu[k] = S.u[k] + hs * (S.ax[k] + 0.5 * hs * S.jx[k]);
                S.ev[k] = S.v[k] + hs * (S.ay[k] + 0.5 * hs * S.jy[k]);
                S.ew[k] = S.w[k] + hs * (S.az[k] + 0.5 * hs * S.jz[k]);
            }
            __syncthreads();
            for (int k = tid; k < n; k += blockDim.x)
                if (S.ti[k] + (1ll << (KMAX - S.lev[k])) == tn) S.act[atomicAdd(&n_act, 1)] = k;
            __syncthreads();
            const int na = n_act;
            const int PA = lanes_per_member(na);
            const int NGA = HTHREADS / PA;
            const int ga = tid / PA, la = tid % PA;
            // evaluate (split over lanes) and correct (lane 0) the active members
            for (int k0 = 0; k0 < na; k0 += NGA) {
                const int slot = k0 + ga;
                const int k = slot < na ? S.act[slot] : 0;
                double a1[6] = {0, 0, 0, 0, 0, 0};
                if (slot < na) herm_part(S, n, k, la, PA, G, m0, tc, h.eps2, a1);
                group_sum(a1, 6, PA);
                if (slot < na && la == 0) {
                    const long long dti = 1ll << (KMAX - S.lev[k]);
                    const double hs = sgn * (double)dti * tick;
                    double a0[3] = {S.ax[k], S.ay[k], S.az[k]};
                    double j0[3] = {S.jx[k], S.jy[k], S.jz[k]};
                    double e[3] = {S.ex[k], S.ey[k], S.ez[k]};
                    double f[3] = {S.eu[k], S.ev[k], S.ew[k]};
                    double a2[3], a3[3], xn[3], un[3];
                    const double ih = 1.0 / hs, ih2 = ih * ih, ih3 = ih2 * ih;
                    const double h3 = hs * hs * hs, h4 = h3 * hs;
                    for (int c = 0; c < 3; ++c) {
                        a2[c] = (-6.0 * (a0[c] - a1[c]) - hs * (4.0 * j0[c] + 2.0 * a1[3 + c])) * ih2;
                        a3[c] = (12.0 * (a0[c] - a1[c]) + 6.0 * hs * (j0[c] + a1[3 + c])) * ih3;
                        xn[c] = e[c] + h4 * (a2[c] * (1.0 / 24.0) + hs * a3[c] * (1.0 / 120.0));
                        un[c] = f[c] + h3 * (a2[c] * (1.0 / 6.0) + hs * a3[c] * (1.0 / 24.0));
                        a2[c] += hs * a3[c];
                    }
                    S.x[k] = xn[0]; S.y[k] = xn[1]; S.z[k] = xn[2];
                    S.u[k] = un[0]; S.v[k] = un[1]; S.w[k] = un[2];
                    S.ax[k] = a1[0]; S.ay[k] = a1[1]; S.az[k] = a1[2];
                    S.jx[k] = a1[3]; S.jy[k] = a1[4]; S.jz[k] = a1[5];
                    S.ti[k] = tn;
                    // Aarseth criterion at the end of the step, then the level
                    double na1 = sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
                    double nj = sqrt(a1[3] * a1[3] + a1[4] * a1[4] + a1[5] * a1[5]);
                    double n2 = sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
                    double n3 = sqrt(a3[0] * a3[0] + a3[1] * a3[1] + a3[2] * a3[2]);
                    double den = nj * n3 + n2 * n2;
                    double dt_c = den > 0.0 ? sqrt(h.eta * (na1 * n2 + nj * nj) / den) : T;
                    int kn = level_of(dt_c, T);
                    const int lv = S.lev[k];
                    if (kn < lv) {  // a larger step: one level, on a commensurate time
                        const int up1 = lv - 1;
                        kn = (tn % (1ll << (KMAX - up1)) == 0) ? up1 : lv;
                    }
                    S.lev[k] = kn;
                }
            }
            ++steps;
        }
        __syncthreads();
        if (capped && tid == 0) atomicOr(d.status, QYM_ST_HERMITE_CAP);
        // item 7: pre-remove the (1-K) part of the coming kick at q1
        for (int k = tid; k < n; k += blockDim.x) {
            S.ex[k] = S.x[k]; S.ey[k] = S.y[k]; S.ez[k] = S.z[k];
        }
        __syncthreads();
        for (int k0 = 0; k0 < n; k0 += NG) {
            int k = k0 + grp;
            double c[3] = {0.0, 0.0, 0.0};
            if (k < n) kcorr_part(S, n, k, lane, P, G, tc, c);
            group_sum(c, 3, P);
            if (k < n && lane == 0) {
                int64_t r = S.ids[k];
                d.q1[r] = S.x[k];
                d.q1[R + r] = S.y[k];
                d.q1[2 * R + r] = S.z[k];
                d.v1[r] = S.u[k] - 0.5 * tau * c[0];
                d.v1[R + r] = S.v[k] - 0.5 * tau * c[1];
                d.v1[2 * R + r] = S.w[k] - 0.5 * tau * c[2];
                d.uf[r] = -1;
            }
        }
        if (tid == 0) {
            atomicAdd(d.ctr + C_SUM_HSTEPS, (unsigned long long)steps);
            atomicMax(d.ctr + C_MAX_HSET, (unsigned long long)steps);
        }
    }
}

cudaError_t hermite_prepare() {
    return cudaFuncSetAttribute(k_hermite, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kHermSmem);
}

cudaError_t launch_hermite(const Dev &d, const qym_params &p, double tau, cudaStream_t st) {
    HermArgs h;
    h.G = p.G;
    h.eps2 = p.eps_H * p.eps_H;
    h.eta = p.eta;
    h.eta_s = p.eta_s;
    h.tau = tau;
    h.max_steps = p.max_hermite_steps;
    k_hermite<<<2 * 152, HTHREADS, kHermSmem, st>>>(d, h);
    return cudaGetLastError();
}

}  // namespace qym
