// hermite.cu -- the close-encounter branch of the hybrid step (Sec. 2.2 and
// Sec. 2.3 items 5-8), one CTA per encounter set, or a thread-block cluster
// (2, 4 or 8 CTAs) for each of the large sets predicted to take longest:
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
// the members whose step ends there are evaluated and corrected, against
// their partners predicted to that time; a partner farther than r_crit
// exerts no force (K = 1), so an FP32 prediction with a bound on its error
// first rules out the pairs that are surely that far, and only the others
// are predicted and evaluated in FP64 (the result is the same as evaluating
// every pair). FP64 instructions issue at one per 64 cycles per warp here, so
// each block step is split by instruction stream across warps: a warp per
// coordinate for predictor and corrector, each pair item on two warps, the
// star's pull on its own warp, fixed-order sums (a cluster's CTAs push their
// parts to each other and add them in rank order, so every copy of the set
// stays bit-identical). Every loop has a cap and reports through the status
// word.
#include <climits>

#include <cooperative_groups.h>

#include "qym_internal.cuh"

namespace qym {
namespace cg = cooperative_groups;

constexpr int HCAP = 320;       // members per set held in shared memory
constexpr int HTHREADS = 256;

// sin and cos of (pi/2) y for y in [0, 1]: y > 1/2 is folded onto 1 - y
// (sin and cos swap), so the argument w = (pi/2) y' stays in [0, pi/4], where
// the Taylor series of sin to w^15 and of cos to w^16 leave truncation errors
// below 7e-17 and 3e-18 (the next terms, w^17/17! and w^18/18!, at pi/4).
struct HalfPi {
    double w, x, x2, x4;  // w = (pi/2) y', y' = y or 1 - y; x = w^2, x^2, x^4
    bool fold;            // y' = 1 - y: sin and cos swap
};
__device__ __forceinline__ HalfPi half_pi_arg(double y) {
    HalfPi a;
    a.fold = y > 0.5;
    a.w = 1.5707963267948966 * (a.fold ? 1.0 - y : y);
    a.x = a.w * a.w;
    a.x2 = a.x * a.x;
    a.x4 = a.x2 * a.x2;
    return a;
}
// both polynomials in x = w^2 by Estrin's scheme (dependent depth 4-5
// instead of 8-9: FP64 operations have long latency on this GPU)
// sin w = w (1 - x/3! + x^2/5! - ... - x^7/15!)
__device__ __forceinline__ double sin_w(const HalfPi &a) {
    const double s01 = fma(-1.0 / 6.0, a.x, 1.0);
    const double s23 = fma(-1.0 / 5040.0, a.x, 1.0 / 120.0);
    const double s45 = fma(-1.0 / 39916800.0, a.x, 1.0 / 362880.0);
    const double s67 = fma(-1.0 / 1307674368000.0, a.x, 1.0 / 6227020800.0);
    const double ps = fma(fma(s67, a.x2, s45), a.x4, fma(s23, a.x2, s01));
    return a.w * ps;
}
// cos w = 1 - x/2! + x^2/4! - ... + x^8/16!
__device__ __forceinline__ double cos_w(const HalfPi &a) {
    const double c01 = fma(-0.5, a.x, 1.0);
    const double c23 = fma(-1.0 / 720.0, a.x, 1.0 / 24.0);
    const double c45 = fma(-1.0 / 3628800.0, a.x, 1.0 / 40320.0);
    const double c67 = fma(-1.0 / 87178291200.0, a.x, 1.0 / 479001600.0);
    const double c8 = (1.0 / 20922789888000.0) * (a.x4 * a.x4);
    return fma(fma(c67, a.x2, c45), a.x4, fma(c23, a.x2, c01)) + c8;
}
__device__ __forceinline__ void sincos_half_pi(double y, double &sn, double &cs) {
    const HalfPi a = half_pi_arg(y);
    const double sw = sin_w(a), pc = cos_w(a);
    sn = a.fold ? pc : sw;
    cs = a.fold ? sw : pc;
}

// Constants of the transition function of one set: K(y) = sin(pi y / 2) with
// y = 1.1 s / r_crit - 0.1 (Sec. 2.1), so y = a s - 0.1 and dy/ds = a.
struct TransC {
    double rc2;  // r_crit^2: K = 1 (and K' = K'' = 0) beyond
    double a;    // 1.1 / r_crit
    double c;    // (pi / 2) a: K' = c cos, K'' = -c^2 sin
    double nc2;  // -c^2
    __device__ __forceinline__ explicit TransC(double rc)
        : rc2(rc * rc), a(1.1 / rc), c(0.5 * kPi * (1.1 / rc)), nc2(-c * c) {}
};

// the transition's argument y = 1.1 s / r_crit - 0.1
__device__ __forceinline__ double trans_y(double s, const TransC &tc) { return fma(tc.a, s, -0.1); }

// K and its first and second derivatives with respect to s
__device__ __forceinline__ void transition(double s, const TransC &tc, double &K, double &Kp,
                                           double &Kpp) {
    const double y = trans_y(s, tc);
    if (y <= 0.0) {
        K = 0.0; Kp = 0.0; Kpp = 0.0;
    } else if (y >= 1.0) {
        K = 1.0; Kp = 0.0; Kpp = 0.0;
    } else {
        double sn, cs;
        sincos_half_pi(y, sn, cs);
        K = sn;
        Kp = tc.c * cs;
        Kpp = tc.nc2 * sn;
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

// shared memory of k_hermite, at file scope so that every array of a set's
// state is a constant offset (no base pointers held in registers or passed
// through the stack of the per-set function)
extern __shared__ __align__(16) unsigned char g_hsmem[];

// CTAs of a cluster sharing one large set: 2, 4 or 8 (one lane group of 8
// pushes), chosen per context at launch; buffers are sized for the largest
constexpr int CLMAX = 8;
#ifndef QYM_HERM_NBIG
#define QYM_HERM_NBIG 24
#endif
constexpr int NBIG = QYM_HERM_NBIG;  // sets of at least this many members use a whole cluster
#ifndef QYM_HERM_F32MIN
#define QYM_HERM_F32MIN 64
#endif
// partners of a CTA plus active members above which the FP32 prediction
// screens the partners before the FP64 one
constexpr int F32MIN = QYM_HERM_F32MIN;
constexpr int ACH = 64;    // active members per force round (exchange, correction)
constexpr int RSL = 16;    // members per force round on a cluster (receive buffer slots)

constexpr int KMAX = 48;

// corrector constants of a level's step h (signed), rows of HermSmem::lvt:
// a2 = (-6 d - h (4 j0 + 2 j1)) / h^2 = A2D d + A2J0 j0 + A2J1 j1,
// a3 = (12 d + 6 h (j0 + j1)) / h^3 = A3D d + A3J (j0 + j1),
// x1 = x_p + h^4/24 a2 + h^5/120 a3, v1 = v_p + h^3/6 a2 + h^4/24 a3,
// and a2 at the end of the step, a2 + h a3 (d = a0 - a1)
enum LvConst : int { LV_H = 0, LV_A2D, LV_A2J0, LV_A2J1, LV_A3D, LV_A3J, LV_H4, LV_H5, LV_H3, LV_N };

struct HermSmem {
    double *ex, *ey, *ez, *eu, *ev, *ew;      // evaluation point of every member
    double *gm;                               // -G m of every member
    double *x, *y, *z, *u, *v, *w;            // state at the member's own time
    double *ax, *ay, *az, *jx, *jy, *jz;      // a, adot at the member's own time
    double *pr;                               // per-lane partial a, adot [6][HTHREADS]
    double *rb;                               // partials received from each CTA [2][CL][6][RSL]
    double *a1s;                              // a, adot of the round's active members [6][ACH]
    double *lvt;                              // corrector constants per level [LV_N][KMAX + 1]
    long long *ti;                            // member time in ticks
    float *f;                                 // x..z, u..w, ax..az, jx..jz cut to FP32 [12][HCAP]
    float *px, *py, *pz, *pd;                 // FP32 prediction and its error bound
    float *cf;                                // step criterion inputs [12][ACH]
    int32_t *lev;                             // member level: step = tau 2^-lev
    int32_t *act;                             // members whose step ends now
    int32_t *ids;
    int32_t *need;                            // member needed in FP64 at this block time
    int32_t *nl;                              // per coordinate warp: those members [3][HCAP]
                                              // (need and nl also hold the two-warp force's
                                              // exchange slots, [2][3][96] doubles)
};

__device__ __forceinline__ HermSmem carve(void *base) {
    double *p = (double *)base;
    HermSmem s;
    s.ex = p; p += HCAP; s.ey = p; p += HCAP; s.ez = p; p += HCAP;
    s.eu = p; p += HCAP; s.ev = p; p += HCAP; s.ew = p; p += HCAP;
    s.gm = p; p += HCAP;
    s.x = p; p += HCAP; s.y = p; p += HCAP; s.z = p; p += HCAP;
    s.u = p; p += HCAP; s.v = p; p += HCAP; s.w = p; p += HCAP;
    s.ax = p; p += HCAP; s.ay = p; p += HCAP; s.az = p; p += HCAP;
    s.jx = p; p += HCAP; s.jy = p; p += HCAP; s.jz = p; p += HCAP;
    s.pr = p; p += 6 * HTHREADS;
    s.rb = p; p += 2 * CLMAX * 6 * RSL;
    s.a1s = p; p += 6 * ACH;
    s.lvt = p; p += LV_N * (KMAX + 1);
    s.ti = (long long *)p; p += HCAP;
    float *fp = (float *)p;
    s.f = fp; fp += 12 * HCAP;
    s.px = fp; fp += HCAP; s.py = fp; fp += HCAP; s.pz = fp; fp += HCAP; s.pd = fp; fp += HCAP;
    s.cf = fp; fp += 12 * ACH;
    int32_t *ip = (int32_t *)fp;
    s.lev = ip; ip += HCAP;
    s.act = ip; ip += HCAP;
    s.ids = ip; ip += HCAP;
    s.need = ip; ip += HCAP;
    s.nl = ip;
    return s;
}
constexpr size_t kHermSmem =
    sizeof(double) * (HCAP * 20 + 6 * HTHREADS + 2 * CLMAX * 6 * RSL + 6 * ACH + LV_N * (KMAX + 1)) +
    sizeof(float) * (16 * HCAP + 12 * ACH) + sizeof(int32_t) * HCAP * 7;
static_assert(2 * 3 * 96 * sizeof(double) <= 4 * HCAP * sizeof(int32_t),
              "the two-warp force's exchange slots overlay need and nl");
// two CTAs per SM (228 KB of shared memory, 1 KB of it per CTA reserved)
static_assert(2 * (kHermSmem + 1024) <= 228 * 1024, "Hermite shared memory above two CTAs per SM");

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

// Work split inside a CTA: each member of a group of n is handled by P
// consecutive lanes (P a power of two, P * n <= HTHREADS when possible); lane
// l of a member's group takes the partners lo + l, lo + l + P, ... below hi;
// the group's partial sums are combined with warp shuffles in a fixed tree.
__device__ __forceinline__ int lanes_per_member(int n, int partners) {
    int p = 32;
    while (p > 1 && (p * n > HTHREADS || p >= 2 * partners)) p >>= 1;
    return p;
}

__device__ __forceinline__ void group_sum(double *v, int cnt, int P) {
    for (int off = P >> 1; off > 0; off >>= 1)
        for (int c = 0; c < cnt; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
}

// partial (1-K)-weighted pair acceleration of member k at the evaluation
// point, unsmoothed (the kick used the bare separation):
// sum_l -G m_l q_kl / q^3 [1 - K + q K'] over the partners of this lane
__device__ void kcorr_part(const HermSmem &S, int lo, int hi, int k, int l0, int P,
                           const TransC &tc, double *c) {
    c[0] = c[1] = c[2] = 0.0;
    for (int l = lo + l0; l < hi; l += P) {
        if (l == k) continue;
        double qx = S.ex[k] - S.ex[l], qy = S.ey[k] - S.ey[l], qz = S.ez[k] - S.ez[l];
        double q2 = qx * qx + qy * qy + qz * qz;
        if (q2 >= tc.rc2) continue;  // K = 1 beyond r_crit: no (1-K) part
        const double qi = rsqrt(q2);
        const double q = q2 * qi;
        double K, Kp, Kpp;
        transition(q, tc, K, Kp, Kpp);
        double wgt = S.gm[l] * (qi * qi * qi) * (1.0 - K + q * Kp);
        c[0] += wgt * qx;
        c[1] += wgt * qy;
        c[2] += wgt * qz;
    }
}

// partial Hermite acceleration and jerk of member k at the evaluation point
// (Sec. 2.2): with `star`, the star term on lane 0 of the group; the pair
// terms with the transition bracket over this lane's partners (one
// reciprocal square root per pair: q = q2 / sqrt(q2), 1/q^3, 1/q^2)
__device__ void herm_part(const HermSmem &S, int lo, int hi, int k, int l0, int P, bool star,
                          double gm0, const TransC &tc, double eps2, double *aj) {
    const double xk = S.ex[k], yk = S.ey[k], zk = S.ez[k];
    const double uk = S.eu[k], vk = S.ev[k], wk = S.ew[k];
    for (int c = 0; c < 6; ++c) aj[c] = 0.0;
    if (star && l0 == 0) {  // star, fixed at the origin
        double s2 = xk * xk + yk * yk + zk * zk + eps2;
        double si = rsqrt(s2);
        double si2 = si * si;
        double rv = xk * uk + yk * vk + zk * wk;
        double c = gm0 * (si2 * si);
        double t = 3.0 * rv * si2;
        aj[0] = c * xk; aj[1] = c * yk; aj[2] = c * zk;
        aj[3] = c * (uk - t * xk); aj[4] = c * (vk - t * yk); aj[5] = c * (wk - t * zk);
    }
    for (int l = lo + l0; l < hi; l += P) {
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
        double cl = S.gm[l] * (qi2 * qi);
        double tl = 3.0 * rvl * qi2;
        aj[0] += cl * br * qx; aj[1] += cl * br * qy; aj[2] += cl * br * qz;
        aj[3] += cl * (rvl * qx * Kpp + (px - tl * qx) * br);
        aj[4] += cl * (rvl * qy * Kpp + (py - tl * qy) * br);
        aj[5] += cl * (rvl * qz * Kpp + (pz - tl * qz) * br);
    }
}

// 2^e as a double, -1022 <= e <= 1023 (from the bits: no FP64 instruction)
__device__ __forceinline__ double pow2d(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// v 2^s as a float, the mantissa truncated, by integer operations on the bits
// (no FP64 instruction): signed zero below the float normal range, +-FLT_MAX
// above it. Used only for the step-size criterion.
__device__ __forceinline__ float to_float_scaled(double v, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int eb = (int)((b >> 52) & 0x7ff);
    if (eb == 0) return __uint_as_float(sign);
    const int e = eb - 1023 + s;
    if (e < -126) return __uint_as_float(sign);
    if (e > 127) return __uint_as_float(sign | 0x7f7fffffu);
    return __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// Step levels by the Aarseth criterion,
// dt_c^2 = eta (|a| |a2| + |j|^2) / (|j| |a3| + |a2|^2), with a, j the new
// acceleration and jerk and a2, a3 the corrector's derivatives: the new level
// is the smallest k with T 2^-k <= dt_c. With g = 2^-lv (lv the level of the
// step just taken), j g, a2 g^2 and a3 g^3 are accelerations scaled alike and
// r = eta (|a||a2 g^2| + |j g|^2) / (|j g||a3 g^3| + |a2 g^2|^2) =
// (dt_c / (T g))^2 T^2, so T 2^-k <= dt_c is T^2 4^(lv - k) <= r. The powers
// of g are applied exactly through the exponents when the inputs are cut to
// FP32, and the criterion runs in FP32 (an FP64 operation costs about fifteen
// FP32 ones here). It only picks a power of two: a level different from an
// FP64 evaluation needs dt_c within ~1e-7 of a level boundary.
// level_from: that level from the criterion's inputs as floats f[c * ACH]
// (stride ACH): a (3), j g (3), a2 g^2 (3), a3 g^3 (3)
__device__ __forceinline__ int level_from(const float *f, int lv, float eta, float T2) {
    float q[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const float x = f[(3 * g) * ACH], y = f[(3 * g + 1) * ACH], z = f[(3 * g + 2) * ACH];
        q[g] = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    }
    const float num = eta * fmaf(q[0], q[2], q[1] * q[1]);
    const float den = fmaf(q[1], q[3], q[2] * q[2]);
    if (!(den > 0.0f)) return 0;
    if (!(num > 0.0f)) return KMAX;
    const float r = num / den;
    if (!(r < INFINITY)) return 0;
    int er, et;
    const float fr = frexpf(r, &er), ft = frexpf(T2, &et);
    const int dd = er - et;
    const int m = (dd & 1) ? (dd - 1) >> 1 : ((ft <= fr) ? dd >> 1 : (dd >> 1) - 1);
    const int k = lv - m;
    return k < 0 ? 0 : (k > KMAX ? KMAX : k);
}

// component c of member k predicted from its own time to tn
__device__ __forceinline__ void predict_c(const HermSmem &S, int k, int c, long long tn,
                                          double stick) {
    const double hs = (double)(tn - S.ti[k]) * stick;
    const double h6 = hs * (1.0 / 6.0);
    double *x = c == 0 ? S.x : (c == 1 ? S.y : S.z);
    double *u = c == 0 ? S.u : (c == 1 ? S.v : S.w);
    double *a = c == 0 ? S.ax : (c == 1 ? S.ay : S.az);
    double *j = c == 0 ? S.jx : (c == 1 ? S.jy : S.jz);
    double *ex = c == 0 ? S.ex : (c == 1 ? S.ey : S.ez);
    double *eu = c == 0 ? S.eu : (c == 1 ? S.ev : S.ew);
    const double ak = a[k], jk = j[k], uk = u[k];
    ex[k] = x[k] + hs * (uk + hs * (0.5 * ak + h6 * jk));
    eu[k] = uk + hs * (ak + 0.5 * hs * jk);
}

// FP32 copies of member k's state (truncated: within 2^-23 of the FP64
// values, relative), kept beside the FP64 state for the FP32 prediction
__device__ __forceinline__ void store_f32(const HermSmem &S, int k) {
    const double *src[12] = {S.x, S.y, S.z, S.u, S.v, S.w, S.ax, S.ay, S.az, S.jx, S.jy, S.jz};
#pragma unroll
    for (int q = 0; q < 12; ++q) S.f[q * HCAP + k] = to_float_scaled(src[q][k], 0);
}

// Member k's position predicted to tn in FP32 from the copies, by the same
// Horner form as the FP64 predictor, and a bound pd on its distance from the
// FP64 prediction. Each input is within 2^-23 of its FP64 value (hs within
// 3 2^-24), and each of the three fmaf roundings adds 2^-24 relative to the
// magnitude of what it rounds, so every term of the polynomial is within
// 15 2^-24 < 2^-20 of its FP64 value, relative to the sum M of the terms'
// magnitudes; pd = 2^-18 (M_x + M_y + M_z) (plus 1e-30 for inputs flushed
// to zero) keeps a factor 4 to spare.
__device__ __forceinline__ void predict_f32(const HermSmem &S, int k, long long tn, float stickf) {
    const float hs = (float)(tn - S.ti[k]) * stickf;
    const float ah = fabsf(hs);
    const float h6 = hs * (1.0f / 6.0f), ah6 = ah * (1.0f / 6.0f);
    float *out[3] = {S.px, S.py, S.pz};
    float m = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float xk = S.f[c * HCAP + k], uk = S.f[(3 + c) * HCAP + k];
        const float ak = S.f[(6 + c) * HCAP + k], jk = S.f[(9 + c) * HCAP + k];
        out[c][k] = fmaf(hs, fmaf(hs, fmaf(h6, jk, 0.5f * ak), uk), xk);
        m += fmaf(ah, fmaf(ah, fmaf(ah6, fabsf(jk), 0.5f * fabsf(ak)), fabsf(uk)), fabsf(xk));
    }
    S.pd[k] = fmaf(m, 0x1p-18f, 1e-30f);
}

// false only when members k and l, both predicted in FP32 to the same time,
// are surely farther apart than r_crit in their FP64 predictions: then the
// FP64 pair test (q^2 + eps^2 >= r_crit^2) rejects the pair as well. The
// separation is within 2^-21 (relative) of that of the FP32 positions, which
// differ from the FP64 ones by at most pd_k + pd_l; rcf >= r_crit (1 + 2^-20).
// Written with explicit roundings so that every call gives the same answer.
__device__ __forceinline__ bool maybe_near(const HermSmem &S, int k, int l, float rcf) {
    const float dx = __fsub_rn(S.px[k], S.px[l]);
    const float dy = __fsub_rn(S.py[k], S.py[l]);
    const float dz = __fsub_rn(S.pz[k], S.pz[l]);
    const float q = __fsqrt_rn(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))));
    return __fmul_rn(q, 1.0f - 0x1p-20f) <= __fadd_rn(rcf, __fadd_rn(S.pd[k], S.pd[l]));
}

// Pieces of the pair force shared by the one-lane form (herm_item) and the
// two-warp form of the block step, written with explicit fused operations
// so that both give the same bits: q^2 + eps^2; q . p; cl = -G m_l / q^3;
// br = 1 - K + q K'; the acceleration cl br q and the jerk cl br p + cq q
// with cq = cl (q . p) (K'' - 3 br / q^2)
__device__ __forceinline__ double pair_q2(double qx, double qy, double qz, double eps2) {
    return fma(qx, qx, fma(qy, qy, fma(qz, qz, eps2)));
}
__device__ __forceinline__ double pair_rv(double qx, double qy, double qz, double px, double py,
                                          double pz) {
    return fma(qx, px, fma(qy, py, qz * pz));
}
__device__ __forceinline__ double pair_cl(double gml, double qi, double qi2) {
    return gml * (qi2 * qi);
}
__device__ __forceinline__ double pair_br(double sq, double K, double Kp) {
    return fma(sq, Kp, 1.0 - K);
}
// m3qi2 = -3 / q^2
__device__ __forceinline__ double pair_cq(double cl, double rvl, double m3qi2, double br,
                                          double Kpp) {
    return (cl * rvl) * fma(m3qi2, br, Kpp);
}

// Hermite a, adot of member k from one item: partner mlo + item of this
// CTA's range (with f32, skipped at once when maybe_near rules it out), or
// the star for item == npart (with `star`)
__device__ __forceinline__ void herm_item(const HermSmem &S, int k, int item, int mlo, int npart,
                                          bool star, double gm0, const TransC &tc, double eps2,
                                          bool f32, float rcf, double *aj) {
    if (item < npart && (mlo + item == k || (f32 && !maybe_near(S, k, mlo + item, rcf)))) return;
    const double xk = S.ex[k], yk = S.ey[k], zk = S.ez[k];
    const double uk = S.eu[k], vk = S.ev[k], wk = S.ew[k];
    if (item == npart) {
        if (!star) return;
        double s2 = xk * xk + yk * yk + zk * zk + eps2;
        double si = rsqrt(s2);
        double si2 = si * si;
        double rv = xk * uk + yk * vk + zk * wk;
        double c = gm0 * (si2 * si);
        double t = 3.0 * rv * si2;
        aj[0] += c * xk; aj[1] += c * yk; aj[2] += c * zk;
        aj[3] += c * (uk - t * xk); aj[4] += c * (vk - t * yk); aj[5] += c * (wk - t * zk);
        return;
    }
    const int l = mlo + item;
    const double qx = xk - S.ex[l], qy = yk - S.ey[l], qz = zk - S.ez[l];
    const double q2 = pair_q2(qx, qy, qz, eps2);
    if (q2 >= tc.rc2) return;  // K = 1, K' = K'' = 0: no force, no jerk
    const double px = uk - S.eu[l], py = vk - S.ev[l], pz = wk - S.ew[l];
    const double qi = rsqrt(q2);
    const double qi2 = qi * qi;
    const double sq = q2 * qi;
    double K, Kp, Kpp;
    transition(sq, tc, K, Kp, Kpp);
    const double rvl = pair_rv(qx, qy, qz, px, py, pz);
    const double cl = pair_cl(S.gm[l], qi, qi2), br = pair_br(sq, K, Kp);
    const double cb = cl * br;
    const double cq = pair_cq(cl, rvl, -3.0 * qi2, br, Kpp);
    aj[0] = fma(cb, qx, aj[0]); aj[1] = fma(cb, qy, aj[1]); aj[2] = fma(cb, qz, aj[2]);
    aj[3] = fma(cb, px, fma(cq, qx, aj[3]));
    aj[4] = fma(cb, py, fma(cq, qy, aj[4]));
    aj[5] = fma(cb, pz, fma(cq, qz, aj[5]));
}

// the pair barrier of warps 2p and 2p + 1 (named barrier 1 + p, 64 threads)
__device__ __forceinline__ void pair_bar(int p) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + p) : "memory");
}

struct HermArgs {
    double G, eps2, eta, eta_s, tau;
    int64_t max_steps;
};

__shared__ int g_next_small;
__shared__ long long g_tn;
__shared__ int g_na;

// Next block time (the earliest end of a member's step) and the members whose
// step ends then, in member order, by one warp; every thread reads (tn, na)
// after the barrier that follows. The end times stay in registers
// between the two passes; the minimum (below 2^49) is taken as the minimum of
// the high words, then of the low words among the lanes that hold it.
__device__ __forceinline__ void next_block(const int32_t *lev, const long long *ti, int32_t *act,
                                           int n) {
    constexpr int NI = HCAP / 32;
    const int wl = threadIdx.x & 31;
    long long te[NI];
    long long t = LLONG_MAX;
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int k = q * 32 + wl;
        te[q] = (k < n) ? ti[k] + (1ll << (KMAX - lev[k])) : LLONG_MAX;
        t = min(t, te[q]);
    }
    const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)(t >> 32));
    const unsigned lo =
        __reduce_min_sync(0xffffffffu, (unsigned)(t >> 32) == hi ? (unsigned)t : 0xffffffffu);
    t = (long long)(((unsigned long long)hi << 32) | lo);
    int na = 0;
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        if (q * 32 >= n) break;
        const bool f = te[q] == t;
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (f) act[na + __popc(b & ((1u << wl) - 1u))] = q * 32 + wl;
        na += __popc(b);
    }
    if (wl == 0) {
        g_tn = t;
        g_na = na;
    }
}

// Copy the member range [lo, hi) of arrays a..: from CTA `r` of the cluster
// into this CTA's shared memory.
__device__ __forceinline__ void pull_range(cg::cluster_group &cl, const HermSmem &S, int r,
                                           int lo, int hi, double *const *arrs, int narr) {
    for (int q = 0; q < narr; ++q) {
        const double *src = cl.map_shared_rank(arrs[q], r);
        for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) arrs[q][k] = src[k];
    }
}

// One set through items 5-7 of the step (Sec. 2.3): K correction at q0,
// Hermite over tau with individual block steps, K correction at q1. With
// COOP the cs CTAs of a cluster share the set: every CTA keeps a full copy of
// the members' state; CTA `rank` evaluates the start-up forces and the K
// corrections of its member range, exchanged once; in each block step it sums
// the forces on the active members from its partner range, all partial sums
// are read from the peers' shared memory in rank order, and every CTA applies
// the same corrector, so the copies stay identical with one cluster barrier
// per exchange round (partials double-buffered).
template <bool COOP, int CLT>
__device__ __noinline__ void hermite_set(const Dev &d, const HermArgs h, int set, int rank,
                                         int cs) {
    const HermSmem S = carve(g_hsmem);
    cg::cluster_group cl = cg::this_cluster();
    const int64_t R = d.rows;
    const int tid = threadIdx.x;
    const int st = d.set_start[set];
    const int n = d.set_start[set + 1] - st;
    if (n < 1) return;
    if (n > HCAP || st + n > d.max_members) {
        if (tid == 0 && rank == 0) atomicOr(d.status, QYM_ST_SET_OVERFLOW);
        if (rank == 0)
            for (int k = tid; k < n && st + k < d.max_members; k += blockDim.x)
                d.uf[d.set_mem[st + k]] = -1;
        return;
    }
    // a system integrated whole by the Hermite this step (whole.cu): its
    // members only leave the union-find
    if (d.wh_flag && d.wh_flag[d.sys_of[d.set_mem[st]]]) {
        if (rank == 0)
            for (int k = tid; k < n; k += blockDim.x) d.uf[d.set_mem[st + k]] = -1;
        return;
    }
    // this CTA's member range (COOP) or all members
    const int mlo = n * rank / cs, mhi = n * (rank + 1) / cs;
    const int P = lanes_per_member(mhi - mlo, n);
    const int NG = HTHREADS / P;
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
    const int64_t star_row = d.offsets[d.sys_of[S.ids[0]]];
    const double gm0 = -h.G * d.m[star_row];
    const TransC tc(d.rcrit[set]);
    const double tau = h.tau;
    // state entering the Kepler drift (after the first kick)
    for (int k = tid; k < n; k += blockDim.x) {
        int64_t r = S.ids[k];
        S.ex[k] = S.x[k] = d.q[r];
        S.ey[k] = S.y[k] = d.q[R + r];
        S.ez[k] = S.z[k] = d.q[2 * R + r];
        S.u[k] = d.v[r];
        S.v[k] = d.v[R + r];
        S.w[k] = d.v[2 * R + r];
        S.gm[k] = -h.G * d.m[r];
    }
    __syncthreads();
    // item 5: remove the (1-K) part of the first kick (own members)
    for (int k0 = mlo; k0 < mhi; k0 += NG) {
        int k = k0 + grp;
        double c[3] = {0.0, 0.0, 0.0};
        if (k < mhi) kcorr_part(S, 0, n, k, lane, P, tc, c);
        group_sum(c, 3, P);
        if (k < mhi && lane == 0) {
            S.u[k] -= 0.5 * tau * c[0];
            S.v[k] -= 0.5 * tau * c[1];
            S.w[k] -= 0.5 * tau * c[2];
        }
    }
    if (COOP) {
        cl.sync();
        double *const arr[3] = {S.u, S.v, S.w};
        for (int r = 0; r < cs; ++r)
            if (r != rank) pull_range(cl, S, r, n * r / cs, n * (r + 1) / cs, arr, 3);
        cl.sync();
    } else {
        __syncthreads();
    }
    for (int k = tid; k < n; k += blockDim.x) {
        S.eu[k] = S.u[k]; S.ev[k] = S.v[k]; S.ew[k] = S.w[k];
    }
    __syncthreads();
    // start-up: a, adot at t = 0 and the levels from eta_s |a| / |adot|
    const double sgn = tau >= 0.0 ? 1.0 : -1.0;
    const double T = fabs(tau);
    const long long TT = 1ll << KMAX;
    const double tick = T / (double)TT;
    const double inv_T = 1.0 / T;
    for (int k0 = mlo; k0 < mhi; k0 += NG) {
        int k = k0 + grp;
        double aj[6] = {0, 0, 0, 0, 0, 0};
        if (k < mhi) herm_part(S, 0, n, k, lane, P, true, gm0, tc, h.eps2, aj);
        group_sum(aj, 6, P);
        if (k < mhi && lane == 0) {
            S.ax[k] = aj[0]; S.ay[k] = aj[1]; S.az[k] = aj[2];
            S.jx[k] = aj[3]; S.jy[k] = aj[4]; S.jz[k] = aj[5];
            double jn = sqrt(aj[3] * aj[3] + aj[4] * aj[4] + aj[5] * aj[5]);
            double dt_c = jn > 0.0 ? h.eta_s * sqrt(aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]) / jn : T;
            S.lev[k] = level_of(dt_c, T);
            S.ti[k] = 0;
        }
    }
    if (COOP) {
        cl.sync();
        double *const arr[6] = {S.ax, S.ay, S.az, S.jx, S.jy, S.jz};
        for (int r = 0; r < cs; ++r) {
            if (r == rank) continue;
            const int lo = n * r / cs, hi = n * (r + 1) / cs;
            pull_range(cl, S, r, lo, hi, arr, 6);
            const int32_t *pl = cl.map_shared_rank(S.lev, r);
            for (int k = lo + tid; k < hi; k += blockDim.x) {
                S.lev[k] = pl[k];
                S.ti[k] = 0;
            }
        }
        cl.sync();
    }
    // Block steps. FP64 instructions are issued at about one warp-instruction
    // per 64 cycles per SM sub-partition here, whatever the number of active
    // lanes, so the work is split by instruction stream across warps (which
    // the sub-partitions serve in parallel): one warp per coordinate for the
    // predictor and the corrector, several warps per member for the forces,
    // one warp per (member, component) for the sums.
    const int warp = tid >> 5, wl = tid & 31;
    const double stick = sgn * tick;
    const double T2d = T * T, T3 = T2d * T, T4 = T3 * T;
    const double iT2 = inv_T * inv_T, iT3 = iT2 * inv_T;
    const float T2f = (float)T2d, etaf = (float)h.eta;
    const float stickf = (float)stick;
    const float rcf = __double2float_ru(d.rcrit[set] * (1.0 + 0x1p-20));
    const int npart = mhi - mlo;
    // the largest range of the cluster: every CTA derives its lane layout and
    // its round count from it, so all CTAs pass the same cluster barriers and
    // lay out their partial sums alike
    const int npmax = (n + cs - 1) / cs;
    // FP32 copies of the start-up state; the corrector's constants per level
    // (products with powers of two, so the table holds the same values)
    __syncthreads();
    for (int k = tid; k < n; k += blockDim.x) store_f32(S, k);
    for (int lv = tid; lv <= KMAX; lv += blockDim.x) {
        double *L = S.lvt + lv;
        const double ih = sgn * inv_T * pow2d(lv), ih2 = iT2 * pow2d(2 * lv);
        L[LV_H * (KMAX + 1)] = sgn * T * pow2d(-lv);
        L[LV_A2D * (KMAX + 1)] = -6.0 * ih2;
        L[LV_A2J0 * (KMAX + 1)] = -4.0 * ih;
        L[LV_A2J1 * (KMAX + 1)] = -2.0 * ih;
        L[LV_A3D * (KMAX + 1)] = 12.0 * (sgn * iT3 * pow2d(3 * lv));
        L[LV_A3J * (KMAX + 1)] = 6.0 * ih2;
        L[LV_H4 * (KMAX + 1)] = (T4 * pow2d(-4 * lv)) * (1.0 / 24.0);
        L[LV_H5 * (KMAX + 1)] = (sgn * T4 * T * pow2d(-5 * lv)) * (1.0 / 120.0);
        L[LV_H3 * (KMAX + 1)] = (sgn * T3 * pow2d(-3 * lv)) * (1.0 / 6.0);
    }
    const bool with_star = rank == 0;
    int64_t steps = 0;
    bool capped = false;
    int buf = 0;
    // the first block time; later ones are found by warp 3 right after it sets
    // the new levels (it wrote every value the scan reads), so one barrier per
    // block step publishes them
    if (warp == 3) next_block(S.lev, S.ti, S.act, n);
    for (;;) {
        __syncthreads();
        const long long tn = g_tn;
        if (tn > TT) break;  // every member has reached tau
        if (steps >= h.max_steps) { capped = true; break; }
        const int na = g_na;
        // Predict this CTA's partners and the active members to tn. Up to two
        // warps' worth, FP64 passes over them all (one warp per coordinate);
        // above that the FP32 prediction first rules out the partners that are
        // surely beyond r_crit of every active member.
        const bool f32 = npmax + na > F32MIN;
        if (!f32) {
            if (warp < 3) {
                for (int i = wl; i < npart + na; i += 32) {
                    int k = mlo + i;
                    if (i >= npart) k = S.act[i - npart];
                    if (i < npart || k < mlo || k >= mhi) predict_c(S, k, warp, tn, stick);
                }
            }
        } else {
            for (int k = tid; k < n; k += HTHREADS) S.need[k] = 0;
            for (int i = tid; i < npart + na; i += HTHREADS) {
                int k = mlo + i;
                if (i >= npart) {
                    k = S.act[i - npart];
                    if (k >= mlo && k < mhi) continue;
                }
                predict_f32(S, k, tn, stickf);
            }
            __syncthreads();
            // members needed in FP64: the active ones and the partners that
            // maybe_near does not rule out for some active member
            for (int i = tid; i < na; i += HTHREADS) S.need[S.act[i]] = 1;
            for (int p = tid; p < na * npart; p += HTHREADS) {
                const int ia = p / npart, l = mlo + (p - ia * npart);
                const int k = S.act[ia];
                if (l != k && maybe_near(S, k, l, rcf)) S.need[l] = 1;
            }
            __syncthreads();
            // their FP64 prediction, one warp per coordinate, each warp listing
            // them in member order for itself
            if (warp < 3) {
                int32_t *nl = S.nl + warp * HCAP;
                int nn = 0;
                for (int k0 = 0; k0 < n; k0 += 32) {
                    const int k = k0 + wl;
                    const bool f = k < n && S.need[k] != 0;
                    const unsigned b = __ballot_sync(0xffffffffu, f);
                    if (f) nl[nn + __popc(b & ((1u << wl) - 1u))] = k;
                    nn += __popc(b);
                }
                __syncwarp();
                for (int i = wl; i < nn; i += 32) predict_c(S, nl[i], warp, tn, stick);
            }
        }
        __syncthreads();
        for (int a0 = 0; a0 < na; a0 += ACH) {
            const int nc = min(ACH, na - a0);
            // pair items on warps 0-6 (LA lanes per member), the star's pull
            // (rank 0) on warp 7, so neither path diverges inside a warp
            int LA = 1;
            while (LA < npmax && LA < 64) LA <<= 1;
            // slots per round (warp 7 holds one star per slot; on a cluster at
            // most RSL, the receive buffer's width). When the round's members
            // fit three warps' worth of lanes, each pair item runs on two warps
            // of different sub-partitions (pair_bar): the even warp takes sin,
            // q . p and the acceleration, the odd warp cos and the jerk, which
            // shortens each warp's FP64 instruction stream by about a third.
            // Either way every partial is the same sum in the same order.
            const int NG = min(COOP ? RSL : 32, (HTHREADS - 32) / LA);
            const bool paired = nc <= min(COOP ? RSL : 32, 96 / LA);
            const int NR = paired ? nc : NG;
            for (int s0 = 0; s0 < nc; s0 += NR) {
                const int cnt = min(NR, nc - s0);
                double *prb = S.pr;
                if (!paired) {
                    double aj[6] = {0, 0, 0, 0, 0, 0};
                    if (warp < 7) {
                        const int slot = s0 + tid / LA, la = tid % LA;
                        if (slot < s0 + cnt) {
                            const int k = S.act[a0 + slot];
                            for (int it = la; it < npart; it += LA)
                                herm_item(S, k, it, mlo, npart, false, gm0, tc, h.eps2, f32, rcf, aj);
                        }
                    } else if (with_star && wl < cnt) {
                        herm_item(S, S.act[a0 + s0 + wl], npart, mlo, npart, true, gm0, tc, h.eps2,
                                  f32, rcf, aj);
                    }
#pragma unroll
                    for (int c = 0; c < 6; ++c) prb[c * HTHREADS + tid] = aj[c];
                } else if (warp < 6) {
                    const int role = warp & 1, vl = (warp >> 1) * 32 + wl;
                    const int slot = vl / LA, la = vl - slot * LA;
                    const bool sv = slot < cnt;
                    const int k = sv ? S.act[a0 + slot] : 0;
                    // exchange slots [2][3][96] (sin, q . p, cos): the FP32
                    // pass's lists, which are idle until the next block time
                    double *xch = reinterpret_cast<double *>(S.need);
                    double acc[3] = {0.0, 0.0, 0.0};
                    int par = 0;
                    for (int it0 = 0; it0 < npart; it0 += LA) {
                        const int l = mlo + it0 + la;
                        double *xs = xch + par * (3 * 96);
                        bool valid = sv && it0 + la < npart && l != k &&
                                     (!f32 || maybe_near(S, k, l, rcf));
                        double qx = 0.0, qy = 0.0, qz = 0.0, qi2 = 0.0, sq = 0.0;
                        double y = 0.0, mine = 0.0, cl = 0.0, m3 = 0.0, px = 0.0, py = 0.0, pz = 0.0;
                        bool fold = false;
                        if (valid) {
                            qx = S.ex[k] - S.ex[l];
                            qy = S.ey[k] - S.ey[l];
                            qz = S.ez[k] - S.ez[l];
                            const double q2 = pair_q2(qx, qy, qz, h.eps2);
                            valid = q2 < tc.rc2;  // beyond r_crit: no force, no jerk
                            if (valid) {
                                const double qi = rsqrt(q2);
                                qi2 = qi * qi;
                                sq = q2 * qi;
                                y = trans_y(sq, tc);
                                if (y > 0.0 && y < 1.0) {
                                    const HalfPi arg = half_pi_arg(y);
                                    fold = arg.fold;
                                    mine = role == 0 ? sin_w(arg) : cos_w(arg);
                                    xs[2 * 96 * role + vl] = mine;
                                }
                                // what does not wait for the partner warp's
                                // polynomial is done before the barrier
                                cl = pair_cl(S.gm[l], qi, qi2);
                                px = S.eu[k] - S.eu[l];
                                py = S.ev[k] - S.ev[l];
                                pz = S.ew[k] - S.ew[l];
                                if (role == 0)
                                    xs[96 + vl] = pair_rv(qx, qy, qz, px, py, pz);
                                else
                                    m3 = -3.0 * qi2;
                            }
                        }
                        __syncwarp();
                        pair_bar(warp >> 1);
                        if (valid) {
                            double K = 0.0, Kp = 0.0, Kpp = 0.0;
                            if (y >= 1.0) {
                                K = 1.0;
                            } else if (y > 0.0) {
                                const double sw = role == 0 ? mine : xs[vl];
                                const double pc = role == 1 ? mine : xs[2 * 96 + vl];
                                const double sn = fold ? pc : sw, cs = fold ? sw : pc;
                                K = sn;
                                Kp = tc.c * cs;
                                Kpp = tc.nc2 * sn;
                            }
                            const double br = pair_br(sq, K, Kp);
                            const double cb = cl * br;
                            if (role == 0) {
                                acc[0] = fma(cb, qx, acc[0]);
                                acc[1] = fma(cb, qy, acc[1]);
                                acc[2] = fma(cb, qz, acc[2]);
                            } else {
                                const double cq = pair_cq(cl, xs[96 + vl], m3, br, Kpp);
                                acc[0] = fma(cb, px, fma(cq, qx, acc[0]));
                                acc[1] = fma(cb, py, fma(cq, qy, acc[1]));
                                acc[2] = fma(cb, pz, fma(cq, qz, acc[2]));
                            }
                        }
                        par ^= 1;
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) prb[(3 * role + c) * HTHREADS + vl] = acc[c];
                } else if (warp == 7) {
                    double aj[6] = {0, 0, 0, 0, 0, 0};
                    if (with_star && wl < cnt)
                        herm_item(S, S.act[a0 + s0 + wl], npart, mlo, npart, true, gm0, tc, h.eps2,
                                  f32, rcf, aj);
#pragma unroll
                    for (int c = 0; c < 6; ++c) prb[c * HTHREADS + tid] = aj[c];
                }
                if (COOP) {
                    // This CTA's part of every (member, component): its LA lanes
                    // summed by a group of eight lanes in a fixed order (plus the
                    // star's pull on rank 0), stored by lane g into CTA g's
                    // receive buffer under this rank; after the cluster barrier
                    // every CTA adds the CTAs' parts in rank order. Receive
                    // buffers are double-buffered: a CTA stores into this one
                    // again only after the next round's cluster barrier, which
                    // every CTA passes after reading it.
                    __syncthreads();
                    double *rbb = S.rb + buf * (CLT * 6 * RSL);
                    const int g = wl & 7;
                    for (int pi0 = warp * 4; pi0 < 6 * cnt; pi0 += HTHREADS / 8) {
                        const int pi = pi0 + (wl >> 3);
                        const bool live = pi < 6 * cnt;
                        const int sl = pi / 6, c = pi - 6 * sl;
                        double v = 0.0;
                        if (live)
                            for (int m = g; m < LA; m += 8) v += prb[c * HTHREADS + sl * LA + m];
                        v += __shfl_xor_sync(0xffffffffu, v, 1);
                        v += __shfl_xor_sync(0xffffffffu, v, 2);
                        v += __shfl_xor_sync(0xffffffffu, v, 4);
                        if (live && with_star) v += prb[c * HTHREADS + 224 + sl];
                        if (live && g < CLT) cl.map_shared_rank(rbb, g)[(rank * 6 + c) * RSL + sl] = v;
                    }
                    cl.sync();
                    for (int pi = tid; pi < 6 * cnt; pi += HTHREADS) {
                        const int sl = pi / 6, c = pi - 6 * sl;
                        double pv[CLT];
#pragma unroll
                        for (int r = 0; r < CLT; ++r) pv[r] = rbb[(r * 6 + c) * RSL + sl];
                        // pairwise tree: rank r with rank r + w, halving w
#pragma unroll
                        for (int w = CLT / 2; w >= 1; w >>= 1) {
#pragma unroll
                            for (int r = 0; r < w; ++r) pv[r] += pv[r + w];
                        }
                        S.a1s[c * ACH + s0 + sl] = pv[0];
                    }
                    buf ^= 1;
                } else {
                    __syncthreads();
                    // sums over the LA lanes of each (member, component), one
                    // warp each, in a fixed order
                    for (int pi = warp; pi < 6 * cnt; pi += HTHREADS / 32) {
                        const int sl = pi / 6, c = pi - 6 * sl;
                        const double *col = prb + c * HTHREADS + sl * LA;
                        double v = 0.0;
                        for (int m = wl; m < LA; m += 32) v += col[m];
                        for (int off = (LA < 32 ? LA : 32) >> 1; off > 0; off >>= 1)
                            v += __shfl_xor_sync(0xffffffffu, v, off);
                        if (wl == 0) S.a1s[c * ACH + s0 + sl] = v + prb[c * HTHREADS + 224 + sl];
                    }
                }
                __syncthreads();
            }
            // corrector, one warp per coordinate (the same in every CTA)
            if (warp < 3) {
                const int c = warp;
                double *xa = c == 0 ? S.x : (c == 1 ? S.y : S.z);
                double *ua = c == 0 ? S.u : (c == 1 ? S.v : S.w);
                double *aa = c == 0 ? S.ax : (c == 1 ? S.ay : S.az);
                double *ja = c == 0 ? S.jx : (c == 1 ? S.jy : S.jz);
                const double *ea = c == 0 ? S.ex : (c == 1 ? S.ey : S.ez);
                const double *fa = c == 0 ? S.eu : (c == 1 ? S.ev : S.ew);
                for (int sl = wl; sl < nc; sl += 32) {
                    const int k = S.act[a0 + sl];
                    const int lv = S.lev[k];
                    const double *L = S.lvt + lv;
                    constexpr int LS = KMAX + 1;
                    const double a1c = S.a1s[c * ACH + sl], j1c = S.a1s[(3 + c) * ACH + sl];
                    const double d = aa[k] - a1c, j0c = ja[k];
                    const double a2 =
                        fma(L[LV_A2D * LS], d, fma(L[LV_A2J0 * LS], j0c, L[LV_A2J1 * LS] * j1c));
                    const double a3 = fma(L[LV_A3D * LS], d, L[LV_A3J * LS] * (j0c + j1c));
                    const double xn = fma(L[LV_H4 * LS], a2, fma(L[LV_H5 * LS], a3, ea[k]));
                    const double un = fma(L[LV_H3 * LS], a2, fma(L[LV_H4 * LS], a3, fa[k]));
                    xa[k] = xn;
                    ua[k] = un;
                    aa[k] = a1c;
                    ja[k] = j1c;
                    S.f[c * HCAP + k] = to_float_scaled(xn, 0);
                    S.f[(3 + c) * HCAP + k] = to_float_scaled(un, 0);
                    S.f[(6 + c) * HCAP + k] = to_float_scaled(a1c, 0);
                    S.f[(9 + c) * HCAP + k] = to_float_scaled(j1c, 0);
                    const double a2e = fma(L[LV_H * LS], a3, a2);  // a2 at the end of the step
                    S.cf[c * ACH + sl] = to_float_scaled(a1c, 0);
                    S.cf[(3 + c) * ACH + sl] = to_float_scaled(j1c, -lv);
                    S.cf[(6 + c) * ACH + sl] = to_float_scaled(a2e, -2 * lv);
                    S.cf[(9 + c) * ACH + sl] = to_float_scaled(a3, -3 * lv);
                }
            }
            __syncthreads();
            // new time and level by the Aarseth criterion (FP32 on scaled
            // inputs); a larger step only by one level and on a commensurate time
            if (warp == 3) {
                for (int sl = wl; sl < nc; sl += 32) {
                    const int k = S.act[a0 + sl];
                    const int lv = S.lev[k];
                    int kn = level_from(S.cf + sl, lv, etaf, T2f);
                    if (kn < lv) {
                        const int up1 = lv - 1;
                        kn = (tn & ((1ll << (KMAX - up1)) - 1)) == 0 ? up1 : lv;
                    }
                    S.lev[k] = kn;
                    S.ti[k] = tn;
                }
            }
        }
        // every thread read (tn, na) before the barriers above; the active
        // list is no longer read in this block step
        if (warp == 3) next_block(S.lev, S.ti, S.act, n);
        ++steps;
    }
    // peers may still read this CTA's partial sums of the last round
    if (COOP) cl.sync(); else __syncthreads();
    if (capped && tid == 0 && rank == 0) atomicOr(d.status, QYM_ST_HERMITE_CAP);
    // item 7: pre-remove the (1-K) part of the coming kick at q1 (own members)
    for (int k = tid; k < n; k += blockDim.x) {
        S.ex[k] = S.x[k]; S.ey[k] = S.y[k]; S.ez[k] = S.z[k];
    }
    __syncthreads();
    for (int k0 = mlo; k0 < mhi; k0 += NG) {
        int k = k0 + grp;
        double c[3] = {0.0, 0.0, 0.0};
        if (k < mhi) kcorr_part(S, 0, n, k, lane, P, tc, c);
        group_sum(c, 3, P);
        if (k < mhi && lane == 0) {
            int64_t r = S.ids[k];
            d.q1[r] = S.x[k];
            d.q1[R + r] = S.y[k];
            d.q1[2 * R + r] = S.z[k];
            d.v1[r] = S.u[k] - 0.5 * tau * c[0];
            d.v1[R + r] = S.v[k] - 0.5 * tau * c[1];
            d.v1[2 * R + r] = S.w[k] - 0.5 * tau * c[2];
            d.uf[r] = -1;
            d.hcost[r] = (int32_t)min(steps, (int64_t)INT_MAX);
        }
    }
    if (tid == 0 && rank == 0) {
        atomicAdd(d.ctr + C_SUM_HSTEPS, (unsigned long long)steps);
        atomicMax(d.ctr + C_MAX_HSET, (unsigned long long)steps);
    }
    // the next set reuses shared memory that peers read above
    if (COOP) cl.sync(); else __syncthreads();
}

// The Hermite kernel's schedule for this step. A set's chain of block steps
// runs on one CTA (or one cluster) from start to end, so the step lasts as
// long as its longest set; which set that is can be foreseen, since a close
// pair stays close over consecutive steps. A set's predicted cost is the
// largest count of block steps among its members' sets of the previous step
// (hcost; 0 for rows that were in no set), raised per member by the set
// builder into hsetcost, which the plan reads and clears. Sets of at least
// NBIG members with the highest predicted cost (then the most members, then
// the lowest index) take the ncl clusters, one each; the other sets form the
// per-CTA queue in descending predicted cost, so the longest chains start
// first. With more than kPlanCap sets the queue keeps the set order and no
// cluster is used.
// One CTA of 1024 threads; the sets are ordered by a bitonic sort of 64-bit
// keys in shared memory.
constexpr int kPlanCap = 4096;
// When a system's step is split over several GPUs (own_hi > 0) this context
// integrates only the sets whose lowest row is its own: sets are numbered in
// the order of their lowest rows, so those are the index range [s_lo, s_hi).
__global__ void __launch_bounds__(1024) k_hermite_plan(Dev d, int ncl) {
    __shared__ unsigned long long key[kPlanCap];
    __shared__ int wsum[32];
    __shared__ int s_range[2];
    const int tid = threadIdx.x;
    const int nall = (int)min((unsigned long long)d.max_sets, d.ctr[C_NSETS]);
    if (tid == 0) {
        int lo = 0, hi = nall;
        if (d.own_hi > 0) {
            // first set whose root is >= own_lo, and >= own_hi (roots ascend)
            int a = 0, b = nall;
            while (a < b) { const int m = (a + b) >> 1; if (d.set_root[m] < d.own_lo) a = m + 1; else b = m; }
            lo = a;
            b = nall;
            while (a < b) { const int m = (a + b) >> 1; if (d.set_root[m] < d.own_hi) a = m + 1; else b = m; }
            hi = a;
        }
        s_range[0] = lo;
        s_range[1] = hi;
    }
    __syncthreads();
    const int s_lo = s_range[0];
    const int nsets = s_range[1] - s_lo;
    if (ncl > kHermMaxClusters) ncl = kHermMaxClusters;
    for (int c = tid; c < kHermMaxClusters; c += blockDim.x) d.hcl[c] = -1;
    for (int k = tid; k < nall; k += blockDim.x)
        if (k < s_lo || k >= s_lo + nsets) d.hsetcost[k] = 0;
    if (nsets > kPlanCap) {
        for (int k = tid; k < nsets; k += blockDim.x) {
            d.hq[k] = s_lo + k;
            d.hsetcost[s_lo + k] = 0;
        }
        if (tid == 0) d.ctr[C_HNQ] = (unsigned long long)nsets;
        return;
    }
    int P = 1;
    while (P < nsets) P <<= 1;
    // key: predicted cost (31 bits) | members (16 bits) | 0xffff - set index
    // (set indices relative to s_lo)
    for (int k = tid; k < P; k += blockDim.x) {
        unsigned long long kk = 0;
        if (k < nsets) {
            const int sk = s_lo + k;
            const int n = d.set_start[sk + 1] - d.set_start[sk];
            const int cost = d.hsetcost[sk];
            d.hsetcost[sk] = 0;
            kk = ((unsigned long long)min(max(cost, 0), 0x7fffffff) << 32) |
                 ((unsigned long long)min(max(n, 0), 0xffff) << 16) | (unsigned long long)(0xffff - k);
        }
        key[k] = kk;
    }
    __syncthreads();
    // descending bitonic sort (padding keys are 0 and sink to the end)
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = tid; k < P; k += blockDim.x) {
                const int o = k ^ stride;
                if (o > k) {
                    const bool desc = (k & size) == 0;
                    const unsigned long long a = key[k], b = key[o];
                    if (desc ? a < b : a > b) {
                        key[k] = b;
                        key[o] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // in sorted order: eligible = at least NBIG members; the first ncl
    // eligible sets go to the clusters, the rest keep their order in the queue
    constexpr int PER = kPlanCap / 1024;
    const int k0 = tid * PER;
    int e[PER], cnt = 0;
    for (int i = 0; i < PER; ++i) {
        const int k = k0 + i;
        e[i] = (k < nsets && (int)((key[k] >> 16) & 0xffff) >= NBIG) ? 1 : 0;
        cnt += e[i];
    }
    // exclusive prefix of cnt over the threads
    const int lane = tid & 31, w = tid >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = incl - cnt;
    for (int k = 0; k < w; ++k) before += wsum[k];
    int total = 0;
    for (int k = 0; k < 32; ++k) total += wsum[k];
    for (int i = 0; i < PER; ++i) {
        const int k = k0 + i;
        if (k >= nsets) break;
        const int set = s_lo + 0xffff - (int)(key[k] & 0xffff);
        if (e[i] && before < ncl) {
            d.hcl[before] = set;
        } else {
            d.hq[k - min(before, ncl)] = set;
        }
        before += e[i];
    }
    if (tid == 0) d.ctr[C_HNQ] = (unsigned long long)(nsets - min(total, ncl));
}

// Each cluster of CLT CTAs first integrates the set the plan gave it (all its
// CTAs on one set), then every CTA takes sets one at a time from the queue, in
// the order of a counter, so CTAs freed early take more.
template <int CLT>
__global__ void __cluster_dims__(CLT, 1, 1) __launch_bounds__(HTHREADS, 2) k_hermite(Dev d, HermArgs h) {
    static_assert(CLT == 2 || CLT == 4 || CLT == 8, "a cluster is 2, 4 or 8 CTAs");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int cid = blockIdx.x / CLT;
    const int cset = cid < kHermMaxClusters ? d.hcl[cid] : -1;
    if (cset >= 0) hermite_set<true, CLT>(d, h, cset, rank, CLT);
    const int nq = (int)d.ctr[C_HNQ];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) g_next_small = (int)atomicAdd(d.ctr + C_HSMALL, 1ull);
        __syncthreads();
        const int k = g_next_small;
        if (k >= nq) break;
        hermite_set<false, 2>(d, h, d.hq[k], 0, 1);
    }
}

// every member of every set leaves the union-find (-1) and, when this context
// integrated only its own sets, the other sets' members get their states and
// costs from the GPUs that did
__global__ void k_uf_clear_members(Dev d) {
    const unsigned long long n = min(d.ctr[C_NMEM], (unsigned long long)d.max_members);
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x)
        d.uf[d.set_mem[k]] = -1;
}

cudaError_t hermite_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_hermite<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kHermSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hermite<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHermSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hermite<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHermSmem);
    return e;
}

// Cluster size for a batch (qym_params.hermite_cluster; 0 = automatic). One
// system holds a few sets, and its longest set gains most from spreading its
// partners over eight SMs (two CTAs per SM). A batch of many systems keeps
// thousands of sets in flight that share the SMs' FP64 units; there the
// longest set does best on a cluster of two CTAs, each alone on its SM
// (measured on the 512-system ensemble: 20.2 ms per step, against 22.7 ms with
// eight-CTA clusters at two CTAs per SM; the 16384-body disk: 1.38 ms against
// 1.48 ms the other way round).
int hermite_cluster_size(const Dev &d, const qym_params &p) {
    if (p.hermite_cluster == 2 || p.hermite_cluster == 4 || p.hermite_cluster == 8)
        return p.hermite_cluster;
    return d.nsys == 1 ? 8 : 2;
}

cudaError_t launch_hermite(const Dev &d, const qym_params &p, double tau, cudaStream_t st) {
    HermArgs h;
    h.G = p.G;
    h.eps2 = p.eps_H * p.eps_H;
    h.eta = p.eta;
    h.eta_s = p.eta_s;
    h.tau = tau;
    h.max_steps = p.max_hermite_steps;
    const int cls = hermite_cluster_size(d, p);
    const int grid = (cls == 2 ? 1 : 2) * 152;  // CTAs per SM x SMs
    static_assert(2 * 152 / 4 <= kHermMaxClusters && 152 / 2 <= kHermMaxClusters,
                  "more clusters than plan entries");
    k_hermite_plan<<<1, 1024, 0, st>>>(d, grid / cls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the plan has read the previous step's costs; this step's sets write theirs
    e = cudaMemsetAsync(d.hcost, 0, sizeof(int32_t) * (size_t)d.rows, st);
    if (e != cudaSuccess) return e;
    switch (cls) {
    case 2: k_hermite<2><<<grid, HTHREADS, kHermSmem, st>>>(d, h); break;
    case 4: k_hermite<4><<<grid, HTHREADS, kHermSmem, st>>>(d, h); break;
    default: k_hermite<8><<<grid, HTHREADS, kHermSmem, st>>>(d, h); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || d.own_hi == 0) return e;
    k_uf_clear_members<<<152, 256, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace qym
