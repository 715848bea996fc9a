// search.cu -- close-encounter candidates by spatial binning after the Kepler
// drift (the survey's next step for dense disks: sorting instead of the
// all-pairs sweep of Sec. 2.4), with a bound that makes the candidate set a
// superset of the pairs the rigorous test (Sec. 2.4, the cubic interpolation
// of d^2) can flag.
//
// The bound. For a pair (i, j) the rigorous test takes the cubic p(s),
// s = t / tau in [0, 1], that matches |dQ|^2 and its slope at both ends. Let
// H_k(s) = a_k + b_k s + c_k s^2 + d_k s^3 be the cubic Hermite interpolant of
// body k's own position (a = q0, b = tau v0, c = 3 (q1 - q0) - tau (2 v0 +
// v1), d = 2 (q0 - q1) + tau (v0 + v1)) and H = H_i - H_j. |H|^2 has the same
// values and slopes at both ends as the data p interpolates, and cubic
// Hermite interpolation reproduces cubics, so |H(s)|^2 - p(s) = s^2 (1 - s)^2
// r(s) with r(s) = A4 + A5 (s + 2) + A6 (s^2 + 2 s + 3), A4 = |c|^2 + 2 b.d,
// A5 = 2 c.d, A6 = |d|^2 (c, d, b those of H). Hence, with s^2 (1 - s)^2 <=
// 1/16, p(s) >= |H(s)|^2 - (|c|^2 + 2 |b||d| + 6 |c||d| + 6 |d|^2) / 16, and a
// pair the test flags (min p < thr^2) has min_s |H(s)| < thr + e_ij with
// e_ij <= e_i + e_j, e_k = (|c_k| + 3 |d_k|) / 4 + sqrt(|tau| V |d_k|) / 2,
// V the largest |v0| of the system (|b| <= |tau| (|v0_i| + |v0_j|)). So if
// the boxes that hold H_i([0, 1]) and H_j([0, 1]), each widened by its body's
// a_E r_H + e_k, do not overlap, the test cannot flag the pair.
//
// The pass. Per body its widened box (k_search_prep); per tile of 256
// consecutive positions (the kick's Morton order for one system, row order in
// a batch) the union of its bodies' boxes (k_search_tiles); tile pairs of a
// system whose boxes overlap (k_search_tilepairs); and per such tile pair,
// each body pair whose boxes overlap is tested with the rigorous test's cubic
// in FP32 on positions relative to a point of the first tile, with an error
// allowance that keeps the FP32 form from rejecting any pair the FP64 test
// (k_refine) can flag; the pairs that pass are the candidates.
#include <algorithm>
#include <vector>

#include "qym_internal.cuh"

namespace qym {

constexpr int kSTile = 256;  // positions per search tile

// V = largest |v0| of each system's bodies, as float bits (non-negative floats
// order like their bit patterns), raised by atomics
__global__ void __launch_bounds__(256) k_search_vmax(Dev d, int32_t *vmax) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    const int64_t R = d.rows;
    const double vx = d.v[r], vy = d.v[R + r], vz = d.v[2 * R + r];
    const float s = __double2float_ru(sqrt(vx * vx + vy * vy + vz * vz));
    atomicMax(vmax + d.sys_of[r], __float_as_int(s));
}

// extremes over s in [0, 1] of a + b s + c s^2 + d s^3
__device__ __forceinline__ void cubic_range(double a, double b, double c, double d, double &lo,
                                            double &hi) {
    const double e = a + b + c + d;
    lo = fmin(a, e);
    hi = fmax(a, e);
    // stationary points: 3 d s^2 + 2 c s + b = 0
    const double A = 3.0 * d, B = 2.0 * c, C = b;
    double s[2];
    int ns = 0;
    if (A != 0.0) {
        const double disc = B * B - 4.0 * A * C;
        if (disc >= 0.0) {
            const double w = -0.5 * (B + copysign(sqrt(disc), B));
            s[ns++] = w / A;
            if (w != 0.0) s[ns++] = C / w;
        }
    } else if (B != 0.0) {
        s[ns++] = -C / B;
    }
    for (int k = 0; k < ns; ++k) {
        const double u = s[k];
        if (u > 0.0 && u < 1.0) {
            const double x = a + u * (b + u * (c + u * d));
            lo = fmin(lo, x);
            hi = fmax(hi, x);
        }
    }
}


// per body: its widened box and its FP32 state, at its position
__global__ void __launch_bounds__(256) k_search_prep(Dev d, SearchArgs s) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    const int64_t R = d.rows;
    const int64_t p = d.inv ? d.inv[r] : r;
    const int sys = d.sys_of[r];
    if (d.offsets[sys] == r) {  // star rows: an empty box
        s.box_lo[p] = make_float4(3e38f, 3e38f, 3e38f, 0.f);
        s.box_hi[p] = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
        return;
    }
    const double tau = s.tau, at = fabs(tau);
    double lo[3], hi[3], cc = 0.0, dd = 0.0, qq = 0.0;
    float q0h[3], q0l[3], q1h[3], q1l[3], vf0[3], vf1[3];
    for (int k = 0; k < 3; ++k) {
        const double a = d.q[k * R + r], v0 = d.v[k * R + r];
        const double e = d.q1[k * R + r], v1 = d.v1[k * R + r];
        const double b = tau * v0;
        const double c = 3.0 * (e - a) - tau * (2.0 * v0 + v1);
        const double dk = 2.0 * (a - e) + tau * (v0 + v1);
        cubic_range(a, b, c, dk, lo[k], hi[k]);
        cc += c * c;
        dd += dk * dk;
        qq = fmax(qq, fmax(fabs(a), fabs(e)));
        split_ds(a, q0h[k], q0l[k]);
        split_ds(e, q1h[k], q1l[k]);
        vf0[k] = (float)v0;
        vf1[k] = (float)v1;
    }
    const double V = (double)__int_as_float(s.vmax[sys]);
    const double C = sqrt(cc), D = sqrt(dd);
    const double ek = 0.25 * (C + 3.0 * D) + 0.5 * sqrt(at * V * D);
    const double thr = s.a_E * d.rH[r];
    // widened by a_E r_H + e_k, and by 1e-12 of the coordinates for the
    // rounding of the cubic's coefficients and extremes here and in the test
    const double w = (thr + ek) * (1.0 + 1e-9) + 1e-12 * qq;
    s.box_lo[p] = make_float4(__double2float_rd(lo[0] - w), __double2float_rd(lo[1] - w),
                              __double2float_rd(lo[2] - w), 0.f);
    s.box_hi[p] = make_float4(__double2float_ru(hi[0] + w), __double2float_ru(hi[1] + w),
                              __double2float_ru(hi[2] + w), 0.f);
    s.x0h[p] = make_float4(q0h[0], q0h[1], q0h[2], __double2float_ru(thr));
    s.x0l[p] = make_float4(q0l[0], q0l[1], q0l[2], 0.f);
    s.x1h[p] = make_float4(q1h[0], q1h[1], q1h[2], 0.f);
    s.x1l[p] = make_float4(q1l[0], q1l[1], q1l[2], 0.f);
    s.v0f[p] = make_float4(vf0[0], vf0[1], vf0[2], 0.f);
    s.v1f[p] = make_float4(vf1[0], vf1[1], vf1[2], 0.f);
}

// per tile: the union of its bodies' boxes
__global__ void __launch_bounds__(kSTile) k_search_tiles(SearchArgs s) {
    __shared__ float sm[kSTile / 32][6];
    const int4 t = s.tiles[blockIdx.x];
    const int64_t p = t.y + threadIdx.x;
    float m[6] = {3e38f, 3e38f, 3e38f, 3e38f, 3e38f, 3e38f};
    if (p < t.z) {
        const float4 a = s.box_lo[p], b = s.box_hi[p];
        m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = -b.x; m[4] = -b.y; m[5] = -b.z;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) m[q] = warp_min(m[q]);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 6; ++q) sm[threadIdx.x >> 5][q] = m[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = sm[0][threadIdx.x];
        for (int w = 1; w < kSTile / 32; ++w) v = fminf(v, sm[w][threadIdx.x]);
        sm[0][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s.tbox[2 * blockIdx.x] = make_float4(sm[0][0], sm[0][1], sm[0][2], 0.f);
        s.tbox[2 * blockIdx.x + 1] = make_float4(-sm[0][3], -sm[0][4], -sm[0][5], 0.f);
    }
}

__device__ __forceinline__ bool boxes_overlap(float4 al, float4 ah, float4 bl, float4 bh) {
    return al.x <= bh.x && bl.x <= ah.x && al.y <= bh.y && bl.y <= ah.y && al.z <= bh.z &&
           bl.z <= ah.z;
}

__global__ void __launch_bounds__(256) k_search_tilepairs(SearchArgs s, int32_t *status) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool hit = false;
    int2 tp = make_int2(0, 0);
    if (k < s.ntpairs) {
        tp = s.tpairs[k];
        hit = boxes_overlap(s.tbox[2 * tp.x], s.tbox[2 * tp.x + 1], s.tbox[2 * tp.y],
                            s.tbox[2 * tp.y + 1]);
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(s.nactive, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) s.active[base + __popc(m & ((1u << lane) - 1u))] = tp;
}

// candidate (i, j), rows, smaller first: warp-aggregated append
__device__ __forceinline__ void push_cand(const Dev &d, int i, int j) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(d.ctr + C_NCAND, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < (unsigned long long)d.max_cand)
        d.cand[idx] = make_int2(i, j);
    else if (lane == leader)
        atomicOr(d.status, QYM_ST_CAND_OVERFLOW);
}

// a + b + c rounded once (two-sum of a + b; c small)
__device__ __forceinline__ float ds3(float a, float b, float c) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return __fadd_rn(s, __fadd_rn(e, c));
}

// The rigorous test's cubic in FP32 for one pair, conservative: true unless
// the FP64 test (same data) certainly finds min p >= thr^2. Positions are
// offsets from a common point (rounded once each, |error| <= 2^-24 |offset|),
// velocities FP32; eq, ev bound the errors of the differences dq, dv.
__device__ __forceinline__ bool cubic_may_flag(const float *oi0, const float *oi1,
                                               const float *vi0, const float *vi1,
                                               const float *oj0, const float *oj1,
                                               const float *vj0, const float *vj1, float thr,
                                               float tau) {
    float dq0[3], dq1[3], dv0[3], dv1[3];
    float m_q = 0.f, m_v = 0.f;  // magnitudes for the error bounds
    for (int k = 0; k < 3; ++k) {
        dq0[k] = oi0[k] - oj0[k];
        dq1[k] = oi1[k] - oj1[k];
        dv0[k] = vi0[k] - vj0[k];
        dv1[k] = vi1[k] - vj1[k];
        m_q = fmaxf(m_q, fmaxf(fabsf(oi0[k]) + fabsf(oj0[k]), fabsf(oi1[k]) + fabsf(oj1[k])));
        m_v = fmaxf(m_v, fmaxf(fabsf(vi0[k]) + fabsf(vj0[k]), fabsf(vi1[k]) + fabsf(vj1[k])));
    }
    const float y0 = dq0[0] * dq0[0] + dq0[1] * dq0[1] + dq0[2] * dq0[2];
    const float y1 = dq1[0] * dq1[0] + dq1[1] * dq1[1] + dq1[2] * dq1[2];
    const float g0 = dq0[0] * dv0[0] + dq0[1] * dv0[1] + dq0[2] * dv0[2];
    const float g1 = dq1[0] * dv1[0] + dq1[1] * dv1[1] + dq1[2] * dv1[2];
    const float s0 = 2.0f * g0 * tau, s1 = 2.0f * g1 * tau;
    const float c2 = 3.0f * (y1 - y0) - 2.0f * s0 - s1;
    const float c3 = 2.0f * (y0 - y1) + s0 + s1;
    float best = fminf(y0, y1);
    const float A = 3.0f * c3, B = 2.0f * c2;
    // also at the inflection point -B / 2A: where the two stationary points
    // meet, a discriminant near zero can come out negative in FP32
    if (A != 0.0f) {
        const float ui = -B / (2.0f * A);
        if (ui > 0.0f && ui < 1.0f) best = fminf(best, y0 + ui * (s0 + ui * (c2 + ui * c3)));
    }
    const float disc = B * B - 4.0f * A * s0;
    if (disc >= 0.0f) {
        const float w = -0.5f * (B + copysignf(sqrtf(disc), B));
        float u[2];
        int nu = 0;
        if (A != 0.0f) u[nu++] = w / A;
        if (w != 0.0f) u[nu++] = s0 / w;
        for (int k = 0; k < nu; ++k)
            if (u[k] > 0.0f && u[k] < 1.0f)
                best = fminf(best, y0 + u[k] * (s0 + u[k] * (c2 + u[k] * c3)));
    }
    // The FP64 test's cubic and this one differ by the inputs' errors (the
    // offsets and velocities each within 2^-24 relative, their differences
    // within eq, ev) carried through y, g (values and slopes enter p with
    // weights at most 1 and 4/27), and by the rounding here (a generous
    // 2^-18 of the terms' magnitudes), and the FP32 root can miss the exact
    // stationary point; the minimum over [0, 1] moves by at most the largest
    // change of p, which the allowance bounds.
    const float eq = 4.0f * 5.96e-8f * m_q, ev = 4.0f * 5.96e-8f * m_v;
    const float nq0 = sqrtf(y0), nq1 = sqrtf(y1);
    const float nv0 = sqrtf(dv0[0] * dv0[0] + dv0[1] * dv0[1] + dv0[2] * dv0[2]);
    const float nv1 = sqrtf(dv1[0] * dv1[0] + dv1[1] * dv1[1] + dv1[2] * dv1[2]);
    const float at = fabsf(tau);
    const float ey = (2.0f * nq0 + eq) * eq + (2.0f * nq1 + eq) * eq;
    const float es = 2.0f * at * ((nq0 + eq) * ev + nv0 * eq + (nq1 + eq) * ev + nv1 * eq);
    const float mag = y0 + y1 + fabsf(s0) + fabsf(s1) + fabsf(c2) + fabsf(c3);
    const float allow = 1.01f * (ey + es) + 3.8e-6f * mag;
    return best - allow < thr * thr * 1.0001f;
}

// one CTA per overlapping tile pair (I, J): tile J staged in shared memory
// relative to a point of tile I, each thread one body of I against all of J
__global__ void __launch_bounds__(kSTile) k_search_pairs(Dev d, SearchArgs s) {
    __shared__ float4 j_lo[kSTile], j_hi[kSTile];
    __shared__ float j_o0[kSTile][3], j_o1[kSTile][3], j_v0[kSTile][3], j_v1[kSTile][3];
    __shared__ float j_thr[kSTile];
    const unsigned long long na = min(*(volatile unsigned long long *)s.nactive,
                                      (unsigned long long)s.ntpairs);
    for (unsigned long long k = blockIdx.x; k < na; k += gridDim.x) {
        const int2 tp = s.active[k];
        const int4 ti = s.tiles[tp.x], tj = s.tiles[tp.y];
        // reference point: the low corner of tile I's box (FP32, both tiles near it)
        const float4 cref = s.tbox[2 * tp.x];
        __syncthreads();
        {
            const int64_t p = tj.y + threadIdx.x;
            if (p < tj.z) {
                j_lo[threadIdx.x] = s.box_lo[p];
                j_hi[threadIdx.x] = s.box_hi[p];
                const float4 a = s.x0h[p], al = s.x0l[p], b = s.x1h[p], bl = s.x1l[p];
                const float4 u = s.v0f[p], w = s.v1f[p];
                j_o0[threadIdx.x][0] = ds3(a.x, -cref.x, al.x);
                j_o0[threadIdx.x][1] = ds3(a.y, -cref.y, al.y);
                j_o0[threadIdx.x][2] = ds3(a.z, -cref.z, al.z);
                j_o1[threadIdx.x][0] = ds3(b.x, -cref.x, bl.x);
                j_o1[threadIdx.x][1] = ds3(b.y, -cref.y, bl.y);
                j_o1[threadIdx.x][2] = ds3(b.z, -cref.z, bl.z);
                j_v0[threadIdx.x][0] = u.x; j_v0[threadIdx.x][1] = u.y; j_v0[threadIdx.x][2] = u.z;
                j_v1[threadIdx.x][0] = w.x; j_v1[threadIdx.x][1] = w.y; j_v1[threadIdx.x][2] = w.z;
                j_thr[threadIdx.x] = a.w;
            }
        }
        __syncthreads();
        const int64_t pi = ti.y + threadIdx.x;
        if (pi >= ti.z) continue;
        const float4 il = s.box_lo[pi], ih = s.box_hi[pi];
        const float4 a = s.x0h[pi], al = s.x0l[pi], b = s.x1h[pi], bl = s.x1l[pi];
        const float4 u = s.v0f[pi], w = s.v1f[pi];
        const float oi0[3] = {ds3(a.x, -cref.x, al.x), ds3(a.y, -cref.y, al.y), ds3(a.z, -cref.z, al.z)};
        const float oi1[3] = {ds3(b.x, -cref.x, bl.x), ds3(b.y, -cref.y, bl.y), ds3(b.z, -cref.z, bl.z)};
        const float vi0[3] = {u.x, u.y, u.z}, vi1[3] = {w.x, w.y, w.z};
        const int ri = d.perm ? d.perm[pi] : (int)pi;
        const int nj = (int)(tj.z - tj.y);
        const int j0 = tp.x == tp.y ? (int)threadIdx.x + 1 : 0;  // same tile: j after i
        for (int jj = j0; jj < nj; ++jj) {
            if (!boxes_overlap(il, ih, j_lo[jj], j_hi[jj])) continue;
            if (!cubic_may_flag(oi0, oi1, vi0, vi1, j_o0[jj], j_o1[jj], j_v0[jj], j_v1[jj],
                                a.w + j_thr[jj], (float)s.tau))
                continue;
            const int rj = d.perm ? d.perm[tj.y + jj] : (int)(tj.y + jj);
            push_cand(d, min(ri, rj), max(ri, rj));
        }
    }
}

cudaError_t launch_binned_search(const Dev &d, const SearchArgs &s0, double tau, double a_E,
                                 cudaStream_t st) {
    SearchArgs s = s0;
    s.tau = tau;
    s.a_E = a_E;
    cudaError_t e = cudaMemsetAsync((void *)s.vmax, 0, sizeof(int32_t) * d.nsys, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.nactive, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((d.rows + 255) / 256);
    k_search_vmax<<<g, 256, 0, st>>>(d, (int32_t *)s.vmax);
    k_search_prep<<<g, 256, 0, st>>>(d, s);
    k_search_tiles<<<s.ntiles, kSTile, 0, st>>>(s);
    k_search_tilepairs<<<(unsigned)((s.ntpairs + 255) / 256), 256, 0, st>>>(s, d.status);
    k_search_pairs<<<4 * 152, kSTile, 0, st>>>(d, s);
    return cudaGetLastError();
}

// tiles of kSTile consecutive positions within each system (positions
// offsets[s] + 1 .. offsets[s + 1] - 1) and every pair (I <= J) of one system
void search_tiles_host(const int64_t *offsets, int32_t nsys, std::vector<int4> &tiles,
                       std::vector<int2> &tpairs) {
    tiles.clear();
    tpairs.clear();
    for (int32_t s = 0; s < nsys; ++s) {
        const int t0 = (int)tiles.size();
        for (int64_t p = offsets[s] + 1; p < offsets[s + 1]; p += kSTile)
            tiles.push_back(make_int4(s, (int)p, (int)std::min<int64_t>(p + kSTile, offsets[s + 1]), 0));
        const int t1 = (int)tiles.size();
        for (int a = t0; a < t1; ++a)
            for (int b = a; b < t1; ++b) tpairs.push_back(make_int2(a, b));
    }
}

}  // namespace qym
