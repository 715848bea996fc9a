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
// The pass. Each body's widened box at its position in tiles of 256
// consecutive positions (the kick's Morton order for one system, row order in
// a batch), and the union of each tile's boxes (k_search_prep; V from the
// first kick's finisher); then
// the tile pairs of a system whose boxes overlap (k_search_tilepairs) and,
// per such pair, each body pair whose boxes overlap tested with the rigorous
// test's cubic in FP32 on positions relative to a point of the first tile,
// with an error allowance that keeps the FP32 form from rejecting any pair the
// FP64 test (k_refine) can flag (k_search_pairs); the pairs that pass are the
// candidates.
#include <algorithm>
#include <vector>

#include "qym_internal.cuh"

namespace qym {

constexpr int kSTile = 256;  // positions per search tile

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


// Four lanes per body (three axes and one idle), 8 bodies per warp: each
// body's widened box and its FP32 state at its position, and the union of the
// boxes of each tile, raised with atomics on order-preserving integer images
// of the floats (order-independent, so deterministic).
__device__ __forceinline__ int fbits(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float fvalue(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void __launch_bounds__(256) k_search_prep(Dev d, SearchArgs s) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = gt >> 2;           // position
    const int k = (int)(gt & 3);         // axis (3: idle)
    const bool body = p < d.rows && d.offsets[d.sys_of[d.perm ? d.perm[p] : p]] != (d.perm ? d.perm[p] : p);
    const int64_t R = d.rows;
    const int64_t r = p < d.rows ? (d.perm ? d.perm[p] : p) : 0;
    const double tau = s.tau;
    double lo = 0.0, hi = 0.0, c2 = 0.0, d2 = 0.0, qa = 0.0;
    float qh = 0.f, ql = 0.f, eh = 0.f, el = 0.f, v0f = 0.f, v1f = 0.f;
    if (body && k < 3) {
        const double a = d.q[k * R + r], v0 = d.v[k * R + r];
        const double e = d.q1[k * R + r], v1 = d.v1[k * R + r];
        const double b = tau * v0;
        const double c = 3.0 * (e - a) - tau * (2.0 * v0 + v1);
        const double dk = 2.0 * (a - e) + tau * (v0 + v1);
        cubic_range(a, b, c, dk, lo, hi);
        c2 = c * c;
        d2 = dk * dk;
        qa = fmax(fabs(a), fabs(e));
        split_ds(a, qh, ql);
        split_ds(e, eh, el);
        v0f = (float)v0;
        v1f = (float)v1;
    }
    // |c|^2, |d|^2 and the largest coordinate over the body's three lanes
    c2 += __shfl_xor_sync(0xffffffffu, c2, 1);
    c2 += __shfl_xor_sync(0xffffffffu, c2, 2);
    d2 += __shfl_xor_sync(0xffffffffu, d2, 1);
    d2 += __shfl_xor_sync(0xffffffffu, d2, 2);
    qa = fmax(qa, __shfl_xor_sync(0xffffffffu, qa, 1));
    qa = fmax(qa, __shfl_xor_sync(0xffffffffu, qa, 2));
    float blo = 3e38f, bhi = -3e38f;
    if (body) {
        const double V = (double)__int_as_float(d.vmax[d.sys_of[r]]);
        const double ek = 0.25 * (sqrt(c2) + 3.0 * sqrt(d2)) + 0.5 * sqrt(fabs(tau) * V * sqrt(d2));
        const double thr = s.a_E * d.rH[r];
        // widened by a_E r_H + e_k, and by 1e-12 of the coordinates for the
        // rounding of the cubic's coefficients and extremes here and in the test
        const double w = (thr + ek) * (1.0 + 1e-9) + 1e-12 * qa;
        if (k < 3) {
            blo = __double2float_rd(lo - w);
            bhi = __double2float_ru(hi + w);
        }
        if (k == 3) ((float *)(s.x0h + p))[3] = __double2float_ru(thr);
    }
    // scatter the lanes' components into the per-position float4s
    if (p < d.rows && k < 3) {
        ((float *)(s.box_lo + p))[k] = body ? blo : 3e38f;
        ((float *)(s.box_hi + p))[k] = body ? bhi : -3e38f;
        ((float *)(s.x0h + p))[k] = qh;
        ((float *)(s.x0l + p))[k] = ql;
        ((float *)(s.x1h + p))[k] = eh;
        ((float *)(s.x1l + p))[k] = el;
        ((float *)(s.v0f + p))[k] = v0f;
        ((float *)(s.v1f + p))[k] = v1f;
    }
    // the tile's box: each lane holds one axis of one body
    if (body && k < 3) {
        const int sys = d.sys_of[r];
        const int64_t tile = s.tile0[sys] + (p - d.offsets[sys] - 1) / kSTile;
        atomicMin(s.tbox_bits + 6 * tile + k, fbits(blo));
        atomicMin(s.tbox_bits + 6 * tile + 3 + k, fbits(-bhi));
    }
}

__device__ __forceinline__ bool boxes_overlap(float4 al, float4 ah, float4 bl, float4 bh) {
    return al.x <= bh.x && bl.x <= ah.x && al.y <= bh.y && bl.y <= ah.y && al.z <= bh.z &&
           bl.z <= ah.z;
}

__device__ __forceinline__ void tile_box(const SearchArgs &s, int t, float4 &lo, float4 &hi) {
    const int *b = s.tbox_bits + 6 * t;
    lo = make_float4(fvalue(b[0]), fvalue(b[1]), fvalue(b[2]), 0.f);
    hi = make_float4(-fvalue(b[3]), -fvalue(b[4]), -fvalue(b[5]), 0.f);
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
    const float t2 = thr * thr * 1.0001f;
    // in the Hermite form p = h00 y0 + h01 y1 + h10 s0 + h11 s1 (h00 + h01 = 1,
    // both >= 0; |h10|, |h11| <= 4/27): p >= min(y0, y1) - 4/27 (|s0| + |s1|)
    if (fminf(y0, y1) - 0.14815f * (fabsf(s0) + fabsf(s1)) - allow >= t2) return false;
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
    return best - allow < t2;
}

// tile pairs of a system whose boxes overlap, appended to the active list
__global__ void __launch_bounds__(256) k_search_tilepairs(Dev d, SearchArgs s) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool hit = false;
    int2 tp = make_int2(0, 0);
    if (k < s.ntpairs) {
        tp = s.tpairs[k];
        float4 al, ah, bl, bh;
        tile_box(s, tp.x, al, ah);
        tile_box(s, tp.y, bl, bh);
        hit = boxes_overlap(al, ah, bl, bh);
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(d.ctr + C_NACTIVE, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) s.active[base + __popc(m & ((1u << lane) - 1u))] = tp;
}

// one CTA per overlapping tile pair (I, J): tile J staged in shared memory
// relative to a point of tile I, each thread one body of I against all of J
__global__ void __launch_bounds__(kSTile) k_search_pairs(Dev d, SearchArgs s) {
    __shared__ float4 j_lo[kSTile], j_hi[kSTile];
    __shared__ float j_o0[kSTile][3], j_o1[kSTile][3], j_v0[kSTile][3], j_v1[kSTile][3];
    __shared__ float j_thr[kSTile];
    const unsigned long long na = min(*(volatile unsigned long long *)(d.ctr + C_NACTIVE),
                                      (unsigned long long)s.ntpairs);
    for (unsigned long long h = blockIdx.x; h < na; h += gridDim.x) {
        const int2 tq = s.active[h];
        const int4 ti = s.tiles[tq.x], tj = s.tiles[tq.y];
        // reference point: the low corner of tile I's box (both tiles near it)
        float4 cref, chi;
        tile_box(s, tq.x, cref, chi);
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
        // the warp's union box: a j whose box misses it is skipped by the
        // whole warp at once
        float4 il = make_float4(3e38f, 3e38f, 3e38f, 0.f), ih = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
        if (pi < ti.z) {
            il = s.box_lo[pi];
            ih = s.box_hi[pi];
        }
        const float4 wl = make_float4(warp_min(il.x), warp_min(il.y), warp_min(il.z), 0.f);
        const float4 wh = make_float4(-warp_min(-ih.x), -warp_min(-ih.y), -warp_min(-ih.z), 0.f);
        if (pi >= ti.z) continue;
        const float4 a = s.x0h[pi], al = s.x0l[pi], b = s.x1h[pi], bl = s.x1l[pi];
        const float4 u = s.v0f[pi], w = s.v1f[pi];
        const float oi0[3] = {ds3(a.x, -cref.x, al.x), ds3(a.y, -cref.y, al.y),
                              ds3(a.z, -cref.z, al.z)};
        const float oi1[3] = {ds3(b.x, -cref.x, bl.x), ds3(b.y, -cref.y, bl.y),
                              ds3(b.z, -cref.z, bl.z)};
        const float vi0[3] = {u.x, u.y, u.z}, vi1[3] = {w.x, w.y, w.z};
        const int ri = d.perm ? d.perm[pi] : (int)pi;
        const int nj = (int)(tj.z - tj.y);
        const int j0 = tq.x == tq.y ? (int)threadIdx.x + 1 : 0;  // same tile: j after i
        for (int jj = j0; jj < nj; ++jj) {
            const float4 jl = j_lo[jj], jh = j_hi[jj];
            if (!boxes_overlap(wl, wh, jl, jh)) continue;
            if (!boxes_overlap(il, ih, jl, jh)) continue;
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
    if (s.ntiles <= 0) return cudaSuccess;
    k_search_prep<<<(unsigned)((4 * d.rows + 255) / 256), 256, 0, st>>>(d, s);
    k_search_tilepairs<<<(unsigned)((s.ntpairs + 255) / 256), 256, 0, st>>>(d, s);
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
