// whole.cu -- the whole-system Hermite of Sec. 2.3, last paragraph: when a
// step's encounter sets put two planets (m >= planet_mass m0) in one set, that
// system's step is redone by the Hermite for every body: from the positions
// after the opening drift and the velocities entering the first kick, every
// body is integrated over tau under H_Kep + H_Int (the star fixed at the
// origin, every pair with its full force: K = 0, r_crit infinite) with the
// same 4th-order scheme and individual block steps as an encounter set
// (Makino & Aarseth; Sec. 2.2), smoothed with eps_H; no K corrections and no
// second kick follow, only the closing drift.
//
// A system of any size: the state lives in global memory and each block step
// is four kernels, enqueued by the host in chunks (the paper computes the
// accelerations and jerks on the GPU and steps on the CPU). As in the mixed
// kick, the pull of the light bodies (m < heavy_mass m0) is an FP32 pair term
// on double-single separations, and the heavy bodies' pull is FP64 (they
// carry almost all of the interaction; a light body's pull enters the sums
// at 1e-7 of itself):
//   k_wh_next     one CTA: the next block time t_n (the earliest end of a
//                 body's step), the bodies whose step ends there in row order,
//                 the split of their partner sums over CTAs; `done` at tau
//   k_wh_predict  every body predicted to t_n from its own time (FP64, and
//                 split into float hi + lo parts)
//   k_wh_force    (active body, partner range) items over a fixed grid: the
//                 range's light pair accelerations and jerks, summed in a
//                 fixed tree
//   k_wh_correct  per active body: its ranges in order, the heavy bodies' and
//                 the star's pull in FP64, the corrector, the Aarseth
//                 criterion and the new level
// Time runs in integer ticks of |tau| / 2^48 as in the set Hermite; a level
// grows by one only on a commensurate block time. Every kernel returns at once
// when `done` is set, so a chunk may run past tau without effect.
#include "qym_internal.cuh"

namespace qym {

namespace {

constexpr int WKMAX = 48;           // levels: steps |tau| 2^-k, k <= WKMAX
constexpr int kForceThreads = 128;  // k_wh_force
constexpr int kMinRange = 64;       // partners per (body, range) item at least

__device__ __forceinline__ int wh_level(double dt_c, double T) {
    // smallest k with T 2^-k <= dt_c, in [0, WKMAX]
    if (!(dt_c > 0.0)) return WKMAX;
    int k = 0;
    double dd = T;
    while (dd > dt_c && k < WKMAX) {
        dd *= 0.5;
        ++k;
    }
    return k;
}

__device__ __forceinline__ double n3(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

// Aarseth: sqrt(eta (|a| |a2| + |j|^2) / (|j| |a3| + |a2|^2)), T when the
// denominator vanishes
__device__ __forceinline__ double wh_aarseth(const double *a, const double *j, const double *a2,
                                             const double *a3, double eta, double T) {
    const double na = n3(a[0], a[1], a[2]), nj = n3(j[0], j[1], j[2]);
    const double n2 = n3(a2[0], a2[1], a2[2]), nn3 = n3(a3[0], a3[1], a3[2]);
    const double den = nj * nn3 + n2 * n2;
    if (!(den > 0.0)) return T;
    return sqrt(eta * (na * n2 + nj * nj) / den);
}

}  // namespace

// load the system's bodies: x = positions after the opening drift, u = the
// velocities entering the first kick; the start-up evaluates every body at
// t = 0 (all active, ranges for that many)
__global__ void k_wh_load(WholeArgs w, const double *q, const double *vpre) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        w.ctl[WC_NA] = w.nb;
        w.ctl[WC_DONE] = 0;
        w.ctl[WC_NCH] = 1;
        *w.tn = 0;
        *w.steps = 0;
    }
    if (i >= w.nb) return;
    const int64_t r = w.r0 + 1 + i;
    for (int c = 0; c < 3; ++c) {
        w.x[c * w.ld + i] = q[c * w.R + r];
        w.u[c * w.ld + i] = vpre[c * w.R + r];
        w.a0[c * w.ld + i] = 0.0;  // (the start-up's prediction to t = 0 reads them)
        w.j0[c * w.ld + i] = 0.0;
    }
    w.ti[i] = 0;
    w.act[i] = (int32_t)i;
}

// one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_wh_next(WholeArgs w) {
    __shared__ long long s_min[32];
    __shared__ int s_cnt[32];
    __shared__ int s_base, s_open;
    if (w.ctl[WC_DONE]) return;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const long long TT = 1ll << WKMAX;
    long long mn = TT;
    int open = 0;
    for (int64_t i = tid; i < w.nb; i += blockDim.x) {
        const long long e = w.ti[i] + (1ll << (WKMAX - w.lev[i]));
        mn = e < mn ? e : mn;
        open |= w.ti[i] < TT;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = t < mn ? t : mn;
    }
    open = __any_sync(0xffffffffu, open);
    if (tid == 0) s_open = 0;
    __syncthreads();
    if (lane == 0) {
        s_min[wp] = mn;
        if (open) atomicOr(&s_open, 1);
    }
    __syncthreads();
    if (tid < 32) {
        long long m2 = tid < (int)(blockDim.x >> 5) ? s_min[tid] : TT;
        for (int o = 16; o > 0; o >>= 1) {
            const long long t = __shfl_xor_sync(0xffffffffu, m2, o);
            m2 = t < m2 ? t : m2;
        }
        if (tid == 0) s_min[0] = m2;
    }
    __syncthreads();
    const long long tn = s_min[0];
    if (!s_open) {  // every body at tau
        if (tid == 0) w.ctl[WC_DONE] = 1;
        return;
    }
    if (*w.steps >= w.max_steps) {
        if (tid == 0) {
            w.ctl[WC_DONE] = 1;
            atomicOr(w.status, QYM_ST_HERMITE_CAP);
        }
        return;
    }
    // the bodies whose step ends at tn, in row order
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < w.nb; b0 += blockDim.x) {
        const int64_t i = b0 + tid;
        const bool a = i < w.nb && w.ti[i] + (1ll << (WKMAX - w.lev[i])) == tn;
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        if (lane == 0) s_cnt[wp] = __popc(bal);
        __syncthreads();
        int before = s_base;
        for (int k = 0; k < wp; ++k) before += s_cnt[k];
        if (a) w.act[before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_cnt[k];
            s_base += t;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int na = s_base;
        w.ctl[WC_NA] = na;
        // ranges per active body: about the grid's worth of items in all,
        // each range at least kMinRange partners
        const int maxr = (int)((w.nb + kMinRange - 1) / kMinRange);
        int nch = w.grid / (na > 0 ? na : 1);
        nch = nch < 1 ? 1 : (nch > maxr ? maxr : nch);
        w.ctl[WC_NCH] = nch;
        *w.tn = tn;
        *w.steps += 1;
    }
}

// every body to t_n from its own time (the oracle's Taylor forms)
__global__ void __launch_bounds__(256) k_wh_predict(WholeArgs w) {
    if (w.ctl[WC_DONE]) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.nb) return;
    const long long tn = *w.tn;
    const double h = w.sg * (double)(tn - w.ti[i]) * w.tick;
    float ph[3], pl[3], vh[3], vl[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t id = c * w.ld + i;
        const double x = w.x[id], u = w.u[id], a = w.a0[id], j = w.j0[id];
        const double xp = x + h * (u + h * (0.5 * a + h * j / 6.0));
        const double up = u + h * (a + 0.5 * h * j);
        w.xp[id] = xp;
        w.up[id] = up;
        split_ds(xp, ph[c], pl[c]);
        split_ds(up, vh[c], vl[c]);
    }
    const double mj = w.m[w.r0 + 1 + i];
    const float gm = mj >= w.heavy_thr ? 0.0f : (float)(w.G * mj);
    w.pf_hi[i] = make_float4(ph[0], ph[1], ph[2], gm);
    w.pf_lo[i] = make_float4(pl[0], pl[1], pl[2], 0.0f);
    w.vf_hi[i] = make_float4(vh[0], vh[1], vh[2], 0.0f);
    w.vf_lo[i] = make_float4(vl[0], vl[1], vl[2], 0.0f);
}

// the light partners' accelerations and jerks on the active bodies over
// partner ranges: item (k, c) = active body k, range c of nch; each thread a
// stride of the range in FP32 (separations as double-single differences, the
// smoothed pair term of the set Hermite with K = 0), its sums then in FP64 by
// warp trees and in warp order
__global__ void __launch_bounds__(kForceThreads) k_wh_force(WholeArgs w) {
    __shared__ double s_part[kForceThreads / 32][6];
    if (w.ctl[WC_DONE]) return;
    const int na = w.ctl[WC_NA], nch = w.ctl[WC_NCH];
    const int64_t items = (int64_t)na * nch;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const float eps2 = (float)w.eps2;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int k = (int)(it / nch), c = (int)(it - (int64_t)k * nch);
        const int64_t i = w.act[k];
        const int64_t lo = w.nb * c / nch, hi = w.nb * (c + 1) / nch;
        const float4 pih = w.pf_hi[i], pil = w.pf_lo[i], vih = w.vf_hi[i], vil = w.vf_lo[i];
        float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int64_t j = lo + tid; j < hi; j += blockDim.x) {
            if (j == i) continue;
            const float4 pjh = w.pf_hi[j], pjl = w.pf_lo[j], vjh = w.vf_hi[j], vjl = w.vf_lo[j];
            const float dx = (pih.x - pjh.x) + (pil.x - pjl.x);
            const float dy = (pih.y - pjh.y) + (pil.y - pjl.y);
            const float dz = (pih.z - pjh.z) + (pil.z - pjl.z);
            const float ex = (vih.x - vjh.x) + (vil.x - vjl.x);
            const float ey = (vih.y - vjh.y) + (vil.y - vjl.y);
            const float ez = (vih.z - vjh.z) + (vil.z - vjl.z);
            const float s2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float is = rsqrt_ftz(s2), is2 = is * is;
            const float g = -pjh.w * is * is2;   // -G m_j / s^3 (0 for a heavy body)
            const float t3 = 3.0f * fmaf(dx, ex, fmaf(dy, ey, dz * ez)) * is2;
            s[0] = fmaf(g, dx, s[0]);
            s[1] = fmaf(g, dy, s[1]);
            s[2] = fmaf(g, dz, s[2]);
            s[3] = fmaf(g, fmaf(-t3, dx, ex), s[3]);
            s[4] = fmaf(g, fmaf(-t3, dy, ey), s[4]);
            s[5] = fmaf(g, fmaf(-t3, dz, ez), s[5]);
        }
        double sd[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) sd[q] = warp_sum((double)s[q]);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 6; ++q) s_part[wp][q] = sd[q];
        __syncthreads();
        if (tid < 6) {
            double v = 0.0;
            for (int k2 = 0; k2 < kForceThreads / 32; ++k2) v += s_part[k2][tid];
            w.part[6 * it + tid] = v;
        }
        __syncthreads();
    }
}

// per active body: the ranges' sums in order plus the star's pull (smoothed,
// the star fixed at the origin), then at start-up the first level, else the
// corrector, the new level and the body's time
__global__ void __launch_bounds__(128) k_wh_correct(WholeArgs w, int startup) {
    if (w.ctl[WC_DONE]) return;
    const int na = w.ctl[WC_NA], nch = w.ctl[WC_NCH];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const int64_t i = w.act[k], ld = w.ld;
    double a1[3], j1[3];
    {
        const double x = w.xp[i], y = w.xp[ld + i], z = w.xp[2 * ld + i];
        const double u = w.up[i], v = w.up[ld + i], ww = w.up[2 * ld + i];
        const double s2 = x * x + y * y + z * z + w.eps2;
        const double is = rsqrt(s2), is2 = is * is;
        const double g = -w.G * w.m0 * is * is2;
        const double t3 = 3.0 * (x * u + y * v + z * ww) * is2;
        a1[0] = g * x; a1[1] = g * y; a1[2] = g * z;
        j1[0] = g * (u - t3 * x); j1[1] = g * (v - t3 * y); j1[2] = g * (ww - t3 * z);
    }
    const double *p = w.part + 6 * (int64_t)k * nch;
    for (int c = 0; c < nch; ++c)
        for (int q = 0; q < 3; ++q) {
            a1[q] += p[6 * c + q];
            j1[q] += p[6 * c + 3 + q];
        }
    // the heavy bodies' pull in FP64 (the oracle's pair term with K = 0)
    for (int h = 0; h < w.nheavy; ++h) {
        const int64_t j = w.heavy[h];
        if (j == i) continue;
        const double dx = w.xp[i] - w.xp[j], dy = w.xp[ld + i] - w.xp[ld + j];
        const double dz = w.xp[2 * ld + i] - w.xp[2 * ld + j];
        const double ex = w.up[i] - w.up[j], ey = w.up[ld + i] - w.up[ld + j];
        const double ez = w.up[2 * ld + i] - w.up[2 * ld + j];
        const double s2 = dx * dx + dy * dy + dz * dz + w.eps2;
        const double s = sqrt(s2);
        const double rv = dx * ex + dy * ey + dz * ez;
        const double g = -w.G * w.m[w.r0 + 1 + j] / (s2 * s);
        a1[0] += g * dx; a1[1] += g * dy; a1[2] += g * dz;
        j1[0] += g * (ex - 3.0 * rv * dx / s2);
        j1[1] += g * (ey - 3.0 * rv * dy / s2);
        j1[2] += g * (ez - 3.0 * rv * dz / s2);
    }
    const double T = w.T;
    if (startup) {
        for (int q = 0; q < 3; ++q) {
            w.a0[q * ld + i] = a1[q];
            w.j0[q * ld + i] = j1[q];
        }
        const double jn = n3(j1[0], j1[1], j1[2]);
        const double dt_c = jn > 0.0 ? w.eta_s * n3(a1[0], a1[1], a1[2]) / jn : T;
        w.lev[i] = wh_level(dt_c, T);
        w.ti[i] = 0;
        return;
    }
    const long long tn = *w.tn;
    const int lv = w.lev[i];
    const long long dti = 1ll << (WKMAX - lv);
    const double h = w.sg * (double)dti * w.tick;
    double a2[3], a3[3];
    for (int q = 0; q < 3; ++q) {
        const int64_t id = q * ld + i;
        const double a0 = w.a0[id], j0 = w.j0[id];
        a2[q] = (-6.0 * (a0 - a1[q]) - h * (4.0 * j0 + 2.0 * j1[q])) / (h * h);
        a3[q] = (12.0 * (a0 - a1[q]) + 6.0 * h * (j0 + j1[q])) / (h * h * h);
        w.x[id] = w.xp[id] + h * h * h * h * (a2[q] / 24.0 + h * a3[q] / 120.0);
        w.u[id] = w.up[id] + h * h * h * (a2[q] / 6.0 + h * a3[q] / 24.0);
        a2[q] += h * a3[q];
        w.a0[id] = a1[q];
        w.j0[id] = j1[q];
    }
    w.ti[i] = tn;
    int kn = wh_level(wh_aarseth(a1, j1, a2, a3, w.eta, T), T);
    if (kn < lv) {
        const int up1 = lv - 1;
        kn = (tn % (1ll << (WKMAX - up1)) == 0) ? up1 : lv;
    }
    w.lev[i] = kn;
}

// the result over the Kepler drift's output rows
__global__ void k_wh_store(WholeArgs w, double *q1, double *v1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w.nb) return;
    const int64_t r = w.r0 + 1 + i;
    for (int c = 0; c < 3; ++c) {
        q1[c * w.R + r] = w.x[c * w.ld + i];
        v1[c * w.R + r] = w.u[c * w.ld + i];
    }
}

// a set of two or more planets: flag its system (one warp per set)
__global__ void __launch_bounds__(256) k_wh_trigger(Dev d, double planet_mass, int32_t *flag) {
    const int nsets = (int)min((unsigned long long)d.max_sets, d.ctr[C_NSETS]);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nsets; s += warps) {
        const int b = d.set_start[s];
        const int e = min(d.set_start[s + 1], d.max_members);  // (an overflow is flagged elsewhere)
        if (b >= e) continue;
        const int sys = d.sys_of[d.set_mem[b]];
        const double mp = planet_mass * d.m[d.offsets[sys]];
        int np = 0;
        for (int k = b + lane; k < e; k += 32) np += d.m[d.set_mem[k]] >= mp;
        for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
        if (lane == 0 && np >= 2) atomicOr(flag + sys, 1);
    }
}

cudaError_t launch_wh_trigger(const Dev &d, double planet_mass, int32_t *flag, cudaStream_t st) {
    k_wh_trigger<<<8, 256, 0, st>>>(d, planet_mass, flag);
    return cudaGetLastError();
}

cudaError_t launch_wh_start(const WholeArgs &w, const double *q, const double *vpre, cudaStream_t st) {
    const unsigned g = (unsigned)((w.nb + 255) / 256);
    k_wh_load<<<g, 256, 0, st>>>(w, q, vpre);
    k_wh_predict<<<g, 256, 0, st>>>(w);  // t_n = 0: the loaded state itself
    k_wh_force<<<w.grid, kForceThreads, 0, st>>>(w);
    k_wh_correct<<<(unsigned)((w.nb + 127) / 128), 128, 0, st>>>(w, 1);
    return cudaGetLastError();
}

cudaError_t launch_wh_blocks(const WholeArgs &w, int nblocks, cudaStream_t st) {
    const unsigned g = (unsigned)((w.nb + 255) / 256);
    for (int b = 0; b < nblocks; ++b) {
        k_wh_next<<<1, 1024, 0, st>>>(w);
        k_wh_predict<<<g, 256, 0, st>>>(w);
        k_wh_force<<<w.grid, kForceThreads, 0, st>>>(w);
        k_wh_correct<<<(unsigned)((w.nb + 127) / 128), 128, 0, st>>>(w, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_wh_store(const WholeArgs &w, double *q1, double *v1, cudaStream_t st) {
    k_wh_store<<<(unsigned)((w.nb + 255) / 256), 256, 0, st>>>(w, q1, v1);
    return cudaGetLastError();
}

}  // namespace qym
