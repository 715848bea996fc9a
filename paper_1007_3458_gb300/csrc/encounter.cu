// encounter.cu -- close-encounter identification after the Kepler drift
// (Sec. 2.3 item 4, Sec. 2.4) and the partition of the encounter pairs into
// non-intersecting sets with their transition radius r_crit (Eq. 9).
//
// The rigorous test is evaluated in FP64 with explicitly rounded operations
// (no contraction into FMA) in a fixed order, so that equal inputs give equal
// bits on any IEEE-754 machine evaluating the same sequence.
#include "qym_internal.cuh"

namespace qym {

#define DM(a, b) __dmul_rn((a), (b))
#define DA(a, b) __dadd_rn((a), (b))
#define DS(a, b) __dsub_rn((a), (b))

// Minimum over [0, tau] of the cubic p(u), u = t / tau, that matches
// d^2 = |dQ|^2 and its slope at both ends (third-order interpolation of the
// minimum separation, Sec. 2.4); clamped at 0.
__device__ double dmin2_cubic(const double *dq0, const double *dv0, const double *dq1,
                              const double *dv1, double tau) {
    double d0 = DA(DA(DM(dq0[0], dq0[0]), DM(dq0[1], dq0[1])), DM(dq0[2], dq0[2]));
    double d1 = DA(DA(DM(dq1[0], dq1[0]), DM(dq1[1], dq1[1])), DM(dq1[2], dq1[2]));
    double g0 = DA(DA(DM(dq0[0], dv0[0]), DM(dq0[1], dv0[1])), DM(dq0[2], dv0[2]));
    double g1 = DA(DA(DM(dq1[0], dv1[0]), DM(dq1[1], dv1[1])), DM(dq1[2], dv1[2]));
    double s0 = DM(DM(2.0, g0), tau);
    double s1 = DM(DM(2.0, g1), tau);
    double c0 = d0, c1 = s0;
    double c2 = DS(DS(DM(3.0, DS(d1, d0)), DM(2.0, s0)), s1);
    double c3 = DA(DA(DM(2.0, DS(d0, d1)), s0), s1);
    double best = d0 < d1 ? d0 : d1;
    // stationary points of p: A u^2 + B u + Cc = 0 with A = 3 c3, B = 2 c2,
    // Cc = c1; roots w / A and Cc / w, w = -(B + sgn(B) sqrt(B^2 - 4 A Cc)) / 2
    double A = DM(3.0, c3), B = DM(2.0, c2), Cc = c1;
    double disc = DS(DM(B, B), DM(DM(4.0, A), Cc));
    if (disc >= 0.0) {
        double sq = __dsqrt_rn(disc);
        double w = DM(-0.5, DA(B, B >= 0.0 ? sq : -sq));
        double u[2];
        int nu = 0;
        if (A != 0.0) u[nu++] = __ddiv_rn(w, A);
        if (w != 0.0) u[nu++] = __ddiv_rn(Cc, w);
        for (int k = 0; k < nu; ++k) {
            double uk = u[k];
            if (uk > 0.0 && uk < 1.0) {
                double p = DA(c0, DM(uk, DA(c1, DM(uk, DA(c2, DM(uk, c3))))));
                if (p < best) best = p;
            }
        }
    }
    return best > 0.0 ? best : 0.0;
}

__device__ __forceinline__ double pair_test(const double *q0, const double *v0,
                                            const double *q1, const double *v1,
                                            const double *rH, int64_t R, int64_t i, int64_t j,
                                            double tau, double a_E, double &thr2) {
    double dq0[3], dv0[3], dq1[3], dv1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dq0[c] = DS(q0[c * R + i], q0[c * R + j]);
        dv0[c] = DS(v0[c * R + i], v0[c * R + j]);
        dq1[c] = DS(q1[c * R + i], q1[c * R + j]);
        dv1[c] = DS(v1[c * R + i], v1[c * R + j]);
    }
    double Rr = DM(a_E, DA(rH[i], rH[j]));
    thr2 = DM(Rr, Rr);
    return dmin2_cubic(dq0, dv0, dq1, dv1, tau);
}

// ---------------------------------------------------------------- public pair test
__global__ void k_pair_test(int64_t rows, const double *q0, const double *v0, const double *q1,
                            const double *v1, const double *rH, double tau, double a_E,
                            int64_t npairs, const int32_t *pairs, double *d2, int32_t *flag) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
    double thr2;
    double dm = pair_test(q0, v0, q1, v1, rH, rows, i, j, tau, a_E, thr2);
    if (d2) d2[k] = dm;
    if (flag) flag[k] = dm < thr2 ? 1 : 0;
}

cudaError_t launch_pair_test(int64_t rows, const double *q0, const double *v0, const double *q1,
                             const double *v1, const double *rH, double tau, double a_E,
                             int64_t npairs, const int32_t *pairs, double *d2, int32_t *flag,
                             cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    int tb = 256;
    k_pair_test<<<(unsigned)((npairs + tb - 1) / tb), tb, 0, st>>>(rows, q0, v0, q1, v1, rH, tau,
                                                                  a_E, npairs, pairs, d2, flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- refine
__device__ __forceinline__ void push_encounter(const Dev &d, int i, int j) {
    unsigned long long k = atomicAdd(d.ctr + C_NENC, 1ull);
    if (k < (unsigned long long)d.max_enc)
        d.enc[k] = make_int2(i, j);
    else
        atomicOr(d.status, QYM_ST_ENC_OVERFLOW);
    if (!d.log_refine) return;
    unsigned long long l = atomicAdd(d.ctr + C_LOG, 1ull);
    if (l < (unsigned long long)d.max_log) {
        d.log[3 * l] = (int64_t)d.ctr[C_STEP];
        d.log[3 * l + 1] = i;
        d.log[3 * l + 2] = j;
    } else {
        atomicOr(d.status, QYM_ST_LOG_OVERFLOW);
    }
}

// rigorous test of the crude candidates: (d.q, d.v) hold the state entering
// the Kepler drift, (d.q1, d.v1) the Kepler result
__global__ void __launch_bounds__(256) k_refine(Dev d, double tau, double a_E) {
    unsigned long long n = d.ctr[C_NCAND];
    if (n > (unsigned long long)d.max_cand) n = d.max_cand;
    const int64_t R = d.rows;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        int2 p = d.cand[k];
        double thr2;
        double dm = pair_test(d.q, d.v, d.q1, d.v1, d.rH, R, p.x, p.y, tau, a_E, thr2);
        if (dm < thr2) push_encounter(d, p.x, p.y);
    }
}

// exact re-search of rows whose crude bounds were exceeded: the row against
// every other body of its system (one CTA per row)
__global__ void __launch_bounds__(256) k_rescan(Dev d, double tau, double a_E) {
    unsigned long long n = d.ctr[C_NRESCAN];
    if (n > (unsigned long long)d.rows) n = d.rows;
    const int64_t R = d.rows;
    for (unsigned long long b = blockIdx.x; b < n; b += gridDim.x) {
        int64_t i = d.rescan[b];
        int sys = d.sys_of[i];
        int64_t lo = d.offsets[sys] + 1, hi = d.offsets[sys + 1];
        for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
            if (j == i) continue;
            int64_t a = i < j ? i : j, c = i < j ? j : i;
            double thr2;
            double dm = pair_test(d.q, d.v, d.q1, d.v1, d.rH, R, a, c, tau, a_E, thr2);
            if (dm < thr2) push_encounter(d, (int)a, (int)c);
        }
    }
}

cudaError_t launch_refine(const Dev &d, double tau, double a_E, cudaStream_t st) {
    k_refine<<<2 * 152, 256, 0, st>>>(d, tau, a_E);
    k_rescan<<<152, 256, 0, st>>>(d, tau, a_E);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sets
// Union-find over the encounter pairs on uf[rows] (-1 = not in any pair):
// roots are the smallest row of each set. Hooking links the larger root under
// the smaller with compare-and-swap; every loop is capped.
constexpr int UF_CAP = 1 << 20;

// Parents are read with volatile (L1-bypassing) loads: links are made with
// atomics in L2, and a cached line could still show a node as unset (-1).
// A negative parent is never followed.
__device__ __forceinline__ int uf_find(int *uf, int x, int &guard) {
    volatile int *u = uf;
    int p = u[x];
    while (p != x && p >= 0 && guard < UF_CAP) {
        x = p;
        p = u[x];
        ++guard;
    }
    return x;
}

__global__ void k_uf_hook(Dev d) {
    unsigned long long n = d.ctr[C_NENC];
    if (n > (unsigned long long)d.max_enc) n = d.max_enc;
    int *uf = d.uf;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        int2 p = d.enc[k];
        atomicCAS(uf + p.x, -1, p.x);
        atomicCAS(uf + p.y, -1, p.y);
        int guard = 0;
        while (guard < UF_CAP) {
            int a = uf_find(uf, p.x, guard), b = uf_find(uf, p.y, guard);
            if (a == b) break;
            if (a > b) { int t = a; a = b; b = t; }
            if (atomicCAS(uf + b, b, a) == b) break;
            ++guard;
        }
        if (guard >= UF_CAP) atomicOr(d.status, QYM_ST_UF_CAP);
    }
}

// per-block counts of roots, for an ordered numbering of the sets
__global__ void __launch_bounds__(1024) k_uf_count(Dev d, int32_t *blk) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int isroot = 0;
    if (r < d.rows) {
        int p = d.uf[r];
        isroot = (p == (int)r);
    }
    int c = __syncthreads_count(isroot);
    if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// exclusive scan of the block counts (one CTA)
__global__ void __launch_bounds__(1024) k_scan_blocks(Dev d, int32_t *blk, int nblk) {
    __shared__ int32_t part[1024];
    int per = (nblk + 1023) / 1024;
    int b0 = threadIdx.x * per;
    int s = 0;
    for (int b = b0; b < b0 + per && b < nblk; ++b) s += blk[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int b = b0; b < b0 + per && b < nblk; ++b) {
        int c = blk[b];
        blk[b] = run;
        run += c;
    }
    if (threadIdx.x == 1023) d.ctr[C_NSETS] = (unsigned long long)part[1023];
}

// number the roots in row order: sid[root] = set index; members are counted
__global__ void __launch_bounds__(1024) k_uf_number(Dev d, const int32_t *blk, int32_t *sid,
                                                    int32_t *size) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int isroot = 0;
    if (r < d.rows) isroot = (d.uf[r] == (int)r);
    unsigned ball = __ballot_sync(0xffffffffu, isroot);
    __shared__ int wsum[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(ball);
    __syncthreads();
    if (threadIdx.x < 32) {
        int x = wsum[threadIdx.x];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        wsum[threadIdx.x] = x;  // inclusive
    }
    __syncthreads();
    if (isroot) {
        int before = (w ? wsum[w - 1] : 0) + __popc(ball & ((1u << lane) - 1u));
        int s = blk[blockIdx.x] + before;
        sid[r] = s;
        size[s] = 0;
        if (s < d.max_sets) d.set_root[s] = (int32_t)r;
    }
}

// each member finds its root (compressing the path), adds itself to its set
// size, raises the set's r_crit (a_H times the largest Hill radius) and the
// set's predicted Hermite cost (the block steps of the member's set in the
// previous step)
__global__ void __launch_bounds__(256) k_uf_members(Dev d, const int32_t *sid, int32_t *size,
                                                    unsigned long long *rc_bits, double a_H) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    int p = d.uf[r];
    if (p < 0) return;
    int guard = 0;
    int root = uf_find(d.uf, (int)r, guard);
    int s = sid[root];
    if (s < 0 || s >= d.max_sets) return;
    atomicAdd(size + s, 1);
    double rc = a_H * d.rH[r];
    atomicMax(rc_bits + s, (unsigned long long)__double_as_longlong(rc));
    const int32_t hc = d.hcost[r];
    if (hc > 0) atomicMax(d.hsetcost + s, hc);
}

// set_start = exclusive scan of set sizes (one CTA); the fill counters reset
__global__ void __launch_bounds__(1024) k_scan_sets(Dev d, int32_t *size, int32_t *fill,
                                                    unsigned long long *rc_bits) {
    __shared__ int32_t part[1024];
    int n = (int)d.ctr[C_NSETS];
    if (n > d.max_sets) n = d.max_sets;
    int per = (n + 1023) / 1024;
    int b0 = threadIdx.x * per;
    int s = 0;
    for (int b = b0; b < b0 + per && b < n; ++b) s += size[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    int mx = 0;
    for (int b = b0; b < b0 + per && b < n; ++b) {
        d.set_start[b] = run;
        run += size[b];
        mx = max(mx, size[b]);
        fill[b] = 0;
        d.rcrit[b] = __longlong_as_double((long long)rc_bits[b]);
        rc_bits[b] = 0ull;
    }
    // largest set
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ int wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 1023) {
        d.set_start[n] = part[1023];
        d.ctr[C_NMEM] = (unsigned long long)part[1023];
        int m = 0;
        for (int k = 0; k < 32; ++k) m = max(m, wmax[k]);
        if ((unsigned long long)m > d.ctr[C_MAX_SET]) d.ctr[C_MAX_SET] = (unsigned long long)m;
        d.ctr[C_SUM_SETS] += (unsigned long long)n;
        if (part[1023] > d.max_members) atomicOr(d.status, QYM_ST_SET_OVERFLOW);
    }
}

__global__ void __launch_bounds__(256) k_uf_place(Dev d, const int32_t *sid, int32_t *fill) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    int p = d.uf[r];
    if (p < 0) return;
    int guard = 0;
    int root = uf_find(d.uf, (int)r, guard);
    int s = sid[root];
    if (s < 0 || s >= d.max_sets) return;
    int pos = d.set_start[s] + atomicAdd(fill + s, 1);
    if (pos < d.max_members) d.set_mem[pos] = (int32_t)r;
}

cudaError_t launch_sets_impl(const Dev &d, double a_H, const SetScratch &s, cudaStream_t st) {
    int nblk = (int)((d.rows + 1023) / 1024);
    k_uf_hook<<<152, 256, 0, st>>>(d);
    k_uf_count<<<nblk, 1024, 0, st>>>(d, s.blk);
    k_scan_blocks<<<1, 1024, 0, st>>>(d, s.blk, nblk);
    k_uf_number<<<nblk, 1024, 0, st>>>(d, s.blk, s.sid, s.size);
    int tb = 256;
    unsigned g = (unsigned)((d.rows + tb - 1) / tb);
    k_uf_members<<<g, tb, 0, st>>>(d, s.sid, s.size, s.rc_bits, a_H);
    k_scan_sets<<<1, 1024, 0, st>>>(d, s.size, s.fill, s.rc_bits);
    k_uf_place<<<g, tb, 0, st>>>(d, s.sid, s.fill);
    return cudaGetLastError();
}

}  // namespace qym
