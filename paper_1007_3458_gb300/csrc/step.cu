// step.cu -- the O(N) kernels of a step: the barycentric-momentum reduction and
// the uniform shift of E_Dft (Sec. 2, Eq. 2), the kick finisher (adds the
// partial accelerations, updates velocities, records |a| and the Hill radii
// used by the encounter test), Hill radii (Eq. 9), and the heliocentric <->
// barycentric velocity conversion (Sec. 2).
#include "qym_internal.cuh"

namespace qym {

// ---------------------------------------------------------------- E_Dft
// chunk partial sums of m_i v_i (bodies only), deterministic tree order
// (a chunk lies in one system, ch.z: its star row is known per chunk)
__global__ void __launch_bounds__(256) k_mom_chunks(Dev d) {
    const int4 ch = d.mchunks[blockIdx.x];
    const int64_t star = d.offsets[ch.z];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    const int64_t R = d.rows;
#pragma unroll 4
    for (int64_t r = ch.x + threadIdx.x; r < ch.y; r += blockDim.x) {
        if (r == star) continue;
        double mm = d.m[r];
        sx += mm * d.v[r];
        sy += mm * d.v[R + r];
        sz += mm * d.v[2 * R + r];
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    sz = warp_sum(sz);
    __shared__ double sh[3][8];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = sx; sh[1][w] = sy; sh[2][w] = sz; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[threadIdx.x][k];
        d.mpart[3 * blockIdx.x + threadIdx.x] = t;
    }
}

// S of each system from its chunks' partial sums, one warp per system: lane l
// adds the chunks l, l + 32, ... in order, then a fixed shuffle tree (the
// loads of a long system's chunk list overlap instead of following one another)
__global__ void k_mom_final(Dev d) {
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= d.nsys) return;
    double t[3] = {0.0, 0.0, 0.0};
    for (int c = d.sys_chunk0[s] + lane; c < d.sys_chunk0[s + 1]; c += 32)
        for (int k = 0; k < 3; ++k) t[k] += d.mpart[3 * c + k];
    for (int k = 0; k < 3; ++k) t[k] = warp_sum(t[k]);
    if (lane < 3) d.S[3 * s + lane] = lane == 0 ? t[0] : (lane == 1 ? t[1] : t[2]);
}

cudaError_t launch_momentum(const Dev &d, cudaStream_t st) {
    k_mom_chunks<<<d.nmchunks, 256, 0, st>>>(d);
    k_mom_final<<<(unsigned)((32 * (int64_t)d.nsys + 127) / 128), 128, 0, st>>>(d);
    return cudaGetLastError();
}

// Hill radius at the body's heliocentric distance: r_H = |Q| (m / 3 m0)^(1/3),
// the factor (m / 3 m0)^(1/3) of each row formed once on the host (hfac)
__device__ __forceinline__ double hill(double qx, double qy, double qz, double hf) {
    double r = sqrt(qx * qx + qy * qy + qz * qz);
    return r * hf;
}

__device__ __forceinline__ float round_up_f(double x) {
    float f = __double2float_ru(x);
    return f;
}

// E_Dft: Q += h S / m0 for h_close then h_open (each a separate half-drift,
// Sec. 2.3 items 10 and 1), read from (qs, vs) and written to (d.q, d.v);
// then the float packs of the coming kick, with the crude encounter reach when
// the coming kick searches for encounters (Sec. 2.4). flag_next = 2: the packs
// of a search that runs after the step's first kick, on the state that enters
// the Kepler drift; the Hill radius of the step is recorded here then.
struct DriftArgs {
    const double *qs, *vs;
    double h_close, h_open, tau, a_E, G;
    double kick_span;  // time of the kick(s) between this pack and the Kepler drift
    double a_allow;    // bound on |a| of that kick as a multiple of the last |a|
    int flag_next, hill_fixed;
};

// the systems whose shifts a CTA of k_drift_pack forms once (its rows span at
// most this many systems; else every row forms its own)
constexpr int kDriftSys = 8;

__global__ void __launch_bounds__(256) k_drift_pack(Dev d, DriftArgs a) {
    // The shifts (h S_k) / m0 of the CTA's systems, the same quotients every
    // row would form: FP64 divisions cost ~385 cycles and ~8 FP64-pipe
    // instructions here, six per row otherwise.
    __shared__ double sh_shift[kDriftSys][6];
    const int64_t R = d.rows;
    const int64_t rb = (int64_t)blockIdx.x * blockDim.x;
    const int s_lo = d.sys_of[rb], s_hi = d.sys_of[min(rb + (int64_t)blockDim.x, R) - 1];
    const bool cached = s_hi - s_lo < kDriftSys;
    if (cached && threadIdx.x < 6 * (s_hi - s_lo + 1)) {
        const int ss = s_lo + threadIdx.x / 6, k = threadIdx.x % 6;
        const double h = k < 3 ? a.h_close : a.h_open;
        sh_shift[threadIdx.x / 6][k] = h * d.S[3 * ss + k % 3] / d.m[d.offsets[ss]];
    }
    __syncthreads();
    int64_t r = rb + threadIdx.x;
    if (r >= R) return;
    const int sys = d.sys_of[r];
    const int64_t star = d.offsets[sys];
    double qx = a.qs[r], qy = a.qs[R + r], qz = a.qs[2 * R + r];
    double vx = a.vs[r], vy = a.vs[R + r], vz = a.vs[2 * R + r];
    if (r == star) {
        qx = qy = qz = vx = vy = vz = 0.0;
    } else {
        double sh[6];
        if (cached) {
#pragma unroll
            for (int k = 0; k < 6; ++k) sh[k] = sh_shift[sys - s_lo][k];
        } else {
            const double m0 = d.m[star];
#pragma unroll
            for (int k = 0; k < 6; ++k) sh[k] = (k < 3 ? a.h_close : a.h_open) * d.S[3 * sys + k % 3] / m0;
        }
        if (a.h_close != 0.0) {
            qx += sh[0];
            qy += sh[1];
            qz += sh[2];
        }
        if (a.h_open != 0.0) {
            qx += sh[3];
            qy += sh[4];
            qz += sh[5];
        }
    }
    d.q[r] = qx; d.q[R + r] = qy; d.q[2 * R + r] = qz;
    if (a.vs != d.v) { d.v[r] = vx; d.v[R + r] = vy; d.v[2 * R + r] = vz; }
    float xh, xl, yh, yl, zh, zl;
    split_ds(qx, xh, xl);
    split_ds(qy, yh, yl);
    split_ds(qz, zh, zl);
    const double mm = d.m[r];
    float reach = 0.0f;
    if (a.flag_next && r != star) {
        // crude reach rho_i = F_i (R_i + |tau| (u_i + w_i)):
        //   R_i  a_E times a bound on this step's Hill radius
        //   u_i  speed relative to the local circular velocity Omega (z x Q)
        //   w_i  bound on the velocity change of the kick(s) before the Kepler
        //        drift: (tau/2) 1.01 |a| (the last kick was at the same
        //        separations), or with merged kicks tau 2 |a| (the last kick
        //        was a step earlier); the finisher checks the bound
        //   F_i  stretch for the Keplerian shear over one step
        const double m0 = d.m[star];
        const double mu = a.G * m0;
        double rH;
        if (a.hill_fixed) {
            rH = d.rH_fixed[r];
        } else {
            rH = hill(qx, qy, qz, d.hfac[r]);  // positions do not change in the kick
        }
        if (a.flag_next == 2) d.rH[r] = rH;
        float rHb = round_up_f(rH * (1.0 + 1e-6));
        d.rH_bound[r] = rHb;
        double rr = sqrt(qx * qx + qy * qy + qz * qz);
        double rho;
        if (d.escape_reach) {
            // QYM_SEARCH_ESCAPE, the paper's crude sweep (Sec. 2.4): a_E times
            // the Hill radius plus the distance covered at the escape
            // velocity over the step
            rho = a.a_E * (double)rHb + fabs(a.tau) * sqrt(2.0 * mu / rr) + 1e-12 * rr;
        } else {
            double Om = sqrt(mu / (rr * rr * rr));
            double ux = vx + Om * qy, uy = vy - Om * qx, uz = vz;
            double u = sqrt(ux * ux + uy * uy + uz * uz);
            double w = fabs(a.kick_span) * a.a_allow * (double)d.amag[r];
            double sh = fmin(0.8, 2.5 * Om * fabs(a.tau));
            double F = 2.0 / (1.0 - sh);
            rho = F * (a.a_E * (double)rHb + fabs(a.tau) * (u + w)) + 1e-12 * rr;
        }
        // kernels test r^2 < c_i + c_j with c = 2 rho^2 >= ... a superset of
        // r < rho_i + rho_j, as (rho_i + rho_j)^2 <= 2 rho_i^2 + 2 rho_j^2;
        // the factor covers the FP32 rounding of r^2 (a few 1e-7 relative,
        // also in the kick's far-tile form)
        reach = round_up_f(2.0 * rho * rho * (1.0 + 4e-6));
    }
    // heavy bodies enter the FP32 tiles with zero mass (their pull is added
    // in FP64 by the finisher); they still take part in the encounter search
    float gm = (d.heavy_split && r != star && mm >= d.heavy_thr[sys]) ? 0.0f : (float)(a.G * mm);
    const int64_t pr = d.inv ? d.inv[r] : r;  // the kick's order
    d.pk_pos[pr] = make_float4(xh, yh, zh, gm);
    d.pk_lo[pr] = make_float4(xl, yl, zl, reach);
}

cudaError_t launch_drift_pack_from(const Dev &d, const double *qs, const double *vs,
                                   double h_close, double h_open, double tau, double a_E,
                                   double G, int flag_next, int hill_fixed, cudaStream_t st,
                                   double kick_span, double a_allow) {
    DriftArgs a;
    a.qs = qs;
    a.vs = vs;
    a.h_close = h_close;
    a.h_open = h_open;
    a.tau = tau;
    a.kick_span = kick_span;
    a.a_allow = a_allow;
    a.a_E = a_E;
    a.G = G;
    a.flag_next = flag_next;
    a.hill_fixed = hill_fixed;
    int tb = 256;
    k_drift_pack<<<(unsigned)((d.rows + tb - 1) / tb), tb, 0, st>>>(d, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- kick finish
// v += dt * sum over slots of the partial accelerations (fixed slot order);
// |a| is kept for the next crude search. After the first kick of a step
// (check != 0) the Hill radius of this step is computed from the state that
// enters the Kepler drift, and (check == 1, the search fused into this kick)
// rows whose crude-search bounds (|a| allowance, Hill radius bound) were
// exceeded are queued for an exact re-search.
struct FinishArgs {
    double *v;          // velocities to update ([3][rows])
    const double *q;    // positions (for the Hill radius)
    double dt, G;
    float a_allow;      // the crude reach's bound on |a| / |a of the last kick|
    int check, hill_fixed;
    int skip_whole;     // v of systems flagged in d.wh_flag stays
};

constexpr int kFinLanes = 4;  // lanes that share one row's partial sums

__global__ void __launch_bounds__(256) k_finish(Dev d, FinishArgs a) {
    // kFinLanes lanes per position of the kick's order: lane q sums the slots
    // q, q + 4, ... (loads coalesced across positions, dependent FP64 adds in
    // chains a quarter as long), the four parts added in a fixed tree; lane 0
    // then does the row's own work
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t pr = gt / kFinLanes;
    const int q = (int)(gt % kFinLanes);
    const int64_t R = d.rows;
    double ax = 0.0, ay = 0.0, az = 0.0;
    const int nslots = d.kick_cnt ? 1 : d.splits;  // the kick added its slots into slot 0
    if (pr < R)
        for (int s = q; s < nslots; s += kFinLanes) {
            const double *p = d.apart + (int64_t)s * 3 * R;
            ax += p[pr];
            ay += p[R + pr];
            az += p[2 * R + pr];
        }
#pragma unroll
    for (int o = 1; o < kFinLanes; o <<= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (pr >= R || q != 0) return;
    const int64_t r = d.perm ? d.perm[pr] : pr;
    if (d.own_hi > 0 && (r < d.own_lo || r >= d.own_hi)) return;  // another GPU's row
    const int sys = d.sys_of[r];
    const int64_t star = d.offsets[sys];
    if (r == star) return;
    if (d.heavy_split) {
        int h0 = d.heavy_start[sys], h1 = d.heavy_start[sys + 1];
        heavy_pull(d.heavy_rows + h0, h1 - h0, r, a.q[r], a.q[R + r], a.q[2 * R + r], a.q, d.m, R,
                   a.G, ax, ay, az);
    }
    double vx = a.v[r], vy = a.v[R + r], vz = a.v[2 * R + r];
    if (!(a.skip_whole && d.wh_flag && d.wh_flag[sys])) {
        vx += a.dt * ax;
        vy += a.dt * ay;
        vz += a.dt * az;
        a.v[r] = vx; a.v[R + r] = vy; a.v[2 * R + r] = vz;
    }
    float an = round_up_f(sqrt(ax * ax + ay * ay + az * az));
    if (a.check) {
        if (d.vmax)  // the binned search's bound takes the largest |v| entering the drift
            atomicMax(d.vmax + sys, __float_as_int(round_up_f(sqrt(vx * vx + vy * vy + vz * vz))));
        double rH = a.hill_fixed ? d.rH_fixed[r] : hill(a.q[r], a.q[R + r], a.q[2 * R + r], d.hfac[r]);
        d.rH[r] = rH;
        // check 1 (the search fused into this kick): audit its reach
        bool bad = a.check == 1 && !d.escape_reach && (an > a.a_allow * d.amag[r] + 1e-30f ||
                                    rH > (double)d.rH_bound[r]);
        if (bad) {
            unsigned long long k = atomicAdd(d.ctr + C_NRESCAN, 1ull);
            if (k < (unsigned long long)R) d.rescan[k] = (int32_t)r;
        }
    }
    d.amag[r] = an;
}

cudaError_t launch_kick_finish_v(const Dev &d, double *v, const double *q, double dt, double G,
                                 int check, int hill_fixed, cudaStream_t st, double a_allow,
                                 int skip_whole) {
    FinishArgs a;
    a.skip_whole = skip_whole;
    a.v = v;
    a.q = q;
    a.dt = dt;
    a.G = G;
    a.a_allow = (float)a_allow;
    a.check = check;
    a.hill_fixed = hill_fixed;
    int tb = 256;
    k_finish<<<(unsigned)((kFinLanes * d.rows + tb - 1) / tb), tb, 0, st>>>(d, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Hill radii at init
__global__ void k_hill_init(Dev d, double G) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    const int64_t R = d.rows;
    const int64_t star = d.offsets[d.sys_of[r]];
    if (r == star) { d.rH_fixed[r] = 0.0; return; }
    d.rH_fixed[r] = hill(d.q[r], d.q[R + r], d.q[2 * R + r], d.hfac[r]);
}

cudaError_t launch_hill_init(const Dev &d, double G, cudaStream_t st) {
    int tb = 256;
    k_hill_init<<<(unsigned)((d.rows + tb - 1) / tb), tb, 0, st>>>(d, G);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- coordinates
// Barycentric velocity of body i: V_i = v_i - sum_k m_k v_k / (m0 + sum_k m_k)
// (heliocentric -> DH, inverse = 0, in place on d.v); heliocentric velocity:
// v_i = V_i + S / m0 with S = sum_k m_k V_k (inverse = 1, into vout).
// Needs d.S = sum m v of the input velocities and, for the forward direction,
// the total body mass per system in mt.
__global__ void k_mass_total(Dev d, double *mt) {
    int s = blockIdx.x;
    int64_t lo = d.offsets[s], hi = d.offsets[s + 1];
    double t = 0.0;
    for (int64_t r = lo + 1 + threadIdx.x; r < hi; r += blockDim.x) t += d.m[r];
    t = warp_sum(t);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) u += sh[k];
        mt[s] = d.m[lo] + u;
    }
}

__global__ void k_to_dh(Dev d, int inverse, const double *mt, double *vout) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    const int64_t R = d.rows;
    const int sys = d.sys_of[r];
    const int64_t star = d.offsets[sys];
    double *dst = inverse ? vout : d.v;
    if (r == star) {
        dst[r] = dst[R + r] = dst[2 * R + r] = 0.0;
        return;
    }
    double den = inverse ? -d.m[star] : mt[sys];
    for (int c = 0; c < 3; ++c) dst[c * R + r] = d.v[c * R + r] - d.S[3 * sys + c] / den;
}

cudaError_t launch_to_dh_impl(const Dev &d, int inverse, double *vout, double *mt_scratch,
                              cudaStream_t st) {
    cudaError_t e = launch_momentum(d, st);
    if (e != cudaSuccess) return e;
    if (!inverse) {
        k_mass_total<<<d.nsys, 256, 0, st>>>(d, mt_scratch);
    }
    int tb = 256;
    k_to_dh<<<(unsigned)((d.rows + tb - 1) / tb), tb, 0, st>>>(d, inverse, mt_scratch, vout);
    return cudaGetLastError();
}

}  // namespace qym
