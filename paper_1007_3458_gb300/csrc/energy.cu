// energy.cu -- total energy of each system (Sec. 2, Eqs. 2-4), FP64:
//   E = |S|^2 / (2 m0) + sum_i [m_i v_i^2 / 2 - G m0 m_i / |Q_i|]
//       - (1/2) sum_{i != j} G m_i m_j / |Q_i - Q_j|        (i, j bodies),
// the pair sum taken over all ordered pairs in tiles (the paper's N^2
// over-count) with the star mass restored for the star terms.
#include "qym_internal.cuh"

namespace qym {

constexpr int ETILE = 256;

// one CTA per item (i0, i1, j0, j1) of one system; writes its partial of
// sum_i [m v^2 / 2 - G m0 m / r - (1/2) m_i sum_j G m_j / r_ij]
__global__ void __launch_bounds__(256) k_energy_items(const int4 *items, const int32_t *isys,
                                                      const int64_t *offsets, int64_t R,
                                                      const double *m, const double *q,
                                                      const double *v, double G, double *part) {
    __shared__ D4 s_q[ETILE];
    __shared__ double red[8];
    const int4 it = items[blockIdx.x];
    const int64_t star = offsets[isys[blockIdx.x]];
    const double m0 = m[star];
    const int64_t i = it.x + threadIdx.x;
    const bool act = i < it.y;
    double xi = 0, yi = 0, zi = 0;
    if (act) { xi = q[i]; yi = q[R + i]; zi = q[2 * R + i]; }
    double phi = 0.0;
    for (int jt = it.z; jt < it.w; jt += ETILE) {
        int n = min(ETILE, it.w - jt);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int64_t j = jt + t;
            s_q[t] = D4{q[j], q[R + j], q[2 * R + j], G * m[j]};
        }
        __syncthreads();
        if (act) {
            for (int t = 0; t < n; ++t) {
                D4 p = s_q[t];
                double dx = xi - p.x, dy = yi - p.y, dz = zi - p.z;
                double r2 = dx * dx + dy * dy + dz * dz;
                phi += (r2 > 0.0) ? p.w * rsqrt(r2) : 0.0;
            }
        }
    }
    double e = 0.0;
    if (act) {
        double mi = m[i];
        double vx = v[i], vy = v[R + i], vz = v[2 * R + i];
        double r = sqrt(xi * xi + yi * yi + zi * zi);
        e = 0.5 * mi * (vx * vx + vy * vy + vz * vz) - G * m0 * mi / r - 0.5 * mi * phi;
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        part[blockIdx.x] = s;
    }
}

// per system: fixed-order sum of its items' partials plus |S|^2 / (2 m0),
// with S = sum m v computed here in fixed order as well
__global__ void k_energy_final(int32_t nsys, const int64_t *offsets, const int32_t *item0,
                               const double *part, const double *m, const double *v, int64_t R,
                               double *E) {
    int s = blockIdx.x;
    if (s >= nsys) return;
    int64_t lo = offsets[s], hi = offsets[s + 1];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t r = lo + 1 + threadIdx.x; r < hi; r += blockDim.x) {
        sx += m[r] * v[r];
        sy += m[r] * v[R + r];
        sz += m[r] * v[2 * R + r];
    }
    __shared__ double sh[3][8];
    sx = warp_sum(sx); sy = warp_sum(sy); sz = warp_sum(sz);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = sx; sh[1][threadIdx.x >> 5] = sy; sh[2][threadIdx.x >> 5] = sz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S[3] = {0, 0, 0};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            for (int c = 0; c < 3; ++c) S[c] += sh[c][k];
        double e = 0.0;
        for (int k = item0[s]; k < item0[s + 1]; ++k) e += part[k];
        E[s] = e + (S[0] * S[0] + S[1] * S[1] + S[2] * S[2]) / (2.0 * m[lo]);
    }
}

// host: items of at most 256 i-rows against the whole system
int32_t energy_items_host(const int64_t *offsets, int32_t nsys, int4 *items, int32_t *isys,
                          int32_t *item0) {
    int32_t n = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        if (item0) item0[s] = n;
        int64_t b0 = offsets[s] + 1, b1 = offsets[s + 1];
        for (int64_t i0 = b0; i0 < b1; i0 += 256) {
            if (items) {
                items[n] = make_int4((int)i0, (int)(i0 + 256 < b1 ? i0 + 256 : b1), (int)b0, (int)b1);
                isys[n] = s;
            }
            ++n;
        }
    }
    if (item0) item0[nsys] = n;
    return n;
}

cudaError_t launch_energy_items(int32_t nitems, const int4 *items, const int32_t *isys,
                                const int32_t *item0, int32_t nsys, const int64_t *offsets,
                                int64_t R, const double *m, const double *q, const double *v,
                                double G, double *part, double *E, cudaStream_t st) {
    if (nitems > 0)
        k_energy_items<<<nitems, 256, 0, st>>>(items, isys, offsets, R, m, q, v, G, part);
    k_energy_final<<<nsys, 256, 0, st>>>(nsys, offsets, item0, part, m, v, R, E);
    return cudaGetLastError();
}

}  // namespace qym
