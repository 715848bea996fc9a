// sort.cu -- the order in which the mixed kick holds a system's bodies: along
// a Morton (Z-order) curve of their positions, so that each tile of 256
// consecutive bodies is compact in space and the kick can treat tiles far
// from a warp's rows with its one-add separation (kick.cu). Only the layout of
// the kick's operand packs follows this order; the state stays in row order,
// and results depend on it only through the grouping of the FP32 tile sums.
//
// Keys: 10 bits per axis of the position scaled into the cube over the
// system's bounding box, interleaved into 30 bits; bodies ordered by (key,
// row). Sort: stable least-significant-digit radix sort of (key, row) over
// four 8-bit digits; deterministic (per-block digit counts, a scan, and ranks
// within a block from warp match masks). (A bitonic sort of the 64-bit words
// (key, row) in one CTA's shared memory took 0.16 ms for 16384 bodies, against
// about 0.04 ms for these 16 launches: each of its 105 stages moves every word
// through shared memory.)
#include <algorithm>
#include <utility>

#include "qym_internal.cuh"

namespace qym {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                       // keys per thread per pass
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per block

int64_t sort_blocks(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

// bounding box of the bodies (rows 1 .. rows-1) as order-preserving integer
// images of their float coordinates (min and -max), reduced with atomics
__device__ __forceinline__ int fkey(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float kfloat(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_sort_box_init(int *box) {
    if (threadIdx.x < 6) box[threadIdx.x] = 0x7fffffff;
}

__global__ void __launch_bounds__(256) k_sort_box(int64_t rows, const double *q, int *box) {
    float m[6] = {3e38f, 3e38f, 3e38f, 3e38f, 3e38f, 3e38f};
    for (int64_t r = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) {
            const float x = (float)q[c * rows + r];
            m[c] = fminf(m[c], x);
            m[c + 3] = fminf(m[c + 3], -x);
        }
    }
    for (int c = 0; c < 6; ++c) {
        const float v = warp_min(m[c]);
        if ((threadIdx.x & 31) == 0) atomicMin(box + c, fkey(v));
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    // 10 bits -> every third bit of 30
    x &= 0x3ff;
    x = (x | (x << 16)) & 0x030000ff;
    x = (x | (x << 8)) & 0x0300f00f;
    x = (x | (x << 4)) & 0x030c30c3;
    x = (x | (x << 2)) & 0x09249249;
    return x;
}

// Morton code of row r from the box (min, -max per axis, as fkey images)
__device__ __forceinline__ uint32_t morton_code(int64_t rows, const double *q, int64_t r,
                                                const int *box) {
    // one scale for the three axes (cubic cells): a thin disk then orders by
    // its plane first instead of splitting its few bodies' heights at the top
    float span = 0.0f;
    for (int c = 0; c < 3; ++c) span = fmaxf(span, -kfloat(box[c + 3]) - kfloat(box[c]));
    uint32_t code = 0;
    for (int c = 0; c < 3; ++c) {
        const float lo = kfloat(box[c]);
        float u = span > 0.0f ? ((float)q[c * rows + r] - lo) / span : 0.0f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        const uint32_t b = min((uint32_t)(u * 1024.0f), 1023u);
        code |= spread10(b) << c;
    }
    return code;
}
__global__ void __launch_bounds__(256) k_sort_keys(int64_t rows, const double *q, const int *box,
                                                    uint32_t *keys, int32_t *vals) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // body k = row k + 1
    if (k >= rows - 1) return;
    const int64_t r = k + 1;
    keys[k] = morton_code(rows, q, r, box);
    vals[k] = (int32_t)r;
}

// digit counts of each block: hist[digit * nblk + block]
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(int64_t n, const uint32_t *keys,
                                                            int shift, uint32_t *hist, int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        const int64_t k = base + it * kSortThreads + threadIdx.x;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of the m = 256 * nblk counts (one CTA)
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t *hist, int m) {
    __shared__ uint32_t part[1024];
    const int per = (m + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int b = b0; b < b0 + per && b < m; ++b) s += hist[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int b = b0; b < b0 + per && b < m; ++b) {
        const uint32_t c = hist[b];
        hist[b] = run;
        run += c;
    }
}

// stable scatter: each block's keys in rounds of 256 (thread order), a key's
// place = the block's offset for its digit + the keys with that digit in
// earlier rounds + those in earlier warps of this round + earlier lanes
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(int64_t n, const uint32_t *kin,
                                                               const int32_t *vin, uint32_t *kout,
                                                               int32_t *vout, int shift,
                                                               const uint32_t *hist, int nblk) {
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[NW][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = hist[tid * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int it = 0; it < kSortItems; ++it) {
        for (int q = 0; q < NW; ++q) wc[q][tid] = 0;
        __syncthreads();
        const int64_t k = base + it * kSortThreads + tid;
        const bool act = k < n;
        const uint32_t key = act ? kin[k] : 0u;
        const int dig = act ? (int)((key >> shift) & 255) : 256 + lane;  // idle lanes apart
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (act && rank == 0) wc[w][dig] = (uint32_t)__popc(peers);
        __syncthreads();
        if (act) {
            uint32_t before = run[dig];
            for (int q = 0; q < w; ++q) before += wc[q][dig];
            const uint32_t pos = before + (uint32_t)rank;
            kout[pos] = key;
            vout[pos] = vin[k];
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int q = 0; q < NW; ++q) tot += wc[q][tid];
        run[tid] += tot;
        __syncthreads();
    }
}

// position p (1 .. rows-1) holds row perm[p]; inv[perm[p]] = p; row 0 stays
__global__ void __launch_bounds__(256) k_sort_perm(int64_t rows, const int32_t *vals,
                                                    int32_t *perm, int32_t *inv) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        perm[0] = 0;
        inv[0] = 0;
    }
    if (k >= rows - 1) return;
    const int32_t r = vals[k];
    perm[k + 1] = r;
    inv[r] = (int32_t)(k + 1);
}

cudaError_t launch_sort_rows(int64_t rows, const double *q, const SortScratch &s, int32_t *perm,
                             int32_t *inv, cudaStream_t st) {
    const int64_t n = rows - 1;
    if (n < 1) return cudaSuccess;
    const int nblk = (int)sort_blocks(n);
    const unsigned g = (unsigned)((n + 255) / 256);
    k_sort_box_init<<<1, 32, 0, st>>>(s.box);
    k_sort_box<<<(unsigned)std::min<int64_t>(g, 4 * 152), 256, 0, st>>>(rows, q, s.box);
    k_sort_keys<<<g, 256, 0, st>>>(rows, q, s.box, s.k0, s.v0);
    uint32_t *ka = s.k0, *kb = s.k1;
    int32_t *va = s.v0, *vb = s.v1;
    for (int shift = 0; shift < 32; shift += 8) {
        k_sort_hist<<<nblk, kSortThreads, 0, st>>>(n, ka, shift, s.hist, nblk);
        k_sort_scan<<<1, 1024, 0, st>>>(s.hist, 256 * nblk);
        k_sort_scatter<<<nblk, kSortThreads, 0, st>>>(n, ka, va, kb, vb, shift, s.hist, nblk);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    k_sort_perm<<<g, 256, 0, st>>>(rows, va, perm, inv);
    return cudaGetLastError();
}

}  // namespace qym
