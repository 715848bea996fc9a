// kick.cu -- E_Int: all-pairs interaction accelerations (Sec. 2, Eq. 4),
//   a_i = -sum_{j >= 1, j != i} G m_j (Q_i - Q_j) / |Q_i - Q_j|^3,
// the star's mass zeroed (its row is simply not in any tile), fused with the
// crude close-encounter search of the first kick of a step (Sec. 2.4).
//
// Work decomposition: one CTA per work item (system, i-block, j-range). The
// i rows of the block live in registers (IPT per thread); j rows stream
// through shared memory in tiles of TILE. Each item writes its partial sums to
// its own slot of apart[slot][3][rows]; the finisher adds the slots in a fixed
// order, so results are deterministic.
//
// Mixed precision (QYM_KICK_MIXED): positions are split into float hi + lo
// parts, the separation is formed as (hi_i - hi_j) + (lo_i - lo_j) (a
// double-single difference, accurate to ~1e-7 relative even for close pairs
// far from the star), the pair force is FP32 with rsqrt, and the FP32 tile sums
// are folded every FOLD pairs into a float two-sum (hi, lo) accumulator that
// is returned as a double. The FP32 arithmetic runs on Blackwell's packed
// FP32x2 instructions, two j rows per instruction.
#include "qym_internal.cuh"

namespace qym {

constexpr int TILE = kKickTile;
constexpr int FOLD = 64;
#ifndef QYM_KICK_UNROLL
#define QYM_KICK_UNROLL 4
#endif
constexpr int kPairUnroll = QYM_KICK_UNROLL;  // j pairs per unrolled step

struct KickArgs {
    const int4 *items;
    const int32_t *slots;
    const float4 *pos;      // (x_hi, y_hi, z_hi, G m)
    const float4 *lo;       // (x_lo, y_lo, z_lo, c = 2 rho^2 of the crude reach rho)
    const double *q;        // [3][rows] (FP64 path)
    const double *m;        // [rows] (FP64 path)
    double G;
    double *apart;
    int64_t rows;
    int2 *cand;
    int64_t max_cand;
    unsigned long long *ncand;
    int4 *fchunk;
    int64_t max_fchunk;
    unsigned long long *nfchunk;
    int32_t *status;
    int32_t far_tiles;      // 1: tiles far from a warp's rows take the one-add separation
    const int32_t *perm;    // row of each position of the packs (NULL: row order)
    const float4 *far;      // (o_x, o_y, o_z, G m): offset from the tile's reference point
    const float4 *tile;     // per tile: (c_x, c_y, c_z, R), box min (x, y, z, -), box max
    int32_t *blk_cnt = nullptr;  // arrivals per i-block (NULL: each slot stays for the finisher)
    int32_t splits = 1;          // items (slots) per i-block
};

// The last CTA of an i-block to finish (arrivals counted per i-block, the
// counter reset by that CTA for the next launch) adds the block's `splits`
// slots into slot 0, in the order a reader of the slots used (lane q of
// four summing slots q, q + 4, ..., the four parts added as (0 + 1) + (2 + 3)),
// and discards the other slots' lines from L2 (PTX discard.global.L2): they
// are dead, and discarded lines are not written back, so the partial sums of
// all splits stay on chip and HBM sees only slot 0. Lines shared with a
// neighbouring i-block's rows are kept.
// (not inlined: as a call it leaves the register allocation of the kick's
// tile loop as it is without this epilogue)
template <int IPT>
__device__ __noinline__ void sum_block_slots(const KickArgs &a, const int (&gi)[IPT], int i_lo,
                                             int i_hi) {
    __shared__ int s_last;
    __syncthreads();  // every thread's slot stores issued
    if (threadIdx.x == 0) {
        // release: the block's slot stores (ordered before by the barrier)
        // precede the arrival; acquire: the last arrival sees every slot
        const int blk = (int)(blockIdx.x / a.splits);
        int old;
        asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;"
                     : "=r"(old)
                     : "l"(a.blk_cnt + blk)
                     : "memory");
        s_last = old == a.splits - 1;
        if (s_last) a.blk_cnt[blk] = 0;
    }
    __syncthreads();
    if (!s_last) return;
    const int64_t rows = a.rows;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        if (gi[k] < i_hi) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double *p = a.apart + (int64_t)c * rows + gi[k];
                const int64_t st = 3 * rows;
                double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
                int s = 0;
                for (; s + 3 < a.splits; s += 4) {
                    p0 += __ldcg(p + s * st);
                    p1 += __ldcg(p + (s + 1) * st);
                    p2 += __ldcg(p + (s + 2) * st);
                    p3 += __ldcg(p + (s + 3) * st);
                }
                if (s < a.splits) p0 += __ldcg(p + s * st);
                if (s + 1 < a.splits) p1 += __ldcg(p + (s + 1) * st);
                if (s + 2 < a.splits) p2 += __ldcg(p + (s + 2) * st);
                a.apart[(int64_t)c * rows + gi[k]] = (p0 + p1) + (p2 + p3);
            }
        }
    }
    __syncthreads();  // every read done before a line goes
    // whole 128-byte lines inside this block's rows of slots 1 .. splits-1:
    // per slot-component row sc, the lines from the first 128-byte boundary
    // at or after row i_lo to the last one at or before row i_hi
    const int L = (int)(((int64_t)(i_hi - i_lo) * 8 + 127) >> 7);  // lines a row range can span
    const int tot = (a.splits - 1) * 3 * L;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
        const int sc = 3 + t / L;
        const uintptr_t base = (uintptr_t)(a.apart + (int64_t)sc * rows);
        const uintptr_t l0 = (base + (uintptr_t)i_lo * 8 + 127) & ~(uintptr_t)127;
        const uintptr_t l1 = (base + (uintptr_t)i_hi * 8) & ~(uintptr_t)127;
        const uintptr_t line = l0 + ((uintptr_t)(t % L) << 7);
        if (line < l1)  // [line, line + 128) inside [start, end)
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
    }
}

// a + b + c for |c| far below |a + b|, rounded once: the rounding error of
// a + b (Knuth's two-sum) joins c before the last rounding
__device__ __forceinline__ float ds_add(float a, float b, float c) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return __fadd_rn(s, __fadd_rn(e, c));
}

// min(a, b, c) in one instruction (the three-input form of sm_100 and later)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// append candidate (i, j) from a divergent branch, warp-aggregated
__device__ __forceinline__ void push_candidate(const KickArgs &a, int i, int j) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.ncand, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < (unsigned long long)a.max_cand)
        a.cand[idx] = make_int2(i, j);
    else if (lane == leader)
        atomicOr(a.status, QYM_ST_CAND_OVERFLOW);
}

// j rows of a tile sit in shared memory in pairs (j = 2p, 2p+1), each pair as
// four float4: (xh0, xh1, yh0, yh1), (zh0, zh1, Gm0, Gm1), (xl0, xl1, yl0,
// yl1), (zl0, zl1, -c0, -c1). A float4's halves are float2 operands of the
// packed FP32 instructions (FADD2 / FMUL2 / FFMA2), so one instruction serves
// both j of a pair for an i row; the i operands are per-thread constants,
// negated and duplicated once. Each lane computes exactly what the scalar
// form (Q_i - Q_j, r^2, rsqrt, m r^-3, force) computes, with the sign of
// the separation flipped: d = Q_j - Q_i, a_i += (G m_j / r^3) d.
struct JPairs {
    float4 *a, *b, *c, *d;
};

// Pair forces of the j pairs [p0, p1) for the IPT rows of a thread. With
// FLAG, each i keeps the minimum over the chunk of r^2 - c_j, c_j = 2 rho_j^2
// (no branch); since (rho_i + rho_j)^2 <= c_i + c_j, a chunk without a
// candidate of i has that minimum >= c_i and needs no further look; a chunk
// with a smaller minimum is recorded and re-tested exactly by k_flag_chunks.
// In a chunk of the diagonal tile the row's own j (r^2 = 0) is left out of
// the minimum. Without FORCE only the search runs (the same separations and
// r^2).
template <int IPT, bool FLAG, bool DIAG, bool FORCE>
__device__ __forceinline__ void mixed_chunk(const JPairs &s, int p0, int p1, int jt,
                                            const int (&gi)[IPT],
                                            const float2 (&nxh)[IPT], const float2 (&nyh)[IPT],
                                            const float2 (&nzh)[IPT], const float2 (&nxl)[IPT],
                                            const float2 (&nyl)[IPT], const float2 (&nzl)[IPT],
                                            float2 (&fx)[IPT], float2 (&fy)[IPT],
                                            float2 (&fz)[IPT], float (&mind)[IPT]) {
#pragma unroll kPairUnroll
    for (int p = p0; p < p1; ++p) {
        const float4 A = s.a[p], B = s.b[p], C = s.c[p], D = s.d[p];
        const float2 xh = make_float2(A.x, A.y), yh = make_float2(A.z, A.w);
        const float2 zh = make_float2(B.x, B.y), gm = make_float2(B.z, B.w);
        const float2 xl = make_float2(C.x, C.y), yl = make_float2(C.z, C.w);
        const float2 zl = make_float2(D.x, D.y), nc = make_float2(D.z, D.w);
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float2 dx = __fadd2_rn(__fadd2_rn(xh, nxh[k]), __fadd2_rn(xl, nxl[k]));
            const float2 dy = __fadd2_rn(__fadd2_rn(yh, nyh[k]), __fadd2_rn(yl, nyl[k]));
            const float2 dz = __fadd2_rn(__fadd2_rn(zh, nzh[k]), __fadd2_rn(zl, nzl[k]));
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            if (FORCE) {
                const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                float2 sm = __fmul2_rn(__fmul2_rn(gm, ri), __fmul2_rn(ri, ri));
                if (DIAG) {
                    sm.x = (r2.x > 0.0f) ? sm.x : 0.0f;
                    sm.y = (r2.y > 0.0f) ? sm.y : 0.0f;
                }
                fx[k] = __ffma2_rn(sm, dx, fx[k]);
                fy[k] = __ffma2_rn(sm, dy, fy[k]);
                fz[k] = __ffma2_rn(sm, dz, fz[k]);
            }
            if (FLAG) {
                float2 t = __fadd2_rn(r2, nc);
                if (DIAG) {  // a row is not its own partner
                    t.x = (jt + 2 * p == gi[k]) ? 3.0e38f : t.x;
                    t.y = (jt + 2 * p + 1 == gi[k]) ? 3.0e38f : t.y;
                }
                mind[k] = fmin3(mind[k], t.x, t.y);
            }
        }
    }
}

// The same for a tile far from every row of the warp (far_tile): the j rows
// are held as FP32 offsets o_j = Q_j - c from the tile's reference point c
// (two j per float4 pair: (ox0, ox1, oy0, oy1), (oz0, oz1, Gm0, Gm1)) and
// each row as d_i = c - Q_i, formed once per tile in double-single and
// rounded; the separation is one packed add o_j + d_i per coordinate instead
// of three. With every pair at least the tile's radius R apart, both offsets
// are at most about the separation, so its relative error stays a few
// 2^-24; the rest (r^2, rsqrt, m r^-3, force, search) is the near form's.
struct JFar {
    float4 *a, *b, *d;  // d: the near layout's fourth float4, for -c0, -c1
};

template <int IPT, bool FLAG, bool FORCE>
__device__ __forceinline__ void far_chunk(const JFar &s, int p0, int p1, const float2 (&dxi)[IPT],
                                          const float2 (&dyi)[IPT], const float2 (&dzi)[IPT],
                                          float2 (&fx)[IPT], float2 (&fy)[IPT], float2 (&fz)[IPT],
                                          float (&mind)[IPT]) {
#pragma unroll kPairUnroll
    for (int p = p0; p < p1; ++p) {
        const float4 A = s.a[p], B = s.b[p];
        const float2 ox = make_float2(A.x, A.y), oy = make_float2(A.z, A.w);
        const float2 oz = make_float2(B.x, B.y), gm = make_float2(B.z, B.w);
        float2 nc = make_float2(0.0f, 0.0f);
        if (FLAG) {
            const float4 D = s.d[p];
            nc = make_float2(D.z, D.w);
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float2 dx = __fadd2_rn(ox, dxi[k]);
            const float2 dy = __fadd2_rn(oy, dyi[k]);
            const float2 dz = __fadd2_rn(oz, dzi[k]);
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            if (FORCE) {
                const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                const float2 sm = __fmul2_rn(__fmul2_rn(gm, ri), __fmul2_rn(ri, ri));
                fx[k] = __ffma2_rn(sm, dx, fx[k]);
                fy[k] = __ffma2_rn(sm, dy, fy[k]);
                fz[k] = __ffma2_rn(sm, dz, fz[k]);
            }
            if (FLAG) {
                const float2 t = __fadd2_rn(r2, nc);
                mind[k] = fmin3(mind[k], t.x, t.y);
            }
        }
    }
}

// record that row i's crude minimum over the j rows [j0, j1) fell below c_i
// (divergent branch, warp-aggregated); k_flag_chunks re-tests them
__device__ __forceinline__ void push_flag(const KickArgs &a, int i, int j0, int j1) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.nfchunk, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < (unsigned long long)a.max_fchunk)
        a.fchunk[idx] = make_int4(i, j0, j1, 0);
    else if (lane == leader)
        atomicOr(a.status, QYM_ST_CAND_OVERFLOW);
}

// FORCE = false: the crude search alone (no partial sums written)
template <int IPT, bool FLAG, bool FORCE>
__global__ void __launch_bounds__(256) k_kick_mixed(KickArgs a) {
    __shared__ float4 s_a[TILE / 2], s_b[TILE / 2], s_c[TILE / 2], s_d[TILE / 2];
    __shared__ float4 s_fa[TILE / 2], s_fb[TILE / 2];
    const JPairs sp{s_a, s_b, s_c, s_d};
    const JFar sf{s_fa, s_fb, s_d};
    const int4 it = a.items[blockIdx.x];
    const int slot = a.slots[blockIdx.x];
    float rho[IPT];
    float2 nxh[IPT], nyh[IPT], nzh[IPT], nxl[IPT], nyl[IPT], nzl[IPT];  // -Q_i, duplicated
    int gi[IPT];
    float ahx[IPT], ahy[IPT], ahz[IPT], alx[IPT], aly[IPT], alz[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        int i = it.x + threadIdx.x + k * blockDim.x;
        gi[k] = i;
        // idle lane: parked far away so its arithmetic stays finite
        float4 p = make_float4(1e18f, 1e18f, 1e18f, 0.0f), l = make_float4(0.f, 0.f, 0.f, -1e30f);
        if (i < it.y) {
            p = a.pos[i];
            l = a.lo[i];
        }
        rho[k] = l.w;
        nxh[k] = make_float2(-p.x, -p.x); nyh[k] = make_float2(-p.y, -p.y);
        nzh[k] = make_float2(-p.z, -p.z); nxl[k] = make_float2(-l.x, -l.x);
        nyl[k] = make_float2(-l.y, -l.y); nzl[k] = make_float2(-l.z, -l.z);
        ahx[k] = ahy[k] = ahz[k] = alx[k] = aly[k] = alz[k] = 0.0f;
    }
    const int i_lo = it.x, i_hi = it.x + (int)(IPT * blockDim.x);
    for (int jt = it.z, n = 0; jt < it.w; jt += n) {
        // windows of at most TILE positions; with far tiles never across the
        // end of a tile (positions 1 + TILE t ..), whose data a window uses
        n = min(TILE, it.w - jt);
        if (a.far_tiles) n = min(n, 1 + ((jt - 1) / TILE + 1) * TILE - jt);
        const int np = (n + 1) >> 1;
        const bool diag = (jt < i_hi) && (jt + n > i_lo);
        // Far tiles (a.far_tiles: the bodies in Morton order, tiles aligned
        // at position 1 + TILE t, their data from k_tile_prep): a warp whose
        // every row lies at least the tile's radius R outside its box takes
        // the one-add separation; every pair is then at least R apart,
        // |o_j| <= R <= r and |d_i| <= 2 r, so that with o_j and d_i each
        // rounded once the separation is within 4 2^-24 r (the row test's
        // own rounding is within its 2% margin).
        bool far = false;
        // quiet (searching kick, a window of another block's tile): no pair
        // of the window can be a candidate, as every row lies farther from
        // the tile's box than its reach and the tile's largest one allow
        // (r^2 >= c_i + c_max, with a 3% and an absolute margin for the FP32
        // box distance): the window takes the plain form, far or near, with
        // no search arithmetic
        bool quiet = false;
        float2 dxi[IPT], dyi[IPT], dzi[IPT];
        float4 m0 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.far_tiles && !diag) {
            const float4 *tm = a.tile + 3 * ((jt - 1) / TILE);
            m0 = tm[0];
            const float4 m1 = tm[1], m2 = tm[2];
            const float R = m0.w;
            bool mine = true, calm = true;
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const float x = -nxh[k].x, y = -nyh[k].x, z = -nzh[k].x;
                const float ex = fmaxf(fmaxf(m1.x - x, x - m2.x), 0.0f);
                const float ey = fmaxf(fmaxf(m1.y - y, y - m2.y), 0.0f);
                const float ez = fmaxf(fmaxf(m1.z - z, z - m2.z), 0.0f);
                const float d2 = ex * ex + ey * ey + ez * ez;
                mine = mine && (d2 >= 1.02f * R * R);
                if (FLAG)
                    calm = calm && (d2 >= 1.03f * (rho[k] + m1.w) + 1e-9f * (x * x + y * y + z * z));
            }
            far = __all_sync(0xffffffffu, mine);
            if (FLAG) quiet = __all_sync(0xffffffffu, calm);
        }
        // which layouts this CTA's warps need
        const bool any_far = __syncthreads_or(far);
        const bool any_near = __syncthreads_or(!far);
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            const int j0 = jt + 2 * t;
            const bool two = 2 * t + 1 < n;
            if (any_near) {
                const float4 p0 = a.pos[j0], l0 = a.lo[j0];
                // an odd tail is padded with a massless row far from everything
                float4 p1 = make_float4(2e18f, 2e18f, 2e18f, 0.0f), l1 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (two) {
                    p1 = a.pos[j0 + 1];
                    l1 = a.lo[j0 + 1];
                }
                s_a[t] = make_float4(p0.x, p1.x, p0.y, p1.y);
                s_b[t] = make_float4(p0.z, p1.z, p0.w, p1.w);
                s_c[t] = make_float4(l0.x, l1.x, l0.y, l1.y);
                s_d[t] = make_float4(l0.z, l1.z, -l0.w, -l1.w);
            }
            if (any_far) {
                const float4 f0 = a.far[j0];
                float4 f1 = make_float4(2e18f, 2e18f, 2e18f, 0.0f);
                float c1 = 0.0f;
                if (two) {
                    f1 = a.far[j0 + 1];
                    c1 = a.lo[j0 + 1].w;
                }
                s_fa[t] = make_float4(f0.x, f1.x, f0.y, f1.y);
                s_fb[t] = make_float4(f0.z, f1.z, f0.w, f1.w);
                if (FLAG && !any_near) s_d[t] = make_float4(0.f, 0.f, -a.lo[j0].w, -c1);
            }
        }
        __syncthreads();
        if (far) {
            // d_i = c - Q_i = (c - x_hi) - x_lo rounded once, duplicated for
            // the packed form
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const float dx = ds_add(m0.x, nxh[k].x, nxl[k].x);
                const float dy = ds_add(m0.y, nyh[k].x, nyl[k].x);
                const float dz = ds_add(m0.z, nzh[k].x, nzl[k].x);
                dxi[k] = make_float2(dx, dx);
                dyi[k] = make_float2(dy, dy);
                dzi[k] = make_float2(dz, dz);
            }
        }
        for (int c = 0; c < np; c += FOLD / 2) {
            const int ce = min(c + FOLD / 2, np);
            float2 fx[IPT], fy[IPT], fz[IPT];
            float mind[IPT];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                fx[k] = fy[k] = fz[k] = make_float2(0.0f, 0.0f);
                mind[k] = 3.0e38f;
            }
            if (far && quiet)
                far_chunk<IPT, false, FORCE>(sf, c, ce, dxi, dyi, dzi, fx, fy, fz, mind);
            else if (far)
                far_chunk<IPT, FLAG, FORCE>(sf, c, ce, dxi, dyi, dzi, fx, fy, fz, mind);
            else if (quiet)
                mixed_chunk<IPT, false, false, FORCE>(sp, c, ce, jt, gi, nxh, nyh, nzh, nxl, nyl,
                                                      nzl, fx, fy, fz, mind);
            else if (diag)
                mixed_chunk<IPT, FLAG, true, FORCE>(sp, c, ce, jt, gi, nxh, nyh, nzh, nxl, nyl, nzl,
                                                    fx, fy, fz, mind);
            else
                mixed_chunk<IPT, FLAG, false, FORCE>(sp, c, ce, jt, gi, nxh, nyh, nzh, nxl, nyl, nzl,
                                                     fx, fy, fz, mind);
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                if (FORCE) {
                    float s, e;
                    two_sum(ahx[k], fx[k].x + fx[k].y, s, e); ahx[k] = s; alx[k] += e;
                    two_sum(ahy[k], fy[k].x + fy[k].y, s, e); ahy[k] = s; aly[k] += e;
                    two_sum(ahz[k], fz[k].x + fz[k].y, s, e); ahz[k] = s; alz[k] += e;
                }
                // only partners j > i become candidates, so a chunk wholly at or
                // below the row needs no record
                const int j1 = jt + min(2 * ce, n);
                if (FLAG && mind[k] < rho[k] && j1 - 1 > gi[k]) push_flag(a, gi[k], jt + 2 * c, j1);
            }
        }
    }
    if (!FORCE) return;
    const int64_t rows = a.rows;
    double *out = a.apart + (int64_t)slot * 3 * rows;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        if (gi[k] < it.y) {
            out[gi[k]] = (double)ahx[k] + (double)alx[k];
            out[rows + gi[k]] = (double)ahy[k] + (double)aly[k];
            out[2 * rows + gi[k]] = (double)ahz[k] + (double)alz[k];
        }
    }
    if (a.blk_cnt) sum_block_slots<IPT>(a, gi, it.x, it.y);
}

// Exact test of the flagged chunks, one warp per entry, lane l on the j rows
// j0 + l and j0 + 32 + l: candidates (i, j), i < j, with r^2 < c_i + c_j, the
// separation formed from the same split positions in the same order as the
// kick forms it, so the candidate set is the kick's own. Entries hold
// positions of the packs' order (each pair once: from the smaller position);
// candidates are rows. The last CTA to finish resets the entry counter for
// the next search kick.
__global__ void __launch_bounds__(256) k_flag_chunks(KickArgs a, unsigned long long *done) {
    unsigned long long n = *(volatile unsigned long long *)a.nfchunk;
    if (n > (unsigned long long)a.max_fchunk) n = a.max_fchunk;
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         e < n; e += warps) {
        const int4 f = a.fchunk[e];
        const float4 pi = a.pos[f.x], li = a.lo[f.x];
        for (int j = f.y + lane; j < f.z; j += 32) {
            if (j <= f.x) continue;
            const float4 pj = a.pos[j], lj = a.lo[j];
            const float dx = (pi.x - pj.x) + (li.x - lj.x);
            const float dy = (pi.y - pj.y) + (li.y - lj.y);
            const float dz = (pi.z - pj.z) + (li.z - lj.z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < li.w + lj.w) {
                // positions of the kick's order -> rows, smaller row first
                int ri = f.x, rj = j;
                if (a.perm) {
                    ri = a.perm[ri];
                    rj = a.perm[rj];
                }
                push_candidate(a, min(ri, rj), max(ri, rj));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1ull) == gridDim.x - 1) {
            *a.nfchunk = 0;
            *done = 0;
        }
    }
}

// ---------------------------------------------------------------- FP64 form
template <int IPT, bool FLAG, bool FORCE>
__global__ void __launch_bounds__(256) k_kick_fp64(KickArgs a) {
    __shared__ D4 s_q[TILE];
    __shared__ float s_rho[TILE];
    const int4 it = a.items[blockIdx.x];
    const int slot = a.slots[blockIdx.x];
    const int64_t rows = a.rows;
    double xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
    float rho[IPT];
    int gi[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        int i = it.x + threadIdx.x + k * blockDim.x;
        gi[k] = i;
        if (i < it.y) {
            xi[k] = a.q[i]; yi[k] = a.q[rows + i]; zi[k] = a.q[2 * rows + i];
            rho[k] = FLAG ? a.lo[i].w : 0.0f;
        } else {
            xi[k] = yi[k] = zi[k] = 1e18;
            rho[k] = -1e30f;
        }
        ax[k] = ay[k] = az[k] = 0.0;
    }
    const double G = a.G;
    for (int jt = it.z; jt < it.w; jt += TILE) {
        const int n = min(TILE, it.w - jt);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            int j = jt + t;
            s_q[t] = D4{a.q[j], a.q[rows + j], a.q[2 * rows + j], G * a.m[j]};
            if (FLAG) s_rho[t] = a.lo[j].w;
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
            const D4 p = s_q[j];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                double dx = xi[k] - p.x, dy = yi[k] - p.y, dz = zi[k] - p.z;
                double r2 = dx * dx + dy * dy + dz * dz;
                if (FORCE) {
                    double ri = rsqrt(r2);
                    double s = p.w * (ri * ri) * ri;
                    s = (r2 > 0.0) ? s : 0.0;
                    ax[k] -= s * dx;
                    ay[k] -= s * dy;
                    az[k] -= s * dz;
                }
                if (FLAG) {
                    if ((float)r2 < rho[k] + s_rho[j]) {
                        int gj = jt + j;
                        if (gi[k] < gj) push_candidate(a, gi[k], gj);
                    }
                }
            }
        }
    }
    if (!FORCE) return;
    double *out = a.apart + (int64_t)slot * 3 * rows;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        if (gi[k] < it.y) {
            out[gi[k]] = ax[k];
            out[rows + gi[k]] = ay[k];
            out[2 * rows + gi[k]] = az[k];
        }
    }
    if (a.blk_cnt) sum_block_slots<IPT>(a, gi, it.x, it.y);
}

// ---------------------------------------------------------------- items
// Items for a batch: for each system (bodies are rows lo+1 .. hi-1), i-blocks
// of threads*ipt rows times `splits` contiguous j-ranges. Every (i-block,
// split) pair gets an item, even when its j-range is empty, so every slot of
// every row is written. Only rows in [i_lo, i_hi) get i-blocks (a rank's own
// rows when a system's step is split over several GPUs); the j-ranges always
// cover the whole system, so a row's partial sums do not depend on the range.
static int64_t items_i_begin(int64_t b0, int64_t i_lo) { return b0 > i_lo ? b0 : i_lo; }
static int64_t items_i_end(int64_t b1, int64_t i_hi) { return b1 < i_hi ? b1 : i_hi; }

int32_t kick_items_count(const int64_t *offsets, int32_t nsys, const KickTune &t, int64_t i_lo,
                         int64_t i_hi) {
    int64_t tot = 0;
    const int64_t ti = (int64_t)t.threads * t.ipt;
    for (int32_t s = 0; s < nsys; ++s) {
        const int64_t a = items_i_begin(offsets[s] + 1, i_lo), b = items_i_end(offsets[s + 1], i_hi);
        const int64_t nb = b - a;
        if (nb > 0) tot += ((nb + ti - 1) / ti) * t.splits;
    }
    return (int32_t)tot;
}

void kick_items_host(const int64_t *offsets, int32_t nsys, const KickTune &t, int4 *items,
                     int32_t *slots, int32_t *nitems, int32_t *splits_used, int32_t max_items,
                     int64_t i_lo, int64_t i_hi, int32_t align) {
    const int64_t ti = (int64_t)t.threads * t.ipt;
    int32_t n = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        int64_t b0 = offsets[s] + 1, b1 = offsets[s + 1];
        int64_t nb = b1 - b0;
        int64_t chunk = (nb + t.splits - 1) / t.splits;
        chunk = (chunk + align - 1) / align * align;  // j-ranges start on half tiles (one inside a tile takes that tile's far data)
        const int64_t ia = items_i_begin(b0, i_lo), ib = items_i_end(b1, i_hi);
        for (int64_t i0 = ia; i0 < ib; i0 += ti) {
            int64_t i1 = i0 + ti < ib ? i0 + ti : ib;
            for (int32_t sp = 0; sp < t.splits; ++sp) {
                int64_t j0 = b0 + sp * chunk, j1 = j0 + chunk;
                if (j0 > b1) j0 = b1;
                if (j1 > b1) j1 = b1;
                if (n < max_items) {
                    items[n] = make_int4((int)i0, (int)i1, (int)j0, (int)j1);
                    slots[n] = sp;
                }
                ++n;
            }
        }
    }
    *nitems = n;
    *splits_used = t.splits;
}

template <bool FLAG, bool FORCE>
static cudaError_t launch_mixed(const KickArgs &a, int nitems, int threads, int ipt,
                                cudaStream_t st) {
    switch (ipt) {
    case 1: k_kick_mixed<1, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    case 2: k_kick_mixed<2, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    case 4: k_kick_mixed<4, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool FLAG, bool FORCE>
static cudaError_t launch_f64(const KickArgs &a, int nitems, int threads, int ipt,
                              cudaStream_t st) {
    switch (ipt) {
    case 1: k_kick_fp64<1, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    case 2: k_kick_fp64<2, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    default: k_kick_fp64<2, FLAG, FORCE><<<nitems, threads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// Per tile of TILE consecutive positions (from position 1; the bodies in
// Morton order): the bounding box of the hi parts, a reference point c at its
// middle, a radius R >= max |Q_j - c| (rounded up, with room for the lo parts
// and the rounding of c), the largest crude-search reach c_j of its bodies
// (tile[1].w), and each body's offset o_j = Q_j - c, rounded once (two-sum of
// x_hi - c, then x_lo added), beside its G m.
__global__ void __launch_bounds__(TILE) k_tile_prep(int64_t npos, const float4 *pos,
                                                    const float4 *lo, float4 *far, float4 *tile) {
    __shared__ float s_m[TILE / 32][7];
    __shared__ float s_c[3];
    const int64_t p = 1 + (int64_t)blockIdx.x * TILE + threadIdx.x;
    const bool act = p < npos;
    float4 P = make_float4(0.f, 0.f, 0.f, 0.f), L = P;
    if (act) {
        P = pos[p];
        L = lo[p];
    }
    // (m[6]: minus the largest search reach c of the tile's bodies)
    float m[7] = {act ? P.x : 3e38f, act ? P.y : 3e38f, act ? P.z : 3e38f,
                  act ? -P.x : 3e38f, act ? -P.y : 3e38f, act ? -P.z : 3e38f,
                  act ? -L.w : 3e38f};
#pragma unroll
    for (int q = 0; q < 7; ++q) m[q] = warp_min(m[q]);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 7; ++q) s_m[threadIdx.x >> 5][q] = m[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        float b[7];
        for (int q = 0; q < 7; ++q) {
            b[q] = s_m[0][q];
            for (int w = 1; w < TILE / 32; ++w) b[q] = fminf(b[q], s_m[w][q]);
        }
        float hr2 = 0.0f, big = 0.0f, c[3];
        for (int q = 0; q < 3; ++q) {
            const float l = b[q], h = -b[q + 3];
            c[q] = 0.5f * (l + h);
            const float e = fmaxf(__fsub_ru(h, c[q]), __fsub_ru(c[q], l));
            hr2 = __fmaf_ru(e, e, hr2);
            big = fmaxf(big, fmaxf(fabsf(l), fabsf(h)));
            s_c[q] = c[q];
        }
        const float R = __fadd_ru(__fsqrt_ru(hr2), 4.0f * 1.1920929e-7f * big);
        float4 *t = tile + 3 * blockIdx.x;
        t[0] = make_float4(c[0], c[1], c[2], R);
        t[1] = make_float4(b[0], b[1], b[2], fmaxf(-b[6], 0.0f));
        t[2] = make_float4(-b[3], -b[4], -b[5], 0.0f);
    }
    __syncthreads();
    if (act)
        far[p] = make_float4(ds_add(P.x, -s_c[0], L.x), ds_add(P.y, -s_c[1], L.y),
                             ds_add(P.z, -s_c[2], L.z), P.w);
}

cudaError_t launch_kick_tiles(const Dev &d, int prec, int flag, double G, int threads, int ipt,
                              cudaStream_t st) {
    if (d.nitems <= 0) return cudaSuccess;
    KickArgs a;
    a.items = d.items;
    a.slots = d.item_slot;
    a.pos = d.pk_pos;
    a.lo = d.pk_lo;
    a.q = d.q;
    a.m = d.m;
    a.G = G;
    a.apart = d.apart;
    a.rows = d.rows;
    a.cand = d.cand;
    a.max_cand = d.max_cand;
    a.ncand = d.ctr + C_NCAND;
    a.fchunk = d.fchunk;
    a.max_fchunk = d.max_fchunk;
    a.nfchunk = d.ctr + C_NFCHUNK;
    a.status = d.status;
    a.far_tiles = (d.perm && d.far && prec == QYM_KICK_MIXED) ? 1 : 0;
    a.perm = d.perm;
    a.far = d.far;
    a.tile = d.tile;
    a.blk_cnt = d.kick_cnt;
    a.splits = d.splits;
    if (a.far_tiles) {
        const int64_t ntiles = (d.rows - 1 + TILE - 1) / TILE;
        k_tile_prep<<<(unsigned)ntiles, TILE, 0, st>>>(d.rows, d.pk_pos, d.pk_lo, d.far, d.tile);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (flag != KICK_FORCE && flag != KICK_SEARCH && flag != KICK_SEARCH_ONLY)
        return cudaErrorInvalidValue;
    if (prec == QYM_KICK_MIXED) {
        if (flag == KICK_FORCE) return launch_mixed<false, true>(a, d.nitems, threads, ipt, st);
        cudaError_t e = flag == KICK_SEARCH
                            ? launch_mixed<true, true>(a, d.nitems, threads, ipt, st)
                            : launch_mixed<true, false>(a, d.nitems, threads, ipt, st);
        if (e) return e;
        // about one entry per row (its own chunk) plus the close pairs
        int64_t blocks = (d.rows + 63) / 64;
        if (blocks > 4 * 152) blocks = 4 * 152;
        if (blocks < 1) blocks = 1;
        k_flag_chunks<<<(int)blocks, 256, 0, st>>>(a, d.ctr + C_FCDONE);
        return cudaGetLastError();
    }
    if (flag == KICK_FORCE) return launch_f64<false, true>(a, d.nitems, threads, ipt, st);
    return flag == KICK_SEARCH ? launch_f64<true, true>(a, d.nitems, threads, ipt, st)
                               : launch_f64<true, false>(a, d.nitems, threads, ipt, st);
}

// ---------------------------------------------------------------- single system
// Workspace for qym_accel_dev: packs + items + partials for one system.
struct SingleLayout {
    size_t off_pos, off_lo, off_items, off_slots, off_apart, off_heavy, total;
    int32_t nitems, splits;
    KickTune tune;
    bool sorted;   // bodies held in Morton order (mixed kick, >= kSortMinBodies bodies)
    size_t off_perm, off_inv, off_box, off_k0, off_k1, off_v0, off_v1, off_hist, off_far, off_tile;
};

// bodies from which a system's mixed kick holds them in Morton order (sort.cu)
constexpr int64_t kSingleSortMin = 2048;

static SingleLayout single_layout(int64_t rows, int prec) {
    SingleLayout L;
    KickTune t;
    t.threads = 128;
    t.ipt = prec == QYM_KICK_MIXED ? 2 : 1;
    int64_t nb = rows - 1;
    int64_t ib = (nb + t.threads * t.ipt - 1) / (t.threads * t.ipt);
    // enough CTAs to cover the GPU a few times over
    int64_t want = 4 * 152;
    int64_t sp = (want + ib - 1) / ib;
    int64_t maxsp = (nb + 255) / 256;  // at least a tile of j per split
    if (sp > maxsp) sp = maxsp;
    if (sp < 1) sp = 1;
    t.splits = (int32_t)sp;
    L.tune = t;
    L.splits = t.splits;
    L.nitems = (int32_t)(ib * sp);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    L.off_pos = o; o = al(o + sizeof(float4) * rows);
    L.off_lo = o; o = al(o + sizeof(float4) * rows);
    L.off_items = o; o = al(o + sizeof(int4) * L.nitems);
    L.off_slots = o; o = al(o + sizeof(int32_t) * L.nitems);
    L.off_apart = o; o = al(o + sizeof(double) * 3 * rows * L.splits);
    L.off_heavy = o; o = al(o + sizeof(int32_t) * (QYM_HEAVY_CAP + 1));
    L.sorted = prec == QYM_KICK_MIXED && nb >= kSingleSortMin;
    L.off_perm = L.off_inv = L.off_box = L.off_k0 = L.off_k1 = L.off_v0 = L.off_v1 = L.off_hist = 0;
    L.off_far = L.off_tile = 0;
    if (L.sorted) {
        L.off_perm = o; o = al(o + sizeof(int32_t) * rows);
        L.off_inv = o; o = al(o + sizeof(int32_t) * rows);
        L.off_box = o; o = al(o + sizeof(int) * 8);
        L.off_k0 = o; o = al(o + sizeof(uint32_t) * rows);
        L.off_k1 = o; o = al(o + sizeof(uint32_t) * rows);
        L.off_v0 = o; o = al(o + sizeof(int32_t) * rows);
        L.off_v1 = o; o = al(o + sizeof(int32_t) * rows);
        L.off_hist = o; o = al(o + sizeof(uint32_t) * 256 * (size_t)sort_blocks(rows));
        L.off_far = o; o = al(o + sizeof(float4) * rows);
        L.off_tile = o; o = al(o + sizeof(float4) * 3 * (size_t)((rows - 1 + TILE - 1) / TILE));
    }
    L.total = o;
    return L;
}

size_t accel_single_workspace(int64_t rows, int prec) {
    if (rows < 2) return 0;
    return single_layout(rows, prec).total;
}

// heavy list of one system: the first QYM_HEAVY_CAP bodies (ascending rows)
// with m >= heavy_mass * m[0]; hl[QYM_HEAVY_CAP] receives their count, and the
// bodies past the cap stay in the FP32 tiles
__global__ void __launch_bounds__(1024) k_heavy_thr_single(int64_t rows, const double *m,
                                                           double heavy_mass, int32_t *hl) {
    // same compaction as k_heavy_single with the threshold taken from m[0]
    __shared__ int base;
    __shared__ int wsum[32];
    const double thr = heavy_mass * m[0];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t r0 = 1; r0 < rows; r0 += blockDim.x) {
        int64_t r = r0 + threadIdx.x;
        int hv = (r < rows && m[r] >= thr) ? 1 : 0;
        unsigned b = __ballot_sync(0xffffffffu, hv);
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int k = 0; k < w; ++k) before += wsum[k];
        int pos = base + before + __popc(b & ((1u << lane) - 1u));
        if (hv && pos < QYM_HEAVY_CAP) hl[pos] = (int32_t)r;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
            base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) hl[QYM_HEAVY_CAP] = base < QYM_HEAVY_CAP ? base : QYM_HEAVY_CAP;
}

__global__ void k_pack_single(int64_t rows, const double *m, const double *q, double G,
                              const int32_t *hl, float4 *pos, float4 *lo, const int32_t *inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int64_t pi = inv ? inv[i] : i;  // the kick's order
    float xh, xl, yh, yl, zh, zl;
    split_ds(q[i], xh, xl);
    split_ds(q[rows + i], yh, yl);
    split_ds(q[2 * rows + i], zh, zl);
    float gm = (float)(G * m[i]);
    if (hl) {
        int nh = hl[QYM_HEAVY_CAP];
        for (int k = 0; k < nh; ++k)
            if (hl[k] == (int32_t)i) gm = 0.0f;
    }
    pos[pi] = make_float4(xh, yh, zh, gm);
    lo[pi] = make_float4(xl, yl, zl, 0.0f);
}

__global__ void k_items_single(int64_t rows, int32_t ti, int32_t splits, int4 *items,
                               int32_t *slots, int32_t nitems, int32_t align) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nitems) return;
    int64_t b0 = 1, b1 = rows, nb = rows - 1;
    int64_t chunk = (nb + splits - 1) / splits;
    chunk = (chunk + align - 1) / align * align;  // j-ranges start on tiles
    int ib = idx / splits, sp = idx % splits;
    int64_t i0 = b0 + (int64_t)ib * ti, i1 = i0 + ti < b1 ? i0 + ti : b1;
    int64_t j0 = b0 + sp * chunk, j1 = j0 + chunk;
    if (j0 > b1) j0 = b1;
    if (j1 > b1) j1 = b1;
    items[idx] = make_int4((int)i0, (int)i1, (int)j0, (int)j1);
    slots[idx] = sp;
}

__global__ void k_sum_partials(int64_t rows, int32_t splits, const double *apart,
                               const int32_t *hl, const double *m, const double *q, double G,
                               double *a, const int32_t *inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    double s[3] = {0.0, 0.0, 0.0};
    if (i > 0) {
        const int64_t pi = inv ? inv[i] : i;  // the kick's order
        for (int c = 0; c < 3; ++c)
            for (int sp = 0; sp < splits; ++sp) s[c] += apart[((int64_t)sp * 3 + c) * rows + pi];
        if (hl)
            heavy_pull(hl, hl[QYM_HEAVY_CAP], i, q[i], q[rows + i], q[2 * rows + i], q, m, rows, G,
                       s[0], s[1], s[2]);
    }
    for (int c = 0; c < 3; ++c) a[c * rows + i] = s[c];
}

cudaError_t launch_accel_single(int64_t rows, const double *m, const double *q, double *a,
                                double G, int prec, double heavy_mass, void *work,
                                size_t work_bytes, cudaStream_t st) {
    SingleLayout L = single_layout(rows, prec);
    if (work_bytes < L.total) return cudaErrorInvalidValue;
    char *w = (char *)work;
    Dev d;
    d.rows = rows;
    d.m = m ? const_cast<double *>(m) : nullptr;
    d.q = const_cast<double *>(q);
    d.pk_pos = (float4 *)(w + L.off_pos);
    d.pk_lo = (float4 *)(w + L.off_lo);
    d.items = (int4 *)(w + L.off_items);
    d.item_slot = (int32_t *)(w + L.off_slots);
    d.apart = (double *)(w + L.off_apart);
    d.nitems = L.nitems;
    d.splits = L.splits;
    int tb = 256;
    // heavy split (mixed kick only): threshold relative to the star mass m[0],
    // read on the device
    int32_t *hl = nullptr;
    if (prec == QYM_KICK_MIXED && heavy_mass > 0.0) {
        hl = (int32_t *)(w + L.off_heavy);
        k_heavy_thr_single<<<1, 1024, 0, st>>>(rows, m, heavy_mass, hl);
    }
    if (L.sorted) {
        // the bodies in Morton order, as the step's kick holds them
        d.perm = (int32_t *)(w + L.off_perm);
        d.inv = (int32_t *)(w + L.off_inv);
        d.far = (float4 *)(w + L.off_far);
        d.tile = (float4 *)(w + L.off_tile);
        SortScratch ss;
        ss.box = (int *)(w + L.off_box);
        ss.k0 = (uint32_t *)(w + L.off_k0);
        ss.k1 = (uint32_t *)(w + L.off_k1);
        ss.v0 = (int32_t *)(w + L.off_v0);
        ss.v1 = (int32_t *)(w + L.off_v1);
        ss.hist = (uint32_t *)(w + L.off_hist);
        cudaError_t e = launch_sort_rows(rows, q, ss, d.perm, d.inv, st);
        if (e != cudaSuccess) return e;
    }
    k_pack_single<<<(unsigned)((rows + tb - 1) / tb), tb, 0, st>>>(rows, m, q, G, hl, d.pk_pos,
                                                                    d.pk_lo, d.inv);
    k_items_single<<<(L.nitems + tb - 1) / tb, tb, 0, st>>>(rows, L.tune.threads * L.tune.ipt,
                                                             L.splits, d.items, d.item_slot,
                                                             L.nitems, L.sorted ? TILE : 1);
    cudaError_t e;
    if (prec == QYM_KICK_MIXED) {
        e = launch_kick_tiles(d, prec, 0, G, L.tune.threads, L.tune.ipt, st);
    } else {
        KickArgs ka;
        ka.items = d.items; ka.slots = d.item_slot; ka.pos = d.pk_pos; ka.lo = d.pk_lo;
        ka.q = q; ka.m = m; ka.G = G; ka.apart = d.apart; ka.rows = rows;
        ka.cand = nullptr; ka.max_cand = 0; ka.ncand = nullptr; ka.status = nullptr;
        ka.fchunk = nullptr; ka.max_fchunk = 0; ka.nfchunk = nullptr; ka.far_tiles = 0;
        ka.perm = nullptr; ka.far = nullptr; ka.tile = nullptr;
        e = launch_f64<false, true>(ka, L.nitems, L.tune.threads, L.tune.ipt, st);
    }
    if (e != cudaSuccess) return e;
    k_sum_partials<<<(unsigned)((rows + tb - 1) / tb), tb, 0, st>>>(rows, L.splits, d.apart, hl, m,
                                                                     q, G, a, d.inv);
    return cudaGetLastError();
}

}  // namespace qym
