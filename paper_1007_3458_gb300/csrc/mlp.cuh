// mlp.cuh -- the learned starting guess of the universal Kepler equation
// (Appendix): a 4 -> 64 -> 64 -> 1 perceptron with GELU (tanh form) on
// dimensionless features of a body's state and step. BF16 weights, FP32
// accumulation; the 64 x 64 layer runs on the tensor cores with
// mma.sync m16n8k16 (bf16 in, f32 out), the 4-wide input layer and the
// 1-wide output layer on the FP32 pipes.
//
// Weights are one float32 vector (the master copy that training updates):
// W1[64][4] b1[64] W2[64][64] b2[64] W3[64] b3 mean[4] std[4] om osd. The
// matrices are rounded to bf16 (nearest, ties to even) as they are loaded.
//
// Fragment layouts (PTX ISA, mma.m16n8k16 with .bf16): lane = 4 g + t;
// A (16 x 16, row major): a0 = (row g, cols 2t, 2t+1), a1 = (row g+8, same
// cols), a2 = (row g, cols 2t+8, 2t+9), a3 = (row g+8, cols 2t+8, 2t+9);
// B (16 x 8): b0 = (rows 2t, 2t+1, col g), b1 = (rows 2t+8, 2t+9, col g);
// C (16 x 8, f32): c0, c1 = (row g, cols 2t, 2t+1), c2, c3 = (row g+8, ...).
// Two C tiles side by side hold exactly one A fragment of the next product,
// so a layer's output feeds the next layer from registers.
#pragma once
#include <cuda_bf16.h>

#include "qym_internal.cuh"

namespace qym {
namespace mlp {

constexpr int H = 64;
constexpr int NW = 4555;
constexpr int W1 = 0, B1 = 256, W2 = 320, B2 = 4416, W3 = 4480, B3 = 4544;
constexpr int MEAN = 4545, STD = 4549, OM = 4553, OSD = 4554;
constexpr int NFROZEN = 10;  // normalisation entries, not trained

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// two floats -> one bf16x2 register, `lo` in the low half
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float lo_of(uint32_t r) { return __uint_as_float(r << 16); }
__device__ __forceinline__ float hi_of(uint32_t r) { return __uint_as_float(r & 0xffff0000u); }

// GELU, tanh form: x/2 (1 + tanh c), c = sqrt(2/pi) (x + 0.044715 x^3),
// evaluated as x / (1 + e^(-2c)); dh receives its derivative
// s + x s (1 - s) 2 c' with s = 1 / (1 + e^(-2c)). c is clamped below at -40
// so that e^(-2c) stays finite (the value there is below 1e-33 x).
__device__ __forceinline__ float gelu(float x, float &dh) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float x2 = x * x;
    const float c = fmaxf(k0 * fmaf(k1 * x2, x, x), -40.0f);
    const float e = __expf(-2.0f * c);
    const float s = __frcp_rn(1.0f + e);
    dh = fmaf(x * s * (1.0f - s) * 2.0f * k0, fmaf(3.0f * k1, x2, 1.0f), s);
    return x * s;
}
__device__ __forceinline__ float gelu(float x) {
    float d;
    return gelu(x, d);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// normalised features fn = (u - mean) / std
__device__ __forceinline__ void normalise(const float *__restrict__ w, const float (&u)[4],
                                          float (&fn)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) fn[i] = (u[i] - w[MEAN + i]) / w[STD + i];
}

// B fragments of layer 2 (B[k][n] = W2[n][k]: a lane's registers are
// consecutive pairs along a row of W2), from the float32 master weights...
struct W2FromGlobal {
    const float *w;
    __device__ __forceinline__ void operator()(int ks, int nt, int g, int t, uint32_t &b0,
                                               uint32_t &b1) const {
        const float *row = w + W2 + 64 * (8 * nt + g) + 16 * ks + 2 * t;
        const float2 lo = *reinterpret_cast<const float2 *>(row);
        const float2 hi = *reinterpret_cast<const float2 *>(row + 8);
        b0 = pack2(lo.x, lo.y);
        b1 = pack2(hi.x, hi.y);
    }
};
// ... or from a bf16 copy in shared memory, rows of `ld` bf16 (ld even):
// s[n * ld + k] = bf16(W2[n][k]) (or any other matrix stored that way).
struct BFromShared {
    const uint32_t *s;
    int ld;
    __device__ __forceinline__ void operator()(int ks, int nt, int g, int t, uint32_t &b0,
                                               uint32_t &b1) const {
        const int base = (8 * nt + g) * ld + 16 * ks + 2 * t;
        b0 = s[base >> 1];
        b1 = s[(base + 8) >> 1];
    }
};

// Layers 1 and 2 of one 16-row tile of a warp. fa, fb: normalised features of
// rows g and g+8. Out: A = bf16(h1) as the A fragments of the four k-steps of
// layer 2, acc = p2 = W2 h1 + b2 in C layout (n-tile nt: cols 8 nt + 2t, +1),
// and with KEEP_D1 d1 = gelu'(p1) in C layout.
template <bool KEEP_D1, class BLoad>
__device__ __forceinline__ void layers12(const float *__restrict__ w, const BLoad &bload,
                                         const float (&fa)[4], const float (&fb)[4], int g, int t,
                                         uint32_t (&A)[4][4], float (&acc)[8][4],
                                         float (&d1)[8][4]) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float h[4];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * nt + 2 * t + e;
            const float4 wr = *reinterpret_cast<const float4 *>(w + W1 + 4 * c);
            const float w0 = bf(wr.x), w1 = bf(wr.y), w2 = bf(wr.z), w3 = bf(wr.w);
            const float bb = w[B1 + c];
            const float pa = fmaf(w3, fa[3], fmaf(w2, fa[2], fmaf(w1, fa[1], fmaf(w0, fa[0], bb))));
            const float pb = fmaf(w3, fb[3], fmaf(w2, fb[2], fmaf(w1, fb[1], fmaf(w0, fb[0], bb))));
            float da, db;
            h[e] = gelu(pa, da);
            h[2 + e] = gelu(pb, db);
            if (KEEP_D1) {
                d1[nt][e] = da;
                d1[nt][2 + e] = db;
            }
        }
        const int ks = nt >> 1, half = nt & 1;
        A[ks][2 * half] = pack2(h[0], h[1]);       // row g
        A[ks][2 * half + 1] = pack2(h[2], h[3]);   // row g+8
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 bb = *reinterpret_cast<const float2 *>(w + B2 + 8 * nt + 2 * t);
        acc[nt][0] = bb.x;
        acc[nt][1] = bb.y;
        acc[nt][2] = bb.x;
        acc[nt][3] = bb.y;
    }
    // p2[s][n] = sum_k h1[s][k] W2[n][k]
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b0, b1;
            bload(ks, nt, g, t, b0, b1);
            mma_bf16(acc[nt], A[ks], b0, b1);
        }
    }
}

// Output layer of a tile: y for rows g and g+8 (summed over the quad, so
// every lane of quad g holds both).
__device__ __forceinline__ void output(const float *__restrict__ w, const float (&acc)[8][4], int t,
                                       float &ya, float &yb) {
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 w3 = *reinterpret_cast<const float2 *>(w + W3 + 8 * nt + 2 * t);
        const float w30 = bf(w3.x), w31 = bf(w3.y);
        sa = fmaf(w30, gelu(acc[nt][0]), sa);
        sa = fmaf(w31, gelu(acc[nt][1]), sa);
        sb = fmaf(w30, gelu(acc[nt][2]), sb);
        sb = fmaf(w31, gelu(acc[nt][3]), sb);
    }
    sa += __shfl_xor_sync(0xffffffffu, sa, 1);
    sb += __shfl_xor_sync(0xffffffffu, sb, 1);
    sa += __shfl_xor_sync(0xffffffffu, sa, 2);
    sb += __shfl_xor_sync(0xffffffffu, sb, 2);
    ya = sa + w[B3];
    yb = sb + w[B3];
}

// Network output y for the 32 samples of a warp, one per lane (fn: the
// lane's normalised features). Every lane of the warp must call it.
__device__ __forceinline__ float warp_forward(const float *__restrict__ w, const float (&fn)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float mine = 0.0f;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        float fa[4], fb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            fa[i] = __shfl_sync(0xffffffffu, fn[i], 16 * mt + g);
            fb[i] = __shfl_sync(0xffffffffu, fn[i], 16 * mt + g + 8);
        }
        uint32_t A[4][4];
        float acc[8][4], d1[8][4];
        layers12<false>(w, W2FromGlobal{w}, fa, fb, g, t, A, acc, d1);
        float ya, yb;
        output(w, acc, t, ya, yb);
        // lane l owns row l & 15 of tile l >> 4, held by lane 4 (row & 7)
        const int r = lane & 15;
        const float va = __shfl_sync(0xffffffffu, ya, 4 * (r & 7));
        const float vb = __shfl_sync(0xffffffffu, yb, 4 * (r & 7));
        if ((lane >> 4) == mt) mine = r < 8 ? va : vb;
    }
    return mine;
}

// Raw features u1..u4 of a body (q, v) about a star of parameter mu for a
// step dt (r0 = |q| > 0, dt != 0), and sigma = s / (1 + s) with
// s = |dt| sqrt(mu / r0^3):
//   u1 = q.v / sqrt(mu r0), u2 = r0 |v|^2 / mu, u3 = ln s,
//   u4 = dt sqrt(mu alpha^3) / (2 pi) for alpha = 2/r0 - |v|^2/mu > 0, else 0.
// Returns whether the orbit is bound (alpha > 0): the domain of the learned
// guess (there |u1| < sqrt 2 and u2 < 2; unbound states, such as bodies deep
// in a planet's well during an encounter, keep the standard guess).
__device__ __forceinline__ bool features(double qx, double qy, double qz, double vx, double vy,
                                         double vz, double r0, double mu, double dt,
                                         float (&u)[4], double &sigma) {
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double rv = qx * vx + qy * vy + qz * vz;
    const double alpha = 2.0 / r0 - v2 / mu;
    const double s = fabs(dt) * sqrt(mu / (r0 * r0 * r0));
    u[0] = (float)(rv / sqrt(mu * r0));
    u[1] = (float)(r0 * v2 / mu);
    u[2] = (float)log(s);
    u[3] = alpha > 0.0 ? (float)(dt * sqrt(mu * alpha * alpha * alpha) / (2.0 * kPi)) : 0.0f;
    sigma = s / (1.0 + s);
    return alpha > 0.0;
}

}  // namespace mlp
}  // namespace qym
