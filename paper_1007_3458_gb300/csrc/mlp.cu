// mlp.cu -- inference and training kernels of the learned Kepler starting
// guess (network and layouts in mlp.cuh).
//
// Training minimises the mean squared error of the network output y against
// yt = (t - om) / osd over rows (u1, u2, u3, u4, t) with Adam. One step is two
// launches:
//   k_mlp_grad    forward and backward of a minibatch; each CTA takes rounds
//                 of 64 rows (16 per warp), keeps the 64 x 64 weight gradient
//                 of its rows in tensor-core accumulators and writes one
//                 partial gradient vector;
//   k_mlp_reduce  sums the partials in a fixed order (deterministic) and
//                 applies the Adam update to the float32 master weights.
// The operands the tensor cores take are bf16: h1 and W2 in the forward
// product, dp2 = dL/dp2 with W2 (for dL/dh1) and with h1 (for dL/dW2) in the
// backward ones. The other sums (dL/dW1, the biases, dL/dW3) stay in FP32.
#include <cmath>

#include "mlp.cuh"

namespace qym {
using namespace mlp;

namespace {
constexpr int GT = 128;   // threads of a gradient CTA (4 warps)
constexpr int GR = 64;    // rows per round
constexpr int LDT = 72;   // bf16 row stride of the transposed tiles (conflict-free)
constexpr int LDF = 65;   // float row stride
constexpr int MAXBLK = 256;
constexpr size_t kGradSmem = 4 * 64 * LDT * sizeof(__nv_bfloat16) + 3 * 64 * LDF * sizeof(float) +
                             64 * 4 * sizeof(float) + 64 * sizeof(float);
}  // namespace

__global__ void __launch_bounds__(256) k_mlp_forward(int64_t n, const float *__restrict__ w,
                                                     const float *__restrict__ u,
                                                     float *__restrict__ y) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float uu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (k < n) {
        const float4 r = *reinterpret_cast<const float4 *>(u + 4 * k);
        uu[0] = r.x; uu[1] = r.y; uu[2] = r.z; uu[3] = r.w;
    }
    float fn[4];
    normalise(w, uu, fn);
    const float out = warp_forward(w, fn);
    if (k < n) y[k] = out;
}

__global__ void __launch_bounds__(GT) k_mlp_grad(const float *__restrict__ w,
                                                 const float *__restrict__ rows, int64_t n,
                                                 float inv_n, float *__restrict__ part,
                                                 float *__restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *h1T = reinterpret_cast<__nv_bfloat16 *>(sm);   // [64 k][LDT]: h1 of row s at col s
    __nv_bfloat16 *dp2T = h1T + 64 * LDT;                          // [64 j][LDT]
    float *dp1s = reinterpret_cast<float *>(dp2T + 64 * LDT);      // [64 s][LDF]
    float *dp2s = dp1s + 64 * LDF;                                 // [64 s][LDF]
    float *h2s = dp2s + 64 * LDF;                                  // [64 s][LDF]
    float *fns = h2s + 64 * LDF;                                   // [64 s][4]
    float *dys = fns + 64 * 4;                                     // [64 s]
    __nv_bfloat16 *w2n = reinterpret_cast<__nv_bfloat16 *>(dys + 64);  // [64 n][LDT] bf16 W2[n][k]
    __nv_bfloat16 *w2k = w2n + 64 * LDT;                                // [64 k][LDT] bf16 W2[j][k] at (k, j)
    __shared__ float red[2][GT / 32];
    {
        unsigned short *a = reinterpret_cast<unsigned short *>(w2n);
        unsigned short *b = reinterpret_cast<unsigned short *>(w2k);
        for (int i = threadIdx.x; i < 64 * 64; i += GT) {
            const int r = i >> 6, c = i & 63;
            const __nv_bfloat16 x = __float2bfloat16_rn(w[W2 + i]);
            const unsigned short xb = *reinterpret_cast<const unsigned short *>(&x);
            a[r * LDT + c] = xb;
            b[c * LDT + r] = xb;
        }
        __syncthreads();
    }
    const BFromShared bW2{reinterpret_cast<const uint32_t *>(w2n), LDT};
    const BFromShared bW2T{reinterpret_cast<const uint32_t *>(w2k), LDT};

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const float om = w[OM], osd = w[OSD];

    float gw2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) gw2[nt][e] = 0.0f;
    float cs[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // column sums of phase 2
    float gb3 = 0.0f, lsum = 0.0f;

    const int64_t nround = (n + GR - 1) / GR;
    for (int64_t rd = blockIdx.x; rd < nround; rd += gridDim.x) {
        const int ra = 16 * warp + g, rb = ra + 8;         // rows of this lane within the round
        const int64_t sa = rd * GR + ra, sb = rd * GR + rb;
        const bool va = sa < n, vb = sb < n;
        float ua[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ub[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        float ta = 0.0f, tb = 0.0f;
        if (va) {
#pragma unroll
            for (int i = 0; i < 4; ++i) ua[i] = rows[5 * sa + i];
            ta = rows[5 * sa + 4];
        }
        if (vb) {
#pragma unroll
            for (int i = 0; i < 4; ++i) ub[i] = rows[5 * sb + i];
            tb = rows[5 * sb + 4];
        }
        float fa[4], fb[4];
        normalise(w, ua, fa);
        normalise(w, ub, fb);
        if (t == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fns[4 * ra + i] = fa[i];
                fns[4 * rb + i] = fb[i];
            }
        }
        uint32_t A[4][4];
        float acc[8][4], d1[8][4];
        layers12<true>(w, bW2, fa, fb, g, t, A, acc, d1);
        // gelu'(p1) waits in dp1s until dL/dh1 is known (same slots, same thread)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = 8 * nt + 2 * t + e;
                dp1s[ra * LDF + c] = d1[nt][e];
                dp1s[rb * LDF + c] = d1[nt][2 + e];
            }
        }
        // bf16 h1, transposed, for the layer-2 weight gradient
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int k = 8 * nt + 2 * t, ks = nt >> 1, half = nt & 1;
            const uint32_t ra2 = A[ks][2 * half], rb2 = A[ks][2 * half + 1];
            const unsigned short *pa = reinterpret_cast<const unsigned short *>(&ra2);
            const unsigned short *pb = reinterpret_cast<const unsigned short *>(&rb2);
            unsigned short *dst = reinterpret_cast<unsigned short *>(h1T);
            dst[k * LDT + ra] = pa[0];
            dst[(k + 1) * LDT + ra] = pa[1];
            dst[k * LDT + rb] = pb[0];
            dst[(k + 1) * LDT + rb] = pb[1];
        }
        // output layer: h2 to shared memory, acc <- gelu'(p2)
        float sya = 0.0f, syb = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = 8 * nt + 2 * t + e;
                const float w3 = bf(w[W3 + c]);
                float da, db;
                const float ha = gelu(acc[nt][e], da), hb = gelu(acc[nt][2 + e], db);
                h2s[ra * LDF + c] = ha;
                h2s[rb * LDF + c] = hb;
                sya = fmaf(w3, ha, sya);
                syb = fmaf(w3, hb, syb);
                acc[nt][e] = da;
                acc[nt][2 + e] = db;
            }
        }
        sya += __shfl_xor_sync(0xffffffffu, sya, 1);
        syb += __shfl_xor_sync(0xffffffffu, syb, 1);
        sya += __shfl_xor_sync(0xffffffffu, sya, 2);
        syb += __shfl_xor_sync(0xffffffffu, syb, 2);
        const float b3 = w[B3];
        const float rra = va ? (sya + b3) - (ta - om) / osd : 0.0f;
        const float rrb = vb ? (syb + b3) - (tb - om) / osd : 0.0f;
        const float dya = 2.0f * rra * inv_n, dyb = 2.0f * rrb * inv_n;
        if (t == 0) {
            dys[ra] = dya;
            dys[rb] = dyb;
            lsum = fmaf(rra, rra, fmaf(rrb, rrb, lsum));
            gb3 += dya + dyb;
        }
        // dp2 = dy W3 gelu'(p2): FP32 copy for the bias gradient, bf16
        // (transposed) for the weight gradient, bf16 A fragments for dL/dh1
        uint32_t dA[4][4];
        unsigned short *dT = reinterpret_cast<unsigned short *>(dp2T);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float p[4];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = 8 * nt + 2 * t + e;
                const float w3 = bf(w[W3 + c]);
                p[e] = dya * w3 * acc[nt][e];
                p[2 + e] = dyb * w3 * acc[nt][2 + e];
                dp2s[ra * LDF + c] = p[e];
                dp2s[rb * LDF + c] = p[2 + e];
            }
            const int ks = nt >> 1, half = nt & 1;
            const uint32_t xa = pack2(p[0], p[1]), xb = pack2(p[2], p[3]);
            dA[ks][2 * half] = xa;
            dA[ks][2 * half + 1] = xb;
            const int c = 8 * nt + 2 * t;
            dT[c * LDT + ra] = (unsigned short)(xa & 0xffffu);
            dT[(c + 1) * LDT + ra] = (unsigned short)(xa >> 16);
            dT[c * LDT + rb] = (unsigned short)(xb & 0xffffu);
            dT[(c + 1) * LDT + rb] = (unsigned short)(xb >> 16);
        }
        // dh1[s][k] = sum_j dp2[s][j] W2[j][k]: B[j][k] = W2[j][k], pairs along
        // j, i.e. along the rows of the transposed copy
        float dh[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) dh[nt][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b0, b1;
                bW2T(ks, nt, g, t, b0, b1);
                mma_bf16(dh[nt], dA[ks], b0, b1);
            }
        }
        // dp1 = dh1 gelu'(p1)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = 8 * nt + 2 * t + e;
                dp1s[ra * LDF + c] *= dh[nt][e];
                dp1s[rb * LDF + c] *= dh[nt][2 + e];
            }
        }
        __syncthreads();
        // dL/dW2[j][k] = sum_s dp2[s][j] h1[s][k]; this warp's rows j = 16 warp + ...
        {
            const uint32_t *dT32 = reinterpret_cast<const uint32_t *>(dp2T);
            const uint32_t *hT32 = reinterpret_cast<const uint32_t *>(h1T);
            const int j0 = 16 * warp + g;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t a[4];
                a[0] = dT32[(j0 * LDT + 16 * ks + 2 * t) >> 1];
                a[1] = dT32[((j0 + 8) * LDT + 16 * ks + 2 * t) >> 1];
                a[2] = dT32[(j0 * LDT + 16 * ks + 2 * t + 8) >> 1];
                a[3] = dT32[((j0 + 8) * LDT + 16 * ks + 2 * t + 8) >> 1];
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int kk = 8 * nt + g;
                    const uint32_t b0 = hT32[(kk * LDT + 16 * ks + 2 * t) >> 1];
                    const uint32_t b1 = hT32[(kk * LDT + 16 * ks + 2 * t + 8) >> 1];
                    mma_bf16(gw2[nt], a, b0, b1);
                }
            }
        }
        // column sums over the round's rows: threads 0-63 take dL/dW1 and
        // dL/db1 of unit j, threads 64-127 dL/db2 and dL/dW3 of unit j
        if (tid < 64) {
            const int j = tid;
            for (int s = 0; s < GR; ++s) {
                const float d = dp1s[s * LDF + j];
                cs[0] += d;
#pragma unroll
                for (int i = 0; i < 4; ++i) cs[1 + i] = fmaf(d, fns[4 * s + i], cs[1 + i]);
            }
        } else {
            const int j = tid - 64;
            for (int s = 0; s < GR; ++s) {
                cs[0] += dp2s[s * LDF + j];
                cs[1] = fmaf(h2s[s * LDF + j], dys[s], cs[1]);
            }
        }
        __syncthreads();
    }
    // one partial gradient per CTA
    float *P = part + (size_t)blockIdx.x * NW;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = 16 * warp + g, k = 8 * nt + 2 * t;
        P[W2 + 64 * j + k] = gw2[nt][0];
        P[W2 + 64 * j + k + 1] = gw2[nt][1];
        P[W2 + 64 * (j + 8) + k] = gw2[nt][2];
        P[W2 + 64 * (j + 8) + k + 1] = gw2[nt][3];
    }
    if (tid < 64) {
        P[B1 + tid] = cs[0];
#pragma unroll
        for (int i = 0; i < 4; ++i) P[W1 + 4 * tid + i] = cs[1 + i];
    } else {
        P[B2 + tid - 64] = cs[0];
        P[W3 + tid - 64] = cs[1];
    }
    // b3 and the loss: lanes with t == 0 hold them
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if (lane == 0) {
        red[0][warp] = gb3;
        red[1][warp] = lsum;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.0f, b = 0.0f;
        for (int i = 0; i < GT / 32; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        P[B3] = a;
        lpart[blockIdx.x] = b;
    }
    if (tid < NFROZEN) P[NW - NFROZEN + tid] = 0.0f;
}

// Sum of nblk partial gradients (fixed order), optional copy to grad, and
// with adam != 0 the Adam update of w, m, v (normalisation entries kept).
// Block 0 also reduces the loss partials into *loss (mean over inv_n).
__global__ void __launch_bounds__(256) k_mlp_reduce(const float *__restrict__ part, int nblk,
                                                    const float *__restrict__ lpart, float inv_n,
                                                    float *__restrict__ grad, float *__restrict__ loss,
                                                    float *__restrict__ w, float *__restrict__ m,
                                                    float *__restrict__ v, int adam, float lr,
                                                    float beta1, float beta2, float eps, float bc1,
                                                    float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NW) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * NW + i];
        const float gi = (float)s;
        if (grad) grad[i] = gi;
        if (adam && i < NW - NFROZEN) {
            const float mm = fmaf(beta1, m[i], (1.0f - beta1) * gi);
            const float vv = fmaf(beta2, v[i], (1.0f - beta2) * gi * gi);
            m[i] = mm;
            v[i] = vv;
            w[i] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
        }
    }
    if (loss && lpart && blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += lpart[b];
        *loss = (float)(s * inv_n);
    }
}

// ------------------------------------------------------------------ host side
size_t mlp_workspace_bytes() { return (size_t)MAXBLK * NW * sizeof(float) + MAXBLK * sizeof(float); }

cudaError_t launch_mlp_forward(int64_t n, const float *w, const float *u, float *y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_mlp_forward<<<(unsigned)blocks, 256, 0, st>>>(n, w, u, y);
    return cudaGetLastError();
}

static cudaError_t grad_partials(int64_t n, const float *w, const float *rows, void *work, int &nblk,
                                 cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGradSmem);
    if (e != cudaSuccess) return e;
    const int64_t rounds = (n + GR - 1) / GR;
    nblk = (int)(rounds < MAXBLK ? rounds : MAXBLK);
    float *part = static_cast<float *>(work);
    float *lpart = part + (size_t)MAXBLK * NW;
    k_mlp_grad<<<nblk, GT, kGradSmem, st>>>(w, rows, n, 1.0f / (float)n, part, lpart);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(int64_t n, const float *w, const float *rows, float *grad, float *loss,
                            void *work, cudaStream_t st) {
    int nblk = 0;
    cudaError_t e = grad_partials(n, w, rows, work, nblk, st);
    if (e != cudaSuccess) return e;
    float *part = static_cast<float *>(work);
    float *lpart = part + (size_t)MAXBLK * NW;
    k_mlp_reduce<<<(NW + 255) / 256, 256, 0, st>>>(part, nblk, lpart, 1.0f / (float)n, grad, loss,
                                                   nullptr, nullptr, nullptr, 0, 0.f, 0.f, 0.f, 0.f,
                                                   1.f, 1.f);
    return cudaGetLastError();
}

static void bias_corr(int64_t t, float beta1, float beta2, float &bc1, float &bc2) {
    bc1 = (float)(1.0 - std::pow((double)beta1, (double)t));
    bc2 = (float)(1.0 - std::pow((double)beta2, (double)t));
}

cudaError_t launch_mlp_adam(float *w, float *m, float *v, const float *grad, int64_t t, float lr,
                            float beta1, float beta2, float eps, cudaStream_t st) {
    float bc1, bc2;
    bias_corr(t, beta1, beta2, bc1, bc2);
    k_mlp_reduce<<<(NW + 255) / 256, 256, 0, st>>>(grad, 1, nullptr, 0.f, nullptr, nullptr, w, m, v,
                                                   1, lr, beta1, beta2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(float *w, float *m, float *v, int64_t t0, const float *rows, int64_t n,
                             int64_t batch, int32_t epochs, float lr, float lr_final, float *losses,
                             void *work, cudaStream_t st) {
    const int64_t nb = (n + batch - 1) / batch;
    const int64_t S = nb * (int64_t)epochs;
    float *part = static_cast<float *>(work);
    float *lpart = part + (size_t)MAXBLK * NW;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    for (int64_t s = 0; s < S; ++s) {
        const int64_t b = s % nb, off = b * batch;
        const int64_t len = (n - off) < batch ? (n - off) : batch;
        int nblk = 0;
        cudaError_t e = grad_partials(len, w, rows + 5 * off, work, nblk, st);
        if (e != cudaSuccess) return e;
        // cosine schedule from lr (s = 0) towards lr_final
        const double lrs = (double)lr_final +
                           0.5 * ((double)lr - (double)lr_final) * (1.0 + std::cos(kPi * (double)s / (double)S));
        float bc1, bc2;
        bias_corr(t0 + s + 1, beta1, beta2, bc1, bc2);
        k_mlp_reduce<<<(NW + 255) / 256, 256, 0, st>>>(part, nblk, lpart, 1.0f / (float)len, nullptr,
                                                       losses ? losses + s : nullptr, w, m, v, 1,
                                                       (float)lrs, beta1, beta2, eps, bc1, bc2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qym
