// The LoD ranking MLP: 48 -> 64 -> 64 -> 1 with ReLU, BF16 tensor-core
// matrix products (mma m16n8k16, FP32 accumulate), FP32 master weights and
// Adam.  One fused kernel runs the forward pass (and, when training, the
// backward pass with per-CTA weight-gradient partials); a second kernel
// reduces the partials in a fixed order and applies Adam.
//
// Warp-level fragments of mma.m16n8k16 (bf16 in, f32 accumulate), lane =
// 4 * g + q (g = lane / 4, q = lane % 4):
//   A 16x16 row-major, 4 registers of two bf16 each (low half = lower column):
//     a0 = A[g][2q, 2q+1]  a1 = A[g+8][2q, 2q+1]  a2 = A[g][2q+8, 2q+9]  a3 = A[g+8][2q+8, 2q+9]
//   B 16x8, two registers:  b0 = B[2q, 2q+1][g]  b1 = B[2q+8, 2q+9][g]
//   C 16x8 f32:  c0, c1 = C[g][2q, 2q+1]   c2, c3 = C[g+8][2q, 2q+1]
// Two neighbouring C tiles of a 16-row block therefore hold exactly the A
// fragment of the next layer's 16-wide k step, so activations stay in
// registers between layers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/crowdsplat.h"
#include "../../include/crowdsplat_lod.h"

namespace {

constexpr int kIn = CS_MLP_IN;      // 48
constexpr int kH = CS_MLP_HIDDEN;   // 64
constexpr int kFeat = CS_LOD_FEATURES;
constexpr int kP = CS_MLP_PARAMS;   // 7361
constexpr int oW1 = 0, oB1 = oW1 + kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
static_assert(oB3 + 1 == kP, "parameter layout");

constexpr int kWarps = 8, kThreads = 32 * kWarps, kTile = 16 * kWarps;  // 128 rows per CTA tile
// shared-memory leading dimensions (bf16 elements), padded so that the 32
// lanes of a fragment load hit 32 different banks
constexpr int kLdW1 = 56;   // W1^T  [64 hidden][48 in]
constexpr int kLdW2 = 72;   // W2^T and W2 [64][64]
constexpr int kLdT = kTile + 8;  // transposed activations [feature][row]

constexpr size_t kW1Elems = (size_t)kH * kLdW1, kW2Elems = (size_t)kH * kLdW2;
constexpr size_t kSmemWeights = (kW1Elems + 2 * kW2Elems) * 2 + (3 * kH + 4) * 4;
constexpr size_t kSmemTrain = kSmemWeights + (size_t)(kIn + 3 * kH) * kLdT * 2 + (3 * kWarps * kH + 2 * kWarps) * 4;

struct Weights {
    const __nv_bfloat16 *w1t;  // [64][kLdW1]: w1t[n][k] = bf16(W1[k][n])
    const __nv_bfloat16 *w2t;  // [64][kLdW2]: w2t[n][k] = bf16(W2[k][n])
    const __nv_bfloat16 *w2n;  // [64][kLdW2]: w2n[k][n] = bf16(W2[k][n])
    const float *master;       // FP32 parameters
};

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t bits16(__nv_bfloat16 v) { return (uint32_t)__bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) { return bits16(lo) | (bits16(hi) << 16); }
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Input x[row][c]: features for c < 32, one-hot band for 32 <= c < 36, zero above.
__device__ __forceinline__ float2 input_pair(const float *__restrict__ feat, int band, bool valid, int row, int c) {
    if (!valid) return make_float2(0.f, 0.f);
    if (c < kFeat) return __ldg(reinterpret_cast<const float2 *>(feat + (size_t)row * kFeat + c));
    const int b = c - kFeat;
    return make_float2(b == band ? 1.f : 0.f, b + 1 == band ? 1.f : 0.f);
}

template <bool kTrain>
__global__ void __launch_bounds__(kThreads, 1) k_mlp(int64_t n, int n_tiles, const float *__restrict__ feat,
                                                     const int32_t *__restrict__ band,
                                                     const float *__restrict__ target, Weights W, float inv_n,
                                                     float *__restrict__ score, float *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *sW1t = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sW2t = sW1t + kW1Elems;
    __nv_bfloat16 *sW2n = sW2t + kW2Elems;
    float *sb1 = reinterpret_cast<float *>(sW2n + kW2Elems);
    float *sb2 = sb1 + kH, *sw3 = sb2 + kH, *sb3 = sw3 + kH;
    __nv_bfloat16 *sXT = reinterpret_cast<__nv_bfloat16 *>(sb3 + 4);  // training only
    __nv_bfloat16 *sH1T = sXT + (size_t)kIn * kLdT;
    __nv_bfloat16 *sD2T = sH1T + (size_t)kH * kLdT;
    __nv_bfloat16 *sD1T = sD2T + (size_t)kH * kLdT;
    float *sRed = reinterpret_cast<float *>(sD1T + (size_t)kH * kLdT);  // [3][kWarps][kH] + [2][kWarps]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    {
        const uint4 *s1 = reinterpret_cast<const uint4 *>(W.w1t);
        const uint4 *s2 = reinterpret_cast<const uint4 *>(W.w2t);
        const uint4 *s3 = reinterpret_cast<const uint4 *>(W.w2n);
        uint4 *d1 = reinterpret_cast<uint4 *>(sW1t), *d2 = reinterpret_cast<uint4 *>(sW2t),
              *d3 = reinterpret_cast<uint4 *>(sW2n);
        for (int i = tid; i < (int)(kW1Elems / 8); i += kThreads) d1[i] = s1[i];
        for (int i = tid; i < (int)(kW2Elems / 8); i += kThreads) {
            d2[i] = s2[i];
            if (kTrain) d3[i] = s3[i];
        }
        for (int i = tid; i < kH; i += kThreads) {
            sb1[i] = W.master[oB1 + i];
            sb2[i] = W.master[oB2 + i];
            sw3[i] = W.master[oW3 + i];
        }
        if (tid == 0) sb3[0] = W.master[oB3];
    }
    __syncthreads();

    // training accumulators (per thread, columns 8 nt + 2 q + e)
    float acc_w3[8][2], acc_b2[8][2], acc_b1[8][2];
    float acc_dw2[4][4], acc_dw1[3][4];
    float acc_b3 = 0.f, acc_loss = 0.f;
    if (kTrain) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int e = 0; e < 2; ++e) acc_w3[i][e] = acc_b2[i][e] = acc_b1[i][e] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc_dw2[i][e] = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc_dw1[i][e] = 0.f;
    }

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r0 = (int64_t)tile * kTile + warp * 16;
        const int64_t ra = r0 + g, rb = r0 + g + 8;
        const bool va = ra < n, vb = rb < n;
        int ba = va ? __ldg(band + ra) : -1, bb = vb ? __ldg(band + rb) : -1;
        if (ba < 0 || ba > 3) ba = -1;  // no band: all-zero one-hot
        if (bb < 0 || bb > 3) bb = -1;
        const int la = warp * 16 + g, lb = la + 8;  // rows within the CTA tile

        // ---- layer 1: z1 = x W1 + b1 -------------------------------------
        uint32_t a1[3][4];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int c = 16 * kk + 8 * half + 2 * q;
                const float2 xa = input_pair(feat, ba, va, (int)ra, c);
                const float2 xb = input_pair(feat, bb, vb, (int)rb, c);
                const __nv_bfloat16 xa0 = __float2bfloat16_rn(xa.x), xa1 = __float2bfloat16_rn(xa.y);
                const __nv_bfloat16 xb0 = __float2bfloat16_rn(xb.x), xb1 = __float2bfloat16_rn(xb.y);
                a1[kk][2 * half] = pack2(xa0, xa1);
                a1[kk][2 * half + 1] = pack2(xb0, xb1);
                if (kTrain) {
                    sXT[c * kLdT + la] = xa0;
                    sXT[(c + 1) * kLdT + la] = xa1;
                    sXT[c * kLdT + lb] = xb0;
                    sXT[(c + 1) * kLdT + lb] = xb1;
                }
            }
        }
        uint32_t a2[4][4];  // bf16 h1 as layer-2 A fragments
        uint32_t mask1 = 0;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + 2 * q;
            float d[4] = {sb1[col], sb1[col + 1], sb1[col], sb1[col + 1]};
            const __nv_bfloat16 *bp = sW1t + (8 * nt + g) * kLdW1 + 2 * q;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) mma16816(d, a1[kk], ld32(bp + 16 * kk), ld32(bp + 16 * kk + 8));
            __nv_bfloat16 h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (d[e] > 0.f) mask1 |= 1u << (4 * nt + e);
                h[e] = __float2bfloat16_rn(fmaxf(d[e], 0.f));
            }
            a2[nt >> 1][(nt & 1) * 2] = pack2(h[0], h[1]);
            a2[nt >> 1][(nt & 1) * 2 + 1] = pack2(h[2], h[3]);
            if (kTrain) {
                sH1T[col * kLdT + la] = h[0];
                sH1T[(col + 1) * kLdT + la] = h[1];
                sH1T[col * kLdT + lb] = h[2];
                sH1T[(col + 1) * kLdT + lb] = h[3];
            }
        }
        // ---- layer 2: z2 = h1 W2 + b2; output y = relu(z2) w3 + b3 --------
        float h2[8][4];
        uint32_t mask2 = 0;
        float pa = 0.f, pb = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + 2 * q;
            float d[4] = {sb2[col], sb2[col + 1], sb2[col], sb2[col + 1]};
            const __nv_bfloat16 *bp = sW2t + (8 * nt + g) * kLdW2 + 2 * q;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma16816(d, a2[kk], ld32(bp + 16 * kk), ld32(bp + 16 * kk + 8));
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (d[e] > 0.f) mask2 |= 1u << (4 * nt + e);
                h2[nt][e] = fmaxf(d[e], 0.f);
            }
            pa += h2[nt][0] * sw3[col] + h2[nt][1] * sw3[col + 1];
            pb += h2[nt][2] * sw3[col] + h2[nt][3] * sw3[col + 1];
        }
        pa += __shfl_xor_sync(0xffffffffu, pa, 1);
        pa += __shfl_xor_sync(0xffffffffu, pa, 2);
        pb += __shfl_xor_sync(0xffffffffu, pb, 1);
        pb += __shfl_xor_sync(0xffffffffu, pb, 2);
        const float ya = pa + sb3[0], yb = pb + sb3[0];
        if (!kTrain) {
            if (q == 0) {
                if (va) score[ra] = ya;
                if (vb) score[rb] = yb;
            }
            continue;
        }
        // ---- backward ---------------------------------------------------
        const float ea = va ? ya - __ldg(target + ra) : 0.f;
        const float eb = vb ? yb - __ldg(target + rb) : 0.f;
        const float dya = 2.f * ea * inv_n, dyb = 2.f * eb * inv_n;
        if (q == 0) {
            acc_loss += ea * ea + eb * eb;
            acc_b3 += dya + dyb;
        }
        uint32_t ad[4][4];  // bf16 dz2 as A fragments (k = second hidden unit)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + 2 * q;
            float dz[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float dy = e < 2 ? dya : dyb;
                dz[e] = (mask2 >> (4 * nt + e)) & 1u ? dy * sw3[col + (e & 1)] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                acc_w3[nt][e] += dya * h2[nt][e] + dyb * h2[nt][2 + e];
                acc_b2[nt][e] += dz[e] + dz[2 + e];
            }
            __nv_bfloat16 hb[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) hb[e] = __float2bfloat16_rn(dz[e]);
            ad[nt >> 1][(nt & 1) * 2] = pack2(hb[0], hb[1]);
            ad[nt >> 1][(nt & 1) * 2 + 1] = pack2(hb[2], hb[3]);
            sD2T[col * kLdT + la] = hb[0];
            sD2T[(col + 1) * kLdT + la] = hb[1];
            sD2T[col * kLdT + lb] = hb[2];
            sD2T[(col + 1) * kLdT + lb] = hb[3];
        }
        // dh1 = dz2 W2^T, dz1 = dh1 * [z1 > 0]
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + 2 * q;
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16 *bp = sW2n + (8 * nt + g) * kLdW2 + 2 * q;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma16816(d, ad[kk], ld32(bp + 16 * kk), ld32(bp + 16 * kk + 8));
            __nv_bfloat16 hb[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float dz = (mask1 >> (4 * nt + e)) & 1u ? d[e] : 0.f;
                if (e < 2) acc_b1[nt][e] += dz; else acc_b1[nt][e - 2] += dz;
                hb[e] = __float2bfloat16_rn(dz);
            }
            sD1T[col * kLdT + la] = hb[0];
            sD1T[(col + 1) * kLdT + la] = hb[1];
            sD1T[col * kLdT + lb] = hb[2];
            sD1T[(col + 1) * kLdT + lb] = hb[3];
        }
        __syncthreads();
        // ---- weight gradients over the tile's 128 rows ------------------
        // dW2[m][n] = sum_r h1[r][m] dz2[r][n]: warp -> m tile warp/2, n tiles 4 (warp%2) + i
        {
            const int mt = warp >> 1;
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks) {
                const __nv_bfloat16 *ap = sH1T + (16 * mt + g) * kLdT + 16 * ks + 2 * q;
                const uint32_t a[4] = {ld32(ap), ld32(ap + 8 * kLdT), ld32(ap + 8), ld32(ap + 8 * kLdT + 8)};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int nt = 4 * (warp & 1) + i;
                    const __nv_bfloat16 *bp = sD2T + (8 * nt + g) * kLdT + 16 * ks + 2 * q;
                    mma16816(acc_dw2[i], a, ld32(bp), ld32(bp + 8));
                }
            }
        }
        // dW1[m][n] = sum_r x[r][m] dz1[r][n]: 3 m tiles x 8 n tiles, 3 per warp
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int id = 3 * warp + i, mt = id >> 3, nt = id & 7;
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ++ks) {
                const __nv_bfloat16 *ap = sXT + (16 * mt + g) * kLdT + 16 * ks + 2 * q;
                const uint32_t a[4] = {ld32(ap), ld32(ap + 8 * kLdT), ld32(ap + 8), ld32(ap + 8 * kLdT + 8)};
                const __nv_bfloat16 *bp = sD1T + (8 * nt + g) * kLdT + 16 * ks + 2 * q;
                mma16816(acc_dw1[i], a, ld32(bp), ld32(bp + 8));
            }
        }
        __syncthreads();  // the transposed tiles are rewritten by the next tile
    }
    if (!kTrain) return;

    // ---- per-CTA partial gradient, written in a fixed order --------------
    float *out = partial + (size_t)blockIdx.x * (kP + 1);
    {
        const int mt = warp >> 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int nt = 4 * (warp & 1) + i;
            const int m = 16 * mt + g, c = 8 * nt + 2 * q;
            out[oW2 + m * kH + c] = acc_dw2[i][0];
            out[oW2 + m * kH + c + 1] = acc_dw2[i][1];
            out[oW2 + (m + 8) * kH + c] = acc_dw2[i][2];
            out[oW2 + (m + 8) * kH + c + 1] = acc_dw2[i][3];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int id = 3 * warp + i, mt = id >> 3, nt = id & 7;
        const int m = 16 * mt + g, c = 8 * nt + 2 * q;
        out[oW1 + m * kH + c] = acc_dw1[i][0];
        out[oW1 + m * kH + c + 1] = acc_dw1[i][1];
        out[oW1 + (m + 8) * kH + c] = acc_dw1[i][2];
        out[oW1 + (m + 8) * kH + c + 1] = acc_dw1[i][3];
    }
    // column sums: over the 8 lanes of equal q, then over warps via shared memory
    float *rw3 = sRed, *rb2 = rw3 + kWarps * kH, *rb1 = rb2 + kWarps * kH, *rs = rb1 + kWarps * kH;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float a = acc_w3[nt][e], b = acc_b2[nt][e], c = acc_b1[nt][e];
#pragma unroll
            for (int s = 4; s < 32; s <<= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, s);
                b += __shfl_xor_sync(0xffffffffu, b, s);
                c += __shfl_xor_sync(0xffffffffu, c, s);
            }
            if (g == 0) {
                const int col = 8 * nt + 2 * q + e;
                rw3[warp * kH + col] = a;
                rb2[warp * kH + col] = b;
                rb1[warp * kH + col] = c;
            }
        }
    float l = acc_loss, b3 = acc_b3;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, s);
        b3 += __shfl_xor_sync(0xffffffffu, b3, s);
    }
    if (lane == 0) {
        rs[warp] = b3;
        rs[kWarps + warp] = l;
    }
    __syncthreads();
    if (tid < kH) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            a += rw3[w * kH + tid];
            b += rb2[w * kH + tid];
            c += rb1[w * kH + tid];
        }
        out[oW3 + tid] = a;
        out[oB2 + tid] = b;
        out[oB1 + tid] = c;
    }
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            a += rs[w];
            b += rs[kWarps + w];
        }
        out[oB3] = a;
        out[kP] = b;  // sum of squared errors
    }
}

// Sum the per-CTA partials (fixed order), then Adam on the FP32 master
// weights and refresh the BF16 copies.  One thread per parameter; thread kP
// sums the squared errors.
__global__ void k_mlp_adam(int n_part, const float *__restrict__ partial, float *__restrict__ master,
                           float *__restrict__ m1, float *__restrict__ m2, float *__restrict__ grad,
                           __nv_bfloat16 *__restrict__ w1t, __nv_bfloat16 *__restrict__ w2t,
                           __nv_bfloat16 *__restrict__ w2n, float lr, float bc1, float bc2, float *__restrict__ sse) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kP) return;
    float s = 0.f;
    for (int c = 0; c < n_part; ++c) s += partial[(size_t)c * (kP + 1) + p];
    if (p == kP) {
        *sse = s;
        return;
    }
    grad[p] = s;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * m1[p] + (1.f - b1) * s;
    const float v = b2 * m2[p] + (1.f - b2) * s * s;
    m1[p] = m;
    m2[p] = v;
    const float th = master[p] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    master[p] = th;
    if (p < oB1) {
        const int k = p / kH, n = p % kH;
        w1t[n * kLdW1 + k] = __float2bfloat16_rn(th);
    } else if (p >= oW2 && p < oB2) {
        const int k = (p - oW2) / kH, n = (p - oW2) % kH;
        w2t[n * kLdW2 + k] = __float2bfloat16_rn(th);
        w2n[k * kLdW2 + n] = __float2bfloat16_rn(th);
    }
}

// BF16 copies of W1 and W2 from the master weights (after set_params).
__global__ void k_mlp_copies(const float *__restrict__ master, __nv_bfloat16 *__restrict__ w1t,
                             __nv_bfloat16 *__restrict__ w2t, __nv_bfloat16 *__restrict__ w2n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < oB1) {
        const int k = p / kH, n = p % kH;
        w1t[n * kLdW1 + k] = __float2bfloat16_rn(master[p]);
    } else if (p >= oW2 && p < oB2) {
        const int k = (p - oW2) / kH, n = (p - oW2) % kH;
        w2t[n * kLdW2 + k] = __float2bfloat16_rn(master[p]);
        w2n[k * kLdW2 + n] = __float2bfloat16_rn(master[p]);
    }
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of a counter.
uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace

struct cs_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    std::string err;
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr, *sse = nullptr, *h_sse = nullptr;
    __nv_bfloat16 *w1t = nullptr, *w2t = nullptr, *w2n = nullptr;
    float *partial = nullptr;
    int n_part_cap = 0;
    int64_t steps = 0;
};

namespace {

int mfail(cs_mlp *m, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    m->err = buf;
    return code;
}

#define MLP_CUDA(m, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            return mfail(m, e_ == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA, "%s: %s", \
                         #call, cudaGetErrorString(e_));                                          \
        }                                                                                         \
    } while (0)

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int grid_for(const cs_mlp *m, int64_t n) {
    const int64_t tiles = (n + kTile - 1) / kTile;
    return (int)std::min<int64_t>(tiles, 2LL * m->n_sm);
}

int refresh_copies(cs_mlp *m) {
    MLP_CUDA(m, cudaMemsetAsync(m->w1t, 0, kW1Elems * 2, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->w2t, 0, kW2Elems * 2, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->w2n, 0, kW2Elems * 2, m->stream));
    k_mlp_copies<<<(kP + 255) / 256, 256, 0, m->stream>>>(m->master, m->w1t, m->w2t, m->w2n);
    MLP_CUDA(m, cudaGetLastError());
    return CS_OK;
}

}  // namespace

extern "C" {

int cs_mlp_create(cs_mlp **out, int32_t device, void *stream, uint64_t seed) {
    if (!out) return CS_ERR_ARG;
    *out = nullptr;
    cs_mlp *m = new cs_mlp();
    m->device = device;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    auto bail = [&](int code) {
        cs_mlp_destroy(m);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(CS_ERR_CUDA);
    if (cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return bail(CS_ERR_CUDA);
    if (cudaMalloc(&m->master, kP * 4) != cudaSuccess || cudaMalloc(&m->m1, kP * 4) != cudaSuccess ||
        cudaMalloc(&m->m2, kP * 4) != cudaSuccess || cudaMalloc(&m->grad, kP * 4) != cudaSuccess ||
        cudaMalloc(&m->sse, 16) != cudaSuccess || cudaMalloc(&m->w1t, kW1Elems * 2) != cudaSuccess ||
        cudaMalloc(&m->w2t, kW2Elems * 2) != cudaSuccess || cudaMalloc(&m->w2n, kW2Elems * 2) != cudaSuccess ||
        cudaMallocHost(&m->h_sse, 16) != cudaSuccess) {
        cudaGetLastError();
        return bail(CS_ERR_OOM);
    }
    if (cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTrain) != cudaSuccess ||
        cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTrain) != cudaSuccess)
        return bail(CS_ERR_CUDA);
    // initial weights from the counter-based generator
    std::vector<float> p(kP, 0.0f);
    auto uni = [&](uint64_t i) {  // uniform in [-1, 1)
        return (float)((double)(splitmix64(seed * 0x100000001B3ull + i) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    };
    const float s1 = std::sqrt(6.0f / 36.0f), s2 = std::sqrt(6.0f / 64.0f), s3 = std::sqrt(3.0f / 64.0f);
    for (int k = 0; k < 36; ++k)
        for (int n = 0; n < kH; ++n) p[oW1 + k * kH + n] = s1 * uni(oW1 + k * kH + n);
    for (int i = 0; i < kH * kH; ++i) p[oW2 + i] = s2 * uni(oW2 + i);
    for (int i = 0; i < kH; ++i) p[oW3 + i] = s3 * uni(oW3 + i);
    int rc = cs_mlp_set_params(m, p.data());
    if (rc != CS_OK) return bail(rc);
    *out = m;
    return CS_OK;
}

void cs_mlp_destroy(cs_mlp *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->master);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->grad);
    cudaFree(m->sse);
    cudaFree(m->w1t);
    cudaFree(m->w2t);
    cudaFree(m->w2n);
    cudaFree(m->partial);
    cudaFreeHost(m->h_sse);
    delete m;
}

const char *cs_mlp_last_error(const cs_mlp *m) { return m ? m->err.c_str() : "null MLP"; }

int cs_mlp_get_params(cs_mlp *m, float *host_out) {
    if (!m) return CS_ERR_ARG;
    if (!host_out) return mfail(m, CS_ERR_ARG, "NULL output");
    MLP_CUDA(m, cudaSetDevice(m->device));
    MLP_CUDA(m, cudaMemcpyAsync(host_out, m->master, kP * 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return CS_OK;
}

int cs_mlp_set_params(cs_mlp *m, const float *host_in) {
    if (!m) return CS_ERR_ARG;
    if (!host_in) return mfail(m, CS_ERR_ARG, "NULL parameters");
    for (int i = 0; i < kP; ++i)
        if (!std::isfinite(host_in[i])) return mfail(m, CS_ERR_ARG, "parameter %d is not finite", i);
    MLP_CUDA(m, cudaSetDevice(m->device));
    MLP_CUDA(m, cudaMemcpyAsync(m->master, host_in, kP * 4, cudaMemcpyHostToDevice, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m1, 0, kP * 4, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m2, 0, kP * 4, m->stream));
    int rc = refresh_copies(m);
    if (rc != CS_OK) return rc;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    m->steps = 0;
    return CS_OK;
}

int cs_mlp_forward(cs_mlp *m, int64_t n, const float *feat, const int32_t *band, float *score_out) {
    if (!m) return CS_ERR_ARG;
    if (n < 0) return mfail(m, CS_ERR_ARG, "n must be >= 0");
    if (n == 0) return CS_OK;
    if (n > (int64_t)INT32_MAX) return mfail(m, CS_ERR_CAPACITY, "n exceeds 2^31 - 1");
    if (!feat || !band || !score_out || !aligned(feat, 8) || !aligned(band, 4) || !aligned(score_out, 4))
        return mfail(m, CS_ERR_ARG, "NULL or misaligned array");
    MLP_CUDA(m, cudaSetDevice(m->device));
    const int tiles = (int)((n + kTile - 1) / kTile);
    Weights W{m->w1t, m->w2t, m->w2n, m->master};
    k_mlp<false><<<grid_for(m, n), kThreads, kSmemWeights, m->stream>>>(n, tiles, feat, band, nullptr, W, 0.f,
                                                                       score_out, nullptr);
    MLP_CUDA(m, cudaGetLastError());
    return CS_OK;
}

int cs_mlp_train_step(cs_mlp *m, int64_t n, const float *feat, const int32_t *band, const float *target, float lr,
                      float *loss_out) {
    if (!m) return CS_ERR_ARG;
    if (n < 1) return mfail(m, CS_ERR_ARG, "n must be >= 1");
    if (n > (int64_t)INT32_MAX) return mfail(m, CS_ERR_CAPACITY, "n exceeds 2^31 - 1");
    if (!(lr > 0.0f) || !std::isfinite(lr)) return mfail(m, CS_ERR_ARG, "lr must be > 0");
    if (!feat || !band || !target || !aligned(feat, 8) || !aligned(band, 4) || !aligned(target, 4))
        return mfail(m, CS_ERR_ARG, "NULL or misaligned array");
    MLP_CUDA(m, cudaSetDevice(m->device));
    const int grid = grid_for(m, n);
    if (grid > m->n_part_cap) {
        MLP_CUDA(m, cudaStreamSynchronize(m->stream));
        cudaFree(m->partial);
        m->partial = nullptr;
        m->n_part_cap = 0;
        MLP_CUDA(m, cudaMalloc(&m->partial, (size_t)grid * (kP + 1) * 4));
        m->n_part_cap = grid;
    }
    const int tiles = (int)((n + kTile - 1) / kTile);
    Weights W{m->w1t, m->w2t, m->w2n, m->master};
    k_mlp<true><<<grid, kThreads, kSmemTrain, m->stream>>>(n, tiles, feat, band, target, W, (float)(1.0 / (double)n),
                                                          nullptr, m->partial);
    MLP_CUDA(m, cudaGetLastError());
    const int64_t t = m->steps + 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)t)), bc2 = (float)(1.0 - std::pow(0.999, (double)t));
    k_mlp_adam<<<(kP + 1 + 255) / 256, 256, 0, m->stream>>>(grid, m->partial, m->master, m->m1, m->m2, m->grad,
                                                              m->w1t, m->w2t, m->w2n, lr, bc1, bc2, m->sse);
    MLP_CUDA(m, cudaGetLastError());
    m->steps = t;
    if (loss_out) {
        MLP_CUDA(m, cudaMemcpyAsync(m->h_sse, m->sse, 4, cudaMemcpyDeviceToHost, m->stream));
        MLP_CUDA(m, cudaStreamSynchronize(m->stream));
        *loss_out = (float)((double)m->h_sse[0] / (double)n);
    }
    return CS_OK;
}

int cs_mlp_get_grad(cs_mlp *m, float *host_out) {
    if (!m) return CS_ERR_ARG;
    if (!host_out) return mfail(m, CS_ERR_ARG, "NULL output");
    if (m->steps == 0) return mfail(m, CS_ERR_STATE, "no training step yet");
    MLP_CUDA(m, cudaSetDevice(m->device));
    MLP_CUDA(m, cudaMemcpyAsync(host_out, m->grad, kP * 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return CS_OK;
}

}  // extern "C"
