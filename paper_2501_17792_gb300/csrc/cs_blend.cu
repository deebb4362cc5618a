// cs_blend.cu -- front-to-back alpha compositing of a CrowdSplat frame.
//
// The 3DGS rasteriser CrowdSplat renders with (cited in Sec. 1 and Sec. 2)
// composites, for every pixel, the depth-sorted splats of its 16x16 tile:
//   q = -(A dx^2 + C dy^2)/2 - B dx dy;  skip q > 0;
//   alpha = min(0.99, o e^q);  skip alpha < 1/255;
//   T' = T (1 - alpha);  stop (without this splat) once T' < 1e-4;
//   C += c alpha T;  T = T'.
// A splat also contributes only where the pixel centre lies in its square
// support box (|dx|, |dy| <= r), which makes the image independent of the
// tile size.  One CTA per tile, one thread per pixel; the CTA stages
// batches of splat records in shared memory and stops once every pixel of
// the tile is saturated.
#include "cs_internal.cuh"

namespace cs {

constexpr int kBlendThreads = kTile * kTile;

__global__ void __launch_bounds__(kBlendThreads) k_blend(int tiles_x, int W, int H,
                                                         const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ pval,
                                                         const float4 *__restrict__ rec,
                                                         float4 *__restrict__ out) {
    __shared__ float4 s0[kBlendThreads];
    __shared__ float4 s1[kBlendThreads];
    __shared__ float4 s2[kBlendThreads];
    const int tile = blockIdx.x;
    const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
    const int px = txi * kTile + (threadIdx.x & (kTile - 1));
    const int py = tyi * kTile + (threadIdx.x / kTile);
    const bool inside = px < W && py < H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    int done = inside ? 0 : 1;
    for (uint32_t base = rg.x; base < rg.y; base += kBlendThreads) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        const uint32_t idx = base + threadIdx.x;
        if (idx < rg.y) {
            const uint32_t s = pval[idx];
            s0[threadIdx.x] = rec[(size_t)s * 3 + 0];
            s1[threadIdx.x] = rec[(size_t)s * 3 + 1];
            s2[threadIdx.x] = rec[(size_t)s * 3 + 2];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)kBlendThreads, rg.y - base);
        if (!done) {
            for (int j = 0; j < nb; ++j) {
                const float4 a = s0[j];   // u, v, A, B
                const float4 b = s1[j];   // C, opacity, radius, depth
                const float dx = fpx - a.x, dy = fpy - a.y;
                if (fabsf(dx) > b.z || fabsf(dy) > b.z) continue;
                const float q = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
                if (q > 0.0f) continue;
                const float alpha = fminf(0.99f, b.y * __expf(q));
                if (alpha < (1.0f / 255.0f)) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < 1e-4f) {
                    done = 1;
                    break;
                }
                const float4 c = s2[j];
                const float wgt = alpha * T;
                cr += c.x * wgt;
                cg += c.y * wgt;
                cb += c.z * wgt;
                T = Tn;
            }
        }
    }
    if (inside) out[(size_t)py * W + px] = make_float4(cr, cg, cb, 1.0f - T);
}

int launch_blend(int tiles_x, int tiles_y, int W, int H, const uint2 *ranges, const uint32_t *pval,
                 const float4 *rec, float4 *out, cudaStream_t st) {
    const int n = tiles_x * tiles_y;
    if (n <= 0) return 0;
    k_blend<<<n, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, out);
    return 1;
}

}  // namespace cs
