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
// tile size.
//
// One CTA per tile, one thread per pixel, each warp an 8x4 block of the
// tile.  The CTA stages batches of 256 splat records in shared memory; the
// thread that loads a splat also marks which of the 8 warp blocks hold a
// pixel the splat can reach (the exact rectangle test of binning), and each
// warp walks only its marked splats (ballot over 32 splats at a time).  The
// CTA stops once every pixel of the tile is saturated.
#include "cs_internal.cuh"

namespace cs {

constexpr int kBlendThreads = kTile * kTile;
constexpr int kBlockW = 8, kBlockH = 4;  // pixels per warp

__global__ void __launch_bounds__(kBlendThreads) k_blend(int tiles_x, int W, int H,
                                                         const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ pval,
                                                         const float4 *__restrict__ rec,
                                                         float4 *__restrict__ out) {
    __shared__ float4 s0[kBlendThreads];
    __shared__ float4 s1[kBlendThreads];
    __shared__ float4 s2[kBlendThreads];
    __shared__ uint8_t smask[kBlendThreads];
    const int tile = blockIdx.x;
    const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = (warp & 1) * kBlockW, by = (warp >> 1) * kBlockH;
    const int tx0 = txi * kTile, ty0 = tyi * kTile;
    const int px = tx0 + bx + (lane & (kBlockW - 1));
    const int py = ty0 + by + (lane / kBlockW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint32_t wbit = 1u << warp;
    const uint2 rg = ranges[tile];
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += kBlendThreads) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        const uint32_t idx = base + threadIdx.x;
        if (idx < rg.y) {
            const uint32_t s = pval[idx];
            const float4 a = rec[(size_t)s * 3 + 0];
            const float4 b = rec[(size_t)s * 3 + 1];
            s0[threadIdx.x] = a;
            s1[threadIdx.x] = b;
            s2[threadIdx.x] = rec[(size_t)s * 3 + 2];
            // warp blocks of this tile that hold a pixel the splat can reach
            int qx0, qx1, qy0, qy1;
            box_range(a.x, b.z, W, qx0, qx1);
            box_range(a.y, b.z, H, qy0, qy1);
            const float fcut = splat_fcut(b.y);
            uint32_t m = 0;
#pragma unroll
            for (int w = 0; w < kBlendThreads / 32; ++w) {
                const int wx0 = max(tx0 + (w & 1) * kBlockW, qx0);
                const int wx1 = min(tx0 + (w & 1) * kBlockW + kBlockW - 1, qx1);
                const int wy0 = max(ty0 + (w >> 1) * kBlockH, qy0);
                const int wy1 = min(ty0 + (w >> 1) * kBlockH + kBlockH - 1, qy1);
                if (wx0 <= wx1 && wy0 <= wy1 &&
                    splat_rect_hits(a.x, a.y, a.z, a.w, b.x, fcut, wx0, wx1, wy0, wy1))
                    m |= 1u << w;
            }
            smask[threadIdx.x] = (uint8_t)m;
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)kBlendThreads, rg.y - base);
        for (int c = 0; c < nb; c += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const bool mine = c + lane < nb && (smask[c + lane] & wbit);
            uint32_t m = __ballot_sync(0xffffffffu, mine);
            while (m) {
                const int j = c + __ffs(m) - 1;
                m &= m - 1;
                if (done) continue;
                const float4 a = s0[j];  // u, v, A, B
                const float4 b = s1[j];  // C, opacity, radius, depth
                const float dx = fpx - a.x, dy = fpy - a.y;
                if (fabsf(dx) > b.z || fabsf(dy) > b.z) continue;
                const float q = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
                if (q > 0.0f) continue;
                const float alpha = fminf(0.99f, b.y * __expf(q));
                if (alpha < (1.0f / 255.0f)) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < 1e-4f) {
                    done = true;
                    continue;
                }
                const float4 col = s2[j];
                const float wgt = alpha * T;
                cr += col.x * wgt;
                cg += col.y * wgt;
                cb += col.z * wgt;
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
