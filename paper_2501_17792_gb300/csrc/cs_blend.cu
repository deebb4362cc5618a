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
// One CTA per tile, one thread per pixel, each warp an 8x4 block of the tile.
// Warps are independent (no CTA-wide barrier): a warp walks the tile's
// depth-ordered pair list 32 entries at a time; each lane loads one splat
// (the 8 warps of a tile share the loads through L1), keeps it if the splat
// can reach a pixel of the warp's block (box overlap, then the exact
// rectangle test of binning), and stages kept splats in the warp's slice of
// shared memory with the exponent pre-scaled to base 2 (e^q = 2^(q log2 e),
// evaluated with the hardware ex2).  The warp then composites the kept splats
// in order and leaves the tile once all 32 pixels are saturated.
#include "cs_internal.cuh"

namespace cs {

constexpr int kBlendThreads = kTile * kTile;
constexpr int kBlendWarps = kBlendThreads / 32;
constexpr int kBlockW = 8, kBlockH = 4;  // pixels per warp
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kBlendThreads) k_blend(int tiles_x, int W, int H,
                                                         const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ pval,
                                                         const float4 *__restrict__ rec,
                                                         float4 *__restrict__ out) {
    // per warp, per lane: {u, v, a, b}, {c, log2 o, r, -}, {r, g, b, -} with
    // a = -A log2e / 2, b = -B log2e, c = -C log2e / 2
    __shared__ float4 sg[kBlendWarps][32][3];
    const int tile = blockIdx.x;
    const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = txi * kTile + (warp & 1) * kBlockW;
    const int by0 = tyi * kTile + (warp >> 1) * kBlockH;
    const int bx1 = min(bx0 + kBlockW - 1, W - 1), by1 = min(by0 + kBlockH - 1, H - 1);
    if (bx0 > bx1 || by0 > by1) return;  // the whole warp block lies outside the image
    const int px = bx0 + (lane & (kBlockW - 1));
    const int py = by0 + (lane / kBlockW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    bool done = !inside;
    float4(*slot)[3] = sg[warp];
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const uint32_t idx = base + lane;
        bool keep = false;
        if (idx < rg.y) {
            const uint32_t s = __ldg(pval + idx);
            const float4 a = __ldg(rec + (size_t)s * 3 + 0);  // u, v, A, B
            const float4 b = __ldg(rec + (size_t)s * 3 + 1);  // C, opacity, radius, depth
            int qx0, qx1, qy0, qy1;
            box_range(a.x, b.z, W, qx0, qx1);
            box_range(a.y, b.z, H, qy0, qy1);
            qx0 = max(qx0, bx0);
            qx1 = min(qx1, bx1);
            qy0 = max(qy0, by0);
            qy1 = min(qy1, by1);
            if (qx0 <= qx1 && qy0 <= qy1)
                keep = splat_rect_hits(a.x, a.y, a.z, a.w, b.x, splat_fcut(b.y), qx0, qx1, qy0, qy1);
            if (keep) {
                const float4 c = __ldg(rec + (size_t)s * 3 + 2);
                slot[lane][0] = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
                slot[lane][1] = make_float4(-0.5f * kLog2e * b.x, __log2f(b.y), b.z, 0.0f);
                slot[lane][2] = c;
            }
        }
        uint32_t m = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            if (done) continue;
            const float4 a = slot[j][0];
            const float4 b = slot[j][1];
            const float dx = fpx - a.x, dy = fpy - a.y;
            if (fmaxf(fabsf(dx), fabsf(dy)) > b.z) continue;
            // p = q log2 e
            const float p = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
            if (p > 0.0f) continue;
            const float alpha = fminf(0.99f, ex2_approx(p + b.y));
            if (alpha < (1.0f / 255.0f)) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < 1e-4f) {
                done = true;
                continue;
            }
            const float4 col = slot[j][2];
            const float wgt = alpha * T;
            cr += col.x * wgt;
            cg += col.y * wgt;
            cb += col.z * wgt;
            T = Tn;
        }
        __syncwarp();
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
