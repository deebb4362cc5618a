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
// The CTA walks the tile's depth-ordered pairs in batches of 256, software
// pipelined: while the warps composite batch k from one half of a shared
// double buffer, each thread holds in registers the record it loaded for
// batch k+1; after compositing it stages that record into the other half
// (with the warp blocks its reach box overlaps as an 8-bit mask, and the
// exponent pre-scaled to base 2: e^q = 2^(q log2 e) on the hardware ex2
// unit) and issues the loads of batch k+2, so global latency hides behind a
// whole batch of compositing.  Each warp walks only the splats marked for
// its block (ballot over 32 at a time); the CTA leaves once every pixel of
// the tile is saturated.
#include "cs_internal.cuh"

namespace cs {

constexpr int kBlendThreads = kTile * kTile;
constexpr int kBlockW = 8, kBlockH = 4;  // pixels per warp
constexpr float kLog2e = 1.4426950408889634f;

// e^q evaluated as 2^(q log2 e) on the hardware ex2 unit
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct StagedRecord {
    float4 a, b, c, q;  // {u, v, A, B}, {C, o, r, depth}, {r, g, b, -}, {reach x, reach y, fcut, log2 o}
    bool have;
};

__device__ __forceinline__ void load_record(StagedRecord &r, const uint32_t *__restrict__ pval,
                                            const float4 *__restrict__ rec, uint32_t idx, uint32_t end) {
    r.have = idx < end;
    if (r.have) {
        const float4 *p = rec + (size_t)__ldg(pval + idx) * kRecVec;
        r.a = __ldg(p + 0);
        r.b = __ldg(p + 1);
        r.c = __ldg(p + 2);
        r.q = __ldg(p + 3);
    }
}

__global__ void __launch_bounds__(kBlendThreads) k_blend(int tiles_x, int W, int H,
                                                         const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ pval,
                                                         const float4 *__restrict__ rec,
                                                         float4 *__restrict__ out) {
    // staged splats: {u, v, a', b'}, {c', log2 o, radius, -}, {r, g, b, -} with
    // p = q log2 e = a' dx^2 + b' dx dy + c' dy^2
    __shared__ float4 s0[2][kBlendThreads];
    __shared__ float4 s1[2][kBlendThreads];
    __shared__ float4 s2[2][kBlendThreads];
    __shared__ uint8_t smask[2][kBlendThreads];
    const int tile = blockIdx.x;
    const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx0 = txi * kTile, ty0 = tyi * kTile;
    const int px = tx0 + (warp & 1) * kBlockW + (lane & (kBlockW - 1));
    const int py = ty0 + (warp >> 1) * kBlockH + (lane / kBlockW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint32_t wbit = 1u << warp;
    const uint2 rg = ranges[tile];
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    bool done = !inside;

    // stage a loaded record into half `h`: pre-scaled exponent, warp-block mask
    auto stage = [&](const StagedRecord &r, int h) {
        uint32_t m = 0;
        if (r.have) {
            const uint32_t rx = __float_as_uint(r.q.x), ry = __float_as_uint(r.q.y);
            const int x0 = (int)(rx & 0xFFFFu) - tx0, x1 = (int)(rx >> 16) - tx0;
            const int y0 = (int)(ry & 0xFFFFu) - ty0, y1 = (int)(ry >> 16) - ty0;
#pragma unroll
            for (int w = 0; w < kBlendThreads / 32; ++w) {
                const int bx = (w & 1) * kBlockW, by = (w >> 1) * kBlockH;
                if (x0 <= bx + kBlockW - 1 && x1 >= bx && y0 <= by + kBlockH - 1 && y1 >= by) m |= 1u << w;
            }
            s0[h][tid] = make_float4(r.a.x, r.a.y, -0.5f * kLog2e * r.a.z, -kLog2e * r.a.w);
            s1[h][tid] = make_float4(-0.5f * kLog2e * r.b.x, r.q.w, r.b.z, 0.0f);
            s2[h][tid] = r.c;
        }
        smask[h][tid] = (uint8_t)m;
    };

    StagedRecord nxt;
    load_record(nxt, pval, rec, rg.x + tid, rg.y);
    stage(nxt, 0);
    load_record(nxt, pval, rec, rg.x + kBlendThreads + tid, rg.y);
    __syncthreads();
    int h = 0;
    for (uint32_t base = rg.x; base < rg.y; base += kBlendThreads, h ^= 1) {
        const int nb = (int)min((uint32_t)kBlendThreads, rg.y - base);
        for (int c = 0; c < nb; c += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const bool mine = (smask[h][c + lane] & wbit) != 0 && c + lane < nb;
            uint32_t m = __ballot_sync(0xffffffffu, mine);
            while (m) {
                const int j = c + __ffs(m) - 1;
                m &= m - 1;
                if (done) continue;
                const float4 a = s0[h][j];  // u, v, a', b'
                const float4 b = s1[h][j];  // c', log2 o, radius
                const float dx = fpx - a.x, dy = fpy - a.y;
                if (fmaxf(fabsf(dx), fabsf(dy)) > b.z) continue;
                const float p = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
                if (p > 0.0f) continue;
                const float alpha = fminf(0.99f, ex2_approx(p + b.y));
                if (alpha < (1.0f / 255.0f)) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < 1e-4f) {
                    done = true;
                    continue;
                }
                const float4 col = s2[h][j];
                const float wgt = alpha * T;
                cr += col.x * wgt;
                cg += col.y * wgt;
                cb += col.z * wgt;
                T = Tn;
            }
        }
        // the other half was last read before the previous barrier: refill it
        // with the next batch (loaded while this one was composited) and
        // start loading the batch after
        if (base + kBlendThreads < rg.y) {
            stage(nxt, h ^ 1);
            load_record(nxt, pval, rec, base + 2 * kBlendThreads + tid, rg.y);
        }
        if (__syncthreads_count(done) == kBlendThreads) break;
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
