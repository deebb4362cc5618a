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
// Pass 1 of a plain frame (k_blend_pp) composites each 8x4 pixel block of
// a tile with a long list with eight warps that split the block's
// depth-ordered pairs into sub-ranges and chain their partial composites,
// and every tile with a short list with one CTA, one warp per block
// (described at the kernel).
//
// The one-pass kernel of statistics frames, the split passes and the
// chunked passes of training frames below take one CTA per tile (or chunk of
// its list), one thread per pixel, each warp an 8x4 block of the tile.  A CTA walks depth-ordered pairs in batches of 256, software
// pipelined:
// while the warps composite batch k from one half of a shared double buffer,
// each thread holds in registers the record it loaded for batch k+1; after
// compositing it stages that record into the other half (with the warp
// blocks its reach box overlaps as an 8-bit mask, and the exponent
// pre-scaled to base 2: e^q = 2^(q log2 e) on the hardware ex2 unit) and
// issues the loads of batch k+2.  Each warp walks only the splats marked for
// its block; the CTA leaves once every pixel is saturated.
//
// Long lists are split in depth order (the compositing operator is
// associative): pass 1 composites the first kBudget pairs of every tile;
// tiles with unsaturated pixels left hand the rest to pass 2, which
// composites chunks of kChunk pairs in parallel, each from T = 1 and only
// for pixels pass 1 left open; the merge pass then combines, per pixel,
// C += T C_k, T *= T_k in order, up to the chunk (if any) inside which the
// pixel meets the stop rule (T T_k < 1e-4); the fix-up pass composites each
// such chunk again, in parallel over chunks, for its stopping pixels from
// their true T, so the stop rule holds exactly as in the definition.
#include <algorithm>

#include "crowdsplat.h"
#include "cs_internal.cuh"

namespace cs {

constexpr int kBlendThreads = kTile * kTile;
constexpr int kBlockW = kBlendBlockW, kBlockH = kBlendBlockH;  // pixels per warp
constexpr float kLog2e = 1.4426950408889634f;
constexpr uint32_t kBudget = kBlendBudget;  // pairs of pass 1 per tile
constexpr uint32_t kChunk = kBlendChunk;    // pairs per pass-2 chunk
constexpr size_t kChunkGrid = 8192;         // CTAs of the chunk and fix-up grids at most
static_assert(kBwdChunk % kBlendThreads == 0, "backward chunk boundaries fall on batch starts");

// e^q evaluated as 2^(q log2 e) on the hardware ex2 unit
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct StagedRecord {
    float4 q, a, c;  // {reach x, reach y, log2 o, C}, {u, v, A, B}, {r, g, b, radius}
    uint32_t s;         // splat id
    bool have;
};

__device__ __forceinline__ void load_record(StagedRecord &r, const uint32_t *__restrict__ pval,
                                            const float4 *__restrict__ rec, uint32_t idx, uint32_t end) {
    r.have = idx < end;
    if (r.have) {
        r.s = __ldg(pval + idx);
        const float4 *p = rec + (size_t)r.s * kRecVec;
        r.q = __ldg(p + 0);
        r.a = __ldg(p + 1);
        r.c = __ldg(p + 2);
    }
}

// kT threads stage batches of kT splats, double-buffered
template <int kT = kBlendThreads>
struct BlendShared {
    // staged splats: {u, v, a', b'}, {c', log2 o, radius, -}, {r, g, b, -} with
    // p = q log2 e = a' dx^2 + b' dx dy + c' dy^2
    float4 s0[2][kT];
    float4 s1[2][kT];
    float4 s2[2][kT];
    uint32_t sid[2][kT];
    uint8_t mask[2][kT];
};

struct Pixel {
    float T, r, g, b;
    uint32_t last;  // one past the last composited pair (training forward)
    bool done;     // saturated, outside the image, or not composited here
    bool stopped;  // met the stop rule in this call
};

// Composite pairs [start, end) of a tile into the calling thread's pixel.
// Every thread of the CTA must call it with the same range.  kMode 1
// (statistics): also add each composited weight alpha * T to
// contrib[splat]; kMode 2 (training): also track the last composited pair.
// kT: threads of the CTA, covering kT / 32 of the tile's 8x4 warp blocks
// from block row brow0 (a 16x16 tile has 8: two columns, four rows).
template <int kMode = 0, int kT = kBlendThreads>
__device__ __forceinline__ void composite_range(BlendShared<kT> &sh, uint32_t start, uint32_t end,
                                                const uint32_t *__restrict__ pval,
                                                const float4 *__restrict__ rec, int tx0, int ty0,
                                                float fpx, float fpy, Pixel &px,
                                                float *__restrict__ contrib = nullptr, int brow0 = 0) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t wbit = 1u << warp;
    auto stage = [&](const StagedRecord &r, int h) {
        uint32_t m = 0;
        if (r.have) {
            const uint32_t rx = __float_as_uint(r.q.x), ry = __float_as_uint(r.q.y);
            const int x0 = (int)(rx & 0xFFFFu) - tx0, x1 = (int)(rx >> 16) - tx0;
            const int y0 = (int)(ry & 0xFFFFu) - ty0, y1 = (int)(ry >> 16) - ty0;
#pragma unroll
            for (int w = 0; w < kT / 32; ++w) {
                const int bx = (w & 1) * kBlockW, by = ((w >> 1) + brow0) * kBlockH;
                if (x0 <= bx + kBlockW - 1 && x1 >= bx && y0 <= by + kBlockH - 1 && y1 >= by) m |= 1u << w;
            }
            sh.s0[h][tid] = make_float4(r.a.x, r.a.y, -0.5f * kLog2e * r.a.z, -kLog2e * r.a.w);
            sh.s1[h][tid] = make_float4(-0.5f * kLog2e * r.q.w, r.q.z, r.c.w, 0.0f);
            sh.s2[h][tid] = r.c;
            if (kMode == 1) sh.sid[h][tid] = r.s;
        }
        sh.mask[h][tid] = (uint8_t)m;
    };
    // the buffers may still be read by a previous call; leave when no pixel is open
    if (__syncthreads_count(px.done) == kT || start >= end) return;
    StagedRecord nxt;
    load_record(nxt, pval, rec, start + tid, end);
    stage(nxt, 0);
    load_record(nxt, pval, rec, start + kT + tid, end);
    __syncthreads();
    int h = 0;
    for (uint32_t base = start; base < end; base += kT, h ^= 1) {
        const int nb = (int)min((uint32_t)kT, end - base);
        for (int c = 0; c < nb; c += 32) {
            if (__all_sync(0xffffffffu, px.done)) break;
            const bool mine = (sh.mask[h][c + lane] & wbit) != 0 && c + lane < nb;
            uint32_t m = __ballot_sync(0xffffffffu, mine);
            while (m) {
                const int j = c + __ffs(m) - 1;
                m &= m - 1;
                if (px.done) continue;
                const float4 a = sh.s0[h][j];  // u, v, a', b'
                const float4 b = sh.s1[h][j];  // c', log2 o, radius
                const float dx = fpx - a.x, dy = fpy - a.y;
                if (fmaxf(fabsf(dx), fabsf(dy)) > b.z) continue;
                const float p = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
                if (p > 0.0f) continue;
                const float alpha = fminf(0.99f, ex2_approx(p + b.y));
                if (alpha < (1.0f / 255.0f)) continue;
                const float Tn = px.T * (1.0f - alpha);
                if (Tn < 1e-4f) {
                    px.done = true;
                    px.stopped = true;
                    continue;
                }
                const float4 col = sh.s2[h][j];
                const float wgt = alpha * px.T;
                if (kMode == 1) atomicAdd(contrib + sh.sid[h][j], wgt);
                if (kMode == 2) px.last = base + (uint32_t)j + 1u;
                px.r += col.x * wgt;
                px.g += col.y * wgt;
                px.b += col.z * wgt;
                px.T = Tn;
            }
        }
        // the other half was last read before the previous barrier: refill it
        // with the next batch (loaded while this one was composited) and
        // start loading the batch after
        if (base + kT < end) {
            stage(nxt, h ^ 1);
            load_record(nxt, pval, rec, base + 2 * kT + tid, end);
        }
        if (__syncthreads_count(px.done) == kT) break;
    }
}

struct TileGeom {
    int tx0, ty0, px, py;
    bool inside;
    float fpx, fpy;
};

// Pixel of the calling thread: warp w of the tile (w0 = the CTA's first)
// covers the 8x4 block at column w % 2, row w / 2.
__device__ __forceinline__ TileGeom tile_geom(int tile, int tiles_x, int W, int H, int ox, int oy, int w0 = 0) {
    TileGeom g;
    const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
    const int warp = w0 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    g.tx0 = txi * kTile;
    g.ty0 = tyi * kTile;
    g.px = g.tx0 + (warp & 1) * kBlockW + (lane & (kBlockW - 1));
    g.py = g.ty0 + (warp >> 1) * kBlockH + (lane / kBlockW);
    g.inside = g.px < W && g.py < H;
    g.fpx = (float)(g.px + ox) + 0.5f;
    g.fpy = (float)(g.py + oy) + 0.5f;
    return g;
}

// One CTA per tile: the first kBudget pairs of the tile (kMode 1,
// statistics: every pair in one pass).  kT threads per CTA: 256 cover a tile,
// 128 half a tile (two CTAs per tile, rows 0-7 and 8-15, each compositing
// the tile's list on its own, so the halves do not wait for each other).
template <int kMode, int kT>
__global__ void __launch_bounds__(kT) k_blend(int tiles_x, int W, int H, const uint2 *__restrict__ ranges,
                                              const uint32_t *__restrict__ pval, const float4 *__restrict__ rec,
                                              float4 *__restrict__ out, BlendWork work) {
    __shared__ BlendShared<kT> sh;
    constexpr int kParts = kBlendThreads / kT;
    const int tile = blockIdx.x / kParts, part = blockIdx.x % kParts;
    const int w0 = part * (kT / 32);  // first warp block of this CTA
    const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy, w0);
    uint2 rg = ranges[tile];
    if (!in_bounds(rg.x <= rg.y && rg.y <= work.n_pairs, kChkPair)) rg.y = rg.x;
    Pixel px{1.0f, 0.0f, 0.0f, 0.0f, rg.x, !g.inside, false};
    const uint32_t end1 = rg.y - rg.x > kBudget && kMode == 0 ? rg.x + kBudget : rg.y;
    composite_range<kMode, kT>(sh, rg.x, end1, pval, rec, g.tx0, g.ty0, g.fpx, g.fpy, px, work.contrib, w0 / 2);
    if (end1 < rg.y && in_bounds(work.cand_slot[tile] >= 0, kChkSlot)) {
        // pairs remain: record the pixel state for pass 2 and the merge (the
        // plan set cand_done to 1; every part clears it unless all its
        // pixels are done)
        const int slot = work.cand_slot[tile];
        const int all = __syncthreads_count(px.done) == kT;
        if (threadIdx.x == 0 && !all) atomicAnd(work.cand_done + slot, 0u);
        work.state[(size_t)slot * kBlendThreads + part * kT + threadIdx.x] =
            make_float4(px.r, px.g, px.b, px.done ? -px.T : px.T);
        if (!all) return;
    }
    if (g.inside) out[(size_t)g.py * W + g.px] = make_float4(px.r, px.g, px.b, 1.0f - px.T);
}

// ---------------------------------------------------------------------------
// Pass 1 of plain frames, pair-parallel.  A CTA of kPpWarps warps
// composites one 8x4 pixel block of a tile, one pixel per lane, in rounds
// of kPpRound pairs: warp k composites pairs
// [32 k, 32 k + 32) of the round for the block's pixels from T = 1 (a
// partial (C_k, T_k), no stop rule); warp 0 then chains the partials in
// depth order, C += T C_k, T *= T_k, and where T T_k would fall below the
// stop threshold it composites sub-range k again from the true T with the
// stop rule, so the stop rule holds exactly as in the sequential definition
// (only it needs the true T; the rest of the operator is associative).  A
// block's dependency chain is one round per kPpRound pairs, split over
// eight warps, instead of every pair in turn: a long list of large splats
// no longer leaves the GPU waiting on a single CTA.
//
// In frames with many busy tiles (blend_key), a tile whose list is shorter
// (below 2^(kPpTileClass - 1) pairs) is one item of its own instead: the CTA stages each batch of kPpRound pairs once
// for the whole tile, with the blocks each reach box meets as one bit mask
// per block, and warp w composites block w's pairs in depth order, as the
// definition reads.  Eight block items would stage every pair eight times
// and pay eight rounds of barriers and chaining; where lists are mid-length
// and many (a 4K frame of a large crowd) the pass is bound by instruction
// issue, and the tile items issue about a fifth fewer instructions there.
//
// Persistent CTAs take items in decreasing schedule key (blend_key: the
// list length class, raised for tile items), so the longest dependency
// chains start first; empty tiles (background) come last.
// ---------------------------------------------------------------------------
constexpr int kPpWarps = 8;
constexpr int kPpThreads = 32 * kPpWarps;
constexpr uint32_t kPpRound = 32 * kPpWarps;
constexpr int kPpBlocks = kTile * kTile / 32;  // 8x4 blocks per tile
constexpr int kPpTileClass = 14;               // lists of fewer than 8,192 pairs: tile items
static_assert((1u << (kPpTileClass - 1)) <= kBlendBudget, "a tile item composites its whole list");

struct PpShared {
    float4 s0[kPpWarps][32];  // u, v, a', b' (as staged by composite_range)
    float4 s1[kPpWarps][32];  // c', log2 o, radius, -
    float4 s2[kPpWarps][32];  // r, g, b, -
    float4 part[kPpWarps][32];
    uint32_t wm[kPpBlocks][kPpWarps];  // tile items: bit l of wm[b][k]: pair 32 k + l meets block b
    uint32_t m[kPpWarps];  // pairs of each sub-range whose reach box meets the block
    uint32_t done;         // pixels of the block that are done
    int tile, kind, blk;   // the current item: kind 0 empty tile, 1 tile item, 2 block item
    int seg_item[kBlendKeys + 1], seg_tile[kBlendKeys + 1];  // first item and tile of each key, decreasing key
};

// List length class of a tile: 0 empty, else 1 + floor(log2 n) (capped).
__device__ __forceinline__ int blend_class(uint32_t n) {
    return n == 0u ? 0 : 1 + min(kBlendClasses - 2, 31 - __clz((int)n));
}

// Schedule key of a tile in pass 1 (larger first), from its class c: 2c + 1
// for block items; for a tile item 2 (c + kPpTileShift), moved up because
// one warp composites each block's pairs in turn (a far longer dependency
// chain than a block item's for the same n, and a CTA held for the whole
// tile); 0 for an empty tile.  Longest chains first keeps the tail of the
// persistent grid short.  Tile items are used only in frames with at least
// kPpTileItemsPerCta busy tiles per persistent CTA: with fewer, block items
// keep more of the GPU busy and the frame is bound by its longest chains,
// not by instruction issue.  The shift, the threshold class and the busy
// tile count were chosen by timing the 1080p 3,500-instance frame (long
// lists), the 4K 10,000-instance frame (mostly mid-length lists) and
// 1280x720 frames of 1 to 5,000 characters.
constexpr int kPpTileShift = 4;
constexpr int kPpTileItemsPerCta = 8;
static_assert(2 * (kBlendClasses - 1) + 1 < kBlendKeys && 2 * (kPpTileClass - 1 + kPpTileShift) < kBlendKeys,
              "schedule keys");
__device__ __forceinline__ int blend_key(int c, bool tiles) {
    return c == 0 ? 0 : (tiles && c < kPpTileClass ? 2 * (c + kPpTileShift) : 2 * c + 1);
}

// Class of the tiles of schedule key k, or -1 when no class maps to it.
__device__ __forceinline__ int key_class(int k, bool tiles) {
    if (k == 0) return 0;
    if (k & 1) {
        const int c = (k - 1) >> 1;
        return c >= 1 && c < kBlendClasses && (!tiles || c >= kPpTileClass) ? c : -1;
    }
    const int c = (k >> 1) - kPpTileShift;
    return tiles && c >= 1 && c < kPpTileClass ? c : -1;
}

// Segments of the schedule in decreasing key, scanned by one warp (two keys
// per lane): segment s = key kBlendKeys - 1 - s starts at tile seg_tile[s]
// of pp_tile and at item seg_item[s] (kPpBlocks items per tile for odd keys,
// block items; one otherwise); entry kBlendKeys holds the totals.  Returns
// whether the frame uses tile items (the same answer in every CTA; forced
// by `items` unless CS_BLEND_ITEMS_AUTO).
static_assert(kBlendKeys == 64 && kBlendClasses <= 32, "one warp: two schedule keys, one class per lane");
__device__ __forceinline__ bool key_segments(const int32_t *__restrict__ meta, int ctas, int items, int *seg_item,
                                             int *seg_tile) {
    const int lane = threadIdx.x & 31, s0 = 2 * lane, k0 = kBlendKeys - 1 - s0, k1 = k0 - 1;
    int busy = lane >= 1 && lane < kBlendClasses ? meta[kBlendCountAt + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) busy += __shfl_xor_sync(0xffffffffu, busy, o);
    const bool tiles = items == CS_BLEND_ITEMS_TILES || (items == CS_BLEND_ITEMS_AUTO && busy >= kPpTileItemsPerCta * ctas);
    const int q0 = key_class(k0, tiles), q1 = key_class(k1, tiles);
    const int c0 = q0 >= 0 ? meta[kBlendCountAt + q0] : 0, c1 = q1 >= 0 ? meta[kBlendCountAt + q1] : 0;
    const int i0 = (k0 & 1) ? c0 * kPpBlocks : c0, i1 = (k1 & 1) ? c1 * kPpBlocks : c1;
    const int ii = (int)warp_inclusive_scan((uint32_t)(i0 + i1));
    const int it = (int)warp_inclusive_scan((uint32_t)(c0 + c1));
    if (seg_item) {
        seg_item[s0] = ii - i0 - i1;
        seg_item[s0 + 1] = ii - i1;
        if (lane == 31) seg_item[kBlendKeys] = ii;
    }
    seg_tile[s0] = it - c0 - c1;
    seg_tile[s0 + 1] = it - c1;
    if (lane == 31) seg_tile[kBlendKeys] = it;
    __syncwarp();
    return tiles;
}

// alpha of a staged splat at a pixel centre; 0 when the splat does not
// contribute there (outside its support box, q > 0, alpha < 1/255).  The
// same arithmetic as composite_range.  kBranchFree evaluates every test
// without branches: a splat that does not contribute then leaves T and C
// unchanged when composited with alpha = 0 (T (1 - 0) = T exactly), so the
// caller needs no test either.  That pays where the pairs of a sub-range
// are composited by many warps at once (no divergence); one warp walking a
// block's pairs in turn is faster skipping early.
template <bool kBranchFree>
__device__ __forceinline__ float staged_alpha(const float4 &a, const float4 &b, float fpx, float fpy) {
    const float dx = fpx - a.x, dy = fpy - a.y;
    if (kBranchFree) {
        const float p = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
        const float alpha = fminf(0.99f, ex2_approx(p + b.y));
        const bool skip = fmaxf(fabsf(dx), fabsf(dy)) > b.z || p > 0.0f || alpha < (1.0f / 255.0f);
        return skip ? 0.0f : alpha;
    }
    if (fmaxf(fabsf(dx), fabsf(dy)) > b.z) return 0.0f;
    const float p = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
    if (p > 0.0f) return 0.0f;
    const float alpha = fminf(0.99f, ex2_approx(p + b.y));
    return alpha < (1.0f / 255.0f) ? 0.0f : alpha;
}

__global__ void __launch_bounds__(kPpThreads, 8) k_blend_pp(int tiles_x, int W, int H, const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ pval,
                                                         const float4 *__restrict__ rec, float4 *__restrict__ out,
                                                         BlendWork work) {
    __shared__ PpShared sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // items in decreasing schedule key
    if (warp == 0) key_segments(work.meta, gridDim.x, work.items, sh.seg_item, sh.seg_tile);
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(reinterpret_cast<unsigned *>(work.meta + 3), 1u);
            int seg = 0;
            while (seg < kBlendKeys && item >= sh.seg_item[seg + 1]) ++seg;
            int tile = -1, kind = 0, blk = 0;
            if (seg < kBlendKeys) {
                const int key = kBlendKeys - 1 - seg, off = item - sh.seg_item[seg];
                const int per = (key & 1) ? kPpBlocks : 1;
                tile = work.pp_tile[sh.seg_tile[seg] + off / per];
                blk = off % per;
                kind = key == 0 ? 0 : ((key & 1) ? 2 : 1);
            }
            sh.tile = tile;
            sh.kind = kind;
            sh.blk = blk;
        }
        __syncthreads();
        const int tile = sh.tile, kind = sh.kind;
        if (tile < 0) return;
        if (!in_bounds(tile < tiles_x * ((H + kTile - 1) / kTile), kChkTile)) {
            __syncthreads();  // the item fields are rewritten for the next item
            continue;
        }
        if (kind != 2) {
            const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
            const int tx0 = txi * kTile, ty0 = tyi * kTile;
            if (kind == 0) {
                // a tile without pairs: background (C = 0, T = 1)
                for (int q = threadIdx.x; q < kTile * kTile; q += kPpThreads) {
                    const int x = tx0 + (q & (kTile - 1)), y = ty0 + q / kTile;
                    if (x < W && y < H) out[(size_t)y * W + x] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
                __syncthreads();  // the item fields are rewritten for the next item
                continue;
            }
            // a short list: the whole tile, warp w compositing block w
            const int px = tx0 + (warp & 1) * kBlockW + (lane & (kBlockW - 1));
            const int py = ty0 + (warp >> 1) * kBlockH + lane / kBlockW;
            const bool inside = px < W && py < H;
            const float fpx = (float)(px + work.ox) + 0.5f, fpy = (float)(py + work.oy) + 0.5f;
            uint2 rg = ranges[tile];
            if (!in_bounds(rg.x <= rg.y && rg.y <= work.n_pairs, kChkPair)) rg.y = rg.x;
            float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
            bool done = !inside;
            float4 *const f0 = &sh.s0[0][0], *const f1 = &sh.s1[0][0], *const f2 = &sh.s2[0][0];
            for (uint32_t base = rg.x; base < rg.y; base += kPpRound) {
                // stage pair base + tid with the blocks its reach box meets
                const uint32_t i = base + threadIdx.x;
                uint32_t bm = 0;
                if (i < rg.y) {
                    const uint32_t s = __ldg(pval + i);
                    const float4 *p = rec + (size_t)s * kRecVec;
                    const float4 rq = __ldg(p);  // reach x, reach y, log2 o, C
                    const uint32_t rx = __float_as_uint(rq.x), ry = __float_as_uint(rq.y);
                    const int x0 = (int)(rx & 0xFFFFu) - tx0, x1 = (int)(rx >> 16) - tx0;
                    const int y0 = (int)(ry & 0xFFFFu) - ty0, y1 = (int)(ry >> 16) - ty0;
#pragma unroll
                    for (int b = 0; b < kPpBlocks; ++b) {
                        const int bx = (b & 1) * kBlockW, by = (b >> 1) * kBlockH;
                        if (x0 <= bx + kBlockW - 1 && x1 >= bx && y0 <= by + kBlockH - 1 && y1 >= by) bm |= 1u << b;
                    }
                    if (bm) {
                        const float4 ra = __ldg(p + 1), rc = __ldg(p + 2);
                        f0[threadIdx.x] = make_float4(ra.x, ra.y, -0.5f * kLog2e * ra.z, -kLog2e * ra.w);
                        f1[threadIdx.x] = make_float4(-0.5f * kLog2e * rq.w, rq.z, rc.w, 0.0f);
                        f2[threadIdx.x] = rc;
                    }
                }
#pragma unroll
                for (int b = 0; b < kPpBlocks; ++b) {
                    const uint32_t word = __ballot_sync(0xffffffffu, (bm >> b) & 1u);
                    if (lane == 0) sh.wm[b][warp] = word;
                }
                __syncthreads();
                for (int k = 0; k < kPpWarps && !done; ++k) {
                    uint32_t m = sh.wm[warp][k];
                    while (m) {
                        const int j = 32 * k + __ffs(m) - 1;
                        m &= m - 1;
                        const float alpha = staged_alpha<false>(f0[j], f1[j], fpx, fpy);
                        if (alpha == 0.0f) continue;
                        const float Tn = T * (1.0f - alpha);
                        if (Tn < 1e-4f) {
                            done = true;
                            break;
                        }
                        const float4 col = f2[j];
                        const float wgt = alpha * T;
                        cr += col.x * wgt;
                        cg += col.y * wgt;
                        cb += col.z * wgt;
                        T = Tn;
                    }
                }
                // the staging buffers are refilled by the next batch
                if (__syncthreads_count(done) == kPpThreads) break;
            }
            if (inside) out[(size_t)py * W + px] = make_float4(cr, cg, cb, 1.0f - T);
            continue;  // the loop's barriers keep the item fields until every thread has read them
        }
        const int blk = sh.blk;
        const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
        const int bx0 = txi * kTile + (blk & 1) * kBlockW, by0 = tyi * kTile + (blk >> 1) * kBlockH;
        const int px = bx0 + (lane & (kBlockW - 1)), py = by0 + lane / kBlockW;
        const bool inside = px < W && py < H;
        const float fpx = (float)(px + work.ox) + 0.5f, fpy = (float)(py + work.oy) + 0.5f;
        uint2 rg = ranges[tile];
        if (!in_bounds(rg.x <= rg.y && rg.y <= work.n_pairs, kChkPair)) rg.y = rg.x;
        const uint32_t end1 = rg.y - rg.x > kBudget ? rg.x + kBudget : rg.y;
        // the block's chained state (warp 0)
        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        bool done = !inside;
        if (warp == 0) {
            const uint32_t dm = __ballot_sync(0xffffffffu, done);
            if (lane == 0) sh.done = dm;
        }
        __syncthreads();
        for (uint32_t base = rg.x; base < end1; base += kPpRound) {
            const uint32_t dmask = sh.done;
            if (dmask == 0xffffffffu) break;
            // stage this warp's sub-range
            const uint32_t i = base + (uint32_t)warp * 32u + (uint32_t)lane;
            bool mine = false;
            if (i < end1) {
                const uint32_t s = __ldg(pval + i);
                const float4 *p = rec + (size_t)s * kRecVec;
                // the reach box first: the rest of the record only for
                // splats whose reach box meets this block
                const float4 rq = __ldg(p);  // reach x, reach y, log2 o, C
                const uint32_t rx = __float_as_uint(rq.x), ry = __float_as_uint(rq.y);
                mine = (int)(rx & 0xFFFFu) <= bx0 + kBlockW - 1 && (int)(rx >> 16) >= bx0 &&
                       (int)(ry & 0xFFFFu) <= by0 + kBlockH - 1 && (int)(ry >> 16) >= by0;
                if (mine) {
                    const float4 ra = __ldg(p + 1), rc = __ldg(p + 2);
                    sh.s0[warp][lane] = make_float4(ra.x, ra.y, -0.5f * kLog2e * ra.z, -kLog2e * ra.w);
                    sh.s1[warp][lane] = make_float4(-0.5f * kLog2e * rq.w, rq.z, rc.w, 0.0f);
                    sh.s2[warp][lane] = rc;
                }
            }
            uint32_t m = __ballot_sync(0xffffffffu, mine);
            if (lane == 0) sh.m[warp] = m;
            __syncwarp();
            // the sub-range's partial composite from T = 1
            float Tk = 1.0f, kr = 0.0f, kg = 0.0f, kb = 0.0f;
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                // a done pixel's partial is computed and left unused
                const float alpha = staged_alpha<true>(sh.s0[warp][j], sh.s1[warp][j], fpx, fpy);
                const float4 col = sh.s2[warp][j];
                const float wgt = alpha * Tk;
                kr += col.x * wgt;
                kg += col.y * wgt;
                kb += col.z * wgt;
                Tk *= 1.0f - alpha;
            }
            sh.part[warp][lane] = make_float4(kr, kg, kb, Tk);
            __syncthreads();
            // chain the partials in depth order
            if (warp == 0) {
                for (int k = 0; k < kPpWarps && !done;) {
                    // the first sub-range from k in which the stop rule can
                    // fall (its transmittances read at once), then the ones
                    // before it applied as wholes, in order
                    float Tq[kPpWarps];
#pragma unroll
                    for (int i = 0; i < kPpWarps; ++i) Tq[i] = i >= k ? sh.part[i][lane].w : 1.0f;
                    int ks = kPpWarps;
                    float Tb = T;
#pragma unroll
                    for (int i = 0; i < kPpWarps; ++i) {
                        if (i < k || ks < kPpWarps) continue;
                        if (Tb * Tq[i] < 1e-4f) ks = i;
                        else Tb *= Tq[i];
                    }
#pragma unroll
                    for (int i = 0; i < kPpWarps; ++i) {
                        if (i < k || i >= ks) continue;
                        // no splat of the sub-range meets the stop rule from this T
                        const float4 q = sh.part[i][lane];
                        cr += T * q.x;
                        cg += T * q.y;
                        cb += T * q.z;
                        T *= q.w;
                    }
                    if (ks == kPpWarps) break;
                    k = ks + 1;
                    // the stop falls inside sub-range ks: composite it from the true T
                    uint32_t mk = sh.m[ks];
                    while (mk) {
                        const int j = __ffs(mk) - 1;
                        mk &= mk - 1;
                        const float alpha = staged_alpha<true>(sh.s0[ks][j], sh.s1[ks][j], fpx, fpy);
                        const float Tn = T * (1.0f - alpha);
                        if (Tn < 1e-4f) {
                            done = true;
                            break;
                        }
                        const float4 col = sh.s2[ks][j];
                        const float wgt = alpha * T;
                        cr += col.x * wgt;
                        cg += col.y * wgt;
                        cb += col.z * wgt;
                        T = Tn;
                    }
                }
                const uint32_t dm = __ballot_sync(0xffffffffu, done);
                if (lane == 0) sh.done = dm;
            }
            __syncthreads();
        }
        if (warp == 0) {
            bool final_out = true;
            const int slot = end1 < rg.y ? work.cand_slot[tile] : -1;
            if (end1 < rg.y && in_bounds(slot >= 0, kChkSlot)) {
                // pairs remain: the state for pass 2 and the merge, as pass 1 records it
                const bool all = __all_sync(0xffffffffu, done);
                if (lane == 0 && !all) atomicAnd(work.cand_done + slot, 0u);
                work.state[(size_t)slot * kBlendThreads + blk * 32 + lane] = make_float4(cr, cg, cb, done ? -T : T);
                final_out = all;
            }
            if (final_out && inside) out[(size_t)py * W + px] = make_float4(cr, cg, cb, 1.0f - T);
        }
        __syncthreads();  // the item fields and the staging buffers are reused by the next item
    }
}

// Pass 2: chunk c of a tile's remaining pairs, from T = 1, for the pixels
// pass 1 left open.  Writes (r, g, b, T) with T negated when the chunk met
// the stop rule.
__global__ void __launch_bounds__(kBlendThreads) k_blend_chunks(int tiles_x, int W, int H,
                                                                const uint2 *__restrict__ ranges,
                                                                const uint32_t *__restrict__ pval,
                                                                const float4 *__restrict__ rec,
                                                                BlendWork work) {
    __shared__ BlendShared<> sh;
    // chunk w of the frame, grid-stride (the grid is capped, not sized for
    // the worst case)
    for (uint32_t w = blockIdx.x; w < (uint32_t)work.meta[1]; w += gridDim.x) {
        const int slot = work.chunk_slot[w];
        if (work.cand_done[slot]) continue;
        const int tile = work.cand_tile[slot];
        const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
        const uint2 rg = ranges[tile];
        if (!in_bounds(rg.y <= work.n_pairs, kChkPair)) continue;
        const uint32_t c = w - work.cand_chunk0[slot];
        const uint32_t start = rg.x + kBudget + c * kChunk;
        const uint32_t end = min(rg.y, start + kChunk);
        const float4 s1 = work.state[(size_t)slot * kBlendThreads + threadIdx.x];
        Pixel px{1.0f, 0.0f, 0.0f, 0.0f, 0u, !g.inside || s1.w < 0.0f, false};
        composite_range(sh, start, end, pval, rec, g.tx0, g.ty0, g.fpx, g.fpy, px);
        work.part[(size_t)w * kBlendThreads + threadIdx.x] = make_float4(px.r, px.g, px.b, px.stopped ? -px.T : px.T);
        __syncthreads();  // the staging buffers are reused by the next chunk
    }
}

// Merge: pass-1 state then the chunks in depth order, per pixel, up to the
// chunk in which the pixel meets the stop rule: such pixels keep their
// state before that chunk (in work.state) and its index (work.stop) for the
// fix-up pass; the others are final.
__global__ void __launch_bounds__(kBlendThreads) k_blend_merge(int tiles_x, int W, int H,
                                                               const uint2 *__restrict__ ranges,
                                                               float4 *__restrict__ out, BlendWork work) {
    const int slot = blockIdx.x;
    if (slot >= work.meta[0] || work.cand_done[slot]) return;
    const int tile = work.cand_tile[slot];
    const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
    const size_t pix = (size_t)slot * kBlendThreads + threadIdx.x;
    const float4 s1 = work.state[pix];
    float T = fabsf(s1.w), r = s1.x, gg = s1.y, b = s1.z;
    bool done = !g.inside || s1.w < 0.0f;
    int32_t stop = -1;
    const uint2 rg = ranges[tile];
    const uint32_t c0 = work.cand_chunk0[slot], c1 = c0 + (rg.y - rg.x - kBudget + kChunk - 1) / kChunk;
    // four chunks' partials loaded at a time (independent loads), applied in order
    for (uint32_t w0 = c0; w0 < c1 && !done; w0 += 4) {
        float4 pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            pk[i] = w0 + i < c1 ? work.part[(size_t)(w0 + i) * kBlendThreads + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 1.f);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (done || w0 + i >= c1) break;
            const float Tk = fabsf(pk[i].w);
            if (T * Tk >= 1e-4f) {
                // no splat of the chunk reaches the stop rule from this T: the
                // chunk's composite applies as a whole
                r += T * pk[i].x;
                gg += T * pk[i].y;
                b += T * pk[i].z;
                T *= Tk;
                done = pk[i].w < 0.0f;
            } else {
                stop = (int32_t)(w0 + i);
                done = true;
            }
        }
    }
    work.stop[pix] = stop;
    if (stop >= 0) work.state[pix] = make_float4(r, gg, b, T);
    else if (g.inside) out[(size_t)g.py * W + g.px] = make_float4(r, gg, b, 1.0f - T);
}

// Fix-up: chunk w composited again, from their true transmittance, for the
// pixels that meet the stop rule inside it.
__global__ void __launch_bounds__(kBlendThreads) k_blend_fix(int tiles_x, int W, int H,
                                                             const uint2 *__restrict__ ranges,
                                                             const uint32_t *__restrict__ pval,
                                                             const float4 *__restrict__ rec,
                                                             float4 *__restrict__ out, BlendWork work) {
    __shared__ BlendShared<> sh;
    for (uint32_t w = blockIdx.x; w < (uint32_t)work.meta[1]; w += gridDim.x) {
        const int slot = work.chunk_slot[w];
        if (work.cand_done[slot]) continue;
        const size_t pix = (size_t)slot * kBlendThreads + threadIdx.x;
        const bool mine = work.stop[pix] == (int32_t)w;
        if (__syncthreads_count(mine) == 0) continue;
        const int tile = work.cand_tile[slot];
        const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
        const uint2 rg = ranges[tile];
        if (!in_bounds(rg.y <= work.n_pairs, kChkPair)) continue;
        const float4 sb = mine ? work.state[pix] : make_float4(0.f, 0.f, 0.f, 1.f);
        Pixel px{sb.w, sb.x, sb.y, sb.z, 0u, !mine, false};
        const uint32_t start = rg.x + kBudget + (w - work.cand_chunk0[slot]) * kChunk;
        composite_range(sh, start, min(rg.y, start + kChunk), pval, rec, g.tx0, g.ty0, g.fpx, g.fpy, px);
        if (mine && g.inside) out[(size_t)g.py * W + g.px] = make_float4(px.r, px.g, px.b, 1.0f - px.T);
        __syncthreads();  // the staging buffers are reused by the next chunk
    }
}

// ---------------------------------------------------------------------------
// Training frames: every tile's list in chunks of kBwdChunk pairs composited
// in parallel, as the split passes of plain frames do (the operator is
// associative), and per pixel the state at each chunk boundary, the end of
// its composited list and its final state for the backward.
//   k_train_counts   chunks per tile (then an exclusive scan numbers them)
//   k_train_chunks   CTA per chunk: its composite from T = 1 for every pixel
//                    of the tile, and one past its last composited pair
//   k_train_merge    CTA per tile: per pixel, the chunks in order, C += T C_k,
//                    T *= T_k, keeping the state before every chunk; up to the
//                    chunk in which T T_k would fall below the stop threshold
//                    (or whose partial met it from T = 1)
//   k_train_fix      CTA per chunk: that chunk again from the pixel's true
//                    state with the stop rule, for the pixels stopping in it
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_train_counts(int n_tiles, const uint2 *__restrict__ ranges,
                                                      uint32_t *__restrict__ cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) cnt[t] = (ranges[t].y - ranges[t].x + kBwdChunk - 1) / kBwdChunk;
}

// tile of chunk w: the last t with chunk0[t] <= w (thread 0, broadcast)
__device__ __forceinline__ int chunk_tile(const uint32_t *__restrict__ chunk0, int n_tiles, uint32_t w, int *s_tile) {
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_tiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (chunk0[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        *s_tile = lo;
    }
    __syncthreads();
    return *s_tile;
}

__global__ void __launch_bounds__(kBlendThreads) k_train_chunks(int tiles_x, int W, int H,
                                                                const uint2 *__restrict__ ranges,
                                                                const uint32_t *__restrict__ pval,
                                                                const float4 *__restrict__ rec, BlendWork work) {
    __shared__ BlendShared<> sh;
    __shared__ int s_tile;
    const int n_tiles = tiles_x * ((H + kTile - 1) / kTile);
    const uint32_t w = blockIdx.x;
    if (w >= work.t_chunk0[n_tiles]) return;
    const int tile = chunk_tile(work.t_chunk0, n_tiles, w, &s_tile);
    const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
    const uint2 rg = ranges[tile];
    const uint32_t a = rg.x + (w - work.t_chunk0[tile]) * kBwdChunk, b = min(rg.y, a + kBwdChunk);
    Pixel px{1.0f, 0.0f, 0.0f, 0.0f, 0u, !g.inside, false};
    composite_range<2>(sh, a, b, pval, rec, g.tx0, g.ty0, g.fpx, g.fpy, px);
    work.t_part[(size_t)w * kBlendThreads + threadIdx.x] = make_float4(px.r, px.g, px.b, px.stopped ? -px.T : px.T);
    work.t_last[(size_t)w * kBlendThreads + threadIdx.x] = px.last;
}

__global__ void __launch_bounds__(kBlendThreads) k_train_merge(int tiles_x, int W, int H,
                                                               const uint2 *__restrict__ ranges,
                                                               float4 *__restrict__ out, BlendWork work) {
    const int tile = blockIdx.x;
    const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
    if (!g.inside) return;
    const size_t pix = (size_t)g.py * W + g.px;
    const uint2 rg = ranges[tile];
    float T = 1.0f, r = 0.0f, gg = 0.0f, b = 0.0f;
    uint32_t last = rg.x;
    int32_t stop = -1;
    const uint32_t c0 = work.t_chunk0[tile], c1 = work.t_chunk0[tile + 1];
    for (uint32_t w = c0; w < c1; ++w) {
        if (w > c0) {
            // the state before pair a of chunk w, for the backward
            const uint32_t a = rg.x + (w - c0) * kBwdChunk;
            work.px_bnd[(size_t)(a / kBwdChunk) * kBlendThreads + threadIdx.x] = make_float4(r, gg, b, T);
        }
        const float4 p = work.t_part[(size_t)w * kBlendThreads + threadIdx.x];
        const float Tk = fabsf(p.w);
        if (p.w >= 0.0f && T * Tk >= 1e-4f) {
            // no splat of the chunk meets the stop rule from this T: it applies as a whole
            r += T * p.x;
            gg += T * p.y;
            b += T * p.z;
            T *= Tk;
            const uint32_t lk = work.t_last[(size_t)w * kBlendThreads + threadIdx.x];
            if (lk) last = lk;
        } else {
            stop = (int32_t)w;
            break;
        }
    }
    work.t_stop[pix] = stop;
    if (stop >= 0) {
        work.t_state[pix] = make_float4(r, gg, b, T);
        work.t_slast[pix] = last;
    } else {
        out[pix] = make_float4(r, gg, b, 1.0f - T);
        work.px_end[pix] = last;
        work.px_fin[pix] = make_float4(r, gg, b, T);
    }
}

__global__ void __launch_bounds__(kBlendThreads) k_train_fix(int tiles_x, int W, int H,
                                                             const uint2 *__restrict__ ranges,
                                                             const uint32_t *__restrict__ pval,
                                                             const float4 *__restrict__ rec,
                                                             float4 *__restrict__ out, BlendWork work) {
    __shared__ BlendShared<> sh;
    __shared__ int s_tile;
    const int n_tiles = tiles_x * ((H + kTile - 1) / kTile);
    const uint32_t w = blockIdx.x;
    if (w >= work.t_chunk0[n_tiles]) return;
    const int tile = chunk_tile(work.t_chunk0, n_tiles, w, &s_tile);
    const TileGeom g = tile_geom(tile, tiles_x, W, H, work.ox, work.oy);
    const size_t pix = (size_t)g.py * W + g.px;
    const bool mine = g.inside && work.t_stop[pix] == (int32_t)w;
    if (__syncthreads_count(mine) == 0) return;
    const uint2 rg = ranges[tile];
    const uint32_t a = rg.x + (w - work.t_chunk0[tile]) * kBwdChunk, b = min(rg.y, a + kBwdChunk);
    const float4 sb = mine ? work.t_state[pix] : make_float4(0.f, 0.f, 0.f, 1.f);
    Pixel px{sb.w, sb.x, sb.y, sb.z, mine ? work.t_slast[pix] : 0u, !mine, false};
    composite_range<2>(sh, a, b, pval, rec, g.tx0, g.ty0, g.fpx, g.fpy, px);
    if (mine) {
        out[pix] = make_float4(px.r, px.g, px.b, 1.0f - px.T);
        work.px_end[pix] = px.last;
        work.px_fin[pix] = make_float4(px.r, px.g, px.b, px.T);
    }
}

// Plan, part 1 (one thread per tile; meta zeroed before): tiles per list
// length class (warp-aggregated atomics), and a slot plus
// ceil((n - kBudget) / kChunk) consecutive chunks for every tile with more
// than kBudget pairs.  Slot and chunk numbers depend on the order of the
// atomics; no result does (a tile's chunks are consecutive and merged in
// order).
__global__ void __launch_bounds__(256) k_blend_count(int n_tiles, const uint2 *__restrict__ ranges, BlendWork work) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const uint32_t n = t < n_tiles ? ranges[t].y - ranges[t].x : 0u;
    const int cls = t < n_tiles ? blend_class(n) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, cls);
    if (cls >= 0 && lane == __ffs(peers) - 1) atomicAdd(work.meta + kBlendCountAt + cls, __popc(peers));
    if (t >= n_tiles) return;
    int slot = -1;
    if (n > kBudget) {
        const uint32_t nk = (n - kBudget + kChunk - 1) / kChunk;
        slot = atomicAdd(work.meta + 0, 1);
        const uint32_t c0 = atomicAdd(reinterpret_cast<unsigned *>(work.meta + 1), nk);
        if (in_bounds((uint32_t)slot < work.max_slots && c0 + nk <= work.max_chunks, kChkSlot)) {
            work.cand_tile[slot] = t;
            work.cand_chunk0[slot] = c0;
            work.cand_done[slot] = 1u;  // cleared by pass 1 unless every pixel is done
            for (uint32_t c = 0; c < nk; ++c) work.chunk_slot[c0 + c] = slot;
        } else {
            slot = -1;
        }
    }
    work.cand_slot[t] = slot;
}

// Plan, part 2: pp_tile in decreasing schedule key (the order inside a key
// is that of the atomics and affects no result).
__global__ void __launch_bounds__(256) k_blend_order(int n_tiles, const uint2 *__restrict__ ranges, int pp_ctas,
                                                     BlendWork work) {
    __shared__ int seg_tile[kBlendKeys + 1];  // first tile of key kBlendKeys - 1 - s
    __shared__ bool tiles;
    if (threadIdx.x < 32) {
        const bool t_ = key_segments(work.meta, pp_ctas, work.items, nullptr, seg_tile);
        if (threadIdx.x == 0) tiles = t_;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const int cls = t < n_tiles ? blend_class(ranges[t].y - ranges[t].x) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, cls);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (cls >= 0 && lane == leader) pos = atomicAdd(work.meta + kBlendCursorAt + cls, __popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & ((1u << lane) - 1u));
    if (cls >= 0) work.pp_tile[seg_tile[kBlendKeys - 1 - blend_key(cls, tiles)] + pos] = t;
}

// Persistent grid of the pair-parallel pass: as many CTAs as fit on the
// device at once.
static unsigned pp_grid() {
    static int cached_device = -1;
    static unsigned grid = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_device) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_pp, kPpThreads, 0);
        grid = (unsigned)std::max(1, sms * std::max(1, per_sm));
        cached_device = dev;
    }
    return grid;
}

int launch_blend(int tiles_x, int tiles_y, int W, int H, const uint2 *ranges, const uint32_t *pval,
                 const float4 *rec, float4 *out, const BlendWork &work, uint32_t n_pairs, cudaStream_t st) {
    const int n = tiles_x * tiles_y;
    if (n <= 0) return 0;
    const size_t max_cand = blend_max_slots((size_t)n, n_pairs);
    const size_t max_chunks = blend_max_chunks((size_t)n, n_pairs);
    if (work.contrib) {
        // statistics: every list composited in one pass
        k_blend<1, kBlendThreads><<<n, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, out, work);
        return 1;
    }
    if (work.px_end) {
        // training forward: every list in parallel chunks, per-pixel state
        // for the backward
        k_train_counts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ranges, work.t_cnt);
        const int sc = exclusive_scan(work.t_cnt, nullptr, work.t_chunk0, (uint32_t)n, work.t_scan, st);
        const unsigned grid = (unsigned)train_max_chunks((size_t)n, n_pairs);
        k_train_chunks<<<grid, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, work);
        k_train_merge<<<n, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, out, work);
        k_train_fix<<<grid, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, out, work);
        return 4 + sc;
    }
    const unsigned tb = (unsigned)((n + 255) / 256);
    if (cudaMemsetAsync(work.meta, 0, kBlendMetaWords * sizeof(int32_t), st) != cudaSuccess) return -1;
    k_blend_count<<<tb, 256, 0, st>>>(n, ranges, work);
    const unsigned grid = pp_grid();
    k_blend_order<<<tb, 256, 0, st>>>(n, ranges, (int)grid, work);
    // pass 1 of every tile: persistent CTAs, longest chains first
    k_blend_pp<<<grid, kPpThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, out, work);
    const int launched = 3;
    // no tile has pairs left after pass 1
    if (n_pairs <= kBudget) return launched;
    // chunk grids capped at kChunkGrid CTAs (grid-stride over the frame's
    // chunks): a frame whose lists all end within the pass-1 budget does not
    // pay for a worst-case grid of CTAs that return at once
    const unsigned chunk_grid = (unsigned)std::min<size_t>(max_chunks, kChunkGrid);
    k_blend_chunks<<<chunk_grid, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, work);
    k_blend_merge<<<(unsigned)max_cand, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, out, work);
    k_blend_fix<<<chunk_grid, kBlendThreads, 0, st>>>(tiles_x, W, H, ranges, pval, rec, out, work);
    return launched + 3;
}

CS_DEFINE_CHECK_READER(check_word_blend)

}  // namespace cs
