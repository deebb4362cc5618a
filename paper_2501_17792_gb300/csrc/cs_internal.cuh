// cs_internal.cuh -- shared declarations of the CrowdSplat CUDA library
// (device data layout, per-frame parameters, kernel launchers).
//
// Device data layout (structure of arrays, one allocation per array, all
// templates concatenated; g = global template-Gaussian index):
//   mean_op[g]  float4 (x, y, z, opacity)          template local frame
//   cov_a[g]    float4 (xx, xy, xz, yy)            canonical covariance R S S^T R^T
//   cov_b[g]    float2 (yz, zz)                    at scale multiplier 1
//   skin_w[g]   float4 top-4 skinning weights
//   skin_i[g]   uint32 four joint ids, one byte each (little end = first)
//   sh          float4 planes: plane p of Gaussian k of template t at
//               sh[t.sh_off + p * t.n + k]; plane p holds the flat SH
//               coefficients 4p..4p+3 of that Gaussian (flat = k*3 + channel)
// With BF16 storage (TemplateArrays::storage) the same attributes sit in
// two 16-byte words per Gaussian (qa, qb) and FP16 SH planes of 8.
// Per instance: B[i][24][12] instance-local skinning transforms (root not
// applied), V[i][12] = camera o root (3x4), C[i][4] = camera centre in the
// instance root frame.
// Per splat s (Gaussian-instance of a visible instance, dense ids grouped by
// (template, level)): a 48-byte record rec[3s..3s+2] float4 = {reach x,
// reach y, log2 opacity, C}, {u, v, A, B}, {r, g, b, radius} where reach x/y
// hold the inclusive pixel range (lo | hi << 16, as float bits) in which
// alpha can reach 1/255 (see splat_reach_box); the compositing reads the
// first word alone to test a splat against a pixel block;
// key[s] depth bits (0xFFFFFFFF culled); rect[s] tile rectangle of the
// support box (x0 | y0 << 16, x1 | y1 << 16), inclusive; bin[s] the tiles
// holding a pixel the compositing uses (the pairs of the splat), as a bin
// word: small splats (reach box within a 3x3 tile window) store the
// window's tile origin and a 9-bit mask, x0 | y0 << 8 | mask << 16; larger
// ones store kBinLarge | count and are re-tested from their record.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cs {

// Debug build with bounds checks (nvcc -DCS_CHECKS=1; build.build(checks=
// True) makes libcrowdsplat_checks.so): an index that a checked access would
// take outside its buffer sets one bit of the translation unit's check word
// and the access is skipped, so the fault is reported (cs_debug_checks)
// instead of reading or writing out of bounds.  The release build compiles
// every check away.
#ifndef CS_CHECKS
#define CS_CHECKS 0
#endif
constexpr uint32_t kChkRecord = 1u;  // splat record, depth key or bin word index >= splats of the frame
constexpr uint32_t kChkPair = 2u;    // pair index >= pairs of the frame
constexpr uint32_t kChkTile = 4u;    // tile index >= tiles of the frame
constexpr uint32_t kChkSplat = 8u;   // splat id written into the pair list >= splats
constexpr uint32_t kChkSort = 16u;   // radix scatter position or gathered index >= elements
constexpr uint32_t kChkSlot = 32u;   // compositing slot or chunk beyond the planned capacity
#if CS_CHECKS
static __device__ uint32_t g_check_word;
__device__ __forceinline__ bool in_bounds(bool ok, uint32_t bit) {
    if (!ok) atomicOr(&g_check_word, bit);
    return ok;
}
// reads and clears this translation unit's check word (synchronous)
#define CS_DEFINE_CHECK_READER(fn)                                  \
    uint32_t fn() {                                                 \
        uint32_t v = 0u, z = 0u;                                    \
        if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu; \
        cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));            \
        return v;                                                   \
    }
#else
__device__ __forceinline__ bool in_bounds(bool, uint32_t) { return true; }
#define CS_DEFINE_CHECK_READER(fn) \
    uint32_t fn() { return 0u; }
#endif
uint32_t check_word_geometry();
uint32_t check_word_sort();
uint32_t check_word_blend();

constexpr int kJoints = 24;
constexpr int kMaxTemplates = 63;
constexpr int kMaxLevels = 4;
constexpr int kTile = 16;
constexpr int kRecVec = 3;  // float4 per splat record (48 bytes)
constexpr uint32_t kBinLarge = 0x80000000u;

// number of pairs (tiles) described by a bin word
__host__ __device__ __forceinline__ uint32_t bin_count(uint32_t b) {
#ifdef __CUDA_ARCH__
    return (b & kBinLarge) ? (b & ~kBinLarge) : (uint32_t)__popc((b >> 16) & 0x1FFu);
#else
    return (b & kBinLarge) ? (b & ~kBinLarge) : (uint32_t)__builtin_popcount((b >> 16) & 0x1FFu);
#endif
}

struct TemplateInfo {
    int32_t g_off;      // first global Gaussian index
    int32_t n;          // Gaussians
    int32_t sh_deg;     // 0..3
    int32_t sh_planes;  // float4 planes per Gaussian
    int64_t sh_off;     // offset of SH plane 0 (float4 planes, or uint4 FP16 planes with BF16 storage)
    int32_t n_level[kMaxLevels];   // Gaussians rendered at each level
    float reach[kMaxLevels];       // bound of |posed local mean - pelvis rest| per level
    float sigma_max[kMaxLevels];   // largest scale x level multiplier per level
    float rest[kJoints * 3];
    int8_t parent[kJoints];
    int8_t depth[kJoints];         // depth in the kinematic tree (root 0)
    int32_t max_depth;
    int32_t lod_idx_off[kMaxLevels];  // level's Gaussian subset in lod_idx, -1: the first n_level
};

struct Group {         // visible instances of one (template, level)
    int32_t tpl, lvl;
    int32_t slot0;     // first slot in the visible list
    int32_t nslots;
    int32_t ng;        // Gaussians per instance (template size at level)
    int32_t splat0;    // first splat id
    int32_t block0;    // first projection CTA (each CTA: 256 Gaussians of one instance)
};

// A group as the projection reads it: the Group fields and those of its
// template (level subset offset, Gaussian and SH offsets, sizes).  The host
// passes all groups of a frame as one kernel parameter (constant bank), so
// every thread reads them through the constant cache.
struct ProjGroup {
    int32_t tpl, lvl, slot0, ng, splat0, block0;
    int32_t g_off, n, sh_deg, sub;  // sub: level subset offset in lod_idx, -1 for a prefix
    int64_t sh_off;
};
constexpr int kMaxGroups = kMaxTemplates * kMaxLevels;
struct ProjGroups {
    ProjGroup g[kMaxGroups];
};

struct CamParams {
    float R[9], t[3];
    float fx, fy, cx, cy;  // of the full image
    int32_t W, H;          // of the rendered window
    int32_t ox, oy;        // window origin in the full image (multiples of the tile size)
    float near_z;
    float center[3];       // camera centre in world coordinates
    float limx, limy;      // EWA clamp of x/z, y/z (1.3 x half field of view)
    int32_t tiles_x, tiles_y;
    float plane[4][4];     // conservative frustum side planes (camera space, unit normals)
    float cull_sigma_k;    // instance cull: 3D growth per unit of Gaussian scale
    // depth keys: float bits of the view depth clamped to [key_lo, key_hi]
    // (bits of bounds of every live depth), minus key_lo; culled = all ones
    uint32_t key_lo, key_hi;
    uint32_t n_splats;     // splats of the frame (bounds of the checked debug build)
};

// Bits of the depth keys of a frame whose live depths lie in float-bit range
// [lo, hi]: live keys are at most hi - lo, the culled key (all ones in these
// bits) must exceed them.
inline int depth_key_bits(uint32_t lo, uint32_t hi) {
    const uint64_t span = (uint64_t)(hi - lo) + 2u;  // live keys 0 .. hi - lo, then the culled key
    int b = 1;
    while (b < 32 && (1ull << b) < span) ++b;
    return b;
}

struct LodParams {
    int32_t n_levels;
    float thresh[kMaxLevels - 1];
    float mult[kMaxLevels];
};

constexpr int kStoreFp32 = 0, kStoreBf16 = 1;  // CS_STORE_FP32 / CS_STORE_BF16

struct TemplateArrays {
    // FP32 storage (CS_STORE_FP32)
    const float4 *mean_op;
    const float4 *cov_a;
    const float2 *cov_b;
    const float4 *skin_w;
    const uint32_t *skin_i;
    const float4 *sh;         // planes of 4 coefficients, TemplateInfo sh_off / sh_planes
    const uint32_t *lod_idx;  // template-local Gaussian indices of subset levels
    // BF16 storage (CS_STORE_BF16): two 16-byte words per Gaussian
    //   qa = bf16 {dx, dy, dz, opacity, cxx, cxy, cxz, cyy}, (dx, dy, dz) the
    //        mean minus the rest position of the Gaussian's first skinning joint
    //   qb = bf16 {cyz, czz, w0, w1, w2, w3}, then the four joint ids (bytes)
    // and FP16 SH planes of 8 coefficients (sh_off / sh_planes count these)
    const uint4 *qa;
    const uint4 *qb;
    const uint4 *sh16;
    int storage;  // CS_STORE_FP32 or CS_STORE_BF16
    // scales (x, y, z, 0) and quaternions (w, x, y, z) as uploaded (FP32
    // storage; read by the backward only)
    const float4 *scale;
    const float4 *quat;
};

// BF16 halves of a 32-bit word, widened exactly to FP32
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// ---------------------------------------------------------------------------
// Reach of a splat: where it can contribute.
//
// A splat contributes to a pixel only where alpha = o e^q >= 1/255, i.e. where
// f(d) = A dx^2 + 2 B dx dy + C dy^2 <= fcut = 2 ln(255 o) (d = pixel centre -
// splat centre, conic (A, B, C)).  The axis-aligned extent of that ellipse,
// widened by kAlphaMargin in the exponent (FP32 rounding) and clipped to the
// support box, is the splat's reach box; binning keeps every tile the reach
// box meets, and the compositing's warp masks test the reach box against
// each 8x4 pixel block.  A tile or block outside it holds no pixel the
// compositing would use, so skipping it leaves every pixel unchanged.
// ---------------------------------------------------------------------------
constexpr float kAlphaMargin = 2e-3f;  // in the exponent: alpha within 0.2 %

__device__ __forceinline__ float splat_fcut(float opacity) {
    // 2 (ln(255 o) + margin); negative when o < 1/255 (never contributes)
    return __fmul_rn(2.0f, __fadd_rn(__logf(__fmul_rn(255.0f, opacity)), kAlphaMargin));
}

// Pixel range [lo, hi] of a splat's support box on one axis (centres within
// r of the mean c, a full-image coordinate), in the coordinates of a window
// starting at full-image pixel o, clipped to [0, size - 1]; lo > hi when
// empty.  The integer shift by o is exact, so a window's ranges are the full
// image's, shifted.
__device__ __forceinline__ void box_range(float c, float r, int o, int size, int &lo, int &hi) {
    const float l = fmaxf(ceilf(__fsub_rn(__fsub_rn(c, r), 0.5f)) - (float)o, 0.0f);
    const float h = fminf(floorf(__fsub_rn(__fadd_rn(c, r), 0.5f)) - (float)o, (float)(size - 1));
    lo = (int)l;
    hi = (l <= h) ? (int)h : (int)l - 1;
}

// Inclusive pixel range, on one axis, of the pixel centres within half-width
// `reach` of the mean: the support box (reach = r) or the axis-aligned extent
// of the ellipse f(d) <= fcut (reach = sqrt(fcut * Sigma2D_axis), widened by
// 1e-4 relative + 0.01 px so FP32 rounding cannot cut a pixel off).
__device__ __forceinline__ float ellipse_reach(float fcut, float sigma_axis) {
    const float x = fmaxf(__fmul_rn(fcut, sigma_axis), 1e-30f);
    return __fadd_rn(__fmul_rn(x * rsqrtf(x), 1.0001f), 0.01f);
}

// Block-wide exclusive scan of one value per thread (blockDim a multiple of
// 32); returns the exclusive prefix, *total (shared) receives the block sum.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const uint32_t inc = warp_inclusive_scan(v);
    __syncthreads();  // warp_sums may still be read by a previous call
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t s = lane < nwarps ? warp_sums[lane] : 0u;
        const uint32_t si = warp_inclusive_scan(s);
        warp_sums[lane] = si - s;
        if (lane == 31) *total = si;
    }
    __syncthreads();
    return inc - v + warp_sums[warp];
}

// meta words written by the cull kernel and read back by the host
enum MetaIndex {
    kMetaVisible = 0, kMetaGroups = 1, kMetaSplats = 2, kMetaLevel0 = 3, kMetaBlocks = 7,
    kMetaZlo = 8, kMetaZhi = 9,  // float bits of a lower / upper bound of every live splat depth
    kMetaWords = 12
};

// Every launch_* function returns the number of kernels it launched.
// Per template Gaussian, add the per-splat sums of contrib (splat ids as
// grouped by the cull kernel; subset levels map through lod_idx).
// ranked LoD (offline): per-Gaussian features and per-template ranking
constexpr int kLodFeatures = 32;
int launch_lod_features(int n_total, int n_tpl, const TemplateInfo *tpls, const TemplateArrays &ta, float *feat,
                        cudaStream_t st);
int launch_lod_targets(int n_total, int n_tpl, int n_bands, const TemplateInfo *tpls, const float *contrib,
                       float floor_, float *target, cudaStream_t st);
int lod_rank(int n_total, int n_tpl, const TemplateInfo *tpls, const float *score, uint32_t *order,
             uint32_t *key0, uint32_t *val0, uint32_t *key1, uint32_t *val1, uint16_t *tk0, uint16_t *tk1,
             uint32_t *scratch, cudaStream_t st);
int launch_contrib_to_template(int n_splats, const Group *groups, int n_groups, const TemplateInfo *tpls,
                               const uint32_t *lod_idx, const float *contrib_splat, float *contrib_tmpl,
                               cudaStream_t st);
// ---- geometry (cs_geometry.cu) ----
int launch_fk(int n_inst, int n_tpl, const int32_t *tid, const float *pose, const TemplateInfo *tpls,
              int max_depth, float *B, cudaStream_t st);
// Cull scratch of n instances (frame totals, then a group byte per
// instance), in 4-byte words.
size_t cull_scratch_words(size_t n_inst);
// Returns the kernels launched, or -1 when the scratch could not be cleared
// (the CUDA error is then cudaGetLastError's).
int launch_cull_group(int n_inst, int n_tpl, const int32_t *tid, const float *root,
                       const TemplateInfo *tpls, const CamParams &cam, const LodParams &lod,
                       int do_cull, float *V, float *Cloc, int32_t *vis, Group *groups,
                       int32_t *meta, int32_t *scratch, cudaStream_t st);
int launch_project(int n_blocks, const Group *groups, const Group *groups_host, int n_groups,
                   const TemplateInfo *tpl_host, const int32_t *vis, const float *B, const float *V,
                   const float *root, const TemplateArrays &ta, const TemplateInfo *tpls,
                   const CamParams &cam, const LodParams &lod, int skin_mode, int sh_frame, float4 *rec,
                   uint32_t *key, uint32_t *bin, cudaStream_t st);
// Tile rectangle of each splat's support box (debug view; recomputed from the
// records: x0 | y0 << 16, x1 | y1 << 16; zero for splats without pairs).
int launch_debug_rects(int n_splats, const float4 *rec, const uint32_t *bins, int W, int H, int ox, int oy,
                       uint2 *rect, cudaStream_t st);
// The records of the last frame expanded to 16 floats per splat (debug
// view; culled splats left unwritten).
int launch_debug_records(int n_splats, const float4 *rec, const uint32_t *sorted_keys, const uint32_t *order,
                         uint32_t key_lo, float4 *out, cudaStream_t st);

// ---- sort and binning (cs_sort.cu) ----
// scratch words needed by exclusive_scan / radix_sort for n elements
size_t scan_scratch_words(size_t n);
size_t radix_scratch_words(size_t n);
// out[0..n] = exclusive prefix sums of in; out[n] = total.
int exclusive_scan(const uint32_t *in, const uint32_t *idx_unused, uint32_t *out, uint32_t n,
                   uint32_t *scratch, cudaStream_t st);
// out[0..n] = exclusive prefix sums of bin_count(bins[i]); out[n] = total.
int exclusive_scan_bins(const uint32_t *bins, uint32_t *out, uint32_t n, uint32_t *scratch, cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs over key bits [0, bits).
// Ping-pongs between (k0, v0) and (k1, v1); *in_second is set to 0 when the
// result is in (k0, v0), 1 when in (k1, v1).  Returns kernels launched.
// When gather_dst is non-null, the last pass also writes, for every output
// position, gather_src[value] to gather_dst (a payload in sorted order).
// With iota_values, the values of the input are taken to be 0 .. n - 1 (v0
// is not read, only written as a ping-pong buffer).
int radix_sort_u32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t n, int bits,
                   uint32_t *scratch, cudaStream_t st, int *in_second,
                   const uint32_t *gather_src = nullptr, uint32_t *gather_dst = nullptr, bool iota_values = false);
int radix_sort_u16(uint16_t *k0, uint32_t *v0, uint16_t *k1, uint32_t *v1, uint32_t n, int bits,
                   uint32_t *scratch, cudaStream_t st, int *in_second);
// Pair emission in two steps around the host's read of the pair count:
// bin_scan_sums writes the per-block sums of the sorted bin words' pair
// counts, exclusively scanned, to sums[0 .. nb) and the total to sums[nb]
// (nb = bin_scan_blocks(n)); launch_emit_pairs_scan then writes every
// splat's pairs (the scan's down-sweep fused into the emission).
size_t bin_scan_blocks(size_t n);
int bin_scan_sums(const uint32_t *bins, uint32_t n, uint32_t *sums, cudaStream_t st);
int launch_emit_pairs_scan(uint32_t n_splats, const uint32_t *order, const uint32_t *bins_sorted,
                           const uint32_t *sums, const float4 *rec, int tiles_x, uint32_t n_tiles, uint16_t *ptile,
                           uint32_t *pval, cudaStream_t st);
int launch_emit_pairs(uint32_t n_splats, const uint32_t *order, const uint32_t *bins_sorted,
                      const uint32_t *pair_off, const float4 *rec, int tiles_x, uint32_t n_tiles, uint16_t *ptile,
                      uint32_t *pval, cudaStream_t st);
int launch_tile_ranges(uint32_t n_pairs, const uint16_t *ptile, uint2 *ranges, uint32_t n_tiles, cudaStream_t st);
int launch_count_live(uint32_t n, const uint32_t *sorted_keys, int32_t *out, cudaStream_t st);

// ---- compositing (cs_blend.cu) ----
// Work buffers of the split compositing of long tile lists (sizes from
// blend_work_sizes): per tile, the slot of a tile with pairs left after the
// first pass (-1 if none); per slot, its tile, its first chunk (one extra
// entry holds the chunk total), whether pass 1 finished it, and the pass-1
// pixel state (r, g, b, T; T negated when saturated); per chunk, the chunk's
// pixel composite (r, g, b, T; T negated when it met the stop rule); per
// slot pixel, the chunk in which it meets the stop rule (-1 if none);
// meta[0] = slots, meta[1] = chunks, meta[3] = the work counter of the
// persistent pass-1 CTAs (plain frames), meta[kBlendCountAt + c] = tiles of
// list length class c, meta[kBlendCursorAt + c] = their fill cursor (all
// zeroed before the plan); pp_tile lists the tiles by decreasing schedule
// key, the empty ones last.
struct BlendWork {
    int32_t *cand_slot;
    int32_t *cand_tile;
    uint32_t *cand_chunk0;
    uint32_t *cand_done;
    float4 *state;
    float4 *part;
    int32_t *meta;
    int32_t *stop;
    // when set: per splat, sum over pixels of its compositing weight
    // alpha * T (added to); lists are then composited in one pass
    float *contrib;
    // when set (training forward, in chunks): per pixel, one past the index
    // of its last composited pair and its final state (r, g, b, T).
    // px_bnd: every pixel's state (r, g, b, T) before pair b of its tile's
    // list, for every b = start + k kBwdChunk (k >= 1) up to the chunk in
    // which the pixel stops, at px_bnd[(b / kBwdChunk) * 256 + pixel of the
    // tile] (b / kBwdChunk is distinct for all such b of a frame: lists are
    // disjoint)
    uint32_t *px_end;
    float4 *px_fin;
    float4 *px_bnd;
    // training forward in chunks of kBwdChunk pairs (numbered tile by tile):
    // chunk counts per tile and their exclusive scan ([tiles + 1]), scan
    // scratch; per chunk and pixel its composite from T = 1 (T negated when
    // it met the stop rule) and one past its last composited pair (0: none);
    // per image pixel the state before its stopping chunk, its last pair so
    // far and that chunk (-1: none)
    uint32_t *t_cnt, *t_chunk0, *t_scan;
    float4 *t_part;
    uint32_t *t_last;
    float4 *t_state;
    uint32_t *t_slast;
    int32_t *t_stop;
    int32_t *pp_tile;     // [tiles]
    int32_t *chunk_slot;  // [chunks]: the slot of each pass-2 chunk
    int32_t ox, oy;       // window origin: pixel (i, j) has its centre at (ox + i + 0.5, oy + j + 0.5)
    int32_t items;        // pass-1 schedule: CS_BLEND_ITEMS_AUTO, _TILES or _BLOCKS
    uint32_t n_pairs, max_slots, max_chunks;  // bounds of the checked debug build
};
constexpr int kBlendKeys = 64;     // schedule keys of pass 1 (see cs_blend.cu)
constexpr int kBlendClasses = 24;  // list length classes: 0 empty, c: 2^(c-1) <= n < 2^c (last: n >= 2^22)
constexpr int kBlendCountAt = 8, kBlendCursorAt = kBlendCountAt + kBlendClasses;
constexpr int kBlendMetaWords = kBlendCursorAt + kBlendClasses;
constexpr int kBlendBlockW = 8, kBlendBlockH = 4;  // pixels of one warp in a 16x16 tile
constexpr uint32_t kBlendBudget = 32768;  // pairs composited by pass 1 per tile
constexpr uint32_t kBlendChunk = 1024;   // pairs per pass-2 chunk
constexpr uint32_t kBwdChunk = 1024;     // pairs per chunk of the compositing backward
// boundary-state slots of a training frame of n_pairs pairs
constexpr size_t bwd_boundary_slots(size_t n_pairs) { return n_pairs / kBwdChunk + 2; }
// kBwdChunk-pair chunks of a frame of n_tiles tiles and n_pairs pairs, at most
constexpr size_t train_max_chunks(size_t n_tiles, size_t n_pairs) { return n_pairs / kBwdChunk + n_tiles; }
constexpr size_t blend_max_slots(size_t n_tiles, size_t n_pairs) {
    return n_tiles < n_pairs / kBlendBudget + 1 ? n_tiles : n_pairs / kBlendBudget + 1;
}
constexpr size_t blend_max_chunks(size_t n_tiles, size_t n_pairs) {
    return n_pairs / kBlendChunk + blend_max_slots(n_tiles, n_pairs) + 1;
}
// Returns the kernels launched, or -1 when the plan's counters could not be
// cleared (the CUDA error is then cudaGetLastError's).
int launch_blend(int tiles_x, int tiles_y, int W, int H, const uint2 *ranges, const uint32_t *pval,
                 const float4 *rec, float4 *out, const BlendWork &work, uint32_t n_pairs, cudaStream_t st);

}  // namespace cs

namespace cs {

// Gradients of the last training frame (cs_backward): everything the four
// backward kernels read and write.
struct BackwardArgs {
    int tiles_x, tiles_y, W, H;
    uint32_t n_pairs;
    const uint2 *ranges;
    const uint32_t *pval;
    const float4 *rec;
    const uint32_t *px_end;
    const float4 *px_fin;   // final (r, g, b, T) per pixel
    const float4 *px_bnd;   // states at the chunk boundaries (BlendWork::px_bnd)
    uint32_t *chunk_cnt;    // [tiles + 1] scratch: backward chunks per tile, then their exclusive scan
    uint32_t *chunk0;
    uint32_t *scan_scratch;
    const float4 *dl_drgba;
    float4 *dsplat;  // [S][3]: du, dv, dA, dB | dC, do, dr, dg | db, -, -, -
    int proj_blocks;
    const Group *groups;
    int n_groups;
    const int32_t *vis;
    const float *B, *V, *Cloc, *root;
    TemplateArrays ta;
    const TemplateInfo *tpls;
    CamParams cam;
    LodParams lod;
    int skin_mode, sh_frame;
    float *g_mean, *g_cov, *g_opacity, *g_sh, *g_B;
    int n_inst, n_tpl;
    const int32_t *tid;
    const float *pose;
    float *g_pose;
    int n_gauss;
    const float4 *scale, *quat;
    float *g_scale, *g_quat;
};
int launch_backward(const BackwardArgs &a, cudaStream_t st);

}  // namespace cs
