// cs_sort.cu -- tile binning and the (tile, depth) sort of a CrowdSplat frame.
//
// The 3DGS rasteriser the paper renders with (CrowdSplat Sec. 1 and Sec. 2
// cite Kerbl et al. 2023) duplicates each splat into every 16x16 tile its
// support box touches and sorts the (tile, depth) keys so that each tile
// can composite its splats front to back.  Here the order is reached in two
// stable stages instead of one 64-bit sort:
//   1. a stable LSD radix sort of the splats by depth key (as many bits as
//      the frame's depth range needs, digits of at most 9 bits);
//   2. pairs are emitted in that depth order (prefix sum of tile counts),
//      then a stable LSD radix sort by tile index (16-bit keys, 13 bits at
//      1080p as 7 + 6) leaves every tile's pairs in (depth, splat id) order.
// Each radix pass is reduce-then-scan (histogram of each digit per block,
// one CTA per digit scanning its row of block counts, scatter): no
// inter-block waits, and the order is deterministic.
#include "cs_internal.cuh"

namespace cs {

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (three kernels: tile sums, spine, down-sweep)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    return block_exclusive_scan(v, total);
}

// element i of a scan input: plain value (MODE 0) or pair count of a bin
// word (MODE 1)
template <int MODE>
__device__ __forceinline__ uint32_t scan_load(const uint32_t *in, uint32_t i) {
    return MODE == 1 ? bin_count(in[i]) : in[i];
}

template <int MODE>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              uint32_t n, uint32_t *__restrict__ sums) {
    __shared__ uint32_t total;
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) v += scan_load<MODE>(in, base + k);
    block_excl_scan(v, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in place, total at sums[nb].
__global__ void __launch_bounds__(kScanThreads) k_scan_spine(uint32_t *__restrict__ sums, uint32_t nb) {
    __shared__ uint32_t total;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += kScanThreads) {
        uint32_t i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t ex = block_excl_scan(v, &total);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

template <int MODE>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *__restrict__ in, uint32_t n,
                                                            const uint32_t *__restrict__ sums,
                                                            uint32_t nb, uint32_t *__restrict__ out) {
    __shared__ uint32_t total;
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? scan_load<MODE>(in, base + k) : 0u;
        s += v[k];
    }
    uint32_t ex = block_excl_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = sums[nb];
}

size_t scan_scratch_words(size_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <int MODE>
static int scan_impl(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *scratch, cudaStream_t st) {
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
        return 0;
    }
    const uint32_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<MODE><<<nb, kScanThreads, 0, st>>>(in, n, scratch);
    k_scan_spine<<<1, kScanThreads, 0, st>>>(scratch, nb);
    k_scan_down<MODE><<<nb, kScanThreads, 0, st>>>(in, n, scratch, nb, out);
    return 3;
}

int exclusive_scan(const uint32_t *in, const uint32_t *, uint32_t *out, uint32_t n, uint32_t *scratch,
                   cudaStream_t st) {
    return scan_impl<0>(in, out, n, scratch, st);
}

int exclusive_scan_bins(const uint32_t *bins, uint32_t *out, uint32_t n, uint32_t *scratch, cudaStream_t st) {
    return scan_impl<1>(bins, out, n, scratch, st);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, digits of up to 9 bits, reduce-then-scan per pass
//
// A sort of b-bit keys takes ceil(b / 9) passes of near-equal digit width
// (13-bit tile keys: 7 + 6 bits; 26-bit depth keys: 9 + 9 + 8; 32-bit keys:
// 4 x 8): a narrower digit needs fewer ballots to rank and smaller count
// tables, a wider one may save a pass.  A block owns
// 4,096 consecutive elements; warp w owns 512 of them, read in 16 rounds of
// 32 consecutive elements (coalesced, all loads issued before any
// shared-memory update).  Histogram pass: per-warp digit counts (shared
// atomics), one row per digit in the global count matrix (digit-major),
// which an exclusive scan turns into each block's global digit offsets.
// Scatter pass: stable ranks from per-warp running counts, the lanes that
// share a digit found with one ballot per digit bit, then a block-local
// sort in shared memory, then each digit's run is written out with
// consecutive threads on consecutive addresses.
// ---------------------------------------------------------------------------

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 16;                              // per lane
constexpr int kRadixTile = kRadixThreads * kRadixItems;      // per block (4,096)
constexpr int kRadixWarpTile = 32 * kRadixItems;             // per warp (512)
constexpr int kRadixMaxBits = 9;
constexpr int kRadixDigits = 1 << kRadixMaxBits;             // largest digit range

template <typename K, int kBits>
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const K *__restrict__ keys, uint32_t n,
                                                              int shift, uint32_t *__restrict__ hist,
                                                              uint32_t nblocks) {
    constexpr uint32_t kDigits = 1u << kBits;
    __shared__ uint32_t h[kRadixWarps][kDigits];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kRadixWarps * (int)kDigits; d += kRadixThreads) (&h[0][0])[d] = 0;
    const uint32_t base = blockIdx.x * kRadixTile + warp * kRadixWarpTile;
    uint32_t dig[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        dig[r] = i < n ? (uint32_t)((keys[i] >> shift) & (kDigits - 1)) : kDigits;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r)
        if (dig[r] < kDigits) atomicAdd(&h[warp][dig[r]], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < (int)kDigits; d += kRadixThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) s += h[w][d];
        hist[(size_t)d * nblocks + blockIdx.x] = s;
    }
}

// Exclusive scan of each digit's row of the (digit, block) count matrix
// (digit-major), one CTA per digit: offs[d][b] = counts of digit d in blocks
// before b; tot[d] = the digit's total.  The scatter adds the digit's base
// (an exclusive scan of tot it computes itself).
__global__ void __launch_bounds__(kScanThreads) k_radix_rowscan(const uint32_t *__restrict__ hist, uint32_t nb,
                                                                uint32_t *__restrict__ offs,
                                                                uint32_t *__restrict__ tot) {
    __shared__ uint32_t total;
    const uint32_t *row = hist + (size_t)blockIdx.x * nb;
    uint32_t *orow = offs + (size_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += kScanTile) {
        const uint32_t i0 = base + threadIdx.x * kScanItems;
        uint32_t v[kScanItems], sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = i0 + k < nb ? row[i0 + k] : 0u;
            sum += v[k];
        }
        uint32_t ex = block_excl_scan(sum, &total) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < nb) orow[i0 + k] = ex;
            ex += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

template <typename K, int kBits>
__global__ void __launch_bounds__(kRadixThreads, 3) k_radix_scatter(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, int shift, const uint32_t *__restrict__ offs,
    const uint32_t *__restrict__ dtot_g, uint32_t nblocks, const uint32_t *__restrict__ gsrc,
    uint32_t *__restrict__ gdst) {
    constexpr uint32_t kDigits = 1u << kBits;
    constexpr int kPer = kDigits > (uint32_t)kRadixThreads ? (int)kDigits / kRadixThreads : 1;  // digits per thread
    __shared__ uint32_t wcnt[kRadixWarps][kDigits];  // running counts, then warp offsets
    __shared__ uint32_t dstart[kDigits];             // block-local start of each digit
    __shared__ uint32_t gbase[kDigits];              // global start of each digit
    __shared__ uint32_t total;
    // block-local sort buffers (dynamic: with 9-bit digits the CTA needs
    // more than the 48 KB of static shared memory)
    extern __shared__ __align__(16) unsigned char radix_dyn[];
    uint32_t *sval = reinterpret_cast<uint32_t *>(radix_dyn);
    K *skey = reinterpret_cast<K *>(radix_dyn + kRadixTile * sizeof(uint32_t));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kRadixWarps * (int)kDigits; d += kRadixThreads) (&wcnt[0][0])[d] = 0;
    const uint32_t blk0 = blockIdx.x * kRadixTile;
    const uint32_t base = blk0 + warp * kRadixWarpTile;
    K k[kRadixItems];
    uint32_t v[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? kin[i] : (K)0;
        v[r] = ok ? (vin ? vin[i] : i) : 0u;
    }
    __syncthreads();
    // stable rank within the warp's 512 elements; packed as digit | rank << 16
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t dr[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & (kDigits - 1)) : kDigits;
        // lanes holding the same digit: agree on all kBits bits, among valid lanes
        unsigned peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < kBits; ++b) {
            const unsigned m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
        const uint32_t before = d < kDigits ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (d < kDigits && (peers & lt) == 0u) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        dr[r] = d | ((before + __popc(peers & lt)) << 16);
    }
    __syncthreads();
    // per digit (thread t: digits t kPer .. t kPer + kPer - 1): exclusive
    // prefix over warps, and the digit's block total; the digit's global
    // total for the digit bases
    uint32_t tot = 0, dtot[kPer], gtot = 0, gt[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int d = threadIdx.x * kPer + j;
        dtot[j] = 0;
        gt[j] = 0;
        if (d < (int)kDigits) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            dtot[j] = run;
            tot += run;
            gt[j] = dtot_g[d];
            gtot += gt[j];
        }
    }
    // block-local digit starts
    uint32_t ex = block_excl_scan(tot, &total);
    // global digit bases: exclusive scan of the digit totals
    uint32_t gex = block_excl_scan(gtot, &total);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int d = threadIdx.x * kPer + j;
        if (d < (int)kDigits) {
            dstart[d] = ex;
            gbase[d] = gex + offs[(size_t)d * nblocks + blockIdx.x];
        }
        ex += dtot[j];
        gex += gt[j];
    }
    __syncthreads();
    // block-local sort in shared memory
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const uint32_t d = dr[r] & 0xFFFFu;
        if (d < kDigits) {
            const uint32_t lp = dstart[d] + wcnt[warp][d] + (dr[r] >> 16);
            skey[lp] = k[r];
            sval[lp] = v[r];
        }
    }
    __syncthreads();
    // runs of equal digits go to consecutive global addresses
    const uint32_t cnt = min((uint32_t)kRadixTile, n - blk0);
#pragma unroll 4
    for (uint32_t p = threadIdx.x; p < cnt; p += kRadixThreads) {
        const K key = skey[p];
        const uint32_t d = (uint32_t)((key >> shift) & (kDigits - 1));
        const uint32_t g = gbase[d] + (p - dstart[d]);
        const uint32_t val = sval[p];
        if (!in_bounds(g < n, kChkSort)) continue;
        kout[g] = key;
        vout[g] = val;
        if (gdst && in_bounds(val < n, kChkSort)) gdst[g] = gsrc[val];
    }
}

size_t radix_scratch_words(size_t n) {
    size_t nb = (n + kRadixTile - 1) / kRadixTile;
    if (nb == 0) nb = 1;
    size_t hist = (size_t)kRadixDigits * nb;
    return 2 * hist + kRadixDigits;
}

// one pass over digit bits [shift, shift + kBits)
template <typename K, int kBits>
static int radix_pass(const K *ki, const uint32_t *vi, K *ko, uint32_t *vo, uint32_t n, int shift, uint32_t nb,
                      uint32_t *scratch, const uint32_t *gsrc, uint32_t *gdst, cudaStream_t st) {
    const uint32_t hn = (1u << kBits) * nb;
    uint32_t *hist = scratch;
    uint32_t *offs = scratch + hn;
    uint32_t *dtot = scratch + 2 * hn;
    constexpr int kDyn = kRadixTile * (int)(sizeof(uint32_t) + sizeof(K));
    static int configured_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaFuncSetAttribute(k_radix_scatter<K, kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
        configured_device = dev;
    }
    k_radix_hist<K, kBits><<<nb, kRadixThreads, 0, st>>>(ki, n, shift, hist, nb);
    k_radix_rowscan<<<1u << kBits, kScanThreads, 0, st>>>(hist, nb, offs, dtot);
    k_radix_scatter<K, kBits><<<nb, kRadixThreads, kDyn, st>>>(ki, vi, ko, vo, n, shift, offs, dtot, nb, gsrc,
                                                              gdst);
    return 3;
}

template <typename K>
static int radix_sort(K *k0, uint32_t *v0, K *k1, uint32_t *v1, uint32_t n, int bits,
                      uint32_t *scratch, cudaStream_t st, int *in_second, const uint32_t *gsrc,
                      uint32_t *gdst, bool iota_values) {
    *in_second = 0;
    if (n == 0 || bits <= 0) return 0;
    int launched = 0;
    const uint32_t nb = (n + kRadixTile - 1) / kRadixTile;
    // fewest passes of at most 9 bits, near-equal widths (4 bits at least)
    const int passes = (bits + kRadixMaxBits - 1) / kRadixMaxBits;
    int cur = 0;
    for (int p = 0, shift = 0; p < passes; ++p) {
        const K *ki = cur ? k1 : k0;
        const uint32_t *vi = p == 0 && iota_values ? nullptr : (cur ? v1 : v0);
        K *ko = cur ? k0 : k1;
        uint32_t *vo = cur ? v0 : v1;
        const int left = bits - shift;
        const int width = std::max(4, (left + (passes - p) - 1) / (passes - p));
        const bool last = p == passes - 1;
        const uint32_t *gs = last ? gsrc : nullptr;
        uint32_t *gd = last ? gdst : nullptr;
        switch (width) {
            case 4: launched += radix_pass<K, 4>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
            case 5: launched += radix_pass<K, 5>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
            case 6: launched += radix_pass<K, 6>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
            case 7: launched += radix_pass<K, 7>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
            case 8: launched += radix_pass<K, 8>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
            default: launched += radix_pass<K, 9>(ki, vi, ko, vo, n, shift, nb, scratch, gs, gd, st); break;
        }
        shift += width;
        cur ^= 1;
    }
    *in_second = cur;
    return launched;
}

int radix_sort_u32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t n, int bits,
                   uint32_t *scratch, cudaStream_t st, int *in_second, const uint32_t *gather_src,
                   uint32_t *gather_dst, bool iota_values) {
    return radix_sort<uint32_t>(k0, v0, k1, v1, n, bits, scratch, st, in_second, gather_src, gather_dst,
                                iota_values);
}

int radix_sort_u16(uint16_t *k0, uint32_t *v0, uint16_t *k1, uint32_t *v1, uint32_t n, int bits,
                   uint32_t *scratch, cudaStream_t st, int *in_second) {
    return radix_sort<uint16_t>(k0, v0, k1, v1, n, bits, scratch, st, in_second, nullptr, nullptr, false);
}

// ---------------------------------------------------------------------------
// pair emission in depth order, tile ranges, live count
// ---------------------------------------------------------------------------

// Pairs of one splat: every tile its reach box meets, written to
// ptile / pval from position o (at most e - o of them).  Small splats carry
// those tiles as a 3x3 mask in their bin word (gathered into depth order by
// the depth sort); larger ones take the reach box from the record.
__device__ __forceinline__ void emit_splat_pairs(uint32_t b, uint32_t s, uint32_t o, uint32_t e,
                                                 const float4 *__restrict__ rec, int tiles_x,
                                                 uint16_t *__restrict__ ptile, uint32_t *__restrict__ pval,
                                                 uint32_t n_tiles, uint32_t n_pairs) {
    if (o >= e || !in_bounds(e <= n_pairs, kChkPair)) return;
    if (!(b & kBinLarge)) {
        const uint32_t x0 = b & 0xFFu, y0 = (b >> 8) & 0xFFu;
        uint32_t m = (b >> 16) & 0x1FFu;
        while (m && o < e) {
            const uint32_t k = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t tile = (y0 + k / 3) * (uint32_t)tiles_x + x0 + k % 3;
            if (in_bounds(tile < n_tiles, kChkTile)) {
                ptile[o] = (uint16_t)tile;
                pval[o] = s;
            }
            ++o;
        }
        return;
    }
    const float4 r3 = rec[(size_t)s * kRecVec];  // reach x, reach y, log2 o, C
    const uint32_t rx = __float_as_uint(r3.x), ry = __float_as_uint(r3.y);
    const int ax0 = (int)(rx & 0xFFFFu), ax1 = (int)(rx >> 16);
    const int ay0 = (int)(ry & 0xFFFFu), ay1 = (int)(ry >> 16);
    for (int yy = ay0 >> 4; yy <= (ay1 >> 4); ++yy) {
        for (int xx = ax0 >> 4; xx <= (ax1 >> 4); ++xx) {
            if (o >= e) return;
            if (in_bounds((uint32_t)(yy * tiles_x + xx) < n_tiles, kChkTile)) {
                ptile[o] = (uint16_t)(yy * tiles_x + xx);
                pval[o] = s;
            }
            ++o;
        }
    }
}

// Thread per sorted splat, offsets from a scan of the sorted bin words.
__global__ void __launch_bounds__(256) k_emit_pairs(uint32_t n, const uint32_t *__restrict__ order,
                                                    const uint32_t *__restrict__ bins,
                                                    const uint32_t *__restrict__ pair_off,
                                                    const float4 *__restrict__ rec, int tiles_x, uint32_t n_tiles,
                                                    uint16_t *__restrict__ ptile,
                                                    uint32_t *__restrict__ pval) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = order[i];
    if (!in_bounds(s < n, kChkSplat)) return;
    emit_splat_pairs(bins[i], s, pair_off[i], pair_off[i + 1], rec, tiles_x, ptile, pval, n_tiles, pair_off[n]);
}

// Pair emission fused with the down-sweep of the pair-count scan: block b
// takes the kScanTile splats from b kScanTile in depth order, in kScanItems
// rounds of kScanThreads consecutive splats (one per thread, coalesced); its
// offset comes from the scanned block sums, each round is scanned in the
// block, so no per-splat offset array is written or read.  A splat whose
// tiles fit a 3x3 window (at most nine pairs) is written by its thread; a
// larger one is queued in shared memory and written by a whole warp, lane l
// taking its tiles l, l + 32, ... in row-major order (coalesced stores, no
// warp waiting on one lane's long loop): exactly the pairs emit_splat_pairs
// writes.
__global__ void __launch_bounds__(kScanThreads) k_emit_pairs_scan(uint32_t n, const uint32_t *__restrict__ order,
                                                                 const uint32_t *__restrict__ bins,
                                                                 const uint32_t *__restrict__ sums,
                                                                 const float4 *__restrict__ rec, int tiles_x,
                                                                 uint32_t n_tiles, uint16_t *__restrict__ ptile,
                                                                 uint32_t *__restrict__ pval) {
    __shared__ uint32_t total, n_large;
    const uint32_t n_pairs = CS_CHECKS ? sums[gridDim.x] : 0xFFFFFFFFu;  // the scan's total
    __shared__ uint4 s_large[kScanThreads];  // splat id, first pair, tile x0 | y0 << 16, tiles per row
    __shared__ uint32_t s_cnt[kScanThreads];  // its pairs
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    uint32_t carry = sums[blockIdx.x];
    if (t == 0) n_large = 0u;
#pragma unroll 1
    for (int r = 0; r < kScanItems; ++r) {
        const uint32_t i = blockIdx.x * kScanTile + r * kScanThreads + t;
        const uint32_t b = i < n ? bins[i] : 0u;
        const uint32_t c = bin_count(b);
        const uint32_t o = carry + block_excl_scan(c, &total);
        if (c && in_bounds(order[i] < n, kChkSplat)) {
            const uint32_t s = order[i];
            if (!(b & kBinLarge)) {
                emit_splat_pairs(b, s, o, o + c, rec, tiles_x, ptile, pval, n_tiles, n_pairs);
            } else {
                const float4 r3 = rec[(size_t)s * kRecVec];  // reach x, reach y, log2 o, C
                const uint32_t rx = __float_as_uint(r3.x), ry = __float_as_uint(r3.y);
                const uint32_t tx0 = (rx & 0xFFFFu) >> 4, ty0 = (ry & 0xFFFFu) >> 4;
                const uint32_t q = atomicAdd(&n_large, 1u);  // queue order: any (own output range)
                s_large[q] = make_uint4(s, o, tx0 | (ty0 << 16), ((rx >> 16) >> 4) - tx0 + 1u);
                s_cnt[q] = c;
            }
        }
        carry += total;
        __syncthreads();
        const uint32_t nl = n_large;
        for (uint32_t q = warp; q < nl; q += kScanThreads / 32) {
            const uint4 L = s_large[q];  // splat id, first pair, tile x0 | y0 << 16, tiles per row
            const uint32_t cnt = s_cnt[q];
            if (!in_bounds(L.y + cnt <= n_pairs, kChkPair)) continue;
            for (uint32_t k = lane; k < cnt; k += 32) {
                const uint32_t row = k / L.w, col = k - row * L.w;
                const uint32_t tile = ((L.z >> 16) + row) * (uint32_t)tiles_x + (L.z & 0xFFFFu) + col;
                if (!in_bounds(tile < n_tiles, kChkTile)) continue;
                ptile[L.y + k] = (uint16_t)tile;
                pval[L.y + k] = L.x;
            }
        }
        __syncthreads();  // the queue is refilled by the next round
        if (t == 0) n_large = 0u;
    }
}

size_t bin_scan_blocks(size_t n) { return (n + kScanTile - 1) / kScanTile; }

int bin_scan_sums(const uint32_t *bins, uint32_t n, uint32_t *sums, cudaStream_t st) {
    if (n == 0) return 0;
    const uint32_t nb = (uint32_t)bin_scan_blocks(n);
    k_scan_reduce<1><<<nb, kScanThreads, 0, st>>>(bins, n, sums);
    k_scan_spine<<<1, kScanThreads, 0, st>>>(sums, nb);
    return 2;
}

int launch_emit_pairs_scan(uint32_t n_splats, const uint32_t *order, const uint32_t *bins_sorted,
                           const uint32_t *sums, const float4 *rec, int tiles_x, uint32_t n_tiles, uint16_t *ptile,
                           uint32_t *pval, cudaStream_t st) {
    if (n_splats == 0) return 0;
    k_emit_pairs_scan<<<(uint32_t)bin_scan_blocks(n_splats), kScanThreads, 0, st>>>(
        n_splats, order, bins_sorted, sums, rec, tiles_x, n_tiles, ptile, pval);
    return 1;
}

int launch_emit_pairs(uint32_t n_splats, const uint32_t *order, const uint32_t *bins_sorted,
                      const uint32_t *pair_off, const float4 *rec, int tiles_x, uint32_t n_tiles, uint16_t *ptile,
                      uint32_t *pval, cudaStream_t st) {
    if (n_splats == 0) return 0;
    k_emit_pairs<<<(n_splats + 255) / 256, 256, 0, st>>>(n_splats, order, bins_sorted, pair_off, rec,
                                                          tiles_x, n_tiles, ptile, pval);
    return 1;
}

// Tile boundaries of the sorted pair list: each thread reads 8 tile keys
// with one 16-byte load (the list starts 16-byte aligned) plus its two
// neighbours, and writes the start / end of every tile that begins / ends
// among its keys.
__global__ void __launch_bounds__(256) k_tile_ranges(uint32_t n, const uint16_t *__restrict__ ptile,
                                                     uint2 *__restrict__ ranges, uint32_t n_tiles) {
    const uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) * 8u;
    if (base >= n) return;
    uint32_t v[8];
    if (base + 8u <= n) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(ptile + base));
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = ww[k] & 0xFFFFu;
            v[2 * k + 1] = ww[k] >> 16;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = base + k < n ? (uint32_t)__ldg(ptile + base + k) : 0x10000u;
    }
    uint32_t prev = base > 0 ? (uint32_t)__ldg(ptile + base - 1) : 0x10000u;
    const uint32_t next = base + 8u < n ? (uint32_t)__ldg(ptile + base + 8) : 0x10000u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t t = v[k];
        if (t > 0xFFFFu) break;  // past the end
        const uint32_t after = k < 7 ? v[k + 1] : next;
        if (in_bounds(t < n_tiles, kChkTile)) {
            if (t != prev) ranges[t].x = base + k;
            if (t != after) ranges[t].y = base + k + 1;
        }
        prev = t;
    }
}

int launch_tile_ranges(uint32_t n_pairs, const uint16_t *ptile, uint2 *ranges, uint32_t n_tiles, cudaStream_t st) {
    if (n_pairs == 0) return 0;
    const uint32_t threads = (n_pairs + 7) / 8;
    k_tile_ranges<<<(threads + 255) / 256, 256, 0, st>>>(n_pairs, ptile, ranges, n_tiles);
    return 1;
}

__global__ void __launch_bounds__(256) k_count_live(uint32_t n, const uint32_t *__restrict__ keys,
                                                    int32_t *__restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool live = keys[i] != 0xFFFFFFFFu;
    const bool next_live = i + 1 < n && keys[i + 1] != 0xFFFFFFFFu;
    if (i == 0 && !live) *out = 0;
    if (live && !next_live) *out = (int32_t)(i + 1);
}

int launch_count_live(uint32_t n, const uint32_t *sorted_keys, int32_t *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    if (n == 0) return 0;
    k_count_live<<<(n + 255) / 256, 256, 0, st>>>(n, sorted_keys, out);
    return 1;
}

CS_DEFINE_CHECK_READER(check_word_sort)

}  // namespace cs
