// cs_geometry.cu -- per-instance and per-Gaussian geometry of a CrowdSplat
// frame: forward kinematics, distance LoD with instance culling and
// grouping, and the fused skinning + EWA projection + SH colour kernel.
//
// CrowdSplat Sec. 2 (stage 2): each duplicated character is animated by
// linear blend skinning of its template, whose attributes other than the
// posed means are shared; a distance band picks the template's level of
// detail.  The projection follows the 3DGS rasteriser the paper renders
// with (cited in Sec. 1 and Sec. 2).
#include "cs_internal.cuh"

namespace cs {

// ---------------------------------------------------------------------------
// forward kinematics: one warp per instance, lane j = joint j
// ---------------------------------------------------------------------------

// Rodrigues' formula in FP32: R = cos(th) I + sinc(th) K + b v v^T with
// K = skew(v), b = (1 - cos th) / th^2 written as 2 sin^2(th/2) / th^2 to
// avoid cancellation; second-order series below th = 1e-8.
__device__ __forceinline__ void rodrigues(float x, float y, float z, float R[9]) {
    float th2 = x * x + y * y + z * z;
    float c, a, b;
    if (th2 < 1e-16f) {
        c = 1.0f - 0.5f * th2;
        a = 1.0f;
        b = 0.5f;
    } else {
        float th = sqrtf(th2);
        float s, hs, hc;
        sincosf(th, &s, &c);
        sincosf(0.5f * th, &hs, &hc);
        a = s / th;
        float h = hs / th;
        b = 2.0f * h * h;
    }
    R[0] = c + b * x * x;     R[1] = -a * z + b * x * y; R[2] = a * y + b * x * z;
    R[3] = a * z + b * x * y; R[4] = c + b * y * y;      R[5] = -a * x + b * y * z;
    R[6] = -a * y + b * x * z; R[7] = a * x + b * y * z; R[8] = c + b * z * z;
}

__global__ void __launch_bounds__(256) k_fk(int n_inst, int n_tpl, const int32_t *__restrict__ tid,
                                            const float *__restrict__ pose,
                                            const TemplateInfo *__restrict__ tpls, int max_depth,
                                            float *__restrict__ B) {
    const int inst = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (inst >= n_inst) return;  // uniform per warp
    const int t = tid[inst];
    if (t < 0 || t >= n_tpl) return;  // such instances are hidden by the cull kernel
    const TemplateInfo &T = tpls[t];
    const int j = lane < kJoints ? lane : kJoints - 1;
    const int par = T.parent[j];
    const int dep = lane < kJoints ? T.depth[j] : 1 << 20;
    float R[9];
    const float *pv = pose + (size_t)inst * kJoints * 3 + j * 3;
    rodrigues(pv[0], pv[1], pv[2], R);
    float jx = T.rest[j * 3 + 0], jy = T.rest[j * 3 + 1], jz = T.rest[j * 3 + 2];
    float lx = jx, ly = jy, lz = jz;
    if (par >= 0) {
        lx -= T.rest[par * 3 + 0];
        ly -= T.rest[par * 3 + 1];
        lz -= T.rest[par * 3 + 2];
    }
    // local transform L = [R | l]; global G = G_parent o L, level by level
    float G[12] = {R[0], R[1], R[2], lx, R[3], R[4], R[5], ly, R[6], R[7], R[8], lz};
    const int src = par >= 0 ? par : j;
    for (int level = 1; level <= max_depth; ++level) {
        float P[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) P[e] = __shfl_sync(0xffffffffu, G[e], src);
        if (dep == level) {
            float N[12];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    N[r * 4 + c] = P[r * 4 + 0] * R[0 * 3 + c] + P[r * 4 + 1] * R[1 * 3 + c] +
                                   P[r * 4 + 2] * R[2 * 3 + c];
                N[r * 4 + 3] = P[r * 4 + 0] * lx + P[r * 4 + 1] * ly + P[r * 4 + 2] * lz + P[r * 4 + 3];
            }
#pragma unroll
            for (int e = 0; e < 12; ++e) G[e] = N[e];
        }
    }
    if (lane < kJoints) {
        // B = G o [I | -J]
        float *o = B + ((size_t)inst * kJoints + j) * 12;
        float4 r0, r1, r2;
        r0 = make_float4(G[0], G[1], G[2], G[3] - (G[0] * jx + G[1] * jy + G[2] * jz));
        r1 = make_float4(G[4], G[5], G[6], G[7] - (G[4] * jx + G[5] * jy + G[6] * jz));
        r2 = make_float4(G[8], G[9], G[10], G[11] - (G[8] * jx + G[9] * jy + G[10] * jz));
        reinterpret_cast<float4 *>(o)[0] = r0;
        reinterpret_cast<float4 *>(o)[1] = r1;
        reinterpret_cast<float4 *>(o)[2] = r2;
    }
}

int launch_fk(int n_inst, int n_tpl, const int32_t *tid, const float *pose, const TemplateInfo *tpls,
              int max_depth, float *B, cudaStream_t st) {
    if (n_inst <= 0) return 0;
    int blocks = (n_inst + 7) / 8;
    k_fk<<<blocks, 256, 0, st>>>(n_inst, n_tpl, tid, pose, tpls, max_depth, B);
    return 1;
}

// ---------------------------------------------------------------------------
// LoD + instance cull + grouping.  Every CTA takes kCullThreads instances
// (LoD band, view transform, cull, depth bound, group byte) and adds its
// group counts and depth bound to the frame's totals; the CTA that finishes
// last (a ticket taken after a memory fence: no CTA waits for another)
// turns the totals into the groups and places every visible instance.
// ---------------------------------------------------------------------------

constexpr int kCullThreads = 1024;
constexpr uint8_t kHidden = 255;
// frame totals in the cull scratch (zeroed before the launch): group counts,
// then the inverted bits of the lowest depth bound, the highest, the ticket
constexpr int kCullZloInv = kMaxGroups, kCullZhi = kMaxGroups + 1, kCullTicket = kMaxGroups + 2;

__global__ void __launch_bounds__(kCullThreads) k_cull_group(
    int n_inst, int n_tpl, const int32_t *__restrict__ tid, const float *__restrict__ root,
    const TemplateInfo *__restrict__ tpls, CamParams cam, LodParams lod, int do_cull,
    float *__restrict__ V, float *__restrict__ Cloc, int32_t *__restrict__ vis,
    Group *__restrict__ groups, int32_t *__restrict__ meta, int32_t *__restrict__ tot,
    uint8_t *__restrict__ grp) {
    __shared__ int32_t gcount[kMaxGroups];
    __shared__ int32_t gslot[kMaxGroups];
    __shared__ int32_t wcount[kCullThreads / 32][kMaxGroups];  // per warp and group
    __shared__ uint32_t zlo_bits, zhi_bits;
    __shared__ bool last;
    const int L = lod.n_levels;
    const int n_grp = n_tpl * L;
    for (int g = threadIdx.x; g < n_grp; g += blockDim.x) gcount[g] = 0;
    if (threadIdx.x == 0) {
        zlo_bits = 0x7F7FFFFFu;  // FLT_MAX
        zhi_bits = __float_as_uint(cam.near_z);
    }
    __syncthreads();

    {
        // every lane of the CTA runs (the depth bound is reduced per warp)
        const int i = (int)blockIdx.x * kCullThreads + threadIdx.x;
        uint32_t zl_bits = 0x7F7FFFFFu, zh_bits = 0u;
        if (i < n_inst) {
            const float *rt = root + (size_t)i * 12;
            float Rr[9] = {rt[0], rt[1], rt[2], rt[4], rt[5], rt[6], rt[8], rt[9], rt[10]};
            float tr[3] = {rt[3], rt[7], rt[11]};
            // distance band: number of thresholds <= distance (CrowdSplat Sec. 2)
            float dx = tr[0] - cam.center[0], dy = tr[1] - cam.center[1], dz = tr[2] - cam.center[2];
            float d = sqrtf(dx * dx + dy * dy + dz * dz);
            int lvl = 0;
            for (int k = 0; k < L - 1; ++k) lvl += (d >= lod.thresh[k]) ? 1 : 0;
            // V = camera o root
            float Vm[12];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    Vm[r * 4 + c] = cam.R[r * 3 + 0] * Rr[0 * 3 + c] + cam.R[r * 3 + 1] * Rr[1 * 3 + c] +
                                    cam.R[r * 3 + 2] * Rr[2 * 3 + c];
                Vm[r * 4 + 3] = cam.R[r * 3 + 0] * tr[0] + cam.R[r * 3 + 1] * tr[1] +
                                cam.R[r * 3 + 2] * tr[2] + cam.t[r];
            }
            float4 *vo = reinterpret_cast<float4 *>(V + (size_t)i * 12);
            vo[0] = make_float4(Vm[0], Vm[1], Vm[2], Vm[3]);
            vo[1] = make_float4(Vm[4], Vm[5], Vm[6], Vm[7]);
            vo[2] = make_float4(Vm[8], Vm[9], Vm[10], Vm[11]);
            // camera centre in the root frame: Rr^T (c - t)
            float e0 = -dx, e1 = -dy, e2 = -dz;
            reinterpret_cast<float4 *>(Cloc)[i] =
                make_float4(Rr[0] * e0 + Rr[3] * e1 + Rr[6] * e2, Rr[1] * e0 + Rr[4] * e1 + Rr[7] * e2,
                            Rr[2] * e0 + Rr[5] * e1 + Rr[8] * e2, 0.0f);
            int t = tid[i];
            bool visible = t >= 0 && t < n_tpl;  // out-of-range ids (device input) are hidden
            if (do_cull && visible) {
                const TemplateInfo &T = tpls[t];
                // bounding sphere: centre = pelvis rest position (posed local
                // means stay within reach of it), grown by the splat support
                float px = T.rest[0], py = T.rest[1], pz = T.rest[2];
                float cxs = Vm[0] * px + Vm[1] * py + Vm[2] * pz + Vm[3];
                float cys = Vm[4] * px + Vm[5] * py + Vm[6] * pz + Vm[7];
                float czs = Vm[8] * px + Vm[9] * py + Vm[10] * pz + Vm[11];
                float reach = T.reach[lvl] * 1.0001f + 1e-4f;
                float grow = reach + cam.cull_sigma_k * T.sigma_max[lvl] + 1e-3f;
                if (czs + reach <= cam.near_z) visible = false;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float s = cam.plane[p][0] * cxs + cam.plane[p][1] * cys + cam.plane[p][2] * czs;
                    if (s > grow) visible = false;
                }
            }
            if (visible) {
                // view-depth interval of the instance's splat means: a mean p
                // lies within reach of the pelvis rest position c (instance
                // frame), so its depth is within |v| reach of v.c + t_z, v the
                // depth row of camera o root (Cauchy-Schwarz); widened for
                // rounding and clipped below at the near plane
                const TemplateInfo &T = tpls[t];
                const float czs = Vm[8] * T.rest[0] + Vm[9] * T.rest[1] + Vm[10] * T.rest[2] + Vm[11];
                const float vn = sqrtf(Vm[8] * Vm[8] + Vm[9] * Vm[9] + Vm[10] * Vm[10]);
                const float ext = T.reach[lvl] * vn * 1.001f + 1e-3f;
                const float zl = fmaxf(cam.near_z, (czs - ext) * 0.999f - 1e-3f);
                const float zh = fmaxf(cam.near_z, (czs + ext) * 1.001f + 1e-3f);
                zl_bits = __float_as_uint(zl);  // positive floats order as their bits
                zh_bits = __float_as_uint(zh);
            }
            uint8_t g = visible ? (uint8_t)(t * L + lvl) : kHidden;
            grp[i] = g;
            if (visible) atomicAdd(&gcount[g], 1);
        }
        // one shared atomic per warp instead of one per visible instance
        zl_bits = __reduce_min_sync(0xffffffffu, zl_bits);
        zh_bits = __reduce_max_sync(0xffffffffu, zh_bits);
        if ((threadIdx.x & 31) == 0) {
            if (zl_bits != 0x7F7FFFFFu) atomicMin(&zlo_bits, zl_bits);
            if (zh_bits != 0u) atomicMax(&zhi_bits, zh_bits);
        }
    }
    __syncthreads();
    // this CTA's counts and depth bound into the frame totals
    for (int g = threadIdx.x; g < n_grp; g += blockDim.x)
        if (gcount[g]) atomicAdd(tot + g, gcount[g]);
    if (threadIdx.x == 0) {
        unsigned *tu = reinterpret_cast<unsigned *>(tot);
        if (zlo_bits != 0x7F7FFFFFu) atomicMax(tu + kCullZloInv, ~zlo_bits);
        atomicMax(tu + kCullZhi, zhi_bits);
    }
    __threadfence();  // the group bytes and totals before the ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(tot + kCullTicket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last CTA: the frame's totals (read past L1: other CTAs wrote them)
    for (int g = threadIdx.x; g < n_grp; g += blockDim.x) gcount[g] = __ldcg(tot + g);
    if (threadIdx.x == 0) {
        const uint32_t zinv = (uint32_t)__ldcg(tot + kCullZloInv);
        zlo_bits = zinv ? ~zinv : 0x7F7FFFFFu;
        zhi_bits = max((uint32_t)__ldcg(tot + kCullZhi), __float_as_uint(cam.near_z));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int slot = 0, ng = 0;
        long long splat = 0, blocks = 0;
        int per_level[kMaxLevels] = {0, 0, 0, 0};
        for (int g = 0; g < n_grp; ++g) {
            gslot[g] = slot;
            int c = gcount[g];
            if (c == 0) continue;
            int t = g / L, l = g % L;
            Group G;
            G.tpl = t;
            G.lvl = l;
            G.slot0 = slot;
            G.nslots = c;
            G.ng = tpls[t].n_level[l];
            G.splat0 = (int32_t)(splat < 0x7fffffffLL ? splat : 0x7fffffffLL);
            G.block0 = (int32_t)(blocks < 0x7fffffffLL ? blocks : 0x7fffffffLL);
            groups[ng++] = G;
            slot += c;
            splat += (long long)c * G.ng;
            blocks += (long long)c * ((G.ng + 255) / 256);
            per_level[l] += c;
        }
        meta[kMetaVisible] = slot;
        meta[kMetaGroups] = ng;
        // splat count, saturated: the host rejects counts >= 2^31
        meta[kMetaSplats] = (int32_t)(splat < 0x7fffffffLL ? splat : 0x7fffffffLL);
        for (int l = 0; l < kMaxLevels; ++l) meta[kMetaLevel0 + l] = per_level[l];
        meta[kMetaBlocks] = (int32_t)(blocks < 0x7fffffffLL ? blocks : 0x7fffffffLL);
        meta[kMetaZlo] = (int32_t)zlo_bits;
        meta[kMetaZhi] = (int32_t)zhi_bits;
    }
    __syncthreads();
    // stable placement, one round of kCullThreads instances at a time: an
    // instance goes to its group's slot plus the instances of its group in
    // earlier rounds (gslot runs on), in earlier warps of the round (a scan
    // of the per-warp counts) and in earlier lanes of its warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < n_inst; i0 += kCullThreads) {
        const int i = i0 + threadIdx.x;
        const int g = i < n_inst ? __ldcg(grp + i) : kHidden;
        const unsigned peers = __match_any_sync(0xffffffffu, g);
        for (int k = lane; k < n_grp; k += 32) wcount[warp][k] = 0;
        __syncwarp();
        if (g != kHidden && lane == __ffs(peers) - 1) wcount[warp][g] = __popc(peers);
        __syncthreads();
        for (int k = threadIdx.x; k < n_grp; k += kCullThreads) {
            int run = gslot[k];
#pragma unroll 8
            for (int w = 0; w < kCullThreads / 32; ++w) {
                const int c = wcount[w][k];
                wcount[w][k] = run;
                run += c;
            }
            gslot[k] = run;
        }
        __syncthreads();
        if (g != kHidden) vis[wcount[warp][g] + __popc(peers & ((1u << lane) - 1u))] = i;
        __syncthreads();  // wcount and gslot are rewritten by the next round
    }
}

size_t cull_scratch_words(size_t n_inst) { return kMaxGroups + 3 + (n_inst + 3) / 4; }

int launch_cull_group(int n_inst, int n_tpl, const int32_t *tid, const float *root,
                       const TemplateInfo *tpls, const CamParams &cam, const LodParams &lod,
                       int do_cull, float *V, float *Cloc, int32_t *vis, Group *groups,
                       int32_t *meta, int32_t *scratch, cudaStream_t st) {
    if (cudaMemsetAsync(scratch, 0, (kMaxGroups + 3) * sizeof(int32_t), st) != cudaSuccess) return -1;
    const unsigned blocks = (unsigned)((n_inst + kCullThreads - 1) / kCullThreads);
    k_cull_group<<<blocks > 0 ? blocks : 1u, kCullThreads, 0, st>>>(
        n_inst, n_tpl, tid, root, tpls, cam, lod, do_cull, V, Cloc, vis, groups, meta, scratch,
        reinterpret_cast<uint8_t *>(scratch + kMaxGroups + 3));
    return 1;
}

// ---------------------------------------------------------------------------
// fused LBS + EWA projection + SH colour: one thread per splat
// ---------------------------------------------------------------------------

// Real SH basis to degree 3 (3DGS sign convention, degree 1 = C1 (-y, z, -x)),
// constants from their closed forms.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    const float C0 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
    const float C1 = 0.4886025119029199f;   // sqrt(3 / (4 pi))
    Y[0] = C0;
    if (deg < 1) return;
    Y[1] = -C1 * y;
    Y[2] = C1 * z;
    Y[3] = -C1 * x;
    if (deg < 2) return;
    const float A2 = 1.0925484305920792f;   // sqrt(15 / pi) / 2
    const float B2 = 0.31539156525252005f;  // sqrt(5 / pi) / 4
    const float E2 = 0.5462742152960396f;   // sqrt(15 / pi) / 4
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = A2 * x * y;
    Y[5] = -A2 * y * z;
    Y[6] = B2 * (2.0f * zz - xx - yy);
    Y[7] = -A2 * x * z;
    Y[8] = E2 * (xx - yy);
    if (deg < 3) return;
    const float K0 = 0.5900435899266435f;  // sqrt(35 / (2 pi)) / 4
    const float K1 = 2.890611442640554f;   // sqrt(105 / pi) / 2
    const float K2 = 0.4570457994644658f;  // sqrt(21 / (2 pi)) / 4
    const float K3 = 0.3731763325901154f;  // sqrt(7 / pi) / 4
    const float K5 = 1.445305721320277f;   // sqrt(105 / pi) / 4
    Y[9] = -K0 * y * (3.0f * xx - yy);
    Y[10] = K1 * x * y * z;
    Y[11] = -K2 * y * (4.0f * zz - xx - yy);
    Y[12] = K3 * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -K2 * x * (4.0f * zz - xx - yy);
    Y[14] = K5 * z * (xx - yy);
    Y[15] = -K0 * x * (xx - 3.0f * yy);
}

template <int DEG>
__device__ __forceinline__ void sh_colour(const float4 *__restrict__ sh, int64_t base, int n,
                                          float dx, float dy, float dz, float rgb[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int P = (K * 3 + 3) / 4;
    float Y[16];
    sh_basis(DEG, dx, dy, dz, Y);
    float c[P * 4];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float4 v = __ldg(sh + base + (int64_t)p * n);
        c[p * 4 + 0] = v.x;
        c[p * 4 + 1] = v.y;
        c[p * 4 + 2] = v.z;
        c[p * 4 + 3] = v.w;
    }
    float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r += Y[k] * c[k * 3 + 0];
        g += Y[k] * c[k * 3 + 1];
        b += Y[k] * c[k * 3 + 2];
    }
    rgb[0] = fmaxf(r + 0.5f, 0.0f);
    rgb[1] = fmaxf(g + 0.5f, 0.0f);
    rgb[2] = fmaxf(b + 0.5f, 0.0f);
}

// The same with FP16 coefficient planes of 8 (BF16 template storage).
template <int DEG>
__device__ __forceinline__ void sh_colour16(const uint4 *__restrict__ sh, int64_t base, int n,
                                            float dx, float dy, float dz, float rgb[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int P = (K * 3 + 7) / 8;
    float Y[16];
    sh_basis(DEG, dx, dy, dz, Y);
    float c[P * 8];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const uint4 v = __ldg(sh + base + (int64_t)p * n);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
            c[p * 8 + 2 * e] = f.x;
            c[p * 8 + 2 * e + 1] = f.y;
        }
    }
    float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r += Y[k] * c[k * 3 + 0];
        g += Y[k] * c[k * 3 + 1];
        b += Y[k] * c[k * 3 + 2];
    }
    rgb[0] = fmaxf(r + 0.5f, 0.0f);
    rgb[1] = fmaxf(g + 0.5f, 0.0f);
    rgb[2] = fmaxf(b + 0.5f, 0.0f);
}

constexpr int kProjThreads = 256;

// ---------------------------------------------------------------------------
// LBS blend on the tensor cores (BF16 template storage).  For the CTA's 256
// Gaussians of one instance, M[256 x 12] = W[256 x 32] Bt^T, W the dense
// skinning weights (joints 24..31 zero) and Bt[12 x 32] the instance's 24
// skinning transforms (row e = matrix entry e of every joint).  The weights
// are BF16 as stored, so W is exact in BF16; the transforms are split into
// BF16 hi + lo parts (split-BF16: W Bt_hi^T + W Bt_lo^T; the third product
// of bf16x3, W_lo Bt_hi^T, vanishes because W_lo = 0), accumulated in FP32
// by mma.sync m16n8k16, then divided by the sum of the four weights.  Fragment layout of mma.m16n8k16 with lane =
// 4 g + q: A regs {A[g][2q..], A[g+8][2q..], A[g][2q+8..], A[g+8][2q+8..]},
// B regs {B[2q..][g], B[2q+8..][g]}, C {C[g][2q], C[g][2q+1], C[g+8][2q],
// C[g+8][2q+1]}.  Every thread of the CTA must call it.
// ---------------------------------------------------------------------------
constexpr int kTcLd = 40;  // bf16 row stride of W and Bt (80 B: conflict-free fragment loads)
constexpr int kTcMld = 13; // float row stride of the result
constexpr int kSkinTcBytes = (kProjThreads * kTcLd + 2 * 16 * kTcLd) * 2;  // 23,040 B
static_assert(kProjThreads * kTcMld * 4 <= kProjThreads * kTcLd * 2, "result aliases W");

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ void skin_blend_tc(const float4 *__restrict__ sB, const float w_in[4], uint32_t joints, bool valid,
                              unsigned char *__restrict__ smem, float M[12]) {
    __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sBh = sW + kProjThreads * kTcLd;
    __nv_bfloat16 *sBl = sBh + 16 * kTcLd;
    float *sM = reinterpret_cast<float *>(smem);
    const int t = threadIdx.x;
    // this thread's row of W: zeros, then its weights (a repeated joint adds up)
    {
        uint4 *row = reinterpret_cast<uint4 *>(sW + t * kTcLd);
#pragma unroll
        for (int i = 0; i < 4; ++i) row[i] = make_uint4(0u, 0u, 0u, 0u);
        float wk[4] = {w_in[0], w_in[1], w_in[2], w_in[3]};
        int jk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) jk[k] = (joints >> (8 * k)) & 0xFF;
#pragma unroll
        for (int k = 1; k < 4; ++k)
#pragma unroll
            for (int k2 = 0; k2 < k; ++k2)
                if (jk[k] >= 0 && jk[k2] == jk[k]) {
                    wk[k2] += wk[k];
                    jk[k] = -1;
                }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (valid && jk[k] >= 0 && jk[k] < kJoints) sW[t * kTcLd + jk[k]] = __float2bfloat16_rn(wk[k]);
    }
    // Bt hi and lo: entry e of joint j, zero beyond 12 entries and 24 joints
    for (int i = t; i < 16 * 32; i += kProjThreads) {
        const int e = i >> 5, j = i & 31;
        float v = 0.0f;
        if (e < 12 && j < kJoints) {
            const float4 b = sB[j * 3 + (e >> 2)];
            const int c = e & 3;
            v = c == 0 ? b.x : (c == 1 ? b.y : (c == 2 ? b.z : b.w));
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        sBh[e * kTcLd + j] = hi;
        sBl[e * kTcLd + j] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    __syncthreads();
    const int warp = t >> 5, lane = t & 31, g = lane >> 2, q = lane & 3;
    float acc[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 32 * warp + 16 * mt;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const __nv_bfloat16 *ap = sW + (r0 + g) * kTcLd + 16 * kk + 2 * q;
            const uint32_t a[4] = {lds32(ap), lds32(ap + 8 * kTcLd), lds32(ap + 8), lds32(ap + 8 * kTcLd + 8)};
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int bo = (8 * nt + g) * kTcLd + 16 * kk + 2 * q;
                mma_bf16_16816(acc[mt][nt], a, lds32(sBh + bo), lds32(sBh + bo + 8));
                mma_bf16_16816(acc[mt][nt], a, lds32(sBl + bo), lds32(sBl + bo + 8));
            }
        }
    }
    __syncthreads();  // W and Bt consumed: the result overwrites W
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int r = 32 * warp + 16 * mt + g, c = 8 * nt + 2 * q;
            if (c < 12) {
                sM[r * kTcMld + c] = acc[mt][nt][0];
                sM[(r + 8) * kTcMld + c] = acc[mt][nt][2];
            }
            if (c + 1 < 12) {
                sM[r * kTcMld + c + 1] = acc[mt][nt][1];
                sM[(r + 8) * kTcMld + c + 1] = acc[mt][nt][3];
            }
        }
    __syncthreads();
    // BF16 weights need not sum to 1: normalise the blend, so that the root
    // transform applied afterwards stays rigid
    const float wsum = w_in[0] + w_in[1] + w_in[2] + w_in[3];
    const float iw = wsum > 0.0f ? 1.0f / wsum : 0.0f;
#pragma unroll
    for (int e = 0; e < 12; ++e) M[e] = sM[t * kTcMld + e] * iw;
}

// The FP32 path stages joint j's transform (12 floats) at word j * kSbwLd
// of shared memory: 13 is odd, so the joints of a warp's 32 lanes fall in
// distinct banks and every 4-byte load of the blend is conflict free (16-byte
// loads of 3 rows per joint would put up to 9 joints in one bank group).
constexpr int kSbwLd = 13;

// Records of a 256-splat chunk staged in shared memory as four planes
// (plane k holds float4 k of every splat; rows padded by two float4 so that
// the transposing reads hit every bank group equally), then written out as
// one contiguous block: each warp store covers 512 consecutive bytes instead
// of one 16-byte piece of 32 different records.
constexpr int kSrecLd = kProjThreads + 2;

// Gaussians chunk * 256 + t of one visible instance (thread t), with the
// instance's 24 skinning transforms staged in shared memory (sB).  Splat ids
// are dense, grouped by (template, level), instance-major within a group.
template <int kStore>
__device__ __forceinline__ void project_chunk(
    const ProjGroup &G, int islot, int chunk, int inst, const float4 *__restrict__ sB, const float *__restrict__ sBw,
    const float4 *__restrict__ sV, unsigned char *s_tc,
    const float *__restrict__ Vm, const float *__restrict__ root, const TemplateArrays &ta,
    const TemplateInfo *__restrict__ tpls, const CamParams &cam, const LodParams &lod, int skin_mode, int sh_frame, float4 *__restrict__ rec, uint32_t *__restrict__ key,
    uint32_t *__restrict__ bin, float4 *srec, uint8_t *slive) {
    const int gg = chunk * kProjThreads + threadIdx.x;
    const bool valid = gg < G.ng;
    // the tensor-core blend needs every thread of the CTA
    if (kStore == kStoreFp32 && !valid) return;
    const int s = G.splat0 + islot * G.ng + gg;
    // the level's Gaussians: a prefix of the template, or a chosen subset
    int gsrc = 0, gi = 0;
    if (valid) {
        gsrc = G.sub >= 0 ? (int)__ldg(ta.lod_idx + G.sub + gg) : gg;
        gi = G.g_off + gsrc;
    }

    // LBS (CrowdSplat Sec. 2): M = sum_k w_k B_{idx_k} (instance local)
    float M[12];
    float4 mo;        // mean (template local), opacity
    float cv[6];      // canonical covariance xx, xy, xz, yy, yz, zz
    if constexpr (kStore == kStoreBf16) {
        const uint4 qa = valid ? __ldg(ta.qa + gi) : make_uint4(0u, 0u, 0u, 0u);
        const uint4 qb = valid ? __ldg(ta.qb + gi) : make_uint4(0u, 0u, 0u, 0u);
        const float wq[4] = {bf16_lo(qb.y), bf16_hi(qb.y), bf16_lo(qb.z), bf16_hi(qb.z)};
        skin_blend_tc(sB, wq, qb.w, valid, s_tc, M);
        if (!valid) return;
        const int j0 = qb.w & 0xFF;
        const float *rest = tpls[G.tpl].rest;
        mo = make_float4(rest[j0 * 3] + bf16_lo(qa.x), rest[j0 * 3 + 1] + bf16_hi(qa.x),
                         rest[j0 * 3 + 2] + bf16_lo(qa.y), bf16_hi(qa.y));
        cv[0] = bf16_lo(qa.z); cv[1] = bf16_hi(qa.z); cv[2] = bf16_lo(qa.w); cv[3] = bf16_hi(qa.w);
        cv[4] = bf16_lo(qb.x); cv[5] = bf16_hi(qb.x);
    } else {
        const float4 w = __ldg(ta.skin_w + gi);
        const uint32_t packed = __ldg(ta.skin_i + gi);
        const float wk[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 12; ++e) M[e] = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // joint j's 12 entries at word j * kSbwLd: the 32 lanes of one
            // load read 32 different banks (or the same word)
            const float *b = sBw + ((packed >> (8 * k)) & 0xFF) * kSbwLd;
#pragma unroll
            for (int e = 0; e < 12; ++e) M[e] += wk[k] * b[e];
        }
        mo = __ldg(ta.mean_op + gi);
        // the covariance is loaded with the other attributes (one round of
        // L2 latency instead of two)
        const float4 ca = __ldg(ta.cov_a + gi);
        const float2 cb = __ldg(ta.cov_b + gi);
        cv[0] = ca.x; cv[1] = ca.y; cv[2] = ca.z; cv[3] = ca.w; cv[4] = cb.x; cv[5] = cb.y;
    }
    // view transform V = camera o root.  FP32 storage: M is already in
    // camera axes (the staged transforms are V_R B_j), only V's translation
    // is left to add; BF16 storage: M is instance local.
    float4 v0, v1, v2;
    float tx, ty, tz;
    if constexpr (kStore == kStoreFp32) {
        v0 = sV[0]; v1 = sV[1]; v2 = sV[2];
        tx = M[0] * mo.x + M[1] * mo.y + M[2] * mo.z + M[3] + v0.w;
        ty = M[4] * mo.x + M[5] * mo.y + M[6] * mo.z + M[7] + v1.w;
        tz = M[8] * mo.x + M[9] * mo.y + M[10] * mo.z + M[11] + v2.w;
    } else {
        const float lx = M[0] * mo.x + M[1] * mo.y + M[2] * mo.z + M[3];
        const float ly = M[4] * mo.x + M[5] * mo.y + M[6] * mo.z + M[7];
        const float lz = M[8] * mo.x + M[9] * mo.y + M[10] * mo.z + M[11];
        const float4 *Vi = reinterpret_cast<const float4 *>(Vm + (size_t)inst * 12);
        v0 = __ldg(Vi); v1 = __ldg(Vi + 1); v2 = __ldg(Vi + 2);
        tx = v0.x * lx + v0.y * ly + v0.z * lz + v0.w;
        ty = v1.x * lx + v1.y * ly + v1.z * lz + v1.w;
        tz = v2.x * lx + v2.y * ly + v2.z * lz + v2.w;
    }

    bool live = tz > cam.near_z;  // also false for NaN
    uint32_t nt = 0, bword = 0;
    if (live) {
        // covariance in camera space: Wc = (V_R A) (m^2 Sigma) (V_R A)^T,
        // A = the 3x3 part of M (full LBS) or identity (means only)
        float W[9];
        if (skin_mode == 0 && kStore == kStoreFp32) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) W[r * 3 + c] = M[r * 4 + c];
        } else if (skin_mode == 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float4 vr = r == 0 ? v0 : (r == 1 ? v1 : v2);
#pragma unroll
                for (int c = 0; c < 3; ++c) W[r * 3 + c] = vr.x * M[c] + vr.y * M[4 + c] + vr.z * M[8 + c];
            }
        } else {
            W[0] = v0.x; W[1] = v0.y; W[2] = v0.z;
            W[3] = v1.x; W[4] = v1.y; W[5] = v1.z;
            W[6] = v2.x; W[7] = v2.y; W[8] = v2.z;
        }
        const float m = lod.mult[G.lvl];
        const float m2 = m * m;
        const float S0 = cv[0] * m2, S1 = cv[1] * m2, S2 = cv[2] * m2, S3 = cv[3] * m2, S4 = cv[4] * m2,
                    S5 = cv[5] * m2;
        // EWA Jacobian at the mean, x/z and y/z clamped (3DGS)
        // hardware reciprocal and square root (relative error ~1e-7): far
        // inside the boundary windows the parity tests derive
        const float iz = __fdividef(1.0f, tz);
        const float txz = fminf(fmaxf(tx * iz, -cam.limx), cam.limx);
        const float tyz = fminf(fmaxf(ty * iz, -cam.limy), cam.limy);
        const float j00 = cam.fx * iz, j02 = -cam.fx * txz * iz;
        const float j11 = cam.fy * iz, j12 = -cam.fy * tyz * iz;
        // T = J W (2x3)
        const float t00 = j00 * W[0] + j02 * W[6], t01 = j00 * W[1] + j02 * W[7], t02 = j00 * W[2] + j02 * W[8];
        const float t10 = j11 * W[3] + j12 * W[6], t11 = j11 * W[4] + j12 * W[7], t12 = j11 * W[5] + j12 * W[8];
        // T Sigma (2x3), Sigma symmetric (S0 S1 S2; S1 S3 S4; S2 S4 S5)
        const float u00 = t00 * S0 + t01 * S1 + t02 * S2;
        const float u01 = t00 * S1 + t01 * S3 + t02 * S4;
        const float u02 = t00 * S2 + t01 * S4 + t02 * S5;
        const float u10 = t10 * S0 + t11 * S1 + t12 * S2;
        const float u11 = t10 * S1 + t11 * S3 + t12 * S4;
        const float u12 = t10 * S2 + t11 * S4 + t12 * S5;
        const float a = u00 * t00 + u01 * t01 + u02 * t02 + 0.3f;
        const float b = u00 * t10 + u01 * t11 + u02 * t12;
        const float c = u10 * t10 + u11 * t11 + u12 * t12 + 0.3f;
        const float det = a * c - b * b;
        live = det > 0.0f;
        if (live) {
            const float idet = __fdividef(1.0f, det);
            const float cA = c * idet, cB = -b * idet, cC = a * idet;
            const float mid = 0.5f * (a + c);
            const float disc = fmaxf(0.1f, mid * mid - det);
            const float lam = mid + disc * rsqrtf(disc);
            const float r = ceilf(3.0f * lam * rsqrtf(lam));
            const float u = cam.fx * tx * iz + cam.cx;
            const float v = cam.fy * ty * iz + cam.cy;
            // pixels with centre inside the support box, clipped to the image
            const float fcut = splat_fcut(mo.w);
            live = r > 0.0f && fcut >= 0.0f && isfinite(u) && isfinite(v) && isfinite(r) && isfinite(cA) &&
                   isfinite(cB) && isfinite(cC);
            int ax0 = 0, ax1 = -1, ay0 = 0, ay1 = -1;
            if (live) {
                // pixel range where alpha can reach 1/255 (ellipse extent)
                // inside the support box: both are centred on the mean, so
                // their intersection is the box of the smaller half-width
                box_range(u, fminf(ellipse_reach(fcut, a), r), cam.ox, cam.W, ax0, ax1);
                box_range(v, fminf(ellipse_reach(fcut, c), r), cam.oy, cam.H, ay0, ay1);
                // the tiles the reach box meets: a 3x3 window of them is kept
                // as a mask (bin word), larger boxes as a count
                if (ax0 <= ax1 && ay0 <= ay1) {
                    const int wx0 = ax0 >> 4, wy0 = ay0 >> 4;
                    const int nx = (ax1 >> 4) - wx0 + 1, ny = (ay1 >> 4) - wy0 + 1;
                    nt = (uint32_t)(nx * ny);
                    if (nx <= 3 && ny <= 3) {
                        const uint32_t row = (1u << nx) - 1u;
                        const uint32_t mask = row | (ny > 1 ? row << 3 : 0u) | (ny > 2 ? row << 6 : 0u);
                        bword = (uint32_t)wx0 | ((uint32_t)wy0 << 8) | (mask << 16);
                    } else {
                        bword = kBinLarge | nt;
                    }
                }
            }
            live = live && nt > 0;
            if (live) {
                // colour: SH at the viewing direction (camera centre -> mean)
                // in the instance's root frame: V_R^T t (V is rigid, the
                // camera centre is at the origin of camera space)
                float ddx = v0.x * tx + v1.x * ty + v2.x * tz;
                float ddy = v0.y * tx + v1.y * ty + v2.y * tz;
                float ddz = v0.z * tx + v1.z * ty + v2.z * tz;
                if (sh_frame == 1) {
                    const float *rt = root + (size_t)inst * 12;
                    const float wx = rt[0] * ddx + rt[1] * ddy + rt[2] * ddz;
                    const float wy = rt[4] * ddx + rt[5] * ddy + rt[6] * ddz;
                    const float wz = rt[8] * ddx + rt[9] * ddy + rt[10] * ddz;
                    ddx = wx; ddy = wy; ddz = wz;
                }
                const float inv = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
                ddx *= inv; ddy *= inv; ddz *= inv;
                float rgb[3];
                const int64_t base = G.sh_off + gsrc;
                if constexpr (kStore == kStoreBf16) {
                    switch (G.sh_deg) {
                        case 0: sh_colour16<0>(ta.sh16, base, G.n, ddx, ddy, ddz, rgb); break;
                        case 1: sh_colour16<1>(ta.sh16, base, G.n, ddx, ddy, ddz, rgb); break;
                        case 2: sh_colour16<2>(ta.sh16, base, G.n, ddx, ddy, ddz, rgb); break;
                        default: sh_colour16<3>(ta.sh16, base, G.n, ddx, ddy, ddz, rgb); break;
                    }
                } else {
                    switch (G.sh_deg) {
                        case 0: sh_colour<0>(ta.sh, base, G.n, ddx, ddy, ddz, rgb); break;
                        case 1: sh_colour<1>(ta.sh, base, G.n, ddx, ddy, ddz, rgb); break;
                        case 2: sh_colour<2>(ta.sh, base, G.n, ddx, ddy, ddz, rgb); break;
                        default: sh_colour<3>(ta.sh, base, G.n, ddx, ddy, ddz, rgb); break;
                    }
                }
                const float4 r0 = make_float4(__uint_as_float((uint32_t)ax0 | ((uint32_t)ax1 << 16)),
                                              __uint_as_float((uint32_t)ay0 | ((uint32_t)ay1 << 16)),
                                              __log2f(mo.w), cC);
                const float4 r1 = make_float4(u, v, cA, cB);
                const float4 r2 = make_float4(rgb[0], rgb[1], rgb[2], r);
                if (srec) {
                    // staged: the CTA writes the chunk's records out coalesced
                    const int t = threadIdx.x;
                    srec[0 * kSrecLd + t] = r0;
                    srec[1 * kSrecLd + t] = r1;
                    srec[2 * kSrecLd + t] = r2;
                    slive[t] = 1;
                } else if (in_bounds((uint32_t)s < cam.n_splats, kChkRecord)) {
                    float4 *ro = rec + (size_t)s * kRecVec;
                    ro[0] = r0;
                    ro[1] = r1;
                    ro[2] = r2;
                }
            }
        }
    }
    if (!in_bounds((uint32_t)s < cam.n_splats, kChkRecord)) return;
    key[s] = live ? min(max(__float_as_uint(tz), cam.key_lo), cam.key_hi) - cam.key_lo : 0xFFFFFFFFu;
    bin[s] = live ? bword : 0u;
}

// Projection CTAs: kChunks consecutive virtual blocks each (8 with FP32
// storage), a virtual block being 256 Gaussians of one visible instance
// (cull_group numbers them: Group::block0).  Consecutive virtual blocks
// mostly belong to one instance, whose transforms are then staged once.  kChunks = 1 for BF16 storage (its
// tensor-core blend reuses shared memory between barriers).
template <int kStore, int kChunks>
__global__ void __launch_bounds__(kProjThreads, 5) k_project(
    const Group *__restrict__ groups, int n_groups, int n_vblocks, const int32_t *__restrict__ vis,
    const float *__restrict__ Bm, const float *__restrict__ Vm, const float *__restrict__ root, TemplateArrays ta, const TemplateInfo *__restrict__ tpls,
    CamParams cam, LodParams lod, int skin_mode, int sh_frame, float4 *__restrict__ rec,
    uint32_t *__restrict__ key, uint32_t *__restrict__ bin, const __grid_constant__ ProjGroups pg) {
    static_assert(kStore == kStoreFp32 || kChunks == 1, "the BF16 blend needs one chunk per CTA");
    __shared__ float4 sB[kStore == kStoreBf16 ? kJoints * 3 : 1];         // skinning transforms B_j (BF16 storage)
    __shared__ float sBw[kStore == kStoreFp32 ? kJoints * kSbwLd : 1];   // V_R B_j (FP32 storage)
    __shared__ float4 sV[3];            // V = camera o root, rows
    __shared__ int s_group[kChunks];
    __shared__ __align__(16) unsigned char s_tc[kStore == kStoreBf16 ? kSkinTcBytes : 16];
    __shared__ float4 s_rec[kStore == kStoreFp32 ? kRecVec * kSrecLd : 1];
    __shared__ uint8_t s_live[kStore == kStoreFp32 ? kProjThreads : 1];
    if (threadIdx.x < 32) {
        // group of each virtual block: the last group with block0 <= vb
        // (block0 ascends from 0), counted by ballots
#pragma unroll
        for (int j = 0; j < kChunks; ++j) {
            const int vb = (int)blockIdx.x * kChunks + j;
            int cnt = 0;
            for (int g0 = 0; g0 < n_groups; g0 += 32) {
                const int g = g0 + (int)threadIdx.x;
                cnt += __popc(__ballot_sync(0xffffffffu, g < n_groups && groups[g].block0 <= vb));
            }
            if (threadIdx.x == 0) s_group[j] = max(cnt - 1, 0);
        }
    }
    __syncthreads();
    int staged = -1;
#pragma unroll 1
    for (int j = 0; j < kChunks; ++j) {
        const int vb = (int)blockIdx.x * kChunks + j;
        if (vb >= n_vblocks) break;
        const ProjGroup &G = pg.g[s_group[j]];
        const int per_inst = (G.ng + kProjThreads - 1) / kProjThreads;
        const int rb = vb - G.block0;
        const int islot = rb / per_inst;
        const int chunk = rb - islot * per_inst;
        const int inst = vis[G.slot0 + islot];
        if (inst != staged) {
            if (j > 0) __syncthreads();  // the previous chunk is done with sB
            const float4 *Bi = reinterpret_cast<const float4 *>(Bm + (size_t)inst * kJoints * 12);
            const float4 *Vi = reinterpret_cast<const float4 *>(Vm + (size_t)inst * 12);
            const int t = (int)threadIdx.x;
            if (kStore == kStoreFp32 && t < kJoints * 3) {
                // row r of V_R B_j: the joint transform in camera axes, without
                // V's translation (the blend stays at instance scale)
                const int jj = t / 3, r = t - 3 * jj;
                const float4 vr = __ldg(Vi + r);
                const float4 b0 = __ldg(Bi + jj * 3), b1 = __ldg(Bi + jj * 3 + 1), b2 = __ldg(Bi + jj * 3 + 2);
                float *o = sBw + jj * kSbwLd + 4 * r;
                o[0] = vr.x * b0.x + vr.y * b1.x + vr.z * b2.x;
                o[1] = vr.x * b0.y + vr.y * b1.y + vr.z * b2.y;
                o[2] = vr.x * b0.z + vr.y * b1.z + vr.z * b2.z;
                o[3] = vr.x * b0.w + vr.y * b1.w + vr.z * b2.w;
            } else if (kStore == kStoreBf16 && t < kJoints * 3) {
                sB[t] = __ldg(Bi + t);
            } else if (t >= kJoints * 3 && t < kJoints * 3 + 3) {
                sV[t - kJoints * 3] = __ldg(Vi + (t - kJoints * 3));
            }
            __syncthreads();
            staged = inst;
        }
        if (kStore == kStoreFp32) {
            s_live[threadIdx.x] = 0;
            project_chunk<kStore>(G, islot, chunk, inst, sB, sBw, sV, s_tc, Vm, root, ta, tpls, cam, lod,
                                  skin_mode, sh_frame, rec, key, bin, s_rec, s_live);
            __syncthreads();
            // the chunk's records (live splats only), 16-byte piece o of the
            // block at o (splat o / kRecVec, piece o % kRecVec), consecutive
            // threads on consecutive pieces
            const size_t s0 = (size_t)G.splat0 + (size_t)islot * G.ng + (size_t)chunk * kProjThreads;
#pragma unroll
            for (int i = 0; i < kRecVec; ++i) {
                const int o = (int)threadIdx.x + i * kProjThreads;
                const int sl = o / kRecVec, k = o - sl * kRecVec;
                if (s_live[sl] && in_bounds(s0 + sl < cam.n_splats, kChkRecord))
                    rec[s0 * kRecVec + o] = s_rec[k * kSrecLd + sl];
            }
            __syncthreads();  // the staging buffers are reused by the next chunk
        } else {
            project_chunk<kStore>(G, islot, chunk, inst, sB, sBw, sV, s_tc, Vm, root, ta, tpls, cam, lod,
                                  skin_mode, sh_frame, rec, key, bin, nullptr, nullptr);
        }
    }
}

constexpr int kProjChunksFp32 = 8;

int launch_project(int n_blocks, const Group *groups, const Group *groups_host, int n_groups,
                   const TemplateInfo *tpl_host, const int32_t *vis, const float *B, const float *V,
                   const float *root, const TemplateArrays &ta, const TemplateInfo *tpls,
                   const CamParams &cam, const LodParams &lod, int skin_mode, int sh_frame, float4 *rec,
                   uint32_t *key, uint32_t *bin, cudaStream_t st) {
    if (n_blocks <= 0 || n_groups <= 0 || n_groups > kMaxGroups) return 0;
    ProjGroups pg;
    for (int i = 0; i < n_groups; ++i) {
        const Group &G = groups_host[i];
        const TemplateInfo &T = tpl_host[G.tpl];
        ProjGroup &P = pg.g[i];
        P.tpl = G.tpl;
        P.lvl = G.lvl;
        P.slot0 = G.slot0;
        P.ng = G.ng;
        P.splat0 = G.splat0;
        P.block0 = G.block0;
        P.g_off = T.g_off;
        P.n = T.n;
        P.sh_deg = T.sh_deg;
        P.sub = T.lod_idx_off[G.lvl];
        P.sh_off = T.sh_off;
    }
    if (ta.storage == kStoreBf16) {
        k_project<kStoreBf16, 1><<<n_blocks, kProjThreads, 0, st>>>(groups, n_groups, n_blocks, vis, B, V, root, ta,
                                                                   tpls, cam, lod, skin_mode, sh_frame, rec,
                                                                   key, bin, pg);
    } else {
        const int grid = (n_blocks + kProjChunksFp32 - 1) / kProjChunksFp32;
        k_project<kStoreFp32, kProjChunksFp32><<<grid, kProjThreads, 0, st>>>(
            groups, n_groups, n_blocks, vis, B, V, root, ta, tpls, cam, lod, skin_mode, sh_frame, rec, key,
            bin, pg);
    }
    return 1;
}

__global__ void __launch_bounds__(256) k_debug_rects(int n, const float4 *__restrict__ rec,
                                                     const uint32_t *__restrict__ bins, int W, int H, int ox,
                                                     int oy, uint2 *__restrict__ rect) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint2 rc = make_uint2(0u, 0u);
    if (bins[s] != 0u) {
        const float4 r1 = rec[(size_t)s * kRecVec + 1], r2 = rec[(size_t)s * kRecVec + 2];
        int px0, px1, py0, py1;
        box_range(r1.x, r2.w, ox, W, px0, px1);
        box_range(r1.y, r2.w, oy, H, py0, py1);
        rc = make_uint2((uint32_t)(px0 >> 4) | ((uint32_t)(py0 >> 4) << 16),
                        (uint32_t)(px1 >> 4) | ((uint32_t)(py1 >> 4) << 16));
    }
    rect[s] = rc;
}

// Debug view of the records: per splat the 16 floats {u, v, A, B}, {C,
// opacity, radius, depth}, {r, g, b, 0}, {reach x, reach y, fcut, log2
// opacity}; opacity from its logarithm (within an ulp), the depth from the
// depth key (exactly: float bits = key + key_lo), fcut as the projection
// computes it.  Thread per position i of the depth order.
__global__ void __launch_bounds__(256) k_debug_records(int n, const float4 *__restrict__ rec,
                                                       const uint32_t *__restrict__ sorted_keys,
                                                       const uint32_t *__restrict__ order, uint32_t key_lo,
                                                       float4 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = order[i], key = sorted_keys[i];
    if (key == 0xFFFFFFFFu) return;  // culled: no record
    const float4 q = rec[(size_t)s * kRecVec], a = rec[(size_t)s * kRecVec + 1], c = rec[(size_t)s * kRecVec + 2];
    const float o = exp2f(q.z);
    float4 *d = out + (size_t)s * 4;
    d[0] = a;
    d[1] = make_float4(q.w, o, c.w, __uint_as_float(key + key_lo));
    d[2] = make_float4(c.x, c.y, c.z, 0.0f);
    d[3] = make_float4(q.x, q.y, splat_fcut(o), q.z);
}

int launch_debug_records(int n_splats, const float4 *rec, const uint32_t *sorted_keys, const uint32_t *order,
                         uint32_t key_lo, float4 *out, cudaStream_t st) {
    if (n_splats <= 0) return 0;
    k_debug_records<<<(n_splats + 255) / 256, 256, 0, st>>>(n_splats, rec, sorted_keys, order, key_lo, out);
    return 1;
}

int launch_debug_rects(int n_splats, const float4 *rec, const uint32_t *bins, int W, int H, int ox, int oy,
                       uint2 *rect, cudaStream_t st) {
    if (n_splats <= 0) return 0;
    k_debug_rects<<<(n_splats + 255) / 256, 256, 0, st>>>(n_splats, rec, bins, W, H, ox, oy, rect);
    return 1;
}

// ---------------------------------------------------------------------------
// contribution statistics: per-splat sums -> per template Gaussian
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_contrib_to_template(int n_splats, const Group *__restrict__ groups,
                                                             int n_groups, const TemplateInfo *__restrict__ tpls,
                                                             const uint32_t *__restrict__ lod_idx,
                                                             const float *__restrict__ cs_,
                                                             float *__restrict__ ct) {
    __shared__ Group sg[kMaxTemplates * kMaxLevels];
    for (int g = threadIdx.x; g < n_groups; g += blockDim.x) sg[g] = groups[g];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_splats) return;
    const float c = cs_[s];
    if (c == 0.0f) return;
    int lo = 0, hi = n_groups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sg[mid].splat0 <= s) lo = mid; else hi = mid - 1;
    }
    const Group &G = sg[lo];
    const int gg = (s - G.splat0) % G.ng;
    const TemplateInfo &T = tpls[G.tpl];
    const int sub = T.lod_idx_off[G.lvl];
    const int gsrc = sub >= 0 ? (int)lod_idx[sub + gg] : gg;
    atomicAdd(ct + T.g_off + gsrc, c);
}

int launch_contrib_to_template(int n_splats, const Group *groups, int n_groups, const TemplateInfo *tpls,
                               const uint32_t *lod_idx, const float *contrib_splat, float *contrib_tmpl,
                               cudaStream_t st) {
    if (n_splats <= 0) return 0;
    k_contrib_to_template<<<(n_splats + 255) / 256, 256, 0, st>>>(n_splats, groups, n_groups, tpls, lod_idx,
                                                                  contrib_splat, contrib_tmpl);
    return 1;
}

CS_DEFINE_CHECK_READER(check_word_geometry)

}  // namespace cs
