// Gradients of a rendered frame: reverse-mode through compositing, EWA
// projection, SH colour, linear blend skinning and forward kinematics.
//
// The loss enters as dL/d(pixel RGBA).  Kernels, in order:
//   k_blend_backward     one CTA per chunk of kBwdChunk pairs of a 16x16
//                        tile's list: each pixel walks its contributors in
//                        the chunk back to front (recomputing alpha, and the
//                        transmittance from the state the forward kept at the
//                        chunk's end, or from its final state), producing
//                        dL/d(u, v, conic, opacity, rgb) per splat, summed
//                        over the tile's pixels before the atomic adds; the
//                        chunks of one list run in parallel
//   k_project_backward   one CTA per (instance, 256 Gaussians), like the
//                        forward projection: recompute, then the chain rule to
//                        the template mean, canonical covariance, opacity and
//                        SH coefficients (summed over instances) and to the
//                        instance's 24 skinning transforms (summed in shared
//                        memory per CTA)
//   k_fk_backward        one thread per instance: skinning transforms to the
//                        24 axis-angle joint rotations
//   k_cov_backward       one thread per template Gaussian: canonical
//                        covariance to scales and quaternion
// Every step differentiates the forward as written (3DGS conventions, the
// readings of the forward kernels); clamps (alpha at 0.99, the EWA x/z and
// y/z limits, colour at 0) pass no gradient where active, and the discrete
// decisions (support box, alpha >= 1/255, the stop rule, the radius) are held
// fixed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kBwdThreads = 256;
constexpr int kBlockW = kBlendBlockW, kBlockH = kBlendBlockH;  // the forward's pixels per warp

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// compositing backward
// ---------------------------------------------------------------------------

struct BwdShared {
    float4 s0[kBwdThreads];  // u, v, a', b' (forward's scaled conic)
    float4 s1[kBwdThreads];  // c', log2 o, radius, o
    float4 s2[kBwdThreads];  // r, g, b, -
    float4 s3[kBwdThreads];  // conic A, B, C, -
    uint32_t sid[kBwdThreads];
    uint8_t mask[kBwdThreads];
    float gsum[kBwdThreads][9];  // the batch's gradients summed over the CTA's warps
    uint32_t max_end;
};

// Backward chunks of each tile's list: ceil(n / kBwdChunk).
__global__ void __launch_bounds__(256) k_bwd_chunk_counts(int n_tiles, const uint2 *__restrict__ ranges,
                                                          uint32_t *__restrict__ cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) cnt[t] = (ranges[t].y - ranges[t].x + kBwdChunk - 1) / kBwdChunk;
}

__global__ void __launch_bounds__(kBwdThreads) k_blend_backward(
    int tiles_x, int W, int H, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
    const float4 *__restrict__ rec, const uint32_t *__restrict__ px_end, const float4 *__restrict__ px_fin,
    const float4 *__restrict__ px_bnd, const uint32_t *__restrict__ chunk0, int n_tiles,
    const float4 *__restrict__ dl_drgba, float4 *__restrict__ dsplat) {
    __shared__ BwdShared sh;
    __shared__ int s_tile;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // chunk w of the frame: the tile whose chunks [chunk0[t], chunk0[t + 1]) hold it
    const uint32_t w = blockIdx.x;
    if (w >= chunk0[n_tiles]) return;
    if (tid == 0) {
        int lo = 0, hi = n_tiles - 1;  // the last t with chunk0[t] <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (chunk0[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        s_tile = lo;
    }
    __syncthreads();
    const int tile = s_tile;
    const int tx0 = (tile % tiles_x) * kTile, ty0 = (tile / tiles_x) * kTile;
    // pixel layout of the forward: warp w covers an 8x4 block
    const int bx = (warp & 1) * kBlockW, by = (warp >> 1) * kBlockH;
    const int px = tx0 + bx + (lane % kBlockW), py = ty0 + by + (lane / kBlockW);
    const bool inside = px < W && py < H;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint2 rg0 = ranges[tile];
    // this chunk: pairs [a, b) of the tile's list
    const uint32_t a_lo = rg0.x + (w - chunk0[tile]) * kBwdChunk;
    const uint32_t b_hi = min(rg0.y, a_lo + kBwdChunk);
    const uint2 rg = make_uint2(a_lo, b_hi);
    uint32_t end = rg.x;
    float Tf = 1.0f;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    float T = 1.0f;                      // transmittance behind the current splat
    float Sr = 0.f, Sg = 0.f, Sb = 0.f;  // colour composited behind it
    if (inside) {
        const size_t p = (size_t)py * W + px;
        const uint32_t e = px_end[p];
        const float4 fin = px_fin[p];
        Tf = fin.w;
        g = dl_drgba[p];
        end = min(e, b_hi);
        if (e <= b_hi) {
            // the pixel's list ends in this chunk: the walk starts from its final state
            T = Tf;
        } else if (end > rg.x) {
            // it goes on past the chunk: the state the forward kept at b, and
            // the colour composited behind b (final minus in front of b)
            const float4 st = px_bnd[(size_t)(b_hi / kBwdChunk) * kBwdThreads + tid];
            T = st.w;
            Sr = fin.x - st.x;
            Sg = fin.y - st.y;
            Sb = fin.z - st.z;
        }
    }
    if (tid == 0) sh.max_end = rg.x;
    __syncthreads();
    atomicMax(&sh.max_end, end);
    __syncthreads();
    const uint32_t hi_all = sh.max_end;
    const uint32_t wbit = 1u << warp;
    for (uint32_t hi = hi_all; hi > rg.x;) {
        const uint32_t lo = hi - rg.x > (uint32_t)kBwdThreads ? hi - kBwdThreads : rg.x;
        const uint32_t nb = hi - lo;
        __syncthreads();  // the previous batch is consumed
        if ((uint32_t)tid < nb) {
            const uint32_t s = __ldg(pval + lo + tid);
            const float4 *r = rec + (size_t)s * kRecVec;
            const float4 q = __ldg(r), a = __ldg(r + 1), c = __ldg(r + 2);  // {rx, ry, log2 o, C}, {u, v, A, B}, {rgb, radius}
            sh.s0[tid] = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
            // 1 / opacity from its logarithm: only the opacity gradient uses it
            sh.s1[tid] = make_float4(-0.5f * kLog2e * q.w, q.z, c.w, exp2f(-q.z));
            sh.s2[tid] = c;
            sh.s3[tid] = make_float4(a.z, a.w, q.w, 0.f);
            sh.sid[tid] = s;
            const uint32_t rx = __float_as_uint(q.x), ry = __float_as_uint(q.y);
            const int x0 = (int)(rx & 0xFFFFu) - tx0, x1 = (int)(rx >> 16) - tx0;
            const int y0 = (int)(ry & 0xFFFFu) - ty0, y1 = (int)(ry >> 16) - ty0;
            uint32_t m = 0;
#pragma unroll
            for (int w = 0; w < kBwdThreads / 32; ++w) {
                const int wx = (w & 1) * kBlockW, wy = (w >> 1) * kBlockH;
                if (x0 <= wx + kBlockW - 1 && x1 >= wx && y0 <= wy + kBlockH - 1 && y1 >= wy) m |= 1u << w;
            }
            sh.mask[tid] = (uint8_t)m;
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) sh.gsum[tid][c] = 0.0f;
        __syncthreads();
        for (int j = (int)nb - 1; j >= 0; --j) {
            if (!(sh.mask[j] & wbit)) continue;  // uniform per warp
            const uint32_t pair = lo + (uint32_t)j;
            float gu = 0.f, gv = 0.f, gA = 0.f, gB = 0.f, gC = 0.f, go = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
            bool contributes = false;
            if (pair < end) {
                // the forward's tests, evaluated the same way
                const float4 a = sh.s0[j];
                const float4 b = sh.s1[j];
                const float dx = fpx - a.x, dy = fpy - a.y;
                if (fmaxf(fabsf(dx), fabsf(dy)) <= b.z) {
                    const float pq = dx * (a.z * dx + a.w * dy) + b.x * dy * dy;
                    if (pq <= 0.0f) {
                        const float araw = ex2_approx(pq + b.y);
                        const float alpha = fminf(0.99f, araw);
                        if (alpha >= (1.0f / 255.0f)) {
                            contributes = true;
                            const float4 c = sh.s2[j];
                            const float4 k = sh.s3[j];
                            // one reciprocal of 1 - alpha for the five quotients (off by
                            // an ulp from dividing each): the walk back divides T by it
                            // at every splat, so the chain waits on a multiply only
                            const float iom = 1.0f / (1.0f - alpha);
                            const float Tb = T * iom;  // transmittance in front of this splat
                            const float wgt = alpha * Tb;
                            gr = wgt * g.x;
                            gg = wgt * g.y;
                            gb = wgt * g.z;
                            // d pixel / d alpha: own colour minus what it hides, and the alpha channel
                            const float galpha = g.x * (c.x * Tb - Sr * iom) + g.y * (c.y * Tb - Sg * iom) +
                                                 g.z * (c.z * Tb - Sb * iom) + g.w * (Tf * iom);
                            Sr += c.x * wgt;
                            Sg += c.y * wgt;
                            Sb += c.z * wgt;
                            T = Tb;
                            if (araw < 0.99f) {
                                // alpha = o e^q: d alpha / d q = alpha, d alpha / d o = e^q
                                const float gq = galpha * araw;
                                go = galpha * araw * b.w;
                                gA = -0.5f * dx * dx * gq;
                                gB = -dx * dy * gq;
                                gC = -0.5f * dy * dy * gq;
                                gu = (k.x * dx + k.y * dy) * gq;
                                gv = (k.y * dx + k.z * dy) * gq;
                            }
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contributes)) {
                // the warp's sums of the nine gradients by a reduce-scatter
                // butterfly (16 shuffles instead of 9 x 5): at the step of
                // distance 16, 8, 4, 2 each lane keeps half of its values
                // and adds its partner's copy of that half; the step of
                // distance 1 completes the sum.  Lane l then holds gradient
                // (l >> 1) & 15, and nine lanes add theirs at once into the
                // batch's shared sums.
                float v[16] = {gu, gv, gA, gB, gC, go, gr, gg, gb, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int half = 8; half >= 1; half >>= 1) {
                    const bool upper = (lane & (2 * half)) != 0;
#pragma unroll
                    for (int i = 0; i < half; ++i) {
                        const float recv = __shfl_xor_sync(0xffffffffu, upper ? v[i] : v[i + half], 2 * half);
                        v[i] = (upper ? v[i + half] : v[i]) + recv;
                    }
                }
                v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                const int comp = (lane >> 1) & 15;
                if ((lane & 1) == 0 && comp < 9) atomicAdd(&sh.gsum[j][comp], v[0]);
            }
        }
        // one set of global adds per (tile, splat) instead of per warp
        __syncthreads();
        if ((uint32_t)tid < nb) {
            float *d = reinterpret_cast<float *>(dsplat + (size_t)sh.sid[tid] * 3);
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                const float x = sh.gsum[tid][c];
                if (x != 0.0f) atomicAdd(d + c, x);
            }
        }
        hi = lo;
    }
}

// ---------------------------------------------------------------------------
// projection backward
// ---------------------------------------------------------------------------

// Real SH basis to degree 3 (3DGS signs) and its gradient with respect to
// the (unnormalised) direction components, from the polynomials.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16], float dY[16][3]) {
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float A2 = 1.0925484305920792f, B2 = 0.31539156525252005f, E2 = 0.5462742152960396f;
    const float K0 = 0.5900435899266435f, K1 = 2.890611442640554f, K2 = 0.4570457994644658f;
    const float K3 = 0.3731763325901154f, K5 = 1.445305721320277f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.f;
        dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
    }
    Y[0] = C0;
    if (deg < 1) return;
    Y[1] = -C1 * y; dY[1][1] = -C1;
    Y[2] = C1 * z;  dY[2][2] = C1;
    Y[3] = -C1 * x; dY[3][0] = -C1;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = A2 * x * y;  dY[4][0] = A2 * y; dY[4][1] = A2 * x;
    Y[5] = -A2 * y * z; dY[5][1] = -A2 * z; dY[5][2] = -A2 * y;
    Y[6] = B2 * (2.f * zz - xx - yy); dY[6][0] = -2.f * B2 * x; dY[6][1] = -2.f * B2 * y; dY[6][2] = 4.f * B2 * z;
    Y[7] = -A2 * x * z; dY[7][0] = -A2 * z; dY[7][2] = -A2 * x;
    Y[8] = E2 * (xx - yy); dY[8][0] = 2.f * E2 * x; dY[8][1] = -2.f * E2 * y;
    if (deg < 3) return;
    Y[9] = -K0 * y * (3.f * xx - yy);
    dY[9][0] = -6.f * K0 * x * y; dY[9][1] = -3.f * K0 * (xx - yy);
    Y[10] = K1 * x * y * z;
    dY[10][0] = K1 * y * z; dY[10][1] = K1 * x * z; dY[10][2] = K1 * x * y;
    Y[11] = -K2 * y * (4.f * zz - xx - yy);
    dY[11][0] = 2.f * K2 * x * y; dY[11][1] = -K2 * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * K2 * y * z;
    Y[12] = K3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
    dY[12][0] = -6.f * K3 * x * z; dY[12][1] = -6.f * K3 * y * z; dY[12][2] = K3 * (6.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -K2 * x * (4.f * zz - xx - yy);
    dY[13][0] = -K2 * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * K2 * x * y; dY[13][2] = -8.f * K2 * x * z;
    Y[14] = K5 * z * (xx - yy);
    dY[14][0] = 2.f * K5 * x * z; dY[14][1] = -2.f * K5 * y * z; dY[14][2] = K5 * (xx - yy);
    Y[15] = -K0 * x * (xx - 3.f * yy);
    dY[15][0] = -3.f * K0 * (xx - yy); dY[15][1] = 6.f * K0 * x * y;
}

__global__ void __launch_bounds__(kBwdThreads) k_project_backward(
    const Group *__restrict__ groups, int n_groups, const int32_t *__restrict__ vis, const float *__restrict__ Bm,
    const float *__restrict__ Vm, const float *__restrict__ Cloc, const float *__restrict__ root, TemplateArrays ta,
    const TemplateInfo *__restrict__ tpls, CamParams cam, LodParams lod, int skin_mode, int sh_frame,
    const float4 *__restrict__ dsplat, float *__restrict__ g_mean, float *__restrict__ g_cov,
    float *__restrict__ g_opacity, float *__restrict__ g_sh, float *__restrict__ g_B) {
    __shared__ float4 sB[kJoints * 3];
    __shared__ float sgB[kJoints * 12];
    __shared__ int s_group;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_groups - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (groups[mid].block0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_group = lo;
    }
    for (int k = threadIdx.x; k < kJoints * 12; k += kBwdThreads) sgB[k] = 0.f;
    __syncthreads();
    const Group G = groups[s_group];
    const int per_inst = (G.ng + kBwdThreads - 1) / kBwdThreads;
    const int rb = (int)blockIdx.x - G.block0;
    const int islot = rb / per_inst;
    const int chunk = rb - islot * per_inst;
    const int inst = vis[G.slot0 + islot];
    {
        const float4 *Bi = reinterpret_cast<const float4 *>(Bm + (size_t)inst * kJoints * 12);
        for (int k = threadIdx.x; k < kJoints * 3; k += kBwdThreads) sB[k] = __ldg(Bi + k);
    }
    __syncthreads();
    const int gg = chunk * kBwdThreads + threadIdx.x;
    const int s = G.splat0 + islot * G.ng + gg;
    float4 d0 = make_float4(0.f, 0.f, 0.f, 0.f), d1 = d0, d2 = d0;
    if (gg < G.ng) {
        d0 = dsplat[(size_t)s * 3];
        d1 = dsplat[(size_t)s * 3 + 1];
        d2 = dsplat[(size_t)s * 3 + 2];
    }
    const bool any = d0.x != 0.f || d0.y != 0.f || d0.z != 0.f || d0.w != 0.f || d1.x != 0.f || d1.y != 0.f ||
                     d1.z != 0.f || d1.w != 0.f || d2.x != 0.f;
    if (any) {
        const TemplateInfo &T = tpls[G.tpl];
        const int sub = T.lod_idx_off[G.lvl];
        const int gsrc = sub >= 0 ? (int)__ldg(ta.lod_idx + sub + gg) : gg;
        const int gi = T.g_off + gsrc;
        // ---- recompute the forward ---------------------------------------
        const float4 w = __ldg(ta.skin_w + gi);
        const uint32_t packed = __ldg(ta.skin_i + gi);
        const float wk[4] = {w.x, w.y, w.z, w.w};
        int jk[4];
        float M[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) M[e] = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            jk[k] = (packed >> (8 * k)) & 0xFF;
            const float4 b0 = sB[jk[k] * 3 + 0], b1 = sB[jk[k] * 3 + 1], b2 = sB[jk[k] * 3 + 2];
            M[0] += wk[k] * b0.x; M[1] += wk[k] * b0.y; M[2] += wk[k] * b0.z; M[3] += wk[k] * b0.w;
            M[4] += wk[k] * b1.x; M[5] += wk[k] * b1.y; M[6] += wk[k] * b1.z; M[7] += wk[k] * b1.w;
            M[8] += wk[k] * b2.x; M[9] += wk[k] * b2.y; M[10] += wk[k] * b2.z; M[11] += wk[k] * b2.w;
        }
        const float4 mo = __ldg(ta.mean_op + gi);
        const float mu[3] = {mo.x, mo.y, mo.z};
        float pl[3];  // posed mean, instance local
#pragma unroll
        for (int r = 0; r < 3; ++r) pl[r] = M[r * 4] * mu[0] + M[r * 4 + 1] * mu[1] + M[r * 4 + 2] * mu[2] + M[r * 4 + 3];
        const float4 *Vi = reinterpret_cast<const float4 *>(Vm + (size_t)inst * 12);
        const float4 v0 = __ldg(Vi), v1 = __ldg(Vi + 1), v2 = __ldg(Vi + 2);
        const float VR[9] = {v0.x, v0.y, v0.z, v1.x, v1.y, v1.z, v2.x, v2.y, v2.z};
        const float tx = v0.x * pl[0] + v0.y * pl[1] + v0.z * pl[2] + v0.w;
        const float ty = v1.x * pl[0] + v1.y * pl[1] + v1.z * pl[2] + v1.w;
        const float tz = v2.x * pl[0] + v2.y * pl[1] + v2.z * pl[2] + v2.w;
        float Wm[9];  // V_R A (full skinning) or V_R (means only)
        if (skin_mode == 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    Wm[r * 3 + c] = VR[r * 3] * M[c] + VR[r * 3 + 1] * M[4 + c] + VR[r * 3 + 2] * M[8 + c];
        } else {
#pragma unroll
            for (int e = 0; e < 9; ++e) Wm[e] = VR[e];
        }
        const float4 ca = __ldg(ta.cov_a + gi);
        const float2 cb = __ldg(ta.cov_b + gi);
        const float m = lod.mult[G.lvl], m2 = m * m;
        const float Sg[9] = {ca.x * m2, ca.y * m2, ca.z * m2, ca.y * m2, ca.w * m2, cb.x * m2,
                             ca.z * m2, cb.x * m2, cb.y * m2};
        const float iz = __fdividef(1.0f, tz);
        const float rx = tx * iz, ry = ty * iz;
        const bool clx = rx < -cam.limx || rx > cam.limx, cly = ry < -cam.limy || ry > cam.limy;
        const float txz = fminf(fmaxf(rx, -cam.limx), cam.limx);
        const float tyz = fminf(fmaxf(ry, -cam.limy), cam.limy);
        const float J[6] = {cam.fx * iz, 0.f, -cam.fx * txz * iz, 0.f, cam.fy * iz, -cam.fy * tyz * iz};
        float Tm[6];  // J W
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Tm[r * 3 + c] = J[r * 3] * Wm[c] + J[r * 3 + 1] * Wm[3 + c] + J[r * 3 + 2] * Wm[6 + c];
        float TS[6];  // T Sigma
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) TS[r * 3 + c] = Tm[r * 3] * Sg[c] + Tm[r * 3 + 1] * Sg[3 + c] + Tm[r * 3 + 2] * Sg[6 + c];
        const float a = TS[0] * Tm[0] + TS[1] * Tm[1] + TS[2] * Tm[2] + 0.3f;
        const float b = TS[0] * Tm[3] + TS[1] * Tm[4] + TS[2] * Tm[5];
        const float c = TS[3] * Tm[3] + TS[4] * Tm[4] + TS[5] * Tm[5] + 0.3f;
        const float idet = 1.0f / (a * c - b * b);
        const float QA = c * idet, QB = -b * idet, QC = a * idet;
        // ---- conic -> 2D covariance: gK = -Q gQ Q ------------------------
        const float gQA = d0.z, gQB = 0.5f * d0.w, gQC = d1.x;  // symmetric matrix of dL/dQ
        // P = gQ Q
        const float P00 = gQA * QA + gQB * QB, P01 = gQA * QB + gQB * QC;
        const float P10 = gQB * QA + gQC * QB, P11 = gQB * QB + gQC * QC;
        const float gK00 = -(QA * P00 + QB * P10), gK01 = -(QA * P01 + QB * P11);
        const float gK11 = -(QB * P01 + QC * P11);
        // G2 = dL/dK as a symmetric matrix (K = T S T^T + 0.3 I)
        const float G00 = gK00, G01 = gK01, G11 = gK11;
        // gT = 2 G2 T S  (2x3)
        float gT[6];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            gT[cc] = 2.f * (G00 * TS[cc] + G01 * TS[3 + cc]);
            gT[3 + cc] = 2.f * (G01 * TS[cc] + G11 * TS[3 + cc]);
        }
        // gS = T^T G2 T (3x3)
        float gS[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float u0 = G00 * Tm[i] + G01 * Tm[3 + i], u1 = G01 * Tm[i] + G11 * Tm[3 + i];
#pragma unroll
            for (int j = 0; j < 3; ++j) gS[i * 3 + j] = u0 * Tm[j] + u1 * Tm[3 + j];
        }
        // T = J W: gJ = gT W^T, gW = J^T gT
        float gJ[6], gW[9];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) gJ[r * 3 + k] = gT[r * 3] * Wm[k * 3] + gT[r * 3 + 1] * Wm[k * 3 + 1] + gT[r * 3 + 2] * Wm[k * 3 + 2];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) gW[k * 3 + cc] = J[k] * gT[cc] + J[3 + k] * gT[3 + cc];
        // camera-space mean: the projection u, v and the Jacobian entries
        float gtx = d0.x * cam.fx * iz, gty = d0.y * cam.fy * iz;
        float gtz = -d0.x * cam.fx * tx * iz * iz - d0.y * cam.fy * ty * iz * iz;
        gtz += -gJ[0] * cam.fx * iz * iz - gJ[4] * cam.fy * iz * iz;
        if (!clx) {
            gtx += -gJ[2] * cam.fx * iz * iz;
            gtz += gJ[2] * 2.f * cam.fx * tx * iz * iz * iz;
        } else {
            gtz += gJ[2] * cam.fx * txz * iz * iz;
        }
        if (!cly) {
            gty += -gJ[5] * cam.fy * iz * iz;
            gtz += gJ[5] * 2.f * cam.fy * ty * iz * iz * iz;
        } else {
            gtz += gJ[5] * cam.fy * tyz * iz * iz;
        }
        // t = V_R p + V_t
        float gp[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) gp[i] = VR[i] * gtx + VR[3 + i] * gty + VR[6 + i] * gtz;
        // ---- colour: SH at the viewing direction --------------------------
        {
            const float4 cl = __ldg(reinterpret_cast<const float4 *>(Cloc) + inst);
            float e[3] = {pl[0] - cl.x, pl[1] - cl.y, pl[2] - cl.z};
            float Rf[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
            if (sh_frame == 1) {
                const float *rt = root + (size_t)inst * 12;
                Rf[0] = rt[0]; Rf[1] = rt[1]; Rf[2] = rt[2];
                Rf[3] = rt[4]; Rf[4] = rt[5]; Rf[5] = rt[6];
                Rf[6] = rt[8]; Rf[7] = rt[9]; Rf[8] = rt[10];
            }
            float ew[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) ew[i] = Rf[i * 3] * e[0] + Rf[i * 3 + 1] * e[1] + Rf[i * 3 + 2] * e[2];
            const float inv = rsqrtf(ew[0] * ew[0] + ew[1] * ew[1] + ew[2] * ew[2]);
            const float dd[3] = {ew[0] * inv, ew[1] * inv, ew[2] * inv};
            float Y[16], dY[16][3];
            sh_basis_grad(T.sh_deg, dd[0], dd[1], dd[2], Y, dY);
            const int K = (T.sh_deg + 1) * (T.sh_deg + 1);
            float pre[3] = {0.5f, 0.5f, 0.5f};
            float coef[48];
            for (int k = 0; k < K; ++k)
                for (int ch = 0; ch < 3; ++ch) {
                    const int f = 3 * k + ch;
                    const float4 v = __ldg(ta.sh + T.sh_off + (int64_t)(f >> 2) * T.n + gsrc);
                    const int q = f & 3;
                    coef[f] = q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
                    pre[ch] += Y[k] * coef[f];
                }
            // colour clamp at 0 passes no gradient
            const float grgb[3] = {pre[0] > 0.f ? d1.z : 0.f, pre[1] > 0.f ? d1.w : 0.f, pre[2] > 0.f ? d2.x : 0.f};
            float gd[3] = {0.f, 0.f, 0.f};
            float *gsh = g_sh + (size_t)gi * 48;
            for (int k = 0; k < K; ++k)
                for (int ch = 0; ch < 3; ++ch) {
                    const float gc = grgb[ch];
                    if (gc == 0.f) continue;
                    atomicAdd(gsh + 3 * k + ch, Y[k] * gc);
                    const float cf = coef[3 * k + ch] * gc;
                    gd[0] += cf * dY[k][0];
                    gd[1] += cf * dY[k][1];
                    gd[2] += cf * dY[k][2];
                }
            // d = ew / |ew|: gew = (gd - d (d . gd)) / |ew|, e = Rf^T ew
            const float dg = dd[0] * gd[0] + dd[1] * gd[1] + dd[2] * gd[2];
            float gew[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) gew[i] = (gd[i] - dd[i] * dg) * inv;
#pragma unroll
            for (int i = 0; i < 3; ++i) gp[i] += Rf[i] * gew[0] + Rf[3 + i] * gew[1] + Rf[6 + i] * gew[2];
        }
        // ---- LBS: p = M [mu; 1], W = V_R A --------------------------------
        float gM[12];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            gM[r * 4 + 0] = gp[r] * mu[0];
            gM[r * 4 + 1] = gp[r] * mu[1];
            gM[r * 4 + 2] = gp[r] * mu[2];
            gM[r * 4 + 3] = gp[r];
        }
        if (skin_mode == 0) {
            // gA = V_R^T gW
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    gM[r * 4 + cc] += VR[r] * gW[cc] + VR[3 + r] * gW[3 + cc] + VR[6 + r] * gW[6 + cc];
        }
        float gmu[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) gmu[cc] = M[cc] * gp[0] + M[4 + cc] * gp[1] + M[8 + cc] * gp[2];
        atomicAdd(g_mean + (size_t)gi * 3 + 0, gmu[0]);
        atomicAdd(g_mean + (size_t)gi * 3 + 1, gmu[1]);
        atomicAdd(g_mean + (size_t)gi * 3 + 2, gmu[2]);
        // canonical covariance (6 stored entries; off-diagonals count twice)
        float *gc = g_cov + (size_t)gi * 6;
        atomicAdd(gc + 0, m2 * gS[0]);
        atomicAdd(gc + 1, m2 * (gS[1] + gS[3]));
        atomicAdd(gc + 2, m2 * (gS[2] + gS[6]));
        atomicAdd(gc + 3, m2 * gS[4]);
        atomicAdd(gc + 4, m2 * (gS[5] + gS[7]));
        atomicAdd(gc + 5, m2 * gS[8]);
        atomicAdd(g_opacity + gi, d1.y);
        // skinning transforms of the instance: dB_j += w_j dM
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (wk[k] == 0.f) continue;
#pragma unroll
            for (int e = 0; e < 12; ++e) atomicAdd(&sgB[jk[k] * 12 + e], wk[k] * gM[e]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kJoints * 12; k += kBwdThreads) {
        const float v = sgB[k];
        if (v != 0.f) atomicAdd(g_B + (size_t)inst * kJoints * 12 + k, v);
    }
}

// ---------------------------------------------------------------------------
// forward kinematics backward
// ---------------------------------------------------------------------------

// R(v) by Rodrigues' formula, and dR/dv_i from the compact formula of
// Gallego and Yezzi, "A compact formula for the derivative of a 3-D rotation
// in exponential coordinates", J. Math. Imaging Vis. 51 (2015):
// dR/dv_i = (v_i [v]x + [v x ((I - R) e_i)]x) R / |v|^2, and the series
// [e_i]x + ([e_i]x [v]x + [v]x [e_i]x) / 2 for small |v|.
__device__ void rodrigues_grad(const float v[3], float R[9], float dR[3][9]) {
    const float th2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float K[9] = {0.f, -v[2], v[1], v[2], 0.f, -v[0], -v[1], v[0], 0.f};
    float K2[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) K2[i * 3 + j] = K[i * 3] * K[j] + K[i * 3 + 1] * K[3 + j] + K[i * 3 + 2] * K[6 + j];
    float a, b;
    if (th2 < 1e-12f) {
        a = 1.f;
        b = 0.5f;
    } else {
        const float th = sqrtf(th2);
        a = sinf(th) / th;
        const float h = sinf(0.5f * th) / th;
        b = 2.f * h * h;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) R[e] = (e % 4 == 0 ? 1.f : 0.f) + a * K[e] + b * K2[e];
    for (int i = 0; i < 3; ++i) {
        float E[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // [e_i]x
        if (i == 0) { E[5] = -1.f; E[7] = 1.f; }
        if (i == 1) { E[2] = 1.f; E[6] = -1.f; }
        if (i == 2) { E[1] = -1.f; E[3] = 1.f; }
        if (th2 < 1e-6f) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float ek = 0.f, ke = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        ek += E[r * 3 + k] * K[k * 3 + c];
                        ke += K[r * 3 + k] * E[k * 3 + c];
                    }
                    dR[i][r * 3 + c] = E[r * 3 + c] + 0.5f * (ek + ke);
                }
        } else {
            // w = v x ((I - R) e_i)
            const float col[3] = {(i == 0 ? 1.f : 0.f) - R[0 * 3 + i], (i == 1 ? 1.f : 0.f) - R[1 * 3 + i],
                                  (i == 2 ? 1.f : 0.f) - R[2 * 3 + i]};
            const float w[3] = {v[1] * col[2] - v[2] * col[1], v[2] * col[0] - v[0] * col[2], v[0] * col[1] - v[1] * col[0]};
            const float S[9] = {0.f, -(v[i] * v[2] + w[2]), v[i] * v[1] + w[1], v[i] * v[2] + w[2], 0.f,
                                -(v[i] * v[0] + w[0]), -(v[i] * v[1] + w[1]), v[i] * v[0] + w[0], 0.f};
            const float inv = 1.f / th2;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    dR[i][r * 3 + c] = (S[r * 3] * R[c] + S[r * 3 + 1] * R[3 + c] + S[r * 3 + 2] * R[6 + c]) * inv;
        }
    }
}

__global__ void k_fk_backward(int n_inst, int n_tpl, const int32_t *__restrict__ tid, const float *__restrict__ pose,
                              const TemplateInfo *__restrict__ tpls, const float *__restrict__ g_B,
                              float *__restrict__ g_pose) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    const int t = tid[inst];
    if (t < 0 || t >= n_tpl) return;
    const TemplateInfo &T = tpls[t];
    // forward: G_j = G_parent o [R_j | J_j - J_parent]
    float GR[kJoints][9], Gt[kJoints][3], Rj[kJoints][9], dRj[kJoints][3][9];
    for (int j = 0; j < kJoints; ++j) {
        const float v[3] = {pose[(size_t)inst * 72 + j * 3], pose[(size_t)inst * 72 + j * 3 + 1],
                            pose[(size_t)inst * 72 + j * 3 + 2]};
        rodrigues_grad(v, Rj[j], dRj[j]);
        const int p = T.parent[j];
        float o[3];
        for (int r = 0; r < 3; ++r) o[r] = T.rest[j * 3 + r] - (p >= 0 ? T.rest[p * 3 + r] : 0.f);
        if (p < 0) {
            for (int e = 0; e < 9; ++e) GR[j][e] = Rj[j][e];
            for (int r = 0; r < 3; ++r) Gt[j][r] = o[r];
        } else {
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c)
                    GR[j][r * 3 + c] = GR[p][r * 3] * Rj[j][c] + GR[p][r * 3 + 1] * Rj[j][3 + c] + GR[p][r * 3 + 2] * Rj[j][6 + c];
                Gt[j][r] = GR[p][r * 3] * o[0] + GR[p][r * 3 + 1] * o[1] + GR[p][r * 3 + 2] * o[2] + Gt[p][r];
            }
        }
    }
    // B_j = [G_R | G_t - G_R J_j]: dG_R = dB_R - dB_t J_j^T, dG_t = dB_t
    float gGR[kJoints][9], gGt[kJoints][3];
    for (int j = 0; j < kJoints; ++j) {
        const float *gb = g_B + ((size_t)inst * kJoints + j) * 12;
        const float J0 = T.rest[j * 3], J1 = T.rest[j * 3 + 1], J2 = T.rest[j * 3 + 2];
        for (int r = 0; r < 3; ++r) {
            const float gbt = gb[r * 4 + 3];
            gGR[j][r * 3 + 0] = gb[r * 4 + 0] - gbt * J0;
            gGR[j][r * 3 + 1] = gb[r * 4 + 1] - gbt * J1;
            gGR[j][r * 3 + 2] = gb[r * 4 + 2] - gbt * J2;
            gGt[j][r] = gbt;
        }
    }
    // children before parents (parents[j] < j)
    for (int j = kJoints - 1; j >= 0; --j) {
        const int p = T.parent[j];
        float gR[9];
        if (p < 0) {
            for (int e = 0; e < 9; ++e) gR[e] = gGR[j][e];
        } else {
            // G_R = G_pR R_j: gR_j = G_pR^T gG_R
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    gR[r * 3 + c] = GR[p][r] * gGR[j][c] + GR[p][3 + r] * gGR[j][3 + c] + GR[p][6 + r] * gGR[j][6 + c];
            float o[3];
            for (int r = 0; r < 3; ++r) o[r] = T.rest[j * 3 + r] - T.rest[p * 3 + r];
            // gG_pR += gG_R R_j^T + gG_t o^T; gG_pt += gG_t
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c)
                    gGR[p][r * 3 + c] += gGR[j][r * 3] * Rj[j][c * 3] + gGR[j][r * 3 + 1] * Rj[j][c * 3 + 1] +
                                         gGR[j][r * 3 + 2] * Rj[j][c * 3 + 2] + gGt[j][r] * o[c];
                gGt[p][r] += gGt[j][r];
            }
        }
        for (int i = 0; i < 3; ++i) {
            float acc = 0.f;
            for (int e = 0; e < 9; ++e) acc += gR[e] * dRj[j][i][e];
            g_pose[(size_t)inst * 72 + j * 3 + i] += acc;
        }
    }
}

// ---------------------------------------------------------------------------
// canonical covariance -> scales and quaternion
// ---------------------------------------------------------------------------

__global__ void k_cov_backward(int n, const float4 *__restrict__ scale, const float4 *__restrict__ quat,
                               const float *__restrict__ g_cov, float *__restrict__ g_scale, float *__restrict__ g_quat) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float *gc = g_cov + (size_t)g * 6;
    // dL/dSigma as a symmetric matrix (off-diagonal stored entries count twice)
    const float Gm[9] = {gc[0], 0.5f * gc[1], 0.5f * gc[2], 0.5f * gc[1], gc[3], 0.5f * gc[4],
                         0.5f * gc[2], 0.5f * gc[4], gc[5]};
    const float4 s4 = scale[g], q4 = quat[g];
    const float s[3] = {s4.x, s4.y, s4.z};
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x / qn, x = q4.y / qn, y = q4.z / qn, z = q4.w / qn;
    const float R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    // Sigma = R diag(s^2) R^T: ds_k = 2 s_k (R^T G R)_kk, dR = 2 G R diag(s^2)
    float GR[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) GR[i * 3 + k] = Gm[i * 3] * R[k] + Gm[i * 3 + 1] * R[3 + k] + Gm[i * 3 + 2] * R[6 + k];
    for (int k = 0; k < 3; ++k) {
        const float d = R[k] * GR[k] + R[3 + k] * GR[3 + k] + R[6 + k] * GR[6 + k];
        g_scale[(size_t)g * 3 + k] += 2.f * s[k] * d;
    }
    float gR[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) gR[i * 3 + k] = 2.f * GR[i * 3 + k] * s[k] * s[k];
    // R(w, x, y, z) of the normalised quaternion
    const float gw = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    const float gx = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                            2.f * x * gR[8]);
    const float gy = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                            2.f * y * gR[8]);
    const float gz = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] +
                            x * gR[6] + y * gR[7]);
    // through the normalisation q / |q|
    const float dot = w * gw + x * gx + y * gy + z * gz;
    g_quat[(size_t)g * 4 + 0] += (gw - w * dot) / qn;
    g_quat[(size_t)g * 4 + 1] += (gx - x * dot) / qn;
    g_quat[(size_t)g * 4 + 2] += (gy - y * dot) / qn;
    g_quat[(size_t)g * 4 + 3] += (gz - z * dot) / qn;
}

}  // namespace

int launch_backward(const BackwardArgs &a, cudaStream_t st) {
    int launched = 0;
    const int T = a.tiles_x * a.tiles_y;
    if (T > 0 && a.n_pairs > 0) {
        // chunks of kBwdChunk pairs per tile, numbered tile by tile; one CTA
        // per chunk walks it back to front from the state the forward kept
        k_bwd_chunk_counts<<<(T + 255) / 256, 256, 0, st>>>(T, a.ranges, a.chunk_cnt);
        launched += 1 + exclusive_scan(a.chunk_cnt, nullptr, a.chunk0, (uint32_t)T, a.scan_scratch, st);
        const unsigned grid = a.n_pairs / kBwdChunk + (unsigned)T;  // at least the chunks of the frame
        k_blend_backward<<<grid, kBwdThreads, 0, st>>>(a.tiles_x, a.W, a.H, a.ranges, a.pval, a.rec, a.px_end,
                                                        a.px_fin, a.px_bnd, a.chunk0, T, a.dl_drgba, a.dsplat);
        ++launched;
    }
    if (a.proj_blocks > 0) {
        k_project_backward<<<a.proj_blocks, kBwdThreads, 0, st>>>(
            a.groups, a.n_groups, a.vis, a.B, a.V, a.Cloc, a.root, a.ta, a.tpls, a.cam, a.lod, a.skin_mode,
            a.sh_frame, a.dsplat, a.g_mean, a.g_cov, a.g_opacity, a.g_sh, a.g_B);
        ++launched;
    }
    if (a.n_inst > 0) {
        k_fk_backward<<<(a.n_inst + 63) / 64, 64, 0, st>>>(a.n_inst, a.n_tpl, a.tid, a.pose, a.tpls, a.g_B, a.g_pose);
        ++launched;
    }
    if (a.n_gauss > 0) {
        k_cov_backward<<<(a.n_gauss + 255) / 256, 256, 0, st>>>(a.n_gauss, a.scale, a.quat, a.g_cov, a.g_scale,
                                                                 a.g_quat);
        ++launched;
    }
    return launched;
}

}  // namespace cs
