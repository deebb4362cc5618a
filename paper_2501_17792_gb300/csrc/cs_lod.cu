// Ranked level of detail: per-Gaussian features and the per-template ranking
// sort.  Both run once per template set, offline; nothing here is on the
// per-frame path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cs_internal.cuh"

namespace cs {

namespace {

__device__ __forceinline__ int template_of(const int32_t *__restrict__ g_off, int n_tpl, int g) {
    int lo = 0, hi = n_tpl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Eigenvalues of a symmetric 3x3 matrix, largest first: the trigonometric
// closed form of O. K. Smith, "Eigenvalues of a symmetric 3x3 matrix",
// Commun. ACM 4(4), 1961.
__device__ void sym3_eigenvalues(double a00, double a01, double a02, double a11, double a12, double a22,
                                 double ev[3]) {
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    const double q = (a00 + a11 + a22) / 3.0;
    const double d0 = a00 - q, d1 = a11 - q, d2 = a22 - q;
    const double p2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1;
    if (p2 <= 1e-300) {
        ev[0] = ev[1] = ev[2] = q;
        return;
    }
    const double p = sqrt(p2 / 6.0);
    // B = (A - q I) / p; r = det(B) / 2
    const double b00 = d0 / p, b11 = d1 / p, b22 = d2 / p;
    const double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
    const double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
    const double r = fmin(1.0, fmax(-1.0, 0.5 * det));
    const double phi = acos(r) / 3.0;
    const double two_pi_3 = 2.0943951023931954923;  // 2 pi / 3
    const double e1 = q + 2.0 * p * cos(phi);
    const double e3 = q + 2.0 * p * cos(phi + two_pi_3);
    ev[0] = e1;
    ev[1] = 3.0 * q - e1 - e3;
    ev[2] = e3;
}

template <int kStore>
__global__ void __launch_bounds__(256) k_lod_features(int n_total, int n_tpl, const TemplateInfo *__restrict__ tpls,
                                                      TemplateArrays ta, float *__restrict__ feat) {
    __shared__ int32_t s_off[kMaxTemplates];
    for (int t = threadIdx.x; t < n_tpl; t += blockDim.x) s_off[t] = tpls[t].g_off;
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    const int t = template_of(s_off, n_tpl, g);
    const TemplateInfo &T = tpls[t];
    const int gl = g - T.g_off;
    float f[kLodFeatures];
    // attributes as stored (BF16 storage: widened to FP32)
    float4 mo, ca, w;  // mean + opacity; covariance xx, xy, xz, yy; skinning weights
    float2 cb;         // covariance yz, zz
    uint32_t si;       // joint ids
    if constexpr (kStore == kStoreBf16) {
        const uint4 qa = ta.qa[g], qb = ta.qb[g];
        const int j0 = qb.w & 0xFF;
        mo = make_float4(T.rest[j0 * 3] + bf16_lo(qa.x), T.rest[j0 * 3 + 1] + bf16_hi(qa.x),
                         T.rest[j0 * 3 + 2] + bf16_lo(qa.y), bf16_hi(qa.y));
        ca = make_float4(bf16_lo(qa.z), bf16_hi(qa.z), bf16_lo(qa.w), bf16_hi(qa.w));
        cb = make_float2(bf16_lo(qb.x), bf16_hi(qb.x));
        w = make_float4(bf16_lo(qb.y), bf16_hi(qb.y), bf16_lo(qb.z), bf16_hi(qb.z));
        si = qb.w;
    } else {
        mo = ta.mean_op[g];
        ca = ta.cov_a[g];
        cb = ta.cov_b[g];
        w = ta.skin_w[g];
        si = ta.skin_i[g];
    }
    double ev[3];
    sym3_eigenvalues(ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, ev);
    double ls[3];
    for (int i = 0; i < 3; ++i) ls[i] = 0.5 * log(fmax(ev[i], 1e-20)) - log(0.01);
    const double o = mo.w;
    for (int i = 0; i < 3; ++i) f[i] = (float)ls[i];
    f[3] = (float)((ls[0] + ls[1] + ls[2]) / 3.0);
    f[4] = (float)(ls[0] - ls[2]);
    f[5] = (float)o;
    const double oc = fmin(fmax(o, 1e-6), 1.0 - 1e-6);
    f[6] = (float)fmin(2.0, fmax(-2.0, log(oc / (1.0 - oc)) / 4.0));
    // o sigma_1 sigma_2 / 1e-4 = o exp(ls0 + ls1)
    f[7] = (float)(log(fmax(o, 1e-12)) + ls[0] + ls[1]) / 4.0f;
    // colour: SH planes hold coefficient k, channel c at flat index 3k + c
    auto coeff = [&](int k, int c) -> double {
        const int fi = 3 * k + c;
        if constexpr (kStore == kStoreBf16) {
            const uint4 pl = ta.sh16[T.sh_off + (int64_t)(fi >> 3) * T.n + gl];
            const int e = fi & 7;
            const uint32_t wd = (e >> 1) == 0 ? pl.x : (e >> 1) == 1 ? pl.y : (e >> 1) == 2 ? pl.z : pl.w;
            return (double)__half2float(__ushort_as_half((unsigned short)(e & 1 ? wd >> 16 : wd & 0xFFFFu)));
        } else {
            const float4 pl = ta.sh[T.sh_off + (int64_t)(fi >> 2) * T.n + gl];
            const int e = fi & 3;
            return e == 0 ? pl.x : e == 1 ? pl.y : e == 2 ? pl.z : pl.w;
        }
    };
    double dc[3];
    for (int c = 0; c < 3; ++c) dc[c] = fmax(0.0, 0.28209479177387814 * coeff(0, c) + 0.5);
    for (int c = 0; c < 3; ++c) f[8 + c] = (float)dc[c];
    f[11] = (float)((dc[0] + dc[1] + dc[2]) / 3.0);
    for (int l = 1; l <= 3; ++l) {
        double ss = 0.0;
        int cnt = 0;
        if (l <= T.sh_deg) {
            for (int k = l * l; k < (l + 1) * (l + 1); ++k)
                for (int c = 0; c < 3; ++c) {
                    const double v = coeff(k, c);
                    ss += v * v;
                    ++cnt;
                }
        }
        f[11 + l] = cnt ? (float)(sqrt(ss / cnt) / 0.3) : 0.0f;
    }
    f[15] = mo.x;
    f[16] = mo.y;
    f[17] = mo.z;
    const double rx = mo.x - T.rest[0], rz = mo.z - T.rest[2];
    f[18] = (float)sqrt(rx * rx + rz * rz);
    float wv[4] = {w.x, w.y, w.z, w.w};
    int jv[4] = {(int)(si & 0xFF), (int)((si >> 8) & 0xFF), (int)((si >> 16) & 0xFF), (int)(si >> 24)};
    // sort the four weights, largest first (ties keep their slot order)
    for (int a = 1; a < 4; ++a)
        for (int b = a; b > 0 && wv[b] > wv[b - 1]; --b) {
            const float tw = wv[b]; wv[b] = wv[b - 1]; wv[b - 1] = tw;
            const int tj = jv[b]; jv[b] = jv[b - 1]; jv[b - 1] = tj;
        }
    for (int k = 0; k < 4; ++k) f[19 + k] = wv[k];
    const int j0 = jv[0];
    f[23] = (float)j0 / 23.0f;
    f[24] = T.max_depth > 0 ? (float)T.depth[j0] / (float)T.max_depth : 0.0f;
    const double dx = mo.x - T.rest[j0 * 3], dy = mo.y - T.rest[j0 * 3 + 1], dz = mo.z - T.rest[j0 * 3 + 2];
    f[25] = (float)(10.0 * sqrt(dx * dx + dy * dy + dz * dz));
    const double tr = fmax((double)ca.x + ca.w + cb.y, 1e-30);
    f[26] = (float)(ca.x / tr);
    f[27] = (float)(ca.w / tr);
    f[28] = (float)(cb.y / tr);
    f[29] = (float)log(tr / 3e-4);
    f[30] = (float)(o * exp(ls[0]));  // o sigma_1 / 0.01
    f[31] = (float)(fmax(dc[0], fmax(dc[1], dc[2])) - fmin(dc[0], fmin(dc[1], dc[2])));
    float4 *dst = reinterpret_cast<float4 *>(feat + (size_t)g * kLodFeatures);
#pragma unroll
    for (int i = 0; i < kLodFeatures / 4; ++i) dst[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
}

// Descending-score key: the order-preserving map of IEEE floats to unsigned
// integers, complemented (-0 mapped to +0 first, so that they tie).
__global__ void k_rank_keys(int n, const float *__restrict__ score, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t b = __float_as_uint(score[i]);
    if (b == 0x80000000u) b = 0u;  // -0 ties with +0
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    key[i] = ~asc;
    val[i] = (uint32_t)i;
}

__global__ void k_rank_template_keys(int n, int n_tpl, const TemplateInfo *__restrict__ tpls,
                                     const uint32_t *__restrict__ val, uint16_t *__restrict__ tkey) {
    __shared__ int32_t s_off[kMaxTemplates];
    for (int t = threadIdx.x; t < n_tpl; t += blockDim.x) s_off[t] = tpls[t].g_off;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    tkey[i] = (uint16_t)template_of(s_off, n_tpl, (int)val[i]);
}

__global__ void k_rank_local(int n, int n_tpl, const TemplateInfo *__restrict__ tpls, const uint32_t *__restrict__ val,
                             uint32_t *__restrict__ order) {
    __shared__ int32_t s_off[kMaxTemplates];
    for (int t = threadIdx.x; t < n_tpl; t += blockDim.x) s_off[t] = tpls[t].g_off;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = (int)val[i];
    order[i] = (uint32_t)(g - s_off[template_of(s_off, n_tpl, g)]);
}

// Regression targets: one CTA per (band, template) sums the template's
// contributions (fixed order: strided per thread, then a tree), then writes
// ln(c / mean + floor) for each of its Gaussians.
__global__ void __launch_bounds__(256) k_lod_targets(int n_total, const TemplateInfo *__restrict__ tpls,
                                                     const float *__restrict__ contrib, float floor_,
                                                     float *__restrict__ target) {
    __shared__ double red[256];
    const int t = blockIdx.x, b = blockIdx.y;
    const int g0 = tpls[t].g_off, n = tpls[t].n;
    const float *c = contrib + (size_t)b * n_total + g0;
    float *o = target + (size_t)b * n_total + g0;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)c[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = fmax(red[0] / (double)n, 1e-30);
    for (int i = threadIdx.x; i < n; i += blockDim.x) o[i] = (float)log((double)c[i] / mean + (double)floor_);
}

}  // namespace

int launch_lod_targets(int n_total, int n_tpl, int n_bands, const TemplateInfo *tpls, const float *contrib,
                       float floor_, float *target, cudaStream_t st) {
    if (n_total <= 0 || n_bands <= 0) return 0;
    k_lod_targets<<<dim3(n_tpl, n_bands), 256, 0, st>>>(n_total, tpls, contrib, floor_, target);
    return 1;
}

int launch_lod_features(int n_total, int n_tpl, const TemplateInfo *tpls, const TemplateArrays &ta, float *feat,
                        cudaStream_t st) {
    if (n_total <= 0) return 0;
    if (ta.storage == kStoreBf16)
        k_lod_features<kStoreBf16><<<(n_total + 255) / 256, 256, 0, st>>>(n_total, n_tpl, tpls, ta, feat);
    else
        k_lod_features<kStoreFp32><<<(n_total + 255) / 256, 256, 0, st>>>(n_total, n_tpl, tpls, ta, feat);
    return 1;
}

int lod_rank(int n_total, int n_tpl, const TemplateInfo *tpls, const float *score, uint32_t *order,
             uint32_t *key0, uint32_t *val0, uint32_t *key1, uint32_t *val1, uint16_t *tk0, uint16_t *tk1,
             uint32_t *scratch, cudaStream_t st) {
    if (n_total <= 0) return 0;
    const int nb = (n_total + 255) / 256;
    int launched = 0;
    k_rank_keys<<<nb, 256, 0, st>>>(n_total, score, key0, val0);
    ++launched;
    int ob = 0;
    launched += radix_sort_u32(key0, val0, key1, val1, (uint32_t)n_total, 32, scratch, st, &ob);
    uint32_t *v = ob ? val1 : val0;
    uint32_t *vo = ob ? val0 : val1;
    k_rank_template_keys<<<nb, 256, 0, st>>>(n_total, n_tpl, tpls, v, tk0);
    ++launched;
    int bits = 1;
    while ((1 << bits) < n_tpl) ++bits;
    int ob2 = 0;
    launched += radix_sort_u16(tk0, v, tk1, vo, (uint32_t)n_total, bits, scratch, st, &ob2);
    k_rank_local<<<nb, 256, 0, st>>>(n_total, n_tpl, tpls, ob2 ? vo : v, order);
    return launched + 1;
}

}  // namespace cs
