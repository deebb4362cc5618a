// cs_api.cu -- the C ABI of libcrowdsplat.so (declared in include/crowdsplat.h):
// context and device-memory management, template upload, LoD and
// per-frame instance state, and the ordering of one frame's kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/crowdsplat.h"
#include "../../include/crowdsplat_lod.h"
#include "../../include/crowdsplat_grad.h"
#include "cs_internal.cuh"

using namespace cs;

namespace {

constexpr int kStages = 8;

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;  // elements
};

}  // namespace

struct cs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // allocation-failure injection (cs_debug_fail_allocs): -1 off, else the
    // number of allocations that still succeed before every one fails
    int fail_after = -1;
    int blend_items = CS_BLEND_ITEMS_AUTO;  // cs_debug_blend_items
    int skin_mode = 0, sh_frame = 0, instance_cull = 1, stage_timing = 0;
    int storage = CS_STORE_FP32;  // template storage precision
    std::string err;

    // templates
    int n_tpl = 0;
    std::vector<TemplateInfo> tpl_host;
    std::vector<std::vector<float>> reach_g, smax_g;  // per Gaussian, for LoD bounds
    // chosen Gaussian subsets per (template, level); empty: the level renders a prefix
    std::vector<std::array<std::vector<uint32_t>, kMaxLevels>> lod_sub;
    std::vector<uint32_t> lod_idx_host;  // all subsets, concatenated
    uint32_t *d_lod_idx = nullptr;
    size_t lod_idx_cap = 0;
    TemplateInfo *d_tpl = nullptr;
    float4 *d_mean_op = nullptr, *d_cov_a = nullptr, *d_skin_w = nullptr, *d_sh = nullptr;
    float2 *d_cov_b = nullptr;
    uint32_t *d_skin_i = nullptr;
    uint4 *d_qa = nullptr, *d_qb = nullptr, *d_sh16 = nullptr;  // BF16 storage
    float4 *d_scale = nullptr, *d_quat = nullptr;              // FP32 storage, for the backward
    size_t n_gauss_total = 0, sh_planes_total = 0;
    int max_depth = 0;

    // LoD
    LodParams lod{};
    float lod_frac[kMaxLevels] = {1, 1, 1, 1};

    // instances
    int n_inst = 0;
    DevBuf<int32_t> tid, vis, cull;  // cull: the cull's frame totals and group bytes
    DevBuf<float> root, pose, B, V, Cloc;
    std::vector<int32_t> tid_host_check;
    DevBuf<Group> groups;
    int32_t *d_meta = nullptr, *h_meta = nullptr;  // pinned mirror
    Group *h_groups = nullptr;                     // pinned mirror of the frame's groups
    uint32_t *h_pairs = nullptr;                   // pinned

    // per-frame buffers
    DevBuf<float4> rec;
    DevBuf<uint32_t> key, ids, key2, ids2, bins, bins_sorted, pair_off, pval, pval2, scratch;
    DevBuf<uint2> rect, ranges;
    DevBuf<uint16_t> ptile, ptile2;
    DevBuf<float4> img;  // for cs_render_to_host
    DevBuf<float4> dbg_rec;  // expanded records (debug view)
    uint32_t key_lo = 0;     // the last frame's depth-key offset
    DevBuf<float> contrib_s;  // per-splat compositing weight sums (cs_render_contrib)
    // training frame (cs_render_train / cs_backward)
    DevBuf<uint32_t> px_end, bwd_cnt, bwd_chunk0, bwd_scratch;
    DevBuf<float4> px_fin, px_bnd;  // training: final state per pixel, states at the backward chunk boundaries
    DevBuf<float4> t_part, t_state;  // training forward: chunk partials, state before each pixel's stopping chunk
    DevBuf<uint32_t> t_last, t_slast;
    DevBuf<int32_t> t_stop;
    DevBuf<float> g_cov, g_B, g_dummy;
    DevBuf<float4> dsplat;
    bool train_valid = false;
    CamParams train_cp{};
    int train_proj_blocks = 0;
    // split compositing of long tile lists
    DevBuf<int32_t> bw_slot, bw_tile, bw_meta, bw_stop, bw_pp, bw_cslot;
    DevBuf<uint32_t> bw_chunk0, bw_done;
    DevBuf<float4> bw_state, bw_part;

    // last frame
    int64_t S = 0, P = 0;
    int n_groups = 0, visible = 0, tiles_x = 0, tiles_y = 0, frame_w = 0, frame_h = 0, frame_ox = 0, frame_oy = 0;
    int order_buf = 0, pair_buf = 0;  // which ping-pong half holds the result
    int per_level[kMaxLevels] = {0, 0, 0, 0};
    int launches = 0;  // kernels launched by the last cs_render
    // stage timing: two event sets used by alternate frames, so a frame's
    // events are read (without waiting) two frames later
    cudaEvent_t ev[2][kStages + 1] = {};
    int ev_cur = 0;           // set used by the last timed frame
    bool ev_pending[2] = {false, false};
    double stage_sum[kStages] = {};
    int64_t stage_frames = 0;
    bool timed = false;
};

namespace {

int fail(cs_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CS_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? CS_ERR_OOM : CS_ERR_CUDA,    \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                        __LINE__);                                                          \
        }                                                                                   \
    } while (0)

#define CS_TRY(expr)              \
    do {                          \
        int r_ = (expr);          \
        if (r_ != CS_OK) return r_; \
    } while (0)

template <typename T>
int ensure(cs_ctx *ctx, DevBuf<T> &b, size_t n, const char *what) {
    if (n <= b.cap && b.p) return CS_OK;
    size_t cap = std::max<size_t>(n + n / 4, 1024);
    if (b.p) {
        CS_CUDA(cudaStreamSynchronize(ctx->stream));
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    const bool injected = ctx->fail_after == 0;
    if (ctx->fail_after > 0) --ctx->fail_after;
    cudaError_t e = injected ? cudaErrorMemoryAllocation : cudaMalloc(&b.p, cap * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(ctx, CS_ERR_OOM, "allocating %s (%zu bytes): %s%s", what, cap * sizeof(T),
                    cudaGetErrorString(e), injected ? " (injected failure)" : "");
    }
    b.cap = cap;
    return CS_OK;
}

template <typename T>
void release(DevBuf<T> &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

template <typename T>
size_t bytes_of(const DevBuf<T> &b) {
    return b.cap * sizeof(T);
}

void free_templates(cs_ctx *c) {
    cudaFree(c->d_tpl);
    cudaFree(c->d_mean_op);
    cudaFree(c->d_cov_a);
    cudaFree(c->d_cov_b);
    cudaFree(c->d_skin_w);
    cudaFree(c->d_skin_i);
    cudaFree(c->d_sh);
    cudaFree(c->d_scale);
    cudaFree(c->d_quat);
    c->d_scale = c->d_quat = nullptr;
    c->train_valid = false;
    cudaFree(c->d_qa);
    cudaFree(c->d_qb);
    cudaFree(c->d_sh16);
    c->d_qa = c->d_qb = c->d_sh16 = nullptr;
    cudaFree(c->d_lod_idx);
    c->d_lod_idx = nullptr;
    c->lod_idx_cap = 0;
    c->lod_sub.clear();
    c->lod_idx_host.clear();
    c->d_tpl = nullptr;
    c->d_mean_op = c->d_cov_a = c->d_skin_w = c->d_sh = nullptr;
    c->d_cov_b = nullptr;
    c->d_skin_i = nullptr;
    c->n_tpl = 0;
    c->n_gauss_total = c->sh_planes_total = 0;
}

// Level sizes, subset offsets and instance-cull bounds of every template for
// the current LoD.  A level with a chosen subset renders exactly that subset;
// otherwise it renders the first round(fraction * n) Gaussians.
void refresh_lod_bounds(cs_ctx *c) {
    c->lod_idx_host.clear();
    for (int t = 0; t < c->n_tpl; ++t) {
        TemplateInfo &T = c->tpl_host[t];
        for (int l = 0; l < kMaxLevels; ++l) {
            int lvl = l < c->lod.n_levels ? l : c->lod.n_levels - 1;
            const std::vector<uint32_t> &sub = c->lod_sub[t][lvl];
            int n;
            if (!sub.empty()) {
                n = (int)sub.size();
                T.lod_idx_off[l] = (int32_t)c->lod_idx_host.size();
                c->lod_idx_host.insert(c->lod_idx_host.end(), sub.begin(), sub.end());
            } else {
                double cnt = std::floor((double)c->lod_frac[lvl] * (double)T.n + 0.5);
                n = (int)std::min<double>(std::max<double>(cnt, 0.0), (double)T.n);
                T.lod_idx_off[l] = -1;
            }
            T.n_level[l] = n;
            float reach = 0.f, smax = 0.f;
            for (int k = 0; k < n; ++k) {
                const int g = sub.empty() ? k : (int)sub[k];
                reach = std::max(reach, c->reach_g[t][g]);
                smax = std::max(smax, c->smax_g[t][g]);
            }
            T.reach[l] = reach;
            T.sigma_max[l] = smax * c->lod.mult[lvl];
        }
    }
}

TemplateArrays template_arrays(const cs_ctx *c) {
    TemplateArrays ta{};
    ta.mean_op = c->d_mean_op;
    ta.cov_a = c->d_cov_a;
    ta.cov_b = c->d_cov_b;
    ta.skin_w = c->d_skin_w;
    ta.skin_i = c->d_skin_i;
    ta.sh = c->d_sh;
    ta.lod_idx = c->d_lod_idx;
    ta.qa = c->d_qa;
    ta.qb = c->d_qb;
    ta.sh16 = c->d_sh16;
    ta.storage = c->storage;
    ta.scale = c->d_scale;
    ta.quat = c->d_quat;
    return ta;
}

// Round to BF16 / FP16 (nearest, ties to even) and return the bits.
uint32_t bf16_bits(float v) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v)); }
float bf16_value(uint32_t bits) {
    uint32_t u = bits << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}
uint32_t f16_bits(float v) { return (uint32_t)__half_as_ushort(__float2half_rn(v)); }

int push_templates(cs_ctx *ctx) {
    const size_t ni = ctx->lod_idx_host.size();
    if (ni > ctx->lod_idx_cap) {
        CS_CUDA(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->d_lod_idx);
        ctx->d_lod_idx = nullptr;
        ctx->lod_idx_cap = 0;
        CS_CUDA(cudaMalloc(&ctx->d_lod_idx, ni * sizeof(uint32_t)));
        ctx->lod_idx_cap = ni;
    }
    if (ni > 0)
        CS_CUDA(cudaMemcpyAsync(ctx->d_lod_idx, ctx->lod_idx_host.data(), ni * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, ctx->stream));
    CS_CUDA(cudaMemcpyAsync(ctx->d_tpl, ctx->tpl_host.data(), sizeof(TemplateInfo) * ctx->n_tpl,
                            cudaMemcpyHostToDevice, ctx->stream));
    CS_CUDA(cudaStreamSynchronize(ctx->stream));
    return CS_OK;
}

// Full-image size of a camera (its own size when it has no window).
void full_size(const cs_camera *cam, int &fw, int &fh) {
    const bool win = cam->full_width != 0 || cam->full_height != 0;
    fw = win ? cam->full_width : cam->width;
    fh = win ? cam->full_height : cam->height;
}

// Window fields of a camera: origin on the tile grid, inside the full image.
bool window_ok(const cs_camera *cam) {
    int fw, fh;
    full_size(cam, fw, fh);
    if (cam->full_width == 0 && cam->full_height == 0) return cam->win_x0 == 0 && cam->win_y0 == 0;
    const int x1 = cam->win_x0 + cam->width, y1 = cam->win_y0 + cam->height;
    return fw >= 1 && fh >= 1 && fw <= CS_MAX_IMAGE_SIDE && fh <= CS_MAX_IMAGE_SIDE && cam->win_x0 >= 0 &&
           cam->win_y0 >= 0 && cam->win_x0 % kTile == 0 && cam->win_y0 % kTile == 0 && x1 <= fw && y1 <= fh &&
           (x1 % kTile == 0 || x1 == fw) && (y1 % kTile == 0 || y1 == fh);
}

void cam_params(const cs_ctx *c, const cs_camera *cam, CamParams &p) {
    p.n_splats = 0;  // set once the cull's counts are read
    for (int i = 0; i < 9; ++i) p.R[i] = cam->R[i];
    for (int i = 0; i < 3; ++i) p.t[i] = cam->t[i];
    p.fx = cam->fx;
    p.fy = cam->fy;
    p.cx = cam->cx;
    p.cy = cam->cy;
    p.W = cam->width;
    p.H = cam->height;
    p.ox = cam->win_x0;
    p.oy = cam->win_y0;
    int fw, fh;
    full_size(cam, fw, fh);
    p.near_z = cam->near_z;
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s -= (double)cam->R[k * 3 + i] * (double)cam->t[k];
        p.center[i] = (float)s;
    }
    // the EWA clamp follows the full image's field of view
    p.limx = (float)(1.3 * (0.5 * fw) / (double)cam->fx);
    p.limy = (float)(1.3 * (0.5 * fh) / (double)cam->fy);
    p.tiles_x = (cam->width + kTile - 1) / kTile;
    p.tiles_y = (cam->height + kTile - 1) / kTile;
    // Conservative instance cull.  A splat's support half-width is at most
    // 3 |J| sigma + 3 sqrt(0.3 + sqrt(0.1)) + 1 px with
    // |J| <= (f_max / z) sqrt(2 + limx^2 + limy^2); the pixel term becomes a
    // margin on the side planes, the sigma term a growth of the bounding
    // sphere (in metres, scaled by f_max / f_min for the plane's own focal).
    const double margin = 3.0 * std::sqrt(0.3 + std::sqrt(0.1)) + 1.0 + 2.0;
    const double fmax = std::max(cam->fx, cam->fy), fmin = std::min(cam->fx, cam->fy);
    p.cull_sigma_k = (float)(3.0 * std::sqrt(2.0 + (double)p.limx * p.limx + (double)p.limy * p.limy) *
                             (fmax / fmin) * 1.01);
    // full-range depth keys until the cull has bounded the frame's depths
    p.key_lo = 0u;
    p.key_hi = 0xFFFFFFFEu;
    // side planes of the rendered window
    const double tr = (cam->win_x0 + cam->width - cam->cx + margin) / cam->fx;
    const double tl = (cam->cx - cam->win_x0 + margin) / cam->fx;
    const double tb = (cam->win_y0 + cam->height - cam->cy + margin) / cam->fy;
    const double tt = (cam->cy - cam->win_y0 + margin) / cam->fy;
    const double planes[4][3] = {{1, 0, -tr}, {-1, 0, -tl}, {0, 1, -tb}, {0, -1, -tt}};
    for (int k = 0; k < 4; ++k) {
        double n = std::sqrt(planes[k][0] * planes[k][0] + planes[k][1] * planes[k][1] +
                             planes[k][2] * planes[k][2]);
        for (int e = 0; e < 3; ++e) p.plane[k][e] = (float)(planes[k][e] / n);
        p.plane[k][3] = 0.f;
    }
}

// Add the stage times of event set k (a completed frame) to the running sums.
// Depth keys of this frame: the cull's bounds of every live depth (float
// bits); no visible instance leaves an empty range.
void set_depth_key_range(CamParams &cp, const int32_t *meta) {
    cp.key_lo = (uint32_t)meta[kMetaZlo];
    cp.key_hi = std::max((uint32_t)meta[kMetaZhi], cp.key_lo);
}

int accumulate_stage_times(cs_ctx *ctx, int k) {
    if (!ctx->ev_pending[k]) return CS_OK;
    CS_CUDA(cudaEventSynchronize(ctx->ev[k][kStages]));
    for (int i = 0; i < kStages; ++i) {
        float t = 0.f;
        CS_CUDA(cudaEventElapsedTime(&t, ctx->ev[k][i], ctx->ev[k][i + 1]));
        ctx->stage_sum[i] += t;
    }
    ctx->stage_frames += 1;
    ctx->ev_pending[k] = false;
    return CS_OK;
}

int bits_for(uint32_t n_values) {
    int b = 0;
    while (b < 32 && (1ull << b) < n_values) ++b;
    return b;
}

}  // namespace

extern "C" {

const char *cs_version(void) { return "crowdsplat-gb300 0.1 (sm_103a)"; }

const char *cs_last_error(const cs_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cs_create(cs_ctx **out, const cs_create_params *p) {
    if (!out || !p) return CS_ERR_ARG;
    *out = nullptr;
    if (p->skin_mode != CS_SKIN_FULL && p->skin_mode != CS_SKIN_MEANS_ONLY) return CS_ERR_ARG;
    if (p->sh_frame != CS_SH_ROOT_FRAME && p->sh_frame != CS_SH_WORLD_FRAME) return CS_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return CS_ERR_CUDA;
    }
    if (p->device < 0 || p->device >= ndev) return CS_ERR_ARG;
    cs_ctx *ctx = new (std::nothrow) cs_ctx();
    if (!ctx) return CS_ERR_OOM;
    ctx->device = p->device;
    ctx->stream = (cudaStream_t)p->stream;
    ctx->skin_mode = p->skin_mode;
    ctx->sh_frame = p->sh_frame;
    ctx->instance_cull = p->instance_cull ? 1 : 0;
    ctx->stage_timing = p->stage_timing ? 1 : 0;
    if (p->template_storage != CS_STORE_FP32 && p->template_storage != CS_STORE_BF16) {
        delete ctx;
        return CS_ERR_ARG;
    }
    ctx->storage = p->template_storage;
    ctx->lod.n_levels = 1;
    for (int l = 0; l < kMaxLevels; ++l) ctx->lod.mult[l] = 1.0f;
    int rc = CS_OK;
    do {
        if (cudaSetDevice(ctx->device) != cudaSuccess) { rc = CS_ERR_CUDA; break; }
        if (cudaMalloc(&ctx->d_meta, kMetaWords * sizeof(int32_t)) != cudaSuccess) { rc = CS_ERR_OOM; break; }
        if (cudaHostAlloc(&ctx->h_meta, kMetaWords * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) { rc = CS_ERR_OOM; break; }
        if (cudaHostAlloc(&ctx->h_pairs, 4 * sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) { rc = CS_ERR_OOM; break; }
        if (cudaHostAlloc(&ctx->h_groups, kMaxGroups * sizeof(Group), cudaHostAllocDefault) != cudaSuccess) { rc = CS_ERR_OOM; break; }
        for (int k = 0; k < 2 && rc == CS_OK; ++k)
            for (int i = 0; i <= kStages; ++i)
                if (cudaEventCreate(&ctx->ev[k][i]) != cudaSuccess) { rc = CS_ERR_CUDA; break; }
    } while (0);
    if (rc != CS_OK) {
        cudaGetLastError();
        cs_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return CS_OK;
}

void cs_destroy(cs_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_templates(ctx);
    release(ctx->tid); release(ctx->vis); release(ctx->cull); release(ctx->root); release(ctx->pose);
    release(ctx->B); release(ctx->V); release(ctx->Cloc); release(ctx->groups);
    release(ctx->rec); release(ctx->key); release(ctx->ids); release(ctx->key2); release(ctx->ids2);
    release(ctx->bins); release(ctx->bins_sorted); release(ctx->pair_off); release(ctx->pval); release(ctx->pval2);
    release(ctx->scratch); release(ctx->rect); release(ctx->ranges); release(ctx->ptile);
    release(ctx->ptile2); release(ctx->img); release(ctx->contrib_s); release(ctx->dbg_rec);
    release(ctx->px_end); release(ctx->px_fin); release(ctx->px_bnd); release(ctx->bwd_cnt); release(ctx->bwd_chunk0);
    release(ctx->bwd_scratch); release(ctx->t_part); release(ctx->t_state); release(ctx->t_last);
    release(ctx->t_slast); release(ctx->t_stop); release(ctx->dsplat); release(ctx->g_cov); release(ctx->g_B);
    release(ctx->g_dummy);
    release(ctx->bw_slot); release(ctx->bw_tile); release(ctx->bw_meta); release(ctx->bw_stop); release(ctx->bw_pp); release(ctx->bw_cslot); release(ctx->bw_chunk0);
    release(ctx->bw_done); release(ctx->bw_state); release(ctx->bw_part);
    if (ctx->d_meta) cudaFree(ctx->d_meta);
    if (ctx->h_meta) cudaFreeHost(ctx->h_meta);
    if (ctx->h_groups) cudaFreeHost(ctx->h_groups);
    if (ctx->h_pairs) cudaFreeHost(ctx->h_pairs);
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i <= kStages; ++i)
            if (ctx->ev[k][i]) cudaEventDestroy(ctx->ev[k][i]);
    cudaGetLastError();
    delete ctx;
}

int cs_upload_templates(cs_ctx *ctx, int32_t n_templates, const cs_template_desc *tp) {
    if (!ctx) return CS_ERR_ARG;
    if (n_templates < 1 || !tp) return fail(ctx, CS_ERR_ARG, "n_templates must be >= 1");
    if (n_templates > CS_MAX_TEMPLATES)
        return fail(ctx, CS_ERR_CAPACITY, "n_templates %d exceeds %d", n_templates, CS_MAX_TEMPLATES);
    CS_CUDA(cudaSetDevice(ctx->device));
    // validate and lay out
    std::vector<TemplateInfo> info(n_templates);
    size_t g_total = 0, planes_total = 0;
    int max_depth = 0;
    for (int t = 0; t < n_templates; ++t) {
        const cs_template_desc &d = tp[t];
        if (d.n_gauss < 1) return fail(ctx, CS_ERR_ARG, "template %d: n_gauss must be >= 1", t);
        if (d.sh_degree < 0 || d.sh_degree > 3)
            return fail(ctx, CS_ERR_ARG, "template %d: sh_degree must be 0..3", t);
        if (!d.means || !d.scales || !d.quats || !d.opacity || !d.sh || !d.skin_idx || !d.skin_w ||
            !d.rest_joints || !d.parents)
            return fail(ctx, CS_ERR_ARG, "template %d: NULL array", t);
        TemplateInfo &T = info[t];
        memset(&T, 0, sizeof T);
        T.g_off = (int32_t)g_total;
        T.n = d.n_gauss;
        T.sh_deg = d.sh_degree;
        int K = (d.sh_degree + 1) * (d.sh_degree + 1);
        T.sh_planes = (K * 3 + 3) / 4;
        T.sh_off = (int64_t)planes_total;
        for (int j = 0; j < kJoints; ++j) {
            int par = d.parents[j];
            if ((j == 0 && par != -1) || (j > 0 && (par < 0 || par >= j)))
                return fail(ctx, CS_ERR_ARG, "template %d: parents[%d] = %d (need -1 for the root, "
                            "0 <= parent < j otherwise)", t, j, par);
            T.parent[j] = (int8_t)par;
            T.depth[j] = (int8_t)(par < 0 ? 0 : T.depth[par] + 1);
            max_depth = std::max(max_depth, (int)T.depth[j]);
            T.max_depth = std::max(T.max_depth, (int32_t)T.depth[j]);
            for (int e = 0; e < 3; ++e) T.rest[j * 3 + e] = d.rest_joints[j * 3 + e];
        }
        g_total += (size_t)d.n_gauss;
        planes_total += (size_t)T.sh_planes * (size_t)d.n_gauss;
        if (g_total >= (size_t)INT32_MAX)
            return fail(ctx, CS_ERR_CAPACITY, "total Gaussians exceed 2^31 - 1");
    }
    // host staging in the device layout, plus per-Gaussian cull bounds
    std::vector<float4> mean_op(g_total), cov_a(g_total), skin_w(g_total), sh(planes_total);
    std::vector<float2> cov_b(g_total);
    std::vector<uint32_t> skin_i(g_total);
    std::vector<std::vector<float>> reach(n_templates), smax(n_templates);
    for (int t = 0; t < n_templates; ++t) {
        const cs_template_desc &d = tp[t];
        TemplateInfo &T = info[t];
        // chain length of each joint: sum of bone lengths up to the root
        double chain[kJoints];
        for (int j = 0; j < kJoints; ++j) {
            if (T.parent[j] < 0) {
                chain[j] = 0.0;
                continue;
            }
            int p = T.parent[j];
            double dx = T.rest[j * 3] - T.rest[p * 3], dy = T.rest[j * 3 + 1] - T.rest[p * 3 + 1],
                   dz = T.rest[j * 3 + 2] - T.rest[p * 3 + 2];
            chain[j] = chain[p] + std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        int K = (d.sh_degree + 1) * (d.sh_degree + 1);
        reach[t].resize(d.n_gauss);
        smax[t].resize(d.n_gauss);
        for (int g = 0; g < d.n_gauss; ++g) {
            size_t gi = (size_t)T.g_off + g;
            double m[3] = {d.means[g * 3], d.means[g * 3 + 1], d.means[g * 3 + 2]};
            double o = d.opacity[g];
            if (!(o >= 0.0 && o <= 1.0)) return fail(ctx, CS_ERR_ARG, "template %d: opacity[%d] not in [0,1]", t, g);
            mean_op[gi] = make_float4(d.means[g * 3], d.means[g * 3 + 1], d.means[g * 3 + 2], d.opacity[g]);
            // canonical covariance R S S^T R^T in double, stored in float
            double q[4] = {d.quats[g * 4], d.quats[g * 4 + 1], d.quats[g * 4 + 2], d.quats[g * 4 + 3]};
            double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            if (!(qn > 0.0) || !std::isfinite(qn)) return fail(ctx, CS_ERR_ARG, "template %d: quats[%d] has zero norm", t, g);
            double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
            double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                           2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                           2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
            double s[3] = {d.scales[g * 3], d.scales[g * 3 + 1], d.scales[g * 3 + 2]};
            if (!(s[0] > 0 && s[1] > 0 && s[2] > 0)) return fail(ctx, CS_ERR_ARG, "template %d: scales[%d] must be > 0", t, g);
            double C[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double a = 0.0;
                    for (int k = 0; k < 3; ++k) a += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];
                    C[i * 3 + j] = a;
                }
            cov_a[gi] = make_float4((float)C[0], (float)C[1], (float)C[2], (float)C[4]);
            cov_b[gi] = make_float2((float)C[5], (float)C[8]);
            double wsum = 0.0, r = 0.0;
            uint32_t packed = 0;
            for (int k = 0; k < 4; ++k) {
                int j = d.skin_idx[g * 4 + k];
                float wk = d.skin_w[g * 4 + k];
                if (j >= kJoints) return fail(ctx, CS_ERR_ARG, "template %d: skin_idx[%d] >= 24", t, g);
                if (!(wk >= 0.0f)) return fail(ctx, CS_ERR_ARG, "template %d: negative skin weight at %d", t, g);
                wsum += wk;
                packed |= (uint32_t)j << (8 * k);
                double dx = m[0] - T.rest[j * 3], dy = m[1] - T.rest[j * 3 + 1], dz = m[2] - T.rest[j * 3 + 2];
                if (wk > 0.0f) r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz) + chain[j]);
            }
            if (std::fabs(wsum - 1.0) > 1e-3)
                return fail(ctx, CS_ERR_ARG, "template %d: skin weights of %d sum to %g (need 1 +- 1e-3)", t, g, wsum);
            skin_w[gi] = make_float4(d.skin_w[g * 4], d.skin_w[g * 4 + 1], d.skin_w[g * 4 + 2], d.skin_w[g * 4 + 3]);
            skin_i[gi] = packed;
            // weights summing to 1 + e can push the blend out by e |pelvis|
            double pel = std::sqrt((double)T.rest[0] * T.rest[0] + (double)T.rest[1] * T.rest[1] + (double)T.rest[2] * T.rest[2]);
            reach[t][g] = (float)((r + std::fabs(wsum - 1.0) * (pel + r)) * wsum + 1e-6);
            smax[t][g] = (float)(std::max(s[0], std::max(s[1], s[2])) * std::max(1.0, wsum));
            const float *shg = d.sh + (size_t)g * K * 3;
            for (int pl = 0; pl < T.sh_planes; ++pl) {
                float v[4];
                for (int e = 0; e < 4; ++e) {
                    int f = pl * 4 + e;
                    v[e] = f < K * 3 ? shg[f] : 0.0f;
                }
                sh[(size_t)T.sh_off + (size_t)pl * T.n + g] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    }
    // BF16 storage: quantise the staged attributes (CS_STORE_BF16 in the header)
    std::vector<uint4> qa, qb, sh16;
    size_t planes16_total = 0;
    if (ctx->storage == CS_STORE_BF16) {
        qa.resize(g_total);
        qb.resize(g_total);
        for (int t = 0; t < n_templates; ++t) {
            TemplateInfo &T = info[t];
            const int K = (T.sh_deg + 1) * (T.sh_deg + 1);
            T.sh_planes = (K * 3 + 7) / 8;
            T.sh_off = (int64_t)planes16_total;
            planes16_total += (size_t)T.sh_planes * (size_t)T.n;
        }
        sh16.assign(planes16_total, make_uint4(0u, 0u, 0u, 0u));
        for (int t = 0; t < n_templates; ++t) {
            const cs_template_desc &d = tp[t];
            TemplateInfo &T = info[t];
            const int K = (d.sh_degree + 1) * (d.sh_degree + 1);
            double chain[kJoints];
            for (int j = 0; j < kJoints; ++j) {
                const int p = T.parent[j];
                if (p < 0) { chain[j] = 0.0; continue; }
                const double dx = T.rest[j * 3] - T.rest[p * 3], dy = T.rest[j * 3 + 1] - T.rest[p * 3 + 1],
                             dz = T.rest[j * 3 + 2] - T.rest[p * 3 + 2];
                chain[j] = chain[p] + std::sqrt(dx * dx + dy * dy + dz * dz);
            }
            const double pel = std::sqrt((double)T.rest[0] * T.rest[0] + (double)T.rest[1] * T.rest[1] +
                                         (double)T.rest[2] * T.rest[2]);
            for (int g = 0; g < d.n_gauss; ++g) {
                const size_t gi = (size_t)T.g_off + g;
                const double m[3] = {d.means[g * 3], d.means[g * 3 + 1], d.means[g * 3 + 2]};
                int js[4];
                float ws[4];
                for (int k = 0; k < 4; ++k) {
                    js[k] = d.skin_idx[g * 4 + k];
                    ws[k] = d.skin_w[g * 4 + k];
                }
                // anchor: the skinning joint nearest to the mean goes to slot 0
                int best = 0;
                double bd = INFINITY;
                for (int k = 0; k < 4; ++k) {
                    const int j = js[k];
                    const double dx = m[0] - T.rest[j * 3], dy = m[1] - T.rest[j * 3 + 1], dz = m[2] - T.rest[j * 3 + 2];
                    const double dd = dx * dx + dy * dy + dz * dz;
                    if (dd < bd) { bd = dd; best = k; }
                }
                std::swap(js[0], js[best]);
                std::swap(ws[0], ws[best]);
                const int a = js[0];
                uint32_t db[3];
                float mq[3];  // the mean the kernels reconstruct (FP32 add)
                for (int e = 0; e < 3; ++e) {
                    db[e] = bf16_bits((float)(m[e] - (double)T.rest[a * 3 + e]));
                    mq[e] = T.rest[a * 3 + e] + bf16_value(db[e]);
                }
                const float4 ca = cov_a[gi];
                const float2 cb = cov_b[gi];
                const uint32_t ob = bf16_bits(d.opacity[g]);
                uint32_t wb[4];
                double wsum = 0.0, r = 0.0;
                uint32_t packed = 0;
                for (int k = 0; k < 4; ++k) {
                    wb[k] = bf16_bits(ws[k]);
                    const double wq = bf16_value(wb[k]);
                    wsum += wq;
                    packed |= (uint32_t)js[k] << (8 * k);
                    const int j = js[k];
                    const double dx = mq[0] - T.rest[j * 3], dy = mq[1] - T.rest[j * 3 + 1], dz = mq[2] - T.rest[j * 3 + 2];
                    if (wq > 0.0) r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz) + chain[j]);
                }
                qa[gi] = make_uint4(db[0] | (db[1] << 16), db[2] | (ob << 16), bf16_bits(ca.x) | (bf16_bits(ca.y) << 16),
                                    bf16_bits(ca.z) | (bf16_bits(ca.w) << 16));
                qb[gi] = make_uint4(bf16_bits(cb.x) | (bf16_bits(cb.y) << 16), wb[0] | (wb[1] << 16),
                                    wb[2] | (wb[3] << 16), packed);
                // cull bounds from the quantised values; the split-BF16 blend
                // and the rounded covariance add small margins
                reach[t][g] = (float)((r + std::fabs(wsum - 1.0) * (pel + r)) * wsum + 1e-4);
                smax[t][g] = (float)(smax[t][g] * 1.01 * std::max(1.0, wsum));
                const float *shg = d.sh + (size_t)g * K * 3;
                for (int pl = 0; pl < T.sh_planes; ++pl) {
                    uint32_t h[8];
                    for (int e = 0; e < 8; ++e) {
                        const int f = pl * 8 + e;
                        h[e] = f16_bits(f < K * 3 ? shg[f] : 0.0f);
                    }
                    sh16[(size_t)T.sh_off + (size_t)pl * T.n + g] =
                        make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
                }
            }
        }
    }
    // device copies
    CS_CUDA(cudaStreamSynchronize(ctx->stream));
    free_templates(ctx);
    CS_CUDA(cudaMalloc(&ctx->d_tpl, sizeof(TemplateInfo) * n_templates));
    if (ctx->storage == CS_STORE_BF16) {
        CS_CUDA(cudaMalloc(&ctx->d_qa, sizeof(uint4) * g_total));
        CS_CUDA(cudaMalloc(&ctx->d_qb, sizeof(uint4) * g_total));
        CS_CUDA(cudaMalloc(&ctx->d_sh16, sizeof(uint4) * std::max<size_t>(planes16_total, 1)));
        CS_CUDA(cudaMemcpy(ctx->d_qa, qa.data(), sizeof(uint4) * g_total, cudaMemcpyHostToDevice));
        CS_CUDA(cudaMemcpy(ctx->d_qb, qb.data(), sizeof(uint4) * g_total, cudaMemcpyHostToDevice));
        CS_CUDA(cudaMemcpy(ctx->d_sh16, sh16.data(), sizeof(uint4) * planes16_total, cudaMemcpyHostToDevice));
        planes_total = planes16_total;
    } else {
    {
        std::vector<float4> sc(g_total), qt(g_total);
        for (int t = 0; t < n_templates; ++t)
            for (int g = 0; g < tp[t].n_gauss; ++g) {
                const size_t gi = (size_t)info[t].g_off + g;
                const float *s3 = tp[t].scales + (size_t)g * 3, *q4 = tp[t].quats + (size_t)g * 4;
                sc[gi] = make_float4(s3[0], s3[1], s3[2], 0.0f);
                qt[gi] = make_float4(q4[0], q4[1], q4[2], q4[3]);
            }
        CS_CUDA(cudaMalloc(&ctx->d_scale, sizeof(float4) * g_total));
        CS_CUDA(cudaMalloc(&ctx->d_quat, sizeof(float4) * g_total));
        CS_CUDA(cudaMemcpy(ctx->d_scale, sc.data(), sizeof(float4) * g_total, cudaMemcpyHostToDevice));
        CS_CUDA(cudaMemcpy(ctx->d_quat, qt.data(), sizeof(float4) * g_total, cudaMemcpyHostToDevice));
    }
    CS_CUDA(cudaMalloc(&ctx->d_mean_op, sizeof(float4) * g_total));
    CS_CUDA(cudaMalloc(&ctx->d_cov_a, sizeof(float4) * g_total));
    CS_CUDA(cudaMalloc(&ctx->d_cov_b, sizeof(float2) * g_total));
    CS_CUDA(cudaMalloc(&ctx->d_skin_w, sizeof(float4) * g_total));
    CS_CUDA(cudaMalloc(&ctx->d_skin_i, sizeof(uint32_t) * g_total));
    CS_CUDA(cudaMalloc(&ctx->d_sh, sizeof(float4) * planes_total));
    CS_CUDA(cudaMemcpy(ctx->d_mean_op, mean_op.data(), sizeof(float4) * g_total, cudaMemcpyHostToDevice));
    CS_CUDA(cudaMemcpy(ctx->d_cov_a, cov_a.data(), sizeof(float4) * g_total, cudaMemcpyHostToDevice));
    CS_CUDA(cudaMemcpy(ctx->d_cov_b, cov_b.data(), sizeof(float2) * g_total, cudaMemcpyHostToDevice));
    CS_CUDA(cudaMemcpy(ctx->d_skin_w, skin_w.data(), sizeof(float4) * g_total, cudaMemcpyHostToDevice));
    CS_CUDA(cudaMemcpy(ctx->d_skin_i, skin_i.data(), sizeof(uint32_t) * g_total, cudaMemcpyHostToDevice));
    CS_CUDA(cudaMemcpy(ctx->d_sh, sh.data(), sizeof(float4) * planes_total, cudaMemcpyHostToDevice));
    }
    ctx->n_tpl = n_templates;
    ctx->tpl_host = info;
    ctx->lod_sub.assign(n_templates, {});
    ctx->reach_g = std::move(reach);
    ctx->smax_g = std::move(smax);
    ctx->n_gauss_total = g_total;
    ctx->sh_planes_total = planes_total;
    ctx->max_depth = max_depth;
    // default LoD: one full-detail level
    ctx->lod.n_levels = 1;
    for (int l = 0; l < kMaxLevels; ++l) {
        ctx->lod.mult[l] = 1.0f;
        ctx->lod_frac[l] = 1.0f;
    }
    refresh_lod_bounds(ctx);
    return push_templates(ctx);
}

int cs_set_lod(cs_ctx *ctx, int32_t n_levels, const float *dist_thresh, const float *fraction,
               const float *scale_mult) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "cs_set_lod before cs_upload_templates");
    if (n_levels < 1 || n_levels > CS_MAX_LEVELS)
        return fail(ctx, CS_ERR_ARG, "n_levels must be 1..%d", CS_MAX_LEVELS);
    if (!fraction || !scale_mult || (n_levels > 1 && !dist_thresh))
        return fail(ctx, CS_ERR_ARG, "NULL LoD array");
    for (int l = 0; l < n_levels; ++l) {
        if (!(fraction[l] > 0.0f && fraction[l] <= 1.0f))
            return fail(ctx, CS_ERR_ARG, "fraction[%d] must be in (0, 1]", l);
        if (!(scale_mult[l] > 0.0f && std::isfinite(scale_mult[l])))
            return fail(ctx, CS_ERR_ARG, "scale_mult[%d] must be > 0", l);
    }
    for (int l = 0; l + 1 < n_levels; ++l) {
        if (!std::isfinite(dist_thresh[l]) || (l > 0 && dist_thresh[l] < dist_thresh[l - 1]))
            return fail(ctx, CS_ERR_ARG, "dist_thresh must be finite and ascending");
    }
    ctx->lod.n_levels = n_levels;
    for (int l = 0; l < kMaxLevels; ++l) {
        int s = l < n_levels ? l : n_levels - 1;
        ctx->lod.mult[l] = scale_mult[s];
        ctx->lod_frac[l] = fraction[s];
        if (l < kMaxLevels - 1) ctx->lod.thresh[l] = l < n_levels - 1 ? dist_thresh[l] : INFINITY;
    }
    CS_CUDA(cudaSetDevice(ctx->device));
    ctx->train_valid = false;
    refresh_lod_bounds(ctx);
    return push_templates(ctx);
}

int cs_set_lod_subset(cs_ctx *ctx, int32_t template_id, int32_t level, int32_t n, const uint32_t *idx) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "cs_set_lod_subset before cs_upload_templates");
    if (template_id < 0 || template_id >= ctx->n_tpl)
        return fail(ctx, CS_ERR_ARG, "template_id %d out of range", template_id);
    if (level < 0 || level >= CS_MAX_LEVELS) return fail(ctx, CS_ERR_ARG, "level must be 0..%d", CS_MAX_LEVELS - 1);
    const int ng = ctx->tpl_host[template_id].n;
    if (n < 0 || n > ng) return fail(ctx, CS_ERR_ARG, "n = %d outside 0..%d", n, ng);
    if (n > 0 && !idx) return fail(ctx, CS_ERR_ARG, "NULL index array");
    std::vector<uint32_t> sub(idx, idx + n);
    std::vector<char> seen(ng, 0);
    for (int k = 0; k < n; ++k) {
        if (sub[k] >= (uint32_t)ng)
            return fail(ctx, CS_ERR_ARG, "idx[%d] = %u outside the template's %d Gaussians", k, sub[k], ng);
        if (seen[sub[k]]) return fail(ctx, CS_ERR_ARG, "idx[%d] = %u repeats an earlier index", k, sub[k]);
        seen[sub[k]] = 1;
    }
    CS_CUDA(cudaSetDevice(ctx->device));
    ctx->lod_sub[template_id][level] = std::move(sub);
    ctx->train_valid = false;
    refresh_lod_bounds(ctx);
    return push_templates(ctx);
}

int cs_set_instances(cs_ctx *ctx, int32_t n, const int32_t *template_id, const float *root,
                     const float *joint_pose, int32_t on_device) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "cs_set_instances before cs_upload_templates");
    if (n < 0) return fail(ctx, CS_ERR_ARG, "n must be >= 0");
    if (n > CS_MAX_INSTANCES) return fail(ctx, CS_ERR_CAPACITY, "n = %d exceeds %d", n, CS_MAX_INSTANCES);
    if (n > 0 && (!template_id || !root || !joint_pose)) return fail(ctx, CS_ERR_ARG, "NULL instance array");
    CS_CUDA(cudaSetDevice(ctx->device));
    size_t want = (size_t)std::max(n, 1);
    CS_TRY(ensure(ctx, ctx->tid, want, "template ids"));
    CS_TRY(ensure(ctx, ctx->vis, want, "visible list"));
    CS_TRY(ensure(ctx, ctx->cull, cull_scratch_words(want), "cull scratch"));
    CS_TRY(ensure(ctx, ctx->root, want * 12, "roots"));
    CS_TRY(ensure(ctx, ctx->pose, want * kJoints * 3, "poses"));
    CS_TRY(ensure(ctx, ctx->B, want * kJoints * 12, "skinning transforms"));
    CS_TRY(ensure(ctx, ctx->V, want * 12, "view transforms"));
    CS_TRY(ensure(ctx, ctx->Cloc, want * 4, "local camera centres"));
    CS_TRY(ensure(ctx, ctx->groups, (size_t)kMaxTemplates * kMaxLevels, "groups"));
    if (n > 0) {
        cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (!on_device) {
            for (int i = 0; i < n; ++i)
                if (template_id[i] < 0 || template_id[i] >= ctx->n_tpl)
                    return fail(ctx, CS_ERR_ARG, "template_id[%d] = %d out of range", i, template_id[i]);
        }
        CS_CUDA(cudaMemcpyAsync(ctx->tid.p, template_id, sizeof(int32_t) * n, kind, ctx->stream));
        CS_CUDA(cudaMemcpyAsync(ctx->root.p, root, sizeof(float) * 12 * n, kind, ctx->stream));
        CS_CUDA(cudaMemcpyAsync(ctx->pose.p, joint_pose, sizeof(float) * kJoints * 3 * n, kind, ctx->stream));
    }
    ctx->n_inst = n;
    ctx->train_valid = false;
    return CS_OK;
}

static int render_impl(cs_ctx *ctx, const cs_camera *cam, float4 *out, cs_frame_stats *stats,
                       float *contrib_tmpl = nullptr, bool train = false) {
    ctx->train_valid = false;  // the frame buffers are about to be rewritten
    if (!cam || !out) return fail(ctx, CS_ERR_ARG, "NULL camera or output");
    if (reinterpret_cast<uintptr_t>(out) & 15u) return fail(ctx, CS_ERR_ARG, "rgba_out must be 16-byte aligned");
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "no templates uploaded");
    if (cam->width < 1 || cam->height < 1 || cam->width > CS_MAX_IMAGE_SIDE || cam->height > CS_MAX_IMAGE_SIDE)
        return fail(ctx, CS_ERR_ARG, "image size %dx%d outside 1..%d", cam->width, cam->height, CS_MAX_IMAGE_SIDE);
    if (!(cam->fx > 0.f && cam->fy > 0.f && cam->near_z > 0.f) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return fail(ctx, CS_ERR_ARG, "focal lengths and near plane must be positive and finite");
    if (!window_ok(cam))
        return fail(ctx, CS_ERR_ARG, "window (%d, %d) + %dx%d of a %dx%d image: its edges must be on the %d-pixel "
                    "tile grid (or the image edge) and the window inside the full image", cam->win_x0, cam->win_y0,
                    cam->width, cam->height, cam->full_width, cam->full_height, kTile);
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(cam->R[i])) return fail(ctx, CS_ERR_ARG, "camera rotation not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(cam->t[i])) return fail(ctx, CS_ERR_ARG, "camera translation not finite");
    CS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    CamParams cp;
    cam_params(ctx, cam, cp);
    const int T = cp.tiles_x * cp.tiles_y;
    const int I = ctx->n_inst;
    const bool timing = ctx->stage_timing != 0;
    ctx->tiles_x = cp.tiles_x;
    ctx->frame_w = cam->width;
    ctx->frame_h = cam->height;
    ctx->frame_ox = cp.ox;
    ctx->frame_oy = cp.oy;
    ctx->tiles_y = cp.tiles_y;
    ctx->timed = false;
    int launched = 0;
    cudaEvent_t *ev = nullptr;
    if (timing) {
        // this frame uses the other set; that set's frame (two frames ago)
        // finished before the last frame's first host read, so this does not wait
        const int k = ctx->ev_cur ^ 1;
        CS_TRY(accumulate_stage_times(ctx, k));
        ctx->ev_cur = k;
        ev = ctx->ev[k];
    }
    CS_TRY(ensure(ctx, ctx->ranges, (size_t)T, "tile ranges"));
    CS_TRY(ensure(ctx, ctx->groups, (size_t)kMaxTemplates * kMaxLevels, "groups"));
    CS_TRY(ensure(ctx, ctx->vis, (size_t)std::max(I, 1), "visible list"));
    CS_TRY(ensure(ctx, ctx->cull, cull_scratch_words((size_t)std::max(I, 1)), "cull scratch"));
    if (timing) CS_CUDA(cudaEventRecord(ev[0], st));

    // 1. forward kinematics
    if (I > 0)
        launched += launch_fk(I, ctx->n_tpl, ctx->tid.p, ctx->pose.p, ctx->d_tpl, ctx->max_depth, ctx->B.p, st);
    if (timing) CS_CUDA(cudaEventRecord(ev[1], st));
    // 2. LoD band, instance cull, grouping by (template, level)
    int64_t S = 0;
    int proj_blocks = 0;
    if (I > 0) {
        launched += launch_cull_group(I, ctx->n_tpl, ctx->tid.p, ctx->root.p, ctx->d_tpl, cp, ctx->lod,
                          ctx->instance_cull, ctx->V.p, ctx->Cloc.p, ctx->vis.p, ctx->groups.p,
                          ctx->d_meta, ctx->cull.p, st);
        CS_CUDA(cudaGetLastError());
        CS_CUDA(cudaMemcpyAsync(ctx->h_meta, ctx->d_meta, kMetaWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CS_CUDA(cudaMemcpyAsync(ctx->h_groups, ctx->groups.p, kMaxGroups * sizeof(Group), cudaMemcpyDeviceToHost, st));
        CS_CUDA(cudaStreamSynchronize(st));
        ctx->visible = ctx->h_meta[kMetaVisible];
        ctx->n_groups = ctx->h_meta[kMetaGroups];
        set_depth_key_range(cp, ctx->h_meta);
        ctx->key_lo = cp.key_lo;
        S = ctx->h_meta[kMetaSplats];
        cp.n_splats = (uint32_t)S;
        proj_blocks = ctx->h_meta[kMetaBlocks];
        for (int l = 0; l < kMaxLevels; ++l) ctx->per_level[l] = ctx->h_meta[kMetaLevel0 + l];
        if (S >= 0x7fffffffLL) return fail(ctx, CS_ERR_CAPACITY, "more than 2^31 - 1 splats in a frame");
    } else {
        ctx->visible = ctx->n_groups = 0;
        for (int l = 0; l < kMaxLevels; ++l) ctx->per_level[l] = 0;
    }
    if (timing) CS_CUDA(cudaEventRecord(ev[2], st));
    ctx->S = S;
    // 3. LBS + EWA projection + SH colour
    const size_t Sa = (size_t)std::max<int64_t>(S, 1);
    CS_TRY(ensure(ctx, ctx->rec, Sa * kRecVec, "splat records"));
    CS_TRY(ensure(ctx, ctx->key, Sa, "depth keys"));
    CS_TRY(ensure(ctx, ctx->ids, Sa, "splat ids"));
    CS_TRY(ensure(ctx, ctx->key2, Sa, "depth keys (ping-pong)"));
    CS_TRY(ensure(ctx, ctx->ids2, Sa, "splat ids (ping-pong)"));
    CS_TRY(ensure(ctx, ctx->bins, Sa, "bin words"));
    CS_TRY(ensure(ctx, ctx->bins_sorted, Sa, "bin words in depth order"));
    CS_TRY(ensure(ctx, ctx->pair_off, bin_scan_blocks(Sa) + 1, "pair-count block sums"));
    CS_TRY(ensure(ctx, ctx->scratch, std::max(radix_scratch_words(Sa), scan_scratch_words(Sa + 1)), "scratch"));
    const TemplateArrays ta = template_arrays(ctx);
    if (S > 0)
        launched += launch_project(proj_blocks, ctx->groups.p, ctx->h_groups, ctx->n_groups, ctx->tpl_host.data(),
                                   ctx->vis.p, ctx->B.p, ctx->V.p, ctx->root.p, ta, ctx->d_tpl, cp, ctx->lod,
                                   ctx->skin_mode, ctx->sh_frame, ctx->rec.p, ctx->key.p, ctx->bins.p, st);
    if (timing) CS_CUDA(cudaEventRecord(ev[3], st));
    // 4. depth sort of the splats (stable, ties by splat id)
    int ob = 0;
    if (S > 0) launched += radix_sort_u32(ctx->key.p, ctx->ids.p, ctx->key2.p, ctx->ids2.p, (uint32_t)S,
                                          depth_key_bits(cp.key_lo, cp.key_hi), ctx->scratch.p, st, &ob,
                                          ctx->bins.p, ctx->bins_sorted.p, true);
    ctx->order_buf = ob;
    uint32_t *order = ob ? ctx->ids2.p : ctx->ids.p;
    uint32_t *sorted_keys = ob ? ctx->key2.p : ctx->key.p;
    if (timing) CS_CUDA(cudaEventRecord(ev[4], st));
    // 5. pair offsets in depth order and pair emission
    // (the per-block sums of the pair counts live in pair_off)
    const size_t nbs = bin_scan_blocks((size_t)S);
    launched += bin_scan_sums(ctx->bins_sorted.p, (uint32_t)S, ctx->pair_off.p, st);
    CS_CUDA(cudaGetLastError());
    if (stats && S > 0) launched += launch_count_live((uint32_t)S, sorted_keys, ctx->d_meta + kMetaWords - 1, st);
    if (S > 0) CS_CUDA(cudaMemcpyAsync(ctx->h_pairs, ctx->pair_off.p + nbs, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    else ctx->h_pairs[0] = 0;
    if (stats) CS_CUDA(cudaMemcpyAsync(ctx->h_pairs + 1, ctx->d_meta + kMetaWords - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CS_CUDA(cudaStreamSynchronize(st));
    const int64_t P = ctx->h_pairs[0];
    ctx->P = P;
    const size_t Pa = (size_t)std::max<int64_t>(P, 1);
    CS_TRY(ensure(ctx, ctx->ptile, Pa, "pair tiles"));
    CS_TRY(ensure(ctx, ctx->ptile2, Pa, "pair tiles (ping-pong)"));
    CS_TRY(ensure(ctx, ctx->pval, Pa, "pair splats"));
    CS_TRY(ensure(ctx, ctx->pval2, Pa, "pair splats (ping-pong)"));
    CS_TRY(ensure(ctx, ctx->scratch, std::max(radix_scratch_words(Pa), radix_scratch_words(Sa)), "scratch"));
    if (P > 0) launched += launch_emit_pairs_scan((uint32_t)S, order, ctx->bins_sorted.p, ctx->pair_off.p, ctx->rec.p,
                                                  cp.tiles_x, (uint32_t)T, ctx->ptile.p, ctx->pval.p, st);
    if (timing) CS_CUDA(cudaEventRecord(ev[5], st));
    // 6. stable sort of the pairs by tile
    int pb = 0;
    if (P > 0) launched += radix_sort_u16(ctx->ptile.p, ctx->pval.p, ctx->ptile2.p, ctx->pval2.p, (uint32_t)P,
                                          bits_for((uint32_t)T), ctx->scratch.p, st, &pb);
    ctx->pair_buf = pb;
    uint16_t *ptile = pb ? ctx->ptile2.p : ctx->ptile.p;
    uint32_t *pval = pb ? ctx->pval2.p : ctx->pval.p;
    if (timing) CS_CUDA(cudaEventRecord(ev[6], st));
    // 7. per-tile ranges
    CS_CUDA(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(uint2) * T, st));
    launched += launch_tile_ranges((uint32_t)P, ptile, ctx->ranges.p, (uint32_t)T, st);
    if (timing) CS_CUDA(cudaEventRecord(ev[7], st));
    // 8. compositing
    {
        const size_t ms = blend_max_slots((size_t)T, (size_t)P), mc = blend_max_chunks((size_t)T, (size_t)P);
        CS_TRY(ensure(ctx, ctx->bw_slot, (size_t)T, "blend slots"));
        CS_TRY(ensure(ctx, ctx->bw_tile, ms, "blend slot tiles"));
        CS_TRY(ensure(ctx, ctx->bw_meta, kBlendMetaWords, "blend plan"));
        CS_TRY(ensure(ctx, ctx->bw_pp, (size_t)T, "blend pair-parallel tiles"));
        CS_TRY(ensure(ctx, ctx->bw_chunk0, ms + 1, "blend chunk offsets"));
        CS_TRY(ensure(ctx, ctx->bw_done, ms, "blend slot flags"));
        CS_TRY(ensure(ctx, ctx->bw_state, ms * 256, "blend pass-1 state"));
        CS_TRY(ensure(ctx, ctx->bw_part, mc * 256, "blend chunk partials"));
        CS_TRY(ensure(ctx, ctx->bw_cslot, mc, "blend chunk slots"));
        CS_TRY(ensure(ctx, ctx->bw_stop, ms * 256, "blend stop chunks"));
    }
    BlendWork bw{ctx->bw_slot.p, ctx->bw_tile.p, ctx->bw_chunk0.p, ctx->bw_done.p, ctx->bw_state.p, ctx->bw_part.p,
                 ctx->bw_meta.p, ctx->bw_stop.p, nullptr};
    bw.pp_tile = ctx->bw_pp.p;
    bw.chunk_slot = ctx->bw_cslot.p;
    bw.ox = cp.ox;
    bw.oy = cp.oy;
    bw.items = ctx->blend_items;
    bw.n_pairs = (uint32_t)P;
    bw.max_slots = (uint32_t)blend_max_slots((size_t)T, (size_t)P);
    bw.max_chunks = (uint32_t)blend_max_chunks((size_t)T, (size_t)P);
    if (contrib_tmpl) {
        CS_TRY(ensure(ctx, ctx->contrib_s, Sa, "splat contributions"));
        CS_CUDA(cudaMemsetAsync(ctx->contrib_s.p, 0, Sa * sizeof(float), st));
        bw.contrib = ctx->contrib_s.p;
    }
    if (train) {
        const size_t npix = (size_t)cam->width * cam->height;
        CS_TRY(ensure(ctx, ctx->px_end, npix, "per-pixel list ends"));
        CS_TRY(ensure(ctx, ctx->px_fin, npix, "per-pixel final state"));
        CS_TRY(ensure(ctx, ctx->px_bnd, bwd_boundary_slots((size_t)P) * 256, "chunk-boundary states"));
        const size_t nt = (size_t)std::max(T, 1), tc = train_max_chunks(nt, (size_t)P);
        CS_TRY(ensure(ctx, ctx->bwd_cnt, nt, "training chunk counts"));
        CS_TRY(ensure(ctx, ctx->bwd_chunk0, nt + 1, "training chunk offsets"));
        CS_TRY(ensure(ctx, ctx->bwd_scratch, scan_scratch_words(nt), "training scan scratch"));
        CS_TRY(ensure(ctx, ctx->t_part, tc * 256, "training chunk partials"));
        CS_TRY(ensure(ctx, ctx->t_last, tc * 256, "training chunk ends"));
        CS_TRY(ensure(ctx, ctx->t_state, npix, "training stop states"));
        CS_TRY(ensure(ctx, ctx->t_slast, npix, "training stop ends"));
        CS_TRY(ensure(ctx, ctx->t_stop, npix, "training stop chunks"));
        bw.px_end = ctx->px_end.p;
        bw.px_fin = ctx->px_fin.p;
        bw.px_bnd = ctx->px_bnd.p;
        bw.t_cnt = ctx->bwd_cnt.p;
        bw.t_chunk0 = ctx->bwd_chunk0.p;
        bw.t_scan = ctx->bwd_scratch.p;
        bw.t_part = ctx->t_part.p;
        bw.t_last = ctx->t_last.p;
        bw.t_state = ctx->t_state.p;
        bw.t_slast = ctx->t_slast.p;
        bw.t_stop = ctx->t_stop.p;
    }
    launched += launch_blend(cp.tiles_x, cp.tiles_y, cam->width, cam->height, ctx->ranges.p, pval, ctx->rec.p, out,
                             bw, (uint32_t)P, st);
    if (contrib_tmpl)
        launched += launch_contrib_to_template((int)S, ctx->groups.p, ctx->n_groups, ctx->d_tpl, ctx->d_lod_idx,
                                               ctx->contrib_s.p, contrib_tmpl, st);
    if (timing) CS_CUDA(cudaEventRecord(ev[8], st));
    CS_CUDA(cudaGetLastError());
    ctx->timed = timing;
    ctx->ev_pending[ctx->ev_cur] = timing;
    ctx->launches = launched;
    if (train) {
        ctx->train_valid = true;
        ctx->train_cp = cp;
        ctx->train_proj_blocks = proj_blocks;
    }
    if (stats) {
        stats->instances = I;
        stats->instances_visible = ctx->visible;
        for (int l = 0; l < CS_MAX_LEVELS; ++l) stats->instances_per_level[l] = ctx->per_level[l];
        stats->splats = S;
        stats->splats_live = S > 0 ? (int64_t)ctx->h_pairs[1] : 0;
        stats->pairs = P;
        stats->tiles_x = cp.tiles_x;
        stats->tiles_y = cp.tiles_y;
        stats->kernel_launches = launched;
        stats->depth_key_bits = S > 0 ? depth_key_bits(cp.key_lo, cp.key_hi) : 0;
    }
    return CS_OK;
}

int cs_render(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats) {
    if (!ctx) return CS_ERR_ARG;
    return render_impl(ctx, cam, reinterpret_cast<float4 *>(rgba_out), stats);
}

int cs_render_contrib(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, float *contrib_out,
                      cs_frame_stats *stats) {
    if (!ctx) return CS_ERR_ARG;
    if (!contrib_out) return fail(ctx, CS_ERR_ARG, "NULL contribution array");
    if (reinterpret_cast<uintptr_t>(contrib_out) & 3u) return fail(ctx, CS_ERR_ARG, "contrib_out must be 4-byte aligned");
    return render_impl(ctx, cam, reinterpret_cast<float4 *>(rgba_out), stats, contrib_out);
}

int cs_lod_features(cs_ctx *ctx, float *feat_out) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "no templates uploaded");
    if (!feat_out || (reinterpret_cast<uintptr_t>(feat_out) & 15u))
        return fail(ctx, CS_ERR_ARG, "feat_out must be a 16-byte aligned device pointer");
    CS_CUDA(cudaSetDevice(ctx->device));
    const TemplateArrays ta = template_arrays(ctx);
    launch_lod_features((int)ctx->n_gauss_total, ctx->n_tpl, ctx->d_tpl, ta, feat_out, ctx->stream);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

int cs_lod_targets(cs_ctx *ctx, int32_t n_bands, const float *contrib, float floor_, float *target_out) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "no templates uploaded");
    if (n_bands < 1 || n_bands > CS_MAX_LEVELS) return fail(ctx, CS_ERR_ARG, "n_bands must be 1..%d", CS_MAX_LEVELS);
    if (!(floor_ > 0.0f) || !std::isfinite(floor_)) return fail(ctx, CS_ERR_ARG, "floor must be > 0");
    if (!contrib || !target_out || (reinterpret_cast<uintptr_t>(contrib) & 3u) ||
        (reinterpret_cast<uintptr_t>(target_out) & 3u))
        return fail(ctx, CS_ERR_ARG, "NULL or misaligned contrib / target_out");
    CS_CUDA(cudaSetDevice(ctx->device));
    launch_lod_targets((int)ctx->n_gauss_total, ctx->n_tpl, n_bands, ctx->d_tpl, contrib, floor_, target_out,
                       ctx->stream);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

int cs_lod_rank(cs_ctx *ctx, const float *score, uint32_t *order_out) {
    if (!ctx) return CS_ERR_ARG;
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "no templates uploaded");
    if (!score || !order_out || (reinterpret_cast<uintptr_t>(score) & 3u) ||
        (reinterpret_cast<uintptr_t>(order_out) & 3u))
        return fail(ctx, CS_ERR_ARG, "NULL or misaligned score / order_out");
    CS_CUDA(cudaSetDevice(ctx->device));
    const size_t n = ctx->n_gauss_total;
    // temporary sort buffers: an offline call, so plain allocations
    // every array starts on a 16-byte boundary
    const size_t w32 = (n + 3) & ~size_t(3), w16 = ((n + 1) / 2 + 3) & ~size_t(3);
    const size_t words = 4 * w32 + 2 * w16 + radix_scratch_words(n) + 4;
    uint32_t *buf = nullptr;
    if (cudaMalloc(&buf, words * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, CS_ERR_OOM, "cs_lod_rank: %zu bytes of sort buffers", words * sizeof(uint32_t));
    }
    uint32_t *k0 = buf, *v0 = k0 + w32, *k1 = v0 + w32, *v1 = k1 + w32;
    uint16_t *t0 = reinterpret_cast<uint16_t *>(v1 + w32), *t1 = reinterpret_cast<uint16_t *>(v1 + w32 + w16);
    uint32_t *scratch = v1 + w32 + 2 * w16;
    lod_rank((int)n, ctx->n_tpl, ctx->d_tpl, score, order_out, k0, v0, k1, v1, t0, t1, scratch, ctx->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(ctx, CS_ERR_CUDA, "cs_lod_rank: %s", cudaGetErrorString(e));
    return CS_OK;
}

int cs_render_train(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats) {
    if (!ctx) return CS_ERR_ARG;
    if (cam && (cam->full_width != 0 || cam->full_height != 0))
        return fail(ctx, CS_ERR_ARG, "training frames render the full image (no window)");
    if (ctx->storage != CS_STORE_FP32) return fail(ctx, CS_ERR_STATE, "gradients need FP32 template storage");
    return render_impl(ctx, cam, reinterpret_cast<float4 *>(rgba_out), stats, nullptr, true);
}

int cs_backward(cs_ctx *ctx, const float *dl_drgba, const cs_grads *grads) {
    if (!ctx) return CS_ERR_ARG;
    if (!dl_drgba || !grads || (reinterpret_cast<uintptr_t>(dl_drgba) & 15u))
        return fail(ctx, CS_ERR_ARG, "NULL or misaligned dl_drgba / grads");
    if (!ctx->train_valid) return fail(ctx, CS_ERR_STATE, "no training frame (cs_render_train) since the last change");
    CS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const CamParams &cp = ctx->train_cp;
    const size_t S = (size_t)std::max<int64_t>(ctx->S, 1), G = std::max<size_t>(ctx->n_gauss_total, 1);
    const size_t I = (size_t)std::max(ctx->n_inst, 1);
    CS_TRY(ensure(ctx, ctx->dsplat, S * 3, "splat gradients"));
    const size_t nt = (size_t)std::max(cp.tiles_x * cp.tiles_y, 1);
    CS_TRY(ensure(ctx, ctx->bwd_cnt, nt, "backward chunk counts"));
    CS_TRY(ensure(ctx, ctx->bwd_chunk0, nt + 1, "backward chunk offsets"));
    CS_TRY(ensure(ctx, ctx->bwd_scratch, scan_scratch_words(nt), "backward scan scratch"));
    CS_TRY(ensure(ctx, ctx->g_cov, G * 6, "covariance gradients"));
    CS_TRY(ensure(ctx, ctx->g_B, I * kJoints * 12, "skinning-transform gradients"));
    // destinations the caller does not want go to one scratch buffer
    CS_TRY(ensure(ctx, ctx->g_dummy, std::max(G * 48, I * kJoints * 3), "gradient scratch"));
    CS_CUDA(cudaMemsetAsync(ctx->dsplat.p, 0, S * 3 * sizeof(float4), st));
    CS_CUDA(cudaMemsetAsync(ctx->g_cov.p, 0, G * 6 * sizeof(float), st));
    CS_CUDA(cudaMemsetAsync(ctx->g_B.p, 0, I * kJoints * 12 * sizeof(float), st));
    BackwardArgs a{};
    a.tiles_x = cp.tiles_x;
    a.tiles_y = cp.tiles_y;
    a.W = cp.W;
    a.H = cp.H;
    a.n_pairs = (uint32_t)ctx->P;
    a.ranges = ctx->ranges.p;
    a.pval = ctx->pair_buf ? ctx->pval2.p : ctx->pval.p;
    a.rec = ctx->rec.p;
    a.px_end = ctx->px_end.p;
    a.px_fin = ctx->px_fin.p;
    a.px_bnd = ctx->px_bnd.p;
    a.chunk_cnt = ctx->bwd_cnt.p;
    a.chunk0 = ctx->bwd_chunk0.p;
    a.scan_scratch = ctx->bwd_scratch.p;
    a.dl_drgba = reinterpret_cast<const float4 *>(dl_drgba);
    a.dsplat = ctx->dsplat.p;
    a.proj_blocks = ctx->S > 0 ? ctx->train_proj_blocks : 0;
    a.groups = ctx->groups.p;
    a.n_groups = ctx->n_groups;
    a.vis = ctx->vis.p;
    a.B = ctx->B.p;
    a.V = ctx->V.p;
    a.Cloc = ctx->Cloc.p;
    a.root = ctx->root.p;
    a.ta = template_arrays(ctx);
    a.tpls = ctx->d_tpl;
    a.cam = cp;
    a.lod = ctx->lod;
    a.skin_mode = ctx->skin_mode;
    a.sh_frame = ctx->sh_frame;
    float *dummy = ctx->g_dummy.p;
    a.g_mean = grads->means ? grads->means : dummy;
    a.g_cov = ctx->g_cov.p;
    a.g_opacity = grads->opacity ? grads->opacity : dummy;
    a.g_sh = grads->sh ? grads->sh : dummy;
    a.g_B = ctx->g_B.p;
    a.n_inst = ctx->n_inst;
    a.n_tpl = ctx->n_tpl;
    a.tid = ctx->tid.p;
    a.pose = ctx->pose.p;
    a.g_pose = grads->pose ? grads->pose : dummy;
    a.n_gauss = (int)ctx->n_gauss_total;
    a.scale = ctx->d_scale;
    a.quat = ctx->d_quat;
    a.g_scale = grads->scales ? grads->scales : dummy;
    a.g_quat = grads->quats ? grads->quats : dummy;
    launch_backward(a, st);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

int cs_render_to_host(cs_ctx *ctx, const cs_camera *cam, float *rgba_host, cs_frame_stats *stats) {
    if (!ctx) return CS_ERR_ARG;
    if (!cam || !rgba_host) return fail(ctx, CS_ERR_ARG, "NULL camera or output");
    if (cam->width < 1 || cam->height < 1 || cam->width > CS_MAX_IMAGE_SIDE || cam->height > CS_MAX_IMAGE_SIDE)
        return fail(ctx, CS_ERR_ARG, "image size %dx%d outside 1..%d", cam->width, cam->height, CS_MAX_IMAGE_SIDE);
    CS_CUDA(cudaSetDevice(ctx->device));
    // page-locked host memory mapped into the device's address space: the
    // compositing kernels write the image straight into it (the stores cross
    // the host link while the frame is composited; no separate copy)
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, rgba_host) != cudaSuccess) {
        cudaGetLastError();  // not a CUDA-known pointer: plain pageable memory
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer &&
        (reinterpret_cast<uintptr_t>(at.devicePointer) & 15u) == 0) {
        CS_TRY(render_impl(ctx, cam, reinterpret_cast<float4 *>(at.devicePointer), stats));
        CS_CUDA(cudaStreamSynchronize(ctx->stream));
        return CS_OK;
    }
    const size_t npix = (size_t)cam->width * cam->height;
    CS_TRY(ensure(ctx, ctx->img, npix, "image"));
    CS_TRY(render_impl(ctx, cam, ctx->img.p, stats));
    CS_CUDA(cudaMemcpyAsync(rgba_host, ctx->img.p, npix * sizeof(float4), cudaMemcpyDeviceToHost, ctx->stream));
    CS_CUDA(cudaStreamSynchronize(ctx->stream));
    return CS_OK;
}

int cs_get_stage_times(cs_ctx *ctx, float *ms, int32_t n, int32_t average, int64_t *frames_out) {
    if (!ctx || !ms || n < 0) return -CS_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        fail(ctx, CS_ERR_CUDA, "cudaSetDevice failed");
        return -CS_ERR_CUDA;
    }
    const int k = std::min<int>(n, kStages);
    if (average) {
        for (int s = 0; s < 2; ++s) {
            int rc = accumulate_stage_times(ctx, s);
            if (rc != CS_OK) return -rc;
        }
        if (ctx->stage_frames == 0) {
            fail(ctx, CS_ERR_STATE, "no timed frame since the last average");
            return -CS_ERR_STATE;
        }
        for (int i = 0; i < k; ++i) ms[i] = (float)(ctx->stage_sum[i] / (double)ctx->stage_frames);
        if (frames_out) *frames_out = ctx->stage_frames;
        for (int i = 0; i < kStages; ++i) ctx->stage_sum[i] = 0.0;
        ctx->stage_frames = 0;
        return k;
    }
    if (!ctx->timed) {
        fail(ctx, CS_ERR_STATE, "no timed frame (stage_timing off or no render yet)");
        return -CS_ERR_STATE;
    }
    cudaEvent_t *ev = ctx->ev[ctx->ev_cur];
    if (cudaEventSynchronize(ev[kStages]) != cudaSuccess) {
        fail(ctx, CS_ERR_CUDA, "event synchronise failed");
        return -CS_ERR_CUDA;
    }
    for (int i = 0; i < k; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) != cudaSuccess) {
            fail(ctx, CS_ERR_CUDA, "event timing failed");
            return -CS_ERR_CUDA;
        }
        ms[i] = t;
    }
    if (frames_out) *frames_out = 1;
    return k;
}

int cs_memory_stats(cs_ctx *ctx, cs_memory_stats_t *out) {
    if (!ctx || !out) return CS_ERR_ARG;
    const int64_t per_g = ctx->storage == CS_STORE_BF16 ? (int64_t)(2 * sizeof(uint4))
                                                       : (int64_t)(sizeof(float4) * 3 + sizeof(float2) + sizeof(uint32_t));
    int64_t tb = (int64_t)ctx->n_gauss_total * per_g + (int64_t)ctx->sh_planes_total * 16 +
                 (int64_t)ctx->n_tpl * sizeof(TemplateInfo) +
                 (int64_t)ctx->lod_idx_cap * sizeof(uint32_t);
    int64_t ib = bytes_of(ctx->tid) + bytes_of(ctx->vis) + bytes_of(ctx->cull) + bytes_of(ctx->root) + bytes_of(ctx->pose) +
                 bytes_of(ctx->B) + bytes_of(ctx->V) + bytes_of(ctx->Cloc) + bytes_of(ctx->groups);
    int64_t fb = bytes_of(ctx->rec) + bytes_of(ctx->key) + bytes_of(ctx->ids) + bytes_of(ctx->key2) +
                 bytes_of(ctx->ids2) + bytes_of(ctx->bins) + bytes_of(ctx->bins_sorted) + bytes_of(ctx->pair_off) + bytes_of(ctx->pval) +
                 bytes_of(ctx->pval2) + bytes_of(ctx->scratch) + bytes_of(ctx->rect) + bytes_of(ctx->ranges) +
                 bytes_of(ctx->ptile) + bytes_of(ctx->ptile2) + bytes_of(ctx->img) + bytes_of(ctx->bw_slot) +
                 bytes_of(ctx->bw_tile) + bytes_of(ctx->bw_meta) + bytes_of(ctx->bw_chunk0) + bytes_of(ctx->bw_done) +
                 bytes_of(ctx->bw_state) + bytes_of(ctx->bw_part) + bytes_of(ctx->bw_stop) + bytes_of(ctx->bw_pp) + bytes_of(ctx->bw_cslot) + bytes_of(ctx->contrib_s) +
                 bytes_of(ctx->px_end) + bytes_of(ctx->px_fin) + bytes_of(ctx->px_bnd) + bytes_of(ctx->bwd_cnt) +
                 bytes_of(ctx->bwd_chunk0) + bytes_of(ctx->bwd_scratch) + bytes_of(ctx->t_part) + bytes_of(ctx->t_last) +
                 bytes_of(ctx->t_state) + bytes_of(ctx->t_slast) + bytes_of(ctx->t_stop) + bytes_of(ctx->dsplat) +
                 bytes_of(ctx->g_cov) +
                 bytes_of(ctx->g_B) + bytes_of(ctx->g_dummy);
    out->template_bytes = tb;
    out->instance_bytes = ib;
    out->frame_bytes = fb;
    out->total_bytes = tb + ib + fb;
    return CS_OK;
}

int cs_debug_fail_allocs(cs_ctx *ctx, int32_t after) {
    if (!ctx) return CS_ERR_ARG;
    ctx->fail_after = after < 0 ? -1 : after;
    return CS_OK;
}

int cs_debug_checks(cs_ctx *ctx, uint32_t *failed, int32_t *enabled) {
    if (!ctx || !failed || !enabled) return ctx ? fail(ctx, CS_ERR_ARG, "cs_debug_checks: NULL output") : CS_ERR_ARG;
    CS_CUDA(cudaSetDevice(ctx->device));
    CS_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint32_t w = check_word_geometry() | check_word_sort() | check_word_blend();
    if (w == 0xFFFFFFFFu) return fail(ctx, CS_ERR_CUDA, "cs_debug_checks: reading the check word failed");
    *failed = w;
    *enabled = CS_CHECKS ? 1 : 0;
    return CS_OK;
}

int cs_debug_blend_items(cs_ctx *ctx, int32_t mode) {
    if (!ctx) return CS_ERR_ARG;
    if (mode != CS_BLEND_ITEMS_AUTO && mode != CS_BLEND_ITEMS_TILES && mode != CS_BLEND_ITEMS_BLOCKS)
        return fail(ctx, CS_ERR_ARG, "cs_debug_blend_items: unknown mode");
    ctx->blend_items = mode;
    return CS_OK;
}

int cs_debug_read(cs_ctx *ctx, int32_t which, void *host_dst, size_t bytes, size_t *size_out) {
    if (!ctx) return CS_ERR_ARG;
    CS_CUDA(cudaSetDevice(ctx->device));
    const void *src = nullptr;
    size_t size = 0;
    const int T = ctx->tiles_x * ctx->tiles_y;
    switch (which) {
        case CS_DBG_SKIN_B: src = ctx->B.p; size = (size_t)ctx->n_inst * kJoints * 12 * sizeof(float); break;
        case CS_DBG_VISIBLE: src = ctx->vis.p; size = (size_t)ctx->visible * sizeof(int32_t); break;
        case CS_DBG_GROUPS: src = ctx->groups.p; size = (size_t)ctx->n_groups * sizeof(Group); break;
        case CS_DBG_RECORDS:
            // the 48-byte records expanded to the 16-float view
            if (ctx->S > 0) {
                CS_TRY(ensure(ctx, ctx->dbg_rec, (size_t)ctx->S * 4, "debug records"));
                CS_CUDA(cudaMemsetAsync(ctx->dbg_rec.p, 0, (size_t)ctx->S * 4 * sizeof(float4), ctx->stream));
                launch_debug_records((int)ctx->S, ctx->rec.p, ctx->order_buf ? ctx->key2.p : ctx->key.p,
                                     ctx->order_buf ? ctx->ids2.p : ctx->ids.p, ctx->key_lo, ctx->dbg_rec.p,
                                     ctx->stream);
                CS_CUDA(cudaGetLastError());
            }
            src = ctx->dbg_rec.p;
            size = (size_t)ctx->S * 4 * sizeof(float4);
            break;
        case CS_DBG_DEPTH_KEYS: src = ctx->order_buf ? ctx->key2.p : ctx->key.p; size = (size_t)ctx->S * 4; break;
        case CS_DBG_RECTS:
            // recomputed from the records of the last frame
            if (ctx->S > 0) {
                CS_TRY(ensure(ctx, ctx->rect, (size_t)ctx->S, "tile rects"));
                launch_debug_rects((int)ctx->S, ctx->rec.p, ctx->bins.p, ctx->frame_w, ctx->frame_h, ctx->frame_ox,
                                   ctx->frame_oy, ctx->rect.p, ctx->stream);
                CS_CUDA(cudaGetLastError());
            }
            src = ctx->rect.p;
            size = (size_t)ctx->S * 8;
            break;
        case CS_DBG_DEPTH_ORDER: src = ctx->order_buf ? ctx->ids2.p : ctx->ids.p; size = (size_t)ctx->S * 4; break;
        case CS_DBG_PAIR_TILES: src = ctx->pair_buf ? ctx->ptile2.p : ctx->ptile.p; size = (size_t)ctx->P * 2; break;
        case CS_DBG_PAIR_SPLATS: src = ctx->pair_buf ? ctx->pval2.p : ctx->pval.p; size = (size_t)ctx->P * 4; break;
        case CS_DBG_TILE_RANGES: src = ctx->ranges.p; size = (size_t)T * 8; break;
        default: return fail(ctx, CS_ERR_ARG, "unknown debug buffer %d", which);
    }
    if (size_out) *size_out = size;
    CS_CUDA(cudaStreamSynchronize(ctx->stream));
    size_t n = std::min(bytes, size);
    if (n > 0) {
        if (!host_dst || !src) return fail(ctx, CS_ERR_ARG, "NULL destination or empty buffer");
        CS_CUDA(cudaMemcpy(host_dst, src, n, cudaMemcpyDeviceToHost));
    }
    return CS_OK;
}

// ---------------------------------------------------------------------------
// cs_render_static: cs_render with its per-frame scratch in one fixed device
// array instead of context-owned allocations.  For callers that must not
// allocate device memory during a frame (real-time threads with an
// allocation ban, engines that own the GPU memory budget).  The array is a
// file-scope __device__ object: every GPU that loads the library holds it
// until the process exits.  Host code cannot use its name as a device
// address; the address comes from cudaGetSymbolAddress, once per device.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

constexpr size_t kStaticSplats = 65536;   // splats of visible instances per frame
constexpr size_t kStaticPairs = 262144;   // (tile, splat) pairs per frame
constexpr size_t kStaticTiles = 16384;    // 16x16 tiles per image (e.g. 2048 x 2048)
constexpr size_t kStaticScratchWords = 98304;  // histograms and scan partials

constexpr size_t a256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffRec = 0;
constexpr size_t kOffKey = kOffRec + a256(kStaticSplats * kRecVec * sizeof(float4));
constexpr size_t kOffIds = kOffKey + a256(kStaticSplats * 4);
constexpr size_t kOffKey2 = kOffIds + a256(kStaticSplats * 4);
constexpr size_t kOffIds2 = kOffKey2 + a256(kStaticSplats * 4);
constexpr size_t kOffBins = kOffIds2 + a256(kStaticSplats * 4);
constexpr size_t kOffBinsSorted = kOffBins + a256(kStaticSplats * 4);
constexpr size_t kOffPairOff = kOffBinsSorted + a256(kStaticSplats * 4);
constexpr size_t kOffPtile = kOffPairOff + a256((kStaticSplats + 1) * 4);
constexpr size_t kOffPtile2 = kOffPtile + a256(kStaticPairs * 2);
constexpr size_t kOffPval = kOffPtile2 + a256(kStaticPairs * 2);
constexpr size_t kOffPval2 = kOffPval + a256(kStaticPairs * 4);
constexpr size_t kOffRanges = kOffPval2 + a256(kStaticPairs * 4);
constexpr size_t kOffScratch = kOffRanges + a256(kStaticTiles * sizeof(uint2));
constexpr size_t kStaticSlots = blend_max_slots(kStaticTiles, kStaticPairs);
constexpr size_t kStaticChunks = blend_max_chunks(kStaticTiles, kStaticPairs);
constexpr size_t kOffBwSlot = kOffScratch + a256(kStaticScratchWords * 4);
constexpr size_t kOffBwTile = kOffBwSlot + a256(kStaticTiles * 4);
constexpr size_t kOffBwMeta = kOffBwTile + a256(kStaticSlots * 4);
constexpr size_t kOffBwChunk0 = kOffBwMeta + a256(kBlendMetaWords * 4);
constexpr size_t kOffBwDone = kOffBwChunk0 + a256((kStaticSlots + 1) * 4);
constexpr size_t kOffBwState = kOffBwDone + a256(kStaticSlots * 4);
constexpr size_t kOffBwPart = kOffBwState + a256(kStaticSlots * 256 * sizeof(float4));
constexpr size_t kOffBwStop = kOffBwPart + a256(kStaticChunks * 256 * sizeof(float4));
constexpr size_t kOffBwPp = kOffBwStop + a256(kStaticSlots * 256 * 4);
constexpr size_t kOffBwCslot = kOffBwPp + a256(kStaticTiles * 4);
constexpr size_t kStaticBytes = kOffBwCslot + a256(kStaticChunks * 4);  // about 9.9 MB
static_assert(kStaticBytes > 9800000 && kStaticBytes < 10000000, "the documented size of the static frame scratch");

}  // namespace

// The frame scratch of cs_render_static (file scope, internal linkage).
static __device__ __align__(256) unsigned char g_static_frame[kStaticBytes];

namespace {

std::mutex g_static_mu;
constexpr int kStaticMaxDevices = 64;
unsigned char *g_static_addr[kStaticMaxDevices] = {};

// Device address of g_static_frame on the current device (looked up once per
// device; the device must be current).
int static_frame_address(cs_ctx *ctx, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (ctx->device < 0 || ctx->device >= kStaticMaxDevices)
        return fail(ctx, CS_ERR_ARG, "cs_render_static supports devices 0..%d", kStaticMaxDevices - 1);
    if (!g_static_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_frame);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(ctx, CS_ERR_CUDA, "cudaGetSymbolAddress of the static frame scratch failed: %s",
                        cudaGetErrorString(e));
        }
        g_static_addr[ctx->device] = static_cast<unsigned char *>(p);
    }
    *out = g_static_addr[ctx->device];
    return CS_OK;
}

}  // namespace

extern "C" {

int cs_render_static(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats) {
    if (!ctx) return CS_ERR_ARG;
    // this call rewrites the context's skinning, visibility and group
    // buffers that a training frame's backward reads: that frame is gone
    ctx->train_valid = false;
    float4 *out = reinterpret_cast<float4 *>(rgba_out);
    if (!cam || !out) return fail(ctx, CS_ERR_ARG, "NULL camera or output");
    if (reinterpret_cast<uintptr_t>(out) & 15u) return fail(ctx, CS_ERR_ARG, "rgba_out must be 16-byte aligned");
    if (ctx->n_tpl == 0) return fail(ctx, CS_ERR_STATE, "no templates uploaded");
    if (cam->width < 1 || cam->height < 1 || cam->width > CS_MAX_IMAGE_SIDE || cam->height > CS_MAX_IMAGE_SIDE)
        return fail(ctx, CS_ERR_ARG, "image size %dx%d outside 1..%d", cam->width, cam->height, CS_MAX_IMAGE_SIDE);
    if (!(cam->fx > 0.f && cam->fy > 0.f && cam->near_z > 0.f) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return fail(ctx, CS_ERR_ARG, "focal lengths and near plane must be positive and finite");
    if (!window_ok(cam))
        return fail(ctx, CS_ERR_ARG, "window (%d, %d) + %dx%d of a %dx%d image: its edges must be on the %d-pixel "
                    "tile grid (or the image edge) and the window inside the full image", cam->win_x0, cam->win_y0,
                    cam->width, cam->height, cam->full_width, cam->full_height, kTile);
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(cam->R[i])) return fail(ctx, CS_ERR_ARG, "camera rotation not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(cam->t[i])) return fail(ctx, CS_ERR_ARG, "camera translation not finite");
    CS_CUDA(cudaSetDevice(ctx->device));
    unsigned char *base = nullptr;
    CS_TRY(static_frame_address(ctx, &base));
    cudaStream_t st = ctx->stream;
    CamParams cp;
    cam_params(ctx, cam, cp);
    const int T = cp.tiles_x * cp.tiles_y;
    if ((size_t)T > kStaticTiles)
        return fail(ctx, CS_ERR_CAPACITY, "cs_render_static: %d tiles exceed the static limit of %zu "
                    "(image at most 2048 x 2048)", T, kStaticTiles);
    const int I = ctx->n_inst;
    float4 *rec = reinterpret_cast<float4 *>(base + kOffRec);
    uint32_t *key = reinterpret_cast<uint32_t *>(base + kOffKey);
    uint32_t *ids = reinterpret_cast<uint32_t *>(base + kOffIds);
    uint32_t *key2 = reinterpret_cast<uint32_t *>(base + kOffKey2);
    uint32_t *ids2 = reinterpret_cast<uint32_t *>(base + kOffIds2);
    uint32_t *bins = reinterpret_cast<uint32_t *>(base + kOffBins);
    uint32_t *bins_sorted = reinterpret_cast<uint32_t *>(base + kOffBinsSorted);
    uint32_t *pair_off = reinterpret_cast<uint32_t *>(base + kOffPairOff);
    uint16_t *ptile0 = reinterpret_cast<uint16_t *>(base + kOffPtile);
    uint16_t *ptile1 = reinterpret_cast<uint16_t *>(base + kOffPtile2);
    uint32_t *pval0 = reinterpret_cast<uint32_t *>(base + kOffPval);
    uint32_t *pval1 = reinterpret_cast<uint32_t *>(base + kOffPval2);
    uint2 *ranges = reinterpret_cast<uint2 *>(base + kOffRanges);
    uint32_t *scratch = reinterpret_cast<uint32_t *>(base + kOffScratch);
    int launched = 0;

    // forward kinematics, LoD, cull and grouping (instance buffers were sized
    // by cs_set_instances; nothing is allocated here)
    if (I > 0) launched += launch_fk(I, ctx->n_tpl, ctx->tid.p, ctx->pose.p, ctx->d_tpl, ctx->max_depth, ctx->B.p, st);
    int64_t S = 0;
    int visible = 0, n_groups = 0, proj_blocks = 0, per_level[kMaxLevels] = {0, 0, 0, 0};
    if (I > 0) {
        launched += launch_cull_group(I, ctx->n_tpl, ctx->tid.p, ctx->root.p, ctx->d_tpl, cp, ctx->lod,
                                      ctx->instance_cull, ctx->V.p, ctx->Cloc.p, ctx->vis.p, ctx->groups.p,
                                      ctx->d_meta, ctx->cull.p, st);
        CS_CUDA(cudaGetLastError());
        CS_CUDA(cudaMemcpyAsync(ctx->h_meta, ctx->d_meta, kMetaWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CS_CUDA(cudaMemcpyAsync(ctx->h_groups, ctx->groups.p, kMaxGroups * sizeof(Group), cudaMemcpyDeviceToHost, st));
        CS_CUDA(cudaStreamSynchronize(st));
        visible = ctx->h_meta[kMetaVisible];
        n_groups = ctx->h_meta[kMetaGroups];
        set_depth_key_range(cp, ctx->h_meta);
        S = ctx->h_meta[kMetaSplats];
        cp.n_splats = (uint32_t)S;
        proj_blocks = ctx->h_meta[kMetaBlocks];
        for (int l = 0; l < kMaxLevels; ++l) per_level[l] = ctx->h_meta[kMetaLevel0 + l];
    }
    if ((size_t)S > kStaticSplats)
        return fail(ctx, CS_ERR_CAPACITY, "cs_render_static: %lld splats exceed the static limit of %zu",
                    (long long)S, kStaticSplats);
    const TemplateArrays ta = template_arrays(ctx);
    if (S > 0)
        launched += launch_project(proj_blocks, ctx->groups.p, ctx->h_groups, n_groups, ctx->tpl_host.data(),
                                   ctx->vis.p, ctx->B.p, ctx->V.p, ctx->root.p, ta, ctx->d_tpl, cp, ctx->lod,
                                   ctx->skin_mode, ctx->sh_frame, rec, key, bins, st);
    if (radix_scratch_words((size_t)std::max<int64_t>(S, 1)) > kStaticScratchWords ||
        scan_scratch_words((size_t)S + 1) > kStaticScratchWords)
        return fail(ctx, CS_ERR_CAPACITY, "cs_render_static: scratch too small for %lld splats", (long long)S);
    int ob = 0;
    if (S > 0) launched += radix_sort_u32(key, ids, key2, ids2, (uint32_t)S, depth_key_bits(cp.key_lo, cp.key_hi),
                                          scratch, st, &ob, bins, bins_sorted, true);
    uint32_t *order = ob ? ids2 : ids;
    uint32_t *sorted_keys = ob ? key2 : key;
    launched += exclusive_scan_bins(bins_sorted, pair_off, (uint32_t)S, scratch, st);
    if (stats && S > 0) launched += launch_count_live((uint32_t)S, sorted_keys, ctx->d_meta + kMetaWords - 1, st);
    CS_CUDA(cudaGetLastError());
    CS_CUDA(cudaMemcpyAsync(ctx->h_pairs, pair_off + S, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (stats) CS_CUDA(cudaMemcpyAsync(ctx->h_pairs + 1, ctx->d_meta + kMetaWords - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CS_CUDA(cudaStreamSynchronize(st));
    const int64_t P = ctx->h_pairs[0];
    if ((size_t)P > kStaticPairs)
        return fail(ctx, CS_ERR_CAPACITY, "cs_render_static: %lld pairs exceed the static limit of %zu",
                    (long long)P, kStaticPairs);
    if (radix_scratch_words((size_t)std::max<int64_t>(P, 1)) > kStaticScratchWords)
        return fail(ctx, CS_ERR_CAPACITY, "cs_render_static: scratch too small for %lld pairs", (long long)P);
    if (P > 0)
        launched += launch_emit_pairs((uint32_t)S, order, bins_sorted, pair_off, rec, cp.tiles_x, (uint32_t)T, ptile0,
                                      pval0, st);
    int pb = 0;
    if (P > 0) launched += radix_sort_u16(ptile0, pval0, ptile1, pval1, (uint32_t)P, bits_for((uint32_t)T),
                                          scratch, st, &pb);
    uint16_t *ptile = pb ? ptile1 : ptile0;
    uint32_t *pval = pb ? pval1 : pval0;
    // the array keeps the previous call's ranges: clear them
    CS_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * T, st));
    launched += launch_tile_ranges((uint32_t)P, ptile, ranges, (uint32_t)T, st);
    BlendWork bw{reinterpret_cast<int32_t *>(base + kOffBwSlot), reinterpret_cast<int32_t *>(base + kOffBwTile),
                 reinterpret_cast<uint32_t *>(base + kOffBwChunk0), reinterpret_cast<uint32_t *>(base + kOffBwDone),
                 reinterpret_cast<float4 *>(base + kOffBwState), reinterpret_cast<float4 *>(base + kOffBwPart),
                 reinterpret_cast<int32_t *>(base + kOffBwMeta), reinterpret_cast<int32_t *>(base + kOffBwStop)};
    bw.pp_tile = reinterpret_cast<int32_t *>(base + kOffBwPp);
    bw.chunk_slot = reinterpret_cast<int32_t *>(base + kOffBwCslot);
    bw.ox = cp.ox;
    bw.oy = cp.oy;
    bw.items = ctx->blend_items;
    bw.n_pairs = (uint32_t)P;
    bw.max_slots = (uint32_t)blend_max_slots((size_t)T, (size_t)P);
    bw.max_chunks = (uint32_t)blend_max_chunks((size_t)T, (size_t)P);
    launched += launch_blend(cp.tiles_x, cp.tiles_y, cam->width, cam->height, ranges, pval, rec, out, bw,
                             (uint32_t)P, st);
    CS_CUDA(cudaGetLastError());
    if (stats) {
        stats->instances = I;
        stats->instances_visible = visible;
        for (int l = 0; l < CS_MAX_LEVELS; ++l) stats->instances_per_level[l] = per_level[l];
        stats->splats = S;
        stats->splats_live = S > 0 ? (int64_t)ctx->h_pairs[1] : 0;
        stats->pairs = P;
        stats->tiles_x = cp.tiles_x;
        stats->tiles_y = cp.tiles_y;
        stats->kernel_launches = launched;
        stats->depth_key_bits = S > 0 ? depth_key_bits(cp.key_lo, cp.key_hi) : 0;
    }
    return CS_OK;
}

}  // extern "C"
