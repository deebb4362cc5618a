/*
 * crowdsplat.h -- C ABI of the GB300 (sm_103a) CrowdSplat crowd-synthesis
 * library (libcrowdsplat.so).
 *
 * The library renders crowds of animated 3D-Gaussian avatars as CrowdSplat
 * (arXiv 2501.17792) describes them: a few avatar templates whose Gaussian
 * attributes are shared by every duplicated character (Sec. 1, third
 * contribution; Sec. 2: only the posed means differ between characters of
 * one template), each character animated by linear blend skinning (Fig. 2,
 * Sec. 2), a distance-based level of detail (Sec. 2: fewer Gaussians farther
 * from the camera), and the 3D Gaussian Splatting rasteriser the paper
 * renders with (Sec. 1 and Sec. 2 cite Kerbl et al. 2023): EWA projection
 * with spherical-harmonic colour, 16x16 tile binning, a (tile, depth) sort,
 * front-to-back alpha compositing.
 *
 * Conventions
 *   - Metres, right-handed.  Camera space is OpenCV-style: x right, y down,
 *     z forward.  Pixel (i, j) has its centre at (i + 0.5, j + 0.5).
 *   - Matrices are row-major float32.
 *   - Every function returns CS_OK (0) or a CS_ERR_* code; the text of the
 *     last error of a context is cs_last_error().  No C++ exception crosses
 *     this boundary.  A context is not thread-safe: calls on one context
 *     must not overlap.
 *   - All GPU work is ordered on the context's stream (cs_create_params.stream).
 *     cs_render returns when its work is enqueued, except for the two short
 *     host reads of the frame's splat and pair counts that size its launches.
 *   - Ownership: the library deep-copies every input before returning, so
 *     the caller may free or reuse its buffers; outputs are caller-owned.
 */
#ifndef CROWDSPLAT_H
#define CROWDSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CS_OK 0
#define CS_ERR_ARG 1      /* invalid argument (the message names it)           */
#define CS_ERR_CUDA 2     /* a CUDA runtime call failed                        */
#define CS_ERR_OOM 3      /* device or host allocation failed                  */
#define CS_ERR_CAPACITY 4 /* a size exceeds a documented maximum               */
#define CS_ERR_TIMEOUT 5  /* a bounded device wait gave up                     */
#define CS_ERR_STATE 6    /* call out of order (e.g. render before upload)     */

/* limits */
#define CS_MAX_TEMPLATES 63
#define CS_MAX_LEVELS 4
#define CS_MAX_INSTANCES 131072
#define CS_MAX_IMAGE_SIDE 4096
#define CS_NUM_JOINTS 24
#define CS_TILE 16

/* skinning modes */
#define CS_SKIN_FULL 0       /* LBS moves means and rotates covariances      */
#define CS_SKIN_MEANS_ONLY 1 /* LBS moves means; covariances follow the root */

/* frame of the SH viewing direction */
#define CS_SH_ROOT_FRAME 0  /* direction expressed in the instance's root frame */
#define CS_SH_WORLD_FRAME 1 /* direction in world coordinates                   */

/* template storage precision (the precision variant of the path) */
#define CS_STORE_FP32 0 /* FP32 attributes: 252 B per Gaussian at SH degree 3        */
#define CS_STORE_BF16 1 /* BF16 mean (as an offset from one of its skinning joints),
                           opacity, covariance and skinning weights, FP16 SH
                           coefficients: 128 B per Gaussian at SH degree 3; the
                           skinning blend runs as a split-BF16 tensor-core product
                           with FP32 accumulation, renormalised by the sum of the
                           rounded weights; projection and compositing stay FP32 */

typedef struct cs_ctx cs_ctx; /* opaque, library-owned */

typedef struct {
    int32_t device;        /* CUDA device ordinal                                      */
    void *stream;          /* cudaStream_t all work is ordered on; NULL = legacy default */
    int32_t skin_mode;     /* CS_SKIN_FULL or CS_SKIN_MEANS_ONLY                       */
    int32_t sh_frame;      /* CS_SH_ROOT_FRAME or CS_SH_WORLD_FRAME                    */
    int32_t instance_cull; /* 1: drop instances whose every splat misses the image
                              (conservative bound; never changes the image); 0: off */
    int32_t stage_timing;  /* 1: record CUDA events per stage (cs_get_stage_times)     */
    int32_t template_storage; /* CS_STORE_FP32 or CS_STORE_BF16 (applies to uploads)  */
} cs_create_params;

/* One avatar template, all pointers HOST memory, read during the call.
 * means[n*3] metres (template local frame); scales[n*3] metres (> 0);
 * quats[n*4] (w,x,y,z), normalised by the library; opacity[n] in [0,1];
 * sh[n*K*3] with K = (sh_degree+1)^2, coefficient-major per Gaussian
 * (sh[(g*K + k)*3 + channel]); skin_idx[n*4] joint ids < 24; skin_w[n*4]
 * non-negative, summing to 1 (+-1e-3); rest_joints[24*3] T-pose joint
 * positions; parents[24] with parents[0] = -1 and parents[j] < j.
 * The stored order defines the levels of detail: level l keeps the first
 * N_l = round(fraction_l * n) Gaussians. */
typedef struct {
    int32_t n_gauss;
    int32_t sh_degree; /* 0..3 */
    const float *means;
    const float *scales;
    const float *quats;
    const float *opacity;
    const float *sh;
    const uint8_t *skin_idx;
    const float *skin_w;
    const float *rest_joints;
    const int32_t *parents;
} cs_template_desc;

/* Pinhole camera: x_cam = R x_world + t; u = fx x/z + cx, v = fy y/z + cy.
 * Splats with view depth z <= near_z are culled.
 * Window: the output holds pixels [win_x0, win_x0 + width) x [win_y0,
 * win_y0 + height) of a full image of full_width x full_height pixels
 * (full_width = full_height = 0: no window, the full image is width x
 * height and win_x0 = win_y0 = 0).  fx, fy, cx, cy are the full image's;
 * the EWA clamp follows the full image's field of view and pixel centres
 * stay at their full-image positions, so a window renders bit for bit the
 * same pixels as the full frame.  The window's edges must lie on the full
 * image's tile grid (multiples of CS_TILE) or on the full image's right and
 * bottom edges, so every tile it holds has the full frame's list, and the
 * window must lie inside the full image (CS_ERR_ARG otherwise).  Splitting a frame into row windows this way lets ranks
 * render disjoint parts of one frame. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;
    int32_t win_x0, win_y0;
    int32_t full_width, full_height;
} cs_camera;

typedef struct {
    int32_t instances;              /* instances set                                  */
    int32_t instances_visible;      /* after the instance cull                        */
    int32_t instances_per_level[CS_MAX_LEVELS];
    int64_t splats;                 /* Gaussian-instances projected                   */
    int64_t splats_live;            /* survived the per-splat culls (0 unless stats
                                       were requested: costs one extra reduction)    */
    int64_t pairs;                  /* (tile, splat) pairs sorted and blended         */
    int32_t tiles_x, tiles_y;
    int32_t kernel_launches;        /* CUDA kernels this frame launched               */
    int32_t depth_key_bits;         /* bits of the depth keys the depth sort ranked   */
} cs_frame_stats;

typedef struct {
    int64_t template_bytes;   /* shared template attributes (persistent)        */
    int64_t instance_bytes;   /* per-instance state and FK output (persistent)  */
    int64_t frame_bytes;      /* per-frame splat, sort and pair buffers         */
    int64_t total_bytes;
} cs_memory_stats_t;

/* Create a context on p->device.  *out receives the handle (NULL on failure).
 * Errors: CS_ERR_ARG (bad mode or device), CS_ERR_CUDA. */
int cs_create(cs_ctx **out, const cs_create_params *p);

/* Destroy a context and free its device memory (synchronises its stream).
 * NULL is accepted. */
void cs_destroy(cs_ctx *ctx);

/* Upload the shared avatar templates (CrowdSplat Sec. 2: attributes other
 * than the posed means are reused by every character of a template).
 * Replaces any previous templates; resets the LoD to one full-detail level.
 * Errors: CS_ERR_ARG (a field out of range: n_gauss < 1, sh_degree > 3,
 * joint id > 23, negative weight, bad parents), CS_ERR_CAPACITY (more than
 * CS_MAX_TEMPLATES), CS_ERR_OOM, CS_ERR_CUDA. */
int cs_upload_templates(cs_ctx *ctx, int32_t n_templates, const cs_template_desc *templates);

/* Distance level of detail (CrowdSplat Sec. 2).  Host arrays:
 * dist_thresh[n_levels-1] ascending metres (an instance whose root is at
 * distance d from the camera centre takes level = number of thresholds <= d);
 * fraction[n_levels] in (0,1] (level l renders the first round(f_l * n)
 * Gaussians of its template); scale_mult[n_levels] > 0 (level l multiplies
 * every Gaussian scale by it).  Errors: CS_ERR_ARG, CS_ERR_STATE (no
 * templates). */
int cs_set_lod(cs_ctx *ctx, int32_t n_levels, const float *dist_thresh, const float *fraction,
               const float *scale_mult);

/* Choose the Gaussians that LoD level `level` of template `template_id`
 * renders (CrowdSplat Sec. 2 varies the number of Gaussians per distance
 * band; the paper fits a separate template per band, this call lets a
 * ranking pick the band's Gaussians from the full template instead).
 * idx[n]: HOST array of distinct template-local Gaussian indices, any
 * order (the order is the splat order inside the level and so breaks depth
 * ties).  The subset replaces the level's prefix of round(fraction * N)
 * Gaussians; the level's scale multiplier still applies.  n = 0 clears the
 * subset (back to the prefix).  Subsets are kept across cs_set_lod and
 * cleared by cs_upload_templates.  Errors: CS_ERR_ARG (template or level
 * out of range, n > N, an index >= N or repeated), CS_ERR_STATE (no
 * templates), CS_ERR_CUDA, CS_ERR_OOM. */
int cs_set_lod_subset(cs_ctx *ctx, int32_t template_id, int32_t level, int32_t n, const uint32_t *idx);

/* Per-frame instance state (CrowdSplat Sec. 2, stage 2: duplicated
 * characters, each with its template and pose).  template_id[n];
 * root[n*12] row-major 3x4 rigid [R|t] from template-local to world
 * coordinates; joint_pose[n*24*3] axis-angle radians per joint.
 * on_device = 0: host pointers (copied host->device on the stream, the call
 * returns once the copy is staged); 1: device pointers (device->device copy).
 * Roots must be rigid (the instance cull assumes unit scale).
 * Errors: CS_ERR_ARG (n < 0, template id out of range when host pointers),
 * CS_ERR_CAPACITY (n > CS_MAX_INSTANCES), CS_ERR_STATE, CS_ERR_OOM, CS_ERR_CUDA. */
int cs_set_instances(cs_ctx *ctx, int32_t n, const int32_t *template_id, const float *root,
                     const float *joint_pose, int32_t on_device);

/* Render one frame of the current instances (the whole hot path: forward
 * kinematics, LoD + cull, LBS + EWA projection + SH colour, tile binning,
 * (tile, depth) sort, compositing).  rgba_out: caller-owned DEVICE buffer of
 * height*width*4 float32, row-major, premultiplied RGB on a black background
 * and alpha = 1 - final transmittance.  stats may be NULL.
 * Errors: CS_ERR_ARG (image side < 1 or > CS_MAX_IMAGE_SIDE, non-positive
 * focal length or near plane, NULL or not 16-byte aligned output), CS_ERR_STATE (no templates or
 * instances), CS_ERR_OOM, CS_ERR_CUDA. */
int cs_render(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats);

/* cs_render that also measures how much each template Gaussian contributes
 * to the image: contrib_out[g] (DEVICE float32 array of the total Gaussian
 * count over all templates, template t's Gaussians at its upload offset) is
 * ADDED the sum, over every pixel and every instance that rendered g, of g's
 * compositing weight alpha * T (T = transmittance in front of it).  Summed
 * over all Gaussians this equals the sum of the frame's alpha channel.
 * Tile lists are composited in one pass (no split of long lists), so the
 * frame is slower than cs_render's; the image is the same up to float
 * rounding order.  Used to build ranked LoD subsets (cs_set_lod_subset);
 * the paper has no counterpart.  Same arguments and errors as cs_render,
 * plus CS_ERR_ARG for a NULL or misaligned contrib_out. */
int cs_render_contrib(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, float *contrib_out,
                      cs_frame_stats *stats);

/* cs_render with the image delivered to rgba_host (HOST memory, H*W*4
 * floats, layout as cs_render's output); returns once the image is there.
 * When rgba_host is page-locked host memory mapped into the device's
 * address space (cudaHostAlloc / cudaHostRegister, e.g. a pinned torch
 * tensor) and 16-byte aligned, the compositing kernels write the image
 * straight into it; otherwise the frame is rendered into an internal device
 * buffer followed by one device->host copy.  Same errors as cs_render. */
int cs_render_to_host(cs_ctx *ctx, const cs_camera *cam, float *rgba_host, cs_frame_stats *stats);

/* cs_render without any device allocation, for callers that may not
 * allocate device memory while a frame is produced: real-time render
 * threads where cudaMalloc's implicit synchronisation and latency are not
 * allowed, and engines that hand the library a fixed memory budget up
 * front.  CrowdSplat has no counterpart of this call; it renders exactly
 * what cs_render renders, with the per-frame scratch (splat records, sort
 * buffers, pair lists, tile ranges) taken from one static device array of
 * about 9.9 MB that every GPU loading the library holds until the process
 * exits.  Limits per frame: 65,536 splats, 262,144 (tile, splat) pairs,
 * 16,384 tiles (e.g. 2048 x 2048); larger frames fail with CS_ERR_CAPACITY
 * and a message naming the limit, leaving rgba_out unwritten.  The
 * instance buffers come from cs_set_instances, which allocates as usual.
 * The first call on a device looks the array's device address up (CUDA may
 * load the library's device code then) and keeps it for the process: make
 * that first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library is loaded, since the kept address
 * would then be stale.  All contexts of the process share the array and it
 * keeps the previous call's contents, so calls that overlap on the GPU
 * (other streams, other contexts on the same device) race; serialise them.
 * No stage times are recorded, and cs_debug_read is unspecified after this
 * call until the next cs_render.  Arguments and other errors as cs_render. */
int cs_render_static(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats);

/* Per-stage milliseconds (needs stage_timing = 1), measured with CUDA events
 * on the context's stream: ms[0..n) = fk, cull+lod (with the host read of
 * the frame's splat count), skin+project, depth sort, pair emit (with the
 * host read of the pair count), tile sort, tile ranges, blend.  average = 0:
 * the last
 * frame (waits for it); average = 1: the mean over every frame rendered
 * since the previous average call (waits for the last one), then restarts
 * the mean.  *frames_out (may be NULL) receives the number of frames
 * covered.  Returns the number of stages written, or -CS_ERR_* on error
 * (-CS_ERR_STATE when no timed frame exists). */
int cs_get_stage_times(cs_ctx *ctx, float *ms, int32_t n, int32_t average, int64_t *frames_out);

/* Device memory held by the context (CrowdSplat Table 1 accounting). */
int cs_memory_stats(cs_ctx *ctx, cs_memory_stats_t *out);

/* Text of the last error on this context ("" if none); valid until the
 * next call on the context. */
const char *cs_last_error(const cs_ctx *ctx);

/* Copy an internal buffer of the last frame to HOST memory (testing and
 * diagnosis).  which = CS_DBG_*; copies min(bytes, size) bytes and stores
 * the buffer's full size in *size_out (may be NULL).  Synchronises. */
#define CS_DBG_SKIN_B 1      /* float [I][24][12]: skinning transforms, instance-local */
#define CS_DBG_VISIBLE 2     /* int32 [V]: visible instance ids in group order         */
#define CS_DBG_GROUPS 3      /* int32 [G][7]: template, level, first slot, slots,
                                gaussians per slot, first splat, first projection CTA  */
#define CS_DBG_RECORDS 4     /* float [S][16]: u, v, conic A, B, C, opacity, radius,
                                depth, r, g, b, 0, reach x, reach y (pixel ranges lo | hi
                                << 16 as float bits), fcut, log2 opacity: the 48-byte
                                splat records expanded for this view (opacity from
                                its logarithm, depth from the depth key); culled
                                splats read as zeros                               */
#define CS_DBG_DEPTH_KEYS 5  /* uint32 [S]: depth keys in depth order: float bits of the
                                depth minus those of the frame's lower depth bound
                                (from the instance cull), 0xFFFFFFFF = culled      */
#define CS_DBG_RECTS 6       /* uint16 [S][4]: tile rect x0, y0, x1, y1 (inclusive)    */
#define CS_DBG_DEPTH_ORDER 7 /* uint32 [S]: splat ids sorted by (depth key, id)        */
#define CS_DBG_PAIR_TILES 8  /* uint16 [P]: tile of each pair, (tile, depth, splat id)
                                order                                              */
#define CS_DBG_PAIR_SPLATS 9 /* uint32 [P]: splat of each pair, same order          */
#define CS_DBG_TILE_RANGES 10 /* uint32 [T][2]: [start, end) of each tile's pairs      */
int cs_debug_read(cs_ctx *ctx, int32_t which, void *host_dst, size_t bytes, size_t *size_out);

/* Testing hook for the out-of-memory paths: after `after` more successful
 * allocations of frame or instance buffers, every such allocation of the
 * context fails with CS_ERR_OOM, exactly as a failed cudaMalloc would (the
 * buffer being grown is released first), until the hook is called again
 * with after < 0 (off, the default).  The failure is made on the host; no
 * GPU call fails.  The context stays usable: once the hook is off, the next
 * call allocates again.  The paper has no counterpart.  Returns CS_OK, or
 * CS_ERR_ARG for a NULL context. */
int cs_debug_fail_allocs(cs_ctx *ctx, int32_t after);

/* Testing hook for the compositing schedule of plain frames: mode
 * CS_BLEND_ITEMS_AUTO (the default) composites every short tile list (under
 * 8,192 pairs) as one work item of its own when the frame has many busy
 * tiles (at least 8 per resident compositing CTA) and block by block
 * otherwise; CS_BLEND_ITEMS_TILES and CS_BLEND_ITEMS_BLOCKS force one or the
 * other for every frame of the context, so that small test frames exercise
 * both.  The image is the same up to rounding order (both composite every
 * pixel's pairs in depth order with the same stop rule).  The paper has no
 * counterpart.  Returns CS_OK, or CS_ERR_ARG for a NULL context or an
 * unknown mode. */
/* Bounds checks of the debug build (compiled with CS_CHECKS=1, the library
 * libcrowdsplat_checks.so that build.build(checks=True) makes; the release
 * library compiles them away): a kernel index outside its buffer (splat
 * record, pair, tile, sort position, compositing slot) sets one bit of a
 * device check word and the access is skipped.  Waits for the context's
 * stream, then stores the word accumulated since the last call in *failed
 * (0: every check passed; bits 1 record, 2 pair, 4 tile, 8 splat id,
 * 16 sort, 32 slot) and clears it, and stores in *enabled whether this
 * library was built with the checks (0 and *failed = 0 otherwise).  The
 * word is per process and device, shared by every context.  The paper has
 * no counterpart.  Returns CS_OK, CS_ERR_ARG for a NULL argument, or
 * CS_ERR_CUDA. */
int cs_debug_checks(cs_ctx *ctx, uint32_t *failed, int32_t *enabled);

#define CS_BLEND_ITEMS_AUTO 0
#define CS_BLEND_ITEMS_TILES 1
#define CS_BLEND_ITEMS_BLOCKS 2
int cs_debug_blend_items(cs_ctx *ctx, int32_t mode);

/* Library version string. */
const char *cs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CROWDSPLAT_H */
