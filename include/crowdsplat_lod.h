/*
 * crowdsplat_lod.h -- ranked level of detail for libcrowdsplat.
 *
 * CrowdSplat (Sec. 2, Fig. 3) renders distant characters with fewer
 * Gaussians: one separately reconstructed template per distance band.
 * This part of the library ranks the Gaussians of each uploaded template
 * per band instead, so that a band keeps the Gaussians that matter most at
 * its distances.  A small MLP maps per-Gaussian features plus the band to a
 * score; it is trained on how much each Gaussian contributes to rendered
 * images (cs_render_contrib).  The ranking runs once per (template, band),
 * offline; a frame pays nothing beyond the per-level index list of
 * cs_set_lod_subset.  The paper has no counterpart of the ranking: it is a
 * replacement for its per-band template fitting, which needs the training
 * videos.
 *
 * All compute runs in the library's CUDA kernels on the context's (or the
 * MLP's) stream.  Pointers marked DEVICE must be device memory of that
 * context's GPU; the caller owns every buffer it passes.  Functions return
 * CS_OK or a CS_ERR_* code (crowdsplat.h); cs_last_error on the render
 * context, or cs_mlp_last_error, gives the message.
 */
#ifndef CROWDSPLAT_LOD_H
#define CROWDSPLAT_LOD_H

#include <stddef.h>
#include <stdint.h>

#include "crowdsplat.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CS_LOD_FEATURES 32 /* per-Gaussian features                         */
#define CS_MLP_IN 48       /* 32 features, 4-way one-hot band, 12 zero pads */
#define CS_MLP_HIDDEN 64   /* two hidden layers of 64 ReLU units            */
/* FP32 parameter vector, in this order:
 *   W1 [48][64] (row = input, column = first hidden unit), b1 [64],
 *   W2 [64][64] (row = first hidden unit, column = second), b2 [64],
 *   w3 [64], b3 [1]                                        = 7,361 floats */
#define CS_MLP_PARAMS (CS_MLP_IN * 64 + 64 + 64 * 64 + 64 + 64 + 1)

/* Per-Gaussian ranking features of every uploaded template, computed on the
 * GPU from the uploaded attributes (FP64 arithmetic, FP32 output).
 * feat_out: DEVICE float32 [n_total][32], n_total = the total Gaussian count
 * over all templates in upload order.  The features are scale-free forms of
 * the Gaussian's size, shape, opacity, colour, position and skinning:
 *   0-2  ln(sigma_i / 0.01 m), sigma_1 >= sigma_2 >= sigma_3 the standard
 *        deviations along the principal axes (covariance eigenvalues)
 *   3    mean of 0-2;  4  ln(sigma_1 / sigma_3)
 *   5    opacity o;  6  logit(o) / 4 (clamped to +-2)
 *   7    ln(o sigma_1 sigma_2 / 1e-4 m^2) / 4 (projected footprint weight)
 *   8-10 degree-0 colour max(0, 0.2820948 c0 + 0.5) per channel
 *   11   their mean;  12-14 root-mean-square of the degree-1, 2, 3
 *        coefficients / 0.3 (0 where the template's degree is lower)
 *   15-17 template-space mean (m);  18  its distance from the vertical
 *        axis through the root joint (m)
 *   19-22 skinning weights, largest first
 *   23   joint of the largest weight / 23;  24 that joint's depth in the
 *        kinematic tree / the tree's depth
 *   25   distance from the mean to that joint's rest position (m) x 10
 *   26-28 covariance diagonal / trace (x, y, z)
 *   29   ln(trace / 3e-4 m^2);  30  o sigma_1 / 0.01 m
 *   31   max - min of the degree-0 colour channels
 * Errors: CS_ERR_ARG (NULL or misaligned feat_out), CS_ERR_STATE (no
 * templates), CS_ERR_CUDA. */
int cs_lod_features(cs_ctx *ctx, float *feat_out);

/* Regression targets of the ranking MLP from contribution sums
 * (cs_render_contrib): contrib DEVICE float32 [n_bands][n_total] (row b =
 * the sums over views of distance band b), target_out DEVICE float32
 * [n_bands][n_total] = ln(c / m + floor), m the mean of c over the
 * Gaussian's template within that band (sum in double).  floor > 0 keeps
 * Gaussians that never contributed finite.  Errors: CS_ERR_ARG (n_bands
 * outside 1..CS_MAX_LEVELS, floor <= 0, NULL or misaligned arrays),
 * CS_ERR_STATE, CS_ERR_CUDA. */
int cs_lod_targets(cs_ctx *ctx, int32_t n_bands, const float *contrib, float floor_, float *target_out);

/* Rank every template's Gaussians by score, highest first.
 * score: DEVICE float32 [n_total] (finite); order_out: DEVICE uint32
 * [n_total]: for template t, order_out[g_off(t) + k] is the template-local
 * index of its k-th highest score (ties: lower index first), g_off(t) the
 * template's upload offset.  The first n entries of template t's segment
 * are the argument of cs_set_lod_subset for a level of n Gaussians.
 * Synchronises the context's stream.  Errors: CS_ERR_ARG, CS_ERR_STATE,
 * CS_ERR_OOM, CS_ERR_CUDA. */
int cs_lod_rank(cs_ctx *ctx, const float *score, uint32_t *order_out);

/* ---------------------------------------------------------------------
 * The ranking MLP: 48 -> 64 -> 64 -> 1, ReLU, hand-written BF16 tensor-core
 * kernels (mma m16n8k16, FP32 accumulate).  Rounding points (the FP64
 * reference rounds at the same places): inputs, W1, W2, the first hidden
 * activations and the back-propagated pre-activation gradients are BF16;
 * biases, w3, the second hidden layer, the output and all sums are FP32.
 * FP32 master weights, Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected), mean-squared-error loss.
 * --------------------------------------------------------------------- */
typedef struct cs_mlp cs_mlp;

/* New MLP on `device`, launching on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  Weights: W1, W2 uniform(+-sqrt(6 / fan_in))
 * (padding rows 36..47 of W1 zero), w3 uniform(+-sqrt(3 / 64)), biases 0,
 * from a counter-based generator keyed by seed.  Adam state zero. */
int cs_mlp_create(cs_mlp **out, int32_t device, void *stream, uint64_t seed);
void cs_mlp_destroy(cs_mlp *m);
const char *cs_mlp_last_error(const cs_mlp *m);

/* FP32 parameters in the CS_MLP_PARAMS layout above; HOST arrays of
 * CS_MLP_PARAMS floats.  set also zeroes the Adam state and step count. */
int cs_mlp_get_params(cs_mlp *m, float *host_out);
int cs_mlp_set_params(cs_mlp *m, const float *host_in);

/* Scores of n rows: feat DEVICE float32 [n][32] (cs_lod_features layout),
 * band DEVICE int32 [n] in 0..3, score_out DEVICE float32 [n].  n >= 0.
 * Errors: CS_ERR_ARG (NULL, misaligned or n < 0), CS_ERR_CUDA.  Band values
 * outside 0..3 give an all-zero one-hot. */
int cs_mlp_forward(cs_mlp *m, int64_t n, const float *feat, const int32_t *band, float *score_out);

/* One Adam step on the batch (feat, band as above, target DEVICE float32
 * [n]) with loss (1/n) sum (y - target)^2 and learning rate lr > 0.
 * *loss_out (HOST, may be NULL) receives the batch loss before the step
 * (the call then synchronises the stream).  Errors: CS_ERR_ARG (n < 1,
 * lr <= 0, NULL or misaligned arrays), CS_ERR_OOM, CS_ERR_CUDA. */
int cs_mlp_train_step(cs_mlp *m, int64_t n, const float *feat, const int32_t *band, const float *target,
                      float lr, float *loss_out);

/* FP32 gradient of the last cs_mlp_train_step (before the Adam update), in
 * the parameter layout; HOST array of CS_MLP_PARAMS floats.  Errors:
 * CS_ERR_STATE before the first step. */
int cs_mlp_get_grad(cs_mlp *m, float *host_out);

#ifdef __cplusplus
}
#endif
#endif /* CROWDSPLAT_LOD_H */
