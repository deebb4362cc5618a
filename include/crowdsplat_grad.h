/*
 * crowdsplat_grad.h -- gradients of a rendered frame (the differentiable
 * variant of the CrowdSplat crowd-synthesis path).
 *
 * CrowdSplat (Sec. 2) fits its avatar templates in stage 1 with the 3DGS
 * training loop, whose gradients run back through compositing, projection
 * and skinning; the crowd stage itself only renders.  These calls give the
 * gradients of a loss on one rendered crowd frame with respect to the shared
 * template attributes and every instance's joint poses, so that templates
 * or poses can be optimised against images rendered by this library.
 *
 * cs_render_train renders like cs_render and keeps what the backward needs;
 * cs_backward takes dL/d(image) and adds the gradients into caller-owned
 * DEVICE buffers.  What is differentiated: front-to-back alpha compositing,
 * alpha = min(0.99, o exp(q)), EWA projection with the Jacobian at the mean
 * (x/z, y/z clamped), SH colour clamped at 0, linear blend skinning of means
 * and covariances, forward kinematics of the axis-angle joint poses, and the
 * covariance R(q) diag(s^2) R(q)^T with the LoD scale multiplier.  Clamps
 * pass no gradient where they are active; the discrete choices of the
 * forward (support box, alpha >= 1/255, the stop rule, the radius, the
 * frustum and LoD culls) are held fixed.  FP32 throughout; FP32 template
 * storage only.
 */
#ifndef CROWDSPLAT_GRAD_H
#define CROWDSPLAT_GRAD_H

#include <stddef.h>
#include <stdint.h>

#include "crowdsplat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Gradient destinations, all DEVICE float32, ADDED to (zero them first for a
 * plain gradient).  n_total = Gaussians over all templates in upload order;
 * n_inst = instances of the last cs_set_instances.  NULL: that gradient is
 * not written. */
typedef struct {
    float *means;   /* [n_total][3] template-local means                     */
    float *scales;  /* [n_total][3]                                          */
    float *quats;   /* [n_total][4] (w, x, y, z) as uploaded (unnormalised)   */
    float *opacity; /* [n_total]                                             */
    float *sh;      /* [n_total][48]: coefficient k, channel c at 3k + c     */
    float *pose;    /* [n_inst][24][3] axis-angle joint rotations            */
} cs_grads;

/* cs_render that also keeps, per pixel, where its list of composited splats
 * ends, its final colour and transmittance, and its state at every 1,024th
 * pair of its tile's list, so that cs_backward can walk each 1,024-pair
 * chunk of a list in parallel (every list is composited in such chunks,
 * merged per pixel in order, so the frame is slower than cs_render's; the
 * image is the same up to float rounding order).  The state stays valid until the next render or any
 * change of templates, LoD, subsets or instances.  Same arguments and
 * errors as cs_render; CS_ERR_STATE with BF16 template storage. */
int cs_render_train(cs_ctx *ctx, const cs_camera *cam, float *rgba_out, cs_frame_stats *stats);

/* Gradients of a loss L on the last cs_render_train frame.  dl_drgba: DEVICE
 * float32 [height][width][4], dL/d(R, G, B, A) per pixel, 16-byte aligned.
 * Runs on the context's stream (returns when enqueued).  Errors: CS_ERR_ARG
 * (NULL or misaligned), CS_ERR_STATE (no valid training frame, or BF16
 * storage), CS_ERR_OOM, CS_ERR_CUDA. */
int cs_backward(cs_ctx *ctx, const float *dl_drgba, const cs_grads *grads);

#ifdef __cplusplus
}
#endif
#endif /* CROWDSPLAT_GRAD_H */
