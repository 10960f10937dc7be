/*
 * lbm_nn.h - C ABI of the warm-start network: a 4-level convolutional U-Net
 * that maps a channel's solid mask and Reynolds number to its steady
 * (rho, u_x, u_y), trained by the library's own forward and backward
 * kernels, and the call that turns a prediction into an initial state.
 *
 * The paper has no learned part.  The network serves the method as an
 * initial guess only: a warm-started run still converges to the plain
 * method's steady state (Eq. 1-8), and a drift check falls back to the
 * plain (cold) start.  Conventions as in lbm.h: plain pointers, status codes,
 * no aborts; the network object owns its device buffers, the caller owns
 * every buffer it passes.
 *
 * Network (parameter order and shapes are those of the FP64 reference):
 *   inputs  [B][8][H][W] float: channel 0 = solid mask (1 solid, 0 fluid),
 *           channel 1 = Re / 100, channels 2..7 = 0;
 *   level l (0..levels-1) has base * 2^l channels; encoder: two 3x3 convs
 *           with ReLU per level, 2x2 average pooling between levels; decoder:
 *           2x nearest upsampling, concatenation [upsampled, skip], two 3x3
 *           convs with ReLU; head: 1x1 conv to 3 channels, no ReLU;
 *   outputs [B][3][H][W] float: the scaled density deviation and velocity
 *           (lbm_warm_start names the scales);
 *   params  per conv, in the order enc0a, enc0b, ..., enc{L-1}b, dec{L-2}a,
 *           dec{L-2}b, ..., dec0b, head: weights [Cout][Cin][k][k] then
 *           biases [Cout], float.
 * Activations and weights are BF16 in the products, accumulated in FP32;
 * master weights and Adam moments are FP32.  H and W must be multiples of
 * 2^(levels-1) and W * H * B below 2^31.
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_unet lbm_unet;

typedef struct {
    int32_t levels;     /* 2..4 */
    int32_t base;       /* channels of level 0, multiple of 8 (32 for the warm start) */
    int32_t height;     /* H = ny */
    int32_t width;      /* W = nx */
    int32_t max_batch;  /* largest B of any call */
    int32_t device;
    uint64_t seed;      /* He-normal initial weights, zero biases */
    void *stream;       /* cudaStream_t, NULL: the network creates one */
} lbm_unet_config;

lbm_status lbm_unet_create(const lbm_unet_config *cfg, lbm_unet **out);
lbm_status lbm_unet_destroy(lbm_unet *net);
const char *lbm_unet_last_error(const lbm_unet *net);

/* Polls of an mbarrier before a wait of the tensor-core convolutions gives
 * up (default 2^24; 0 gives up at the first wait).  A CTA whose wait gave up
 * issues no further MMA, waits (at most 2^24 polls) for the MMAs it issued,
 * frees its tensor memory and stores nothing; the next call that
 * synchronises (a host-array forward, lbm_unet_gradients,
 * lbm_unet_train_step with a loss) returns LBM_ETIMEOUT once and clears the
 * flag.  The outputs and parameters of the calls since are then undefined:
 * set them again.  LBM_EINVAL for polls < 0. */
lbm_status lbm_unet_set_wait_limit(lbm_unet *net, int64_t polls);

/* Number of floats in the parameter vector, and its FP32 master copy. */
int64_t lbm_unet_param_count(const lbm_unet *net);
lbm_status lbm_unet_get_params(lbm_unet *net, float *params, int32_t on_device);
lbm_status lbm_unet_set_params(lbm_unet *net, const float *params, int32_t on_device);

/* Forward pass of B samples (in, out as above; on_device: both are device
 * pointers, else host).  Waits for the stream when they are host arrays. */
lbm_status lbm_unet_forward(lbm_unet *net, const float *in, float *out, int32_t batch,
                            int32_t on_device);

/* Loss (mean over fluid nodes and the 3 channels of the squared difference
 * between output and target) and its gradient with respect to every
 * parameter, without an update.  target [B][3][H][W], fluid [B][H][W] (1
 * fluid, 0 solid); grads receives lbm_unet_param_count floats in parameter
 * order. */
lbm_status lbm_unet_gradients(lbm_unet *net, const float *in, const float *target,
                              const float *fluid, int32_t batch, float *grads, double *loss,
                              int32_t on_device);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * loss of one mini-batch; *loss (when not NULL) receives the loss before
 * the step. */
lbm_status lbm_unet_train_step(lbm_unet *net, const float *in, const float *target,
                               const float *fluid, int32_t batch, float lr, double *loss,
                               int32_t on_device);

/* Network input of one case from its owner map (lbm_get_owner layout,
 * device int32 [H][W]) and Reynolds number: writes [8][H][W] floats at
 * in_device. */
lbm_status lbm_unet_input(lbm_unet *net, const int32_t *owner_device, double reynolds,
                          float *in_device);

/* Network input of the case held by ctx (the warm start's learned part; the
 * paper has no counterpart), [8][ny][nx] device floats at in_device, from its
 * solid table and Reynolds number: 0 the solid mask, 1 Re / 100,
 * 2 log10(Re) / 2, 3 the signed distance to the nearest disk surface / 16
 * (clipped to [-1, 4]), 4 the axial distance from that disk's centre in its
 * radii / 8 (clipped to [-1, 4], positive downstream), 5 the channel's
 * parabola 4 y'(ny - y') / ny^2 with y' = y + 1/2, 6 x / nx, 7 y' / ny - 1/2.
 * Enqueued on the context's stream.  LBM_EINVAL for Re <= 0. */
lbm_status lbm_case_input(lbm_ctx *ctx, double reynolds, float *in_device);

/* Flags of lbm_warm_start. */
enum { LBM_WS_BASE = 1, LBM_WS_FLUX = 2 };

/* Initial state of ctx from a network output [3][H][W] (device floats):
 * at every fluid node f = f^eq(rho, u) (Eq. 8) with
 *   rho = 1 + rho_scale p0, u = u_scale (p1, p2)                  (flags 0)
 *   rho = rho_P(x) + rho_scale p0, u = (u_P(y), 0) + u_scale (p1, p2)
 *                                                        (LBM_WS_BASE)
 * where (rho_P, u_P) is the empty channel's Poiseuille flow of the context
 * (bc_x = LBM_OPEN): u_P = the inlet parabola, rho_P = rho0 + 24 nu umax
 * (nx - 1 - x) / ny^2 (the pressure drop of that flow, rho0 at the outlet),
 * nu = (tau - 1/2) / 3.  With LBM_WS_BASE | LBM_WS_FLUX, u_x of every
 * column is then scaled so that the column's mass flux sum_y rho u_x over
 * its fluid nodes equals the inlet's, sum over column 0 of rho u_P (a steady
 * flow carries that flux through every column).  The domain must be H x W;
 * solid nodes keep their state.  LBM_EINVAL for other flags, or a base
 * without an open channel. */
lbm_status lbm_warm_start(lbm_ctx *ctx, const float *prediction_device, double u_scale,
                          double rho_scale, int32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NN_H */
