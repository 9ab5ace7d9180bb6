/*
 * sr_net.h - C-ABI of the learned warm start for the self-repelling snake.
 *
 * The paper starts Alg. 1 from a thresholded or hand-placed level set
 * (Sec. 5).  This part proposes phi0 instead with a small convolutional
 * encoder-decoder, trained on (image, converged phi) pairs that the plain
 * Split Bregman solver of sr.h produces; the plain iteration then finishes
 * the solve from that phi0.  There is no paper equation for the network; its
 * definition is the one below.
 *
 * Network (6 layers, 3x3 zero-padded cross-correlations, bias, ReLU after
 * every layer but the last; H and W multiples of 4):
 *     f (1 ch)  -> conv 1->32,   ReLU -> 2x2 average pool
 *               -> conv 32->64,  ReLU -> 2x2 average pool
 *               -> conv 64->128, ReLU
 *               -> conv 128->64, ReLU -> 2x nearest upsample
 *               -> conv 64->32,  ReLU -> 2x nearest upsample
 *               -> conv 32->1 = y,    phi0 = c * y.
 * Training loss: 1/(2n) sum (y - clip(phi*, -c, c) / c)^2 over the n pixels
 * of the batch, c = phi_clip.  Optimiser: Adam with bias correction
 * (beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Precision.  Activations and their gradients are bfloat16 in NHWC layout.
 * Layers 1-5 run on the tensor cores with bf16 operands (weights rounded to
 * bf16) and fp32 accumulation; the one-channel output layer runs in fp32 on
 * the float weights.  Parameters, their gradients, the Adam moments, the
 * output y, dL/dy and the loss (fp64) are kept in higher precision.
 *
 * Parameters.  One flat float32 vector of sr_net_param_count() entries:
 * layer after layer, W in (Cout, 3, 3, Cin) order followed by the Cout
 * biases.  The caller draws the initial values and passes them in.
 *
 * Pointers are device pointers on the device current at sr_net_create,
 * unless a function says "host".  Image batches are B planes of H x W
 * float32, row-major and packed (plane k starts at k * H * W).  The caller
 * owns every buffer it passes; no call keeps a pointer after it returns.
 * All work is enqueued on the stream given to sr_net_create; calls return
 * once it is enqueued.  Every call returns an sr_status and none exits,
 * aborts or traps the device.
 */
#ifndef SR_NET_H
#define SR_NET_H

#include <stdint.h>

#include "sr.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SR_NET_LAYERS 6

/* (Cin, Cout) of layer k in [0, SR_NET_LAYERS). */
sr_status sr_net_layer_shape(int k, int* cin, int* cout);
/* Number of float32 parameters (185217). */
long long sr_net_param_count(void);

typedef struct sr_net sr_net;

/* Allocate the network's workspace for batches of up to max_batch images of
 * H x W (H, W multiples of 4 in [8, 4096]; phi_clip > 0).  Parameters start
 * at zero: call sr_net_set_params before use. */
sr_status sr_net_create(int H, int W, int max_batch, float phi_clip, void* cuda_stream,
                        sr_net** out);
void sr_net_destroy(sr_net* net);
const char* sr_net_last_error(const sr_net* net);

/* Copy sr_net_param_count() floats in (device pointer); resets the Adam
 * moments and step count. */
sr_status sr_net_set_params(sr_net* net, const float* theta);
/* Copy the parameters, or the gradient of the last sr_net_gradients or
 * sr_net_train_step call, out (device pointers). */
sr_status sr_net_get_params(sr_net* net, float* theta);
sr_status sr_net_get_grads(sr_net* net, float* grad);

/* phi0 = c * y for B <= max_batch images f (device planes). */
sr_status sr_net_forward(sr_net* net, const float* f, int B, float* phi0);
/* Forward and backward pass on (f, phi_star); leaves the gradient in the
 * network.  loss (device, one double) receives the loss unless NULL. */
sr_status sr_net_gradients(sr_net* net, const float* f, const float* phi_star, int B,
                           double* loss);
/* sr_net_gradients followed by one Adam step with learning rate lr. */
sr_status sr_net_train_step(sr_net* net, const float* f, const float* phi_star, int B, float lr,
                            double* loss);
/* Kernel launches the network has enqueued (reset to zero when reset != 0). */
long long sr_net_kernel_launches(sr_net* net, int reset);

/* ---------------------------------------------------------------------------
 * Layer-level entry points (the kernels the network runs), for tests.
 * bf16 tensors are passed as their uint16 bit patterns, NHWC, packed.
 * ------------------------------------------------------------------------- */
#define SR_CONV_RELU 0   /* y (bf16) = max(conv(x, w) + bias, 0)             */
#define SR_CONV_PLAIN 1  /* y (bf16) = conv(x, w) (+ bias when bias != NULL)  */
#define SR_CONV_MASK 2   /* y (bf16) = conv(x, w) where ref > 0, else 0       */
#define SR_CONV_OUT1 3   /* y (float32 plane) = out_scale * (conv + bias), output channel 0 */

/* 3x3 zero-padded cross-correlation of x [B, H, W, cin] with w [cout, 3, 3,
 * cin]: y[b,i,j,o] = sum_{ky,kx,c} x[b,i+ky-1,j+kx-1,c] w[o,ky,kx,c].
 * cin a multiple of 16, cout 16, 32 or a multiple of 64.  ref [B, H, W,
 * cout] for SR_CONV_MASK.  y is bf16 [B, H, W, cout], or a float32 plane
 * [B, H, W] for SR_CONV_OUT1. */
sr_status sr_conv3x3(const uint16_t* x, int B, int H, int W, int cin, const uint16_t* w,
                     const float* bias, int cout, int mode, const uint16_t* ref, void* y,
                     float out_scale, void* cuda_stream);
/* Input gradient of that convolution: dx = conv^T(dy) [B, H, W, cin] (bf16),
 * with w in the forward layout; SR_CONV_PLAIN or SR_CONV_MASK (ref [B, H,
 * W, cin]).  cout a multiple of 16, cin 16, 32 or a multiple of 64. */
sr_status sr_conv3x3_dgrad(const uint16_t* dy, int B, int H, int W, int cout, const uint16_t* w,
                           int cin, int mode, const uint16_t* ref, uint16_t* dx,
                           void* cuda_stream);
/* Weight and bias gradients, ADDED into dw [cout_real, 3, 3, cin_real] and
 * db [cout_real] (float32; db may be NULL): dw[o,ky,kx,c] += sum_{b,i,j}
 * dy[b,i,j,o] x[b,i+ky-1,j+kx-1,c] over o < cout_real, c < cin_real, with
 * dy [B, H, W, cout] and x [B, H, W, cin] bf16 (cin and cout each 16, 32 or a
 * multiple of 64). */
sr_status sr_conv3x3_wgrad(const uint16_t* dy, const uint16_t* x, int B, int H, int W, int cin,
                           int cout, int cin_real, int cout_real, float* dw, float* db,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SR_NET_H */
