/*
 * unet.h -- C ABI of the learned warm start of the Poisson solve (part of
 * libpic_gb300.so).
 *
 * The solve of Eq. (1) in each PIC step starts from an initial guess; the
 * plain form starts from the previous step's potential. The learned form adds
 * a correction predicted by a small 3-D U-Net from the residual that the
 * previous potential leaves, and the multigrid-preconditioned CG then runs to
 * the configured tolerance exactly as before, so the field accuracy does not
 * depend on the network (it can only change the iteration count). The paper
 * has no network: it solves Eq. (1) by FEM; this is the scope's learned
 * variant of that solve.
 *
 * Network (BF16 weights and activations, FP32 accumulation on the tensor
 * cores): input 2 channels, four levels of 16/32/64/128 channels, two 3x3x3
 * convolutions with ReLU per level, 2x2x2 average pooling down, nearest x2
 * upsampling and channel concatenation [upsampled, skip] up, a 1x1x1
 * convolution to one output channel, zero padding, no biases. Weights are
 * exchanged with the host as one flat FP32 array: for each 3x3x3 convolution
 * in the order e0a e0b e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b d0a d0b the
 * array w[co][ci][a][b][c] (tap (a, b, c) reads the input at offset
 * (a-1, b-1, c-1) in (z, y, x)), then the output weights w[0][ci] (16).
 *
 * Volumes are dense FP32 device arrays [c][D][H][W] (x fastest) with D, H, W
 * multiples of 8; the library keeps its activations in its own layout.
 * Status codes are those of pic.h. All work runs on the stream given to
 * unet_create; calls that return host data synchronise it.
 */
#ifndef PIC_GB300_UNET_H
#define PIC_GB300_UNET_H

#include <stdint.h>

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet_handle unet_handle; /* opaque */

/* Number of FP32 values in the flat weight array (and in the gradient array). */
int64_t unet_num_weights(void);

/* A network for volumes of D x H x W voxels (multiples of 8, D, H, W >= 8).
 * Allocates its weights (FP32 master copy, BF16 operand images, Adam moments)
 * and every activation and gradient buffer of one sample. Weights start at
 * zero. PIC_EINVAL for bad sizes, PIC_ENOMEM, PIC_ECUDA. */
pic_status unet_create(int32_t D, int32_t H, int32_t W, void* cuda_stream, unet_handle** out);
pic_status unet_destroy(unet_handle* net);

/* Copy the weights in (host, n = unet_num_weights() FP32 values, layout
 * above; resets the Adam moments and step) or out. */
pic_status unet_set_weights(unet_handle* net, const float* host_w, int64_t n);
pic_status unet_get_weights(unet_handle* net, float* host_w, int64_t n);

/* Forward pass: x_dev = 2 x D x H x W FP32 (device), y_dev = D x H x W FP32
 * (device, written). */
pic_status unet_forward(unet_handle* net, const float* x_dev, float* y_dev);

/* Backward pass of the last unet_forward for a given output gradient dy_dev
 * (D x H x W FP32, device): the weight gradients replace the gradient array,
 * which unet_get_grads copies out (host, n FP32 values, layout of the
 * weights). */
pic_status unet_backward(unet_handle* net, const float* dy_dev);
pic_status unet_get_grads(unet_handle* net, float* host_g, int64_t n);

/* One training step on one sample: forward on x_dev, loss
 * L = mean over the voxels of planes z < loss_planes of (y - t)^2 with the
 * target t_dev (D x H x W FP32, device), backward, and one Adam update
 * (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) of the FP32 master
 * weights, whose BF16 images the next pass uses. *loss (host, may be NULL)
 * receives L of the forward pass before the update; reading it synchronises. */
pic_status unet_train_step(unet_handle* net, const float* x_dev, const float* t_dev, int32_t loss_planes, float lr,
                           double* loss);

/* Test hooks (synchronous; they allocate scratch device memory for the call):
 * one 3x3x3 convolution of the network, `layer` in 0..13 in the order above,
 * on dense FP32 device volumes at that layer's resolution
 * (D >> l) x (H >> l) x (W >> l), level l = 0 for e0* and d0*, 1 for e1* d1*,
 * 2 for e2* d2*, 3 for e3*. unet_layer_forward: y[cout] = conv(x[cin]) with the
 * layer's BF16 weights (x rounded to BF16 on entry), ReLU if relu != 0.
 * unet_layer_backward: for output gradient dz[cout], writes dx[cin] (data
 * gradient, unmasked; may be NULL) and the layer's weight gradient to dw_host
 * (host, 27 cin cout FP32 values in the layout w[co][ci][a][b][c]).
 * PIC_EINVAL for a bad layer or a null argument. */
pic_status unet_layer_forward(unet_handle* net, int32_t layer, const float* x_dev, float* y_dev, int32_t relu);
pic_status unet_layer_backward(unet_handle* net, int32_t layer, const float* x_dev, const float* dz_dev, float* dx_dev,
                               float* dw_host, int64_t n_dw);

/* One training step on the warm start's own objective: forward on x_dev
 * (2 x D x H x W, channel 0 the scaled residual r / s of the previous
 * potential), loss L = mean over the unknown planes (all but the last) of
 * (r / s - A y)^2 -- the scaled residual the warm start phi_prev + s y leaves,
 * A the 7-point operator of Eq. (1) with zero values on the cathode plane below
 * the volume and on its last (anode) plane, periodic x/y -- then backward with
 * dL/dy = -(2 / n) A (r / s - A y) and one Adam update as unet_train_step.
 * *loss (host, may be NULL) receives L before the update. */
pic_status unet_train_step_residual(unet_handle* net, const float* x_dev, float lr, double* loss);

/* Timing of the forward convolutions: with on != 0 every later forward pass
 * records CUDA events on the network's stream around each of the 14
 * convolutions (layer order above; not inside a stream capture, such as a
 * recorded PIC step); unet_get_layer_times adds up, per layer,
 * the elapsed milliseconds (ms[14]) and the number of timed launches
 * (count[14]) since profiling was switched on (either pointer may be NULL;
 * synchronises). Switching on or off resets the sums. */
pic_status unet_set_profiling(unet_handle* net, int32_t on);
pic_status unet_get_layer_times(unet_handle* net, double* ms, int64_t* count);

/* Text of the last error on this network (static storage, never NULL). */
const char* unet_last_error(unet_handle* net);

/* Kernel launches issued by the network so far in this process. */
uint64_t unet_launch_count(void);

/* ---- warm start of the PIC solve -------------------------------------------
 * pic_set_warm_unet: instance `inst` of h starts every later solve from
 *   phi0 = phi_prev + s f(r / s, ramp)
 * on the unknown nodes, where r = b - A phi_prev is the residual of the
 * previous potential (A the scaled 7-point operator, b the right-hand side of
 * the step), s its root mean square, ramp = k / nz the position between the
 * electrodes of node plane k, and f the network; network voxel (d, j, i) is
 * node (i, j, k = d + 1), so the network volume is nz x ny x nx (multiples of
 * 8; its last plane lies on the anode, where the input is 0 and the output is
 * not used). The solve then runs to cg_rtol as before. net = NULL returns to
 * the instance's configured warm start. The network must outlive its use and
 * is not owned by the handle. Recorded steps are dropped.
 * PIC_EINVAL for a volume that does not match the grid or a bad instance. */
pic_status pic_set_warm_unet(pic_handle* h, int32_t inst, unet_handle* net);

/* Training samples from a run: given the potentials of two consecutive steps
 * (device, FP64, nodes (nz+1) x ny x nx, layout [k][j][i]) of a grid with
 * nz x ny x nx matching the network volume, writes x_dev (2 x D x H x W) =
 * (A delta / s, ramp) and t_dev (D x H x W) = delta / s with
 * delta = phi_new - phi_old on the unknown nodes, s the root mean square of
 * A delta (0 on the last plane), and *s_out (host, may be NULL) = s. This is
 * the pair the warm start meets: r = A delta when phi_new solves the step. */
pic_status unet_make_sample(unet_handle* net, const double* phi_new_dev, const double* phi_old_dev, float* x_dev,
                            float* t_dev, double* s_out);

/* Copy the potential of an instance (FP64, nodes, layout [k][j][i]) into a
 * caller-owned device array (no host round trip). */
pic_status pic_get_phi_device(pic_handle* h, int32_t inst, double* dev_out);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_UNET_H */
