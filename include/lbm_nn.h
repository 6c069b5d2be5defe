/*
 * lbm_nn.h -- C ABI of the warm-start surrogate of liblbm_gb300.so.
 *
 * The paper solves each lattice from rest; it has no learned component.
 * This surrogate is library plumbing around the method: a small
 * convolutional encoder-decoder ("WarmNet") that maps per-cell inputs of a
 * lattice instance to an initial guess of its steady fields, from which
 * lbm_init_fields / lbm_batch_init_fields start the unmodified scheme.  Its
 * forward pass, backward pass and Adam update run as CUDA kernels: the 3x3
 * convolutions (forward, input gradient, weight gradient) as implicit GEMMs
 * on the fifth-generation tensor cores (tcgen05.mma with BF16 operands and an
 * FP32 accumulator in tensor memory); pooling, upsampling, skip additions,
 * the output stage, the loss and the optimizer as plain kernels.
 *
 * Network (levels l = 0 .. L-1, channels c[l]):
 *   encoder: x = relu(conv(x)); x = relu(conv(x)); e[l] = x;
 *            x = avgpool2(x) unless l = L-1
 *   decoder, l = L-2 .. 0: x = upsample2(x); x = relu(conv(x));
 *            x = x + e[l]; x = relu(conv(x))
 *   output:  y = conv(x) (c[0] -> 3 channels), then the fixed output stage
 *            out = unstagger(smooth(y))
 * A convolution computes out(y, x) = b + sum_{dy,dx} in(y+dy-1, x+dx-1)
 * W[dy][dx] with zero padding.  Inputs have 4 channels, outputs 3.
 * Output stage (no parameters; a cell is fluid where input channel 0, the
 * solid flag, is below 1/2): smooth applies [1, 2, 1] / 4 along x and then
 * along y, with solid cells and cells outside the grid taken as 0, and sets
 * solid cells to 0; unstagger removes from output channel 1 (u_x) its
 * component along (-1)^x and from channel 2 (u_y) its component along
 * (-1)^y over each instance's fluid cells.  The lattice Boltzmann scheme
 * keeps the staggered momenta sum (-1)^(x+n) rho u_x and
 * sum (-1)^(y+n) rho u_y exactly (lbm.h, lbm_diagnostics), so a warm start
 * carrying them would settle on a different state from the rest start; the
 * output stage gives predictions none.  Both maps are self-adjoint; the
 * backward pass applies them in reverse order.
 *
 * Storage: activations BF16 NHWC with channels padded to a multiple of 8;
 * weights kept as FP32 masters with BF16 copies; gradients of activations
 * BF16, of parameters FP32; the output stage, its result and the loss
 * gradient FP32.  Loss: sum over fluid cells (fluid != 0) of the
 * squared output error, divided by 3 x the number of fluid cells.
 *
 * Parameter vector (lbm_nn_get_params / set_params / gradients): for each
 * convolution in forward order, its weights in (dy, dx, cin, cout) order
 * (cout fastest) followed by its cout biases, as float.
 *
 * Conventions as in lbm.h: lbm_status returns, host arrays copied, work on
 * the stream given at creation; every call here is synchronous.  Every wait
 * of the tensor-core GEMMs is bounded: one that runs out leaves its tile
 * unstored and the call returns LBM_ERR_TIMEOUT.
 */
#ifndef LBM_GB300_NN_H
#define LBM_GB300_NN_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_nn lbm_nn;

/* Create a network of `levels` (1 .. 6) levels with channels[l] (1 .. 512)
 * channels, for batches of up to max_batch (>= 1) instances of height x
 * width cells (multiples of 2^(levels-1), at most 4096 each).  Weights
 * start He-normal from `seed` (zero biases); Adam moments at zero.
 * Errors: LBM_ERR_INVALID, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_nn_create(int levels, const int* channels, int max_batch, int height,
                         int width, uint64_t seed, void* cuda_stream, lbm_nn** out);
void lbm_nn_destroy(lbm_nn* nn);

/* Number of floats of the parameter vector. */
size_t lbm_nn_param_count(const lbm_nn* nn);
lbm_status lbm_nn_get_params(lbm_nn* nn, float* params);
/* Replaces the parameters (and resets the Adam moments and step). */
lbm_status lbm_nn_set_params(lbm_nn* nn, const float* params);

/* y (n x height x width x 3 floats) from x (n x height x width x 4 floats),
 * host arrays, 1 <= n <= max_batch. */
lbm_status lbm_nn_forward(lbm_nn* nn, const float* x, int n, float* y);

/* Prolongation of outputs to a grid `factor` (1 .. 16) times finer, for
 * instances larger than the network's grid: y (n x height x width x 3
 * floats, e.g. lbm_nn_forward's output on block-averaged inputs) is
 * interpolated bilinearly between cell centres (the centre of fine cell
 * (Y, X) at coarse coordinates ((Y + 1/2) / factor - 1/2, ...), clamped to
 * the outermost coarse centres), set to 0 on the solid fine cells, and put
 * through the fixed output stage at the fine resolution with the fine
 * fluid flags (fluid: n x H x W bytes, nonzero = fluid, H = factor x
 * height, W = factor x width), so that the result carries no staggered
 * momentum on the fine lattice either.  out: n x H x W x 3 floats.  Host
 * arrays, 1 <= n <= max_batch; the fine buffers are allocated on the first
 * call at a size and kept until lbm_nn_destroy.  Errors: LBM_ERR_INVALID,
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_nn_prolong(lbm_nn* nn, const float* y, int n, int factor, const uint8_t* fluid,
                          float* out);

/* Loss and parameter gradients (param_count floats, nullable) of a batch:
 * x as above, target n x height x width x 3, fluid n x height x width
 * bytes.  Does not change the parameters. */
lbm_status lbm_nn_gradients(lbm_nn* nn, const float* x, const float* target,
                            const uint8_t* fluid, int n, float* loss, float* grads);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * learning rate lr on the gradients of the batch; *loss (nullable) gets the
 * loss before the step. */
lbm_status lbm_nn_train_step(lbm_nn* nn, const float* x, const float* target,
                             const uint8_t* fluid, int n, float lr, float* loss);

/* Number of kernel launches issued so far. */
int64_t lbm_nn_launch_count(const lbm_nn* nn);

const char* lbm_nn_last_error(const lbm_nn* nn);

#ifdef __cplusplus
}
#endif
#endif
