/* maclab_ws.h -- learned warm start for steady-state runs of the streaming
 * MacLABSWE step (Zhou, arXiv:1902.02999).
 *
 * The paper has no counterpart to anything in this header.  Its Section 3
 * procedure iterates "until a solution is reached"; the iteration always
 * decides the answer.  This component only proposes the starting state
 * (h, u, v) of that iteration: a residual convolutional network, run on a
 * coarse grid of R x R cells (each cell the mean of 4 x 4 fine nodes),
 * maps the problem inputs (still-water depth, node mask, wind, friction) to
 * a steady (eta, u, v); the proposal is interpolated back to the fine grid
 * and handed to maclab_set_state, and the plain iteration then converges
 * from it.
 *
 * Network (all tensors NHWC, channels padded to 16 at the input and output):
 *   H_1     = conv3x3(X; W_0, b_0)                      16 -> C channels
 *   H_{l+1} = H_l + conv3x3_{d_l}(relu(H_l); W_l, b_l)  l = 1..L, dilation d_l
 *   Y       = conv3x3(relu(H_{L+1}); W_out, b_out)      C -> 16 channels
 * 3 x 3 convolutions with zero padding; weights W[tap][c_out][c_in] with
 * tap = 3 (dy + 1) + (dx + 1), the input pixel of tap (dy, dx) being
 * (y + d dy, x + d dx).  Activations are stored in bfloat16, products are
 * summed in float (tensor-core instructions), master weights and their
 * Adam moments are float.  Loss = sum_p w_p sum_{c < out_ch} (Y - T)^2 with
 * caller-normalised weights w (sum 1 over the batch).
 *
 * All pointers named *_dev are device pointers (float unless stated); the
 * handle owns its weights, moments and activation buffers.  Every call runs
 * on the handle's stream; calls that return a host value synchronise.
 * Errors: MACLAB_E_ARG for bad sizes or NULL pointers, MACLAB_E_CUDA for a
 * failed launch or a tensor-core wait that timed out (reported by the next
 * call that synchronises), MACLAB_E_NOMEM when device memory runs out
 * (status codes of maclab.h); maclab_last_error(NULL) gives the message.
 */
#ifndef MACLAB_WS_H
#define MACLAB_WS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct maclab_ws_s* maclab_ws_t;

#define MACLAB_WS_IO 16   /* padded input / output channels */
#define MACLAB_WS_CELL 4  /* fine nodes per coarse cell along each axis */

typedef struct {
    int res;           /* coarse grid R (cells per side), a multiple of 64 */
    int channels;      /* C, a multiple of 64 */
    int blocks;        /* residual blocks L, 0..64 */
    int dilation[64];  /* d_l >= 1 of block l (entries past L unused) */
    int max_batch;     /* largest batch the activation buffers hold */
    uint64_t seed;     /* weight initialisation (SplitMix64 stream) */
    int tensor_path;   /* 0 (default): every convolution and weight
                          gradient on tcgen05, operands staged by TMA
                          (channel counts 16 or multiples of 64 in, 16 or
                          multiples of 128 out; other shapes on mma.sync);
                          1: the 128 -> 128 convolutions on tcgen05 with
                          operands staged by cp.async, the rest on mma.sync;
                          2: everything on mma.sync.  Other values are
                          rejected. */
} maclab_ws_config;

/* Create a network with freshly initialised weights (He-scaled normal
 * weights from the seed, zero biases; the last layer starts at zero). */
int maclab_ws_create(const maclab_ws_config* cfg, void* stream, maclab_ws_t* out);
void maclab_ws_destroy(maclab_ws_t ws);

/* Number of float parameters; parameter vector in the order
 * W_0, b_0, W_1, b_1, ..., W_L, b_L, W_out, b_out (host copies). */
int maclab_ws_param_count(maclab_ws_t ws, int64_t* n);
int maclab_ws_get_params(maclab_ws_t ws, float* host, int64_t n);
int maclab_ws_set_params(maclab_ws_t ws, const float* host, int64_t n);

/* Y = net(X) for `batch` samples: x_dev [batch][R][R][16], y_dev
 * [batch][R][R][16]. */
int maclab_ws_forward(maclab_ws_t ws, int batch, const float* x_dev, float* y_dev);

/* Loss and gradients (host copy, same order as the parameters) without
 * changing the weights: t_dev targets [batch][R][R][16], w_dev weights
 * [batch][R][R]; out_ch channels enter the loss.  For gradient checks. */
int maclab_ws_gradients(maclab_ws_t ws, int batch, int out_ch, const float* x_dev, const float* t_dev,
                        const float* w_dev, float* grad_host, int64_t n, double* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * loss of the batch; *loss (may be NULL) receives the loss before the step.
 * Does not synchronise when loss is NULL. */
int maclab_ws_train_step(maclab_ws_t ws, int batch, int out_ch, const float* x_dev, const float* t_dev,
                         const float* w_dev, float lr, double* loss);

/* Checks of single layers.  With keep on, the backward pass of
 * maclab_ws_gradients / maclab_ws_train_step leaves the loss gradient with
 * respect to every H_l in a buffer of its own (L + 1 more activation-sized
 * bf16 buffers, allocated on the first call with on = 1 and kept until
 * destroy) instead of overwriting two.  MACLAB_E_NOMEM if they do not fit. */
int maclab_ws_keep_gradients(maclab_ws_t ws, int on);

/* Float copy into out_dev of a tensor the handle stores, as of the last
 * call, for the first `batch` samples of that call:
 *   what 0: H_{index+1} (index 0..L) [batch][R][R][C], bf16 as stored,
 *           after a forward, gradients or train step;
 *   what 1: d loss / d H_{index+1} (index 0..L) [batch][R][R][C], bf16 as
 *           stored, after a gradients or train step taken with keep on;
 *   what 2: d loss / d Y [batch][R][R][16], bf16 as stored, after a
 *           gradients or train step (index 0);
 *   what 3: Y [batch][R][R][16], float (index 0).
 * n must equal the element count.  MACLAB_E_ARG when the tensor is not
 * there (no such call since the last forward pass, or batch too large).
 * Runs on the handle's stream; does not synchronise. */
int maclab_ws_inspect(maclab_ws_t ws, int what, int index, int batch, float* out_dev, int64_t n);

/* Problem inputs of one fine n x n grid -> coarse network input and, when
 * eta/u/v are given, coarse targets.  n = R * MACLAB_WS_CELL.
 *   D_dev     [n][n] still-water depth h_ref - z_b (m)
 *   mask_dev  [n][n] uint8 node types of maclab.h
 *   wind_u, wind_v, Cb, dx: the problem's uniform wind (m/s), friction
 *             and lattice size (m)
 *   eta/u/v_dev [n][pitch] a state (may be NULL: no targets)
 *   scale[4]  divisors of (depth, eta, u, v) making the channels O(1)
 *   x_dev [R][R][16]: fluid fraction, mean depth / scale[0], wind_u / 5,
 *     wind_v / 5, 100 Cb, cell x and y in [-1, 1], dx / 2, zeros
 *   t_dev [R][R][16]: fluid means of eta / scale[1], u / scale[2],
 *     v / scale[3], zeros; w_dev [R][R] fluid fraction. */
int maclab_ws_encode(maclab_ws_t ws, int n, const float* D_dev, const uint8_t* mask_dev, double wind_u,
                     double wind_v, double Cb, double dx, const float* eta_dev, const float* u_dev, const float* v_dev,
                     int pitch, const double scale[4], float* x_dev, float* t_dev, float* w_dev);

/* Coarse output y_dev [R][R][16] -> fine proposal (h, u, v) as double
 * [n][n] device arrays: channels 0..2 times scale[1..3], bilinear between
 * cell centres (clamped at the border), h = D + eta; solid nodes get
 * h = D, u = v = 0 and no-slip nodes u = v = 0.  When mass_eta is finite,
 * eta is then shifted by one constant over the non-solid nodes so that it
 * sums to mass_eta there: the iteration conserves mass exactly in a closed
 * basin, so its steady state depends on the initial volume (mass_eta = 0
 * for a basin filled to its still-water level h_ref). */
int maclab_ws_decode(maclab_ws_t ws, int n, const float* y_dev, const float* D_dev, const uint8_t* mask_dev,
                     const double scale[4], double mass_eta, double* h_dev, double* u_dev, double* v_dev);

#ifdef __cplusplus
}
#endif

#endif /* MACLAB_WS_H */
