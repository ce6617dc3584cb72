/*
 * ni_cnn.h - C ABI of the learned warm start of libni.
 *
 * Not part of the paper (an extension beyond it; the paper names learned
 * component heuristics only as future work in its conclusions).  A 6-layer
 * 3x3 convolutional network, 32 channels, ReLU after layers 1-5:
 *   input  4 channels per pixel: (n_x, n_y, n_z, mask)
 *   output 5 channels per pixel: a log-depth (up to one constant per map) and
 *          4 edge-weight logits (right, down, left, up).
 * Convolutions are "valid": an output tile of T x T pixels needs an input tile
 * of (T + 12) x (T + 12) (6-pixel halo; pixels outside the image are zero).
 * Weights and activations are BF16, products are accumulated in FP32 on the
 * tensor cores (mma.sync m16n8k16); the optimiser keeps FP32 master weights.
 *
 * Parameter vector layout (FP32, ni_cnn_num_params() values), layer by layer:
 *   W_l[3][3][cin][cout] (row-major) followed by b_l[cout], for
 *   (cin, cout) = (4,32), (32,32) x 4, (32,5).
 *
 * All array pointers are DEVICE pointers unless the name says host.  Layouts are
 * NHWC float32.  Errors are returned as ni_status; no call aborts.
 */
#ifndef NI_CNN_H_
#define NI_CNN_H_

#include "ni.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ni_cnn ni_cnn;

/* Number of FP32 parameters (39,621). */
int ni_cnn_num_params(void);

/* Network for batches of up to max_batch tiles of tile x tile output pixels
 * (tile >= 16, a multiple of 16).  Parameters start at He-normal values drawn
 * from a counter-based generator keyed by `seed`. */
ni_status ni_cnn_create(int max_batch, int tile, uint64_t seed, ni_cnn** out);
ni_status ni_cnn_destroy(ni_cnn* net);

/* Copy the FP32 parameters to / from host memory (ni_cnn_num_params() floats);
 * set_params also refreshes the BF16 copies and resets the optimiser state. */
ni_status ni_cnn_get_params(ni_cnn* net, float* host_params);
ni_status ni_cnn_set_params(ni_cnn* net, const float* host_params);

/* Forward pass: in = float[B][tile+12][tile+12][4], out = float[B][tile][tile][5]. */
ni_status ni_cnn_forward(ni_cnn* net, const float* in, int B, float* out, ni_stream_t stream);

/* Loss and gradients of one batch (no parameter update):
 *   depth term: mean over intra-component edges (a, b) of both pixels valid and
 *     target_lab[a] == target_lab[b] >= 0 of ((z_a - z_b) - (t_a - t_b))^2
 *     (right and down edges; z = output channel 0, t = target_z);
 *   weight term: mean over valid pixels and directions (right, down, left, up)
 *     with a valid neighbour of the binary cross-entropy between sigmoid(logit)
 *     and target_w in [0, 1];
 *   loss = depth + w_weight * weight.
 * target_z float[B][tile][tile], target_lab int32[B][tile][tile] (-1 invalid),
 * target_w float[B][tile][tile][4].  loss_host[0..2] = (loss, depth, weight).
 * grad_host (may be NULL) receives d loss / d params (ni_cnn_num_params() floats). */
ni_status ni_cnn_loss_grad(ni_cnn* net, const float* in, const float* target_z, const int32_t* target_lab,
                           const float* target_w, int B, float w_weight, double* loss_host, float* grad_host,
                           ni_stream_t stream);

/* ni_cnn_loss_grad followed by one Adam step (beta1 0.9, beta2 0.999, eps 1e-8). */
ni_status ni_cnn_train_step(ni_cnn* net, const float* in, const float* target_z, const int32_t* target_lab,
                            const float* target_w, int B, float w_weight, float lr, double* loss_host,
                            ni_stream_t stream);

/* BiNI edge weights w^BiNI (Sec. 3.1, Eq. 4) of a solved log-depth map, the
 * training targets of the weight channels: for each valid pixel a and direction
 * d (right, down, left, up) with a valid neighbour b,
 *   sigma_k(gamma^2 ((z_{-b} - z_a)^2 - (z_b - z_a)^2)), gamma = f n_a.tau_a,
 * -b the opposite neighbour (its term 0 when it is outside or invalid); 0 for
 * missing neighbours.  normals float[H][W][4], mask uint8[H][W], logdepth
 * float[H][W], out float[H][W][4]. */
ni_status ni_cnn_edge_targets(const float* normals, const uint8_t* mask, const float* logdepth, int H, int W,
                              const ni_camera* cam, double k, float* out, ni_stream_t stream);

/* Input tiles of a map for the network: tiles of tile x tile output pixels in
 * raster order (ceil(H/tile) x ceil(W/tile)), each with its 6-pixel halo, from
 * normals float[H][W][4] and mask uint8[H][W]; pixels outside the image are 0.
 * out = float[ntiles][tile+12][tile+12][4]. */
ni_status ni_cnn_make_tiles(const float* normals, const uint8_t* mask, int H, int W, int tile, float* out,
                            ni_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* NI_CNN_H_ */
