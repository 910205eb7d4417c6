/*
 * xslam_mlp.h -- the learned pose proposal: a small perceptron trained on the GPU with hand-written
 * tensor-core (tcgen05, BF16 operands, FP32 accumulation) forward and backward kernels, and its use
 * as the start pose of the coarsest ICP level of the X-KinectFusion step.
 *
 * X-SLAM has no such network: its ICP starts each frame at the previous pose (Sec. 4.1). The network
 * here maps two depth frames to the camera motion between them; it is trained on frame pairs and
 * the poses the method itself tracks, and plain ICP from the constant-velocity start stays both the
 * fallback and the judge (xslam_set_proposal).
 *
 * Network (layers l = 1..L, widths n_0..n_L, at most 6 layers): a_0 = q(x), z_l = a_{l-1} q(W_l)^T + b_l,
 * a_l = q(relu(z_l)) for l < L, y = z_L, with q the rounding to bfloat16 (nearest, ties to even):
 * weights and activations are BF16, every product sum is accumulated in FP32 and the biases are FP32.
 * Loss of a batch of B rows with targets t: E = 1/(2B) sum |y - t|^2. Gradient: dz_L = (y - t)/B and
 * dW_l = q(dz_l)^T a_{l-1}, db_l = sum over rows of dz_l, dz_{l-1} = (q(dz_l) q(W_l)) * [a_{l-1} > 0]
 * (the roundings pass the gradient through unchanged). Optimiser: Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected) on FP32 master weights; the BF16 copies are refreshed after each step.
 *
 * Input features (xslam_mlp_features): a W x H depth map (W a multiple of 80, H of 60) becomes 80 x 60
 * block means of its depths inside [depth_min, depth_max], divided by 4 m (0 for a block without
 * one), BF16, row-major. A frame pair (i, j) is the row [f_i, f_j] of 9600 values.
 *
 * Parameter layout on the host (xslam_mlp_set_params / get_params / gradient): for l = 1..L, W_l as
 * n_l x n_{l-1} row-major FP32, then b_l (n_l values).
 *
 * Conventions are those of xslam.h (status codes, device pointers of the create-time device, one host
 * thread at a time per object, work ordered on an internal stream after the caller's stream).
 */
#ifndef XSLAM_MLP_H
#define XSLAM_MLP_H

#include <stddef.h>

#include "xslam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xslam_mlp_s* xslam_mlp_t;

/* Create a network with n_layers (1..6) layers of widths sizes[0..n_layers] (sizes[0] a multiple of 64,
 * every width 1..16384) for batches of up to max_batch rows (1..4096). Internally every width but the
 * input's is padded with zeros to a multiple of 64. Weights start at zero (use xslam_mlp_set_params).
 * Allocates every buffer the later calls use except the training permutation (xslam_mlp_train).
 * Errors: XSLAM_EINVAL, XSLAM_ENOMEM, XSLAM_ECUDA. */
xslam_status xslam_mlp_create(xslam_mlp_t* out, int n_layers, const int* sizes, int max_batch, void* cuda_stream);

/* Free the network (synchronises). NULL: no-op. */
xslam_status xslam_mlp_destroy(xslam_mlp_t m);

/* Number of FP32 parameters in the host layout. */
size_t xslam_mlp_param_count(xslam_mlp_t m);

/* Set the FP32 master parameters from host params[param_count] (layout above), reset the Adam moments
 * and step, and round the BF16 copies. Synchronises. */
xslam_status xslam_mlp_set_params(xslam_mlp_t m, const float* params);

/* Copy the FP32 master parameters to host params[param_count]. Synchronises. */
xslam_status xslam_mlp_get_params(xslam_mlp_t m, float* params);

/* Forward pass: x device BF16 [B x sizes[0]] row-major, 1 <= B <= max_batch; writes device FP32
 * y [B x sizes[L]]. Synchronises. Errors: XSLAM_EINVAL, XSLAM_ETIMEOUT (a tensor-core wait ran out). */
xslam_status xslam_mlp_forward(xslam_mlp_t m, const void* x, int B, float* y);

/* Loss and gradient of one batch without a parameter update: x device BF16 [B x sizes[0]], targets
 * device FP32 [B x sizes[L]], B a multiple of 64 up to max_batch. Writes host grad[param_count]
 * (layout above; NULL skips) and *loss (NULL skips). Synchronises. Errors as xslam_mlp_forward. */
xslam_status xslam_mlp_gradient(xslam_mlp_t m, const void* x, const float* targets, int B, float* grad, double* loss);

/* 80 x 60 features of n device depth frames depth[n x H x W] into device BF16 out[n x 4800]
 * (the depth range as in xslam_config). Asynchronous on the caller's stream cuda_stream. */
xslam_status xslam_mlp_features(const float* depth, int n, int W, int H, float depth_min, float depth_max, void* out,
                                void* cuda_stream);

/* Host-side training targets: for each of the n_pairs pairs (i, j) = (pairs[2p], pairs[2p+1]) of the
 * host poses[n_poses x 12] (3x4 camera-to-world, row-major), out[6p..6p+5] = log(T_i^-1 T_j) / scale,
 * the twist (phi, rho) of the motion from camera i to camera j in camera i's frame, divided
 * component-wise by scale[6] (rotation angles below pi). Errors: XSLAM_EINVAL (index out of range). */
xslam_status xslam_mlp_pair_targets(const double* poses, int n_poses, const int* pairs, int n_pairs,
                                    const float* scale, float* out);

/* Train with Adam at learning rate lr for `epochs` passes over n_pairs training pairs: feat device
 * BF16 [n_feat x 4800] frame features, pairs device int [n_pairs x 2] (frame indices, earlier frame
 * first), targets device FP32 [n_pairs x sizes[L]]. sizes[0] must be 9600. Each epoch visits the pairs
 * in an order drawn from seed (splitmix64 and Fisher-Yates on the host) in batches of `batch` rows
 * (a multiple of 64 up to max_batch; a last incomplete batch is skipped); one step per batch is a
 * replay of a CUDA graph of the whole step. mirror = 1 (6 outputs holding the twists of
 * xslam_mlp_pair_targets, cameras whose principal point is the image centre): each visit of a pair
 * reflects it at random left-right and/or top-bottom, both feature maps and the target (the twist of
 * the reflected motion: phi_y, phi_z, rho_x negated left-right; phi_x, phi_z, rho_y top-bottom).
 * epoch_loss (host, NULL allowed) receives each epoch's mean batch loss. Allocates the device
 * permutation (n_pairs ints) when it is larger than any before. Synchronises. Errors: XSLAM_EINVAL
 * (also a pair naming a frame outside the feature table), XSLAM_ENOMEM, XSLAM_ETIMEOUT, XSLAM_ECUDA. */
xslam_status xslam_mlp_train(xslam_mlp_t m, const void* feat, int n_feat, const int* pairs, const float* targets,
                             int n_pairs, int batch, int epochs, float lr, unsigned long long seed, int mirror,
                             float* epoch_loss);

/* One BF16 GEMM on the tensor cores: C[M x N] = A[M x K] B[N x K]^T, all device, A and B BF16
 * row-major (16-byte aligned), C FP32, K a multiple of 64. splits = 1: the product is written to C
 * directly; splits > 1: K is cut into ranges of whole 64-wide slices (at most `splits` of them) whose
 * FP32 partial products go to device workspace[splits x M x N] and are then added into C in range
 * order. Ordered on cuda_stream, which the call synchronises. Calls from several host threads at once
 * share one device error flag. Errors: XSLAM_EINVAL (shape, splits > K / 64, missing workspace),
 * XSLAM_ETIMEOUT, XSLAM_ECUDA. */
xslam_status xslam_gemm_bf16(const void* A, const void* B, int M, int N, int K, float* C, int splits, float* workspace,
                             void* cuda_stream);

/*
 * Attach network m as the learned proposal of handle h (NULL m: detach). From the next frame on,
 * with T_1 = T_{k-1}: the network reads the features of the previous and current depth frames and
 * its output y gives xi = scale * y (scale[6], host); two ICP runs go from the coarsest level down to
 * judge_level (0..icp_levels-1), run A from the handle's configured start (cfg.icp_seed) and run B
 * from T_1 exp(xi); each is judged by J = mean over that level's pixels with a depth of
 * min(r^2, g^2), r the point-to-plane residual against the model point at the nearest pixel of the
 * pixel's projection into the model camera (g^2 where there is none or |p - V| > g, g the distance
 * gate); run B is kept if it did not fail and J_B <= J_A, and the kept run continues to level 0.
 * The network must have sizes[0] = 9600 and sizes[L] = 6, the image size must be a multiple of
 * 80 x 60, the configuration Gauss-Newton ICP, and m must outlive its attachment (not be trained while
 * attached). Allocates the handle's inference buffers. Counters: xslam_counters. Errors:
 * XSLAM_EINVAL, XSLAM_ENOMEM, XSLAM_ECUDA.
 */
xslam_status xslam_set_proposal(xslam_t h, xslam_mlp_t m, const float* scale, int judge_level);

/*
 * Device counters of h since create or the last reset through this call (synchronises):
 * out[0] Gauss-Newton ICP iterations computed, counted when a stop tolerance is set (cfg.icp_stop > 0;
 * iterations skipped after a failure or after their level converged are not counted; without a
 * tolerance every frame runs the fixed counts and this counter stays 0), out[1] frames whose proposal
 * was judged, out[2] proposals accepted. reset = 1 zeroes the three counters after reading.
 */
xslam_status xslam_counters(xslam_t h, unsigned long long* out, int reset);

/* Message of the last failed call on m (NULL m: of the last failed call made without an object). */
const char* xslam_mlp_last_error(xslam_mlp_t m);

#ifdef __cplusplus
}
#endif

#endif /* XSLAM_MLP_H */
