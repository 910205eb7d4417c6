/*
 * xslam_plain.h -- the plain FP64 complex-step X-KinectFusion step on the GPU: the comparison path.
 *
 * This is X-SLAM's scheme taken literally (Sec. 3 and Sec. 4.1): every quantity of the frame step is a
 * complex<double> with the full complex products of Eq. csfd (no simplified arithmetic), one complex
 * run per perturbed input ("perturbing variables one by one", Sec. 6), each run with its own complex
 * TSDF volume stored as an array of structures (complex F, real W per voxel), complex pose, complex
 * depth pyramid and complex model maps. The kernels follow the same algorithms and readings as the
 * batched FP32 path of xslam.h (range gate, optional bilateral filter, 3-level pyramid, projective
 * point-to-plane ICP with the 6x6 normal equations, TSDF update, ray casting, read-out) with one
 * thread per pixel or voxel and no lane batching, no culling, no CUDA graphs and no tuning. It exists
 * so that the batched path can be measured against it; its results agree with the FP64 oracle to
 * rounding.
 *
 * Conventions are those of xslam.h (poses row-major 3x4 camera to world in double, depth float32
 * metres with 0 = no return, status codes, one host thread per handle, work ordered after the
 * caller's stream).
 */
#ifndef XSLAM_PLAIN_H
#define XSLAM_PLAIN_H

#include "xslam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xslam_plain_s* xslam_plain_t;

/* Allocates max_runs complex runs of an nx*ny*nz volume (24 bytes per voxel and run: Re F, Im F, W)
 * with their pyramids and model maps. Arguments as for xslam_create (cfg NULL = defaults; w_max 0 =
 * no cap). max_runs in 1..16. Errors: XSLAM_EINVAL (bad argument), XSLAM_ENOMEM, XSLAM_ECUDA. */
xslam_status xslam_plain_create(xslam_plain_t* out, int nx, int ny, int nz, float voxel_m, float trunc_m,
                                const float origin_m[3], const xslam_intrinsics* K, const xslam_config* cfg,
                                int max_runs, void* cuda_stream);

/* Frees every device and host buffer of h (NULL: no-op). */
xslam_status xslam_plain_destroy(xslam_plain_t h);

/* Frame-0 pose (real) of every run; only before the first frame (else XSLAM_ESTATE). */
xslam_status xslam_plain_set_pose(xslam_plain_t h, const double T[12]);

/* One frame of every run (Sec. 4.1). seeds: K perturbations (kinds and limits as in xslam.h:
 * POSE0 0..5, TRUNC, DEPTH with index -1; 1e-30 <= |h| <= 1e-3), K in 0..max_runs; K = 0 runs one
 * unperturbed complex run. Seeds are fixed at the first frame (a change gives XSLAM_ESTATE).
 * Outputs (host, NULL allowed): pose_out[12] = Re T of run 0; dpose_out[12 K] = Im T / h per run;
 * dtwist_out[6 K] the same derivative as a left twist (omega, v). The call synchronises with the
 * device. XSLAM_ENOTRACK: ICP failed in run 0; every run was fused at its previous pose. */
xslam_status xslam_plain_frame(xslam_plain_t h, const float* depth, int depth_on_device, const xslam_seed* seeds,
                               int K, double* pose_out, double* dpose_out, double* dtwist_out);

/* Copies one part of run r's volume into out (device, nx*ny*nz doubles): part 0 = Re F, 1 = Im F / h,
 * 2 = W. Errors: XSLAM_EINVAL. */
xslam_status xslam_plain_read_tsdf(xslam_plain_t h, int run, int part, double* out);

/* Message of the last failed call on h (NULL h: of the last failed xslam_plain_create). */
const char* xslam_plain_last_error(xslam_plain_t h);

#ifdef __cplusplus
}
#endif

#endif /* XSLAM_PLAIN_H */
