/*
 * xslam_batch.h -- many independent X-KinectFusion trajectories advanced together on one GPU.
 *
 * The per-frame step of X-SLAM (Sec. 4.1) is a serial chain of small launches (27 per frame with a
 * 3-level pyramid), which leaves most of a GB300 idle when one trajectory runs alone. A batch groups
 * handles created with xslam_create -- each with its own volume size, voxel size, intrinsics, image
 * size, configuration, lanes and seeds -- and advances every active one by a frame per call. One call
 * replays one CUDA graph: a kernel gathers each active trajectory's depth frame from the caller's
 * pointers into its handle, then every trajectory's frame chain runs as its own branch of the graph,
 * so the trajectories' kernels overlap on the GPU. Trajectories of uneven length leave the batch by
 * passing NULL for their frame; the graph is rebuilt when the active set changes. The paper runs one
 * trajectory at a time and has no counterpart of this call; every trajectory's results are the ones
 * xslam_frame gives for the same frames (bit for bit: the same kernels on the same grids).
 *
 * Conventions are those of xslam.h.
 */
#ifndef XSLAM_BATCH_H
#define XSLAM_BATCH_H

#include "xslam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xslam_batch_s* xslam_batch_t;

/* Groups n handles (1 <= n <= 256). Every handle must be before its first frame, with its lanes set
 * by xslam_set_lanes and its frame-0 pose by xslam_set_pose; the batch records both (they are what
 * xslam_batch_autotune restores). The handles stay owned by the caller, must outlive the batch, and
 * must not be used on their own while it exists. Work is ordered after cuda_stream (event edges both
 * ways, as in xslam_create). Errors: XSLAM_EINVAL (bad argument, a handle past frame 0 or listed
 * twice), XSLAM_ENOMEM, XSLAM_ECUDA. */
xslam_status xslam_batch_create(xslam_batch_t* out, int n, xslam_t const* handles, void* cuda_stream);

/* Frees the batch (not the handles). NULL: no-op. */
xslam_status xslam_batch_destroy(xslam_batch_t b);

/* Advances every trajectory i with depths[i] != NULL by one frame. depths: n device pointers, each
 * to an H_i x W_i float32 depth map in metres (0 = no return) of handle i's image size; it is read
 * before the call's work completes, so it must stay valid until the next xslam_batch_sync. A NULL
 * entry leaves trajectory i where it is. Asynchronous: the call returns once the work is enqueued.
 * Errors: XSLAM_EINVAL (no active trajectory, NULL array), XSLAM_ECUDA. */
xslam_status xslam_batch_step(xslam_batch_t b, const float* const* depths);

/* Waits for the steps enqueued so far. n_failed (NULL allowed): n ints, the number of frames whose
 * ICP failed (XSLAM_ENOTRACK) per trajectory since its first frame. */
xslam_status xslam_batch_sync(xslam_batch_t b, int* n_failed);

/* Pose and derivative blocks of trajectory i after its last frame (as xslam_frame returns them; NULL
 * outputs are skipped). Synchronises. */
xslam_status xslam_batch_read(xslam_batch_t b, int i, double* pose_out, double* dpose_out, double* dtwist_out);

/* Per-trajectory latency of the last step: ms[i] = time from the start of the step to the end of
 * trajectory i's frame chain (0 for a trajectory that did not advance). Synchronises. */
xslam_status xslam_batch_latency(xslam_batch_t b, float* ms);

/* Autotuner of the ICP grid. For each candidate (the default grid of every trajectory and level
 * divided by 1, 2, 4, 8 and 16, at least one block), runs `steps` >= 3 batch steps from frame 0 on the
 * given frames (frames[s * n + i] = trajectory i's depth at step s, device pointers, NULL = inactive)
 * and times steps 2.. with CUDA events (steps 0 and 1 build the graphs); then keeps the fastest
 * candidate, restores every handle to frame 0 (empty volume, the lanes and pose recorded at
 * xslam_batch_create) and returns the chosen divisor in *divisor and the candidates' milliseconds per
 * step in ms_per_step[5] (NULL allowed). Errors: XSLAM_EINVAL (steps < 3, NULL frames), as step. */
xslam_status xslam_batch_autotune(xslam_batch_t b, const float* const* frames, int steps, int* divisor,
                                  float* ms_per_step);

/* Message of the last failed call on b (NULL b: of the last failed xslam_batch_create). */
const char* xslam_batch_last_error(xslam_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* XSLAM_BATCH_H */
