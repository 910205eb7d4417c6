/*
 * xslam_batch.h -- many independent X-KinectFusion trajectories advanced together on one GPU.
 *
 * The per-frame step of X-SLAM (Sec. 4.1) is a serial chain of small launches (27 per frame with a
 * 3-level pyramid), which leaves most of a GB300 idle when one trajectory runs alone. A batch groups
 * handles created with xslam_create -- each with its own volume size, voxel size, intrinsics, image
 * size, configuration, lanes and seeds -- and advances every active one by a frame per call. One call
 * replays one CUDA graph: a kernel gathers each active trajectory's depth frame from the caller's
 * pointers into its handle; then, when every handle runs the plain frame chain (Gauss-Newton ICP with
 * fixed iteration counts from the previous pose; POSE0, TRUNC or all-pixel DEPTH lanes), each stage of
 * the step is one launch over all active trajectories (the range gate, the filter, each pyramid level,
 * each ICP iteration, the tile lists, the update per lane count, the ray cast, the read-out), a block
 * working for one trajectory with that trajectory's own grid, so small trajectories fill the GPU
 * together; otherwise every trajectory's own frame chain runs as a branch of the graph. Trajectories of
 * uneven length leave the batch by passing NULL for their frame; the graph is rebuilt when the active
 * set changes. The paper runs one trajectory at a time and has no counterpart of this call; every
 * trajectory's results are the ones xslam_frame gives for the same frames (bit for bit: the same
 * arithmetic on the same per-trajectory grids).
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
 * ways, as in xslam_create). Errors: XSLAM_EINVAL (bad argument, a handle past frame 0, listed twice or
 * in another live batch), XSLAM_ENOMEM, XSLAM_ECUDA. */
xslam_status xslam_batch_create(xslam_batch_t* out, int n, xslam_t const* handles, void* cuda_stream);

/* Frees the batch (not the handles, which get back the launch shapes they had at xslam_batch_create and
 * may then join another batch). NULL: no-op. */
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

/* Autotuner of the step's launch shapes. A coordinate search, each coordinate tried with the best
 * choices of the coordinates before it: the mode (segmented launches or every trajectory's own chain as
 * a graph branch; only when every handle runs the plain frame chain, see xslam_batch_create); the ICP
 * grid of every trajectory and level divided by 1, 2, 4, 8, 16 or 32 (at least one block); then, in segmented
 * mode, the fusion grid (the default, or 1, 2 or 4 blocks per SM for every trajectory) and the ray-cast
 * tile (32 x 8, 16 x 16 or 64 x 4 pixels). The fusion tile is the 8 x 8 x 8 brick of the TSDF layout and
 * is not tuned. Each candidate runs `steps` >= 3 batch steps from frame 0 on the given frames
 * (frames[s * n + i] = trajectory i's depth at step s, device pointers, NULL = inactive) and times steps
 * 2.. with CUDA events (steps 0 and 1 build the graphs). Then the best choices are kept, every handle is
 * restored to frame 0 (empty volume, the lanes and pose recorded at xslam_batch_create), choice[4]
 * receives the ICP divisor, the fusion blocks per SM (0 = default), the tile (0 = 32 x 8, 1 = 16 x 16,
 * 2 = 64 x 4) and the mode (0 = segmented, 1 = branches), and ms_per_step[15] (NULL allowed) the
 * candidates' milliseconds per step in the order tried, zeros after the last.
 * Errors: XSLAM_EINVAL (steps < 3, NULL frames or choice), as step. */
xslam_status xslam_batch_autotune(xslam_batch_t b, const float* const* frames, int steps, int* choice,
                                  float* ms_per_step);

/* Sets the launch shapes as xslam_batch_autotune returns them in choice[4] (ICP divisor >= 1, fusion
 * blocks per SM 0..32, tile 0..2, mode 0..1; mode 0 falls back to branches when a handle does not run the
 * plain frame chain). The handles keep their state. Errors: XSLAM_EINVAL. Synchronises. */
xslam_status xslam_batch_set_shapes(xslam_batch_t b, const int* choice);

/* Launch profile of the segmented step (tracing, not for timed runs: the events it adds between the
 * launches keep each launch from overlapping the next one's start). enable != 0 records a CUDA event
 * after every launch of the step's graph, which is rebuilt at the next step; 0 removes them.
 * Synchronises. */
xslam_status xslam_batch_profile(xslam_batch_t b, int enable);

/* The launches of the last step in order (profile on, segmented mode; *n = 0 otherwise): kind[q]
 * (0 measurement stage, 1 seed, 2 ICP iteration, 3 tile lists, 4 surface update, 5 ray cast, 6 read-out),
 * arg[q] (measurement: 0 gate, 1 filter, 1 + l pyramid level l; ICP: the largest lane count; surface
 * update: the lane count; ray cast: the tile), blocks[q] (the grid) and ms[q], the time from the end of
 * the previous launch (the first: from the step's start, including the frame gather). *n receives the
 * number of launches; at most cap entries are written; any output array may be NULL. Synchronises. */
xslam_status xslam_batch_profile_read(xslam_batch_t b, int cap, int* kind, int* arg, int* blocks, float* ms,
                                      int* n);

/* Message of the last failed call on b (NULL b: of the last failed xslam_batch_create). */
const char* xslam_batch_last_error(xslam_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* XSLAM_BATCH_H */
