/*
 * xslam.h -- C ABI of the GB300 (sm_103a) X-KinectFusion step in complex-step (CSFD) arithmetic.
 *
 * The method is X-SLAM (Peng, Yang, Shao, Jiang, Zhou, ACM TOG 43(4) art. 79, 2024): a dense SLAM
 * step (surface measurement, projective point-to-plane ICP, TSDF surface update, ray casting; Sec.
 * 4.1) evaluated on complex numbers so that Im(f(x + h i)) / h is the derivative of every result with
 * respect to a perturbed input (Sec. 3, Eq. csfd). Following the simplified complex arithmetic of
 * Sec. 3 (Eq. csfd_simplify_multiplication / csfd_simplify_division: products of two imaginary parts
 * are dropped), each perturbed input j = 1..K owns one FP32 imaginary lane next to one shared real
 * lane; the 6x6 Gauss-Newton solve, its final cross-block sum and the SE(3) pose composition run in
 * FP64.
 *
 * Conventions for every call:
 *   - a pose is a row-major 3x4 array [R | t] in double, camera to world (the paper's T_{g,k});
 *   - a pose "lane block" is (1 + K) consecutive 12-double poses: lane 0 is the real pose, lane j is
 *     the imaginary part Im(T*) of perturbation j (the raw value, h_j included);
 *   - depth images are float32 metres along the camera z axis, row-major H x W, 0 = no return;
 *   - device pointers must belong to the CUDA device that was current at xslam_create; host pointers
 *     are ordinary (preferably pinned) host memory;
 *   - every call returns an xslam_status; on an error other than XSLAM_ENOTRACK the handle's state
 *     is unchanged and xslam_last_error() describes the problem;
 *   - a handle is used by one host thread at a time; work is ordered on the handle's internal
 *     stream, which is ordered after the caller's stream given at create (event edges both ways).
 */
#ifndef XSLAM_H
#define XSLAM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xslam_s* xslam_t;

typedef enum {
  XSLAM_OK = 0,
  XSLAM_EINVAL = 1,   /* bad argument or unsupported option                         */
  XSLAM_ENOMEM = 2,   /* device or host allocation failed (create, set_proposal)    */
  XSLAM_ECUDA = 3,    /* a CUDA runtime call failed; see xslam_last_error           */
  XSLAM_ETIMEOUT = 4, /* a device-side wait exceeded its budget                     */
  XSLAM_ENOTRACK = 5, /* soft: ICP failed; the frame was fused at the previous pose */
  XSLAM_ESTATE = 6    /* call not valid in the handle's current state               */
} xslam_status;

/*
 * Which input a lane perturbs (X-SLAM Sec. 4.1). The two per-frame pose kinds promote frame k's own pose
 * (Eq. lie) and restart at every frame: before frame k > 0 the lane drops the imaginary parts earlier
 * frames left in its pose lanes, its TSDF plane and its model maps, so that Im(X_k) / h is the
 * derivative of frame k's results with respect to frame k's pose alone (the paper's dF_k / dxi_{k,i}
 * and Eq. pvnpxi), not a sum over frames. At frame 0 both equal POSE0.
 */
typedef enum {
  XSLAM_SEED_POSE0 = 0, /* index 0..5: left twist (phi then rho) of frame 0's pose, Eq. lie / pvnpxi    */
  XSLAM_SEED_POSE = 1,  /* index 0..5: left twist of frame k's pose before ICP, i.e. ICP's start (the
                           previous pose, or the constant-velocity / proposal starts; both runs of the
                           proposal are perturbed): dpose_out is d T_k / d xi_{k,0}, which ICP's
                           contraction makes small once it converges                                  */
  XSLAM_SEED_TRUNC = 2, /* the truncation distance mu (Sec. 4.1, Psi)                                   */
  XSLAM_SEED_DEPTH = 3, /* index -1: every valid pixel of every frame, D* = D + h i (Eq. csfd_depth);
                           index p in 0..W H - 1: level-0 pixel p of every frame (its perturbation
                           passes through the bilateral filter and the pyramid like the depth)         */
  XSLAM_SEED_POSE_TRACKED = 4 /* index 0..5: left twist of frame k's tracked pose T_{g,k} (the ICP result)
                           as the surface update and the ray cast use it (Eq. lie, Eq. pvnpxi, and
                           dF_k / dxi_{k,i} of the surface update): dpose_out is G_index T_k exactly;
                           xslam_read_tsdf and the model maps carry the derivatives                   */
} xslam_seed_kind;

typedef struct {
  int kind;   /* xslam_seed_kind                                                   */
  int index;  /* twist component 0..5 (pose kinds); -1 or a pixel (DEPTH); 0 (TRUNC) */
  double h;   /* imaginary step; the read-out divides Im by h                      */
} xslam_seed;

typedef struct {
  float fx, fy, cx, cy; /* pinhole intrinsics K of pyramid level 0; pixel centres at integers */
  int width, height;    /* level-0 image size; both must be divisible by 2^(icp_levels-1)      */
} xslam_intrinsics;

/* Every constant the paper leaves open (defaults from xslam_default_config in brackets). */
typedef struct {
  int icp_levels;        /* pyramid levels used by ICP, 1..3 [3]                                   */
  int icp_iters[4];      /* Gauss-Newton iterations per level, finest first [10, 5, 4]              */
  float dist_gate_m;     /* reject a correspondence with |p' - q| above this [0.1]                 */
  float normal_gate_deg; /* reject if the measured and model normals differ more than this [20]    */
  float disc_gate_m;     /* depth-discontinuity gate on a bilinear cell (Sec. 4.1) [0.1]           */
  float min_corr_frac;   /* fewer correspondences than this fraction of a level fails ICP [0.1]    */
  float ray_step_vox;    /* ray-casting step in voxels of camera depth [1]                          */
  float depth_min_m;     /* valid depth range; also the ray-casting range [0.2]                     */
  float depth_max_m;     /* [4.0]                                                                   */
  float pyr_range_m;     /* pyramid smoothing skips taps farther than this from the centre [0.09]  */
  int bilateral;         /* 1: bilateral filter of the gated raw depth (Sec. 4.1; 7x7, spatial
                            sigma 4.5 px, range sigma 0.03 m), 0: off [0]                         */
  float w_max;           /* cap of the TSDF weight after each update; <= 0 means none [0]           */
  int icp_newton;        /* 1: Newton ICP (Sec. 4.1, second-order ICP; the Hessian of each iteration's
                            energy by the second-order complex step), for the real pose only: lanes
                            must be 0 (XSLAM_EINVAL otherwise); 0: Gauss-Newton [0]                  */
  float icp_newton_eta;  /* Newton ICP: an iteration uses the Hessian when the mean squared residual is
                            at most this (m^2) and the Hessian is positive definite, else the
                            Gauss-Newton matrix of the same exact first derivatives [1e-4]          */
  int icp_seed;          /* ICP start of frame k: 0 the previous pose T_{k-1} (Sec. 4.1), 1 constant
                            velocity T_{k-1} T_{k-2}^-1 T_{k-1} (T_0 at k = 1), on every lane [0]    */
  float icp_stop;        /* > 0: a pyramid level ends after an iteration whose real step (twist
                            norm) is below this; the remaining iterations of the level are skipped
                            (Gauss-Newton ICP only); 0: fixed iteration counts [0]                  */
} xslam_config;

/* Fill *cfg with the defaults above. */
void xslam_default_config(xslam_config* cfg);

/*
 * Create a handle owning a TSDF volume of nx*ny*nz voxels of voxel_m metres whose min corner is at
 * origin_m (voxel centres at origin + (i + 0.5) voxel, linear index x + nx (y + ny z)), truncation
 * distance trunc_m (mu), intrinsics K, options cfg (NULL = defaults), room for up to max_lanes
 * imaginary lanes (0..15), ordered after the CUDA stream cuda_stream (a cudaStream_t; NULL = the
 * legacy default stream). Allocates all device memory the later calls use (the frame pipeline
 * included); no other call allocates, except xslam_set_proposal (include/xslam_mlp.h), which
 * allocates the attached network's inference buffers.
 * The volume starts unobserved (F = 1, W = 0) and the first frame's pose is the identity until
 * xslam_set_pose. Errors: XSLAM_EINVAL (sizes, intrinsics, lanes, config), XSLAM_ENOMEM, XSLAM_ECUDA.
 */
xslam_status xslam_create(xslam_t* out, int nx, int ny, int nz, float voxel_m, float trunc_m,
                          const float origin_m[3], const xslam_intrinsics* K, const xslam_config* cfg,
                          int max_lanes, void* cuda_stream);

/* Free the handle and all its device memory (synchronises its stream). NULL is accepted. */
xslam_status xslam_destroy(xslam_t h);

/* Clear the volume to unobserved, forget the lanes and go back to frame 0 (keeps the pose). */
xslam_status xslam_reset(xslam_t h);

/* Set the real pose of the next frame (only before frame 0, XSLAM_ESTATE afterwards); host array. */
xslam_status xslam_set_pose(xslam_t h, const double T_world_cam[12]);

/*
 * One X-KinectFusion step (Sec. 4.1) on depth map `depth` (H x W float32; device pointer if
 * depth_on_device, else host): range gate, bilateral filter (if the configuration says so), 3-level
 * Gaussian pyramid, multi-level projective
 * point-to-plane ICP from the previous pose against the previous frame's ray-cast model (frame 0
 * keeps its pose), TSDF update at the new pose, ray cast at the new pose; every step on 1 + K lanes.
 * seeds[K] (K <= max_lanes) define the lanes; they are fixed by the first frame after create/reset
 * and must be repeated unchanged afterwards (XSLAM_ESTATE otherwise).
 * Outputs (host arrays, each may be NULL): pose_out[12] = Re T_k; dpose_out[12 K] = Im T_k / h_j
 * (lane-major, 12 per lane); dtwist_out[6 K] = the same derivative as a left twist (omega, v) with
 * [omega] = dR R^T, v = dt - omega x t. If all three are NULL and depth is on the device the call only
 * enqueues work and returns without synchronising (use xslam_sync for ICP failures).
 * Returns XSLAM_ENOTRACK (outputs filled) if ICP failed at some level: too few correspondences or a
 * non-positive-definite normal matrix; the frame is then fused at the previous pose.
 */
xslam_status xslam_frame(xslam_t h, const float* depth, int depth_on_device, const xslam_seed* seeds,
                         int K, double* pose_out, double* dpose_out, double* dtwist_out);

/* Wait for the handle's work; returns XSLAM_ENOTRACK if any frame since the last xslam_sync failed
 * to track, *n_failed (may be NULL) receives how many. Frames run through xslam_frame_submit report
 * their failures to xslam_frame_wait instead and are not counted here. */
xslam_status xslam_sync(xslam_t h, int* n_failed);

/* Frames that may be submitted and not yet waited for (xslam_frame_submit). */
#define XSLAM_PIPELINE 4

/*
 * Pipelined form of xslam_frame (the same Sec. 4.1 step, same arguments, same results bit for bit):
 * enqueue the frame and return without waiting for it; *ticket receives the frame's number, which
 * xslam_frame_wait takes to deliver its outputs. This lets a caller submit frame k + 1 before it reads
 * frame k's pose, so the host's own work, the depth upload and the result read overlap the GPU's
 * frames. A host depth map (pinned memory for an asynchronous copy) is uploaded on a second stream
 * into one of two device staging buffers while the frame before runs; the caller keeps it unchanged
 * until xslam_frame_wait(ticket) returns. A device depth map is copied on the handle's stream.
 * Frames run in submission order, each from the one before, as xslam_frame runs them; the two calls
 * may be mixed. Returns XSLAM_ESTATE when XSLAM_PIPELINE frames are outstanding (wait for the oldest
 * first), and the errors of xslam_frame's argument checks, before anything is enqueued. xslam_reset
 * finishes and drops the outstanding frames; xslam_destroy finishes them.
 */
xslam_status xslam_frame_submit(xslam_t h, const float* depth, int depth_on_device, const xslam_seed* seeds,
                                int K, long long* ticket);

/*
 * Wait for submitted frame `ticket` and write its outputs (host arrays, each may be NULL; layout as in
 * xslam_frame). Tickets are waited for in submission order: `ticket` must be the oldest outstanding
 * one (XSLAM_EINVAL otherwise). Returns XSLAM_ENOTRACK (outputs filled) if that frame failed to
 * track, XSLAM_ETIMEOUT if a tensor-core wait of the proposal network ran out during it.
 */
xslam_status xslam_frame_wait(xslam_t h, long long ticket, double* pose_out, double* dpose_out,
                              double* dtwist_out);

/*
 * Ray cast the volume (Sec. 4.1, "Ray casting"; Eq. surface_prediction) at pose lanes T (host,
 * (1 + K) x 12 as described above; NULL = the handle's current pose lanes), K = the handle's lane
 * count. Writes device arrays: depth[H W] = Re alpha0 of the vertex (camera z, 0 = no surface),
 * vmap and nmap [(1 + K) x 3 x H x W]: plane (lane * 3 + c) holds component c of lane `lane` of the
 * global-frame vertex / normal (lane 0 real, lane j the raw imaginary part). Any of the three may be
 * NULL. Does not change the model used by the next frame.
 */
xslam_status xslam_raycast(xslam_t h, const double* T, float* depth, float* vmap, float* nmap);

/*
 * Relocalisation loss of a query depth frame and its derivatives with respect to the query pose
 * (Sec. 5.2 with the point-to-plane reading): E(T_q) = mean over pixels of r_u^2 with
 * r_u = ((T_q V_q(u)) - V_g(u)) . N_g(u), where V_g, N_g are ray cast from the volume at T_q itself and
 * V_q = D_q K^-1 u (pixels whose vertex or model is invalid, or that fail the distance gate, are
 * skipped). query_depth is a device pointer (range gated, and bilaterally filtered if the handle's
 * configuration says so). Derivatives are with respect to a left twist xi of T_q (phi then rho).
 * order 1: *loss and grad[6] (Eq. csfd on six lanes, one per twist component). Needs max_lanes >= 6
 *   and a handle with no frame-sequence lanes in use (call between sequences or on a separate handle).
 * order 2: *loss, grad[6] and hess[21], the upper triangle of the Hessian row by row ((0,0), (0,1),
 *   ..., (0,5), (1,1), ...), from the second-order (bicomplex) step of Sec. 3 in truncated arithmetic:
 *   each of the 21 pairs j <= k evaluates the ray-cast refinement and the residual on numbers
 *   a + b e1 + c e2 + d e1 e2 (e1^2 = e2^2 = 0) from T = exp(e1 G_j + e2 G_k) T_q, with the real pose's
 *   ray-cast and gating decisions. Any handle (no lanes needed); the handle's frame state is kept.
 * Any output pointer may be NULL. Errors: XSLAM_EINVAL (NULL input, order not 1 or 2, non-finite T_q).
 */
xslam_status xslam_grad(xslam_t h, const float* query_depth, const double T_q[12], int order, double* loss,
                        double grad[6], double* hess);

/*
 * The loss, gradient and Hessian of xslam_grad order 2 (outputs as there) by the plain FP64 path: Sec. 3's
 * bicomplex step as printed, numbers a + b i1 + c i2 + d i1 i2 with i1^2 = i2^2 = -1 and every product
 * kept, step h = 1e-20 in each of the 21 start poses exp(h i1 G_j + h i2 G_k) T_q, one thread per pixel,
 * and every decision in FP64 (the pixel's own march with the ray cast's sampling rules, the cells of
 * the hit pair and of the gradient samples, the distance gate). The comparison path of the FP32
 * truncated arithmetic; the handle's volume is read and not changed. Any handle.
 * Errors: XSLAM_EINVAL (NULL input, non-finite T_q).
 */
xslam_status xslam_grad_plain64(xslam_t h, const float* query_depth, const double T_q[12], double* loss,
                                double grad[6], double* hess);

/*
 * The paper's relocalisation loss (Sec. 5.2, TSDF-difference reading) of a query depth frame and its
 * derivatives with respect to the query pose: with (F_q, W_q) the handle's volume (F_r, W_r) after the
 * surface update (Sec. 4.1) of the query frame at T_q, E(T_q) = sum over the observed voxels (W_r > 0)
 * of (F_r - F_q)^2, which is the sum over the observed voxels the query updates of
 * ((F_r - F_D) / (W_r + 1))^2. The volume itself is not changed. query_depth is a device pointer [H W]
 * (range gated, and bilaterally filtered if the handle's configuration says so, as a frame's depth is).
 * Derivatives are with respect to a left twist xi of T_q (phi then rho), from the bicomplex step of
 * Sec. 3 in truncated arithmetic with the real pose's update decisions (voxels updated, voxels clamped
 * at F_D = 1, which carry no derivative, and the pixel cells):
 * order 1: *loss and grad[6] (hess gets zeros);
 * order 2: *loss, grad[6] and hess[21], the upper triangle row by row as in xslam_grad.
 * *n_voxels = the number of observed voxels the query updates (the terms of the sum). The FP32 sums are
 * taken in an order that depends on the blocks' scheduling: repeated calls agree to rounding, not bit for
 * bit. Any handle; any output pointer may be NULL.
 * Errors: XSLAM_EINVAL (NULL input, order not 1 or 2, non-finite T_q).
 */
xslam_status xslam_grad_tsdf(xslam_t h, const float* query_depth, const double T_q[12], int order, double* loss,
                             double grad[6], double* hess, long long* n_voxels);

/*
 * The same loss, gradient and full Hessian (outputs as xslam_grad_tsdf order 2) by the plain FP64 path:
 * Sec. 3's bicomplex step as printed, numbers a + b i1 + c i2 + d i1 i2 with i1^2 = i2^2 = -1 and every
 * product kept, step h = 1e-20, the update's decisions taken in FP64. The comparison path of the FP32
 * truncated arithmetic; the handle's volume (FP32) is read and not changed. Errors as xslam_grad_tsdf.
 */
xslam_status xslam_grad_tsdf_plain64(xslam_t h, const float* query_depth, const double T_q[12], double* loss,
                                     double grad[6], double* hess, long long* n_voxels);

/* Copy one plane of the volume to device array out[nx ny nz]: lane 0 = F (unobserved voxels read
 * 1), lane j >= 1 = Im F / h_j of lane j, lane -1 = the weight W. */
xslam_status xslam_read_tsdf(xslam_t h, int lane, float* out);

/* Stage-level entry points (used to test each step alone; same conventions). */

/* Set the lanes from seeds[K] without running a frame (frame counter unchanged). */
xslam_status xslam_set_lanes(xslam_t h, const xslam_seed* seeds, int K);
/* Set the current pose lanes from a host (1 + K) x 12 block. */
xslam_status xslam_set_pose_lanes(xslam_t h, const double* T);
/* Read the current pose lanes into a host (1 + K) x 12 block. */
xslam_status xslam_get_pose_lanes(xslam_t h, double* T);
/* Overwrite one plane of the volume from device array in[nx ny nz] (lane as in xslam_read_tsdf; for
 * lane j >= 1 the values are the raw imaginary parts, not divided by h). Write lane 0 before lane -1:
 * writing the weights marks every voxel with W = 0 as unobserved. */
xslam_status xslam_write_tsdf(xslam_t h, int lane, const float* in);
/* Surface measurement of device depth[H W] (range gate and Gaussian pyramid, Sec. 4.1); level l of
 * the result is copied to device out[(H >> l)(W >> l)] if out is not NULL. */
xslam_status xslam_measure(xslam_t h, const float* depth, int level, float* out);
/* TSDF surface update (Sec. 4.1, "Surface Update") of device depth[H W] at the current pose lanes. */
xslam_status xslam_integrate(xslam_t h, const float* depth);
/* Replace the model maps used by ICP: device depth[H W], vmap and nmap [(1 + K) x 3 x H x W] as
 * written by xslam_raycast, predicted at the pose lanes T_prev (host (1 + K) x 12). */
xslam_status xslam_set_model(xslam_t h, const float* depth, const float* vmap, const float* nmap,
                             const double* T_prev);
/* One ICP normal-equation build (Sec. 4.1, Eq. icp and "icp approx") at pyramid level `level` of the
 * last xslam_measure, at pose lanes Tj (host (1 + K) x 12) against the current model: writes host
 * out[(1 + K) x 27] = per lane the 21 upper-triangle entries of A = sum J J^T (row-major) then the 6
 * entries of sum J r (lane 0 real, lane j raw imaginary), and *n_valid. */
xslam_status xslam_icp_system(xslam_t h, int level, const double* Tj, double* out, int* n_valid);

/* Stage profiling (tracing). Stages of the frame step: */
#define XSLAM_NSTAGE 5
enum { XSLAM_STAGE_PREPARE = 0,   /* range gate, bilateral filter, pyramid     */
       XSLAM_STAGE_ICP = 1,       /* every ICP iteration of the frame          */
       XSLAM_STAGE_INTEGRATE = 2, /* TSDF surface update                       */
       XSLAM_STAGE_RAYCAST = 3,   /* ray cast of the model for the next frame  */
       XSLAM_STAGE_OTHER = 4 };   /* pose-lane seeding and read-out            */
/* enable = 1: later frames run without CUDA graphs and bracket each stage with CUDA events on the
 * handle's stream; totals and the counters restart. enable = 0: stop (totals are kept). */
xslam_status xslam_profile(xslam_t h, int enable);
/* Synchronise and read the totals since profiling was enabled: ms[XSLAM_NSTAGE] device milliseconds
 * per stage, launches[XSLAM_NSTAGE] kernel launches per stage, counters[3] = voxels updated by the
 * TSDF update, pixels with a ray-cast surface, frames. Any pointer may be NULL. */
xslam_status xslam_profile_read(xslam_t h, double* ms, long long* launches, double* counters);

/*
 * ICP normal equations without any allocation. The paper has no counterpart: this is a deployment
 * variant of xslam_icp_system for callers that cannot allocate device memory where they need it (code
 * inside a framework-owned memory pool, real-time loops in which cudaMalloc would synchronise the
 * device, plug-ins that may only use buffers their host hands them). Stateless: every input and output
 * is the caller's; all scratch (block partial sums, block ticket, pose lanes, result) lives in one
 * file-scope device array of about 290 KB that every GPU which loads the library keeps until exit.
 *   depth   device, pyramid level `level` (0..2) of the measured depth: (H >> level) x (W >> level)
 *   K       level-0 intrinsics and size (H, W divisible by 2^level, at least 4 pixels per level)
 *   model   device, level-0 model maps as (1 + 6 (1 + K_lanes)) planes of H x W: depth, vertex lanes,
 *           normal lanes (the layout of xslam_set_model / xslam_raycast)
 *   Tj, T_prev  host (1 + K_lanes) x 12 pose lanes (current estimate; pose the model was cast at)
 *   seeds   the K_lanes seeds (DEPTH seeds on every pixel enter the measured vertices; single-pixel
 *           DEPTH seeds need a handle and are rejected; the per-frame pose kinds take no derivative
 *           from T_prev's lanes or the model's; the others enter only through the pose lanes and the
 *           model); cfg may be NULL (defaults)
 *   out     host (1 + K_lanes) x 27, as in xslam_icp_system; n_valid may be NULL
 *   cuda_stream  the stream the call is ordered on (NULL = legacy default); the call synchronises it
 * Limits: K_lanes <= 15 and at most 160 thread blocks (the grid this library picks on a GB300 is at
 * most one block per SM); larger requests return XSLAM_EINVAL with a message in
 * xslam_last_error(NULL). Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first lookup on a device may load the library's device code, so make
 * the first call on each device before any stream capture. Calls share the
 * array: calls that overlap on the GPU (other streams, other host threads) race; the call clears the
 * scratch it needs cleared (ticket, status) itself. No cudaMalloc, cudaFree or allocating library
 * routine is called.
 */
xslam_status xslam_icp_system_noalloc(const float* depth, int level, const xslam_intrinsics* K, const float* model,
                                      const double* Tj, const double* T_prev, const xslam_seed* seeds, int K_lanes,
                                      const xslam_config* cfg, double* out, int* n_valid, void* cuda_stream);

/* Host utility (no GPU work): out = exp(xi) T for a left twist xi = (phi, rho) (Sec. 4.1, Eq. lie,
 * Eq. rotvector, Eq. rotation_jacobi), with the library's FP64 SE(3) exponential, the formula of the ICP
 * pose update. xi[6], T[12] and out[12] are host arrays (3x4 row-major poses); out may alias T.
 * Returns XSLAM_EINVAL if a pointer is NULL or xi is not finite. */
xslam_status xslam_se3_exp_compose(const double* xi, const double* T, double* out);

/* Description of the last error on this handle; with h = NULL, of the last failed call made without a
 * handle (xslam_create, xslam_icp_system_noalloc). */
const char* xslam_last_error(xslam_t h);

#ifdef __cplusplus
}
#endif
#endif /* XSLAM_H */
