// Internal definitions shared by the CUDA translation units of libxslam (not part of the C ABI).
//
// Lane model (X-SLAM Sec. 3, simplified CSFD arithmetic): a perturbed quantity x* = x + sum_j x_j i_j
// is stored as one real value x and K imaginary values x_j. Products of two imaginary parts are
// dropped (Eq. csfd_simplify_multiplication), so every imaginary part is the directional derivative
// times h_j and is computed by the tangent (first-order) rule from the real values. Discrete
// decisions (gates, floors, zero-crossing tests) use real parts only; the imaginary parts follow the
// chosen branch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xslam {

constexpr int kMaxLanes = 16;        // 1 real + up to 15 imaginary lanes
constexpr int kNT = 27;              // 21 upper-triangle entries of J J^T + 6 of J r
constexpr int kResSys = 12 + 18 * (kMaxLanes - 1);       // offset of the last ICP system in `result`
constexpr int kResLen = kResSys + kNT * kMaxLanes + 8;   // doubles in `result` (+ loss / grad scratch)
constexpr float kUnobserved = 2.f;      // Re F of a voxel with W = 0 (observed values lie in [-1, 1])
// the same in the march's linear copy: a quiet NaN, which every trilinear sample of its cell carries
__host__ __device__ __forceinline__ float unobserved_lin() {
#ifdef __CUDA_ARCH__
  return __int_as_float(0x7fc00000);
#else
  const unsigned u = 0x7fc00000u;
  float f;
  __builtin_memcpy(&f, &u, sizeof(f));
  return f;
#endif
}
constexpr float kCellBias = 0.015625f;  // 2^-6 pixel: ICP bilinear-cell tie breaker (first iteration
                                        // evaluates u_hat on integer pixels by construction)

// Everything a kernel needs besides buffers; passed by value.
struct Params {
  // volume: nx x ny x nz voxels stored in nbx x nby x nbz bricks of 8 x 8 x 8 (vox_index)
  int nx, ny, nz;
  int nbx, nby, nbz;
  float voxel, mu, ox, oy, oz;
  float w_max;              // <= 0: no cap
  // camera (level 0)
  float fx, fy, cx, cy;
  int W, H;
  // lanes: L = 1 + K
  int L;
  float dmu[kMaxLanes];     // Im mu of each lane (TRUNC seeds), lane 0 unused
  float dD[kMaxLanes];      // Im D of each lane (DEPTH seeds on every pixel), lane 0 unused
  int dpix[kMaxLanes];      // single-pixel DEPTH seed: its level-0 pixel (the lane's Im depth maps
                            // Buffers::dlane hold the perturbation at every level); -1 otherwise
  unsigned fresh;           // bit l: lane l restarts at every frame (per-frame pose seeds): its earlier
                            // imaginary parts of the previous pose and the model maps do not enter ICP
  double h[kMaxLanes];      // step of each lane for the read-out
  // gates and ranges
  float dist_gate2, cos_normal_gate, disc_gate, min_corr_frac;
  float depth_min, depth_max, pyr_range;
  int bilateral;            // 1: bilateral filter of the gated raw depth before the pyramid
  float ray_step;           // dalpha in metres of camera depth
  float icp_newton_eta;     // Newton ICP: mean squared residual (m^2) below which the Hessian is used
  float icp_stop;           // > 0: a level ends after a real step |x| below this (twist norm)
  int m0, m1;               // ray samples alpha_m = m * ray_step, m0 <= m <= m1
  float inv_mu;             // 1 / mu (the lanes' tangents multiply by it)
};

// Device buffers owned by a handle.
struct Buffers {
  float* F;         // L planes of vox_plane floats: lane 0 = Re F (kUnobserved where W = 0), lane j = Im F (raw)
  float* Wt;        // one plane
  float* F0lin;     // Re F again, in the linear layout x + nx (y + ny z): the ray-cast march's copy
                    // (unobserved_lin() where W = 0)
  float* depth_in;  // H*W raw input
  float* gated;     // H*W range-gated input (bilateral filter source)
  float* pyr[3];    // range-gated level 0 and its two coarser levels
  float* model;     // (1 + 6 L) planes of H*W: depth_g, V lanes (3 L), N lanes (3 L)
  double* pose;     // L x 12 current pose lanes
  double* pose_prev;// L x 12 pose lanes at which the model was ray cast
  float* partial;   // ICP per-block partial sums: nblk x L x 27
  int* partial_n;   // ICP per-block correspondence counts
  unsigned* ticket; // last-block-done counter
  int* status;      // [0] ICP failed in this frame, [1] frames failed since last sync, [2] last n_valid,
                    // [3] level converged, [4] tensor-core wait timed out
  double* result;   // read-out: 12 (pose) + 12 K (dpose) + 6 K (dtwist) + 27 L (last system)
  unsigned long long* stats;  // kNStat counters (kStat* below); NULL in the allocation-free calls
  int* hit;                   // per pixel: index m of the first sample of the ray-cast hit pair, -1 = none
  int* tiles;                 // fusion: tiles the frame can touch (fuse_tile_count entries at most)
  unsigned* tile_ctr;         // fusion: [0] listed tiles, [1] finished blocks (both 0 between launches),
                              // [2] tiles of the last update (tiles_prev), kept for the restarted lanes
  int* tiles_prev;            // fusion: the tiles of the last update (written when Params::fresh != 0)
  float* dlane;               // single-pixel DEPTH lanes: Im D at levels 0, 1, 2 (dlane_offset), lane l
                              // at (l - 1) dlane_stride; zero outside the seed's windows
};

// Im depth map of lane l (single-pixel DEPTH seed) at pyramid level `level`
__host__ __device__ inline size_t dlane_stride(const Params& p) {
  const size_t hw = (size_t)p.W * p.H;
  return hw + (hw >> 2) + (hw >> 4);
}
__host__ __device__ inline size_t dlane_offset(const Params& p, int lane, int level) {
  const size_t hw = (size_t)p.W * p.H;
  const size_t lo = level == 0 ? 0 : (level == 1 ? hw : hw + (hw >> 2));
  return (size_t)(lane - 1) * dlane_stride(p) + lo;
}

// device counters of a handle (Buffers::stats)
enum : int {
  kStatVoxels = 0,    // voxels updated by fusion
  kStatHits = 1,      // pixels with a ray-cast surface
  kStatIcpIters = 2,  // ICP iterations computed (not skipped after a failure or convergence)
  kStatJudged = 3,    // frames whose learned proposal was judged
  kStatAccepted = 4,  // ... and accepted
  kNStat = 8
};

// Learned proposal and constant-velocity start (proposal.cu), per handle
struct PropBuffers {
  double* pose_pp;   // L x 12: T_{k-2} lanes (the pose before the model's)
  double* candA;     // L x 12: the first ICP run's result while the second runs
  double* candB;     // L x 12: the proposal's start pose
  double* judge;     // [0] J of run A, [1] J of run B
  int* failA;        // run A failed
  double* partial;   // judge: per-block sums (2 per block)
  unsigned* ticket;  // judge: last-block-done counter
  void* row;         // BF16 network input [2 x 4800]: previous frame's features, then the current's
  void* prev;        // BF16 previous frame's features [4800]
  float* y;          // network output (padded to 64)
};

// GEMM launch plan (gemm.cu): K split into `splits` ranges of kb_per_split 64-wide slices
struct GemmPlan {
  int splits = 1, kb_per_split = 1;
};
GemmPlan gemm_plan(int M, int N, int K, int target_ctas);
bool gemm_shape_ok(int M, int N, int K);
cudaError_t gemm_configure();
cudaError_t launch_gemm_bf16(const void* A, const void* B, int M, int N, int K, const GemmPlan& g, float* C, int* err,
                             cudaStream_t s);

__host__ __device__ inline size_t vox_count(const Params& p) {
  return (size_t)p.nx * p.ny * p.nz;
}

// TSDF layout in HBM: bricks of 8 x 8 x 8 voxels, 512 consecutive floats each (x fastest, then y, then
// z inside the brick), bricks in x-fastest order; a plane is padded to whole bricks (padding voxels
// stay unobserved). A fusion tile is one brick (2 KB of one plane, read and written in full lines) and
// a ray-cast cell's 8 corners lie in one brick unless it straddles a brick face.
constexpr int kBrick = 8;
__host__ __device__ inline size_t vox_plane(const Params& p) { return (size_t)p.nbx * p.nby * p.nbz * 512; }

__host__ __device__ inline unsigned vox_index(const Params& p, int i, int j, int k) {
  return ((((unsigned)(k >> 3) * (unsigned)p.nby + (unsigned)(j >> 3)) * (unsigned)p.nbx + (unsigned)(i >> 3)) << 9) +
         ((unsigned)(k & 7) << 6) + ((unsigned)(j & 7) << 3) + (unsigned)(i & 7);
}

// index of voxel (i, j, k) and the offsets to (i + 1, j, k), (i, j + 1, k) and (i, j, k + 1)
struct CellAddr {
  unsigned b, dx, dy, dz;
};
__host__ __device__ inline CellAddr cell_addr(const Params& p, int i, int j, int k) {
  CellAddr c;
  c.b = vox_index(p, i, j, k);
  c.dx = (i & 7) != 7 ? 1u : 512u - 7u;
  c.dy = (j & 7) != 7 ? 8u : (unsigned)p.nbx * 512u - 56u;
  c.dz = (k & 7) != 7 ? 64u : (unsigned)p.nbx * (unsigned)p.nby * 512u - 448u;
  return c;
}

// ---------------------------------------------------------------------------------------------
// Programmatic dependent launch. Every kernel of the frame chain is launched with programmatic stream
// serialization and begins with pdl_enter(): griddepcontrol.wait returns once the preceding kernel in
// the stream has completed and its writes are visible, and launch_dependents then lets the next kernel
// be scheduled, so that its blocks are resident (and past their own launch latency) when this one ends.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// false when the environment sets XSLAM_PDL=0 (plain stream-ordered launches, for comparison)
bool pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------------------------
// Segmented launches (batches of trajectories, batch.cu): one launch runs a kernel over several
// trajectories, each with its own parameters, buffers and grid. Segment i owns the blocks
// [block0, block0 + nblk) of the launch; a block finds its segment by binary search and then works as
// block (blockIdx.x - block0) of a grid of nblk blocks of its trajectory, so every trajectory sees the
// same grid, the same work split and the same per-trajectory tickets as in a launch of its own.
// ---------------------------------------------------------------------------------------------
struct TrajDesc {
  Params p;
  Buffers b;
  const int* kinds;  // lane seed kinds and indices (device)
  const int* index;
};
struct Seg {
  int traj;    // index into the TrajDesc table
  int block0;  // first block of the launch that belongs to this segment
  int nblk;    // the trajectory's grid (1-D) or its blocks along x times along y (2-D kernels)
  int arg;     // per-segment argument: the pyramid level (and flags) or the 2-D grid's width in blocks
};
struct SegTable {
  const TrajDesc* desc;
  const Seg* seg;
  int nseg;
};
__device__ __forceinline__ int seg_find(const SegTable& t, int bx) {
  int lo = 0, hi = t.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.seg[mid].block0 <= bx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------------
// launches (each defined in its own translation unit)
// ---------------------------------------------------------------------------------------------
cudaError_t launch_prepare(const Params& p, const Buffers& b, int levels, cudaStream_t s);
// segmented measurement stage: 0 range gate (segment grids of ceil(W H / 256) blocks), 1 bilateral
// filter, 1 + l pyramid level l (2-D grids of 32 x 8 blocks over the output, arg = width in blocks)
cudaError_t launch_prepare_seg(const SegTable& t, int nblocks, int stage, cudaStream_t s);
cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s);
// The fusion tile list (Buffers::tiles, tile_ctr) of the frame pose `pose` (device, 12 doubles); the
// consumer of the list clears the counters.
cudaError_t launch_fuse_tiles(const Params& p, const Buffers& b, const double* pose, cudaStream_t s);
// The TSDF-difference relocalisation loss of the depth map `depth` fused at `pose`, with its gradient
// and Hessian (order 2) or gradient (order 1) from the 21 truncated-bicomplex poses `poses`: out[29] =
// E, g[6], H[21], updated-voxel count (tsdf_loss.cu).
cudaError_t launch_tsdf_hess(const Params& p, const Buffers& b, const float* depth, const double* pose,
                             const float* poses, int order, double* out, int nblk, cudaStream_t s);
// The same loss, gradient and Hessian in the plain FP64 bicomplex arithmetic (full products, step h
// folded into the 21 start poses `poses`).
cudaError_t launch_tsdf_hess64(const Params& p, const Buffers& b, const float* depth, const double* pose,
                               const double* poses, double h, double* out, int nblk, cudaStream_t s);
int fuse_tile_count(const Params& p);
int fuse_tiles_grid(const Params& p);  // grids of the single-trajectory fusion launches
int integrate_grid(const Params& p);
// segmented fusion launches (every segment's trajectory of L lanes for the update)
cudaError_t launch_fuse_tiles_seg(const SegTable& t, int nblocks, cudaStream_t s);
cudaError_t launch_integrate_seg(const SegTable& t, int nblocks, int L, cudaStream_t s);
cudaError_t launch_raycast(const Params& p, const Buffers& b, const double* pose, float* depth,
                           float* vmap, float* nmap, bool ignore_imag_volume, bool set_prev, cudaStream_t s);
// the frame chain's ray cast (march and refinement into each handle's model) of every segment; blocks of
// tile_w x (256 / tile_w) pixels, segment grids of nblk = ceil(W / tile_w) ceil(H / (256 / tile_w))
// blocks, arg = ceil(W / tile_w)
cudaError_t launch_raycast_seg(const SegTable& t, int nblocks, int tile_w, cudaStream_t s);
// the real march alone: hit[pixel] = first sample of the hit pair, -1 = none
cudaError_t launch_march(const Params& p, const Buffers& b, const double* pose, cudaStream_t s);
// Newton ICP iteration (icp_newton.cu): real pose, lanes unused
cudaError_t launch_icp_newton(const Params& p, const Buffers& b, int level, int flags, int nblk, cudaStream_t s);
int icp_newton_blocks(int level_pixels, int sms);
cudaError_t launch_icp(const Params& p, const Buffers& b, int level, int iter_flags, int nblk, cudaStream_t s);
cudaError_t launch_seed_pose(const Params& p, const Buffers& b, const int* kinds, const int* index, cudaStream_t s);
// Per-frame pose lanes (aux.cu). mode bit 0: restart (zero the lanes of Params::fresh in the pose, the
// previous pose and T_{k-2}); bit 1: ICP's start, lanes of kind POSE = h G_index Re(pose) (and of
// candB, the proposal's start, if not NULL); bit 2: the tracked pose, lanes of kind POSE_TRACKED.
cudaError_t launch_seed_frame(const Params& p, const Buffers& b, double* pose_pp, double* candB, const int* kinds,
                              const int* index, int mode, cudaStream_t s);
// Im depth maps of the single-pixel DEPTH lanes at every level of the pyramid (measure.cu)
cudaError_t launch_depth_lanes(const Params& p, const Buffers& b, int levels, cudaStream_t s);
// zero the restarted lanes' TSDF planes over the tiles of the last update (fuse.cu)
cudaError_t launch_clear_fresh(const Params& p, const Buffers& b, cudaStream_t s);
cudaError_t launch_readout(const Params& p, const Buffers& b, cudaStream_t s);
// segmented: mode 0 frame 0's pose lanes, mode 1 the read-out (a block per segment)
cudaError_t launch_lanes_seg(const SegTable& t, int mode, cudaStream_t s);
// segmented Gauss-Newton iteration: segment arg = level | flags << 4 (fixed counts, no stop tolerance)
cudaError_t launch_icp_seg(const SegTable& t, int nblocks, int max_lanes, cudaStream_t s);
// relocalisation loss, gradient and Hessian (hess.cu); poses: 21 x 12 truncated-bicomplex pose
// elements (4 floats each), out: [E, g(6), H upper (21), count]
cudaError_t launch_hess(const Params& p, const Buffers& b, const float* depth, const float* poses, double* out,
                        int nblk, cudaStream_t s);
// the same loss, gradient and Hessian by the plain FP64 path (full bicomplex products, FP64 march and
// decisions); poses: 21 x 12 bicomplex pose elements (4 doubles each) with the step h folded in
cudaError_t launch_hess64(const Params& p, const Buffers& b, const float* depth, const double* poses, double h,
                          double* out, int nblk, cudaStream_t s);
cudaError_t launch_loss(const Params& p, const Buffers& b, const float* depth, const float* model,
                        const double* pose, double* out, int nblk, cudaStream_t s);
int icp_blocks(int level_pixels, int L);
cudaError_t icp_configure();

// learned proposal / constant-velocity start (proposal.cu)
constexpr int kFeatW = 80, kFeatH = 60, kFeat = kFeatW * kFeatH;
// 80 x 60 block-mean features of n depth frames (frame f at D + f W H) into out + f out_stride (BF16);
// with prev != NULL (n = 1): out[0..kFeat) = prev, out[kFeat..2 kFeat) = the features, prev = the features
cudaError_t launch_features(const float* D, int n, int W, int H, float dmin, float dmax, void* out, size_t out_stride,
                            void* prev, cudaStream_t s);
// start poses: mode bit 0 constant velocity (else T_{k-1}), bit 1 proposal (T_{k-1} exp(scale y)),
// bit 2 frame 0 (only records T_{k-2} := T_0)
cudaError_t launch_prop_seed(const Params& p, const Buffers& b, const PropBuffers& q, const float* scale, int mode,
                             cudaStream_t s);
// judge of the current pose at `level`; phase 0 stores run A and starts run B, phase 1 selects; final:
// phase 1 also closes the frame (fallback to T_{k-1} and failure count)
cudaError_t launch_prop_judge(const Params& p, const Buffers& b, const PropBuffers& q, int level, int phase, int final_,
                              int nblk, cudaStream_t s);

// message of the last failed call made without a handle (returned by xslam_last_error(NULL))
void set_handleless_error(const char* msg);

// ICP iteration flags
enum : int { kIcpFirst = 1, kIcpLast = 2, kIcpNoUpdate = 4 };

}  // namespace xslam
