// C ABI of libxslam (declared in include/xslam.h): handle, device memory, frame driver, stage calls.
//
// The frame step of X-SLAM Sec. 4.1 is a fixed chain of launches on the handle's own stream:
//   frame 0:  range gate -> seed pose lanes -> TSDF update -> ray cast -> read-out
//   frame k:  range gate + pyramid -> ICP iterations (one launch each, coarse to fine) -> TSDF
//             update -> ray cast -> read-out
// Each chain is captured once into a CUDA graph and replayed per frame (kernel arguments only point at
// handle-owned buffers, so a replay needs nothing but the new depth copied into the input buffer).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "../../include/xslam.h"
#include "handle.cuh"
#include "mlp.cuh"
#include "internal.cuh"
#include "se3.cuh"

using namespace xslam;

static std::string g_create_err;

bool xslam::pdl_enabled() {
  static const bool on = [] {
    const char* env = getenv("XSLAM_PDL");
    return !(env && env[0] == '0');
  }();
  return on;
}

void xslam::set_handleless_error(const char* msg) { g_create_err = msg; }

static xslam_status fail(xslam_t h, xslam_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return st;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(h, XSLAM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

extern "C" void xslam_default_config(xslam_config* c) {
  if (!c) return;
  c->icp_levels = 3;
  c->icp_iters[0] = 10;
  c->icp_iters[1] = 5;
  c->icp_iters[2] = 4;
  c->icp_iters[3] = 0;
  c->dist_gate_m = 0.1f;
  c->normal_gate_deg = 20.f;
  c->disc_gate_m = 0.1f;
  c->min_corr_frac = 0.1f;
  c->ray_step_vox = 1.f;
  c->depth_min_m = 0.2f;
  c->depth_max_m = 4.f;
  c->pyr_range_m = 0.09f;
  c->bilateral = 0;
  c->w_max = 0.f;
  c->icp_newton = 0;
  c->icp_newton_eta = 1e-4f;
  c->icp_seed = 0;
  c->icp_stop = 0.f;
}

// the frame pipeline's copy stream, staging buffers, events and pinned output slots (below)
static void pipe_free(xslam_t h);
static xslam_status pipe_alloc(xslam_t h);

static void drop_graphs(xslam_t h) {
  if (h->g_first) cudaGraphExecDestroy(h->g_first);
  if (h->g_track) cudaGraphExecDestroy(h->g_track);
  h->g_first = h->g_track = nullptr;
}

static xslam_status enter(xslam_t h) {
  CU(cudaEventRecord(h->ev_in, h->user));
  CU(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  return XSLAM_OK;
}

static xslam_status leave(xslam_t h) {
  CU(cudaEventRecord(h->ev_out, h->s));
  CU(cudaStreamWaitEvent(h->user, h->ev_out, 0));
  return XSLAM_OK;
}

static int ray_m0(double dmin, double step) { return (int)std::ceil(dmin / step - 1e-4); }
static int ray_m1(double dmax, double step) { return (int)std::floor(dmax / step + 1e-4); }

extern "C" xslam_status xslam_create(xslam_t* out, int nx, int ny, int nz, float voxel_m, float trunc_m,
                                     const float origin_m[3], const xslam_intrinsics* K, const xslam_config* cfg,
                                     int max_lanes, void* cuda_stream) {
  xslam_t h = nullptr;
  if (!out) return fail(h, XSLAM_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2 ||
      (size_t)((nx + 7) / 8) * ((ny + 7) / 8) * ((nz + 7) / 8) * 512 >= ((size_t)1 << 31))
    return fail(h, XSLAM_EINVAL, "volume dimensions must be >= 2 with fewer than 2^31 voxels in whole 8^3 bricks");
  if (!(voxel_m > 0.f) || !(trunc_m > 0.f)) return fail(h, XSLAM_EINVAL, "voxel and truncation must be > 0");
  if (!origin_m || !K) return fail(h, XSLAM_EINVAL, "origin and intrinsics are required");
  if (max_lanes < 0 || max_lanes > kMaxLanes - 1) return fail(h, XSLAM_EINVAL, "max_lanes must be in 0..15");
  xslam_config c;
  if (cfg) c = *cfg;
  else xslam_default_config(&c);
  if (c.icp_levels < 1 || c.icp_levels > 3) return fail(h, XSLAM_EINVAL, "icp_levels must be 1..3");
  for (int l = 0; l < c.icp_levels; ++l)
    if (c.icp_iters[l] < 0 || c.icp_iters[l] > 100) return fail(h, XSLAM_EINVAL, "icp_iters must be 0..100");
  if (c.bilateral != 0 && c.bilateral != 1) return fail(h, XSLAM_EINVAL, "bilateral must be 0 or 1");
  if (c.icp_newton != 0 && c.icp_newton != 1) return fail(h, XSLAM_EINVAL, "icp_newton must be 0 or 1");
  if (c.icp_seed != 0 && c.icp_seed != 1) return fail(h, XSLAM_EINVAL, "icp_seed must be 0 or 1");
  if (!(c.icp_stop >= 0.f) || !std::isfinite(c.icp_stop)) return fail(h, XSLAM_EINVAL, "icp_stop must be >= 0");
  if (c.icp_stop > 0.f && c.icp_newton) return fail(h, XSLAM_EINVAL, "icp_stop applies to Gauss-Newton ICP only");
  const int div = 1 << (c.icp_levels - 1);
  if (K->width < 4 * div || K->height < 4 * div || K->width % div || K->height % div)
    return fail(h, XSLAM_EINVAL, "image size must be divisible by 2^(icp_levels-1) and at least 4 pixels per level");
  if (!(K->fx > 0.f) || !(K->fy > 0.f)) return fail(h, XSLAM_EINVAL, "focal lengths must be > 0");
  if (!(c.depth_max_m > c.depth_min_m) || !(c.depth_min_m >= 0.f) || !(c.ray_step_vox > 0.f))
    return fail(h, XSLAM_EINVAL, "bad depth range or ray step");

  h = new (std::nothrow) xslam_s();
  if (!h) return fail(nullptr, XSLAM_ENOMEM, "host allocation failed");
  h->cfg = c;
  h->max_lanes = max_lanes;
  h->user = (cudaStream_t)cuda_stream;
  const char* env = getenv("XSLAM_GRAPHS");
  h->use_graphs = !(env && env[0] == '0');
  Params& p = h->p;
  memset(&p, 0, sizeof(p));
  p.nx = nx; p.ny = ny; p.nz = nz;
  p.nbx = (nx + kBrick - 1) / kBrick; p.nby = (ny + kBrick - 1) / kBrick; p.nbz = (nz + kBrick - 1) / kBrick;
  p.voxel = voxel_m; p.mu = trunc_m; p.inv_mu = 1.f / trunc_m;
  p.ox = origin_m[0]; p.oy = origin_m[1]; p.oz = origin_m[2];
  p.w_max = c.w_max;
  p.fx = K->fx; p.fy = K->fy; p.cx = K->cx; p.cy = K->cy;
  p.W = K->width; p.H = K->height;
  p.L = 1;
  for (int l = 0; l < kMaxLanes; ++l) p.dpix[l] = -1;
  p.dist_gate2 = c.dist_gate_m * c.dist_gate_m;
  p.cos_normal_gate = (float)std::cos(c.normal_gate_deg * M_PI / 180.0);
  p.disc_gate = c.disc_gate_m;
  p.min_corr_frac = c.min_corr_frac;
  p.depth_min = c.depth_min_m;
  p.depth_max = c.depth_max_m;
  p.pyr_range = c.pyr_range_m;
  p.bilateral = c.bilateral;
  p.icp_newton_eta = c.icp_newton_eta;
  p.icp_stop = c.icp_stop;
  const double step = (double)c.ray_step_vox * (double)voxel_m;
  p.ray_step = (float)step;
  p.m0 = ray_m0(c.depth_min_m, step);
  p.m1 = ray_m1(c.depth_max_m, step);

  auto cleanup = [&](xslam_status st, const std::string& m) {
    xslam_destroy(h);
    return fail(nullptr, st, m);
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cleanup(XSLAM_ECUDA, "no CUDA device");
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (icp_configure() != cudaSuccess) return cleanup(XSLAM_ECUDA, "cannot configure the ICP kernel's shared memory");
  if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(XSLAM_ECUDA, "stream/event creation failed");

  const size_t n = vox_plane(p), hw = (size_t)p.W * p.H;
  const int Lmax = 1 + max_lanes;
  Buffers& b = h->b;
  memset(&b, 0, sizeof(b));
  int nblk_max = 1;
  for (int l = 0; l < 3; ++l) {
    const int np = (p.W >> l) * (p.H >> l);
    h->nblk[l] = icp_blocks(np, Lmax);
    nblk_max = std::max(nblk_max, h->nblk[l]);
  }
  nblk_max = std::max(nblk_max, 4 * h->nsm);  // k_loss grid
  h->nblk_max = nblk_max;
  bool ok = true;
  ok &= cudaMalloc(&b.F, sizeof(float) * n * Lmax) == cudaSuccess;
  ok &= cudaMalloc(&b.Wt, sizeof(float) * n) == cudaSuccess;
  ok &= cudaMalloc(&b.F0lin, sizeof(float) * vox_count(p)) == cudaSuccess;
  ok &= cudaMalloc(&b.depth_in, sizeof(float) * hw) == cudaSuccess;
  ok &= cudaMalloc(&b.gated, sizeof(float) * hw) == cudaSuccess;
  for (int l = 0; l < 3; ++l) ok &= cudaMalloc(&b.pyr[l], sizeof(float) * (hw >> (2 * l))) == cudaSuccess;
  ok &= cudaMalloc(&b.model, sizeof(float) * hw * (1 + 6 * Lmax)) == cudaSuccess;
  ok &= cudaMalloc(&b.pose, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&b.pose_prev, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->pose_tmp, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->hess_poses, sizeof(float) * 21 * 12 * 4) == cudaSuccess;
  ok &= cudaMalloc(&h->hess_poses64, sizeof(double) * 21 * 12 * 4) == cudaSuccess;
  ok &= cudaMalloc(&b.partial, sizeof(float) * (size_t)(nblk_max + 4) * kNT * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&b.partial_n, sizeof(int) * nblk_max) == cudaSuccess;
  ok &= cudaMalloc(&b.ticket, sizeof(unsigned)) == cudaSuccess;
  ok &= cudaMalloc(&b.status, sizeof(int) * 8) == cudaSuccess;
  ok &= cudaMalloc(&b.result, sizeof(double) * kResLen) == cudaSuccess;
  ok &= cudaMalloc(&b.stats, sizeof(unsigned long long) * kNStat) == cudaSuccess;
  h->judge_nblk = std::min(2 * h->nsm, std::max(1, (int)((hw + 255) / 256)));
  ok &= cudaMalloc(&h->q.pose_pp, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->q.candA, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->q.candB, sizeof(double) * 12 * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->q.judge, sizeof(double) * 2) == cudaSuccess;
  ok &= cudaMalloc(&h->q.failA, sizeof(int)) == cudaSuccess;
  ok &= cudaMalloc(&h->q.partial, sizeof(double) * 2 * h->judge_nblk) == cudaSuccess;
  ok &= cudaMalloc(&h->q.ticket, sizeof(unsigned)) == cudaSuccess;
  ok &= cudaMalloc(&b.hit, sizeof(int) * hw) == cudaSuccess;
  ok &= cudaMalloc(&b.tiles, sizeof(int) * (size_t)fuse_tile_count(p)) == cudaSuccess;
  ok &= cudaMalloc(&b.tiles_prev, sizeof(int) * (size_t)fuse_tile_count(p)) == cudaSuccess;
  ok &= cudaMalloc(&b.tile_ctr, sizeof(unsigned) * 4) == cudaSuccess;
  if (max_lanes > 0) ok &= cudaMalloc(&b.dlane, sizeof(float) * dlane_stride(p) * max_lanes) == cudaSuccess;
  ok &= cudaMalloc(&h->d_kinds, sizeof(int) * kMaxLanes) == cudaSuccess;
  ok &= cudaMalloc(&h->d_index, sizeof(int) * kMaxLanes) == cudaSuccess;
  if (max_lanes >= 6) ok &= cudaMalloc(&h->model_q, sizeof(float) * hw * (1 + 6 * 7)) == cudaSuccess;
  ok &= cudaMallocHost(&h->h_result, sizeof(double) * kResLen) == cudaSuccess;
  ok &= cudaMallocHost(&h->h_status, sizeof(int) * 8) == cudaSuccess;
  ok = ok && pipe_alloc(h) == XSLAM_OK;
  if (!ok) return cleanup(XSLAM_ENOMEM, "device or pinned allocation failed");
  *out = h;
  xslam_status st = xslam_reset(h);
  if (st != XSLAM_OK) {
    std::string m = h->err;
    *out = nullptr;
    return cleanup(st, m);
  }
  double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  cudaMemcpyAsync(b.pose, I, sizeof(I), cudaMemcpyHostToDevice, h->s);
  if (cudaStreamSynchronize(h->s) != cudaSuccess) {
    *out = nullptr;
    return cleanup(XSLAM_ECUDA, "initialisation failed");
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_destroy(xslam_t h) {
  if (!h) return XSLAM_OK;
  if (h->s) cudaStreamSynchronize(h->s);
  pipe_free(h);
  drop_graphs(h);
  Buffers& b = h->b;
  cudaFree(b.F); cudaFree(b.Wt); cudaFree(b.F0lin); cudaFree(b.depth_in); cudaFree(b.gated);
  for (int l = 0; l < 3; ++l) cudaFree(b.pyr[l]);
  cudaFree(b.model); cudaFree(b.pose); cudaFree(b.pose_prev); cudaFree(h->pose_tmp); cudaFree(h->hess_poses); cudaFree(h->hess_poses64);
  cudaFree(b.partial); cudaFree(b.partial_n); cudaFree(b.ticket); cudaFree(b.status); cudaFree(b.result); cudaFree(b.stats); cudaFree(b.hit);
  cudaFree(b.tiles); cudaFree(b.tiles_prev); cudaFree(b.tile_ctr); cudaFree(b.dlane);
  cudaFree(h->q.pose_pp); cudaFree(h->q.candA); cudaFree(h->q.candB); cudaFree(h->q.judge); cudaFree(h->q.failA);
  cudaFree(h->q.partial); cudaFree(h->q.ticket); cudaFree(h->q.row); cudaFree(h->q.prev); cudaFree(h->q.y);
  for (int l = 0; l < 8; ++l) cudaFree(h->prop_act[l]);
  cudaFree(h->prop_ws);
  for (int st = 0; st < XSLAM_NSTAGE; ++st)
    for (int i = 0; i < kProfRing; ++i)
      for (int k = 0; k < 2; ++k)
        if (h->pev[st][i][k]) cudaEventDestroy(h->pev[st][i][k]);
  cudaFree(h->d_kinds); cudaFree(h->d_index); cudaFree(h->model_q);
  if (h->h_result) cudaFreeHost(h->h_result);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
  return XSLAM_OK;
}

// volume: F = 1 (all lanes: lane 0 = 1, lanes >= 1 = 0), W = 0
__global__ void k_fill(float* a, size_t n, float v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = v;
}
// plane read-out into the linear layout x + nx (y + ny z): mode 0 = Re F (unobserved voxels read 1, the
// sentinel is internal), 1 = scaled by s (imaginary lanes), 2 = as stored (weights)
__global__ void k_read_plane(Params p, const float* a, float* o, int mode, double s) {
  const size_t n = vox_count(p);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = (int)((i / p.nx) % p.ny), z = (int)(i / ((size_t)p.nx * p.ny));
    const float v = a[vox_index(p, x, y, z)];
    o[i] = mode == 0 ? (v > 1.f ? 1.f : v) : (mode == 1 ? (float)((double)v * s) : v);
  }
}
// plane write from the linear layout
__global__ void k_write_plane(Params p, const float* in, float* a) {
  const size_t n = vox_count(p);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = (int)((i / p.nx) % p.ny), z = (int)(i / ((size_t)p.nx * p.ny));
    a[vox_index(p, x, y, z)] = in[i];
  }
}
// after W is written: voxels with W = 0 are unobserved (the brick plane and the march's linear copy)
__global__ void k_mark_unobserved(float* F, const float* W, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(W[i] > 0.f)) F[i] = kUnobserved;
}
__global__ void k_mark_unobserved_lin(Params p, float* Flin, const float* W) {
  const size_t n = vox_count(p);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % p.nx), y = (int)((i / p.nx) % p.ny), z = (int)(i / ((size_t)p.nx * p.ny));
    if (!(W[vox_index(p, x, y, z)] > 0.f)) Flin[i] = unobserved_lin();
  }
}

extern "C" xslam_status xslam_reset(xslam_t h) {
  if (!h) return XSLAM_EINVAL;
  const size_t n = vox_plane(h->p);
  const int Lmax = 1 + h->max_lanes;
  const unsigned g = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)h->nsm * 32);
  k_fill<<<g, 256, 0, h->s>>>(h->b.F, n, kUnobserved);
  CU(cudaGetLastError());
  k_fill<<<g, 256, 0, h->s>>>(h->b.F0lin, vox_count(h->p), unobserved_lin());
  CU(cudaGetLastError());
  if (Lmax > 1) CU(cudaMemsetAsync(h->b.F + n, 0, sizeof(float) * n * (Lmax - 1), h->s));
  CU(cudaMemsetAsync(h->b.Wt, 0, sizeof(float) * n, h->s));
  CU(cudaMemsetAsync(h->b.model, 0, sizeof(float) * (size_t)h->p.W * h->p.H * (1 + 6 * Lmax), h->s));
  CU(cudaMemsetAsync(h->b.ticket, 0, sizeof(unsigned), h->s));
  CU(cudaMemsetAsync(h->b.partial, 0, sizeof(float) * (size_t)(h->nblk_max + 4) * kNT * kMaxLanes, h->s));
  CU(cudaMemsetAsync(h->b.status, 0, sizeof(int) * 8, h->s));
  CU(cudaMemsetAsync(h->q.pose_pp, 0, sizeof(double) * 12 * kMaxLanes, h->s));
  CU(cudaMemsetAsync(h->q.ticket, 0, sizeof(unsigned), h->s));
  CU(cudaMemsetAsync(h->q.failA, 0, sizeof(int), h->s));
  CU(cudaMemsetAsync(h->b.pose + 12, 0, sizeof(double) * 12 * (kMaxLanes - 1), h->s));
  CU(cudaMemsetAsync(h->b.result, 0, sizeof(double) * kResLen, h->s));
  CU(cudaMemsetAsync(h->b.stats, 0, sizeof(unsigned long long) * kNStat, h->s));
  CU(cudaMemsetAsync(h->b.tile_ctr, 0, sizeof(unsigned) * 4, h->s));
  if (h->b.dlane) CU(cudaMemsetAsync(h->b.dlane, 0, sizeof(float) * dlane_stride(h->p) * h->max_lanes, h->s));
  h->frame = 0;
  h->K = 0;
  h->p.L = 1;
  drop_graphs(h);
  CU(cudaStreamSynchronize(h->s));
  h->t_done = h->t_next;  // frames submitted before the reset are finished and their outputs dropped
  return XSLAM_OK;
}

extern "C" xslam_status xslam_set_pose(xslam_t h, const double* T) {
  if (!h || !T) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (h->frame > 0) return fail(h, XSLAM_ESTATE, "the pose can only be set before the first frame");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T[i])) return fail(h, XSLAM_EINVAL, "pose has a non-finite entry");
  CU(cudaMemcpyAsync(h->b.pose, T, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
  CU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

static bool same_seeds(xslam_t h, const xslam_seed* s, int K) {
  if (K != h->K) return false;
  for (int j = 0; j < K; ++j)
    if (s[j].kind != h->seeds[j].kind || s[j].index != h->seeds[j].index || s[j].h != h->seeds[j].h) return false;
  return true;
}

extern "C" xslam_status xslam_set_lanes(xslam_t h, const xslam_seed* seeds, int K) {
  if (!h) return XSLAM_EINVAL;
  if (K < 0 || K > h->max_lanes) return fail(h, XSLAM_EINVAL, "K must be in 0..max_lanes");
  if (K > 0 && !seeds) return fail(h, XSLAM_EINVAL, "seeds is NULL");
  if (K > 0 && h->cfg.icp_newton) return fail(h, XSLAM_EINVAL, "Newton ICP runs the real pose only (K must be 0)");
  int kinds[kMaxLanes] = {0}, index[kMaxLanes] = {0};
  Params p = h->p;
  p.L = 1 + K;
  p.fresh = 0u;
  for (int l = 0; l < kMaxLanes; ++l) {
    p.dmu[l] = 0.f;
    p.dD[l] = 0.f;
    p.dpix[l] = -1;
    p.h[l] = 1.0;
  }
  for (int j = 0; j < K; ++j) {
    const xslam_seed& s = seeds[j];
    if (!std::isfinite(s.h) || s.h == 0.0 || std::fabs(s.h) > 1e-3 || std::fabs(s.h) < 1e-30)
      return fail(h, XSLAM_EINVAL, "seed h must satisfy 1e-30 <= |h| <= 1e-3");
    switch (s.kind) {
      case XSLAM_SEED_POSE0:
        if (s.index < 0 || s.index > 5) return fail(h, XSLAM_EINVAL, "POSE0 index must be 0..5");
        break;
      case XSLAM_SEED_POSE:
      case XSLAM_SEED_POSE_TRACKED:
        if (s.index < 0 || s.index > 5) return fail(h, XSLAM_EINVAL, "POSE and POSE_TRACKED index must be 0..5");
        p.fresh |= 1u << (j + 1);
        break;
      case XSLAM_SEED_TRUNC:
        p.dmu[j + 1] = (float)s.h;
        break;
      case XSLAM_SEED_DEPTH:
        if (s.index == -1) {
          p.dD[j + 1] = (float)s.h;
        } else if (s.index >= 0 && s.index < p.W * p.H) {
          p.dpix[j + 1] = s.index;
        } else {
          return fail(h, XSLAM_EINVAL, "DEPTH index must be -1 (every pixel) or a pixel 0..W H - 1");
        }
        break;
      default:
        return fail(h, XSLAM_EINVAL, "unknown seed kind");
    }
    kinds[j + 1] = s.kind;
    index[j + 1] = s.index;
    p.h[j + 1] = s.h;
  }
  CU(cudaMemcpyAsync(h->d_kinds, kinds, sizeof(kinds), cudaMemcpyHostToDevice, h->s));
  CU(cudaMemcpyAsync(h->d_index, index, sizeof(index), cudaMemcpyHostToDevice, h->s));
  // the single-pixel lanes' maps are zero outside their windows, which each frame rewrites
  if (h->b.dlane) CU(cudaMemsetAsync(h->b.dlane, 0, sizeof(float) * dlane_stride(p) * h->max_lanes, h->s));
  CU(cudaStreamSynchronize(h->s));
  h->p = p;
  h->K = K;
  for (int j = 0; j < K; ++j) h->seeds[j] = seeds[j];
  drop_graphs(h);
  return XSLAM_OK;
}

static xslam_status copy_depth(xslam_t h, const float* depth, int on_device) {
  const size_t bytes = sizeof(float) * h->p.W * h->p.H;
  CU(cudaMemcpyAsync(h->b.depth_in, depth, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
  return XSLAM_OK;
}

static void stage_begin(xslam_t h, int st) {
  if (h->profiling) cudaEventRecord(h->pev[st][h->pcount[st] % kProfRing][0], h->s);
}
static void stage_end(xslam_t h, int st, int launches) {
  if (!h->profiling) return;
  cudaEventRecord(h->pev[st][h->pcount[st] % kProfRing][1], h->s);
  h->pcount[st] += 1;
  h->plaunch[st] += launches;
}

static bool uses_start(xslam_t h) { return h->cfg.icp_seed == 1 || h->mlp != nullptr; }
static bool has_depth_lanes(xslam_t h) {
  for (int l = 1; l < h->p.L; ++l)
    if (h->p.dpix[l] >= 0) return true;
  return false;
}
static bool has_kind(xslam_t h, int kind) {
  for (int j = 0; j < h->K; ++j)
    if (h->seeds[j].kind == kind) return true;
  return false;
}

static cudaError_t enqueue_first(xslam_t h) {
  cudaError_t e;
  const size_t hw = (size_t)h->p.W * h->p.H;
  stage_begin(h, XSLAM_STAGE_PREPARE);
  if ((e = launch_prepare(h->p, h->b, 1, h->s)) != cudaSuccess) return e;
  const bool dl = has_depth_lanes(h);
  if (dl && (e = launch_depth_lanes(h->p, h->b, 1, h->s)) != cudaSuccess) return e;
  stage_end(h, XSLAM_STAGE_PREPARE, 1 + h->p.bilateral + (dl ? 1 : 0));
  stage_begin(h, XSLAM_STAGE_OTHER);
  if ((e = launch_seed_pose(h->p, h->b, h->d_kinds, h->d_index, h->s)) != cudaSuccess) return e;
  int n_other = 1;
  if (uses_start(h)) {
    if ((e = launch_prop_seed(h->p, h->b, h->q, h->prop_scale, 4, h->s)) != cudaSuccess) return e;
    ++n_other;
  }
  if (h->mlp) {
    if ((e = launch_features(h->b.depth_in, 1, h->p.W, h->p.H, h->p.depth_min, h->p.depth_max, h->q.row, 0, h->q.prev,
                             h->s)) != cudaSuccess)
      return e;
    ++n_other;
  }
  stage_end(h, XSLAM_STAGE_OTHER, n_other);
  stage_begin(h, XSLAM_STAGE_INTEGRATE);
  if ((e = launch_integrate(h->p, h->b, h->s)) != cudaSuccess) return e;
  stage_end(h, XSLAM_STAGE_INTEGRATE, 2 + (h->p.fresh ? 1 : 0));
  stage_begin(h, XSLAM_STAGE_RAYCAST);
  if ((e = launch_raycast(h->p, h->b, h->b.pose, h->b.model, h->b.model + hw, h->b.model + hw * (1 + 3 * h->p.L),
                          false, true, h->s)) != cudaSuccess)
    return e;
  stage_end(h, XSLAM_STAGE_RAYCAST, 2);
  stage_begin(h, XSLAM_STAGE_OTHER);
  e = launch_readout(h->p, h->b, h->s);
  stage_end(h, XSLAM_STAGE_OTHER, 1);
  return e;
}

// ICP iterations of pyramid levels first .. last (first >= last), coarse to fine, on the current pose
// lanes; close = the range's last iteration closes the frame (fallback to T_{k-1}, failure count)
static cudaError_t enqueue_icp_levels(xslam_t h, int first, int last, bool close, int* n_icp) {
  int last_level = -1;
  for (int l = first; l >= last; --l)
    if (h->cfg.icp_iters[l] > 0) last_level = l;
  for (int l = first; l >= last; --l) {
    for (int it = 0; it < h->cfg.icp_iters[l]; ++it) {
      int flags = it == 0 ? kIcpFirst : 0;
      if (close && l == last_level && it == h->cfg.icp_iters[l] - 1) flags |= kIcpLast;
      cudaError_t e;
      if (h->cfg.icp_newton)
        e = launch_icp_newton(h->p, h->b, l, flags, icp_newton_blocks((h->p.W >> l) * (h->p.H >> l), h->nsm), h->s);
      else
        e = launch_icp(h->p, h->b, l, flags, h->nblk[l], h->s);
      if (e != cudaSuccess) return e;
      ++*n_icp;
    }
  }
  return cudaSuccess;
}

static cudaError_t enqueue_track(xslam_t h) {
  cudaError_t e;
  const int levels = h->cfg.icp_levels;
  stage_begin(h, XSLAM_STAGE_PREPARE);
  if ((e = launch_prepare(h->p, h->b, levels, h->s)) != cudaSuccess) return e;
  const bool dl = has_depth_lanes(h);
  if (dl && (e = launch_depth_lanes(h->p, h->b, levels, h->s)) != cudaSuccess) return e;
  stage_end(h, XSLAM_STAGE_PREPARE, levels + h->p.bilateral + (dl ? 1 : 0));
  // per-frame pose lanes restart: the imaginary parts the last frame left in the pose lanes go, and
  // (without a start-pose kernel to follow) ICP's start is perturbed at once
  const bool fresh = h->p.fresh != 0u;
  const bool start_kind = has_kind(h, XSLAM_SEED_POSE);
  if (fresh) {
    stage_begin(h, XSLAM_STAGE_OTHER);
    const int mode = 1 | (uses_start(h) ? 0 : 2);
    if ((e = launch_seed_frame(h->p, h->b, h->q.pose_pp, nullptr, h->d_kinds, h->d_index, mode, h->s)) != cudaSuccess)
      return e;
    stage_end(h, XSLAM_STAGE_OTHER, 1);
  }
  if (uses_start(h)) {
    // the proposal's forward pass and the start poses
    stage_begin(h, XSLAM_STAGE_OTHER);
    int n_other = 1;
    if (h->mlp) {
      if ((e = launch_features(h->b.depth_in, 1, h->p.W, h->p.H, h->p.depth_min, h->p.depth_max, h->q.row, 0,
                               h->q.prev, h->s)) != cudaSuccess)
        return e;
      if ((e = mlp_enqueue_forward(h->mlp, h->q.row, 1, (__nv_bfloat16* const*)h->prop_act, h->prop_ws, h->q.y, 64, 6,
                                   h->b.status + 4, h->s)) != cudaSuccess)
        return e;
      n_other += 1 + 2 * h->mlp->L;
    }
    const int mode = (h->cfg.icp_seed == 1 ? 1 : 0) | (h->mlp ? 2 : 0);
    if ((e = launch_prop_seed(h->p, h->b, h->q, h->prop_scale, mode, h->s)) != cudaSuccess) return e;
    if (fresh && start_kind) {
      if ((e = launch_seed_frame(h->p, h->b, nullptr, h->mlp ? h->q.candB : nullptr, h->d_kinds, h->d_index, 2,
                                 h->s)) != cudaSuccess)
        return e;
      ++n_other;
    }
    stage_end(h, XSLAM_STAGE_OTHER, n_other);
  }
  int n_icp = 0;
  stage_begin(h, XSLAM_STAGE_ICP);
  if (h->mlp) {
    const int J = std::min(h->judge_level, levels - 1);
    for (int run = 0; run < 2; ++run) {
      if ((e = enqueue_icp_levels(h, levels - 1, J, false, &n_icp)) != cudaSuccess) return e;
      if ((e = launch_prop_judge(h->p, h->b, h->q, J, run, run == 1 && J == 0, h->judge_nblk, h->s)) != cudaSuccess)
        return e;
      ++n_icp;
    }
    if (J > 0 && (e = enqueue_icp_levels(h, J - 1, 0, true, &n_icp)) != cudaSuccess) return e;
  } else {
    if ((e = enqueue_icp_levels(h, levels - 1, 0, true, &n_icp)) != cudaSuccess) return e;
  }
  stage_end(h, XSLAM_STAGE_ICP, n_icp);
  if (has_kind(h, XSLAM_SEED_POSE_TRACKED)) {
    // the tracked pose T_{g,k} enters the surface update and the ray cast perturbed
    stage_begin(h, XSLAM_STAGE_OTHER);
    if ((e = launch_seed_frame(h->p, h->b, nullptr, nullptr, h->d_kinds, h->d_index, 4, h->s)) != cudaSuccess) return e;
    stage_end(h, XSLAM_STAGE_OTHER, 1);
  }
  stage_begin(h, XSLAM_STAGE_INTEGRATE);
  if ((e = launch_integrate(h->p, h->b, h->s)) != cudaSuccess) return e;
  stage_end(h, XSLAM_STAGE_INTEGRATE, 2 + (h->p.fresh ? 1 : 0));
  const size_t hw = (size_t)h->p.W * h->p.H;
  stage_begin(h, XSLAM_STAGE_RAYCAST);
  if ((e = launch_raycast(h->p, h->b, h->b.pose, h->b.model, h->b.model + hw, h->b.model + hw * (1 + 3 * h->p.L),
                          false, true, h->s)) != cudaSuccess)
    return e;
  stage_end(h, XSLAM_STAGE_RAYCAST, 2);
  stage_begin(h, XSLAM_STAGE_OTHER);
  e = launch_readout(h->p, h->b, h->s);
  stage_end(h, XSLAM_STAGE_OTHER, 1);
  return e;
}

cudaError_t xslam::enqueue_chain(xslam_t h, bool first) { return first ? enqueue_first(h) : enqueue_track(h); }

void xslam::handle_drop_graphs(xslam_t h) { drop_graphs(h); }

// Fold the recorded event pairs into the per-stage totals (synchronises the stream).
static xslam_status prof_accumulate(xslam_t h) {
  CU(cudaStreamSynchronize(h->s));
  for (int st = 0; st < XSLAM_NSTAGE; ++st) {
    const int n = h->pcount[st] < kProfRing ? h->pcount[st] : kProfRing;
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, h->pev[st][i][0], h->pev[st][i][1]));
      h->pms[st] += ms;
    }
    h->pcount[st] = 0;
  }
  return XSLAM_OK;
}

static xslam_status run_chain(xslam_t h, bool first) {
  cudaGraphExec_t* ge = first ? &h->g_first : &h->g_track;
  if (h->profiling) {
    for (int st = 0; st < XSLAM_NSTAGE; ++st)
      if (h->pcount[st] + 2 > kProfRing) {
        xslam_status s2 = prof_accumulate(h);
        if (s2 != XSLAM_OK) return s2;
        break;
      }
    CU(first ? enqueue_first(h) : enqueue_track(h));
    h->pframes += 1;
    return XSLAM_OK;
  }
  if (!h->use_graphs) {
    CU(first ? enqueue_first(h) : enqueue_track(h));
    return XSLAM_OK;
  }
  if (!*ge) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = first ? enqueue_first(h) : enqueue_track(h);
    cudaError_t e2 = cudaStreamEndCapture(h->s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(h, XSLAM_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(ge, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
      *ge = nullptr;
      return fail(h, XSLAM_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e3));
    }
  }
  CU(cudaGraphLaunch(*ge, h->s));
  return XSLAM_OK;
}

// the read-out block of a finished frame (host copy of `result`): pose, dpose and dtwist of K lanes
static void copy_outputs(const double* res, int K, double* pose_out, double* dpose_out, double* dtwist_out) {
  if (pose_out) memcpy(pose_out, res, sizeof(double) * 12);
  if (dpose_out) memcpy(dpose_out, res + 12, sizeof(double) * 12 * K);
  if (dtwist_out) memcpy(dtwist_out, res + 12 + 12 * (kMaxLanes - 1), sizeof(double) * 6 * K);
}

// the lane checks of a frame call: frame 0 fixes the lanes, later frames must repeat them
static xslam_status frame_lanes(xslam_t h, const xslam_seed* seeds, int K) {
  if (K < 0 || K > h->max_lanes) return fail(h, XSLAM_EINVAL, "K must be in 0..max_lanes");
  if (h->frame == 0) return xslam_set_lanes(h, seeds, K);
  if (!same_seeds(h, seeds, K)) return fail(h, XSLAM_ESTATE, "seeds must not change after the first frame (xslam_reset first)");
  return XSLAM_OK;
}

extern "C" xslam_status xslam_frame(xslam_t h, const float* depth, int depth_on_device, const xslam_seed* seeds, int K,
                                    double* pose_out, double* dpose_out, double* dtwist_out) {
  if (!h) return XSLAM_EINVAL;
  if (!depth) return fail(h, XSLAM_EINVAL, "depth is NULL");
  xslam_status st = frame_lanes(h, seeds, K);
  if (st != XSLAM_OK) return st;
  if ((st = enter(h)) != XSLAM_OK) return st;
  if (st != XSLAM_OK) return st;
  if ((st = copy_depth(h, depth, depth_on_device)) != XSLAM_OK) return st;
  if ((st = run_chain(h, h->frame == 0)) != XSLAM_OK) return st;
  h->frame += 1;
  const bool want = pose_out || dpose_out || dtwist_out;
  if (!want && depth_on_device) return leave(h);
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResSys, cudaMemcpyDeviceToHost, h->s));
  CU(cudaMemcpyAsync(h->h_status, h->b.status, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->s));
  if ((st = leave(h)) != XSLAM_OK) return st;
  CU(cudaStreamSynchronize(h->s));
  if (h->h_status[4]) {
    CU(cudaMemsetAsync(h->b.status + 4, 0, sizeof(int), h->s));
    CU(cudaStreamSynchronize(h->s));
    return fail(h, XSLAM_ETIMEOUT, "a tensor-core wait of the proposal network ran out");
  }
  copy_outputs(h->h_result, h->K, pose_out, dpose_out, dtwist_out);
  if (h->h_status[1] > 0) {
    CU(cudaMemsetAsync(h->b.status + 1, 0, sizeof(int), h->s));
    CU(cudaStreamSynchronize(h->s));
    h->err = "ICP failed to track (too few correspondences or singular normal equations)";
    return XSLAM_ENOTRACK;
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_sync(xslam_t h, int* n_failed) {
  if (!h) return XSLAM_EINVAL;
  CU(cudaMemcpyAsync(h->h_status, h->b.status, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->s));
  CU(cudaMemsetAsync(h->b.status + 1, 0, sizeof(int), h->s));
  CU(cudaMemsetAsync(h->b.status + 4, 0, sizeof(int), h->s));
  CU(cudaStreamSynchronize(h->s));
  if (n_failed) *n_failed = h->h_status[1];
  if (h->h_status[4]) return fail(h, XSLAM_ETIMEOUT, "a tensor-core wait of the proposal network ran out");
  if (h->h_status[1] > 0) {
    h->err = "ICP failed to track on some frames";
    return XSLAM_ENOTRACK;
  }
  return XSLAM_OK;
}

// ---- pipelined frames ----------------------------------------------------------------------------
static void pipe_free(xslam_t h) {
  if (h->cs) {
    cudaStreamSynchronize(h->cs);
    cudaStreamDestroy(h->cs);
    h->cs = nullptr;
  }
  for (int i = 0; i < 2; ++i) {
    if (h->stage[i]) cudaFree(h->stage[i]);
    if (h->ev_h2d[i]) cudaEventDestroy(h->ev_h2d[i]);
    if (h->ev_used[i]) cudaEventDestroy(h->ev_used[i]);
    h->stage[i] = nullptr;
    h->ev_h2d[i] = h->ev_used[i] = nullptr;
  }
  for (int i = 0; i < XSLAM_PIPELINE; ++i) {
    if (h->ev_res[i]) cudaEventDestroy(h->ev_res[i]);
    h->ev_res[i] = nullptr;
  }
  if (h->h_ring) cudaFreeHost(h->h_ring);
  if (h->h_sring) cudaFreeHost(h->h_sring);
  h->h_ring = nullptr;
  h->h_sring = nullptr;
}

// the copy stream, staging buffers, events and pinned output slots of xslam_frame_submit (at create)
static xslam_status pipe_alloc(xslam_t h) {
  const size_t hw = (size_t)h->p.W * h->p.H;
  bool ok = cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 2; ++i) {
    ok = ok && cudaMalloc(&h->stage[i], sizeof(float) * hw) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&h->ev_h2d[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming) == cudaSuccess;
  }
  for (int i = 0; i < XSLAM_PIPELINE; ++i)
    ok = ok && cudaEventCreateWithFlags(&h->ev_res[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMallocHost(&h->h_sring, sizeof(int) * 8 * XSLAM_PIPELINE) == cudaSuccess;
  ok = ok && cudaMallocHost(&h->h_ring, sizeof(double) * kResSys * XSLAM_PIPELINE) == cudaSuccess;
  if (!ok) {
    pipe_free(h);
    return fail(h, XSLAM_ENOMEM, "allocation of the frame pipeline failed");
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_frame_submit(xslam_t h, const float* depth, int depth_on_device, const xslam_seed* seeds,
                                           int K, long long* ticket) {
  if (!h) return XSLAM_EINVAL;
  if (!depth || !ticket) return fail(h, XSLAM_EINVAL, "depth or ticket is NULL");
  if (h->t_next - h->t_done >= XSLAM_PIPELINE)
    return fail(h, XSLAM_ESTATE, "XSLAM_PIPELINE frames are outstanding: wait for the oldest first");
  xslam_status st = frame_lanes(h, seeds, K);
  if (st != XSLAM_OK) return st;
  if ((st = enter(h)) != XSLAM_OK) return st;
  const size_t bytes = sizeof(float) * h->p.W * h->p.H;
  if (depth_on_device) {
    CU(cudaMemcpyAsync(h->b.depth_in, depth, bytes, cudaMemcpyDeviceToDevice, h->s));
  } else {
    // upload on the copy stream while the frames before run; the frame's stream takes it from there
    const int i = h->stage_next;
    h->stage_next ^= 1;
    CU(cudaStreamWaitEvent(h->cs, h->ev_used[i], 0));  // the frame two back has consumed this buffer
    CU(cudaMemcpyAsync(h->stage[i], depth, bytes, cudaMemcpyHostToDevice, h->cs));
    CU(cudaEventRecord(h->ev_h2d[i], h->cs));
    CU(cudaStreamWaitEvent(h->s, h->ev_h2d[i], 0));
    CU(cudaMemcpyAsync(h->b.depth_in, h->stage[i], bytes, cudaMemcpyDeviceToDevice, h->s));
    CU(cudaEventRecord(h->ev_used[i], h->s));
  }
  if ((st = run_chain(h, h->frame == 0)) != XSLAM_OK) return st;
  h->frame += 1;
  // the frame's read-out block and status words to its slot; the failure and timeout words restart
  // at 0 for the next frame, so each slot reports its own frame
  const int slot = (int)(h->t_next % XSLAM_PIPELINE);
  CU(cudaMemcpyAsync(h->h_ring + (size_t)slot * kResSys, h->b.result, sizeof(double) * kResSys,
                     cudaMemcpyDeviceToHost, h->s));
  CU(cudaMemcpyAsync(h->h_sring + 8 * slot, h->b.status, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->s));
  CU(cudaMemsetAsync(h->b.status + 1, 0, sizeof(int), h->s));
  CU(cudaMemsetAsync(h->b.status + 4, 0, sizeof(int), h->s));
  CU(cudaEventRecord(h->ev_res[slot], h->s));
  h->ring_K[slot] = h->K;
  *ticket = h->t_next++;
  return leave(h);
}

extern "C" xslam_status xslam_frame_wait(xslam_t h, long long ticket, double* pose_out, double* dpose_out,
                                         double* dtwist_out) {
  if (!h) return XSLAM_EINVAL;
  if (h->t_done >= h->t_next || ticket != h->t_done)
    return fail(h, XSLAM_EINVAL, "ticket is not the oldest outstanding frame");
  const int slot = (int)(ticket % XSLAM_PIPELINE);
  CU(cudaEventSynchronize(h->ev_res[slot]));
  h->t_done += 1;
  const int* stat = h->h_sring + 8 * slot;
  if (stat[4]) return fail(h, XSLAM_ETIMEOUT, "a tensor-core wait of the proposal network ran out");
  copy_outputs(h->h_ring + (size_t)slot * kResSys, h->ring_K[slot], pose_out, dpose_out, dtwist_out);
  if (stat[1] > 0) {
    h->err = "ICP failed to track (too few correspondences or singular normal equations)";
    return XSLAM_ENOTRACK;
  }
  return XSLAM_OK;
}

static xslam_status upload_pose_lanes(xslam_t h, double* dst, const double* T) {
  const int L = h->p.L;
  for (int i = 0; i < 12 * L; ++i)
    if (!std::isfinite(T[i])) return fail(h, XSLAM_EINVAL, "pose lanes have a non-finite entry");
  CU(cudaMemcpyAsync(dst, T, sizeof(double) * 12 * L, cudaMemcpyHostToDevice, h->s));
  return XSLAM_OK;
}

extern "C" xslam_status xslam_raycast(xslam_t h, const double* T, float* depth, float* vmap, float* nmap) {
  if (!h) return XSLAM_EINVAL;
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  const double* pose = h->b.pose;
  if (T) {
    if ((st = upload_pose_lanes(h, h->pose_tmp, T)) != XSLAM_OK) return st;
    pose = h->pose_tmp;
  }
  CU(launch_raycast(h->p, h->b, pose, depth, vmap, nmap, false, false, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_read_tsdf(xslam_t h, int lane, float* out) {
  if (!h || !out) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (lane < -1 || lane > h->K) return fail(h, XSLAM_EINVAL, "lane must be -1..K");
  const size_t n = vox_count(h->p), np = vox_plane(h->p);
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  const unsigned g = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)h->nsm * 32);
  if (lane == -1)
    k_read_plane<<<g, 256, 0, h->s>>>(h->p, h->b.Wt, out, 2, 1.0);
  else if (lane == 0)
    k_read_plane<<<g, 256, 0, h->s>>>(h->p, h->b.F, out, 0, 1.0);
  else
    k_read_plane<<<g, 256, 0, h->s>>>(h->p, h->b.F + (size_t)lane * np, out, 1, 1.0 / h->p.h[lane]);
  CU(cudaGetLastError());
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_write_tsdf(xslam_t h, int lane, const float* in) {
  if (!h || !in) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (lane < -1 || lane > h->K) return fail(h, XSLAM_EINVAL, "lane must be -1..K");
  const size_t n = vox_count(h->p), np = vox_plane(h->p);
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  float* dst = lane == -1 ? h->b.Wt : h->b.F + (size_t)lane * np;
  const unsigned g = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)h->nsm * 32);
  k_write_plane<<<g, 256, 0, h->s>>>(h->p, in, dst);
  CU(cudaGetLastError());
  if (lane == 0) CU(cudaMemcpyAsync(h->b.F0lin, in, sizeof(float) * n, cudaMemcpyDeviceToDevice, h->s));
  if (lane == -1) {
    const unsigned gp = (unsigned)std::min<size_t>((np + 255) / 256, (size_t)h->nsm * 32);
    k_mark_unobserved<<<gp, 256, 0, h->s>>>(h->b.F, h->b.Wt, np);
    CU(cudaGetLastError());
    k_mark_unobserved_lin<<<g, 256, 0, h->s>>>(h->p, h->b.F0lin, h->b.Wt);
    CU(cudaGetLastError());
  }

  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_set_pose_lanes(xslam_t h, const double* T) {
  if (!h || !T) return fail(h, XSLAM_EINVAL, "NULL argument");
  xslam_status st = upload_pose_lanes(h, h->b.pose, T);
  if (st != XSLAM_OK) return st;
  CU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

extern "C" xslam_status xslam_get_pose_lanes(xslam_t h, double* T) {
  if (!h || !T) return fail(h, XSLAM_EINVAL, "NULL argument");
  CU(cudaMemcpyAsync(T, h->b.pose, sizeof(double) * 12 * h->p.L, cudaMemcpyDeviceToHost, h->s));
  CU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

extern "C" xslam_status xslam_measure(xslam_t h, const float* depth, int level, float* out) {
  if (!h || !depth) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (level < 0 || level >= h->cfg.icp_levels) return fail(h, XSLAM_EINVAL, "level out of range");
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  if ((st = copy_depth(h, depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(h->p, h->b, h->cfg.icp_levels, h->s));
  if (out) {
    const size_t npx = (size_t)(h->p.W >> level) * (h->p.H >> level);
    CU(cudaMemcpyAsync(out, h->b.pyr[level], sizeof(float) * npx, cudaMemcpyDeviceToDevice, h->s));
  }
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_integrate(xslam_t h, const float* depth) {
  if (!h || !depth) return fail(h, XSLAM_EINVAL, "NULL argument");
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  if ((st = copy_depth(h, depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(h->p, h->b, 1, h->s));
  CU(launch_integrate(h->p, h->b, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_set_model(xslam_t h, const float* depth, const float* vmap, const float* nmap,
                                        const double* T_prev) {
  if (!h || !depth || !vmap || !nmap || !T_prev) return fail(h, XSLAM_EINVAL, "NULL argument");
  const size_t hw = (size_t)h->p.W * h->p.H;
  const int L = h->p.L;
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  CU(cudaMemcpyAsync(h->b.model, depth, sizeof(float) * hw, cudaMemcpyDeviceToDevice, h->s));
  CU(cudaMemcpyAsync(h->b.model + hw, vmap, sizeof(float) * hw * 3 * L, cudaMemcpyDeviceToDevice, h->s));
  CU(cudaMemcpyAsync(h->b.model + hw * (1 + 3 * L), nmap, sizeof(float) * hw * 3 * L, cudaMemcpyDeviceToDevice, h->s));
  if ((st = upload_pose_lanes(h, h->b.pose_prev, T_prev)) != XSLAM_OK) return st;
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  return st;
}

extern "C" xslam_status xslam_icp_system(xslam_t h, int level, const double* Tj, double* out, int* n_valid) {
  if (!h || !Tj || !out) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (level < 0 || level >= h->cfg.icp_levels) return fail(h, XSLAM_EINVAL, "level out of range");
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  if ((st = upload_pose_lanes(h, h->b.pose, Tj)) != XSLAM_OK) return st;
  CU(launch_icp(h->p, h->b, level, kIcpNoUpdate, h->nblk[level], h->s));
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
  CU(cudaMemcpyAsync(h->h_status, h->b.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  memcpy(out, h->h_result + kResSys, sizeof(double) * kNT * h->p.L);
  if (n_valid) *n_valid = h->h_status[2];
  return st;
}

// The 21 truncated-bicomplex start poses exp(e1 G_j + e2 G_k) T_q (j <= k) of the order-2 loss:
// (I + e1 G_j + e2 G_k + e1 e2 (G_j G_k + G_k G_j) / 2) T_q, exact with e1^2 = e2^2 = 0; G_j the
// generators of the left twist (phi then rho). Out: [pair][element][a, e1, e2, e1 e2] in R, with the e1
// and e2 parts scaled by the step h and the e1 e2 part by h^2 (h = 1 for the truncated FP32 arithmetic;
// a tiny h for the full bicomplex FP64 path, whose dropped i1^2, i2^2 terms are O(h^2) in the real part).
template <typename R>
static void hess_poses(const double* Tq, R* out, double h = 1.0) {
  double G[6][4][4] = {};
  for (int j = 0; j < 3; ++j) {  // [e_j]x
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    G[j][b][a] = 1.0;
    G[j][a][b] = -1.0;
  }
  for (int j = 3; j < 6; ++j) G[j][j - 3][3] = 1.0;
  double T[4][4] = {};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) T[r][c] = Tq[4 * r + c];
  T[3][3] = 1.0;
  auto mul = [](const double A[4][4], const double B[4][4], double C[4][4]) {
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) s += A[r][k] * B[k][c];
        C[r][c] = s;
      }
  };
  int q = 0;
  for (int j = 0; j < 6; ++j)
    for (int k = j; k < 6; ++k, ++q) {
      double GjT[4][4], GkT[4][4], GjGk[4][4], GkGj[4][4], S[4][4], ST[4][4];
      mul(G[j], T, GjT);
      mul(G[k], T, GkT);
      mul(G[j], G[k], GjGk);
      mul(G[k], G[j], GkGj);
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) S[r][c] = 0.5 * (GjGk[r][c] + GkGj[r][c]);
      mul(S, T, ST);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
          R* o = out + 4 * (12 * q + 4 * r + c);
          o[0] = (R)T[r][c];
          o[1] = (R)(h * GjT[r][c]);
          o[2] = (R)(h * GkT[r][c]);
          o[3] = (R)(h * h * ST[r][c]);
        }
    }
}

extern "C" xslam_status xslam_grad(xslam_t h, const float* query_depth, const double* T_q, int order, double* loss,
                                   double* grad, double* hess) {
  if (!h || !query_depth || !T_q) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (order != 1 && order != 2) return fail(h, XSLAM_EINVAL, "order must be 1 or 2");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_q[i])) return fail(h, XSLAM_EINVAL, "T_q has a non-finite entry");
  if (order == 2) {
    float hp[21 * 12 * 4];
    hess_poses(T_q, hp);
    xslam_status st = enter(h);
    if (st != XSLAM_OK) return st;
    CU(cudaMemcpyAsync(h->hess_poses, hp, sizeof(hp), cudaMemcpyHostToDevice, h->s));
    CU(cudaMemcpyAsync(h->pose_tmp, T_q, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
    if ((st = copy_depth(h, query_depth, 1)) != XSLAM_OK) return st;
    CU(launch_prepare(h->p, h->b, 1, h->s));
    CU(launch_march(h->p, h->b, h->pose_tmp, h->s));
    const int nblk = std::min((int)((size_t)h->p.W * h->p.H + 127) / 128, 4 * h->nsm);
    CU(launch_hess(h->p, h->b, h->b.pyr[0], h->hess_poses, h->b.result + kResSys, nblk, h->s));
    CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
    st = leave(h);
    CU(cudaStreamSynchronize(h->s));
    const double* r = h->h_result + kResSys;
    if (loss) *loss = r[0];
    if (grad)
      for (int j = 0; j < 6; ++j) grad[j] = r[1 + j];
    if (hess)
      for (int q = 0; q < 21; ++q) hess[q] = r[7 + q];
    return st;
  }
  if (h->max_lanes < 6 || !h->model_q) return fail(h, XSLAM_EINVAL, "xslam_grad needs max_lanes >= 6");
  if (h->K != 0) return fail(h, XSLAM_ESTATE, "xslam_grad needs a handle without sequence lanes (reset first)");
  Params p = h->p;
  p.L = 7;
  for (int l = 1; l < 7; ++l) {
    p.dmu[l] = 0.f;
    p.dD[l] = 0.f;
    p.h[l] = 1e-10;
  }
  int kinds[kMaxLanes] = {0}, index[kMaxLanes] = {0};
  for (int l = 1; l < 7; ++l) index[l] = l - 1;
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  CU(cudaMemcpyAsync(h->d_kinds, kinds, sizeof(kinds), cudaMemcpyHostToDevice, h->s));
  CU(cudaMemcpyAsync(h->d_index, index, sizeof(index), cudaMemcpyHostToDevice, h->s));
  CU(cudaMemcpyAsync(h->pose_tmp, T_q, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
  Buffers bq = h->b;
  bq.pose = h->pose_tmp;
  CU(launch_seed_pose(p, bq, h->d_kinds, h->d_index, h->s));
  const size_t hw = (size_t)p.W * p.H;
  CU(launch_raycast(p, bq, h->pose_tmp, h->model_q, h->model_q + hw, h->model_q + hw * (1 + 3 * 7), true, false, h->s));
  if ((st = copy_depth(h, query_depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(p, h->b, 1, h->s));
  CU(launch_loss(p, h->b, h->b.pyr[0], h->model_q, h->pose_tmp, h->b.result + kResSys, 4 * h->nsm, h->s));
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  if (loss) *loss = h->h_result[kResSys];
  if (grad)
    for (int j = 0; j < 6; ++j) grad[j] = h->h_result[kResSys + 1 + j];
  return st;
}

extern "C" xslam_status xslam_grad_plain64(xslam_t h, const float* query_depth, const double* T_q, double* loss,
                                           double* grad, double* hess) {
  if (!h || !query_depth || !T_q) return fail(h, XSLAM_EINVAL, "NULL argument");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_q[i])) return fail(h, XSLAM_EINVAL, "T_q has a non-finite entry");
  const double step = 1e-20;
  double hp[21 * 12 * 4];
  hess_poses(T_q, hp, step);
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  CU(cudaMemcpyAsync(h->hess_poses64, hp, sizeof(hp), cudaMemcpyHostToDevice, h->s));
  if ((st = copy_depth(h, query_depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(h->p, h->b, 1, h->s));
  const int nblk = std::min((int)((size_t)h->p.W * h->p.H + 127) / 128, 4 * h->nsm);
  CU(launch_hess64(h->p, h->b, h->b.pyr[0], h->hess_poses64, step, h->b.result + kResSys, nblk, h->s));
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  const double* r = h->h_result + kResSys;
  if (loss) *loss = r[0];
  if (grad)
    for (int j = 0; j < 6; ++j) grad[j] = r[1 + j];
  if (hess)
    for (int q = 0; q < 21; ++q) hess[q] = r[7 + q];
  return st;
}

extern "C" xslam_status xslam_grad_tsdf(xslam_t h, const float* query_depth, const double* T_q, int order,
                                        double* loss, double* grad, double* hess, long long* n_voxels) {
  if (!h || !query_depth || !T_q) return fail(h, XSLAM_EINVAL, "NULL argument");
  if (order != 1 && order != 2) return fail(h, XSLAM_EINVAL, "order must be 1 or 2");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_q[i])) return fail(h, XSLAM_EINVAL, "T_q has a non-finite entry");
  float hp[21 * 12 * 4];
  hess_poses(T_q, hp);
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  CU(cudaMemcpyAsync(h->hess_poses, hp, sizeof(hp), cudaMemcpyHostToDevice, h->s));
  CU(cudaMemcpyAsync(h->pose_tmp, T_q, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
  if ((st = copy_depth(h, query_depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(h->p, h->b, 1, h->s));
  // two resident blocks per SM take tiles from the list by work stealing
  const int nblk = std::max(1, std::min(fuse_tile_count(h->p), 2 * h->nsm));
  CU(launch_tsdf_hess(h->p, h->b, h->b.pyr[0], h->pose_tmp, h->hess_poses, order, h->b.result + kResSys, nblk,
                      h->s));
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  const double* r = h->h_result + kResSys;
  if (loss) *loss = r[0];
  if (grad)
    for (int j = 0; j < 6; ++j) grad[j] = r[1 + j];
  if (hess)
    for (int q = 0; q < 21; ++q) hess[q] = r[7 + q];
  if (n_voxels) *n_voxels = (long long)r[28];
  return st;
}

extern "C" xslam_status xslam_grad_tsdf_plain64(xslam_t h, const float* query_depth, const double* T_q,
                                                double* loss, double* grad, double* hess, long long* n_voxels) {
  if (!h || !query_depth || !T_q) return fail(h, XSLAM_EINVAL, "NULL argument");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T_q[i])) return fail(h, XSLAM_EINVAL, "T_q has a non-finite entry");
  constexpr double kStep = 1e-20;
  double hp[21 * 12 * 4];
  hess_poses(T_q, hp, kStep);
  xslam_status st = enter(h);
  if (st != XSLAM_OK) return st;
  CU(cudaMemcpyAsync(h->hess_poses64, hp, sizeof(hp), cudaMemcpyHostToDevice, h->s));
  CU(cudaMemcpyAsync(h->pose_tmp, T_q, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
  if ((st = copy_depth(h, query_depth, 1)) != XSLAM_OK) return st;
  CU(launch_prepare(h->p, h->b, 1, h->s));
  const int nblk = std::max(1, std::min(fuse_tile_count(h->p), 4 * h->nsm));
  CU(launch_tsdf_hess64(h->p, h->b, h->b.pyr[0], h->pose_tmp, h->hess_poses64, kStep, h->b.result + kResSys, nblk,
                        h->s));
  CU(cudaMemcpyAsync(h->h_result, h->b.result, sizeof(double) * kResLen, cudaMemcpyDeviceToHost, h->s));
  st = leave(h);
  CU(cudaStreamSynchronize(h->s));
  const double* r = h->h_result + kResSys;
  if (loss) *loss = r[0];
  if (grad)
    for (int j = 0; j < 6; ++j) grad[j] = r[1 + j];
  if (hess)
    for (int q = 0; q < 21; ++q) hess[q] = r[7 + q];
  if (n_voxels) *n_voxels = (long long)r[28];
  return st;
}

extern "C" xslam_status xslam_profile(xslam_t h, int enable) {
  if (!h) return XSLAM_EINVAL;
  if (enable && !h->profiling) {
    for (int st = 0; st < XSLAM_NSTAGE; ++st)
      for (int i = 0; i < kProfRing; ++i)
        for (int k = 0; k < 2; ++k)
          if (!h->pev[st][i][k]) CU(cudaEventCreate(&h->pev[st][i][k]));
    for (int st = 0; st < XSLAM_NSTAGE; ++st) {
      h->pcount[st] = 0;
      h->pms[st] = 0;
      h->plaunch[st] = 0;
    }
    h->pframes = 0;
    CU(cudaMemsetAsync(h->b.stats, 0, sizeof(unsigned long long) * kStatIcpIters, h->s));
  CU(cudaMemsetAsync(h->b.tile_ctr, 0, sizeof(unsigned) * 4, h->s));
  if (h->b.dlane) CU(cudaMemsetAsync(h->b.dlane, 0, sizeof(float) * dlane_stride(h->p) * h->max_lanes, h->s));
  }
  if (!enable && h->profiling) {
    xslam_status st = prof_accumulate(h);
    if (st != XSLAM_OK) return st;
  }
  h->profiling = enable != 0;
  CU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

extern "C" xslam_status xslam_profile_read(xslam_t h, double* ms, long long* launches, double* counters) {
  if (!h) return XSLAM_EINVAL;
  xslam_status st = prof_accumulate(h);
  if (st != XSLAM_OK) return st;
  unsigned long long c[2] = {0, 0};
  CU(cudaMemcpy(c, h->b.stats, sizeof(c), cudaMemcpyDeviceToHost));
  for (int i = 0; i < XSLAM_NSTAGE; ++i) {
    if (ms) ms[i] = h->pms[i];
    if (launches) launches[i] = h->plaunch[i];
  }
  if (counters) {
    counters[0] = (double)c[0];
    counters[1] = (double)c[1];
    counters[2] = (double)h->pframes;
  }
  return XSLAM_OK;
}

extern "C" const char* xslam_last_error(xslam_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

extern "C" xslam_status xslam_set_proposal(xslam_t h, xslam_mlp_t m, const float* scale, int judge_level) {
  if (!h) return XSLAM_EINVAL;
  if (m) {
    if (!scale) return fail(h, XSLAM_EINVAL, "scale is NULL");
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(scale[k])) return fail(h, XSLAM_EINVAL, "scale has a non-finite entry");
    if (m->n[0] != 2 * kFeat || m->n[m->L] != 6)
      return fail(h, XSLAM_EINVAL, "the proposal network must map 9600 inputs to 6 outputs");
    if (h->p.W % kFeatW || h->p.H % kFeatH) return fail(h, XSLAM_EINVAL, "the image size must be a multiple of 80 x 60");
    if (h->cfg.icp_newton) return fail(h, XSLAM_EINVAL, "the proposal needs Gauss-Newton ICP");
    if (judge_level < 0 || judge_level >= h->cfg.icp_levels)
      return fail(h, XSLAM_EINVAL, "judge_level must be 0..icp_levels-1");
  }
  CU(cudaStreamSynchronize(h->s));
  for (int l = 0; l < 8; ++l) {
    cudaFree(h->prop_act[l]);
    h->prop_act[l] = nullptr;
  }
  cudaFree(h->prop_ws);
  cudaFree(h->q.row);
  cudaFree(h->q.prev);
  cudaFree(h->q.y);
  h->prop_ws = nullptr;
  h->q.row = h->q.prev = nullptr;
  h->q.y = nullptr;
  h->mlp = nullptr;
  drop_graphs(h);
  if (!m) return XSLAM_OK;
  bool ok = true;
  for (int l = 1; l < m->L; ++l)
    ok &= cudaMalloc(&h->prop_act[l], sizeof(__nv_bfloat16) * m->np[l]) == cudaSuccess;
  ok &= cudaMalloc(&h->prop_ws, sizeof(float) * std::max<size_t>(16, mlp_ws_floats(m, 1))) == cudaSuccess;
  ok &= cudaMalloc(&h->q.row, sizeof(__nv_bfloat16) * 2 * kFeat) == cudaSuccess;
  ok &= cudaMalloc(&h->q.prev, sizeof(__nv_bfloat16) * kFeat) == cudaSuccess;
  ok &= cudaMalloc(&h->q.y, sizeof(float) * 64) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (int l = 0; l < 8; ++l) {
      cudaFree(h->prop_act[l]);
      h->prop_act[l] = nullptr;
    }
    cudaFree(h->prop_ws);
    cudaFree(h->q.row);
    cudaFree(h->q.prev);
    cudaFree(h->q.y);
    h->prop_ws = nullptr;
    h->q.row = h->q.prev = nullptr;
    h->q.y = nullptr;
    return fail(h, XSLAM_ENOMEM, "proposal buffers");
  }
  CU(cudaMemsetAsync(h->q.row, 0, sizeof(__nv_bfloat16) * 2 * kFeat, h->s));
  CU(cudaMemsetAsync(h->q.prev, 0, sizeof(__nv_bfloat16) * kFeat, h->s));
  CU(cudaMemsetAsync(h->q.y, 0, sizeof(float) * 64, h->s));
  CU(gemm_configure());
  CU(cudaStreamSynchronize(h->s));
  for (int k = 0; k < 6; ++k) h->prop_scale[k] = scale[k];
  h->judge_level = judge_level;
  h->mlp = m;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_counters(xslam_t h, unsigned long long* out, int reset) {
  if (!h) return XSLAM_EINVAL;
  unsigned long long c[kNStat] = {};
  CU(cudaStreamSynchronize(h->s));
  CU(cudaMemcpy(c, h->b.stats, sizeof(c), cudaMemcpyDeviceToHost));
  if (out) {
    out[0] = c[kStatIcpIters];
    out[1] = c[kStatJudged];
    out[2] = c[kStatAccepted];
  }
  if (reset) {
    CU(cudaMemsetAsync(h->b.stats + kStatIcpIters, 0, sizeof(unsigned long long) * 3, h->s));
    CU(cudaStreamSynchronize(h->s));
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_se3_exp_compose(const double* xi, const double* T, double* out) {
  if (!xi || !T || !out) return XSLAM_EINVAL;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(xi[i])) return XSLAM_EINVAL;
  const double zero[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  SeCoef k;
  se3_coef_lane(xi, zero, k);
  double E[12], R[12];
  for (int e = 0; e < 12; ++e) E[e] = se3_exp_element(xi, zero, k, false, e);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) {
      double v = E[4 * r] * T[c] + E[4 * r + 1] * T[4 + c] + E[4 * r + 2] * T[8 + c];
      if (c == 3) v += E[4 * r + 3];
      R[4 * r + c] = v;
    }
  for (int e = 0; e < 12; ++e) out[e] = R[e];
  return XSLAM_OK;
}
