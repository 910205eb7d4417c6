// xslam_icp_system_noalloc: the ICP normal-equation build without any allocation.
//
// Some callers cannot allocate device memory at the point where they need this computation: code that
// runs inside a framework-owned memory pool or arena that forbids foreign cudaMalloc, real-time loops
// where cudaMalloc/cudaFree would synchronise the device and break the frame budget, and plug-ins that
// may only touch buffers their host hands them. For them this entry point keeps every scratch buffer
// (per-block partial sums, the block ticket, the pose lanes and the result) in one file-scope
// __device__ array, so the call needs only the caller's inputs and outputs.
//
// The array has a fixed size (kNoAllocBytes below) and is shared by every call on a device: calls
// that overlap on the GPU race on it. Each call clears what must start at zero (ticket, status).
#include <cmath>
#include <cstring>

#include "../../include/xslam.h"
#include "internal.cuh"

using namespace xslam;

namespace {

constexpr int kNoAllocMaxBlocks = 160;  // grid bound: at least the number of SMs of a GB300 (152)
constexpr size_t kPartialFloats = (size_t)kNT * kMaxLanes * (kNoAllocMaxBlocks + 4);
constexpr size_t kOffPartial = 0;
constexpr size_t kOffPartialN = kOffPartial + sizeof(float) * kPartialFloats;
constexpr size_t kOffTicket = kOffPartialN + sizeof(int) * kNoAllocMaxBlocks;
constexpr size_t kOffStatus = kOffTicket + 256;
constexpr size_t kOffPose = kOffStatus + 256;
constexpr size_t kOffPosePrev = kOffPose + sizeof(double) * 12 * kMaxLanes;
constexpr size_t kOffResult = kOffPosePrev + sizeof(double) * 12 * kMaxLanes;
constexpr size_t kNoAllocBytes = kOffResult + sizeof(double) * kResLen;  // ~290 KB

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array on the current device. Host code cannot use the symbol itself (in host
// code it names a host-side stand-in), so every call looks the address up with the current device's
// context current: a cached address would go stale once cudaDeviceReset rebuilds the context, and the
// lookup after the first (which may load the module) is a host-side table read.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

xslam_status fail(xslam_status st, const char* msg) {
  set_handleless_error(msg);  // readable through xslam_last_error(NULL)
  return st;
}

}  // namespace

extern "C" xslam_status xslam_icp_system_noalloc(const float* depth, int level, const xslam_intrinsics* K,
                                                 const float* model, const double* Tj, const double* T_prev,
                                                 const xslam_seed* seeds, int K_lanes, const xslam_config* cfg,
                                                 double* out, int* n_valid, void* cuda_stream) {
  if (!depth || !K || !model || !Tj || !T_prev || !out) return fail(XSLAM_EINVAL, "NULL argument");
  if (level < 0 || level > 2) return fail(XSLAM_EINVAL, "level must be 0, 1 or 2");
  if (K_lanes < 0 || K_lanes > kMaxLanes - 1) return fail(XSLAM_EINVAL, "K must be in 0..15");
  if (K_lanes > 0 && !seeds) return fail(XSLAM_EINVAL, "seeds is NULL");
  const int s = 1 << level;
  if (K->width < 4 * s || K->height < 4 * s || K->width % s || K->height % s)
    return fail(XSLAM_EINVAL, "image size must be divisible by 2^level and at least 4 pixels per level");
  xslam_config c;
  if (cfg) c = *cfg;
  else xslam_default_config(&c);

  Params p;
  memset(&p, 0, sizeof(p));
  p.fx = K->fx;
  p.fy = K->fy;
  p.cx = K->cx;
  p.cy = K->cy;
  p.W = K->width;
  p.H = K->height;
  p.L = 1 + K_lanes;
  for (int l = 0; l < kMaxLanes; ++l) {
    p.h[l] = 1.0;
    p.dpix[l] = -1;
  }
  for (int j = 0; j < K_lanes; ++j) {
    if (seeds[j].kind == XSLAM_SEED_DEPTH) {
      if (seeds[j].index != -1)
        return fail(XSLAM_EINVAL, "single-pixel DEPTH seeds need a handle (xslam_icp_system); index must be -1 here");
      p.dD[j + 1] = (float)seeds[j].h;
    }
    if (seeds[j].kind == XSLAM_SEED_POSE || seeds[j].kind == XSLAM_SEED_POSE_TRACKED) p.fresh |= 1u << (j + 1);
    p.h[j + 1] = seeds[j].h;
  }
  p.dist_gate2 = c.dist_gate_m * c.dist_gate_m;
  p.cos_normal_gate = (float)std::cos(c.normal_gate_deg * 3.14159265358979323846 / 180.0);
  p.disc_gate = c.disc_gate_m;
  p.min_corr_frac = c.min_corr_frac;

  const int nblk = icp_blocks((p.W >> level) * (p.H >> level), p.L);
  if (nblk > kNoAllocMaxBlocks) return fail(XSLAM_EINVAL, "grid larger than the scratch array allows");

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(XSLAM_ECUDA, cudaGetErrorString(e));
  unsigned char* sc = (unsigned char*)base;
  Buffers b;
  memset(&b, 0, sizeof(b));
  b.pyr[0] = b.pyr[1] = b.pyr[2] = const_cast<float*>(depth);
  b.model = const_cast<float*>(model);
  b.partial = (float*)(sc + kOffPartial);
  b.partial_n = (int*)(sc + kOffPartialN);
  b.ticket = (unsigned*)(sc + kOffTicket);
  b.status = (int*)(sc + kOffStatus);
  b.pose = (double*)(sc + kOffPose);
  b.pose_prev = (double*)(sc + kOffPosePrev);
  b.result = (double*)(sc + kOffResult);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t pose_bytes = sizeof(double) * 12 * p.L;
  if ((e = cudaMemsetAsync(b.ticket, 0, sizeof(unsigned), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.status, 0, sizeof(int) * 4, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b.pose, Tj, pose_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b.pose_prev, T_prev, pose_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = icp_configure()) != cudaSuccess || (e = launch_icp(p, b, level, kIcpNoUpdate, nblk, st)) != cudaSuccess)
    return fail(XSLAM_ECUDA, cudaGetErrorString(e));
  int nv = 0;
  if ((e = cudaMemcpyAsync(out, b.result + kResSys, sizeof(double) * kNT * p.L, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(&nv, b.status + 2, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(XSLAM_ECUDA, cudaGetErrorString(e));
  if (n_valid) *n_valid = nv;
  return XSLAM_OK;
}
