// TSDF surface update (X-SLAM Sec. 4.1, "Surface Update") on 1 + K lanes, and the brick summary the
// ray caster uses to cross free space.
//
// Per voxel p (centre origin + (i + 0.5) voxel): p_c = R^T (p - t) at the frame pose, x = pi(K p_c);
// L(x) = bilinear depth (four valid taps, depth-discontinuity gate); sdf = L(x) - z_c (the paper's
// |K^-1 x|^-1 |t - p| is exactly z_c, read with the sign that makes free space positive); null if
// sdf < -mu; F_D = min(1, sdf / mu); F <- (W F + F_D) / (W + 1); W <- W + 1 (optionally capped).
// Which voxels are updated depends only on the voxel coordinates, the real pose and the depth map,
// so culled voxels cost no volume traffic. Imaginary lanes follow by the tangent rule through the
// same arithmetic (pose lanes through p_c and x, TRUNC lanes through mu, DEPTH lanes through L).
//
// Thread block = 32 x 8 voxel columns, each thread walking 8 voxels along z: the block covers four
// 8^3 bricks. A block whose box lies entirely behind the camera or beyond one image edge is skipped
// (exact: the projection of a convex set in front of the camera is the hull of its corners'
// projections); its voxels and bricks are unchanged. Otherwise, after the update, each brick's flag
// records whether all its voxels hold exactly F = 1 (observed free space) or are all unobserved.
#include "internal.cuh"

namespace xslam {

constexpr int kBX = 32, kBY = 8, kBZ = 8;

// Update voxel (i, j, k) if the frame observes it; returns the (new or unchanged) real TSDF value.
__device__ __forceinline__ float fuse_voxel(const Params& p, const float* __restrict__ D, const float (*sT)[12],
                                            float* __restrict__ F, float* __restrict__ Wt, int i, int j, int k,
                                            size_t n, bool& updated) {
  const size_t v = (size_t)i + (size_t)p.nx * ((size_t)j + (size_t)p.ny * k);
  updated = false;
  const float* T = sT[0];
  const float dx = p.ox + (i + 0.5f) * p.voxel - T[3];
  const float dy = p.oy + (j + 0.5f) * p.voxel - T[7];
  const float dz = p.oz + (k + 0.5f) * p.voxel - T[11];
  const float pcx = T[0] * dx + T[4] * dy + T[8] * dz;
  const float pcy = T[1] * dx + T[5] * dy + T[9] * dz;
  const float pcz = T[2] * dx + T[6] * dy + T[10] * dz;
  if (!(pcz > 0.f)) return F[v];
  const float invz = 1.f / pcz;
  const float qx = pcx * invz, qy = pcy * invz;
  const float x = p.fx * qx + p.cx;
  const float y = p.fy * qy + p.cy;
  if (!(x >= 0.f && x < (float)(p.W - 1) && y >= 0.f && y < (float)(p.H - 1))) return F[v];
  const int i0 = (int)x, j0 = (int)y;  // x, y >= 0: truncation is floor
  const float a = x - i0, bb = y - j0;
  const float* row0 = D + (size_t)j0 * p.W + i0;
  const float d00 = __ldg(row0), d10 = __ldg(row0 + 1), d01 = __ldg(row0 + p.W), d11 = __ldg(row0 + p.W + 1);
  if (!(d00 > 0.f && d10 > 0.f && d01 > 0.f && d11 > 0.f)) return F[v];
  if (!(fabsf(d10 - d00) + fabsf(d01 - d00) + fabsf(d11 - d00) < p.disc_gate)) return F[v];
  const float Lx = (1.f - a) * (1.f - bb) * d00 + a * (1.f - bb) * d10 + (1.f - a) * bb * d01 + a * bb * d11;
  const float sdf = Lx - pcz;
  if (sdf < -p.mu) return F[v];
  const bool clamp = sdf >= p.mu;
  const float FD = clamp ? 1.f : sdf / p.mu;

  const float w = Wt[v];
  const float w1 = w + 1.f;
  const float inv = 1.f / w1;
  const float Fn = (w * F[v] + FD) / w1;  // an unobserved voxel (w = 0) takes F_D whatever its sentinel value
  F[v] = Fn;
  Wt[v] = (p.w_max > 0.f) ? fminf(w1, p.w_max) : w1;
  updated = true;

  // tangents of L with respect to the pixel coordinates
  const float dLda = (1.f - bb) * (d10 - d00) + bb * (d11 - d01);
  const float dLdb = (1.f - a) * (d01 - d00) + a * (d11 - d10);
  for (int l = 1; l < p.L; ++l) {
    const float* Tl = sT[l];
    // p_c' = dR^T (p - t) - R^T dt
    const float ex = Tl[3], ey = Tl[7], ez = Tl[11];
    const float pcx_l = Tl[0] * dx + Tl[4] * dy + Tl[8] * dz - (T[0] * ex + T[4] * ey + T[8] * ez);
    const float pcy_l = Tl[1] * dx + Tl[5] * dy + Tl[9] * dz - (T[1] * ex + T[5] * ey + T[9] * ez);
    const float pcz_l = Tl[2] * dx + Tl[6] * dy + Tl[10] * dz - (T[2] * ex + T[6] * ey + T[10] * ez);
    const float x_l = p.fx * (pcx_l - qx * pcz_l) * invz;
    const float y_l = p.fy * (pcy_l - qy * pcz_l) * invz;
    const float L_l = dLda * x_l + dLdb * y_l + p.dD[l];
    const float sdf_l = L_l - pcz_l;
    const float FD_l = clamp ? 0.f : (sdf_l - FD * p.dmu[l]) / p.mu;
    float* Fl = F + (size_t)l * n + v;
    *Fl = (w * (*Fl) + FD_l) * inv;
  }
  return Fn;
}

// Flags of the four bricks of a block from per-thread (free, empty) over its z voxels.
__device__ __forceinline__ void write_brick_flags(const Params& p, bool fr, bool em, unsigned char* __restrict__ flags,
                                                  int bx0, int by, int bz, unsigned* s_and) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tx < 4 && ty == 0) s_and[tx] = 3u;
  __syncthreads();
  const unsigned fb = __ballot_sync(0xffffffffu, fr), eb = __ballot_sync(0xffffffffu, em);
  if (tx == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned mq = 0xffu << (8 * q);
      if ((fb & mq) != mq) atomicAnd(&s_and[q], ~1u);
      if ((eb & mq) != mq) atomicAnd(&s_and[q], ~2u);
    }
  }
  __syncthreads();
  if (tx < 4 && ty == 0) {
    const int bx = bx0 + tx;
    if (bx < p.bnx)
      flags[(size_t)bx + (size_t)p.bnx * ((size_t)by + (size_t)p.bny * bz)] = (unsigned char)(s_and[tx] & 3u);
  }
}

__global__ void __launch_bounds__(kBX * kBY) k_integrate(Params p, const float* __restrict__ D,
                                                        const double* __restrict__ pose, float* __restrict__ F,
                                                        float* __restrict__ Wt, unsigned char* __restrict__ flags,
                                                        unsigned long long* __restrict__ stats) {
  __shared__ float sT[kMaxLanes][12];
  __shared__ int s_out[8];
  __shared__ unsigned s_and[4];
  const int tid = threadIdx.x + kBX * threadIdx.y;
  for (int i = tid; i < p.L * 12; i += kBX * kBY) sT[i / 12][i % 12] = (float)pose[i];
  __syncthreads();
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY, k0 = blockIdx.z * kBZ;
  if (tid < 8) {
    // corner of the block's box (padded by half a voxel around the voxel centres)
    const float* T = sT[0];
    const float cx = p.ox + ((tid & 1) ? min(i0 + kBX, p.nx) : i0) * p.voxel;
    const float cy = p.oy + ((tid & 2) ? min(j0 + kBY, p.ny) : j0) * p.voxel;
    const float cz = p.oz + ((tid & 4) ? min(k0 + kBZ, p.nz) : k0) * p.voxel;
    const float dx = cx - T[3], dy = cy - T[7], dz = cz - T[11];
    const float px = T[0] * dx + T[4] * dy + T[8] * dz;
    const float py = T[1] * dx + T[5] * dy + T[9] * dz;
    const float pz = T[2] * dx + T[6] * dy + T[10] * dz;
    int code;  // bit 0: behind, 1: left, 2: right, 3: above, 4: below
    if (!(pz > 0.f)) {
      code = 1;  // a corner behind the camera only agrees with "behind"
    } else {
      const float x = p.fx * px / pz + p.cx, y = p.fy * py / pz + p.cy;
      code = (x < 0.f ? 2 : 0) | (x >= (float)(p.W - 1) ? 4 : 0) | (y < 0.f ? 8 : 0) | (y >= (float)(p.H - 1) ? 16 : 0);
    }
    s_out[tid] = code;
  }
  __syncthreads();
  {
    int all = 31;
#pragma unroll
    for (int c = 0; c < 8; ++c) all &= s_out[c];
    if (all) return;  // nothing in this box can be updated: voxels and brick flags unchanged
  }
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const size_t n = vox_count(p);
  bool fr = true, em = true;
  int cnt = 0;
  if (i < p.nx && j < p.ny) {
    for (int dk = 0; dk < kBZ; ++dk) {
      const int k = k0 + dk;
      if (k >= p.nz) break;
      bool upd;
      const float f = fuse_voxel(p, D, sT, F, Wt, i, j, k, n, upd);
      cnt += upd;
      fr = fr && f == 1.f;
      em = em && f == kUnobserved;
    }
  }
  write_brick_flags(p, fr, em, flags, blockIdx.x * (kBX / 8), blockIdx.y, blockIdx.z, s_and);
  // updated-voxel count: warp sums, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (threadIdx.x == 0 && cnt) atomicAdd(stats, (unsigned long long)cnt);
}

// Flags of every brick from the volume as it stands (after the volume is written directly).
__global__ void __launch_bounds__(kBX * kBY) k_brick_flags(Params p, const float* __restrict__ F,
                                                          unsigned char* __restrict__ flags) {
  __shared__ unsigned s_and[4];
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k0 = blockIdx.z * kBZ;
  bool fr = true, em = true;
  if (i < p.nx && j < p.ny) {
    for (int dk = 0; dk < kBZ; ++dk) {
      const int k = k0 + dk;
      if (k >= p.nz) break;
      const float f = F[(size_t)i + (size_t)p.nx * ((size_t)j + (size_t)p.ny * k)];
      fr = fr && f == 1.f;
      em = em && f == kUnobserved;
    }
  }
  write_brick_flags(p, fr, em, flags, blockIdx.x * (kBX / 8), blockIdx.y, blockIdx.z, s_and);
}

cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s) {
  dim3 blk(kBX, kBY, 1), grd((p.nx + kBX - 1) / kBX, (p.ny + kBY - 1) / kBY, (p.nz + kBZ - 1) / kBZ);
  k_integrate<<<grd, blk, 0, s>>>(p, b.pyr[0], b.pose, b.F, b.Wt, b.bricks, b.stats);
  return cudaGetLastError();
}

cudaError_t launch_brick_flags(const Params& p, const Buffers& b, cudaStream_t s) {
  dim3 blk(kBX, kBY, 1), grd((p.nx + kBX - 1) / kBX, (p.ny + kBY - 1) / kBY, (p.nz + kBZ - 1) / kBZ);
  k_brick_flags<<<grd, blk, 0, s>>>(p, b.F, b.bricks);
  return cudaGetLastError();
}

}  // namespace xslam
