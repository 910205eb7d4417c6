// TSDF surface update (X-SLAM Sec. 4.1, "Surface Update") on 1 + K lanes.
//
// Per voxel p (centre origin + (i + 0.5) voxel): p_c = R^T (p - t) at the frame pose, x = pi(K p_c);
// L(x) = bilinear depth (four valid taps, depth-discontinuity gate); sdf = L(x) - z_c (the paper's
// |K^-1 x|^-1 |t - p| is exactly z_c, read with the sign that makes free space positive); null if
// sdf < -mu; F_D = min(1, sdf / mu); F <- (W F + F_D) / (W + 1); W <- W + 1 (optionally capped).
// Which voxels are updated depends only on the voxel coordinates, the real pose and the depth map,
// so culled voxels cost no volume traffic. Imaginary lanes follow by the tangent rule through the
// same arithmetic (pose lanes through p_c and x, TRUNC lanes through mu, DEPTH lanes through L).
//
// Thread block = 32 x 8 voxel columns, each thread walking 8 voxels along z. A block whose box lies
// entirely behind the camera or beyond one image edge is skipped (exact: the projection of a convex
// set in front of the camera is the hull of its corners' projections).
#include "internal.cuh"

namespace xslam {

constexpr int kBX = 32, kBY = 8, kBZ = 8;

// Update voxel (i, j, k) if the frame observes it; returns whether it did.
__device__ __forceinline__ bool fuse_voxel(const Params& p, const float* __restrict__ D, const float (*sT)[12],
                                           float* __restrict__ F, float* __restrict__ Wt, int i, int j, int k,
                                           size_t n) {
  const size_t v = (size_t)i + (size_t)p.nx * ((size_t)j + (size_t)p.ny * k);
  const float* T = sT[0];
  const float dx = p.ox + (i + 0.5f) * p.voxel - T[3];
  const float dy = p.oy + (j + 0.5f) * p.voxel - T[7];
  const float dz = p.oz + (k + 0.5f) * p.voxel - T[11];
  const float pcx = T[0] * dx + T[4] * dy + T[8] * dz;
  const float pcy = T[1] * dx + T[5] * dy + T[9] * dz;
  const float pcz = T[2] * dx + T[6] * dy + T[10] * dz;
  if (!(pcz > 0.f)) return false;
  const float invz = 1.f / pcz;
  const float qx = pcx * invz, qy = pcy * invz;
  const float x = p.fx * qx + p.cx;
  const float y = p.fy * qy + p.cy;
  if (!(x >= 0.f && x < (float)(p.W - 1) && y >= 0.f && y < (float)(p.H - 1))) return false;
  const int i0 = (int)x, j0 = (int)y;  // x, y >= 0: truncation is floor
  const float a = x - i0, bb = y - j0;
  const float* row0 = D + (size_t)j0 * p.W + i0;
  const float d00 = __ldg(row0), d10 = __ldg(row0 + 1), d01 = __ldg(row0 + p.W), d11 = __ldg(row0 + p.W + 1);
  if (!(d00 > 0.f && d10 > 0.f && d01 > 0.f && d11 > 0.f)) return false;
  if (!(fabsf(d10 - d00) + fabsf(d01 - d00) + fabsf(d11 - d00) < p.disc_gate)) return false;
  const float Lx = (1.f - a) * (1.f - bb) * d00 + a * (1.f - bb) * d10 + (1.f - a) * bb * d01 + a * bb * d11;
  const float sdf = Lx - pcz;
  if (sdf < -p.mu) return false;
  const bool clamp = sdf >= p.mu;
  const float FD = clamp ? 1.f : sdf / p.mu;

  const float w = Wt[v];
  const float w1 = w + 1.f;
  const float inv = 1.f / w1;
  const float Fn = (w * F[v] + FD) / w1;  // an unobserved voxel (w = 0) takes F_D whatever its sentinel value
  F[v] = Fn;
  Wt[v] = (p.w_max > 0.f) ? fminf(w1, p.w_max) : w1;

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
  return true;
}

__global__ void __launch_bounds__(kBX * kBY) k_integrate(Params p, const float* __restrict__ D,
                                                        const double* __restrict__ pose, float* __restrict__ F,
                                                        float* __restrict__ Wt, unsigned long long* __restrict__ stats) {
  pdl_enter();
  __shared__ float sT[kMaxLanes][12];
  __shared__ int s_out[8];
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
    if (all) return;  // nothing in this box can be updated
  }
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const size_t n = vox_count(p);
  int cnt = 0;
  if (i < p.nx && j < p.ny) {
    for (int dk = 0; dk < kBZ; ++dk) {
      const int k = k0 + dk;
      if (k >= p.nz) break;
      cnt += fuse_voxel(p, D, sT, F, Wt, i, j, k, n);
    }
  }
  // updated-voxel count: warp sums, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (threadIdx.x == 0 && cnt) atomicAdd(stats, (unsigned long long)cnt);
}

cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s) {
  dim3 blk(kBX, kBY, 1), grd((p.nx + kBX - 1) / kBX, (p.ny + kBY - 1) / kBY, (p.nz + kBZ - 1) / kBZ);
  const cudaError_t e = launch_pdl(k_integrate, grd, blk, 0, s, p, b.pyr[0], b.pose, b.F, b.Wt, b.stats);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace xslam
