// TSDF surface update (X-SLAM Sec. 4.1, "Surface Update") on 1 + K lanes.
//
// Per voxel p (centre origin + (i + 0.5) voxel): p_c = R^T (p - t) at the frame pose, x = pi(K p_c);
// L(x) = bilinear depth (four valid taps, depth-discontinuity gate); sdf = L(x) - z_c (the paper's
// |K^-1 x|^-1 |t - p| is exactly z_c, read with the sign that makes free space positive); null if
// sdf < -mu; F_D = min(1, sdf / mu); F <- (W F + F_D) / (W + 1); W <- W + 1 (optionally capped).
// Which voxels are updated depends only on the voxel coordinates, the real pose and the depth map,
// so culled voxels cost no volume traffic. Imaginary lanes follow by the tangent rule through the
// same arithmetic (pose lanes through p_c and x, TRUNC lanes through mu, DEPTH lanes through L).
#include "internal.cuh"

namespace xslam {

__device__ __forceinline__ bool fuse_voxel(const Params& p, const float* __restrict__ D, const float (*sT)[12],
                                           float* __restrict__ F, float* __restrict__ Wt, size_t v, size_t n) {
  const int i = (int)(v % p.nx);
  const int j = (int)((v / p.nx) % p.ny);
  const int k = (int)(v / ((size_t)p.nx * p.ny));

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
  const int i0 = (int)floorf(x), j0 = (int)floorf(y);
  const float a = x - i0, bb = y - j0;
  const float* row0 = D + (size_t)j0 * p.W + i0;
  const float d00 = row0[0], d10 = row0[1], d01 = row0[p.W], d11 = row0[p.W + 1];
  if (!(d00 > 0.f && d10 > 0.f && d01 > 0.f && d11 > 0.f)) return false;
  if (!(fabsf(d10 - d00) + fabsf(d01 - d00) + fabsf(d11 - d00) < p.disc_gate)) return false;
  const float Lx = (1.f - a) * (1.f - bb) * d00 + a * (1.f - bb) * d10 + (1.f - a) * bb * d01 + a * bb * d11;
  const float sdf = Lx - pcz;
  if (sdf < -p.mu) return false;
  const bool clamp = sdf >= p.mu;
  const float FD = clamp ? 1.f : sdf / p.mu;

  const float w = Wt[v];
  const float inv = 1.f / (w + 1.f);
  F[v] = (w * F[v] + FD) * inv;
  Wt[v] = (p.w_max > 0.f) ? fminf(w + 1.f, p.w_max) : w + 1.f;

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

__global__ void __launch_bounds__(256) k_integrate(Params p, const float* __restrict__ D,
                                                   const double* __restrict__ pose, float* __restrict__ F,
                                                   float* __restrict__ Wt, unsigned long long* __restrict__ stats) {
  __shared__ float sT[kMaxLanes][12];
  for (int i = threadIdx.x; i < p.L * 12; i += blockDim.x) sT[i / 12][i % 12] = (float)pose[i];
  __syncthreads();
  const size_t n = vox_count(p);
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool upd = v < n && fuse_voxel(p, D, sT, F, Wt, v, n);
  const int c = __syncthreads_count(upd);
  if (threadIdx.x == 0 && c) atomicAdd(stats, (unsigned long long)c);
}

cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s) {
  const size_t n = vox_count(p);
  const unsigned grid = (unsigned)((n + 255) / 256);
  k_integrate<<<grid, 256, 0, s>>>(p, b.pyr[0], b.pose, b.F, b.Wt, b.stats);
  return cudaGetLastError();
}

}  // namespace xslam
