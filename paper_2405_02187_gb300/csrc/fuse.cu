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
// The volume is cut into 8 x 8 x 8 tiles, the bricks of the TSDF layout. A first kernel lists the
// tiles the frame can touch (a tile whose box lies entirely behind the camera or beyond one image edge
// cannot: exact, as the projection of a convex set in front of the camera is the hull of its corners'
// projections); a fixed grid then walks the list, a block per tile and a thread per voxel, so each
// tile is 2 KB of every plane read and written in full lines (small tiles: at 640x480 in a 256^3 room
// an 8^3 tile list holds about twice the updated voxels, a 32 x 8 x 8 one nearly four times). The
// update kernel is instantiated for each lane count, so every lane of a voxel is loaded before any is
// stored (one memory round trip per voxel rather than one per lane).
#include <algorithm>

#include "internal.cuh"

namespace xslam {

constexpr int kBX = 8, kBY = 8, kBZ = 8;  // tile of voxels: one brick of the TSDF layout
constexpr int kFuseThreads = kBX * kBY * kBZ;  // a thread per voxel of a tile

// Update voxel (i, j, k) if the frame observes it; returns whether it did. NL = 1 + K lanes.
template <int NL>
__device__ __forceinline__ bool fuse_voxel(const Params& p, const float* __restrict__ D, const float (*sT)[12],
                                           const float (*sC)[3],
                                           float* __restrict__ F, float* __restrict__ Wt,
                                           float* __restrict__ F0lin, int i, int j, int k, size_t n, size_t v) {
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

  // every lane of the voxel is loaded before any is stored: the loads then leave together (one
  // memory round trip per voxel) instead of one round trip per lane behind each store to F
  const float w = Wt[v];
  const float f0 = F[v];
  float fl[NL];
#pragma unroll
  for (int l = 1; l < NL; ++l) fl[l] = F[(size_t)l * n + v];
  const float w1 = w + 1.f;
  const float inv = 1.f / w1;
  const float Fn = (w * f0 + FD) / w1;  // an unobserved voxel (w = 0) takes F_D whatever its sentinel value
  F[v] = Fn;
  F0lin[(size_t)i + (size_t)p.nx * ((size_t)j + (size_t)p.ny * k)] = Fn;
  Wt[v] = (p.w_max > 0.f) ? fminf(w1, p.w_max) : w1;

  if (clamp) {  // F_D = 1 whatever the lane: no tangent
#pragma unroll
    for (int l = 1; l < NL; ++l) F[(size_t)l * n + v] = w * fl[l] * inv;
    return true;
  }
  // The tangent of sdf = L(x) - z_c is linear in the lane's p_c': with x' = fx (p_cx' - q_x p_cz') / z,
  // y' = fy (p_cy' - q_y p_cz') / z and the bilinear L's slopes dL/da, dL/db,
  // sdf' = c_x p_cx' + c_y p_cy' + c_z p_cz' + D', c_x = dL/da fx / z, c_y = dL/db fy / z,
  // c_z = -(c_x q_x + c_y q_y) - 1.
  const float dLda = (1.f - bb) * (d10 - d00) + bb * (d11 - d01);
  const float dLdb = (1.f - a) * (d01 - d00) + a * (d11 - d10);
  const float c_x = dLda * p.fx * invz, c_y = dLdb * p.fy * invz;
  const float c_z = -(c_x * qx + c_y * qy) - 1.f;
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    const float* Tl = sT[l];
    // p_c' = dR^T (p - t) - R^T dt, the second term a per-lane constant
    const float pcx_l = Tl[0] * dx + Tl[4] * dy + Tl[8] * dz + sC[l][0];
    const float pcy_l = Tl[1] * dx + Tl[5] * dy + Tl[9] * dz + sC[l][1];
    const float pcz_l = Tl[2] * dx + Tl[6] * dy + Tl[10] * dz + sC[l][2];
    const float sdf_l = c_x * pcx_l + c_y * pcy_l + c_z * pcz_l + p.dD[l];
    const float FD_l = (sdf_l - FD * p.dmu[l]) * p.inv_mu;
    F[(size_t)l * n + v] = (w * fl[l] + FD_l) * inv;
  }
  return true;
}

// One thread per 8 x 8 x 8 tile: a tile any of whose voxels the frame can update is appended to the
// list (warp-aggregated atomics). The test is the exact corner test: the tile's box (padded by half a
// voxel around the voxel centres) is skipped if all 8 corners lie behind the camera or beyond the
// same image edge.
__global__ void __launch_bounds__(256) k_fuse_tiles(Params p, const double* __restrict__ pose, int* __restrict__ tiles,
                                                   unsigned* __restrict__ ctr) {
  pdl_enter();
  const int ntx = (p.nx + kBX - 1) / kBX, nty = (p.ny + kBY - 1) / kBY, ntz = (p.nz + kBZ - 1) / kBZ;
  const int nt = ntx * nty * ntz;
  float T[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T[e] = (float)pose[e];
  for (int t0 = blockIdx.x * blockDim.x; t0 < nt; t0 += gridDim.x * blockDim.x) {
    const int t = t0 + threadIdx.x;
    bool keep = false;
    if (t < nt) {
      const int i0 = (t % ntx) * kBX, j0 = ((t / ntx) % nty) * kBY, k0 = (t / (ntx * nty)) * kBZ;
      int all = 31;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float cx = p.ox + ((c & 1) ? min(i0 + kBX, p.nx) : i0) * p.voxel;
        const float cy = p.oy + ((c & 2) ? min(j0 + kBY, p.ny) : j0) * p.voxel;
        const float cz = p.oz + ((c & 4) ? min(k0 + kBZ, p.nz) : k0) * p.voxel;
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
        all &= code;
      }
      keep = all == 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m) {
      const int lane = threadIdx.x & 31;
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(ctr, (unsigned)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) tiles[base + __popc(m & ((1u << lane) - 1u))] = t;
    }
  }
}

// Fixed grid over the tile list; a block takes one tile at a time, a thread per voxel: thread t of the
// block is the brick's voxel t (x = t mod 8, y = t / 8 mod 8, z = t / 64), so a warp reads and writes
// 128 consecutive bytes of every plane. The last block to finish clears the list counters for the next
// launch.
template <int NL>
__global__ void __launch_bounds__(kFuseThreads, NL <= 9 ? 2 : 1) k_integrate(Params p, const float* __restrict__ D,
                                                        const double* __restrict__ pose, float* __restrict__ F,
                                                        float* __restrict__ Wt, float* __restrict__ F0lin,
                                                        unsigned long long* __restrict__ stats,
                                                        const int* __restrict__ tiles, unsigned* __restrict__ ctr) {
  pdl_enter();
  __shared__ float sT[NL][12];
  __shared__ float sC[NL][3];  // -R^T dt of each lane: the voxel-independent part of its p_c tangent
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  for (int i = tid; i < NL * 12; i += blockDim.x) sT[i / 12][i % 12] = (float)pose[i];
  if (tid < NL * 3) {
    const int l = tid / 3, c = tid % 3;
    sC[l][c] = -((float)pose[c] * (float)pose[12 * l + 3] + (float)pose[4 + c] * (float)pose[12 * l + 7] +
                 (float)pose[8 + c] * (float)pose[12 * l + 11]);
  }
  __syncthreads();
  const unsigned count = ctr[0];
  const int ntx = (p.nx + kBX - 1) / kBX, nty = (p.ny + kBY - 1) / kBY;
  const size_t n = vox_plane(p);
  const int cx = tid & 7, cy = (tid >> 3) & 7, cz = tid >> 6;
  int cnt = 0;
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const int t = tiles[q];
    const int i = (t % ntx) * kBX + cx, j = ((t / ntx) % nty) * kBY + cy, k = (t / (ntx * nty)) * kBZ + cz;
    // the tile is brick t, whose voxel tid sits at t 512 + tid
    if (i < p.nx && j < p.ny && k < p.nz)
      cnt += fuse_voxel<NL>(p, D, sT, sC, F, Wt, F0lin, i, j, k, n, ((size_t)t << 9) + tid);
  }
  // updated-voxel count: warp sums, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((tid & 31) == 0 && cnt) atomicAdd(stats, (unsigned long long)cnt);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(ctr + 1, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && tid == 0) {
    ctr[0] = 0u;
    ctr[1] = 0u;
  }
}

template <int NL>
static cudaError_t launch_integrate_nl(const Params& p, const Buffers& b, int grid, cudaStream_t s) {
  return launch_pdl(k_integrate<NL>, dim3(grid), dim3(kFuseThreads), 0, s, p, b.pyr[0], b.pose, b.F, b.Wt, b.F0lin,
                    b.stats, b.tiles, b.tile_ctr);
}

int fuse_tile_count(const Params& p) {
  return ((p.nx + kBX - 1) / kBX) * ((p.ny + kBY - 1) / kBY) * ((p.nz + kBZ - 1) / kBZ);
}

cudaError_t launch_fuse_tiles(const Params& p, const Buffers& b, const double* pose, cudaStream_t s) {
  int dev = 0, sms = 0;  // the current device's SM count (queried per call: a handle may live on any device)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nt = fuse_tile_count(p);
  return launch_pdl(k_fuse_tiles, dim3(std::min((nt + 255) / 256, 4 * sms)), dim3(256), 0, s, p, pose, b.tiles,
                    b.tile_ctr);
}

cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s) {
  int dev = 0, sms = 0;  // the current device's SM count (queried per call: a handle may live on any device)
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nt = fuse_tile_count(p);
  cudaError_t e = launch_fuse_tiles(p, b, b.pose, s);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(nt, 4 * sms));
  switch (p.L) {
    case 1: return launch_integrate_nl<1>(p, b, grid, s);
    case 2: return launch_integrate_nl<2>(p, b, grid, s);
    case 3: return launch_integrate_nl<3>(p, b, grid, s);
    case 4: return launch_integrate_nl<4>(p, b, grid, s);
    case 5: return launch_integrate_nl<5>(p, b, grid, s);
    case 6: return launch_integrate_nl<6>(p, b, grid, s);
    case 7: return launch_integrate_nl<7>(p, b, grid, s);
    case 8: return launch_integrate_nl<8>(p, b, grid, s);
    case 9: return launch_integrate_nl<9>(p, b, grid, s);
    case 10: return launch_integrate_nl<10>(p, b, grid, s);
    case 11: return launch_integrate_nl<11>(p, b, grid, s);
    case 12: return launch_integrate_nl<12>(p, b, grid, s);
    case 13: return launch_integrate_nl<13>(p, b, grid, s);
    case 14: return launch_integrate_nl<14>(p, b, grid, s);
    case 15: return launch_integrate_nl<15>(p, b, grid, s);
    case 16: return launch_integrate_nl<16>(p, b, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace xslam
