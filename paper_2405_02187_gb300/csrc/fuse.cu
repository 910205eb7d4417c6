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

// Real part of the update of voxel (i, j, k) at offset (dx, dy, dz) = centre - t from the camera centre:
// whether the frame updates it, and what its lanes need. NL = 1 + K lanes.
struct VoxDec {
  float FD;             // F_D (real)
  float cxl, cyl, czl;  // the sdf tangent as a linear form of the lane's p_c' (unclamped voxels)
  bool clamp;           // F_D = 1 on every lane: no tangent
};

__device__ __forceinline__ bool fuse_decide(const Params& p, const float* __restrict__ D, const float* T, float dx,
                                            float dy, float dz, VoxDec& o) {
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
  o.clamp = sdf >= p.mu;
  o.FD = o.clamp ? 1.f : sdf / p.mu;
  // The tangent of sdf = L(x) - z_c is linear in the lane's p_c': with x' = fx (p_cx' - q_x p_cz') / z,
  // y' = fy (p_cy' - q_y p_cz') / z and the bilinear L's slopes dL/da, dL/db,
  // sdf' = c_x p_cx' + c_y p_cy' + c_z p_cz' + D', c_x = dL/da fx / z, c_y = dL/db fy / z,
  // c_z = -(c_x q_x + c_y q_y) - 1.
  const float dLda = (1.f - bb) * (d10 - d00) + bb * (d11 - d01);
  const float dLdb = (1.f - a) * (d01 - d00) + a * (d11 - d10);
  o.cxl = dLda * p.fx * invz;
  o.cyl = dLdb * p.fy * invz;
  o.czl = -(o.cxl * qx + o.cyl * qy) - 1.f;
  return true;
}

// The lane-l tangent of F_D of an unclamped voxel: sdf' from the lane's p_c' = dR^T (p - t) - R^T dt
// (the second term a per-lane constant sC) and D' (all-pixel DEPTH h, or the single-pixel lane's Im
// depth map bilinear in the real cell), then F_D' = (sdf' - F_D mu') / mu.
__device__ __forceinline__ float fuse_lane_FD(const Params& p, const float* __restrict__ dlane, const float* sT0,
                                              const float* Tl, const float* C, int l, const VoxDec& o, float dx,
                                              float dy, float dz) {
  const float pcx_l = Tl[0] * dx + Tl[4] * dy + Tl[8] * dz + C[0];
  const float pcy_l = Tl[1] * dx + Tl[5] * dy + Tl[9] * dz + C[1];
  const float pcz_l = Tl[2] * dx + Tl[6] * dy + Tl[10] * dz + C[2];
  float Dl = p.dD[l];
  if (p.dpix[l] >= 0) {
    // the projection again (the real pose's, as fuse_decide took it)
    const float* T = sT0;
    const float pcx = T[0] * dx + T[4] * dy + T[8] * dz;
    const float pcy = T[1] * dx + T[5] * dy + T[9] * dz;
    const float invz = 1.f / (T[2] * dx + T[6] * dy + T[10] * dz);
    const float x = p.fx * (pcx * invz) + p.cx, y = p.fy * (pcy * invz) + p.cy;
    const int i0 = (int)x, j0 = (int)y;
    const float a = x - i0, bb = y - j0;
    const float* m = dlane + dlane_offset(p, l, 0) + (size_t)j0 * p.W + i0;
    Dl += (1.f - a) * (1.f - bb) * m[0] + a * (1.f - bb) * m[1] + (1.f - a) * bb * m[p.W] + a * bb * m[p.W + 1];
  }
  const float sdf_l = o.cxl * pcx_l + o.cyl * pcy_l + o.czl * pcz_l + Dl;
  return (sdf_l - o.FD * p.dmu[l]) * p.inv_mu;
}

// One thread per 8 x 8 x 8 tile: a tile any of whose voxels the frame can update is appended to the
// list (warp-aggregated atomics). The test is the exact corner test: the tile's box (padded by half a
// voxel around the voxel centres) is skipped if all 8 corners lie behind the camera or beyond the
// same image edge.
// bx, gx: this block's index in its trajectory's grid and that grid's size
__device__ __forceinline__ void fuse_tiles_body(const Params& p, const double* __restrict__ pose,
                                                int* __restrict__ tiles, unsigned* __restrict__ ctr, int bx, int gx) {
  const int ntx = (p.nx + kBX - 1) / kBX, nty = (p.ny + kBY - 1) / kBY, ntz = (p.nz + kBZ - 1) / kBZ;
  const int nt = ntx * nty * ntz;
  float T[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T[e] = (float)pose[e];
  for (int t0 = bx * blockDim.x; t0 < nt; t0 += gx * blockDim.x) {
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

__global__ void __launch_bounds__(256) k_fuse_tiles(Params p, const double* __restrict__ pose, int* __restrict__ tiles,
                                                   unsigned* __restrict__ ctr) {
  pdl_enter();
  fuse_tiles_body(p, pose, tiles, ctr, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_fuse_tiles_seg(SegTable st) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  fuse_tiles_body(d.p, d.b.pose, d.b.tiles, d.b.tile_ctr, blockIdx.x - sg.block0, sg.nblk);
}

// Fixed grid over the tile list; a block takes one tile at a time, a thread per 4 x-consecutive voxels of
// a brick row: thread t holds voxels 4 (t mod 2) .. + 3 of row y = t / 2 mod 8, z = t / 16, so a warp's
// 128-bit loads and stores cover 512 consecutive bytes of every plane. A thread first takes the real
// decisions of its 4 voxels; if the frame updates any of them it loads W and every lane of all 4 (one
// 16-byte load per plane, all issued before any store), updates the observed ones and stores the 4
// (the others unchanged). The last block to finish clears the list counters for the next launch.
constexpr int kQuadThreads = 128;

// resident blocks of 128 threads per SM: register budgets of 64, 96 and 128 per thread by lane count
__host__ __device__ constexpr int fuse_blocks_per_sm(int NL) { return NL <= 2 ? 8 : (NL <= 9 ? 5 : 4); }

template <int NL>
__device__ __forceinline__ void integrate_body(const Params& p, const float* __restrict__ D,
                                               const double* __restrict__ pose, float* __restrict__ F,
                                               float* __restrict__ Wt, float* __restrict__ F0lin,
                                               unsigned long long* __restrict__ stats, const int* __restrict__ tiles,
                                               unsigned* __restrict__ ctr, const float* __restrict__ dlane,
                                               int* __restrict__ tiles_prev, int bx, int gx) {
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
  const int qx = (tid & 1) * 4, cy = (tid >> 1) & 7, cz = tid >> 4;
  const int off = cz * 64 + cy * 8 + qx;  // the quad's first voxel in the brick
  const bool lin4 = (p.nx & 3) == 0;      // the linear copy's rows keep 16-byte alignment
  const float* T = sT[0];
  int cnt = 0;
  for (unsigned q = bx; q < count; q += gx) {
    const int t = tiles[q];
    if (p.fresh && tid == 0) tiles_prev[q] = t;  // the next frame clears its restarted lanes here
    const int i0 = (t % ntx) * kBX + qx, j = ((t / ntx) % nty) * kBY + cy, k = (t / (ntx * nty)) * kBZ + cz;
    if (j >= p.ny || k >= p.nz) continue;
    const float dy = p.oy + (j + 0.5f) * p.voxel - T[7];
    const float dz = p.oz + (k + 0.5f) * p.voxel - T[11];
    VoxDec dec[4];
    unsigned upd = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float dx = p.ox + (i0 + v + 0.5f) * p.voxel - T[3];
      if (i0 + v < p.nx && fuse_decide(p, D, T, dx, dy, dz, dec[v])) upd |= 1u << v;
    }
    if (!upd) continue;
    const size_t base = ((size_t)t << 9) + off;
    float4 w4 = *reinterpret_cast<const float4*>(Wt + base);
    float4 f4[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) f4[l] = *reinterpret_cast<const float4*>(F + (size_t)l * n + base);
    float w[4] = {w4.x, w4.y, w4.z, w4.w};
    float f[NL][4];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      f[l][0] = f4[l].x;
      f[l][1] = f4[l].y;
      f[l][2] = f4[l].z;
      f[l][3] = f4[l].w;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (!((upd >> v) & 1u)) continue;
      const float w0 = w[v];
      const float w1 = w0 + 1.f;
      const float inv = 1.f / w1;
      f[0][v] = (w0 * f[0][v] + dec[v].FD) / w1;  // an unobserved voxel (w = 0) takes F_D whatever its sentinel
      w[v] = (p.w_max > 0.f) ? fminf(w1, p.w_max) : w1;
      if (dec[v].clamp) {  // F_D = 1 whatever the lane: no tangent
#pragma unroll
        for (int l = 1; l < NL; ++l) f[l][v] = w0 * f[l][v] * inv;
      } else {
        const float dx = p.ox + (i0 + v + 0.5f) * p.voxel - T[3];
#pragma unroll
        for (int l = 1; l < NL; ++l)
          f[l][v] = (w0 * f[l][v] + fuse_lane_FD(p, dlane, T, sT[l], sC[l], l, dec[v], dx, dy, dz)) * inv;
      }
    }
    *reinterpret_cast<float4*>(Wt + base) = make_float4(w[0], w[1], w[2], w[3]);
#pragma unroll
    for (int l = 0; l < NL; ++l)
      *reinterpret_cast<float4*>(F + (size_t)l * n + base) = make_float4(f[l][0], f[l][1], f[l][2], f[l][3]);
    // the march's linear copy of Re F (unchanged voxels rewrite the value they hold; an unobserved one
    // its NaN there)
    const size_t li = (size_t)i0 + (size_t)p.nx * ((size_t)j + (size_t)p.ny * k);
    if (lin4 && i0 + 3 < p.nx) {
      float o[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v] = w[v] > 0.f ? f[0][v] : unobserved_lin();
      *reinterpret_cast<float4*>(F0lin + li) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if ((upd >> v) & 1u) F0lin[li + v] = f[0][v];
    }
    cnt += __popc(upd);
  }
  // updated-voxel count: warp sums, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((tid & 31) == 0 && cnt) atomicAdd(stats, (unsigned long long)cnt);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(ctr + 1, 1u) == (unsigned)gx - 1;
  }
  __syncthreads();
  if (s_last && tid == 0) {
    ctr[2] = p.fresh ? count : 0u;
    ctr[0] = 0u;
    ctr[1] = 0u;
  }
}

template <int NL>
__global__ void __launch_bounds__(kQuadThreads, fuse_blocks_per_sm(NL)) k_integrate(Params p, const float* __restrict__ D,
                                                        const double* __restrict__ pose, float* __restrict__ F,
                                                        float* __restrict__ Wt, float* __restrict__ F0lin,
                                                        unsigned long long* __restrict__ stats,
                                                        const int* __restrict__ tiles, unsigned* __restrict__ ctr,
                                                        const float* __restrict__ dlane, int* __restrict__ tiles_prev) {
  pdl_enter();
  integrate_body<NL>(p, D, pose, F, Wt, F0lin, stats, tiles, ctr, dlane, tiles_prev, blockIdx.x, gridDim.x);
}

// every segment's trajectory has NL lanes
template <int NL>
__global__ void __launch_bounds__(kQuadThreads, fuse_blocks_per_sm(NL)) k_integrate_seg(SegTable st) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  const Buffers& b = d.b;
  integrate_body<NL>(d.p, b.pyr[0], b.pose, b.F, b.Wt, b.F0lin, b.stats, b.tiles, b.tile_ctr, b.dlane, b.tiles_prev,
                     blockIdx.x - sg.block0, sg.nblk);
}

// Restarted lanes (per-frame pose seeds): before frame k's update their TSDF planes must hold no
// imaginary part, so that Im F_k is frame k's derivative alone. Only the bricks of the last update can
// hold one: a block per brick of that list zeroes those lanes' planes there.
__global__ void __launch_bounds__(kFuseThreads) k_clear_fresh(Params p, float* __restrict__ F,
                                                               const int* __restrict__ tiles_prev,
                                                               const unsigned* __restrict__ ctr) {
  pdl_enter();
  const unsigned count = ctr[2];
  const size_t n = vox_plane(p);
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const size_t v = ((size_t)tiles_prev[q] << 9) + threadIdx.x;
    for (int l = 1; l < p.L; ++l)
      if ((p.fresh >> l) & 1u) F[(size_t)l * n + v] = 0.f;
  }
}

template <int NL>
static cudaError_t launch_integrate_nl(const Params& p, const Buffers& b, int grid, cudaStream_t s) {
  return launch_pdl(k_integrate<NL>, dim3(grid), dim3(kQuadThreads), 0, s, p, b.pyr[0], b.pose, b.F, b.Wt, b.F0lin,
                    b.stats, b.tiles, b.tile_ctr, (const float*)b.dlane, b.tiles_prev);
}

int fuse_tile_count(const Params& p) {
  return ((p.nx + kBX - 1) / kBX) * ((p.ny + kBY - 1) / kBY) * ((p.nz + kBZ - 1) / kBZ);
}

static int device_sms() {  // the current device's SM count (queried per call: a handle may live on any device)
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int fuse_tiles_grid(const Params& p) { return std::max(1, std::min((fuse_tile_count(p) + 255) / 256, 4 * device_sms())); }

int integrate_grid(const Params& p) {
  return std::max(1, std::min(fuse_tile_count(p), fuse_blocks_per_sm(p.L) * device_sms()));  // the resident blocks
}

cudaError_t launch_fuse_tiles(const Params& p, const Buffers& b, const double* pose, cudaStream_t s) {
  return launch_pdl(k_fuse_tiles, dim3(fuse_tiles_grid(p)), dim3(256), 0, s, p, pose, b.tiles, b.tile_ctr);
}

cudaError_t launch_clear_fresh(const Params& p, const Buffers& b, cudaStream_t s) {
  return launch_pdl(k_clear_fresh, dim3(std::max(1, std::min(fuse_tile_count(p), 4 * device_sms()))),
                    dim3(kFuseThreads), 0, s, p, b.F, (const int*)b.tiles_prev, (const unsigned*)b.tile_ctr);
}

template <int NL>
static cudaError_t launch_integrate_seg_nl(const SegTable& t, int nblocks, cudaStream_t s) {
  return launch_pdl(k_integrate_seg<NL>, dim3(nblocks), dim3(kQuadThreads), 0, s, t);
}

cudaError_t launch_fuse_tiles_seg(const SegTable& t, int nblocks, cudaStream_t s) {
  return launch_pdl(k_fuse_tiles_seg, dim3(nblocks), dim3(256), 0, s, t);
}

#define XSLAM_LANE_SWITCH(L, CALL)                                                                   \
  switch (L) {                                                                                       \
    case 1: return CALL(1); case 2: return CALL(2); case 3: return CALL(3); case 4: return CALL(4);  \
    case 5: return CALL(5); case 6: return CALL(6); case 7: return CALL(7); case 8: return CALL(8);  \
    case 9: return CALL(9); case 10: return CALL(10); case 11: return CALL(11);                      \
    case 12: return CALL(12); case 13: return CALL(13); case 14: return CALL(14);                    \
    case 15: return CALL(15); case 16: return CALL(16);                                              \
    default: return cudaErrorInvalidValue;                                                           \
  }

cudaError_t launch_integrate_seg(const SegTable& t, int nblocks, int L, cudaStream_t s) {
#define XSLAM_SEG(NL) launch_integrate_seg_nl<NL>(t, nblocks, s)
  XSLAM_LANE_SWITCH(L, XSLAM_SEG)
#undef XSLAM_SEG
}

cudaError_t launch_integrate(const Params& p, const Buffers& b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (p.fresh && (e = launch_clear_fresh(p, b, s)) != cudaSuccess) return e;
  e = launch_fuse_tiles(p, b, b.pose, s);
  if (e != cudaSuccess) return e;
  const int grid = integrate_grid(p);
#define XSLAM_ONE(NL) launch_integrate_nl<NL>(p, b, grid, s)
  XSLAM_LANE_SWITCH(p.L, XSLAM_ONE)
#undef XSLAM_ONE
}

}  // namespace xslam
