// The paper's relocalisation loss (X-SLAM Sec. 5.2): the query frame D_q fused into the reference
// volume at the query pose T gives (F_q, W_q) = surface_update(M_r, T, D_q), and
//   E(T) = sum_p (F_r(p) - F_q(p))^2 = sum over the observed voxels the query updates of
//          ((F_r - F_D) / (W_r + 1))^2,
// since F_q = (W_r F_r + F_D) / (W_r + 1) there and F_q = F_r elsewhere. The sum runs over the voxels the
// reference has observed (W_r > 0): an unobserved voxel has no TSDF value to compare, and counting it
// would reward poses that see less of the map. Its gradient and Hessian with respect to a left twist of T come from
// the truncated-bicomplex step (Sec. 3, simplified arithmetic): for each of the 21 pairs j <= k the
// update's arithmetic runs on numbers a + b e1 + c e2 + d e1 e2 from T = exp(e1 G_j + e2 G_k) T_q,
// with the real pose's decisions (which voxels are updated, which are clamped at F_D = 1, the pixel
// cells). A clamped voxel has no derivative.
//
// The voxels are those of the fusion tile list built for the query pose; a 256-thread block takes one
// 8 x 8 x 8 tile (two voxels per thread) at a time. Order 1 runs the 6 diagonal pairs only (their e1
// parts are the gradient). Per-thread sums of g and H live in shared memory
// (indexed by the pair at run time), then block sums, FP64 cross-block sums in the last block.
#include "hd.cuh"
#include "internal.cuh"

namespace xslam {

namespace {

constexpr int kPairs = 21;
constexpr int kOut = 29;  // count, E, g[6], H[21]
constexpr int kThreads = 256;

}  // namespace

__global__ void __launch_bounds__(kThreads) k_tsdf_hess(Params p, const float* __restrict__ D, const float* __restrict__ F,
                                                       const float* __restrict__ Wt, const float* __restrict__ poses,
                                                       int order, const int* __restrict__ tiles,
                                                       unsigned* __restrict__ ctr,
                                                       float* __restrict__ partial, unsigned* __restrict__ ticket,
                                                       double* __restrict__ out) {
  pdl_enter();
  __shared__ HD sT[kPairs][12];
  __shared__ int sjk[kPairs][2];
  __shared__ float s_red[kThreads / 32][kOut];
  __shared__ float s_acc[kOut - 2][kThreads];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < kPairs * 12; i += blockDim.x) {
    const float* q = poses + 4 * i;
    sT[i / 12][i % 12] = {q[0], q[1], q[2], q[3]};
  }
  if (threadIdx.x < kPairs) {
    int q = threadIdx.x, j = 0;
    while (q >= 6 - j) {
      q -= 6 - j;
      ++j;
    }
    sjk[threadIdx.x][0] = j;
    sjk[threadIdx.x][1] = j + q;
  }
  for (int q = 0; q < kOut - 2; ++q) s_acc[q][threadIdx.x] = 0.f;
  __syncthreads();
  float T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = sT[0][e].a;
  float n_acc = 0.f, e_acc = 0.f;
  const unsigned count = ctr[0];
  const int ntx = (p.nx + 7) / 8, nty = (p.ny + 7) / 8;
  const float inv_mu = 1.f / p.mu;
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const int t = tiles[q];
    for (int half = 0; half < 2; ++half) {
      const int lv = threadIdx.x + half * kThreads;  // the voxel's index inside the brick
      const int i = (t % ntx) * 8 + (lv & 7), j = ((t / ntx) % nty) * 8 + ((lv >> 3) & 7),
                k = (t / (ntx * nty)) * 8 + (lv >> 6);
      if (i >= p.nx || j >= p.ny || k >= p.nz) continue;
      // ---- the surface update's decisions at the real pose ----
      const float px = p.ox + (i + 0.5f) * p.voxel, py = p.oy + (j + 0.5f) * p.voxel, pz = p.oz + (k + 0.5f) * p.voxel;
      const float dx = px - T0[3], dy = py - T0[7], dz = pz - T0[11];
      const float pcx = T0[0] * dx + T0[4] * dy + T0[8] * dz;
      const float pcy = T0[1] * dx + T0[5] * dy + T0[9] * dz;
      const float pcz = T0[2] * dx + T0[6] * dy + T0[10] * dz;
      if (!(pcz > 0.f)) continue;
      const float invz = 1.f / pcz;
      const float x = p.fx * (pcx * invz) + p.cx, y = p.fy * (pcy * invz) + p.cy;
      if (!(x >= 0.f && x < (float)(p.W - 1) && y >= 0.f && y < (float)(p.H - 1))) continue;
      const int i0 = (int)x, j0 = (int)y;
      const float a = x - i0, bb = y - j0;
      const float* row0 = D + (size_t)j0 * p.W + i0;
      const float d00 = __ldg(row0), d10 = __ldg(row0 + 1), d01 = __ldg(row0 + p.W), d11 = __ldg(row0 + p.W + 1);
      if (!(d00 > 0.f && d10 > 0.f && d01 > 0.f && d11 > 0.f)) continue;
      if (!(fabsf(d10 - d00) + fabsf(d01 - d00) + fabsf(d11 - d00) < p.disc_gate)) continue;
      const float L = (1.f - a) * (1.f - bb) * d00 + a * (1.f - bb) * d10 + (1.f - a) * bb * d01 + a * bb * d11;
      const float sdf = L - pcz;
      if (sdf < -p.mu) continue;
      const bool clamp = sdf >= p.mu;
      const size_t v = ((size_t)t << 9) + lv;
      const float w = Wt[v];
      if (!(w > 0.f)) continue;  // an unobserved reference voxel has no TSDF value to compare
      const float Fr = F[v];
      const float iw = 1.f / (w + 1.f);
      const float e = (Fr - (clamp ? 1.f : sdf / p.mu)) * iw;  // F_D rounded as the surface update rounds it
      n_acc += 1.f;
      e_acc += e * e;
      if (clamp) continue;
      // ---- the 21 second-order directions ----
      for (int qq = 0; qq < kPairs; ++qq) {
        if (order == 1 && sjk[qq][0] != sjk[qq][1]) continue;  // the gradient needs the diagonal pairs only
        const HD* T = sT[qq];
        const HD dv[3] = {hd(px) - T[3], hd(py) - T[7], hd(pz) - T[11]};
        HD pc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) pc[c] = T[c] * dv[0] + T[4 + c] * dv[1] + T[8 + c] * dv[2];
        const HD iz = inv(pc[2]);
        const HD A = p.fx * (pc[0] * iz) + (p.cx - (float)i0);
        const HD B = p.fy * (pc[1] * iz) + (p.cy - (float)j0);
        const HD x0 = (d10 - d00) * A + d00, x1 = (d11 - d01) * A + d01;
        const HD Lh = x0 + B * (x1 - x0);
        const HD eh = iw * (hd(Fr) - inv_mu * (Lh - pc[2]));
        // eh.a equals e up to rounding order; e itself (the value the loss sums) makes g vanish exactly
        // where the query repeats the fused frame
        s_acc[6 + qq][threadIdx.x] += 2.f * (e * eh.d + eh.b * eh.c);
        if (sjk[qq][0] == sjk[qq][1]) s_acc[sjk[qq][0]][threadIdx.x] += 2.f * e * eh.b;
      }
    }
  }
  // block sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[kOut];
  acc[0] = n_acc;
  acc[1] = e_acc;
#pragma unroll
  for (int q = 2; q < kOut; ++q) acc[q] = s_acc[q - 2][threadIdx.x];
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    float xs = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
    if (lane == 0) s_red[warp][q] = xs;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    float s = 0.f;
    for (int wv = 0; wv < kThreads / 32; ++wv) s += s_red[wv][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_sum[kOut];
  for (int q = warp; q < kOut; q += kThreads / 32) {
    double s = 0.0;
    for (int kk = lane; kk < (int)gridDim.x; kk += 32) s += (double)__ldcg(&partial[(size_t)q * gridDim.x + kk]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_sum[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = s_sum[1];
    for (int q = 0; q < 6; ++q) out[1 + q] = s_sum[2 + q];
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_sum[8 + q];
    out[28] = s_sum[0];
    *ticket = 0u;
    ctr[0] = 0u;  // the tile list is consumed: ready for the next fusion or loss
    ctr[1] = 0u;
  }
}

// ---- the plain FP64 path: Sec. 3's bicomplex step as printed ----
// Numbers a + b i1 + c i2 + d i1 i2 with i1^2 = i2^2 = -1 (i1 i2 = i2 i1), every product kept, in FP64,
// with the step h folded into the start poses (b, c scaled by h, d by h^2): g = Im_1 E / h and
// H = Im_12 E / h^2. The update's decisions are taken in FP64 too. This is the comparison path of the
// truncated FP32 kernel above: same loss, same voxels, the paper's arithmetic.
struct BC {
  double a, b, c, d;
};
__device__ __forceinline__ BC bc(double a) { return {a, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ BC operator+(BC x, BC y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ BC operator-(BC x, BC y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
__device__ __forceinline__ BC operator+(BC x, double s) { return {x.a + s, x.b, x.c, x.d}; }
__device__ __forceinline__ BC operator*(double s, BC x) { return {s * x.a, s * x.b, s * x.c, s * x.d}; }
__device__ __forceinline__ BC operator*(BC x, BC y) {
  return {x.a * y.a - x.b * y.b - x.c * y.c + x.d * y.d, x.a * y.b + x.b * y.a - x.c * y.d - x.d * y.c,
          x.a * y.c + x.c * y.a - x.b * y.d - x.d * y.b, x.a * y.d + x.d * y.a + x.b * y.c + x.c * y.b};
}
// 1/z: with z = z1 + z2 i2 (z1 = a + b i1, z2 = c + d i1 complex in i1), 1/z = (z1 - z2 i2) / (z1^2 + z2^2)
__device__ __forceinline__ BC binv(BC z) {
  const double p = z.a * z.a - z.b * z.b + z.c * z.c - z.d * z.d, q = 2.0 * (z.a * z.b + z.c * z.d);
  const double n = p * p + q * q, r = p / n, s = -q / n;  // 1/(p + q i1) = r + s i1
  return {z.a * r - z.b * s, z.a * s + z.b * r, -(z.c * r - z.d * s), -(z.c * s + z.d * r)};
}

__global__ void __launch_bounds__(kThreads) k_tsdf_hess64(Params p, const float* __restrict__ D,
                                                         const float* __restrict__ F, const float* __restrict__ Wt,
                                                         const double* __restrict__ poses, double inv_h,
                                                         const int* __restrict__ tiles, unsigned* __restrict__ ctr,
                                                         double* __restrict__ partial, unsigned* __restrict__ ticket,
                                                         double* __restrict__ out) {
  pdl_enter();
  constexpr int kJ[kPairs] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
  constexpr int kK[kPairs] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};
  __shared__ BC sT[kPairs][12];
  __shared__ double s_red[kThreads / 32][kOut];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < kPairs * 12; i += blockDim.x) {
    const double* q = poses + 4 * i;
    sT[i / 12][i % 12] = {q[0], q[1], q[2], q[3]};
  }
  __syncthreads();
  double T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = sT[0][e].a;
  double acc[kOut];
#pragma unroll
  for (int q = 0; q < kOut; ++q) acc[q] = 0.0;
  const unsigned count = ctr[0];
  const int ntx = (p.nx + 7) / 8, nty = (p.ny + 7) / 8;
  const double mu = p.mu, vox = p.voxel, fx = p.fx, fy = p.fy, cx = p.cx, cy = p.cy;
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const int t = tiles[q];
    for (int half = 0; half < 2; ++half) {
      const int lv = threadIdx.x + half * kThreads;
      const int i = (t % ntx) * 8 + (lv & 7), j = ((t / ntx) % nty) * 8 + ((lv >> 3) & 7),
                k = (t / (ntx * nty)) * 8 + (lv >> 6);
      if (i >= p.nx || j >= p.ny || k >= p.nz) continue;
      const double px = p.ox + (i + 0.5) * vox, py = p.oy + (j + 0.5) * vox, pz = p.oz + (k + 0.5) * vox;
      const double dx = px - T0[3], dy = py - T0[7], dz = pz - T0[11];
      const double pcx = T0[0] * dx + T0[4] * dy + T0[8] * dz;
      const double pcy = T0[1] * dx + T0[5] * dy + T0[9] * dz;
      const double pcz = T0[2] * dx + T0[6] * dy + T0[10] * dz;
      if (!(pcz > 0.0)) continue;
      const double x = fx * (pcx / pcz) + cx, y = fy * (pcy / pcz) + cy;
      if (!(x >= 0.0 && x < (double)(p.W - 1) && y >= 0.0 && y < (double)(p.H - 1))) continue;
      const int i0 = (int)x, j0 = (int)y;
      const double a = x - i0, bb = y - j0;
      const float* row0 = D + (size_t)j0 * p.W + i0;
      const double d00 = __ldg(row0), d10 = __ldg(row0 + 1), d01 = __ldg(row0 + p.W), d11 = __ldg(row0 + p.W + 1);
      if (!(d00 > 0.0 && d10 > 0.0 && d01 > 0.0 && d11 > 0.0)) continue;
      if (!(fabs(d10 - d00) + fabs(d01 - d00) + fabs(d11 - d00) < (double)p.disc_gate)) continue;
      const double L = (1.0 - a) * (1.0 - bb) * d00 + a * (1.0 - bb) * d10 + (1.0 - a) * bb * d01 + a * bb * d11;
      const double sdf = L - pcz;
      if (sdf < -mu) continue;
      const bool clamp = sdf >= mu;
      const size_t v = ((size_t)t << 9) + lv;
      const double w = Wt[v];
      if (!(w > 0.0)) continue;
      const double Fr = F[v];
      const double iw = 1.0 / (w + 1.0);
      const double e = (Fr - (clamp ? 1.0 : sdf / mu)) * iw;
      acc[0] += 1.0;
      acc[1] += e * e;
      if (clamp) continue;
#pragma unroll
      for (int qq = 0; qq < kPairs; ++qq) {
        const BC* T = sT[qq];
        const BC dv[3] = {bc(px) - T[3], bc(py) - T[7], bc(pz) - T[11]};
        BC pc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) pc[c] = T[c] * dv[0] + T[4 + c] * dv[1] + T[8 + c] * dv[2];
        const BC iz = binv(pc[2]);
        const BC A = fx * (pc[0] * iz) + (cx - (double)i0);
        const BC B = fy * (pc[1] * iz) + (cy - (double)j0);
        const BC x0 = (d10 - d00) * A + d00, x1 = (d11 - d01) * A + d01;
        const BC Lh = x0 + B * (x1 - x0);
        const BC eh = iw * (bc(Fr) - (1.0 / mu) * (Lh - pc[2]));
        const BC e2 = eh * eh;
        acc[8 + qq] += e2.d;
        if (kJ[qq] == kK[qq]) acc[2 + kJ[qq]] += e2.b;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    double xs = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
    if (lane == 0) s_red[warp][q] = xs;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int wv = 0; wv < kThreads / 32; ++wv) s += s_red[wv][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_sum[kOut];
  for (int q = warp; q < kOut; q += kThreads / 32) {
    double s = 0.0;
    for (int kk = lane; kk < (int)gridDim.x; kk += 32) s += __ldcg(&partial[(size_t)q * gridDim.x + kk]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_sum[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = s_sum[1];
    for (int q = 0; q < 6; ++q) out[1 + q] = s_sum[2 + q] * inv_h;
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_sum[8 + q] * inv_h * inv_h;
    out[28] = s_sum[0];
    *ticket = 0u;
    ctr[0] = 0u;
    ctr[1] = 0u;
  }
}

cudaError_t launch_tsdf_hess64(const Params& p, const Buffers& b, const float* depth, const double* pose,
                               const double* poses, double h, double* out, int nblk, cudaStream_t s) {
  cudaError_t e = launch_fuse_tiles(p, b, pose, s);
  if (e != cudaSuccess) return e;
  // the float partial buffer holds (blocks + 4) x 27 x 16 floats: room for 29 doubles per block
  return launch_pdl(k_tsdf_hess64, dim3(nblk), dim3(kThreads), 0, s, p, depth, (const float*)b.F, (const float*)b.Wt,
                    poses, 1.0 / h, (const int*)b.tiles, b.tile_ctr, reinterpret_cast<double*>(b.partial), b.ticket,
                    out);
}

cudaError_t launch_tsdf_hess(const Params& p, const Buffers& b, const float* depth, const double* pose,
                             const float* poses, int order, double* out, int nblk, cudaStream_t s) {
  cudaError_t e = launch_fuse_tiles(p, b, pose, s);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_tsdf_hess, dim3(nblk), dim3(kThreads), 0, s, p, depth, (const float*)b.F, (const float*)b.Wt,
                    poses, order, (const int*)b.tiles, b.tile_ctr, b.partial, b.ticket, out);
}

}  // namespace xslam
