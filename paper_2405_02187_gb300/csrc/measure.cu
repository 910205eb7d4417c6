// Surface measurement (X-SLAM Sec. 4.1): range gate of the raw depth, optional bilateral filter
// ("applying a bilateral filter to the raw depth map for noise reduction"; 7x7 window, spatial sigma
// 4.5 px, range sigma 0.03 m, valid taps only) and the Gaussian pyramid.
//
// Level l+1 at pixel u is the 5x5 binomial ([1 4 6 4 1]/16 per axis) average of level l around
// pixel 2u over the taps that are valid and within pyr_range of the centre depth; invalid where the
// centre is invalid ("A coarser level depth is computed by applying Gaussian smoothing over D_k(u)").
// Depth lanes are not stored: the only depth seed on the GPU perturbs every valid pixel by the same
// h; the bilateral weights depend only on depth differences and the pyramid weights are constant,
// and both averages are normalised, so the perturbation stays h at every valid pixel of every level.
#include "internal.cuh"

namespace xslam {

__global__ void k_gate(const float* __restrict__ in, float* __restrict__ out, int n, float dmin, float dmax) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float d = in[i];
  out[i] = (d >= dmin && d <= dmax) ? d : 0.f;
}

__global__ void k_bilateral(const float* __restrict__ src, float* __restrict__ dst, int W, int H) {
  pdl_enter();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= W || v >= H) return;
  const float c = src[v * W + u];
  float out = 0.f;
  if (c > 0.f) {
    const float inv2ss = 1.f / (2.f * 4.5f * 4.5f), inv2sr = 1.f / (2.f * 0.03f * 0.03f);
    float acc = 0.f, wsum = 0.f;
    for (int dy = -3; dy <= 3; ++dy) {
      const int y = v + dy;
      if (y < 0 || y >= H) continue;
      for (int dx = -3; dx <= 3; ++dx) {
        const int x = u + dx;
        if (x < 0 || x >= W) continue;
        const float t = src[y * W + x];
        if (t > 0.f) {
          const float d = t - c;
          const float w = expf(-(float)(dx * dx + dy * dy) * inv2ss - d * d * inv2sr);
          acc += w * t;
          wsum += w;
        }
      }
    }
    out = acc / wsum;  // the centre tap has weight 1
  }
  dst[v * W + u] = out;
}

__global__ void k_pyr_down(const float* __restrict__ src, int Ws, int Hs, float* __restrict__ dst, int Wd, int Hd,
                           float range) {
  pdl_enter();
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= Wd || v >= Hd) return;
  const int sx = 2 * u, sy = 2 * v;
  const float c = src[sy * Ws + sx];
  float out = 0.f;
  if (c > 0.f) {
    const float k[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
    float acc = 0.f, wsum = 0.f;
    for (int dy = -2; dy <= 2; ++dy) {
      const int y = sy + dy;
      if (y < 0 || y >= Hs) continue;
      for (int dx = -2; dx <= 2; ++dx) {
        const int x = sx + dx;
        if (x < 0 || x >= Ws) continue;
        const float t = src[y * Ws + x];
        if (t > 0.f && fabsf(t - c) < range) {
          const float w = k[dy + 2] * k[dx + 2];
          acc += w * t;
          wsum += w;
        }
      }
    }
    out = acc / wsum;  // wsum >= 36/256 (the centre tap)
  }
  dst[v * Wd + u] = out;
}

cudaError_t launch_prepare(const Params& p, const Buffers& b, int levels, cudaStream_t s) {
  const int n = p.W * p.H;
  cudaError_t e;
  if (p.bilateral) {
    // gate into the full-size scratch image, filter into level 0
    e = launch_pdl(k_gate, dim3((n + 255) / 256), dim3(256), 0, s, b.depth_in, b.gated, n, p.depth_min, p.depth_max);
    dim3 blk(32, 8), grd((p.W + 31) / 32, (p.H + 7) / 8);
    if (e == cudaSuccess) e = launch_pdl(k_bilateral, grd, blk, 0, s, b.gated, b.pyr[0], p.W, p.H);
  } else {
    e = launch_pdl(k_gate, dim3((n + 255) / 256), dim3(256), 0, s, b.depth_in, b.pyr[0], n, p.depth_min, p.depth_max);
  }
  for (int l = 1; l < levels; ++l) {
    const int Ws = p.W >> (l - 1), Hs = p.H >> (l - 1), Wd = p.W >> l, Hd = p.H >> l;
    dim3 blk(32, 8), grd((Wd + 31) / 32, (Hd + 7) / 8);
    if (e == cudaSuccess) e = launch_pdl(k_pyr_down, grd, blk, 0, s, b.pyr[l - 1], Ws, Hs, b.pyr[l], Wd, Hd, p.pyr_range);
  }
  return e;
}

}  // namespace xslam
