// Surface measurement (X-SLAM Sec. 4.1): range gate of the raw depth, optional bilateral filter
// ("applying a bilateral filter to the raw depth map for noise reduction"; 7x7 window, spatial sigma
// 4.5 px, range sigma 0.03 m, valid taps only) and the Gaussian pyramid.
//
// Level l+1 at pixel u is the 5x5 binomial ([1 4 6 4 1]/16 per axis) average of level l around
// pixel 2u over the taps that are valid and within pyr_range of the centre depth; invalid where the
// centre is invalid ("A coarser level depth is computed by applying Gaussian smoothing over D_k(u)").
// A DEPTH seed on every pixel needs no stored lane: it perturbs every valid pixel by the same h, the
// bilateral weights depend only on depth differences and the pyramid weights are constant, and both
// averages are normalised, so the perturbation stays h at every valid pixel of every level. A DEPTH seed
// on one pixel s has an Im depth map per level (k_depth_lanes): at level 0 the tangent of the bilateral
// filter (its range weights now move with the perturbation) over the 7x7 window around s, at levels 1
// and 2 the pyramid's average of the finer level's map with the real part's weights ("The perturbed hi
// is also Gaussian smoothed"); outside those windows the maps stay zero.
#include "internal.cuh"

namespace xslam {

__device__ __forceinline__ void gate_body(const float* __restrict__ in, float* __restrict__ out, int n, float dmin,
                                          float dmax, int bx) {
  int i = bx * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float d = in[i];
  out[i] = (d >= dmin && d <= dmax) ? d : 0.f;
}

__global__ void k_gate(const float* __restrict__ in, float* __restrict__ out, int n, float dmin, float dmax) {
  pdl_enter();
  gate_body(in, out, n, dmin, dmax, blockIdx.x);
}

__device__ __forceinline__ void bilateral_body(const float* __restrict__ src, float* __restrict__ dst, int W, int H,
                                               int bx, int by) {
  const int u = bx * blockDim.x + threadIdx.x;
  const int v = by * blockDim.y + threadIdx.y;
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

__global__ void k_bilateral(const float* __restrict__ src, float* __restrict__ dst, int W, int H) {
  pdl_enter();
  bilateral_body(src, dst, W, H, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ void pyr_down_body(const float* __restrict__ src, int Ws, int Hs, float* __restrict__ dst,
                                              int Wd, int Hd, float range, int bx, int by) {
  int u = bx * blockDim.x + threadIdx.x;
  int v = by * blockDim.y + threadIdx.y;
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

__global__ void k_pyr_down(const float* __restrict__ src, int Ws, int Hs, float* __restrict__ dst, int Wd, int Hd,
                           float range) {
  pdl_enter();
  pyr_down_body(src, Ws, Hs, dst, Wd, Hd, range, blockIdx.x, blockIdx.y);
}

// Segmented measurement stages (batches): stage 0 the range gate (1-D grids of 256-thread blocks, into
// the filter's source or level 0), stage 1 the bilateral filter, stage 1 + l level l of the pyramid
// (2-D grids of 32 x 8 blocks; a segment's arg is its grid's width in blocks).
__global__ void __launch_bounds__(256) k_prepare_seg(SegTable st, int stage) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  const Params& p = d.p;
  const Buffers& b = d.b;
  const int lb = blockIdx.x - sg.block0;
  if (stage == 0) {
    gate_body(b.depth_in, p.bilateral ? b.gated : b.pyr[0], p.W * p.H, p.depth_min, p.depth_max, lb);
  } else if (stage == 1) {
    bilateral_body(b.gated, b.pyr[0], p.W, p.H, lb % sg.arg, lb / sg.arg);
  } else {
    const int l = stage - 1;
    pyr_down_body(b.pyr[l - 1], p.W >> (l - 1), p.H >> (l - 1), b.pyr[l], p.W >> l, p.H >> l, p.pyr_range,
                  lb % sg.arg, lb / sg.arg);
  }
}

cudaError_t launch_prepare_seg(const SegTable& t, int nblocks, int stage, cudaStream_t s) {
  const dim3 blk = stage == 0 ? dim3(256) : dim3(32, 8);
  return launch_pdl(k_prepare_seg, dim3(nblocks), blk, 0, s, t, stage);
}

// Im depth maps of single-pixel DEPTH lanes, one block per lane (blockIdx.x + 1). The seed pixel s carries
// h if its range-gated depth is valid. Level 0 with the filter on: at output u (valid) with real input
// D, filtered value D'(u) and weights w_t = exp(-|t - u|^2 / 2 ss^2 - (D_t - D_u)^2 / 2 sr^2), the
// tangent is [sum_t w_t dD_t - sum_t w_t (D_t - D_u) / sr^2 (dD_t - dD_u) (D_t - D'(u))] / sum_t w_t
// with dD_t = h [t = s]; without the filter the map is h at s. Level l + 1 at u: the pyramid's
// normalised average of level l's map over the taps the real average used.
__global__ void k_depth_lanes(Params p, const float* __restrict__ src0, const float* __restrict__ pyr0,
                              const float* __restrict__ pyr1, const float* __restrict__ pyr2, float* __restrict__ dlane,
                              int levels) {
  pdl_enter();
  const int l = blockIdx.x + 1;
  if (l >= p.L || p.dpix[l] < 0) return;
  const int W = p.W, H = p.H;
  const int sx = p.dpix[l] % W, sy = p.dpix[l] / W;
  const float h = (float)p.h[l];
  const bool seed_ok = src0[p.dpix[l]] > 0.f;
  // level 0
  const int R0 = p.bilateral ? 3 : 0;
  int lox = max(sx - R0, 0), hix = min(sx + R0, W - 1), loy = max(sy - R0, 0), hiy = min(sy + R0, H - 1);
  float* d0 = dlane + dlane_offset(p, l, 0);
  const int n0 = (hix - lox + 1) * (hiy - loy + 1);
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    const int u = lox + i % (hix - lox + 1), v = loy + i / (hix - lox + 1);
    const float c = src0[v * W + u];
    float out = 0.f;
    if (seed_ok && c > 0.f) {
      if (!p.bilateral) {
        out = (u == sx && v == sy) ? h : 0.f;
      } else {
        const float inv2ss = 1.f / (2.f * 4.5f * 4.5f), inv2sr = 1.f / (2.f * 0.03f * 0.03f);
        const float isr2 = 1.f / (0.03f * 0.03f);
        const float Df = pyr0[v * W + u];
        const float dDu = (u == sx && v == sy) ? h : 0.f;
        float num = 0.f, wsum = 0.f;
        for (int dy = -3; dy <= 3; ++dy) {
          const int y = v + dy;
          if (y < 0 || y >= H) continue;
          for (int dx = -3; dx <= 3; ++dx) {
            const int x = u + dx;
            if (x < 0 || x >= W) continue;
            const float t = src0[y * W + x];
            if (!(t > 0.f)) continue;
            const float d = t - c;
            const float w = expf(-(float)(dx * dx + dy * dy) * inv2ss - d * d * inv2sr);
            const float dDt = (x == sx && y == sy) ? h : 0.f;
            num += w * dDt - w * d * isr2 * (dDt - dDu) * (t - Df);
            wsum += w;
          }
        }
        out = num / wsum;
      }
    }
    d0[v * W + u] = out;
  }
  __syncthreads();
  // levels 1 and 2: the windows of the pixels whose 5x5 taps around 2u reach the finer window
  const float k5[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
  const float* fine = pyr0;
  const float* dfine = d0;
  for (int lv = 1; lv < levels; ++lv) {
    const int Wf = W >> (lv - 1), Hf = H >> (lv - 1), Wc = W >> lv, Hc = H >> lv;
    const float* coarse = lv == 1 ? pyr1 : pyr2;
    float* dc = dlane + dlane_offset(p, l, lv);
    const int nlox = max((lox - 2 + 1) >> 1, 0), nhix = min((hix + 2) >> 1, Wc - 1);
    const int nloy = max((loy - 2 + 1) >> 1, 0), nhiy = min((hiy + 2) >> 1, Hc - 1);
    const int n = (nhix - nlox + 1) * (nhiy - nloy + 1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int u = nlox + i % (nhix - nlox + 1), v = nloy + i / (nhix - nlox + 1);
      float out = 0.f;
      if (coarse[v * Wc + u] > 0.f) {
        const float c = fine[(2 * v) * Wf + 2 * u];
        float num = 0.f, wsum = 0.f;
        for (int dy = -2; dy <= 2; ++dy) {
          const int y = 2 * v + dy;
          if (y < 0 || y >= Hf) continue;
          for (int dx = -2; dx <= 2; ++dx) {
            const int x = 2 * u + dx;
            if (x < 0 || x >= Wf) continue;
            const float t = fine[y * Wf + x];
            if (t > 0.f && fabsf(t - c) < p.pyr_range) {
              const float w = k5[dy + 2] * k5[dx + 2];
              num += w * dfine[y * Wf + x];
              wsum += w;
            }
          }
        }
        out = num / wsum;
      }
      dc[v * Wc + u] = out;
    }
    __syncthreads();
    fine = coarse;
    dfine = dc;
    lox = nlox;
    hix = nhix;
    loy = nloy;
    hiy = nhiy;
  }
}

cudaError_t launch_depth_lanes(const Params& p, const Buffers& b, int levels, cudaStream_t s) {
  if (p.L < 2) return cudaSuccess;
  const float* src0 = p.bilateral ? b.gated : b.pyr[0];
  return launch_pdl(k_depth_lanes, dim3(p.L - 1), dim3(256), 0, s, p, src0, b.pyr[0], b.pyr[1], b.pyr[2], b.dlane,
                    levels);
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
