// Relocalisation loss with its gradient and Hessian in one pass (xslam_grad, order 2).
//
// E(T) = mean over accepted pixels u of r_u^2, r_u = (T V_q(u) - V_g(u)) . N_g(u), with V_g, N_g ray
// cast from the TSDF at T itself (the point-to-plane reading of X-SLAM Sec. 5.2). The second
// derivatives with respect to a left twist xi of T follow the bicomplex step of Sec. 3 in its
// simplified (truncated) form: a number a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0 carries f,
// df/dxi_j, df/dxi_k and d2f/dxi_j dxi_k exactly (unit steps; no truncation error, no cancellation).
// Pair (j, k) starts from T = exp(e1 G_j + e2 G_k) T_q = (I + e1 G_j + e2 G_k + e1 e2 (G_j G_k + G_k
// G_j) / 2) T_q, the 21 pairs j <= k giving the upper triangle.
//
// Every discrete decision is the real pose's: the hit sample pair of the march (k_march at T_q), the
// cells of the two hit samples and of the six gradient samples, their validity, and the distance
// gate. One thread takes a pixel: it loads the 8 cells' corner values once and then evaluates the
// ray-cast refinement and the residual on the 21 pairs. Block sums in FP32, the cross-block sum of
// the last block in FP64.
#include "bc.cuh"
#include "hd.cuh"
#include "internal.cuh"
#include "raycast.cuh"

namespace xslam {

namespace {

// corner values of the cell containing (gx, gy, gz) (voxel-centre coordinates); false outside the
// volume or with an unobserved corner. c[dx + 2 dy + 4 dz].
__device__ __forceinline__ bool load_cell(const Params& p, const float* __restrict__ F, float gx, float gy, float gz,
                                          int& i, int& j, int& k, float* c) {
  if (!(gx >= 0.f && gx < (float)(p.nx - 1) && gy >= 0.f && gy < (float)(p.ny - 1) && gz >= 0.f &&
        gz < (float)(p.nz - 1)))
    return false;
  i = (int)gx;
  j = (int)gy;
  k = (int)gz;
  const CellAddr a = cell_addr(p, i, j, k);
  const unsigned b = a.b, sx = a.dx, sy = a.dy, sz = a.dz;
  c[0] = __ldg(F + b);
  c[1] = __ldg(F + b + sx);
  c[2] = __ldg(F + b + sy);
  c[3] = __ldg(F + b + sx + sy);
  c[4] = __ldg(F + b + sz);
  c[5] = __ldg(F + b + sx + sz);
  c[6] = __ldg(F + b + sy + sz);
  c[7] = __ldg(F + b + sx + sy + sz);
  float mx = c[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) mx = fmaxf(mx, c[q]);
  return mx <= 1.f;  // the unobserved sentinel is above 1
}

__device__ __forceinline__ float tri(const float* c, float fx, float fy, float fz) {
  const float x00 = c[0] + fx * (c[1] - c[0]), x10 = c[2] + fx * (c[3] - c[2]);
  const float x01 = c[4] + fx * (c[5] - c[4]), x11 = c[6] + fx * (c[7] - c[6]);
  const float y0 = x00 + fy * (x10 - x00), y1 = x01 + fy * (x11 - x01);
  return y0 + fz * (y1 - y0);
}

// trilinear interpolation with truncated-bicomplex weights (the cell's values are real)
__device__ __forceinline__ HD tri_hd(const float* c, HD fx, HD fy, HD fz) {
  HD x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float lo = c[2 * q], dd = c[2 * q + 1] - c[2 * q];
    x[q] = {lo + fx.a * dd, fx.b * dd, fx.c * dd, fx.d * dd};
  }
  const HD y0 = x[0] + fy * (x[1] - x[0]), y1 = x[2] + fy * (x[3] - x[2]);
  return y0 + fz * (y1 - y0);
}

constexpr int kPairs = 21;
constexpr int kOut = 29;  // count, E, g[6], H[21]
constexpr int kHessThreads = 128;

}  // namespace

__global__ void __launch_bounds__(kHessThreads) k_hess(Params p, const float* __restrict__ F, const float* __restrict__ D,
                                                      const int* __restrict__ hit, const float* __restrict__ poses,
                                                      float* __restrict__ partial, unsigned* __restrict__ ticket,
                                                      double* __restrict__ out) {
  pdl_enter();
  __shared__ HD sT[kPairs][12];
  __shared__ int sjk[kPairs][2];
  __shared__ float s_red[kHessThreads / 32][kOut];
  __shared__ float s_acc[kOut - 2][kHessThreads];  // per-thread g and H sums (indexed by the pair at run time)
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
  __syncthreads();
  float acc[kOut];
#pragma unroll
  for (int q = 0; q < kOut; ++q) acc[q] = 0.f;
  for (int q = 0; q < kOut - 2; ++q) s_acc[q][threadIdx.x] = 0.f;
  const float inv_vox = 1.f / p.voxel;
  const float og[3] = {p.ox, p.oy, p.oz};
  float T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = sT[0][e].a;
  const size_t hw = (size_t)p.W * p.H;
  for (size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x; pix < hw; pix += (size_t)gridDim.x * blockDim.x) {
    const int m = hit[pix];
    const float dq = D[pix];
    if (m < 0 || !(dq > 0.f)) continue;
    const int u = (int)(pix % p.W), v = (int)(pix / p.W);
    const Ray ry = make_ray(p, T0, u, v);
    // ---- the real refinement: decisions and cell values ----
    float cv[8][8];
    int ci[8][3];
    const float am = m * p.ray_step, an = (m + 1) * p.ray_step;
    bool ok = load_cell(p, F, ry.g0x + am * ry.gdx, ry.g0y + am * ry.gdy, ry.g0z + am * ry.gdz, ci[0][0], ci[0][1],
                        ci[0][2], cv[0]);
    ok = ok && load_cell(p, F, ry.g0x + an * ry.gdx, ry.g0y + an * ry.gdy, ry.g0z + an * ry.gdz, ci[1][0], ci[1][1],
                         ci[1][2], cv[1]);
    if (!ok) continue;
    const float gm[3] = {ry.g0x + am * ry.gdx, ry.g0y + am * ry.gdy, ry.g0z + am * ry.gdz};
    const float gn[3] = {ry.g0x + an * ry.gdx, ry.g0y + an * ry.gdy, ry.g0z + an * ry.gdz};
    const float Fm = tri(cv[0], gm[0] - ci[0][0], gm[1] - ci[0][1], gm[2] - ci[0][2]);
    const float Fn = tri(cv[1], gn[0] - ci[1][0], gn[1] - ci[1][1], gn[2] - ci[1][2]);
    const float alpha0 = am - p.ray_step * Fm / (Fn - Fm);
    const float v0[3] = {T0[3] + alpha0 * ry.dirx, T0[7] + alpha0 * ry.diry, T0[11] + alpha0 * ry.dirz};
    const float gc[3] = {(v0[0] - og[0]) * inv_vox - 0.5f, (v0[1] - og[1]) * inv_vox - 0.5f,
                         (v0[2] - og[2]) * inv_vox - 0.5f};
    float grad[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      float val[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int q = 2 + 2 * ax + s;
        float g3[3] = {gc[0], gc[1], gc[2]};
        g3[ax] += s ? -1.f : 1.f;
        ok = ok && load_cell(p, F, g3[0], g3[1], g3[2], ci[q][0], ci[q][1], ci[q][2], cv[q]);
        val[s] = ok ? tri(cv[q], g3[0] - ci[q][0], g3[1] - ci[q][1], g3[2] - ci[q][2]) : 0.f;
      }
      grad[ax] = (val[0] - val[1]) * 0.5f * inv_vox;
    }
    if (!ok) continue;
    const float n2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
    if (!(n2 > 0.f)) continue;
    const float Vq[3] = {dq * ry.rx, dq * ry.ry, dq};
    float df[3], r0 = 0.f;
    {
      const float in = rsqrtf(n2);
      float d2 = 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float pr = T0[4 * r] * Vq[0] + T0[4 * r + 1] * Vq[1] + T0[4 * r + 2] * Vq[2] + T0[4 * r + 3];
        df[r] = pr - v0[r];
        d2 += df[r] * df[r];
        r0 += df[r] * grad[r] * in;
      }
      if (!(d2 <= p.dist_gate2)) continue;
    }
    acc[0] += 1.f;
    acc[1] += r0 * r0;
    // ---- the 21 second-order directions ----
    for (int q = 0; q < kPairs; ++q) {
      const HD* T = sT[q];
      HD dir[3], t[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        dir[r] = ry.rx * T[4 * r] + ry.ry * T[4 * r + 1] + T[4 * r + 2];
        t[r] = T[4 * r + 3];
      }
      HD Fs[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float al = s ? an : am;
        HD f[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) f[r] = (inv_vox * (t[r] + al * dir[r])) + (-og[r] * inv_vox - 0.5f - (float)ci[s][r]);
        Fs[s] = tri_hd(cv[s], f[0], f[1], f[2]);
      }
      const HD alpha = hd(am) - p.ray_step * (Fs[0] / (Fs[1] - Fs[0]));
      HD vv[3], gg[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        vv[r] = alpha * dir[r] + t[r];
        gg[r] = (inv_vox * vv[r]) + (-og[r] * inv_vox - 0.5f);
      }
      HD gr[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        HD val[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int cq = 2 + 2 * ax + s;
          HD f[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) f[r] = gg[r] + ((r == ax ? (s ? -1.f : 1.f) : 0.f) - (float)ci[cq][r]);
          val[s] = tri_hd(cv[cq], f[0], f[1], f[2]);
        }
        gr[ax] = (0.5f * inv_vox) * (val[0] - val[1]);
      }
      const HD nn = hsqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
      const HD rn = inv(nn);
      HD res = hd(0.f);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const HD pr = Vq[0] * T[4 * r] + Vq[1] * T[4 * r + 1] + Vq[2] * T[4 * r + 2] + T[4 * r + 3];
        res = res + (pr - vv[r]) * (gr[r] * rn);
      }
      s_acc[6 + q][threadIdx.x] += 2.f * (res.a * res.d + res.b * res.c);
      if (sjk[q][0] == sjk[q][1]) s_acc[sjk[q][0]][threadIdx.x] += 2.f * res.a * res.b;
    }
  }
  // block sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 2; q < kOut; ++q) acc[q] = s_acc[q - 2][threadIdx.x];
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    float x = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    float s = 0.f;
    for (int w = 0; w < kHessThreads / 32; ++w) s += s_red[w][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: value q summed in FP64 by warp q % 4 (lanes striding over the blocks)
  __shared__ double s_sum[kOut];
  for (int q = warp; q < kOut; q += kHessThreads / 32) {
    double s = 0.0;
    for (int k = lane; k < (int)gridDim.x; k += 32) s += (double)__ldcg(&partial[(size_t)q * gridDim.x + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_sum[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double n = s_sum[0];
    const double in = n > 0 ? 1.0 / n : 0.0;
    out[0] = s_sum[1] * in;
    for (int q = 0; q < 6; ++q) out[1 + q] = s_sum[2 + q] * in;
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_sum[8 + q] * in;
    out[28] = n;
    *ticket = 0u;
  }
}

// ---------------------------------------------------------------------------------------------------
// The plain FP64 path of the same loss, gradient and Hessian: Sec. 3's bicomplex step as printed (bc.cuh:
// two imaginary units squaring to -1, every product kept, step h = 1e-20 folded into the 21 start
// poses), one thread per pixel, and every decision taken in FP64: its own march along the pixel's ray
// (the ray cast's sampling rules: samples alpha_m = m dalpha within the volume's slab, valid when the 8
// corners are observed, the first pair F_m > 0 >= F_{m+1} is the hit, F_m <= 0 < F_{m+1} ends the ray),
// the cells of the hit pair and of the six gradient samples, and the distance gate. The volume's FP32
// values are read as they are. The comparison path of the truncated FP32 kernel above.
// ---------------------------------------------------------------------------------------------------
namespace {

constexpr int kHess64Threads = 128;

// corner values (FP64) of the cell containing (gx, gy, gz); false outside the volume or unobserved
__device__ __forceinline__ bool load_cell64(const Params& p, const float* __restrict__ F, double gx, double gy,
                                            double gz, int* ijk, double* c) {
  if (!(gx >= 0.0 && gx < (double)(p.nx - 1) && gy >= 0.0 && gy < (double)(p.ny - 1) && gz >= 0.0 &&
        gz < (double)(p.nz - 1)))
    return false;
  ijk[0] = (int)gx;
  ijk[1] = (int)gy;
  ijk[2] = (int)gz;
  const CellAddr a = cell_addr(p, ijk[0], ijk[1], ijk[2]);
  const unsigned b = a.b, sx = a.dx, sy = a.dy, sz = a.dz;
  const unsigned off[8] = {0u, sx, sy, sx + sy, sz, sx + sz, sy + sz, sx + sy + sz};
  double mx = -2.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c[q] = (double)__ldg(F + b + off[q]);
    mx = fmax(mx, c[q]);
  }
  return mx <= 1.0;  // the unobserved sentinel is above 1
}

__device__ __forceinline__ double tri64(const double* c, double fx, double fy, double fz) {
  const double x00 = c[0] + fx * (c[1] - c[0]), x10 = c[2] + fx * (c[3] - c[2]);
  const double x01 = c[4] + fx * (c[5] - c[4]), x11 = c[6] + fx * (c[7] - c[6]);
  const double y0 = x00 + fy * (x10 - x00), y1 = x01 + fy * (x11 - x01);
  return y0 + fz * (y1 - y0);
}

__device__ __forceinline__ BC tri_bc(const double* c, BC fx, BC fy, BC fz) {
  BC x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = (c[2 * q + 1] - c[2 * q]) * fx + c[2 * q];
  const BC y0 = x[0] + fy * (x[1] - x[0]), y1 = x[2] + fy * (x[3] - x[2]);
  return y0 + fz * (y1 - y0);
}

// the first sample m of the ray's hit pair, -1 if none (the march of the ray cast, in FP64)
__device__ int march64(const Params& p, const float* __restrict__ F, const double* g0, const double* gd) {
  const double step = (double)p.ray_step;
  double lo = p.m0 * step, hi = p.m1 * step;
  const int nn[3] = {p.nx, p.ny, p.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (gd[a] != 0.0) {
      const double t1 = (0.0 - g0[a]) / gd[a], t2 = ((double)(nn[a] - 1) - g0[a]) / gd[a];
      lo = fmax(lo, fmin(t1, t2));
      hi = fmin(hi, fmax(t1, t2));
    } else if (!(g0[a] >= 0.0 && g0[a] < (double)(nn[a] - 1))) {
      hi = -1.0;
    }
  }
  const int m_lo = max(p.m0, (int)floor(lo / step) - 1), m_hi = min(p.m1, (int)ceil(hi / step) + 1);
  bool prev_valid = false, prev_pos = false;
  for (int m = m_lo; m <= m_hi; ++m) {
    const double al = m * step;
    int ijk[3];
    double c[8];
    const double g[3] = {g0[0] + al * gd[0], g0[1] + al * gd[1], g0[2] + al * gd[2]};
    const bool ok = load_cell64(p, F, g[0], g[1], g[2], ijk, c);
    const bool pos = ok && tri64(c, g[0] - ijk[0], g[1] - ijk[1], g[2] - ijk[2]) > 0.0;
    if (prev_valid && ok) {
      if (prev_pos && !pos) return m - 1;
      if (!prev_pos && pos) return -1;
    }
    prev_valid = ok;
    prev_pos = pos;
  }
  return -1;
}

}  // namespace

__global__ void __launch_bounds__(kHess64Threads) k_hess64(Params p, const float* __restrict__ F,
                                                          const float* __restrict__ D, const double* __restrict__ poses,
                                                          double inv_h, double* __restrict__ partial,
                                                          unsigned* __restrict__ ticket, double* __restrict__ out) {
  pdl_enter();
  __shared__ BC sT[kPairs][12];
  __shared__ int sjk[kPairs][2];
  __shared__ double s_acc[kOut][kHess64Threads];  // per-thread sums: count, E, g[6], H[21]
  __shared__ double s_red[kHess64Threads / 32][kOut];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < kPairs * 12; i += blockDim.x) {
    const double* q = poses + 4 * i;
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
  for (int q = 0; q < kOut; ++q) s_acc[q][threadIdx.x] = 0.0;
  __syncthreads();
  double T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = sT[0][e].a;
  const double inv_vox = 1.0 / (double)p.voxel, step = (double)p.ray_step;
  const double og[3] = {(double)p.ox, (double)p.oy, (double)p.oz};
  const double fx = p.fx, fy = p.fy, cx = p.cx, cy = p.cy;
  const size_t hw = (size_t)p.W * p.H;
  for (size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x; pix < hw; pix += (size_t)gridDim.x * blockDim.x) {
    const double dq = D[pix];
    if (!(dq > 0.0)) continue;
    const int u = (int)(pix % p.W), v = (int)(pix / p.W);
    const double rx = (u - cx) / fx, ry = (v - cy) / fy;
    double dir[3], g0[3], gd[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dir[r] = T0[4 * r] * rx + T0[4 * r + 1] * ry + T0[4 * r + 2];
      g0[r] = (T0[4 * r + 3] - og[r]) * inv_vox - 0.5;
      gd[r] = dir[r] * inv_vox;
    }
    const int m = march64(p, F, g0, gd);
    if (m < 0) continue;
    // ---- the real refinement: decisions and cell values ----
    double cv[8][8];
    int ci[8][3];
    const double am = m * step, an = (m + 1) * step;
    double gs[2][3];
    for (int r = 0; r < 3; ++r) {
      gs[0][r] = g0[r] + am * gd[r];
      gs[1][r] = g0[r] + an * gd[r];
    }
    if (!load_cell64(p, F, gs[0][0], gs[0][1], gs[0][2], ci[0], cv[0]) ||
        !load_cell64(p, F, gs[1][0], gs[1][1], gs[1][2], ci[1], cv[1]))
      continue;
    const double Fm = tri64(cv[0], gs[0][0] - ci[0][0], gs[0][1] - ci[0][1], gs[0][2] - ci[0][2]);
    const double Fn = tri64(cv[1], gs[1][0] - ci[1][0], gs[1][1] - ci[1][1], gs[1][2] - ci[1][2]);
    const double alpha0 = am - step * Fm / (Fn - Fm);
    double v0[3], gc[3];
    for (int r = 0; r < 3; ++r) {
      v0[r] = T0[4 * r + 3] + alpha0 * dir[r];
      gc[r] = (v0[r] - og[r]) * inv_vox - 0.5;
    }
    bool ok = true;
    double grad[3];
    for (int ax = 0; ax < 3 && ok; ++ax) {
      double val[2];
      for (int s = 0; s < 2 && ok; ++s) {
        const int q = 2 + 2 * ax + s;
        double g3[3] = {gc[0], gc[1], gc[2]};
        g3[ax] += s ? -1.0 : 1.0;
        ok = load_cell64(p, F, g3[0], g3[1], g3[2], ci[q], cv[q]);
        val[s] = ok ? tri64(cv[q], g3[0] - ci[q][0], g3[1] - ci[q][1], g3[2] - ci[q][2]) : 0.0;
      }
      grad[ax] = (val[0] - val[1]) * 0.5 * inv_vox;
    }
    if (!ok) continue;
    const double n2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
    if (!(n2 > 0.0)) continue;
    const double Vq[3] = {dq * rx, dq * ry, dq};
    double d2 = 0.0, r0 = 0.0;
    const double in = 1.0 / sqrt(n2);
    for (int r = 0; r < 3; ++r) {
      const double pr = T0[4 * r] * Vq[0] + T0[4 * r + 1] * Vq[1] + T0[4 * r + 2] * Vq[2] + T0[4 * r + 3];
      const double df = pr - v0[r];
      d2 += df * df;
      r0 += df * grad[r] * in;
    }
    if (!(d2 <= (double)p.dist_gate2)) continue;
    s_acc[0][threadIdx.x] += 1.0;
    s_acc[1][threadIdx.x] += r0 * r0;
    // ---- the 21 pairs in full bicomplex arithmetic ----
    for (int q = 0; q < kPairs; ++q) {
      const BC* T = sT[q];
      BC dq3[3], t[3];
      for (int r = 0; r < 3; ++r) {
        dq3[r] = rx * T[4 * r] + ry * T[4 * r + 1] + T[4 * r + 2];
        t[r] = T[4 * r + 3];
      }
      BC Fs[2];
      for (int s = 0; s < 2; ++s) {
        const double al = s ? an : am;
        BC f[3];
        for (int r = 0; r < 3; ++r) f[r] = inv_vox * (t[r] + al * dq3[r]) + (-og[r] * inv_vox - 0.5 - (double)ci[s][r]);
        Fs[s] = tri_bc(cv[s], f[0], f[1], f[2]);
      }
      const BC alpha = bc(am) - step * (Fs[0] * binv(Fs[1] - Fs[0]));
      BC vv[3], gg[3];
      for (int r = 0; r < 3; ++r) {
        vv[r] = alpha * dq3[r] + t[r];
        gg[r] = inv_vox * vv[r] + (-og[r] * inv_vox - 0.5);
      }
      BC gr[3];
      for (int ax = 0; ax < 3; ++ax) {
        BC val[2];
        for (int s = 0; s < 2; ++s) {
          const int cq = 2 + 2 * ax + s;
          BC f[3];
          for (int r = 0; r < 3; ++r) f[r] = gg[r] + ((r == ax ? (s ? -1.0 : 1.0) : 0.0) - (double)ci[cq][r]);
          val[s] = tri_bc(cv[cq], f[0], f[1], f[2]);
        }
        gr[ax] = (0.5 * inv_vox) * (val[0] - val[1]);
      }
      const BC rn = binv(bsqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]));
      BC res = bc(0.0);
      for (int r = 0; r < 3; ++r) {
        const BC pr = Vq[0] * T[4 * r] + Vq[1] * T[4 * r + 1] + Vq[2] * T[4 * r + 2] + T[4 * r + 3];
        res = res + (pr - vv[r]) * (gr[r] * rn);
      }
      const BC r2 = res * res;
      s_acc[8 + q][threadIdx.x] += r2.d;
      if (sjk[q][0] == sjk[q][1]) s_acc[2 + sjk[q][0]][threadIdx.x] += r2.b;
    }
  }
  // block sums (FP64), then the last block's cross-block sum in block order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < kOut; ++q) {
    double x = s_acc[q][threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int w = 0; w < kHess64Threads / 32; ++w) s += s_red[w][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) s += __ldcg(&partial[(size_t)threadIdx.x * gridDim.x + k]);
    s_red[0][threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double n = s_red[0][0];
    const double inn = n > 0 ? 1.0 / n : 0.0;
    out[0] = s_red[0][1] * inn;
    for (int q = 0; q < 6; ++q) out[1 + q] = s_red[0][2 + q] * inn * inv_h;
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_red[0][8 + q] * inn * inv_h * inv_h;
    out[28] = n;
    *ticket = 0u;
  }
}

cudaError_t launch_hess64(const Params& p, const Buffers& b, const float* depth, const double* poses, double h,
                          double* out, int nblk, cudaStream_t s) {
  // the float partial buffer holds (blocks + 4) x 27 x 16 floats: room for 29 doubles per block
  return launch_pdl(k_hess64, dim3(nblk), dim3(kHess64Threads), 0, s, p, (const float*)b.F, depth, poses, 1.0 / h,
                    reinterpret_cast<double*>(b.partial), b.ticket, out);
}

cudaError_t launch_hess(const Params& p, const Buffers& b, const float* depth, const float* poses, double* out,
                        int nblk, cudaStream_t s) {
  return launch_pdl(k_hess, dim3(nblk), dim3(kHessThreads), 0, s, p, b.F, depth, b.hit, poses, b.partial, b.ticket,
                    out);
}

}  // namespace xslam
