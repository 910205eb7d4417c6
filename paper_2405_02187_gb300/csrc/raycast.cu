// Ray casting of the TSDF (X-SLAM Sec. 4.1, "Ray casting"; Eq. surface_prediction) on 1 + K lanes.
//
// Pixel u casts r(alpha) = alpha R K^-1 u_dot + t with alpha the camera depth. Samples sit at
// alpha_m = m * dalpha (m0 <= m <= m1); a sample is valid if its trilinear cell is inside the volume
// and its 8 corners are observed (W > 0). The march uses real parts only: the first pair of
// consecutive valid samples with F_m > 0 >= F_{m+1} is the hit; a pair with F_m <= 0 < F_{m+1} ends
// the ray. The hit pair is re-evaluated on every lane (complex pose, complex TSDF, same cells):
// alpha0 = alpha_m - dalpha F_m / (F_{m+1} - F_m), V_g = r(alpha0), N_g = grad F / |grad F| from
// central differences of the trilinear F at V_g +- one voxel per axis.
// Samples outside the volume are invalid, so the march starts and stops at the volume's bounds
// (widened by one sample), which visits every valid sample in the same order. In the march's linear
// copy of Re F an unobserved voxel holds a quiet NaN, which the trilinear interpolation carries to the
// sample: a sample's validity and value come from the 8 loads alone.
// Two kernels: k_march (real lane only; each thread keeps the corner loads of 4 consecutive samples in
// flight to hide the gather latency) records per pixel the index of the hit pair's first sample; k_refine
// re-evaluates the pair and the six normal samples on every lane and writes the model maps.
#include "internal.cuh"
#include "raycast.cuh"

namespace xslam {

constexpr int kMarchU = 4;  // samples of a ray whose corner loads are in flight together

// (bx, by): this block's coordinates in its trajectory's 2-D grid
__device__ __forceinline__ void march_body(const Params& p, const float* __restrict__ F, const double* __restrict__ pose,
                                           int* __restrict__ hit, int bx, int by) {
  __shared__ float sT[12];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if (tid < 12) sT[tid] = (float)pose[tid];
  __syncthreads();
  const int u = bx * blockDim.x + threadIdx.x;
  const int v = by * blockDim.y + threadIdx.y;
  if (u >= p.W || v >= p.H) return;
  const Ray ry = make_ray(p, sT, u, v);
  // alpha interval where 0 <= g < n - 1 on every axis (slab test), widened by one sample
  float lo = p.m0 * p.ray_step, hi = p.m1 * p.ray_step;
  {
    const float g0[3] = {ry.g0x, ry.g0y, ry.g0z}, gd[3] = {ry.gdx, ry.gdy, ry.gdz};
    const int nn[3] = {p.nx, p.ny, p.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (gd[a] != 0.f) {
        const float t1 = (0.f - g0[a]) / gd[a], t2 = ((float)(nn[a] - 1) - g0[a]) / gd[a];
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
      } else if (!(g0[a] >= 0.f && g0[a] < (float)(nn[a] - 1))) {
        hi = -1.f;
      }
    }
  }
  const int m_lo = max(p.m0, (int)floorf(lo / p.ray_step) - 1);
  const int m_hi = min(p.m1, (int)ceilf(hi / p.ray_step) + 1);
  // kMarchU samples per trip: all their corner loads are issued before the first is tested (the march
  // is bound by the latency of those loads); the samples are then taken in order, as one at a time
  int m_hit = -1;
  bool prev_valid = false, prev_pos = false;
  for (int m0 = m_lo; m0 <= m_hi; m0 += kMarchU) {
    MarchSample sm[kMarchU];
#pragma unroll
    for (int q = 0; q < kMarchU; ++q) {
      const float al = (m0 + q) * p.ray_step;
      march_load(p, F, ry.g0x + al * ry.gdx, ry.g0y + al * ry.gdy, ry.g0z + al * ry.gdz, m0 + q <= m_hi, sm[q]);
    }
    bool stop = false;
#pragma unroll
    for (int q = 0; q < kMarchU; ++q) {
      if (stop || m0 + q > m_hi) continue;
      float val;
      const bool ok = march_value(sm[q], val);
      if (prev_valid && ok) {
        const bool pos = val > 0.f;
        if (prev_pos && !pos) {  // the hit pair: samples m - 1 and m
          m_hit = m0 + q - 1;
          stop = true;
          continue;
        }
        if (!prev_pos && pos) {  // from behind a surface into free space: no hit
          stop = true;
          continue;
        }
      }
      prev_valid = ok;
      prev_pos = ok && val > 0.f;
    }
    if (stop) break;
  }
  hit[(size_t)v * p.W + u] = m_hit;
}

__global__ void __launch_bounds__(256) k_march(Params p, const float* __restrict__ F, const double* __restrict__ pose,
                                               int* __restrict__ hit) {
  pdl_enter();
  march_body(p, F, pose, hit, blockIdx.x, blockIdx.y);
}

// segments: nblk = blocks of the trajectory's grid, arg = its width in blocks
__global__ void __launch_bounds__(256) k_march_seg(SegTable st) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  const int lb = blockIdx.x - sg.block0;
  march_body(d.p, d.b.F0lin, d.b.pose, d.b.hit, lb % sg.arg, lb / sg.arg);
}

__device__ __forceinline__ void refine_body(const Params& p, const float* __restrict__ F,
                                            const double* __restrict__ pose, const int* __restrict__ hit,
                                            float* __restrict__ out_depth, float* __restrict__ vmap,
                                            float* __restrict__ nmap, int ignore_imag, double* __restrict__ pose_prev,
                                            unsigned long long* __restrict__ hits, int bx, int by) {
  __shared__ float sT[kMaxLanes][12];
  for (int i = threadIdx.x + blockDim.x * threadIdx.y; i < p.L * 12; i += blockDim.x * blockDim.y) {
    sT[i / 12][i % 12] = (float)pose[i];
    if (pose_prev && bx == 0 && by == 0) pose_prev[i] = pose[i];
  }
  __syncthreads();
  const int u = bx * blockDim.x + threadIdx.x;
  const int v = by * blockDim.y + threadIdx.y;
  if (u >= p.W || v >= p.H) return;
  const size_t hw = (size_t)p.W * p.H;
  const size_t pix = (size_t)v * p.W + u;
  const size_t n = vox_plane(p);
  const float* T = sT[0];
  const Ray ry = make_ray(p, T, u, v);
  const float inv_vox = 1.f / p.voxel;
  const int m_hit = hit[pix];

  bool good = false;
  float alpha0 = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, nrm = 1.f;
  Tri tm, tn, ts[6];
  float am = 0.f, an = 0.f, den = 1.f;
  if (m_hit >= 0) {
    am = m_hit * p.ray_step;
    an = (m_hit + 1) * p.ray_step;
    bool ok = tri_real(p, F, ry.g0x + am * ry.gdx, ry.g0y + am * ry.gdy, ry.g0z + am * ry.gdz, tm, true);
    ok &= tri_real(p, F, ry.g0x + an * ry.gdx, ry.g0y + an * ry.gdy, ry.g0z + an * ry.gdz, tn, true);
    if (ok) {
      den = tn.val - tm.val;
      alpha0 = am - p.ray_step * tm.val / den;
      vx = T[3] + alpha0 * ry.dirx;
      vy = T[7] + alpha0 * ry.diry;
      vz = T[11] + alpha0 * ry.dirz;
      const float gx = (vx - p.ox) * inv_vox - 0.5f, gy = (vy - p.oy) * inv_vox - 0.5f,
                  gz = (vz - p.oz) * inv_vox - 0.5f;
      ok &= tri_real(p, F, gx + 1.f, gy, gz, ts[0], true);
      ok &= tri_real(p, F, gx - 1.f, gy, gz, ts[1], true);
      ok &= tri_real(p, F, gx, gy + 1.f, gz, ts[2], true);
      ok &= tri_real(p, F, gx, gy - 1.f, gz, ts[3], true);
      ok &= tri_real(p, F, gx, gy, gz + 1.f, ts[4], true);
      ok &= tri_real(p, F, gx, gy, gz - 1.f, ts[5], true);
      if (ok) {
        const float s = 0.5f * inv_vox;
        nx = (ts[0].val - ts[1].val) * s;
        ny = (ts[2].val - ts[3].val) * s;
        nz = (ts[4].val - ts[5].val) * s;
        const float n2 = nx * nx + ny * ny + nz * nz;
        if (n2 > 0.f) {
          nrm = sqrtf(n2);
          good = true;
        }
      }
    }
  }
  if (out_depth) out_depth[pix] = good ? alpha0 : 0.f;
  if (hits) {
    const unsigned m = __ballot_sync(__activemask(), good);
    if (good && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(hits, (unsigned long long)__popc(m));
  }
  if (!vmap && !nmap) return;
  if (!good) {
    for (int l = 0; l < p.L; ++l)
      for (int c = 0; c < 3; ++c) {
        if (vmap) vmap[(size_t)(3 * l + c) * hw + pix] = 0.f;
        if (nmap) nmap[(size_t)(3 * l + c) * hw + pix] = 0.f;
      }
    return;
  }
  const float Nx = nx / nrm, Ny = ny / nrm, Nz = nz / nrm;
  if (vmap) {
    vmap[pix] = vx;
    vmap[hw + pix] = vy;
    vmap[2 * hw + pix] = vz;
  }
  if (nmap) {
    nmap[pix] = Nx;
    nmap[hw + pix] = Ny;
    nmap[2 * hw + pix] = Nz;
  }
  const float s = 0.5f * inv_vox;
  for (int l = 1; l < p.L; ++l) {
    const float* Tl = sT[l];
    const float* Fl = ignore_imag ? nullptr : F + (size_t)l * n;
    const float dlx = Tl[0] * ry.rx + Tl[1] * ry.ry + Tl[2];
    const float dly = Tl[4] * ry.rx + Tl[5] * ry.ry + Tl[6];
    const float dlz = Tl[8] * ry.rx + Tl[9] * ry.ry + Tl[10];
    // sample positions move by alpha * dir_l + t_l
    const float Fm_l = tri_lane(p, Fl, tm, (am * dlx + Tl[3]) * inv_vox, (am * dly + Tl[7]) * inv_vox,
                                (am * dlz + Tl[11]) * inv_vox);
    const float Fn_l = tri_lane(p, Fl, tn, (an * dlx + Tl[3]) * inv_vox, (an * dly + Tl[7]) * inv_vox,
                                (an * dlz + Tl[11]) * inv_vox);
    const float a0_l = -p.ray_step * (Fm_l * tn.val - tm.val * Fn_l) / (den * den);
    const float vlx = a0_l * ry.dirx + alpha0 * dlx + Tl[3];
    const float vly = a0_l * ry.diry + alpha0 * dly + Tl[7];
    const float vlz = a0_l * ry.dirz + alpha0 * dlz + Tl[11];
    const float glx = vlx * inv_vox, gly = vly * inv_vox, glz = vlz * inv_vox;
    const float gxl = (tri_lane(p, Fl, ts[0], glx, gly, glz) - tri_lane(p, Fl, ts[1], glx, gly, glz)) * s;
    const float gyl = (tri_lane(p, Fl, ts[2], glx, gly, glz) - tri_lane(p, Fl, ts[3], glx, gly, glz)) * s;
    const float gzl = (tri_lane(p, Fl, ts[4], glx, gly, glz) - tri_lane(p, Fl, ts[5], glx, gly, glz)) * s;
    const float dot = Nx * gxl + Ny * gyl + Nz * gzl;
    if (vmap) {
      vmap[(size_t)(3 * l) * hw + pix] = vlx;
      vmap[(size_t)(3 * l + 1) * hw + pix] = vly;
      vmap[(size_t)(3 * l + 2) * hw + pix] = vlz;
    }
    if (nmap) {
      nmap[(size_t)(3 * l) * hw + pix] = (gxl - Nx * dot) / nrm;
      nmap[(size_t)(3 * l + 1) * hw + pix] = (gyl - Ny * dot) / nrm;
      nmap[(size_t)(3 * l + 2) * hw + pix] = (gzl - Nz * dot) / nrm;
    }
  }
}

__global__ void __launch_bounds__(256) k_refine(Params p, const float* __restrict__ F, const double* __restrict__ pose,
                                                const int* __restrict__ hit, float* __restrict__ out_depth,
                                                float* __restrict__ vmap, float* __restrict__ nmap, int ignore_imag,
                                                double* __restrict__ pose_prev, unsigned long long* __restrict__ hits) {
  pdl_enter();
  refine_body(p, F, pose, hit, out_depth, vmap, nmap, ignore_imag, pose_prev, hits, blockIdx.x, blockIdx.y);
}

// the frame chain's refinement of every segment: the model maps of its handle, T_{k-1} := T_k
__global__ void __launch_bounds__(256) k_refine_seg(SegTable st) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  const Buffers& b = d.b;
  const size_t hw = (size_t)d.p.W * d.p.H;
  const int lb = blockIdx.x - sg.block0;
  refine_body(d.p, b.F, b.pose, b.hit, b.model, b.model + hw, b.model + hw * (1 + 3 * d.p.L), 0, b.pose_prev,
              b.stats + 1, lb % sg.arg, lb / sg.arg);
}

cudaError_t launch_raycast_seg(const SegTable& t, int nblocks, int tile_w, cudaStream_t s) {
  const dim3 blk(tile_w, 256 / tile_w);
  cudaError_t e = launch_pdl(k_march_seg, dim3(nblocks), blk, 0, s, t);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_refine_seg, dim3(nblocks), blk, 0, s, t);
}

cudaError_t launch_march(const Params& p, const Buffers& b, const double* pose, cudaStream_t s) {
  dim3 blk(32, 8), grd((p.W + 31) / 32, (p.H + 7) / 8);
  return launch_pdl(k_march, grd, blk, 0, s, p, b.F0lin, pose, b.hit);
}

cudaError_t launch_raycast(const Params& p, const Buffers& b, const double* pose, float* depth, float* vmap,
                           float* nmap, bool ignore_imag_volume, bool set_prev, cudaStream_t s) {
  dim3 blk(32, 8), grd((p.W + 31) / 32, (p.H + 7) / 8);
  cudaError_t e = launch_pdl(k_march, grd, blk, 0, s, p, b.F0lin, pose, b.hit);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_refine, grd, blk, 0, s, p, b.F, pose, b.hit, depth, vmap, nmap, ignore_imag_volume ? 1 : 0,
                    set_prev ? b.pose_prev : nullptr, set_prev ? b.stats + 1 : nullptr);
}

}  // namespace xslam
