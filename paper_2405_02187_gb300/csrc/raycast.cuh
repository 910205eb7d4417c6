// Ray-cast helpers shared by the ray cast (raycast.cu) and the relocalisation Hessian (hess.cu):
// the real trilinear sample with its cell and validity, and the ray of a pixel in continuous voxel
// coordinates (X-SLAM Sec. 4.1, "Ray casting").
#pragma once

#include "internal.cuh"

namespace xslam {

struct Tri {
  CellAddr a;      // brick index of the min corner and the steps to its neighbours
  float fx, fy, fz;
  float val;       // trilinear F (real lane)
  float g[3];      // d val / d g (continuous voxel coordinates)
};

// Cell and real trilinear value at continuous voxel coordinate (gx, gy, gz). Returns false if the
// cell is outside the volume or a corner is unobserved.
__device__ __forceinline__ bool tri_real(const Params& p, const float* __restrict__ F, float gx, float gy, float gz,
                                         Tri& t, bool want_grad) {
  if (!(gx >= 0.f && gx < (float)(p.nx - 1) && gy >= 0.f && gy < (float)(p.ny - 1) && gz >= 0.f &&
        gz < (float)(p.nz - 1)))
    return false;
  const int i = (int)gx, j = (int)gy, k = (int)gz;  // gx >= 0: truncation is floor
  const CellAddr a = cell_addr(p, i, j, k);
  const unsigned b = a.b, sx = a.dx, sy = a.dy, sz = a.dz;
  const float c000 = __ldg(F + b), c100 = __ldg(F + b + sx), c010 = __ldg(F + b + sy), c110 = __ldg(F + b + sx + sy);
  const float c001 = __ldg(F + b + sz), c101 = __ldg(F + b + sx + sz), c011 = __ldg(F + b + sy + sz),
              c111 = __ldg(F + b + sx + sy + sz);
  const float mx = fmaxf(fmaxf(fmaxf(c000, c100), fmaxf(c010, c110)), fmaxf(fmaxf(c001, c101), fmaxf(c011, c111)));
  if (!(mx <= 1.f)) return false;  // an unobserved corner
  const float fx = gx - i, fy = gy - j, fz = gz - k;
  const float x00 = c000 + fx * (c100 - c000), x10 = c010 + fx * (c110 - c010);
  const float x01 = c001 + fx * (c101 - c001), x11 = c011 + fx * (c111 - c011);
  const float y0 = x00 + fy * (x10 - x00), y1 = x01 + fy * (x11 - x01);
  t.val = y0 + fz * (y1 - y0);
  t.a = a;
  t.fx = fx;
  t.fy = fy;
  t.fz = fz;
  if (want_grad) {
    const float dx00 = c100 - c000, dx10 = c110 - c010, dx01 = c101 - c001, dx11 = c111 - c011;
    t.g[0] = (1.f - fz) * ((1.f - fy) * dx00 + fy * dx10) + fz * ((1.f - fy) * dx01 + fy * dx11);
    t.g[1] = (1.f - fz) * (x10 - x00) + fz * (x11 - x01);
    t.g[2] = y1 - y0;
  }
  return true;
}

// The march's sample: validity and real trilinear value from the linear-layout copy of Re F (the
// brick layout's index arithmetic would cost more than the march's loads, which hit L1), in two parts so
// that several samples of a ray have their corner loads in flight at once. The cell is inside the volume
// iff floor(g) lies in [0, n - 2] on every axis (the same test as 0 <= g < n - 1 for finite g; a
// rounding-down conversion and one unsigned compare per axis). march_load issues the 8 corner loads
// without a branch: a sample outside the volume (or past the ray's last one, live = false) reads cell 0
// (inside the volume: every axis has at least 2 voxels) and is marked out. An unobserved corner holds a NaN, which every lerp of march_value carries to the
// value, so validity is the sample being in and its value a number.
struct MarchSample {
  float c[8];  // corners c[dx + 2 dy + 4 dz]
  float fx, fy, fz;
  bool in;
};

__device__ __forceinline__ void march_load(const Params& p, const float* __restrict__ Flin, float gx, float gy, float gz,
                                           bool live, MarchSample& s) {
  const int i = __float2int_rd(gx), j = __float2int_rd(gy), k = __float2int_rd(gz);
  s.in = live && (unsigned)i < (unsigned)(p.nx - 1) && (unsigned)j < (unsigned)(p.ny - 1) &&
         (unsigned)k < (unsigned)(p.nz - 1);
  const unsigned sy = (unsigned)p.nx, sz = (unsigned)p.nx * (unsigned)p.ny;
  const unsigned b = s.in ? (unsigned)i + sy * (unsigned)j + sz * (unsigned)k : 0u;
  s.fx = gx - i;
  s.fy = gy - j;
  s.fz = gz - k;
  s.c[0] = __ldg(Flin + b);
  s.c[1] = __ldg(Flin + b + 1);
  s.c[2] = __ldg(Flin + b + sy);
  s.c[3] = __ldg(Flin + b + 1 + sy);
  s.c[4] = __ldg(Flin + b + sz);
  s.c[5] = __ldg(Flin + b + 1 + sz);
  s.c[6] = __ldg(Flin + b + sy + sz);
  s.c[7] = __ldg(Flin + b + 1 + sy + sz);
}

__device__ __forceinline__ bool march_value(const MarchSample& s, float& val) {
  const float x00 = s.c[0] + s.fx * (s.c[1] - s.c[0]), x10 = s.c[2] + s.fx * (s.c[3] - s.c[2]);
  const float x01 = s.c[4] + s.fx * (s.c[5] - s.c[4]), x11 = s.c[6] + s.fx * (s.c[7] - s.c[6]);
  const float y0 = x00 + s.fy * (x10 - x00), y1 = x01 + s.fy * (x11 - x01);
  val = y0 + s.fz * (y1 - y0);
  return s.in && val == val;  // false outside, or for a NaN: an unobserved corner
}

// Imaginary part of the trilinear F on lane plane Fl at the cell of t, with the sample position
// moving by gl (voxel units): grad . gl + sum_c w_c Im F_c.
__device__ __forceinline__ float tri_lane(const Params& p, const float* __restrict__ Fl, const Tri& t, float glx,
                                          float gly, float glz) {
  float v = t.g[0] * glx + t.g[1] * gly + t.g[2] * glz;
  if (Fl) {
    const unsigned b = t.a.b, sx = t.a.dx, sy = t.a.dy, sz = t.a.dz;
    const float x00 = __ldg(Fl + b) + t.fx * (__ldg(Fl + b + sx) - __ldg(Fl + b));
    const float x10 = __ldg(Fl + b + sy) + t.fx * (__ldg(Fl + b + sx + sy) - __ldg(Fl + b + sy));
    const float x01 = __ldg(Fl + b + sz) + t.fx * (__ldg(Fl + b + sx + sz) - __ldg(Fl + b + sz));
    const float x11 = __ldg(Fl + b + sy + sz) + t.fx * (__ldg(Fl + b + sx + sy + sz) - __ldg(Fl + b + sy + sz));
    const float y0 = x00 + t.fy * (x10 - x00), y1 = x01 + t.fy * (x11 - x01);
    v += y0 + t.fz * (y1 - y0);
  }
  return v;
}

// The ray of pixel (u, v) in continuous voxel coordinates: g(alpha) = g0 + alpha * gd (real pose).
struct Ray {
  float rx, ry;               // K^-1 (u, v, 1)
  float dirx, diry, dirz;     // R K^-1 (u, v, 1)
  float g0x, g0y, g0z, gdx, gdy, gdz;
};

__device__ __forceinline__ Ray make_ray(const Params& p, const float* T, int u, int v) {
  Ray r;
  r.rx = (u - p.cx) / p.fx;
  r.ry = (v - p.cy) / p.fy;
  r.dirx = T[0] * r.rx + T[1] * r.ry + T[2];
  r.diry = T[4] * r.rx + T[5] * r.ry + T[6];
  r.dirz = T[8] * r.rx + T[9] * r.ry + T[10];
  const float inv_vox = 1.f / p.voxel;
  r.g0x = (T[3] - p.ox) * inv_vox - 0.5f;
  r.g0y = (T[7] - p.oy) * inv_vox - 0.5f;
  r.g0z = (T[11] - p.oz) * inv_vox - 0.5f;
  r.gdx = r.dirx * inv_vox;
  r.gdy = r.diry * inv_vox;
  r.gdz = r.dirz * inv_vox;
  return r;
}

}  // namespace xslam
