// Plain FP64 complex-step X-KinectFusion (include/xslam_plain.h): the comparison path.
//
// X-SLAM's scheme taken literally: the frame step of Sec. 4.1 in complex<double> with the full complex
// products of Eq. csfd, one complex run per perturbation (Sec. 6, "perturbing variables one by
// one"), each run with its own array-of-structures volume (Re F, Im F, W per voxel), pose, pyramid,
// vertex/normal maps and model maps. One thread per pixel or voxel, every voxel visited by the TSDF
// update, the march evaluated on complex samples, one launch per step, no CUDA graphs. Discrete
// decisions (validity, gates, cells, the zero crossing) are taken on real parts and the imaginary
// part follows the chosen branch; the readings are those of the batched FP32 path (xslam.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/xslam_plain.h"

namespace {

// ---------------------------------------------------------------------------------------------
// complex<double> with the full products (Sec. 3, Eq. csfd)
// ---------------------------------------------------------------------------------------------
struct cd {
  double r, i;
};
__host__ __device__ inline cd C(double r, double i = 0.0) { return {r, i}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return {a.r + b.r, a.i + b.i}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return {a.r - b.r, a.i - b.i}; }
__host__ __device__ inline cd operator-(cd a) { return {-a.r, -a.i}; }
__host__ __device__ inline cd operator*(cd a, cd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__host__ __device__ inline cd operator*(double s, cd a) { return {s * a.r, s * a.i}; }
__host__ __device__ inline cd operator*(cd a, double s) { return {s * a.r, s * a.i}; }
__host__ __device__ inline cd operator/(cd a, cd b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__host__ __device__ inline cd operator/(cd a, double s) { return {a.r / s, a.i / s}; }
__host__ __device__ inline cd& operator+=(cd& a, cd b) {
  a.r += b.r;
  a.i += b.i;
  return a;
}
__device__ inline double cabs_(cd z) { return hypot(z.r, z.i); }
// principal square root
__device__ inline cd csqrt_(cd z) {
  const double m = hypot(z.r, z.i);
  if (m == 0.0) return C(0.0);
  if (z.r >= 0.0) {
    const double t = sqrt(0.5 * (m + z.r));
    return C(t, z.i / (2.0 * t));
  }
  const double t = sqrt(0.5 * (m - z.r));
  return C(fabs(z.i) / (2.0 * t), copysign(t, z.i));
}
__device__ inline cd cexp_(cd z) {
  double s, c;
  sincos(z.i, &s, &c);
  const double e = exp(z.r);
  return C(e * c, e * s);
}
__device__ inline cd csin_(cd z) {
  double s, c;
  sincos(z.r, &s, &c);
  return C(s * cosh(z.i), c * sinh(z.i));
}
__device__ inline cd ccos_(cd z) {
  double s, c;
  sincos(z.r, &s, &c);
  return C(c * cosh(z.i), -s * sinh(z.i));
}

struct PP {
  int nx, ny, nz, W, H, levels;
  int iters[4];
  double voxel, ox, oy, oz, fx, fy, cx, cy;
  double dist_gate, cos_gate, disc_gate, min_corr_frac, depth_min, depth_max, pyr_range, ray_step, w_max;
  int bilateral, m0, m1;
};

constexpr int kT = 256;      // threads per block everywhere
constexpr int kNV = 55;      // ICP partial: 27 complex values (54 doubles) + the count
constexpr double kCellBias = 0.015625;  // 2^-6: bilinear cell tie-break of the ICP lookup

// ---------------------------------------------------------------------------------------------
// SE(3) (Sec. 4.1, Eq. lie / rotvector / rotation_jacobi; plain transpose, theta^2 = phi . phi)
// ---------------------------------------------------------------------------------------------
__device__ void hat3(const cd* v, cd* M) {
  M[0] = C(0.0); M[1] = -v[2]; M[2] = v[1];
  M[3] = v[2]; M[4] = C(0.0); M[5] = -v[0];
  M[6] = -v[1]; M[7] = v[0]; M[8] = C(0.0);
}
__device__ void mat3mul(const cd* A, const cd* B, cd* O) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) O[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}
// T = exp(xi) as a 3x4 [R | V rho]
__device__ void cse3_exp(const cd* xi, cd* T) {
  const cd* phi = xi;
  const cd th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  cd R[9], V[9];
  if (cabs_(th2) < 1e-4) {
    // exponential power series: R = sum P^n / n!, V = sum P^n / (n + 1)!
    cd P[9], term[9], tmp[9];
    hat3(phi, P);
    for (int e = 0; e < 9; ++e) {
      const double id = (e % 4 == 0) ? 1.0 : 0.0;
      R[e] = C(id);
      V[e] = C(id);
      term[e] = C(id);
    }
    double f0 = 1.0, f1 = 1.0;  // n!, (n + 1)!
    for (int n = 1; n < 12; ++n) {
      mat3mul(term, P, tmp);
      for (int e = 0; e < 9; ++e) term[e] = tmp[e];
      f0 *= n;
      f1 *= (n + 1);
      for (int e = 0; e < 9; ++e) {
        R[e] += term[e] / f0;
        V[e] += term[e] / f1;
      }
    }
  } else {
    const cd th = csqrt_(th2);
    cd a[3] = {phi[0] / th, phi[1] / th, phi[2] / th};
    const cd c = ccos_(th), s = csin_(th);
    const cd sa = s / th, ca = (C(1.0) - c) / th;
    cd Ah[9];
    hat3(a, Ah);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) {
        const cd aa = a[r] * a[q];
        const cd id = C(r == q ? 1.0 : 0.0);
        R[3 * r + q] = c * id + (C(1.0) - c) * aa + s * Ah[3 * r + q];
        V[3 * r + q] = sa * id + (C(1.0) - sa) * aa + ca * Ah[3 * r + q];
      }
  }
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) T[4 * r + q] = R[3 * r + q];
    T[4 * r + 3] = V[3 * r] * xi[3] + V[3 * r + 1] * xi[4] + V[3 * r + 2] * xi[5];
  }
}
// O = A * B for 3x4 rigid transforms
__device__ void ccompose(const cd* A, const cd* B, cd* O) {
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      cd v = A[4 * r] * B[c] + A[4 * r + 1] * B[4 + c] + A[4 * r + 2] * B[8 + c];
      if (c == 3) v += A[4 * r + 3];
      O[4 * r + c] = v;
    }
  }
}
// T^-1 = [R^T | -R^T t]
__device__ void cinverse(const cd* T, cd* O) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) O[4 * r + c] = T[4 * c + r];
  for (int r = 0; r < 3; ++r) O[4 * r + 3] = -(O[4 * r] * T[3] + O[4 * r + 1] * T[7] + O[4 * r + 2] * T[11]);
}
__device__ inline void cxform(const cd* T, const cd* p, cd* o) {
  for (int r = 0; r < 3; ++r) o[r] = T[4 * r] * p[0] + T[4 * r + 1] * p[1] + T[4 * r + 2] * p[2] + T[4 * r + 3];
}

// ---------------------------------------------------------------------------------------------
// surface measurement (Sec. 4.1)
// ---------------------------------------------------------------------------------------------
__global__ void k_p_fill(double* vox, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    vox[3 * i] = 1.0;
    vox[3 * i + 1] = 0.0;
    vox[3 * i + 2] = 0.0;
  }
}

// D* = D + hD i on valid pixels (Eq. csfd_depth), then the range gate on the real part
__global__ void k_p_gate(const float* __restrict__ depth, cd* __restrict__ out, int n, double hD, double dmin,
                         double dmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = depth[i];
  const cd D = d > 0.0 ? C(d, hD) : C(0.0);
  out[i] = (D.r >= dmin && D.r <= dmax) ? D : C(0.0);
}

// 7x7 bilateral filter over valid taps, Gaussian spatial (4.5 px) and range (0.03 m) weights
// evaluated on the complex depths
__global__ void k_p_bilateral(const cd* __restrict__ in, cd* __restrict__ out, int W, int H) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int u = p % W, v = p / W;
  const cd c = in[p];
  if (!(c.r > 0.0)) {
    out[p] = C(0.0);
    return;
  }
  const double ss = 2.0 * 4.5 * 4.5, sr = 2.0 * 0.03 * 0.03;
  cd acc = C(0.0), ws = C(0.0);
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      const int x = u + dx, y = v + dy;
      if (x < 0 || x >= W || y < 0 || y >= H) continue;
      const cd t = in[y * W + x];
      if (!(t.r > 0.0)) continue;
      const cd d = t - c;
      const cd w = cexp_(C(-(dx * dx + dy * dy) / ss) - (d * d) / sr);
      acc += w * t;
      ws += w;
    }
  out[p] = acc / ws;
}

// level l+1 at (u, v): 5x5 binomial over taps around (2u, 2v) that are valid and within range of the
// centre; invalid at an invalid centre
__global__ void k_p_pyr_down(const cd* __restrict__ in, int Wi, int Hi, cd* __restrict__ out, int Wo, int Ho,
                             double range) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Wo * Ho) return;
  const int u = p % Wo, v = p / Wo;
  const double B[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
  const cd c = in[(2 * v) * Wi + 2 * u];
  if (!(c.r > 0.0)) {
    out[p] = C(0.0);
    return;
  }
  cd acc = C(0.0);
  double ws = 0.0;
  for (int dy = -2; dy <= 2; ++dy)
    for (int dx = -2; dx <= 2; ++dx) {
      const int x = 2 * u + dx, y = 2 * v + dy;
      if (x < 0 || x >= Wi || y < 0 || y >= Hi) continue;
      const cd t = in[y * Wi + x];
      if (!(t.r > 0.0 && fabs(t.r - c.r) < range)) continue;
      const double w = B[dy + 2] * B[dx + 2];
      acc += w * t;
      ws += w;
    }
  out[p] = acc / ws;
}

// V = D K^-1 u (Eq. vertex); N = normalised cross product of the forward differences (Eq. normal)
__global__ void k_p_vertex_normal(const cd* __restrict__ D, int W, int H, double fx, double fy, double cx, double cy,
                                  cd* __restrict__ vn, unsigned char* __restrict__ valid) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int u = p % W, v = p / W;
  auto vert = [&](int x, int y, cd* o) {
    const cd d = D[y * W + x];
    o[0] = d * ((x - cx) / fx);
    o[1] = d * ((y - cy) / fy);
    o[2] = d;
  };
  cd V[3];
  vert(u, v, V);
  bool ok = u < W - 1 && v < H - 1 && D[p].r > 0.0;
  cd N[3] = {C(0.0), C(0.0), C(0.0)};
  if (ok) ok = D[p + 1].r > 0.0 && D[p + W].r > 0.0;
  if (ok) {
    cd Vx[3], Vy[3], ex[3], ey[3];
    vert(u + 1, v, Vx);
    vert(u, v + 1, Vy);
    for (int r = 0; r < 3; ++r) {
      ex[r] = Vx[r] - V[r];
      ey[r] = Vy[r] - V[r];
    }
    const cd c[3] = {ex[1] * ey[2] - ex[2] * ey[1], ex[2] * ey[0] - ex[0] * ey[2], ex[0] * ey[1] - ex[1] * ey[0]};
    const cd n2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    ok = n2.r > 0.0;
    if (ok) {
      const cd nn = csqrt_(n2);
      for (int r = 0; r < 3; ++r) N[r] = c[r] / nn;
    }
  }
  for (int r = 0; r < 3; ++r) {
    vn[6 * (size_t)p + r] = V[r];
    vn[6 * (size_t)p + 3 + r] = N[r];
  }
  valid[p] = ok ? 1 : 0;
}

// ---------------------------------------------------------------------------------------------
// ICP (Sec. 4.1, Eq. icp / "icp approx"): per-pixel residual and Jacobian, per-block sums
// ---------------------------------------------------------------------------------------------
struct Lv {
  int W, H, s;
  double fx, fy, cx, cy;
};

__global__ void __launch_bounds__(kT) k_p_icp(PP p, Lv lv, const cd* __restrict__ vn, const unsigned char* __restrict__ nvalid,
                                              const double* __restrict__ mdep, const cd* __restrict__ mvn,
                                              const cd* __restrict__ Tj_g, const cd* __restrict__ Tprev_g,
                                              double* __restrict__ part, const int* __restrict__ st) {
  if (st[0]) return;  // this frame's ICP already failed
  __shared__ cd sT[12], sI[12];
  __shared__ double s_red[kT / 32][kNV];
  if (threadIdx.x < 12) sT[threadIdx.x] = Tj_g[threadIdx.x];
  if (threadIdx.x == 0) {
    cd Tp[12];
    for (int e = 0; e < 12; ++e) Tp[e] = Tprev_g[e];
    cinverse(Tp, sI);
  }
  __syncthreads();
  cd acc[27];
  for (int q = 0; q < 27; ++q) acc[q] = C(0.0);
  double cnt = 0.0;
  const int npx = lv.W * lv.H;
  const int W0 = p.W;
  for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < npx; px += gridDim.x * blockDim.x) {
    if (!nvalid[px]) continue;
    const cd* V = vn + 6 * (size_t)px;
    cd pp[3], pc[3];
    cxform(sT, V, pp);
    cxform(sI, pp, pc);
    const cd z = pc[2];
    if (!(z.r > 0.0)) continue;
    const cd ux = lv.fx * pc[0] / z + C(lv.cx), uy = lv.fy * pc[1] / z + C(lv.cy);
    const double ci = floor(ux.r + kCellBias), cj = floor(uy.r + kCellBias);
    if (!(ci >= 0.0 && ci <= lv.W - 2 && cj >= 0.0 && cj <= lv.H - 2)) continue;
    const cd a = ux - C(ci), b = uy - C(cj);
    const size_t t00 = (size_t)((int)cj * lv.s) * W0 + (size_t)((int)ci * lv.s);
    const size_t t10 = t00 + lv.s, t01 = t00 + (size_t)lv.s * W0, t11 = t01 + lv.s;
    const double d00 = mdep[t00], d10 = mdep[t10], d01 = mdep[t01], d11 = mdep[t11];
    if (!(d00 > 0.0 && d10 > 0.0 && d01 > 0.0 && d11 > 0.0)) continue;
    if (!(fabs(d10 - d00) + fabs(d01 - d00) + fabs(d11 - d00) < p.disc_gate)) continue;
    const cd w00 = (C(1.0) - a) * (C(1.0) - b), w10 = a * (C(1.0) - b), w01 = (C(1.0) - a) * b, w11 = a * b;
    cd q[3], n[3];
    for (int r = 0; r < 3; ++r) {
      q[r] = w00 * mvn[6 * t00 + r] + w10 * mvn[6 * t10 + r] + w01 * mvn[6 * t01 + r] + w11 * mvn[6 * t11 + r];
      n[r] = w00 * mvn[6 * t00 + 3 + r] + w10 * mvn[6 * t10 + 3 + r] + w01 * mvn[6 * t01 + 3 + r] +
             w11 * mvn[6 * t11 + 3 + r];
    }
    cd diff[3];
    double d2 = 0.0;
    for (int r = 0; r < 3; ++r) {
      diff[r] = pp[r] - q[r];
      d2 += diff[r].r * diff[r].r;
    }
    if (!(d2 <= p.dist_gate * p.dist_gate)) continue;
    double nw[3], nre2 = 0.0, dot = 0.0;
    for (int r = 0; r < 3; ++r) {
      nw[r] = V[3].r * sT[4 * r].r + V[4].r * sT[4 * r + 1].r + V[5].r * sT[4 * r + 2].r;
      nre2 += n[r].r * n[r].r;
      dot += nw[r] * n[r].r;
    }
    if (!(fabs(dot) >= p.cos_gate * sqrt(nre2))) continue;
    const cd res = diff[0] * n[0] + diff[1] * n[1] + diff[2] * n[2];
    const cd J[6] = {pp[1] * n[2] - pp[2] * n[1], pp[2] * n[0] - pp[0] * n[2], pp[0] * n[1] - pp[1] * n[0],
                     n[0], n[1], n[2]};
    int e = 0;
    for (int i = 0; i < 6; ++i)
      for (int k = i; k < 6; ++k) acc[e++] += J[i] * J[k];
    for (int i = 0; i < 6; ++i) acc[21 + i] += J[i] * res;
    cnt += 1.0;
  }
  // block sums: warp shuffles, then across warps in a fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < kNV; ++v) {
    double x = v < 54 ? ((v & 1) ? acc[v >> 1].i : acc[v >> 1].r) : cnt;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < kNV) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += s_red[w][threadIdx.x];
    part[(size_t)blockIdx.x * kNV + threadIdx.x] = s;
  }
}

// cross-block sum, then the complex 6x6 solve and T <- exp(x) T (one block)
__global__ void __launch_bounds__(kT) k_p_solve(PP p, int nblk, int npx, const double* __restrict__ part, cd* T,
                                                int* st) {
  if (st[0]) return;
  __shared__ double s_sum[kNV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = warp; v < kNV; v += kT / 32) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * kNV + v];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_sum[v] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (s_sum[54] < p.min_corr_frac * npx) {
    st[0] = 1;
    return;
  }
  cd A[36], g[6];
  int e = 0;
  for (int i = 0; i < 6; ++i)
    for (int k = i; k < 6; ++k) {
      A[6 * i + k] = A[6 * k + i] = C(s_sum[2 * e], s_sum[2 * e + 1]);
      ++e;
    }
  for (int i = 0; i < 6; ++i) g[i] = C(-s_sum[2 * (21 + i)], -s_sum[2 * (21 + i) + 1]);  // b = -sum J r
  // positive definiteness of the real part (real Cholesky pivots)
  double L[36];
  for (int j = 0; j < 6; ++j) {
    double d = A[6 * j + j].r;
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0)) {
      st[0] = 1;
      return;
    }
    L[6 * j + j] = sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double s = A[6 * i + j].r;
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s / L[6 * j + j];
    }
  }
  // complex symmetric LDL^T (no conjugation), then the two triangular solves
  cd Lc[36], Dg[6];
  for (int j = 0; j < 6; ++j) {
    cd d = A[6 * j + j];
    for (int k = 0; k < j; ++k) d = d - Lc[6 * j + k] * Lc[6 * j + k] * Dg[k];
    Dg[j] = d;
    for (int i = j + 1; i < 6; ++i) {
      cd s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s = s - Lc[6 * i + k] * Lc[6 * j + k] * Dg[k];
      Lc[6 * i + j] = s / d;
    }
  }
  cd y[6], x[6];
  for (int i = 0; i < 6; ++i) {
    cd s = g[i];
    for (int k = 0; k < i; ++k) s = s - Lc[6 * i + k] * y[k];
    y[i] = s;
  }
  for (int i = 5; i >= 0; --i) {
    cd s = y[i] / Dg[i];
    for (int k = i + 1; k < 6; ++k) s = s - Lc[6 * k + i] * x[k];
    x[i] = s;
  }
  cd E[12], Told[12], Tn[12];
  cse3_exp(x, E);
  for (int i = 0; i < 12; ++i) Told[i] = T[i];
  ccompose(E, Told, Tn);
  for (int i = 0; i < 12; ++i) T[i] = Tn[i];
}

// frame start: T_{k-1} kept for the fallback; status cleared
__global__ void k_p_icp_begin(const cd* T, cd* Tprev, int* st) {
  if (threadIdx.x < 12) Tprev[threadIdx.x] = T[threadIdx.x];
  if (threadIdx.x == 0) st[0] = 0;
}
// frame end: a failed ICP falls back to T_{k-1}
__global__ void k_p_icp_end(cd* T, const cd* Tprev, int* st) {
  __shared__ int failed;
  if (threadIdx.x == 0) failed = st[0];
  __syncthreads();
  if (failed && threadIdx.x < 12) T[threadIdx.x] = Tprev[threadIdx.x];
  if (failed && threadIdx.x == 0) st[1] += 1;
}

// ---------------------------------------------------------------------------------------------
// TSDF update (Sec. 4.1 "Surface Update", Eq. bi_interpolate): every voxel of the volume
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) k_p_integrate(PP p, double* __restrict__ vox, const cd* __restrict__ D,
                                                    const cd* __restrict__ Tg, cd mu) {
  __shared__ cd sI[12], st_[3];
  if (threadIdx.x == 0) {
    cd T[12];
    for (int e = 0; e < 12; ++e) T[e] = Tg[e];
    cinverse(T, sI);
    st_[0] = T[3];
    st_[1] = T[7];
    st_[2] = T[11];
  }
  __syncthreads();
  const size_t n = (size_t)p.nx * p.ny * p.nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % p.nx), j = (int)((idx / p.nx) % p.ny), k = (int)(idx / ((size_t)p.nx * p.ny));
    const cd pw[3] = {C(p.ox + (i + 0.5) * p.voxel), C(p.oy + (j + 0.5) * p.voxel), C(p.oz + (k + 0.5) * p.voxel)};
    cd pc[3];
    cxform(sI, pw, pc);
    const cd z = pc[2];
    if (!(z.r > 0.0)) continue;
    const cd x = p.fx * pc[0] / z + C(p.cx), y = p.fy * pc[1] / z + C(p.cy);
    if (!(x.r >= 0.0 && x.r < p.W - 1 && y.r >= 0.0 && y.r < p.H - 1)) continue;
    const int i0 = (int)floor(x.r), j0 = (int)floor(y.r);
    const cd a = x - C((double)i0), b = y - C((double)j0);
    const size_t t00 = (size_t)j0 * p.W + i0;
    const cd d00 = D[t00], d10 = D[t00 + 1], d01 = D[t00 + p.W], d11 = D[t00 + p.W + 1];
    if (!(d00.r > 0.0 && d10.r > 0.0 && d01.r > 0.0 && d11.r > 0.0)) continue;
    if (!(fabs(d10.r - d00.r) + fabs(d01.r - d00.r) + fabs(d11.r - d00.r) < p.disc_gate)) continue;
    const cd L = (C(1.0) - a) * (C(1.0) - b) * d00 + a * (C(1.0) - b) * d10 + (C(1.0) - a) * b * d01 + a * b * d11;
    const cd rx = (x - C(p.cx)) / p.fx, ry = (y - C(p.cy)) / p.fy;
    const cd lam = csqrt_(rx * rx + ry * ry + C(1.0));
    const cd dv[3] = {st_[0] - pw[0], st_[1] - pw[1], st_[2] - pw[2]};
    const cd dist = csqrt_(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    const cd sdf = L - dist / lam;
    if (!(sdf.r >= -mu.r)) continue;
    const cd FD = sdf.r >= mu.r ? C(1.0) : sdf / mu;
    double* v = vox + 3 * idx;
    const double w = v[2];
    const cd F = (w * C(v[0], v[1]) + FD) / (w + 1.0);
    v[0] = F.r;
    v[1] = F.i;
    v[2] = fmin(w + 1.0, p.w_max);
  }
}

// ---------------------------------------------------------------------------------------------
// ray casting (Sec. 4.1 "Ray casting", Eq. surface_prediction): complex samples along each ray
// ---------------------------------------------------------------------------------------------
// trilinear F at continuous voxel coordinates g (voxel centres at integers); false outside the
// volume or where a corner is unobserved (W = 0)
__device__ bool ctri(const PP& p, const double* __restrict__ vox, const cd* g, cd& val) {
  const double gx = g[0].r, gy = g[1].r, gz = g[2].r;
  if (!(gx >= 0.0 && gx < p.nx - 1 && gy >= 0.0 && gy < p.ny - 1 && gz >= 0.0 && gz < p.nz - 1)) return false;
  const int i0 = (int)floor(gx), j0 = (int)floor(gy), k0 = (int)floor(gz);
  const cd f[3] = {g[0] - C((double)i0), g[1] - C((double)j0), g[2] - C((double)k0)};
  cd acc = C(0.0);
  bool ok = true;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const size_t lin = (size_t)(i0 + dx) + (size_t)p.nx * ((size_t)(j0 + dy) + (size_t)p.ny * (k0 + dz));
        const cd w = (dx ? f[0] : C(1.0) - f[0]) * (dy ? f[1] : C(1.0) - f[1]) * (dz ? f[2] : C(1.0) - f[2]);
        acc += w * C(vox[3 * lin], vox[3 * lin + 1]);
        ok = ok && vox[3 * lin + 2] > 0.0;
      }
  val = acc;
  return ok;
}

__global__ void __launch_bounds__(kT) k_p_raycast(PP p, const double* __restrict__ vox, const cd* __restrict__ Tg,
                                                  double* __restrict__ mdep, cd* __restrict__ mvn) {
  __shared__ cd sT[12];
  if (threadIdx.x < 12) sT[threadIdx.x] = Tg[threadIdx.x];
  __syncthreads();
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= p.W * p.H) return;
  const int u = px % p.W, v = px / p.W;
  const double ray[3] = {(u - p.cx) / p.fx, (v - p.cy) / p.fy, 1.0};
  cd dir[3], t[3];
  for (int r = 0; r < 3; ++r) {
    dir[r] = sT[4 * r] * ray[0] + sT[4 * r + 1] * ray[1] + sT[4 * r + 2] * ray[2];
    t[r] = sT[4 * r + 3];
  }
  const double org[3] = {p.ox, p.oy, p.oz};
  auto coords = [&](const cd* pt, cd* g) {
    for (int r = 0; r < 3; ++r) g[r] = (pt[r] - C(org[r])) / p.voxel - C(0.5);
  };
  const double step = p.ray_step;
  bool pv = false, ppos = false, hit = false;
  int mh = 0;
  for (int m = p.m0; m <= p.m1; ++m) {
    const double a = m * step;
    cd pt[3], g[3], val = C(0.0);
    for (int r = 0; r < 3; ++r) pt[r] = t[r] + a * dir[r];
    coords(pt, g);
    const bool ok = ctri(p, vox, g, val);
    const bool pos = val.r > 0.0;
    if (pv && ok) {
      if (ppos && !pos) {
        hit = true;
        mh = m - 1;
        break;
      }
      if (!ppos && pos) break;
    }
    pv = ok;
    ppos = pos;
  }
  bool good = false;
  cd V[3], N[3];
  double dep = 0.0;
  if (hit) {
    cd Fs[2];
    bool ok = true;
    for (int s = 0; s < 2; ++s) {
      const double a = (mh + s) * step;
      cd pt[3], g[3];
      for (int r = 0; r < 3; ++r) pt[r] = t[r] + a * dir[r];
      coords(pt, g);
      ok = ctri(p, vox, g, Fs[s]) && ok;
    }
    const cd alpha0 = C(mh * step) - step * Fs[0] / (Fs[1] - Fs[0]);
    for (int r = 0; r < 3; ++r) V[r] = alpha0 * dir[r] + t[r];
    cd grad[3];
    for (int ax = 0; ax < 3; ++ax) {
      cd vals[2];
      for (int s = 0; s < 2; ++s) {
        cd pt[3], g[3];
        for (int r = 0; r < 3; ++r) pt[r] = V[r] + C(r == ax ? (s == 0 ? p.voxel : -p.voxel) : 0.0);
        coords(pt, g);
        ok = ctri(p, vox, g, vals[s]) && ok;
      }
      grad[ax] = (vals[0] - vals[1]) / (2.0 * p.voxel);
    }
    const cd g2 = grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2];
    if (ok && g2.r > 0.0) {
      const cd nn = csqrt_(g2);
      for (int r = 0; r < 3; ++r) N[r] = grad[r] / nn;
      dep = alpha0.r;
      good = true;
    }
  }
  mdep[px] = good ? dep : 0.0;
  for (int r = 0; r < 3; ++r) {
    mvn[6 * (size_t)px + r] = good ? V[r] : C(0.0);
    mvn[6 * (size_t)px + 3 + r] = good ? N[r] : C(0.0);
  }
}

// ---------------------------------------------------------------------------------------------
// seeds and read-out (Eq. lie, Eq. csfd, Eq. pvnpxi)
// ---------------------------------------------------------------------------------------------
__global__ void k_p_set_pose(cd* T, const double* T0) {
  if (threadIdx.x < 12) T[threadIdx.x] = C(T0[threadIdx.x]);
}
// T0* = exp(h i e_j) T0
__global__ void k_p_seed_pose(cd* T, double h, int j) {
  if (threadIdx.x != 0) return;
  cd xi[6], E[12], T0[12], O[12];
  for (int e = 0; e < 6; ++e) xi[e] = C(0.0);
  xi[j] = C(0.0, h);
  cse3_exp(xi, E);
  for (int e = 0; e < 12; ++e) T0[e] = T[e];
  ccompose(E, T0, O);
  for (int e = 0; e < 12; ++e) T[e] = O[e];
}
// out: Re T (12), Im T / h (12), the left twist (omega, v) of that derivative (6)
__global__ void k_p_readout(const cd* T, double h, double* out) {
  if (threadIdx.x != 0) return;
  double R[12], dT[12];
  for (int e = 0; e < 12; ++e) {
    R[e] = T[e].r;
    dT[e] = h != 0.0 ? T[e].i / h : 0.0;
    out[e] = R[e];
    out[12 + e] = dT[e];
  }
  double Wm[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Wm[3 * r + c] = dT[4 * r] * R[4 * c] + dT[4 * r + 1] * R[4 * c + 1] + dT[4 * r + 2] * R[4 * c + 2];
  const double w0 = 0.5 * (Wm[7] - Wm[5]), w1 = 0.5 * (Wm[2] - Wm[6]), w2 = 0.5 * (Wm[3] - Wm[1]);
  out[24] = w0;
  out[25] = w1;
  out[26] = w2;
  out[27] = dT[3] - (w1 * R[11] - w2 * R[7]);
  out[28] = dT[7] - (w2 * R[3] - w0 * R[11]);
  out[29] = dT[11] - (w0 * R[7] - w1 * R[3]);
}

__global__ void k_p_read(const double* vox, size_t n, int part, double scale, double* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = vox[3 * i + part] * scale;
}

struct Run {
  double* vox = nullptr;
  cd* dep[3] = {};
  cd* tmp = nullptr;
  cd* vn[3] = {};
  unsigned char* nv[3] = {};
  double* mdep = nullptr;
  cd* mvn = nullptr;
  cd* T = nullptr;
  cd* Tprev = nullptr;
  double* part = nullptr;
  int* st = nullptr;
  double* out = nullptr;
};

std::string g_plain_err;

}  // namespace

struct xslam_plain_s {
  PP p;
  int max_runs = 0;
  int K = 0;
  int frame = 0;
  xslam_seed seeds[16];
  std::vector<Run> runs;
  cudaStream_t s = nullptr, user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  float* din = nullptr;
  double* h_out = nullptr;
  int* h_st = nullptr;
  int nblk0 = 1;
  int nsm = 148;
  double mu = 0.0;
  std::string err;
};

static xslam_status pfail(xslam_plain_t h, xslam_status st, const std::string& m) {
  if (h) h->err = m;
  else g_plain_err = m;
  return st;
}

#define PCU(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return pfail(h, XSLAM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

static void free_all(xslam_plain_t h) {
  for (Run& r : h->runs) {
    cudaFree(r.vox);
    for (int l = 0; l < 3; ++l) {
      cudaFree(r.dep[l]);
      cudaFree(r.vn[l]);
      cudaFree(r.nv[l]);
    }
    cudaFree(r.tmp);
    cudaFree(r.mdep);
    cudaFree(r.mvn);
    cudaFree(r.T);
    cudaFree(r.Tprev);
    cudaFree(r.part);
    cudaFree(r.st);
    cudaFree(r.out);
  }
  h->runs.clear();
  cudaFree(h->din);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->s) cudaStreamDestroy(h->s);
}

extern "C" xslam_status xslam_plain_create(xslam_plain_t* out, int nx, int ny, int nz, float voxel_m, float trunc_m,
                                           const float origin_m[3], const xslam_intrinsics* K, const xslam_config* cfg,
                                           int max_runs, void* cuda_stream) {
  xslam_plain_t h = nullptr;
  if (!out || !origin_m || !K) return pfail(h, XSLAM_EINVAL, "NULL argument");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2) return pfail(h, XSLAM_EINVAL, "volume dims must be >= 2");
  if (!(voxel_m > 0.f) || !(trunc_m > 0.f)) return pfail(h, XSLAM_EINVAL, "voxel and truncation must be > 0");
  if (K->width < 8 || K->height < 8 || !(K->fx > 0.f) || !(K->fy > 0.f))
    return pfail(h, XSLAM_EINVAL, "bad intrinsics");
  if (max_runs < 1 || max_runs > 16) return pfail(h, XSLAM_EINVAL, "max_runs must be in 1..16");
  xslam_config c;
  if (cfg) c = *cfg;
  else xslam_default_config(&c);
  if (c.icp_levels < 1 || c.icp_levels > 3) return pfail(h, XSLAM_EINVAL, "icp_levels must be in 1..3");
  if (c.icp_newton) return pfail(h, XSLAM_EINVAL, "the plain path runs Gauss-Newton ICP only");
  if (c.icp_seed != 0 || c.icp_stop != 0.f)
    return pfail(h, XSLAM_EINVAL, "the plain path starts ICP at the previous pose with fixed iteration counts");
  for (int l = 0; l < c.icp_levels; ++l)
    if (c.icp_iters[l] < 0 || c.icp_iters[l] > 100) return pfail(h, XSLAM_EINVAL, "icp_iters must be in 0..100");
  if (!(c.ray_step_vox > 0.f) || !(c.depth_max_m > c.depth_min_m) || !(c.depth_min_m > 0.f))
    return pfail(h, XSLAM_EINVAL, "bad ray step or depth range");
  h = new xslam_plain_s();
  PP& p = h->p;
  p.nx = nx; p.ny = ny; p.nz = nz;
  p.W = K->width; p.H = K->height;
  p.levels = c.icp_levels;
  for (int l = 0; l < 4; ++l) p.iters[l] = l < c.icp_levels ? c.icp_iters[l] : 0;
  p.voxel = voxel_m;
  p.ox = origin_m[0]; p.oy = origin_m[1]; p.oz = origin_m[2];
  p.fx = K->fx; p.fy = K->fy; p.cx = K->cx; p.cy = K->cy;
  p.dist_gate = c.dist_gate_m;
  p.cos_gate = std::cos((double)c.normal_gate_deg * 3.14159265358979323846 / 180.0);
  p.disc_gate = c.disc_gate_m;
  p.min_corr_frac = c.min_corr_frac;
  p.depth_min = c.depth_min_m;
  p.depth_max = c.depth_max_m;
  p.pyr_range = c.pyr_range_m;
  p.ray_step = (double)c.ray_step_vox * (double)voxel_m;
  p.w_max = c.w_max > 0.f ? (double)c.w_max : INFINITY;
  p.bilateral = c.bilateral;
  p.m0 = (int)std::ceil(p.depth_min / p.ray_step - 1e-4);
  p.m1 = (int)std::floor(p.depth_max / p.ray_step + 1e-4);
  h->mu = trunc_m;
  h->max_runs = max_runs;
  h->user = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t hw = (size_t)p.W * p.H, n = (size_t)nx * ny * nz;
  h->nblk0 = (int)((hw + kT - 1) / kT);
  bool ok = cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaMalloc(&h->din, sizeof(float) * hw) == cudaSuccess;
  ok &= cudaMallocHost(&h->h_out, sizeof(double) * 30 * max_runs) == cudaSuccess;
  ok &= cudaMallocHost(&h->h_st, sizeof(int) * 4 * max_runs) == cudaSuccess;
  h->runs.resize(max_runs);
  for (Run& r : h->runs) {
    if (!ok) break;
    ok &= cudaMalloc(&r.vox, sizeof(double) * 3 * n) == cudaSuccess;
    for (int l = 0; l < 3; ++l) {
      const size_t hl = (size_t)(p.W >> l) * (p.H >> l);
      ok &= cudaMalloc(&r.dep[l], sizeof(cd) * hl) == cudaSuccess;
      ok &= cudaMalloc(&r.vn[l], sizeof(cd) * 6 * hl) == cudaSuccess;
      ok &= cudaMalloc(&r.nv[l], hl) == cudaSuccess;
    }
    ok &= cudaMalloc(&r.tmp, sizeof(cd) * hw) == cudaSuccess;
    ok &= cudaMalloc(&r.mdep, sizeof(double) * hw) == cudaSuccess;
    ok &= cudaMalloc(&r.mvn, sizeof(cd) * 6 * hw) == cudaSuccess;
    ok &= cudaMalloc(&r.T, sizeof(cd) * 12) == cudaSuccess;
    ok &= cudaMalloc(&r.Tprev, sizeof(cd) * 12) == cudaSuccess;
    ok &= cudaMalloc(&r.part, sizeof(double) * kNV * h->nblk0) == cudaSuccess;
    ok &= cudaMalloc(&r.st, sizeof(int) * 4) == cudaSuccess;
    ok &= cudaMalloc(&r.out, sizeof(double) * 30) == cudaSuccess;
  }
  if (!ok) {
    free_all(h);
    delete h;
    return pfail(nullptr, XSLAM_ENOMEM, "device or pinned allocation failed");
  }
  const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  double* dI = nullptr;
  if (cudaMalloc(&dI, sizeof(I)) != cudaSuccess) {
    free_all(h);
    delete h;
    return pfail(nullptr, XSLAM_ENOMEM, "device allocation failed");
  }
  cudaMemcpyAsync(dI, I, sizeof(I), cudaMemcpyHostToDevice, h->s);
  for (Run& r : h->runs) {
    k_p_fill<<<h->nsm * 8, kT, 0, h->s>>>(r.vox, n);
    k_p_set_pose<<<1, 32, 0, h->s>>>(r.T, dI);
    cudaMemsetAsync(r.st, 0, sizeof(int) * 4, h->s);
    cudaMemsetAsync(r.mdep, 0, sizeof(double) * hw, h->s);
    cudaMemsetAsync(r.mvn, 0, sizeof(cd) * 6 * hw, h->s);
  }
  const cudaError_t e = cudaStreamSynchronize(h->s);
  cudaFree(dI);
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return pfail(nullptr, XSLAM_ECUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  }
  *out = h;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_plain_destroy(xslam_plain_t h) {
  if (!h) return XSLAM_OK;
  cudaStreamSynchronize(h->s);
  free_all(h);
  delete h;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_plain_set_pose(xslam_plain_t h, const double T[12]) {
  if (!h || !T) return pfail(h, XSLAM_EINVAL, "NULL argument");
  if (h->frame > 0) return pfail(h, XSLAM_ESTATE, "the pose can only be set before the first frame");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(T[i])) return pfail(h, XSLAM_EINVAL, "pose has a non-finite entry");
  double* dT = h->runs[0].out;  // 30-double scratch, rewritten by every read-out
  PCU(cudaMemcpyAsync(dT, T, sizeof(double) * 12, cudaMemcpyHostToDevice, h->s));
  for (Run& r : h->runs) k_p_set_pose<<<1, 32, 0, h->s>>>(r.T, dT);
  PCU(cudaGetLastError());
  PCU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

static xslam_status check_seeds(xslam_plain_t h, const xslam_seed* seeds, int K) {
  if (K < 0 || K > h->max_runs) return pfail(h, XSLAM_EINVAL, "K must be in 0..max_runs");
  if (K > 0 && !seeds) return pfail(h, XSLAM_EINVAL, "seeds is NULL");
  for (int j = 0; j < K; ++j) {
    const xslam_seed& s = seeds[j];
    if (!std::isfinite(s.h) || std::fabs(s.h) > 1e-3 || std::fabs(s.h) < 1e-30)
      return pfail(h, XSLAM_EINVAL, "seed h must satisfy 1e-30 <= |h| <= 1e-3");
    if (s.kind == XSLAM_SEED_POSE0) {
      if (s.index < 0 || s.index > 5) return pfail(h, XSLAM_EINVAL, "POSE0 index must be 0..5");
    } else if (s.kind == XSLAM_SEED_DEPTH) {
      if (s.index != -1) return pfail(h, XSLAM_EINVAL, "only DEPTH seeds on every pixel (index -1) are built");
    } else if (s.kind != XSLAM_SEED_TRUNC) {
      return pfail(h, XSLAM_EINVAL, "seed kind not built (POSE0, TRUNC and DEPTH are)");
    }
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_plain_frame(xslam_plain_t h, const float* depth, int depth_on_device,
                                          const xslam_seed* seeds, int K, double* pose_out, double* dpose_out,
                                          double* dtwist_out) {
  if (!h) return XSLAM_EINVAL;
  if (!depth) return pfail(h, XSLAM_EINVAL, "depth is NULL");
  xslam_status st = check_seeds(h, seeds, K);
  if (st != XSLAM_OK) return st;
  if (h->frame == 0) {
    h->K = K;
    for (int j = 0; j < K; ++j) h->seeds[j] = seeds[j];
  } else {
    bool same = K == h->K;
    for (int j = 0; same && j < K; ++j)
      same = seeds[j].kind == h->seeds[j].kind && seeds[j].index == h->seeds[j].index && seeds[j].h == h->seeds[j].h;
    if (!same) return pfail(h, XSLAM_ESTATE, "seeds must not change after the first frame");
  }
  const PP& p = h->p;
  const int W = p.W, H = p.H, hw = W * H;
  PCU(cudaEventRecord(h->ev_in, h->user));
  PCU(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  PCU(cudaMemcpyAsync(h->din, depth, sizeof(float) * hw, depth_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      h->s));
  const int nr = std::max(K, 1);
  const size_t n = (size_t)p.nx * p.ny * p.nz;
  for (int ri = 0; ri < nr; ++ri) {
    Run& r = h->runs[ri];
    const xslam_seed* sd = K > 0 ? &h->seeds[ri] : nullptr;
    const double hD = (sd && sd->kind == XSLAM_SEED_DEPTH) ? sd->h : 0.0;
    const cd mu = C(h->mu, (sd && sd->kind == XSLAM_SEED_TRUNC) ? sd->h : 0.0);
    // surface measurement
    k_p_gate<<<(hw + kT - 1) / kT, kT, 0, h->s>>>(h->din, p.bilateral ? r.tmp : r.dep[0], hw, hD, p.depth_min,
                                                    p.depth_max);
    if (p.bilateral) k_p_bilateral<<<(hw + kT - 1) / kT, kT, 0, h->s>>>(r.tmp, r.dep[0], W, H);
    for (int l = 1; l < p.levels; ++l) {
      const int Wo = W >> l, Ho = H >> l;
      k_p_pyr_down<<<(Wo * Ho + kT - 1) / kT, kT, 0, h->s>>>(r.dep[l - 1], W >> (l - 1), H >> (l - 1), r.dep[l], Wo,
                                                             Ho, p.pyr_range);
    }
    if (h->frame == 0) {
      if (sd && sd->kind == XSLAM_SEED_POSE0) k_p_seed_pose<<<1, 32, 0, h->s>>>(r.T, sd->h, sd->index);
    } else {
      for (int l = 0; l < p.levels; ++l) {
        const int Wl = W >> l, Hl = H >> l;
        const double s = (double)(1 << l);
        k_p_vertex_normal<<<(Wl * Hl + kT - 1) / kT, kT, 0, h->s>>>(r.dep[l], Wl, Hl, p.fx / s, p.fy / s, p.cx / s,
                                                                    p.cy / s, r.vn[l], r.nv[l]);
      }
      k_p_icp_begin<<<1, 32, 0, h->s>>>(r.T, r.Tprev, r.st);
      for (int l = p.levels - 1; l >= 0; --l) {
        const double s = (double)(1 << l);
        const Lv lv{W >> l, H >> l, 1 << l, p.fx / s, p.fy / s, p.cx / s, p.cy / s};
        const int npx = lv.W * lv.H;
        const int nblk = (npx + kT - 1) / kT;
        for (int it = 0; it < p.iters[l]; ++it) {
          k_p_icp<<<nblk, kT, 0, h->s>>>(p, lv, r.vn[l], r.nv[l], r.mdep, r.mvn, r.T, r.Tprev, r.part, r.st);
          k_p_solve<<<1, kT, 0, h->s>>>(p, nblk, npx, r.part, r.T, r.st);
        }
      }
      k_p_icp_end<<<1, 32, 0, h->s>>>(r.T, r.Tprev, r.st);
    }
    k_p_integrate<<<(unsigned)((n + kT - 1) / kT), kT, 0, h->s>>>(p, r.vox, r.dep[0], r.T, mu);
    k_p_raycast<<<(hw + kT - 1) / kT, kT, 0, h->s>>>(p, r.vox, r.T, r.mdep, r.mvn);
    k_p_readout<<<1, 32, 0, h->s>>>(r.T, sd ? sd->h : 0.0, r.out);
    PCU(cudaGetLastError());
    PCU(cudaMemcpyAsync(h->h_out + 30 * ri, r.out, sizeof(double) * 30, cudaMemcpyDeviceToHost, h->s));
    PCU(cudaMemcpyAsync(h->h_st + 4 * ri, r.st, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->s));
  }
  PCU(cudaEventRecord(h->ev_out, h->s));
  PCU(cudaStreamWaitEvent(h->user, h->ev_out, 0));
  PCU(cudaStreamSynchronize(h->s));
  const int failed = h->frame > 0 ? h->h_st[0] : 0;
  h->frame += 1;
  if (pose_out)
    for (int i = 0; i < 12; ++i) pose_out[i] = h->h_out[i];
  for (int j = 0; j < K; ++j) {
    if (dpose_out)
      for (int i = 0; i < 12; ++i) dpose_out[12 * j + i] = h->h_out[30 * j + 12 + i];
    if (dtwist_out)
      for (int i = 0; i < 6; ++i) dtwist_out[6 * j + i] = h->h_out[30 * j + 24 + i];
  }
  if (failed) {
    h->err = "ICP failed; the frame was fused at the previous pose";
    return XSLAM_ENOTRACK;
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_plain_read_tsdf(xslam_plain_t h, int run, int part, double* out) {
  if (!h || !out) return pfail(h, XSLAM_EINVAL, "NULL argument");
  if (run < 0 || run >= h->max_runs) return pfail(h, XSLAM_EINVAL, "run out of range");
  if (part < 0 || part > 2) return pfail(h, XSLAM_EINVAL, "part must be 0 (Re F), 1 (Im F / h) or 2 (W)");
  double scale = 1.0;
  if (part == 1 && run < h->K) scale = 1.0 / h->seeds[run].h;
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  PCU(cudaEventRecord(h->ev_in, h->user));
  PCU(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  k_p_read<<<h->nsm * 8, kT, 0, h->s>>>(h->runs[run].vox, n, part, scale, out);
  PCU(cudaGetLastError());
  PCU(cudaEventRecord(h->ev_out, h->s));
  PCU(cudaStreamWaitEvent(h->user, h->ev_out, 0));
  PCU(cudaStreamSynchronize(h->s));
  return XSLAM_OK;
}

extern "C" const char* xslam_plain_last_error(xslam_plain_t h) {
  return h ? h->err.c_str() : g_plain_err.c_str();
}
