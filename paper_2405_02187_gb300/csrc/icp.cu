// Projective point-to-plane ICP (X-SLAM Sec. 4.1, "Differentiable ICP") on 1 + K lanes: one launch
// per Gauss-Newton iteration.
//
// Per pixel u of pyramid level l: V = D K_l^-1 u, N = normalize((V(u+x) - V) x (V(u+y) - V)) (Eq. vertex,
// Eq. normal), p' = T_j V, u_hat = pi(K_l T_{k-1}^-1 p'), q and n = bilinear model vertex / normal at
// u_hat (level-0 model maps read at pixel 2^l u_hat), r = (p' - q).n, J = [(p' x n)^T, n^T]; the
// normal equations A = sum J J^T, g = sum J r (Eq. icp, Eq. "icp approx") are reduced, A x = -g is
// solved and T_{j+1} = exp(x) T_j.
//
// GB300 mapping: one launch per Gauss-Newton iteration, blocks of 16 warps, at most one block per SM.
// A warp takes one chunk of 32 consecutive pixels of the level at a time (a pixel per thread; at a
// coarse level a chunk's lanes may be split over up to 3 warps, icp_groups), computes its real part,
// then every lane's tangent in turn from the lane's affine map of the camera-frame point and its own
// model taps. The 27 terms of each lane are summed over the warp right away by a transpose reduction
// (thread t ends with value t), so a thread holds no accumulators across chunks and warps never wait
// for each other; the warps' sums go to shared memory, the block's to value-major partials. The last
// block to finish (ticket counter, no grid-wide wait) adds the partials in double-FP32, factors the
// real 6x6 matrix (FP32 square-root-free Cholesky, one refinement of every right-hand side with
// double-FP32 residuals), solves the K + 1 right-hand sides (x_0 from the real part, x_j = A^-1 (-g_j -
// A_j x_0) for each lane) and composes exp(x) T_j on every lane (FP32 increment, FP64 composition).
#include "internal.cuh"
#include "se3.cuh"

namespace xslam {

constexpr int kMaxPartials = 256;  // upper bound of the grid size (partials per value)

// row stride of the value-major partials: a multiple of 4 floats (float4 reads); the last block of
// the grid writes zeros into the padding of every row
__host__ __device__ __forceinline__ int icp_pstride(int nblk) { return (nblk + 3) & ~3; }

struct Lvl {
  int W, H, s, level;
  float fx, fy, cx, cy;
};

// index of (r, c), r <= c, in the row-major packed upper triangle of a 6x6 matrix
__host__ __device__ constexpr int up6(int r, int c) { return r * 6 - r * (r - 1) / 2 + (c - r); }

// Double-FP32 numbers (hi + lo, |lo| <= ulp(hi) / 2: about 48 significant bits) for the tail's sums and
// residuals. GB300's FP64 units make a dependent FP64 operation cost far more than the handful of FP32
// operations of an error-free transformation: Knuth's two-sum, and the exact product error of an FMA.
// The _rn intrinsics keep the compiler from contracting a product into a neighbouring sum.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|, or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  DF s = two_sum(x.h, y.h);
  const DF t = two_sum(x.l, y.l);
  s.l = __fadd_rn(s.l, t.h);
  s = quick_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ DF df_add_f(DF x, float y) {
  DF s = two_sum(x.h, y);
  s.l = __fadd_rn(s.l, x.l);
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.h, -x.l}; }
// x y for a float y: the high part's exact product (rounded product + FMA residual) and the low part's
__device__ __forceinline__ DF df_mul_f(DF x, float y) {
  const float p = __fmul_rn(x.h, y);
  const float e = fmaf(x.l, y, fmaf(x.h, y, -p));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -p)));
  return quick_two_sum(p, e);
}

// The 6x6 solve. A = L D L^T is factored in FP32 (square-root-free Cholesky) and every right-hand
// side is solved by mixed-precision iterative refinement: x = S(b), r = b - A x in double-FP32 (A and b
// are the double-FP32 sums), x += S(r), with S the FP32 forward/back substitution; one round brings the
// relative error from ~cond(A) 2^-24 to ~(cond(A) 2^-24)^2. The steps of the tail run SIMT-parallel: one
// thread per (system, row) or per matrix element.
struct Ldl32 {
  float L[15];  // strictly lower part, row-major packed: (i, k) for k < i at i(i-1)/2 + k
  float rD[6];  // 1 / D
};

__device__ __forceinline__ int lo6(int i, int k) { return i * (i - 1) / 2 + k; }

// returns false if a pivot is not positive (A not positive definite in FP32); A packed upper, FP32
__device__ bool ldl32(const float* __restrict__ A, Ldl32& f) {
  float D[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = A[up6(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= f.L[lo6(j, k)] * f.L[lo6(j, k)] * D[k];
    if (!(d > 0.f)) return false;
    D[j] = d;
    f.rD[j] = 1.f / d;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float s = A[up6(j, i)];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= f.L[lo6(i, k)] * f.L[lo6(j, k)] * D[k];
      f.L[lo6(i, j)] = s * f.rD[j];
    }
  }
  return true;
}

__device__ __forceinline__ void subst32(const Ldl32& f, const float* b, float* x) {
  float y[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= f.L[lo6(i, k)] * y[k];
    y[i] = s;
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    float s = y[i] * f.rD[i];
#pragma unroll
    for (int k = i + 1; k < 6; ++k) s -= f.L[lo6(k, i)] * x[k];
    x[i] = s;
  }
}

// Shared memory of the ICP kernels (static part; the per-pixel records are dynamic).
constexpr int kIcpThreads = 512;  // 16 warps; a warp takes one chunk of 32 pixels at a time
constexpr int kIcpWarps = kIcpThreads / 32;
// dynamic shared memory of the ICP kernels for L lanes: the warps' sums [warp][lane][27]
__host__ __device__ __forceinline__ int icp_dyn_bytes(int L) { return (int)sizeof(float) * kIcpWarps * L * kNT; }


// The tangent of a lane's camera-frame point is affine in the pixel's vertex V: with the pose lanes
// (T, T_l) and the model's pose lanes (P, P_l),
//   p_c' = P_l^T (T V + t - t_P) + P^T (T_l V + t_l - t_Pl + T V_l) = A_l V + b_l + P^T T V_l,
// A_l = P_l^T T + P^T T_l, b_l = P_l^T (t - t_P) + P^T (t_l - t_Pl), and V_l = dD_l (rx, ry, 1) for a
// DEPTH lane, whose P^T T V_l = dD_l (p_c - b_0) / d with b_0 = P^T (t - t_P). Per launch, per lane.
struct IcpLane {
  float A[9];
  float b[3];
};

// Shared memory of the ICP kernels.
struct IcpShared {
  float sT[kMaxLanes][12];   // pose lanes of the current iterate (FP32 copy for the pixel work)
  float sP[kMaxLanes][12];   // pose lanes the model was ray cast at
  IcpLane sL[kMaxLanes];     // per-lane affine maps of the camera-frame tangent
  float sb0[3];
  int s_cnt[kIcpWarps];
  float sAh[kMaxLanes * kNT], sAl[kMaxLanes * kNT];  // the summed normal equations, double-FP32
  float sx0h[6], sx0l[6];                            // x_0 (refined), double-FP32
  double sx[kMaxLanes][6];
  Ldl32 s_ldl;
  float s_halfh[2 * kNT * kMaxLanes], s_halfl[2 * kNT * kMaxLanes];
  float sxf[kMaxLanes][6], srf[kMaxLanes][6], sdf[kMaxLanes][6];
  SeCoefF scf[kMaxLanes];
  float sxs[kMaxLanes][6];
  float sdl[kMaxLanes][12];
  int s_ncorr, s_fail;
};

// Load the pose lanes into S and form the lanes' affine maps; zero the warps' sums (wacc). A restarted
// lane (per-frame pose seed) carries no derivative in the model's pose: its P_l is taken as zero.
__device__ __forceinline__ void icp_prologue(const Params& p, const double* __restrict__ pose,
                                             const double* __restrict__ pose_prev, IcpShared& S, int L,
                                             float* __restrict__ wacc) {
  for (int i = threadIdx.x; i < L * 12; i += blockDim.x) {
    S.sT[i / 12][i % 12] = (float)pose[i];
    const bool fresh = (i >= 12) && ((p.fresh >> (i / 12)) & 1u);
    S.sP[i / 12][i % 12] = fresh ? 0.f : (float)pose_prev[i];
  }
  for (int i = threadIdx.x; i < kIcpWarps * L * kNT; i += blockDim.x) wacc[i] = 0.f;
  __syncthreads();
  const float* T = S.sT[0];
  const float* P = S.sP[0];
  const int t = threadIdx.x;
  if (t < 3) S.sb0[t] = P[t] * (T[3] - P[3]) + P[4 + t] * (T[7] - P[7]) + P[8 + t] * (T[11] - P[11]);
  if (t >= 32 && t < 32 + 12 * (L - 1)) {
    const int l = 1 + (t - 32) / 12, e = (t - 32) % 12;
    const float* Tl = S.sT[l];
    const float* Pl = S.sP[l];
    if (e < 9) {
      const int r = e / 3, c = e % 3;  // A[r][c] = sum_k Pl[k][r] T[k][c] + P[k][r] Tl[k][c]
      float a = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) a += Pl[4 * k + r] * T[4 * k + c] + P[4 * k + r] * Tl[4 * k + c];
      S.sL[l].A[e] = a;
    } else {
      const int r = e - 9;
      float bv = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        bv += Pl[4 * k + r] * (T[4 * k + 3] - P[4 * k + 3]) + P[4 * k + r] * (Tl[4 * k + 3] - Pl[4 * k + 3]);
      S.sL[l].b[r] = bv;
    }
  }
  __syncthreads();
}

// Sum over the warp of 32 values per thread such that thread t ends with the sum of value t: five
// exchange steps, each sending half of the values still held to the partner lane and keeping the half
// that belongs to this lane's bit (31 shuffles for the 32 values).
template <int N>
__device__ __forceinline__ void transpose_step(float* v, int lid) {
  const bool hi = (lid & N) != 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float send = hi ? v[i] : v[i + N];
    const float keep = hi ? v[i + N] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, N);
  }
}

__device__ __forceinline__ float warp_transpose_sum(float* v, int lid) {
  transpose_step<16>(v, lid);
  transpose_step<8>(v, lid);
  transpose_step<4>(v, lid);
  transpose_step<2>(v, lid);
  transpose_step<1>(v, lid);
  return v[0];
}

// Lane groups of a level: where the level has fewer chunks than the grid has warps (the coarse levels),
// a chunk's imaginary lanes are split over G warps, each of which forms the chunk's real correspondence
// itself, so that a chunk's chain of dependent lane loads is about 1/G as long. Group 0 also adds the real
// sums and the correspondence count. G = 3 from 4 lanes up (two imaginary lanes a group at K = 6), 2 for
// 3 lanes, 1 for fewer or where G warps a chunk do not fit the grid; then no group is left without a lane.
__host__ __device__ __forceinline__ int icp_groups(int nchunk, int nwarps, int L) {
  int G = L >= 4 ? 3 : (L == 3 ? 2 : 1);
  while (G > 1 && nchunk * G > nwarps) --G;
  if (G > 1) {
    const int per = (L - 1 + G - 1) / G;
    G = (L - 1 + per - 1) / per;
  }
  return G;
}

// The level's chunks c0, c0 + cstride, ... of 32 pixels for this warp (lane `lid` = pixel). For each
// pixel: the real part (V = D K_l^-1 u, the measured normal for the gate, p' = T V, the projection
// u_hat = pi(K_l P^-1 p'), the bilinear model vertex q and normal n at u_hat with their slopes in the
// cell, the gates, r = (p' - q) . n, J = [(p' x n)^T, n^T]); then for every lane its tangent of r and
// J from the lane's affine map, its depth perturbation and its own model taps. Each lane's 27 terms
// (J J^T upper triangle, J r; the tangent lanes J J_l^T + J_l J^T and J r_l + J_l r) are summed over
// the warp at once (warp_transpose_sum) and added to this warp's sums wacc[lane][27] in shared memory;
// cnt counts the correspondences. The warp is lane group grp of G (icp_groups).
__device__ __forceinline__ void icp_chunks(const Params& p, const Buffers& b, const Lvl& lv, IcpShared& S, int L,
                                           int warp, int lid, int c0, int cstride, int nchunk, int& cnt,
                                           float* __restrict__ wacc, int grp, int G) {
  const int per = (L - 1 + G - 1) / G;  // imaginary lanes of a group
  const int l_lo = 1 + grp * per, l_hi = min(L, l_lo + per);
  const bool real_sums = grp == 0;
  const float* D = lv.s == 1 ? b.pyr[0] : (lv.s == 2 ? b.pyr[1] : b.pyr[2]);
  const unsigned hw0 = (unsigned)p.W * (unsigned)p.H;
  const float* mdep = b.model;
  const float* mV = b.model + hw0;
  const float* mN = b.model + (size_t)hw0 * (1 + 3 * L);
  const int npx = lv.W * lv.H;
  const float* T = S.sT[0];
  const float* P = S.sP[0];
  for (int ch = c0; ch < nchunk; ch += cstride) {
    const int px = (ch << 5) + lid;
    bool ok = px < npx;
    const int u = ok ? px % lv.W : 0, v = ok ? px / lv.W : 0;
    ok = ok && u < lv.W - 1 && v < lv.H - 1;
    float d0 = 0.f, dxp = 0.f, dyp = 0.f;
    if (ok) {
      d0 = D[px];
      dxp = D[px + 1];
      dyp = D[px + lv.W];
    }
    ok = ok && d0 > 0.f && dxp > 0.f && dyp > 0.f;
    const float rx = (u - lv.cx) / lv.fx, ry = (v - lv.cy) / lv.fy;
    const float rx1 = (u + 1 - lv.cx) / lv.fx, ry1 = (v + 1 - lv.cy) / lv.fy;
    const float V[3] = {d0 * rx, d0 * ry, d0};
    const float ex[3] = {dxp * rx1 - V[0], dxp * ry - V[1], dxp - V[2]};
    const float ey[3] = {dyp * rx - V[0], dyp * ry1 - V[1], dyp - V[2]};
    const float c[3] = {ex[1] * ey[2] - ex[2] * ey[1], ex[2] * ey[0] - ex[0] * ey[2], ex[0] * ey[1] - ex[1] * ey[0]};
    const float n2m = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    ok = ok && n2m > 0.f;
    const float inm = ok ? 1.f / sqrtf(n2m) : 0.f;
    const float Nm[3] = {c[0] * inm, c[1] * inm, c[2] * inm};
    float pp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) pp[r] = T[4 * r] * V[0] + T[4 * r + 1] * V[1] + T[4 * r + 2] * V[2] + T[4 * r + 3];
    const float e0 = pp[0] - P[3], e1 = pp[1] - P[7], e2 = pp[2] - P[11];
    const float pc[3] = {P[0] * e0 + P[4] * e1 + P[8] * e2, P[1] * e0 + P[5] * e1 + P[9] * e2,
                         P[2] * e0 + P[6] * e1 + P[10] * e2};
    ok = ok && pc[2] > 0.f;
    const float iz = ok ? 1.f / pc[2] : 0.f;
    const float qx = pc[0] * iz, qy = pc[1] * iz;
    const float ux = lv.fx * qx + lv.cx, uy = lv.fy * qy + lv.cy;
    const float ci = floorf(ux + kCellBias), cj = floorf(uy + kCellBias);
    ok = ok && ci >= 0.f && ci <= (float)(lv.W - 2) && cj >= 0.f && cj <= (float)(lv.H - 2);
    const int i0 = ok ? (int)ci : 0, j0 = ok ? (int)cj : 0;
    const float a = ok ? ux - ci : 0.f, bb = ok ? uy - cj : 0.f;
    // the four taps of the cell in the level-0 model maps (32-bit offsets)
    const unsigned t00 = (unsigned)(j0 * lv.s) * (unsigned)p.W + (unsigned)(i0 * lv.s);
    const unsigned t10 = t00 + lv.s, t01 = t00 + (unsigned)lv.s * (unsigned)p.W, t11 = t01 + lv.s;
    float g00 = 0.f, g10 = 0.f, g01 = 0.f, g11 = 0.f;
    if (ok) {
      g00 = mdep[t00];
      g10 = mdep[t10];
      g01 = mdep[t01];
      g11 = mdep[t11];
    }
    ok = ok && g00 > 0.f && g10 > 0.f && g01 > 0.f && g11 > 0.f;
    ok = ok && fabsf(g10 - g00) + fabsf(g01 - g00) + fabsf(g11 - g00) < p.disc_gate;
    const float w00 = (1.f - a) * (1.f - bb), w10 = a * (1.f - bb), w01 = (1.f - a) * bb, w11 = a * bb;
    float q[3], nn[3], dqa[3], dqb[3], dna[3], dnb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float* Vp = mV + r * hw0;
      const float* Np = mN + r * hw0;
      const float v00 = Vp[t00], v10 = Vp[t10], v01 = Vp[t01], v11 = Vp[t11];
      const float m00 = Np[t00], m10 = Np[t10], m01 = Np[t01], m11 = Np[t11];
      q[r] = w00 * v00 + w10 * v10 + w01 * v01 + w11 * v11;
      nn[r] = w00 * m00 + w10 * m10 + w01 * m01 + w11 * m11;
      dqa[r] = (1.f - bb) * (v10 - v00) + bb * (v11 - v01);
      dqb[r] = (1.f - a) * (v01 - v00) + a * (v11 - v10);
      dna[r] = (1.f - bb) * (m10 - m00) + bb * (m11 - m01);
      dnb[r] = (1.f - a) * (m01 - m00) + a * (m11 - m10);
    }
    const float df[3] = {pp[0] - q[0], pp[1] - q[1], pp[2] - q[2]};
    ok = ok && df[0] * df[0] + df[1] * df[1] + df[2] * df[2] <= p.dist_gate2;
    float nw[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) nw[r] = T[4 * r] * Nm[0] + T[4 * r + 1] * Nm[1] + T[4 * r + 2] * Nm[2];
    const float nl2 = nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2];
    ok = ok && fabsf(nw[0] * nn[0] + nw[1] * nn[1] + nw[2] * nn[2]) >= p.cos_normal_gate * sqrtf(nl2);
    if (!__any_sync(0xffffffffu, ok)) continue;
    if (real_sums) cnt += ok ? 1 : 0;
    // a pixel without a correspondence adds zeros: its J and r are zero and its lanes stay finite
    const float m = ok ? 1.f : 0.f;
    const float res = m * (df[0] * nn[0] + df[1] * nn[1] + df[2] * nn[2]);
    const float J[6] = {m * (pp[1] * nn[2] - pp[2] * nn[1]), m * (pp[2] * nn[0] - pp[0] * nn[2]),
                        m * (pp[0] * nn[1] - pp[1] * nn[0]), m * nn[0], m * nn[1], m * nn[2]};
    float cv[32];
    {
      int k = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = r; cc < 6; ++cc) cv[k++] = J[r] * J[cc];
#pragma unroll
      for (int r = 0; r < 6; ++r) cv[21 + r] = J[r] * res;
#pragma unroll
      for (int r = 27; r < 32; ++r) cv[r] = 0.f;
    }
    if (real_sums) {
      const float sum = warp_transpose_sum(cv, lid);
      if (lid < kNT) wacc[lid] += sum;
    }
    if (l_lo >= l_hi) continue;
    // what the lanes share: the model pose's P^T T ray for DEPTH lanes, T ray likewise
    const float id0 = ok ? 1.f / d0 : 0.f;
    const float Cray[3] = {(pc[0] - S.sb0[0]) * id0, (pc[1] - S.sb0[1]) * id0, (pc[2] - S.sb0[2]) * id0};
    const float Tray[3] = {(pp[0] - T[3]) * id0, (pp[1] - T[7]) * id0, (pp[2] - T[11]) * id0};
    for (int l = l_lo; l < l_hi; ++l) {
      const float* Tl = S.sT[l];
      const IcpLane& LA = S.sL[l];
      float dDl = p.dD[l];
      if (p.dpix[l] >= 0 && ok) dDl += b.dlane[dlane_offset(p, l, lv.level) + px];
      float ppl[3], pcl[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ppl[r] = Tl[4 * r] * V[0] + Tl[4 * r + 1] * V[1] + Tl[4 * r + 2] * V[2] + Tl[4 * r + 3] + dDl * Tray[r];
        pcl[r] = LA.A[3 * r] * V[0] + LA.A[3 * r + 1] * V[1] + LA.A[3 * r + 2] * V[2] + LA.b[r] + dDl * Cray[r];
      }
      const float al = lv.fx * (pcl[0] - qx * pcl[2]) * iz;
      const float bl = lv.fy * (pcl[1] - qy * pcl[2]) * iz;
      float ql[3], nl[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ql[r] = dqa[r] * al + dqb[r] * bl;
        nl[r] = dna[r] * al + dnb[r] * bl;
      }
      if (!((p.fresh >> l) & 1u)) {
        const float* mVl = mV + (unsigned)(3 * l) * hw0;
        const float* mNl = mN + (unsigned)(3 * l) * hw0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float* Vpl = mVl + r * hw0;
          const float* Npl = mNl + r * hw0;
          ql[r] += w00 * Vpl[t00] + w10 * Vpl[t10] + w01 * Vpl[t01] + w11 * Vpl[t11];
          nl[r] += w00 * Npl[t00] + w10 * Npl[t10] + w01 * Npl[t01] + w11 * Npl[t11];
        }
      }
      const float dfl[3] = {ppl[0] - ql[0], ppl[1] - ql[1], ppl[2] - ql[2]};
      const float resl = m * (dfl[0] * nn[0] + dfl[1] * nn[1] + dfl[2] * nn[2] + df[0] * nl[0] + df[1] * nl[1] +
                              df[2] * nl[2]);
      const float Jl[6] = {m * (ppl[1] * nn[2] - ppl[2] * nn[1] + pp[1] * nl[2] - pp[2] * nl[1]),
                           m * (ppl[2] * nn[0] - ppl[0] * nn[2] + pp[2] * nl[0] - pp[0] * nl[2]),
                           m * (ppl[0] * nn[1] - ppl[1] * nn[0] + pp[0] * nl[1] - pp[1] * nl[0]),
                           m * nl[0], m * nl[1], m * nl[2]};
      int k = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = r; cc < 6; ++cc, ++k) cv[k] = J[r] * Jl[cc] + Jl[r] * J[cc];
#pragma unroll
      for (int r = 0; r < 6; ++r) cv[21 + r] = J[r] * resl + Jl[r] * res;
#pragma unroll
      for (int r = 27; r < 32; ++r) cv[r] = 0.f;
      const float sum = warp_transpose_sum(cv, lid);
      if (lid < kNT) wacc[l * kNT + lid] += sum;
    }
  }
}

// Block sums: the warps' sums (wacc [warp][lane][27]) added in warp order into column `col` of the
// value-major partials ([value][stride], so that the cross-block sum reads each value's row with
// coalesced loads), the correspondence count into partial_n[col]. The last column of a launch pads its
// rows with zeros up to the stride.
__device__ __forceinline__ void icp_block_sums(IcpShared& S, int cnt, int L, int warp, int lid,
                                               const float* __restrict__ wacc, float* __restrict__ partial,
                                               int pst, int col, int ncol, int* __restrict__ partial_n) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lid == 0) S.s_cnt[warp] = cnt;
  __syncthreads();
  for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kIcpWarps; ++w) s += wacc[w * L * kNT + i];
    partial[(size_t)i * pst + col] = s;
    if (col == ncol - 1)  // the row padding of this launch's stride reads as zero
      for (int k = ncol; k < pst; ++k) partial[(size_t)i * pst + k] = 0.f;
  }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < kIcpWarps; ++w) c += S.s_cnt[w];
    partial_n[col] = c;
  }
}

// Cross-block sum of the partials of `ncol` blocks into S.sAh / S.sAl (27 L values, double-FP32) and
// S.s_ncorr. Value v is summed by two threads, one per half of its row: all float4 loads of a half (up
// to 20, i.e. up to 160 columns) issued together, FP32 sums of 16 partials, double-FP32 accumulation of
// those sums and of the two halves. The order is fixed by the column count alone: every block that runs
// it gets the same bits.
__device__ __forceinline__ void icp_cross_sum(IcpShared& S, const float* __restrict__ partial, int pst, int ncol,
                                              const int* __restrict__ partial_n, int L, int warp, int lid) {
  const int NV = L * kNT;
  if (warp == (int)(blockDim.x >> 5) - 1) {
    // the last warp adds the per-block correspondence counts: 8 loads per lane in flight at once
    int c = 0;
    for (int k0 = 0; k0 < ncol; k0 += 256) {
      int q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + lid + 32 * j;
        q[j] = k < ncol ? __ldcg(&partial_n[k]) : 0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) c += q[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lid == 0) S.s_ncorr = c;
  }
  const int n4 = pst >> 2, h4 = (n4 + 1) >> 1;
  for (int t = threadIdx.x; t < 2 * NV; t += blockDim.x) {
    const int v = t >> 1, half = t & 1;
    const float4* row = reinterpret_cast<const float4*>(partial + (size_t)v * pst) + half * h4;
    const int cnt = half ? n4 - h4 : h4;
    DF acc = {0.f, 0.f};
    for (int c0 = 0; c0 < cnt; c0 += 20) {
      float4 q[20];
#pragma unroll
      for (int j = 0; j < 20; ++j) q[j] = (c0 + j < cnt) ? __ldcg(row + c0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      float f[5];
#pragma unroll
      for (int g = 0; g < 5; ++g) {
        f[g] = 0.f;
#pragma unroll
        for (int j = 4 * g; j < 4 * g + 4; ++j) f[g] += (q[j].x + q[j].y) + (q[j].z + q[j].w);
      }
      // the five group sums added as a tree
      acc = df_add(acc, df_add_f(df_add(two_sum(f[0], f[1]), two_sum(f[2], f[3])), f[4]));
    }
    S.s_halfh[t] = acc.h;
    S.s_halfl[t] = acc.l;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += blockDim.x) {
    const DF a = df_add({S.s_halfh[2 * v], S.s_halfl[2 * v]}, {S.s_halfh[2 * v + 1], S.s_halfl[2 * v + 1]});
    S.sAh[v] = a.h;
    S.sAl[v] = a.l;
  }
  __syncthreads();
}

// The 6x6 solve of the summed normal equations: factor the real A once, x_0 = A^-1 (-g_0) and
// x_l = A^-1 (-g_l - A_l x_0) on every lane, each refined once with double-FP32 residuals. Sets S.s_fail
// (too few correspondences, A not positive definite, or `skip`) and S.sx.
__device__ __forceinline__ DF sA_df(const IcpShared& S, int i) { return {S.sAh[i], S.sAl[i]}; }

// base - (p0 + ... + p5) with the products summed as a tree (3 levels instead of a chain of 6)
__device__ __forceinline__ DF df_sub_sum6(DF base, const DF* pr) {
  const DF s = df_add(df_add(df_add(pr[0], pr[1]), df_add(pr[2], pr[3])), df_add(pr[4], pr[5]));
  return df_add(base, df_neg(s));
}

__device__ __forceinline__ void icp_solve(const Params& p, IcpShared& S, int L, int npx, bool skip, bool update) {
  const int t = threadIdx.x;
  if (t == 0) {
    int fail = skip;
    if (!fail && (float)S.s_ncorr < p.min_corr_frac * (float)npx) fail = 1;
    if (!fail && !ldl32(S.sAh, S.s_ldl)) fail = 1;  // the high parts: the sums rounded to FP32
    if (!fail) {
      float b0[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) b0[i] = -S.sAh[21 + i];
      subst32(S.s_ldl, b0, S.sxf[0]);
    }
    S.s_fail = fail;
  }
  __syncthreads();
  const bool go = update && !S.s_fail;
  // real lane: residual -g_0 - A x_0 in double-FP32 (thread i = row), FP32 correction
  if (go && t < 6) {
    DF pr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) pr[k] = df_mul_f(sA_df(S, t <= k ? up6(t, k) : up6(k, t)), S.sxf[0][k]);
    S.srf[0][t] = df_sub_sum6(df_neg(sA_df(S, 21 + t)), pr).h;
  }
  __syncthreads();
  if (go && t == 0) subst32(S.s_ldl, S.srf[0], S.sdf[0]);
  __syncthreads();
  if (go && t < 6) {
    const DF x = two_sum(S.sxf[0][t], S.sdf[0][t]);  // exact
    S.sx0h[t] = x.h;
    S.sx0l[t] = x.l;
    S.sx[0][t] = (double)x.h + (double)x.l;
  }
  __syncthreads();
  // imaginary lanes: right-hand sides -g_l - A_l x_0 in double-FP32, thread (l, i)
  const int ls = 1 + t / 6, li = t % 6;
  const bool lane_thread = go && t < 6 * (L - 1);
  DF rhs = {0.f, 0.f};
  if (lane_thread) {
    const int o = ls * kNT;
    DF pr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) pr[k] = df_mul(sA_df(S, o + (li <= k ? up6(li, k) : up6(k, li))), DF{S.sx0h[k], S.sx0l[k]});
    rhs = df_sub_sum6(df_neg(sA_df(S, o + 21 + li)), pr);
    S.srf[ls][li] = rhs.h;
  }
  __syncthreads();
  if (go && t >= 1 && t < L) subst32(S.s_ldl, S.srf[t], S.sxf[t]);
  __syncthreads();
  if (lane_thread) {
    DF pr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) pr[k] = df_mul_f(sA_df(S, li <= k ? up6(li, k) : up6(k, li)), S.sxf[ls][k]);
    S.srf[ls][li] = df_sub_sum6(rhs, pr).h;
  }
  __syncthreads();
  if (go && t >= 1 && t < L) subst32(S.s_ldl, S.srf[t], S.sdf[t]);
  __syncthreads();
  if (lane_thread) S.sx[ls][li] = (double)S.sxf[ls][li] + (double)S.sdf[ls][li];
  __syncthreads();
}

// Pose update T <- exp(x) T on every lane of the pose lanes at `pose` (in place): delta = exp(x) - I in
// FP32 (coefficients once per lane, then one thread per (lane, element)), T + delta T composed in FP64
// one element per thread.
__device__ __forceinline__ void icp_update(IcpShared& S, int L, double* pose) {
  const int t = threadIdx.x;
  const bool elem = t < 12 * L;
  // this thread's element (l, e = 4 r + c) reads 7 values of the old pose: loaded first, so that their
  // latency passes while the increments are formed
  double te = 0.0, t0c[3] = {0.0, 0.0, 0.0}, tlc[3] = {0.0, 0.0, 0.0};
  if (elem) {
    const int l = t / 12, e = t % 12, c = e & 3;
    te = pose[12 * l + e];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      t0c[q] = pose[4 * q + c];
      tlc[q] = pose[12 * l + 4 * q + c];
    }
  }
  if (t < 6 * L) S.sxs[t / 6][t % 6] = (float)S.sx[t / 6][t % 6];
  __syncthreads();
  if (t < L) se3_coef_lane_f(S.sxs[0], S.sxs[t], S.scf[t]);
  __syncthreads();
  if (elem) {
    const int l = t / 12, e = t % 12;
    S.sdl[l][e] = se3_delta_element(S.sxs[0], S.sxs[l], S.scf[l], l > 0, e);
  }
  __syncthreads();
  double tn = 0.0;
  if (elem) {
    const int l = t / 12, e = t % 12, r = e >> 2, c = e & 3;
    // lane 0: T0 + d0 T0; lane l: Tl + dl T0 + d0 Tl (translation column adds the delta's own column)
    tn = te + (double)S.sdl[l][4 * r] * t0c[0] + (double)S.sdl[l][4 * r + 1] * t0c[1] +
         (double)S.sdl[l][4 * r + 2] * t0c[2] + (c == 3 ? (double)S.sdl[l][4 * r + 3] : 0.0);
    if (l > 0)
      tn += (double)S.sdl[0][4 * r] * tlc[0] + (double)S.sdl[0][4 * r + 1] * tlc[1] +
            (double)S.sdl[0][4 * r + 2] * tlc[2];
  }
  __syncthreads();
  if (elem) pose[t] = tn;
  __syncthreads();
}

// the pyramid level's image size and intrinsics
__device__ __forceinline__ Lvl icp_level(const Params& p, int level) {
  Lvl lv;
  lv.s = 1 << level;
  lv.level = level;
  lv.W = p.W >> level;
  lv.H = p.H >> level;
  lv.fx = p.fx / lv.s;
  lv.fy = p.fy / lv.s;
  lv.cx = p.cx / lv.s;
  lv.cy = p.cy / lv.s;
  return lv;
}

// One Gauss-Newton iteration; (bx, gx): this block in its trajectory's grid. The last block to finish
// (ticket counter) sums, solves and updates. kStop: the stop tolerance p.icp_stop is in use (and the
// iteration counter): a launch after its level converged returns at once. Without it the kernel is the
// fixed-count iteration of the method.
template <bool kStop>
__device__ __forceinline__ void icp_body(const Params& p, const Buffers& b, const Lvl& lv, int flags, int bx, int gx) {
  const int L = p.L;
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  __shared__ IcpShared S;
  __shared__ int s_skip, s_last, s_conv;
  extern __shared__ __align__(16) float icp_wacc[];  // icp_dyn_bytes(L): the warps' sums

  if (threadIdx.x == 0) {
    s_skip = b.status[0];
    // status[3]: the level converged (a step below p.icp_stop); only its first iteration ignores it
    if (kStop) s_conv = (flags & (kIcpFirst | kIcpNoUpdate)) ? 0 : b.status[3];
  }
  icp_prologue(p, b.pose, b.pose_prev, S, L, icp_wacc);
  if (kStop && (s_skip || s_conv) && !(flags & kIcpNoUpdate)) {
    // nothing to compute after a failure or after the level converged; the frame's last iteration
    // still closes the frame: fall back to T_{k-1} on a failure and count it
    if ((flags & kIcpLast) && bx == 0) {
      if (s_skip && threadIdx.x < 12 * L) b.pose[threadIdx.x] = b.pose_prev[threadIdx.x];
      if (threadIdx.x == 0) {
        if (s_skip) {
          b.status[1] += 1;
          b.status[2] = 0;
        }
        b.status[0] = 0;
        b.status[3] = 0;
      }
    }
    return;
  }

  int cnt = 0;
  const int npx = lv.W * lv.H;
  const int nchunk = (npx + 31) >> 5;
  const int G = icp_groups(nchunk, gx * kIcpWarps, L);
  const int gw = bx * kIcpWarps + warp, nslot = (gx * kIcpWarps) / G;  // chunk slots of G warps each
  if (!s_skip && gw < nslot * G)
    icp_chunks(p, b, lv, S, L, warp, lid, gw / G, nslot, nchunk, cnt, icp_wacc + warp * L * kNT, gw % G, G);

  const int pst = icp_pstride(gx);
  icp_block_sums(S, cnt, L, warp, lid, icp_wacc, b.partial, pst, bx, gx, b.partial_n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(b.ticket, 1u);
    s_last = (t == gx - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) *b.ticket = 0u;  // ready for the next launch

  // ---------------- last block: double-FP32 cross-block sum, solve, update ----------------
  icp_cross_sum(S, b.partial, pst, gx, b.partial_n, L, warp, lid);
  if (flags & kIcpNoUpdate) {
    for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) b.result[kResSys + i] = (double)S.sAh[i] + (double)S.sAl[i];
    if (threadIdx.x == 0) b.status[2] = S.s_ncorr;
    return;
  }
  icp_solve(p, S, L, npx, s_skip, true);
  const bool go = !S.s_fail;
  if (go) icp_update(S, L, b.pose);
  if (kStop) {
    if (threadIdx.x == 0) {
      if (S.s_fail) b.status[0] = 1;
      b.status[2] = S.s_ncorr;
      double x2 = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) x2 += S.sx[0][k] * S.sx[0][k];
      b.status[3] = (go && x2 < (double)p.icp_stop * (double)p.icp_stop) ? 1 : 0;
      if (b.stats) b.stats[kStatIcpIters] += 1;
    }
  } else if (threadIdx.x == 0 && S.s_fail && !s_skip) {
    b.status[0] = 1;
  }
  if (flags & kIcpLast) {
    __syncthreads();
    const int failed = b.status[0];
    const int t = threadIdx.x;
    if (failed && t < 12 * L) b.pose[t] = b.pose_prev[t];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (failed) b.status[1] += 1;
      b.status[0] = 0;
      b.status[2] = S.s_ncorr;
    }
  }
}

template <bool kStop>
__global__ void __launch_bounds__(kIcpThreads, 1) k_icp(Params p, Buffers b, Lvl lv, int flags) {
  pdl_enter();
  icp_body<kStop>(p, b, lv, flags, blockIdx.x, gridDim.x);
}

// segments: arg = pyramid level | iteration flags << 4 (fixed-count iterations)
__global__ void __launch_bounds__(kIcpThreads, 1) k_icp_seg(SegTable st) {
  pdl_enter();
  const Seg sg = st.seg[seg_find(st, blockIdx.x)];
  const TrajDesc& d = st.desc[sg.traj];
  icp_body<false>(d.p, d.b, icp_level(d.p, sg.arg & 15), sg.arg >> 4, blockIdx.x - sg.block0, sg.nblk);
}

cudaError_t launch_icp_seg(const SegTable& t, int nblocks, int max_lanes, cudaStream_t s) {
  return launch_pdl(k_icp_seg, dim3(nblocks), dim3(kIcpThreads), (size_t)icp_dyn_bytes(max_lanes), s, t);
}

// the kernels' dynamic shared memory above the default 48 KB (once per device of the process)
cudaError_t icp_configure() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  const int bytes = icp_dyn_bytes(kMaxLanes);
  if ((e = cudaFuncSetAttribute(k_icp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_icp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_icp_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if (dev >= 0 && dev < 64) done[dev] = true;
  return cudaSuccess;
}

int icp_blocks(int level_pixels, int L) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one chunk of 32 pixels per warp (per lane group) at least: small levels get fewer blocks (fewer
  // partials to add)
  const int nchunk = (level_pixels + 31) / 32;
  const int G = icp_groups(nchunk, sms * kIcpWarps, L);
  int nblk = (nchunk * G + kIcpWarps - 1) / kIcpWarps;
  if (nblk > sms) nblk = sms;
  if (nblk > kMaxPartials) nblk = kMaxPartials;
  if (nblk < 1) nblk = 1;
  return nblk;
}

cudaError_t launch_icp(const Params& p, const Buffers& b, int level, int flags, int nblk, cudaStream_t s) {
  Lvl lv;
  lv.s = 1 << level;
  lv.level = level;
  lv.W = p.W >> level;
  lv.H = p.H >> level;
  lv.fx = p.fx / lv.s;
  lv.fy = p.fy / lv.s;
  lv.cx = p.cx / lv.s;
  lv.cy = p.cy / lv.s;
  const size_t dyn = (size_t)icp_dyn_bytes(p.L);
  const cudaError_t e = p.icp_stop > 0.f
                            ? launch_pdl(k_icp<true>, dim3(nblk), dim3(kIcpThreads), dyn, s, p, b, lv, flags)
                            : launch_pdl(k_icp<false>, dim3(nblk), dim3(kIcpThreads), dyn, s, p, b, lv, flags);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace xslam
