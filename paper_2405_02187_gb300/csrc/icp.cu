// Projective point-to-plane ICP (X-SLAM Sec. 4.1, "Differentiable ICP") on 1 + K lanes: one launch
// per Gauss-Newton iteration.
//
// Per pixel u of pyramid level l: V = D K_l^-1 u, N = normalize((V(u+x) - V) x (V(u+y) - V)) (Eq. vertex,
// Eq. normal), p' = T_j V, u_hat = pi(K_l T_{k-1}^-1 p'), q and n = bilinear model vertex / normal at
// u_hat (level-0 model maps read at pixel 2^l u_hat), r = (p' - q).n, J = [(p' x n)^T, n^T]; the
// normal equations A = sum J J^T, g = sum J r (Eq. icp, Eq. "icp approx") are reduced, A x = -g is
// solved and T_{j+1} = exp(x) T_j.
//
// GB300 mapping: a block holds L = 1 + K warps per replica; warp `lane` of a replica computes the
// real part of its 32 pixels and, if lane > 0, the tangent of that lane, accumulating only 27 FP32
// sums per thread; replicas of a block share pixel chunks through L1. Warp shuffles and shared
// memory reduce each block to one FP32 partial per lane; the last block to finish (ticket counter,
// no grid-wide wait) adds the partials in FP64, factors the real 6x6 matrix by Cholesky (FP64), solves
// the K + 1 right-hand sides (x_0 from the real part, x_j = A^-1 (-g_j - A_j x_0) for each lane) and
// composes exp(x) T_j on every lane in FP64.
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

// The 6x6 solve. A = L D L^T is factored in FP32 (square-root-free Cholesky) and every right-hand
// side is solved by mixed-precision iterative refinement: x = S(b), r = b - A x in FP64 (A and b are
// the FP64 sums), x += S(r), with S the FP32 forward/back substitution; one round brings the relative
// error from ~cond(A) 2^-24 to ~(cond(A) 2^-24)^2. On GB300 every FP64 warp instruction occupies the
// SM sub-partition's FP64 pipe for ~64-80 cycles whatever the number of active threads, so the FP64
// steps of the tail run SIMT-parallel: one thread per (system, row) or per matrix element.
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

__device__ __forceinline__ void accum(float* acc, const float* Ja, const float ra, const float* Jb, const float rb) {
  // acc += Ja Jb^T + Jb Ja^T (upper triangle) and Ja rb + Jb ra; called with (J, r, J, r) * 0.5 for
  // the real lane and with (J, r, J_l, r_l) for a tangent lane.
  int q = 0;
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = r; c < 6; ++c) acc[q++] += Ja[r] * Jb[c] + Jb[r] * Ja[c];
#pragma unroll
  for (int r = 0; r < 6; ++r) acc[21 + r] += Ja[r] * rb + Jb[r] * ra;
}

// fields of the per-pixel record handed from the real warp to the lane warps (SoA, [field][32])
enum : int {
  RV = 0, RD, RRX, RRY, RE, RQX = RE + 3, RQY, RIZ, RA, RB, RT, RPP, RN = RPP + 3, RDF = RN + 3, RDQA = RDF + 3,
  RDQB = RDQA + 3, RDNA = RDQB + 3, RDNB = RDNA + 3, RJ = RDNB + 3, RRES = RJ + 6, kRec
};
constexpr int kMaxReps = 4;

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Shared memory of the ICP kernels (static part; the per-pixel records are dynamic).
struct IcpShared {
  float sT[kMaxLanes][12];   // pose lanes of the current iterate (FP32 copy for the pixel work)
  float sP[kMaxLanes][12];   // pose lanes the model was ray cast at
  float sZero[12];
  float s_red[kNT * kMaxLanes];  // [rep][lane][27]; reps * L <= 16 by construction
  int s_cnt[32];
  double sA[kMaxLanes * kNT];
  double sx[kMaxLanes][6];
  Ldl32 s_ldl;
  double s_half[2 * kNT * kMaxLanes];
  float sAf[kNT * kMaxLanes];
  float sxf[kMaxLanes][6], srf[kMaxLanes][6], sdf[kMaxLanes][6];
  SeCoefF scf[kMaxLanes];
  float sxs[kMaxLanes][6];
  float sdl[kMaxLanes][12];
  int s_ncorr, s_fail;
};

// Level-l pixel chunks of this replica: groups gbase, gbase + gstride, ... of L chunks of 32 pixels.
// Every warp of the replica computes the real part of one chunk of the group (correspondence, residual,
// Jacobian, bilinear derivatives) into a shared-memory record; after a named barrier every warp reads
// all L records and adds the sums of its own lane: lane 0 the real normal equations, lane l > 0 their
// tangent, for which it loads only lane l's model taps. A second barrier frees the records.
__device__ __forceinline__ void icp_pixels(const Params& p, const Buffers& b, const Lvl& lv, const IcpShared& S,
                                           float* __restrict__ recs, int L, int ln, int lid, int rep, int gbase,
                                           int gstride, int nloop, float* acc, int& cnt) {
  const float* D = lv.s == 1 ? b.pyr[0] : (lv.s == 2 ? b.pyr[1] : b.pyr[2]);
  const size_t hw0 = (size_t)p.W * p.H;
  const float* mdep = b.model;
  const float* mV = b.model + hw0;
  const float* mN = b.model + hw0 * (1 + 3 * L);
  const int npx = lv.W * lv.H;
  for (int it = 0; it < nloop; ++it) {
    const int ch = (gbase + it * gstride) * L + ln;
    {
      // ---------------- real part (every warp produces one chunk's records) ----------------
      float* rec = recs + ln * kRec * 32;
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
      const float* T = S.sT[0];
      const float* P = S.sP[0];
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
      const float pcx = P[0] * e0 + P[4] * e1 + P[8] * e2;
      const float pcy = P[1] * e0 + P[5] * e1 + P[9] * e2;
      const float pcz = P[2] * e0 + P[6] * e1 + P[10] * e2;
      ok = ok && pcz > 0.f;
      const float iz = ok ? 1.f / pcz : 0.f;
      const float qx = pcx * iz, qy = pcy * iz;
      const float ux = lv.fx * qx + lv.cx, uy = lv.fy * qy + lv.cy;
      const float ci = floorf(ux + kCellBias), cj = floorf(uy + kCellBias);
      ok = ok && ci >= 0.f && ci <= (float)(lv.W - 2) && cj >= 0.f && cj <= (float)(lv.H - 2);
      const int i0 = ok ? (int)ci : 0, j0 = ok ? (int)cj : 0;
      const float a = ux - ci, bb = uy - cj;
      const size_t t00 = (size_t)(j0 * lv.s) * p.W + (size_t)(i0 * lv.s);
      const size_t t10 = t00 + lv.s, t01 = t00 + (size_t)lv.s * p.W, t11 = t01 + lv.s;
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
      float q[3] = {0.f, 0.f, 0.f}, nn[3] = {0.f, 0.f, 0.f};
      float dqa[3] = {0.f, 0.f, 0.f}, dqb[3] = {0.f, 0.f, 0.f}, dna[3] = {0.f, 0.f, 0.f}, dnb[3] = {0.f, 0.f, 0.f};
      if (ok) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float* Vp = mV + (size_t)r * hw0;
          const float* Np = mN + (size_t)r * hw0;
          const float v00 = Vp[t00], v10 = Vp[t10], v01 = Vp[t01], v11 = Vp[t11];
          const float m00 = Np[t00], m10 = Np[t10], m01 = Np[t01], m11 = Np[t11];
          q[r] = w00 * v00 + w10 * v10 + w01 * v01 + w11 * v11;
          nn[r] = w00 * m00 + w10 * m10 + w01 * m01 + w11 * m11;
          dqa[r] = (1.f - bb) * (v10 - v00) + bb * (v11 - v01);
          dqb[r] = (1.f - a) * (v01 - v00) + a * (v11 - v10);
          dna[r] = (1.f - bb) * (m10 - m00) + bb * (m11 - m01);
          dnb[r] = (1.f - a) * (m01 - m00) + a * (m11 - m10);
        }
      }
      const float df[3] = {pp[0] - q[0], pp[1] - q[1], pp[2] - q[2]};
      ok = ok && df[0] * df[0] + df[1] * df[1] + df[2] * df[2] <= p.dist_gate2;
      float nw[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) nw[r] = T[4 * r] * Nm[0] + T[4 * r + 1] * Nm[1] + T[4 * r + 2] * Nm[2];
      const float nl2 = nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2];
      ok = ok && fabsf(nw[0] * nn[0] + nw[1] * nn[1] + nw[2] * nn[2]) >= p.cos_normal_gate * sqrtf(nl2);
      const float res = df[0] * nn[0] + df[1] * nn[1] + df[2] * nn[2];
      const float J[6] = {pp[1] * nn[2] - pp[2] * nn[1], pp[2] * nn[0] - pp[0] * nn[2], pp[0] * nn[1] - pp[1] * nn[0],
                          nn[0], nn[1], nn[2]};
      {
        float* R_ = rec + lid;
        R_[RV * 32] = __int_as_float(ok ? px + 1 : 0);  // 0: no correspondence; else the pixel + 1
        if (ok) {
          R_[RD * 32] = d0;
          R_[RRX * 32] = rx;
          R_[RRY * 32] = ry;
          R_[RE * 32] = e0;
          R_[(RE + 1) * 32] = e1;
          R_[(RE + 2) * 32] = e2;
          R_[RQX * 32] = qx;
          R_[RQY * 32] = qy;
          R_[RIZ * 32] = iz;
          R_[RA * 32] = a;
          R_[RB * 32] = bb;
          R_[RT * 32] = __int_as_float((int)t00);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            R_[(RPP + r) * 32] = pp[r];
            R_[(RN + r) * 32] = nn[r];
            R_[(RDF + r) * 32] = df[r];
            R_[(RDQA + r) * 32] = dqa[r];
            R_[(RDQB + r) * 32] = dqb[r];
            R_[(RDNA + r) * 32] = dna[r];
            R_[(RDNB + r) * 32] = dnb[r];
          }
#pragma unroll
          for (int r = 0; r < 6; ++r) R_[(RJ + r) * 32] = J[r];
          R_[RRES * 32] = res;
        }
      }
    }
    named_barrier(1 + rep, 32 * L);
    for (int j = 0; j < L; ++j) {
      // ---------------- lane `ln` of the records of chunk j (consumer) ----------------
      const float* R_ = recs + j * kRec * 32 + lid;
      if (!__float_as_int(R_[RV * 32])) continue;
      if (ln == 0) {
        ++cnt;
        float J[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) J[r] = R_[(RJ + r) * 32];
        const float res = R_[RRES * 32];
        const float hJ[6] = {0.5f * J[0], 0.5f * J[1], 0.5f * J[2], 0.5f * J[3], 0.5f * J[4], 0.5f * J[5]};
        accum(acc, hJ, 0.5f * res, J, res);
      } else {
        const float* T = S.sT[0];
        const float* P = S.sP[0];
        const float* Tl = S.sT[ln];
        // a restarted lane (per-frame pose seed) carries no derivative in the previous pose or the model
        const bool fresh = (p.fresh >> ln) & 1u;
        const float* Pl = fresh ? S.sZero : S.sP[ln];
        const float d0 = R_[RD * 32], rx = R_[RRX * 32], ry = R_[RRY * 32];
        const float V[3] = {d0 * rx, d0 * ry, d0};
        float dDl = p.dD[ln];
        if (p.dpix[ln] >= 0)  // single-pixel DEPTH lane: the level's Im depth map at this pixel
          dDl += b.dlane[dlane_offset(p, ln, lv.level) + (__float_as_int(R_[RV * 32]) - 1)];
        const float Vl[3] = {dDl * rx, dDl * ry, dDl};
        const float e0 = R_[RE * 32], e1 = R_[(RE + 1) * 32], e2 = R_[(RE + 2) * 32];
        const float qx = R_[RQX * 32], qy = R_[RQY * 32], iz = R_[RIZ * 32];
        const float a = R_[RA * 32], bb = R_[RB * 32];
        const size_t t00 = (size_t)__float_as_int(R_[RT * 32]);
        const size_t t10 = t00 + lv.s, t01 = t00 + (size_t)lv.s * p.W, t11 = t01 + lv.s;
        float pp[3], nn[3], df[3], J[6];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          pp[r] = R_[(RPP + r) * 32];
          nn[r] = R_[(RN + r) * 32];
          df[r] = R_[(RDF + r) * 32];
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) J[r] = R_[(RJ + r) * 32];
        const float res = R_[RRES * 32];
        float ppl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
          ppl[r] = Tl[4 * r] * V[0] + Tl[4 * r + 1] * V[1] + Tl[4 * r + 2] * V[2] + Tl[4 * r + 3] +
                   T[4 * r] * Vl[0] + T[4 * r + 1] * Vl[1] + T[4 * r + 2] * Vl[2];
        const float el0 = ppl[0] - Pl[3], el1 = ppl[1] - Pl[7], el2 = ppl[2] - Pl[11];
        const float pcxl = Pl[0] * e0 + Pl[4] * e1 + Pl[8] * e2 + P[0] * el0 + P[4] * el1 + P[8] * el2;
        const float pcyl = Pl[1] * e0 + Pl[5] * e1 + Pl[9] * e2 + P[1] * el0 + P[5] * el1 + P[9] * el2;
        const float pczl = Pl[2] * e0 + Pl[6] * e1 + Pl[10] * e2 + P[2] * el0 + P[6] * el1 + P[10] * el2;
        const float al = lv.fx * (pcxl - qx * pczl) * iz;
        const float bl = lv.fy * (pcyl - qy * pczl) * iz;
        const float w00 = (1.f - a) * (1.f - bb), w10 = a * (1.f - bb), w01 = (1.f - a) * bb, w11 = a * bb;
        const float* mVl = mV + (size_t)(3 * ln) * hw0;
        const float* mNl = mN + (size_t)(3 * ln) * hw0;
        float ql[3], nl[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          ql[r] = R_[(RDQA + r) * 32] * al + R_[(RDQB + r) * 32] * bl;
          nl[r] = R_[(RDNA + r) * 32] * al + R_[(RDNB + r) * 32] * bl;
        }
        if (!fresh) {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float* Vpl = mVl + (size_t)r * hw0;
            const float* Npl = mNl + (size_t)r * hw0;
            ql[r] += w00 * Vpl[t00] + w10 * Vpl[t10] + w01 * Vpl[t01] + w11 * Vpl[t11];
            nl[r] += w00 * Npl[t00] + w10 * Npl[t10] + w01 * Npl[t01] + w11 * Npl[t11];
          }
        }
        const float dfl[3] = {ppl[0] - ql[0], ppl[1] - ql[1], ppl[2] - ql[2]};
        const float resl = dfl[0] * nn[0] + dfl[1] * nn[1] + dfl[2] * nn[2] + df[0] * nl[0] + df[1] * nl[1] + df[2] * nl[2];
        const float Jl[6] = {ppl[1] * nn[2] - ppl[2] * nn[1] + pp[1] * nl[2] - pp[2] * nl[1],
                             ppl[2] * nn[0] - ppl[0] * nn[2] + pp[2] * nl[0] - pp[0] * nl[2],
                             ppl[0] * nn[1] - ppl[1] * nn[0] + pp[0] * nl[1] - pp[1] * nl[0],
                             nl[0], nl[1], nl[2]};
        accum(acc, J, res, Jl, resl);
      }
    }
    named_barrier(1 + rep, 32 * L);
  }
}

// Block reduction of the threads' sums: warp shuffles, then the replicas of a lane added in shared
// memory; the block's 27 L sums go to column `col` of the value-major partials ([value][stride], so that
// the cross-block sum reads each value's row with coalesced loads) and its correspondence count to
// partial_n[col]. The last column of a launch pads its rows with zeros up to the stride.
__device__ __forceinline__ void icp_block_sums(IcpShared& S, float* acc, int cnt, int L, int reps, int ln, int rep,
                                               int warp, int lid, float* __restrict__ partial, int pst, int col,
                                               int ncol, int* __restrict__ partial_n) {
#pragma unroll
  for (int q = 0; q < kNT; ++q) {
    float x = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    acc[q] = x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lid == 0) {
#pragma unroll
    for (int q = 0; q < kNT; ++q) S.s_red[(rep * L + ln) * kNT + q] = acc[q];
    S.s_cnt[warp] = cnt;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < reps; ++r) s += S.s_red[r * L * kNT + i];
    partial[(size_t)i * pst + col] = s;
    if (col == ncol - 1)  // the row padding of this launch's stride reads as zero
      for (int k = ncol; k < pst; ++k) partial[(size_t)i * pst + k] = 0.f;
  }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < reps; ++r) c += S.s_cnt[r * L];
    partial_n[col] = c;
  }
}

// FP64 cross-block sum of the partials of `ncol` blocks into S.sA (27 L values) and S.s_ncorr. Value v
// is summed by two threads, one per half of its row: all float4 loads of a half (up to 20, i.e. up to
// 160 columns) issued together, FP32 sums of 16 partials, FP64 accumulation of those sums, FP64 add of
// the two halves. Different values sit in different lanes, so each FP64 warp instruction adds 32 values.
// The order is fixed by the column count alone: every block that runs it gets the same bits.
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
    double acc = 0.0;
    for (int c0 = 0; c0 < cnt; c0 += 20) {
      float4 q[20];
#pragma unroll
      for (int j = 0; j < 20; ++j) q[j] = (c0 + j < cnt) ? __ldcg(row + c0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int g = 0; g < 5; ++g) {
        float f = 0.f;
#pragma unroll
        for (int j = 4 * g; j < 4 * g + 4; ++j) f += (q[j].x + q[j].y) + (q[j].z + q[j].w);
        acc += (double)f;
      }
    }
    S.s_half[t] = acc;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += blockDim.x) S.sA[v] = S.s_half[2 * v] + S.s_half[2 * v + 1];
  __syncthreads();
}

// The 6x6 solve of the summed normal equations: factor the real A once, x_0 = A^-1 (-g_0) and
// x_l = A^-1 (-g_l - A_l x_0) on every lane, each refined once with FP64 residuals. Sets S.s_fail (too
// few correspondences, A not positive definite, or `skip`) and S.sx.
__device__ __forceinline__ void icp_solve(const Params& p, IcpShared& S, int L, int npx, bool skip, bool update) {
  const int NV = L * kNT;
  const int t = threadIdx.x;
  for (int v = t; v < NV; v += blockDim.x) S.sAf[v] = (float)S.sA[v];
  __syncthreads();
  if (t == 0) {
    int fail = skip;
    if (!fail && (float)S.s_ncorr < p.min_corr_frac * (float)npx) fail = 1;
    if (!fail && !ldl32(S.sAf, S.s_ldl)) fail = 1;
    if (!fail) {
      float b0[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) b0[i] = -S.sAf[21 + i];
      subst32(S.s_ldl, b0, S.sxf[0]);
    }
    S.s_fail = fail;
  }
  __syncthreads();
  const bool go = update && !S.s_fail;
  // real lane: residual in FP64 (thread i = row), FP32 correction
  if (go && t < 6) {
    double r = -S.sA[21 + t];
#pragma unroll
    for (int k = 0; k < 6; ++k) r = fma(-S.sA[t <= k ? up6(t, k) : up6(k, t)], (double)S.sxf[0][k], r);
    S.srf[0][t] = (float)r;
  }
  __syncthreads();
  if (go && t == 0) subst32(S.s_ldl, S.srf[0], S.sdf[0]);
  __syncthreads();
  if (go && t < 6) S.sx[0][t] = (double)S.sxf[0][t] + (double)S.sdf[0][t];
  __syncthreads();
  // imaginary lanes: right-hand sides in FP64, thread (l, i)
  const int ls = 1 + t / 6, li = t % 6;
  const bool lane_thread = go && t < 6 * (L - 1);
  double rhs = 0.0;
  if (lane_thread) {
    const double* Al = S.sA + ls * kNT;
    rhs = -Al[21 + li];
#pragma unroll
    for (int k = 0; k < 6; ++k) rhs = fma(-Al[li <= k ? up6(li, k) : up6(k, li)], S.sx[0][k], rhs);
    S.srf[ls][li] = (float)rhs;
  }
  __syncthreads();
  if (go && t >= 1 && t < L) subst32(S.s_ldl, S.srf[t], S.sxf[t]);
  __syncthreads();
  if (lane_thread) {
    double r = rhs;
#pragma unroll
    for (int k = 0; k < 6; ++k) r = fma(-S.sA[li <= k ? up6(li, k) : up6(k, li)], (double)S.sxf[ls][k], r);
    S.srf[ls][li] = (float)r;
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
  if (t < 6 * L) S.sxs[t / 6][t % 6] = (float)S.sx[t / 6][t % 6];
  __syncthreads();
  if (t < L) se3_coef_lane_f(S.sxs[0], S.sxs[t], S.scf[t]);
  __syncthreads();
  if (t < 12 * L) {
    const int l = t / 12, e = t % 12;
    S.sdl[l][e] = se3_delta_element(S.sxs[0], S.sxs[l], S.scf[l], l > 0, e);
  }
  __syncthreads();
  double tn = 0.0;
  if (t < 12 * L) {
    const int l = t / 12, e = t % 12, r = e >> 2, c = e & 3;
    const double* T0 = pose;
    const double* Tl = pose + 12 * l;
    // lane 0: T0 + d0 T0; lane l: Tl + dl T0 + d0 Tl (translation column adds the delta's own column)
    tn = Tl[e] + (double)S.sdl[l][4 * r] * T0[c] + (double)S.sdl[l][4 * r + 1] * T0[4 + c] +
         (double)S.sdl[l][4 * r + 2] * T0[8 + c] + (c == 3 ? (double)S.sdl[l][4 * r + 3] : 0.0);
    if (l > 0)
      tn += (double)S.sdl[0][4 * r] * Tl[c] + (double)S.sdl[0][4 * r + 1] * Tl[4 + c] +
            (double)S.sdl[0][4 * r + 2] * Tl[8 + c];
  }
  __syncthreads();
  if (t < 12 * L) pose[t] = tn;
  __syncthreads();
}

// kStop: the stop tolerance p.icp_stop is in use (and the iteration counter): a launch after its level
// converged returns at once. Without it the kernel is the fixed-count iteration of the method.
// One launch per iteration; the last block to finish (ticket counter) sums, solves and updates. The
// frame chain runs k_icp_run instead; this kernel serves the stage calls (kIcpNoUpdate).
template <bool kStop>
__global__ void __launch_bounds__(512, 1) k_icp(Params p, Buffers b, Lvl lv, int flags, int reps) {
  pdl_enter();
  const int L = p.L;
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  const int ln = warp % L, rep = warp / L;
  __shared__ IcpShared S;
  __shared__ int s_skip, s_last, s_conv;
  extern __shared__ float s_rec[];  // [rep][chunk of the group][field][pixel]: reps * L * kRec * 32 floats

  if (threadIdx.x == 0) {
    s_skip = b.status[0];
    // status[3]: the level converged (a step below p.icp_stop); only its first iteration ignores it
    if (kStop) s_conv = (flags & (kIcpFirst | kIcpNoUpdate)) ? 0 : b.status[3];
  }
  for (int i = threadIdx.x; i < L * 12; i += blockDim.x) {
    S.sT[i / 12][i % 12] = (float)b.pose[i];
    S.sP[i / 12][i % 12] = (float)b.pose_prev[i];
  }
  if (threadIdx.x < 12) S.sZero[threadIdx.x] = 0.f;
  __syncthreads();
  if (kStop && (s_skip || s_conv) && !(flags & kIcpNoUpdate)) {
    // nothing to compute after a failure or after the level converged; the frame's last iteration
    // still closes the frame: fall back to T_{k-1} on a failure and count it
    if ((flags & kIcpLast) && blockIdx.x == 0) {
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

  float acc[kNT];
#pragma unroll
  for (int q = 0; q < kNT; ++q) acc[q] = 0.f;
  int cnt = 0;
  const int npx = lv.W * lv.H;
  const int nchunk = (npx + 31) >> 5;
  const int ngroup = (nchunk + L - 1) / L;
  const int gbase = blockIdx.x * reps + rep, gstride = gridDim.x * reps;
  const int nloop = (!s_skip && gbase < ngroup) ? (ngroup - gbase + gstride - 1) / gstride : 0;
  icp_pixels(p, b, lv, S, s_rec + (size_t)rep * L * kRec * 32, L, ln, lid, rep, gbase, gstride, nloop, acc, cnt);

  const int pst = icp_pstride(gridDim.x);
  icp_block_sums(S, acc, cnt, L, reps, ln, rep, warp, lid, b.partial, pst, blockIdx.x, gridDim.x, b.partial_n);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(b.ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) *b.ticket = 0u;  // ready for the next launch

  // ---------------- last block: FP64 cross-block sum, solve, update ----------------
  icp_cross_sum(S, b.partial, pst, gridDim.x, b.partial_n, L, warp, lid);
  if (flags & kIcpNoUpdate) {
    for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) b.result[kResSys + i] = S.sA[i];
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

// ---------------------------------------------------------------------------------------------------
// All the iterations of a range of pyramid levels in one cooperative launch (every block resident):
// per iteration each block adds its pixels into its column of the partial sums (two buffers, used
// alternately), the grid meets at a barrier, and every block then takes the same FP64 cross-block sum,
// solve and update itself, keeping the pose lanes in its own shared memory, so no second barrier is
// needed: the next iteration's partials go to the other buffer, which no block can still be reading
// (a block writes iteration j + 1's partials only after every block arrived at iteration j's
// barrier, i.e. finished reading iteration j - 1's). Block 0 writes the pose lanes and the status at
// the end. Every wait is bounded: a barrier that does not fill within its poll budget sets status[5]
// and the blocks leave the launch.
// ---------------------------------------------------------------------------------------------------
constexpr unsigned kBarrierPolls = 1u << 22;  // ~0.3 s at the poll interval below

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// returns false if the barrier timed out
__device__ __forceinline__ bool grid_barrier(unsigned* arrive, unsigned target, int* timeout_flag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(arrive, 1u);
    unsigned polls = 0;
    int ok = 1;
    while (ld_acquire_gpu(arrive) < target) {
      if (++polls > kBarrierPolls) {
        ok = 0;
        atomicExch(timeout_flag, 1);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct IcpRange {
  int first, last;   // pyramid levels, coarse (first) to fine (last)
  int iters[3];      // iterations per level
  int close;         // the range's last iteration closes the frame (fallback to T_{k-1}, failure count)
};

template <bool kStop>
__global__ void __launch_bounds__(512, 1) k_icp_run(Params p, Buffers b, IcpRange rg, int reps) {
  // no launch_dependents: the next kernel must not take SM resources while this grid is resident
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int L = p.L;
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  const int ln = warp % L, rep = warp / L;
  __shared__ IcpShared S;
  __shared__ double sTd[kMaxLanes * 12];  // this block's copy of the pose lanes (FP64)
  extern __shared__ float s_rec[];
  float* recs = s_rec + (size_t)rep * L * kRec * 32;
  const int nblk = gridDim.x;
  const int pst = icp_pstride(nblk);
  const size_t pbuf = (size_t)kNT * L * pst;  // floats of one partial buffer

  for (int i = threadIdx.x; i < L * 12; i += blockDim.x) {
    sTd[i] = b.pose[i];
    S.sT[i / 12][i % 12] = (float)sTd[i];
    S.sP[i / 12][i % 12] = (float)b.pose_prev[i];
  }
  if (threadIdx.x < 12) S.sZero[threadIdx.x] = 0.f;
  bool skip = b.status[0] != 0;           // the frame failed in an earlier range
  bool conv = kStop && b.status[3] != 0;  // the level converged in an earlier range
  int ncorr_last = b.status[2];
  unsigned gen = 0;                       // barriers passed
  bool timed_out = false;
  __syncthreads();

  for (int l = rg.first; l >= rg.last && !timed_out; --l) {
    Lvl lv;
    lv.s = 1 << l;
    lv.level = l;
    lv.W = p.W >> l;
    lv.H = p.H >> l;
    lv.fx = p.fx / lv.s;
    lv.fy = p.fy / lv.s;
    lv.cx = p.cx / lv.s;
    lv.cy = p.cy / lv.s;
    const int npx = lv.W * lv.H;
    const int nchunk = (npx + 31) >> 5;
    const int ngroup = (nchunk + L - 1) / L;
    const int gbase = blockIdx.x * reps + rep, gstride = nblk * reps;
    for (int it = 0; it < rg.iters[l]; ++it) {
      const bool last = rg.close && l == rg.last && it == rg.iters[l] - 1;
      if (it == 0) conv = false;
      if (!(skip || (kStop && conv))) {
        float acc[kNT];
#pragma unroll
        for (int q = 0; q < kNT; ++q) acc[q] = 0.f;
        int cnt = 0;
        const int nloop = gbase < ngroup ? (ngroup - gbase + gstride - 1) / gstride : 0;
        icp_pixels(p, b, lv, S, recs, L, ln, lid, rep, gbase, gstride, nloop, acc, cnt);
        float* part = b.partial + (gen & 1u) * pbuf;
        int* part_n = b.partial_n + (gen & 1u) * nblk;
        icp_block_sums(S, acc, cnt, L, reps, ln, rep, warp, lid, part, pst, blockIdx.x, nblk, part_n);
        ++gen;
        if (!grid_barrier(b.grid_bar, gen * (unsigned)nblk, b.status + 5)) {
          timed_out = true;
          break;
        }
        icp_cross_sum(S, part, pst, nblk, part_n, L, warp, lid);
        icp_solve(p, S, L, npx, false, true);
        ncorr_last = S.s_ncorr;
        if (S.s_fail) {
          skip = true;
        } else {
          icp_update(S, L, sTd);
          for (int i = threadIdx.x; i < L * 12; i += blockDim.x) S.sT[i / 12][i % 12] = (float)sTd[i];
        }
        if (kStop) {
          double x2 = 0.0;
#pragma unroll
          for (int k = 0; k < 6; ++k) x2 += S.sx[0][k] * S.sx[0][k];
          conv = !S.s_fail && x2 < (double)p.icp_stop * (double)p.icp_stop;
          if (blockIdx.x == 0 && threadIdx.x == 0 && b.stats) b.stats[kStatIcpIters] += 1;
        }
        __syncthreads();
      }
      if (last) {
        // close the frame: a failed frame falls back to T_{k-1} on every lane and is counted
        if (skip) {
          for (int i = threadIdx.x; i < L * 12; i += blockDim.x) sTd[i] = b.pose_prev[i];
          if (blockIdx.x == 0 && threadIdx.x == 0) b.status[1] += 1;
          ncorr_last = 0;
        }
        skip = false;
        conv = false;
        __syncthreads();
      }
    }
  }
  if (blockIdx.x == 0 && !timed_out) {
    for (int i = threadIdx.x; i < L * 12; i += blockDim.x) b.pose[i] = sTd[i];
    if (threadIdx.x == 0) {
      b.status[0] = skip ? 1 : 0;
      b.status[2] = ncorr_last;
      b.status[3] = conv ? 1 : 0;
    }
  }
  // leave: the last block out resets the barrier counter for the next launch (every block has
  // passed its last barrier when it counts itself out)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.grid_bar + 1, 1u) == (unsigned)nblk - 1) {
      b.grid_bar[0] = 0u;
      b.grid_bar[1] = 0u;
    }
  }
}

static size_t icp_rec_bytes(int reps, int L) { return sizeof(float) * (size_t)reps * L * kRec * 32; }

cudaError_t icp_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_icp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_icp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_icp_run<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_icp_run<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  return e;
}

int icp_reps(int L) {
  int reps = 16 / L;
  if (reps > kMaxReps) reps = kMaxReps;
  return reps < 1 ? 1 : reps;
}

int icp_blocks(int level_pixels, int L) {
  const int reps = icp_reps(L);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // at least 4 chunks of 32 pixels per warp: small levels get fewer blocks (fewer partials to add)
  const int nchunk = (level_pixels + 31) / 32;
  int nblk = (nchunk + 4 * reps - 1) / (4 * reps);
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
  int reps = icp_reps(p.L);
  const int threads = 32 * p.L * reps;
  const cudaError_t e = p.icp_stop > 0.f
                            ? launch_pdl(k_icp<true>, dim3(nblk), dim3(threads), icp_rec_bytes(reps, p.L), s, p, b, lv,
                                         flags, reps)
                            : launch_pdl(k_icp<false>, dim3(nblk), dim3(threads), icp_rec_bytes(reps, p.L), s, p, b, lv,
                                         flags, reps);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// blocks of the cooperative ICP launch: as many as are resident at once (one per SM), at most
// kMaxPartials (the partial buffers' column bound)
int icp_run_blocks(int L) {
  const int reps = icp_reps(L);
  const size_t smem = icp_rec_bytes(reps, L);
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_icp_run<false>, 32 * L * reps, smem) != cudaSuccess)
    per_sm = 1;
  int n = sms * (per_sm < 1 ? 1 : per_sm);
  return n > kMaxPartials ? kMaxPartials : n;
}

cudaError_t launch_icp_run(const Params& p, const Buffers& b, int first, int last, const int* iters, bool close,
                           int nblk, cudaStream_t s) {
  IcpRange rg;
  rg.first = first;
  rg.last = last;
  for (int l = 0; l < 3; ++l) rg.iters[l] = iters[l];
  rg.close = close ? 1 : 0;
  const int reps = icp_reps(p.L);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk);
  cfg.blockDim = dim3(32 * p.L * reps);
  cfg.dynamicSmemBytes = icp_rec_bytes(reps, p.L);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = p.icp_stop > 0.f ? cudaLaunchKernelEx(&cfg, k_icp_run<true>, p, b, rg, reps)
                                         : cudaLaunchKernelEx(&cfg, k_icp_run<false>, p, b, rg, reps);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace xslam
