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
  int W, H, s;
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

// kStop: the stop tolerance p.icp_stop is in use (and the iteration counter): a launch after its level
// converged returns at once. Without it the kernel is the fixed-count iteration of the method.
template <bool kStop>
__global__ void __launch_bounds__(512, 1) k_icp(Params p, Buffers b, Lvl lv, int flags, int reps) {
  pdl_enter();
  const int L = p.L;
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  const int ln = warp % L, rep = warp / L;
  __shared__ float sT[kMaxLanes][12];
  __shared__ float sP[kMaxLanes][12];
  __shared__ int s_skip, s_last;
  __shared__ float s_red[kNT * kMaxLanes];  // [rep][lane][27]; reps * L <= 16 by construction
  __shared__ int s_cnt[32];
  __shared__ double sA[kMaxLanes * kNT];
  __shared__ double sx[kMaxLanes][6];
  __shared__ Ldl32 s_ldl;
  __shared__ double s_half[2 * kNT * kMaxLanes];
  __shared__ float sAf[kNT * kMaxLanes];
  __shared__ float sxf[kMaxLanes][6], srf[kMaxLanes][6], sdf[kMaxLanes][6];
  __shared__ SeCoefF scf[kMaxLanes];
  __shared__ float sxs[kMaxLanes][6];
  __shared__ float sdl[kMaxLanes][12];
  __shared__ int s_ncorr, s_fail, s_conv;
  extern __shared__ float s_rec[];  // [rep][chunk of the group][field][pixel]: reps * L * kRec * 32 floats

  if (threadIdx.x == 0) {
    s_skip = b.status[0];
    // status[3]: the level converged (a step below p.icp_stop); only its first iteration ignores it
    if (kStop) s_conv = (flags & (kIcpFirst | kIcpNoUpdate)) ? 0 : b.status[3];
  }
  for (int i = threadIdx.x; i < L * 12; i += blockDim.x) {
    sT[i / 12][i % 12] = (float)b.pose[i];
    sP[i / 12][i % 12] = (float)b.pose_prev[i];
  }
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

  // Work unit: a group of L chunks of 32 pixels per replica. Every warp of the replica computes the
  // real part of one chunk of the group (correspondence, residual, Jacobian, bilinear derivatives) into
  // a shared-memory record; after a named barrier every warp reads all L records and adds the sums of
  // its own lane: lane 0 the real normal equations, lane l > 0 their tangent, for which it loads only
  // lane l's model taps. A second barrier frees the records for the next group.
  int nloop = 0, gbase = 0, gstride = 1;
  const int npx = lv.W * lv.H;
  const int nchunk = (npx + 31) >> 5;
  {
    const int ngroup = (nchunk + L - 1) / L;
    gbase = blockIdx.x * reps + rep;
    gstride = gridDim.x * reps;
    nloop = (!s_skip && gbase < ngroup) ? (ngroup - gbase + gstride - 1) / gstride : 0;
  }
  const float* D = lv.s == 1 ? b.pyr[0] : (lv.s == 2 ? b.pyr[1] : b.pyr[2]);
  const size_t hw0 = (size_t)p.W * p.H;
  const float* mdep = b.model;
  const float* mV = b.model + hw0;
  const float* mN = b.model + hw0 * (1 + 3 * L);
  float* recs = s_rec + (size_t)rep * L * kRec * 32;
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
      const float* T = sT[0];
      const float* P = sP[0];
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
        R_[RV * 32] = __int_as_float(ok ? 1 : 0);
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
        const float* T = sT[0];
        const float* P = sP[0];
        const float* Tl = sT[ln];
        const float* Pl = sP[ln];
        const float d0 = R_[RD * 32], rx = R_[RRX * 32], ry = R_[RRY * 32];
        const float V[3] = {d0 * rx, d0 * ry, d0};
        const float dDl = p.dD[ln];
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
          const float* Vpl = mVl + (size_t)r * hw0;
          const float* Npl = mNl + (size_t)r * hw0;
          ql[r] = R_[(RDQA + r) * 32] * al + R_[(RDQB + r) * 32] * bl + w00 * Vpl[t00] + w10 * Vpl[t10] +
                  w01 * Vpl[t01] + w11 * Vpl[t11];
          nl[r] = R_[(RDNA + r) * 32] * al + R_[(RDNB + r) * 32] * bl + w00 * Npl[t00] + w10 * Npl[t10] +
                  w01 * Npl[t01] + w11 * Npl[t11];
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

  // ---------------- block reduction ----------------
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
    for (int q = 0; q < kNT; ++q) s_red[(rep * L + ln) * kNT + q] = acc[q];
    s_cnt[warp] = cnt;
  }
  __syncthreads();
  // partials are stored value-major ([value][block]) so that the last block reads each value's
  // per-block sums with coalesced warp loads
  const int pst = icp_pstride(gridDim.x);
  for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < reps; ++r) s += s_red[r * L * kNT + i];
    b.partial[(size_t)i * pst + blockIdx.x] = s;
    if (blockIdx.x == gridDim.x - 1)  // the row padding of this launch's stride reads as zero
      for (int k = gridDim.x; k < pst; ++k) b.partial[(size_t)i * pst + k] = 0.f;
  }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < reps; ++r) c += s_cnt[r * L];
    b.partial_n[blockIdx.x] = c;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(b.ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---------------- last block: FP64 cross-block sum ----------------
  // value v is summed by two threads, one per half of its row of block partials: all float4 loads of a
  // half (up to 20, i.e. grids of up to 160 blocks) issued together, so the read costs one L2 round
  // trip; FP32 sums of 16 partials, FP64 accumulation of those sums, FP64 add of the two halves.
  // Different values sit in different lanes, so each FP64 warp instruction adds 32 values.
  const int NV = L * kNT;
  const int pstride = icp_pstride(gridDim.x);
  if (warp == (int)(blockDim.x >> 5) - 1) {
    // the last warp adds the per-block correspondence counts: 8 loads per lane in flight at once
    int c = 0;
    for (int k0 = 0; k0 < (int)gridDim.x; k0 += 256) {
      int q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + lid + 32 * j;
        q[j] = k < (int)gridDim.x ? __ldcg(&b.partial_n[k]) : 0;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) c += q[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lid == 0) {
      s_ncorr = c;
      *b.ticket = 0u;  // ready for the next launch
    }
  }
  const int n4 = pstride >> 2, h4 = (n4 + 1) >> 1;
  for (int t = threadIdx.x; t < 2 * NV; t += blockDim.x) {
    const int v = t >> 1, half = t & 1;
    const float4* row = reinterpret_cast<const float4*>(b.partial + (size_t)v * pstride) + half * h4;
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
    s_half[t] = acc;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += blockDim.x) sA[v] = s_half[2 * v] + s_half[2 * v + 1];
  __syncthreads();

  const bool update = !s_skip && !(flags & kIcpNoUpdate);
  if (flags & kIcpNoUpdate) {
    for (int i = threadIdx.x; i < L * kNT; i += blockDim.x) b.result[kResSys + i] = sA[i];
    if (threadIdx.x == 0) b.status[2] = s_ncorr;
    return;
  }
  // factor the real 6x6 A once, then x_0 = A^-1 (-g_0) and x_l = A^-1 (-g_l - A_l x_0)
  const int t = threadIdx.x;
  for (int v = t; v < NV; v += blockDim.x) sAf[v] = (float)sA[v];
  __syncthreads();
  if (t == 0) {
    int fail = s_skip;
    if (!fail && (float)s_ncorr < p.min_corr_frac * (float)(lv.W * lv.H)) fail = 1;
    if (!fail && !ldl32(sAf, s_ldl)) fail = 1;
    if (!fail) {
      float b0[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) b0[i] = -sAf[21 + i];
      subst32(s_ldl, b0, sxf[0]);
    }
    s_fail = fail;
  }
  __syncthreads();
  const bool go = update && !s_fail;
  // real lane: residual in FP64 (thread i = row), FP32 correction
  if (go && t < 6) {
    double r = -sA[21 + t];
#pragma unroll
    for (int k = 0; k < 6; ++k) r = fma(-sA[t <= k ? up6(t, k) : up6(k, t)], (double)sxf[0][k], r);
    srf[0][t] = (float)r;
  }
  __syncthreads();
  if (go && t == 0) subst32(s_ldl, srf[0], sdf[0]);
  __syncthreads();
  if (go && t < 6) sx[0][t] = (double)sxf[0][t] + (double)sdf[0][t];
  __syncthreads();
  // imaginary lanes: right-hand sides in FP64, thread (l, i)
  const int ls = 1 + t / 6, li = t % 6;
  const bool lane_thread = go && t < 6 * (L - 1);
  double rhs = 0.0;
  if (lane_thread) {
    const double* Al = sA + ls * kNT;
    rhs = -Al[21 + li];
#pragma unroll
    for (int k = 0; k < 6; ++k) rhs = fma(-Al[li <= k ? up6(li, k) : up6(k, li)], sx[0][k], rhs);
    srf[ls][li] = (float)rhs;
  }
  __syncthreads();
  if (go && t >= 1 && t < L) subst32(s_ldl, srf[t], sxf[t]);
  __syncthreads();
  if (lane_thread) {
    double r = rhs;
#pragma unroll
    for (int k = 0; k < 6; ++k) r = fma(-sA[li <= k ? up6(li, k) : up6(k, li)], (double)sxf[ls][k], r);
    srf[ls][li] = (float)r;
  }
  __syncthreads();
  if (go && t >= 1 && t < L) subst32(s_ldl, srf[t], sdf[t]);
  __syncthreads();
  if (lane_thread) sx[ls][li] = (double)sxf[ls][li] + (double)sdf[ls][li];
  __syncthreads();

  // pose update T <- exp(x) T on every lane: delta = exp(x) - I in FP32 (coefficients once per lane,
  // then one thread per (lane, element)), T + delta T composed in FP64 one element per thread
  if (go && t < 6 * L) sxs[t / 6][t % 6] = (float)sx[t / 6][t % 6];
  __syncthreads();
  if (go && t < L) se3_coef_lane_f(sxs[0], sxs[t], scf[t]);
  __syncthreads();
  if (go && t < 12 * L) {
    const int l = t / 12, e = t % 12;
    sdl[l][e] = se3_delta_element(sxs[0], sxs[l], scf[l], l > 0, e);
  }
  __syncthreads();
  double tn = 0.0;
  if (go && t < 12 * L) {
    const int l = t / 12, e = t % 12, r = e >> 2, c = e & 3;
    const double* T0 = b.pose;
    const double* Tl = b.pose + 12 * l;
    // lane 0: T0 + d0 T0; lane l: Tl + dl T0 + d0 Tl (translation column adds the delta's own column)
    tn = Tl[e] + (double)sdl[l][4 * r] * T0[c] + (double)sdl[l][4 * r + 1] * T0[4 + c] +
         (double)sdl[l][4 * r + 2] * T0[8 + c] + (c == 3 ? (double)sdl[l][4 * r + 3] : 0.0);
    if (l > 0)
      tn += (double)sdl[0][4 * r] * Tl[c] + (double)sdl[0][4 * r + 1] * Tl[4 + c] + (double)sdl[0][4 * r + 2] * Tl[8 + c];
  }
  __syncthreads();
  if (go && t < 12 * L) b.pose[t] = tn;
  if (kStop) {
    if (threadIdx.x == 0) {
      if (s_fail) b.status[0] = 1;
      b.status[2] = s_ncorr;
      double x2 = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) x2 += sx[0][k] * sx[0][k];
      b.status[3] = (go && x2 < (double)p.icp_stop * (double)p.icp_stop) ? 1 : 0;
      if (b.stats) b.stats[kStatIcpIters] += 1;
    }
  } else if (threadIdx.x == 0 && s_fail && !s_skip) {
    b.status[0] = 1;
  }
  if (flags & kIcpLast) {
    __syncthreads();
    const int failed = b.status[0];
    if (failed && t < 12 * L) b.pose[t] = b.pose_prev[t];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (failed) b.status[1] += 1;
      b.status[0] = 0;
      b.status[2] = s_ncorr;
    }
  }
}

static size_t icp_rec_bytes(int reps, int L) { return sizeof(float) * (size_t)reps * L * kRec * 32; }

cudaError_t icp_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_icp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_icp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
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

}  // namespace xslam
