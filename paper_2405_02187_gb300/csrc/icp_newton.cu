// Newton ICP (X-SLAM Sec. 4.1: "a second-order ICP procedure using Newton's method at each ICP step",
// the Hessian by the second-order complex step, Eq. csfd_hessian), for the real pose.
//
// One launch per iteration. The energy of the iteration is E(xi) = sum_u r_u(exp(xi) T_j)^2 with the
// correspondences' bilinear cells, validity and gates fixed at the real T_j (exactly as the
// Gauss-Newton kernel decides them); r, the projection u_hat and the bilinear model point and normal
// follow xi exactly. Its gradient g and Hessian H come from 21 truncated-bicomplex evaluations per pixel
// (pair j <= k from exp(e1 G_j + e2 G_k) T_j); beside them each pixel adds the point-to-plane
// Gauss-Newton system A = sum J J^T, b = -sum J r (correspondences held fixed). The last block sums all
// in FP64 (Cholesky factors in FP64 too) and steps with the switch of Sec. 5.2: Newton, xi = -H^-1 g,
// when the mean squared residual is at most eta and H is positive definite, else the Gauss-Newton
// step A xi = b (A not positive definite: the frame fails); eta = inf: Newton only, a singular H damped
// as H + mu I, mu = 10^(k-4) trace(H)/6 for the first k = 1..6 that is positive definite (none: the
// frame fails). T_{j+1} = exp(xi) T_j in FP64; the frame failure protocol is the Gauss-Newton kernel's.
#include "hd.cuh"
#include "internal.cuh"
#include "se3.cuh"

namespace xslam {

namespace {

constexpr int kPairs = 21;
constexpr int kOut = 56;  // count, E, g[6], H[21], A[21], b[6]
constexpr int kNThreads = 128;
constexpr float kCellBiasN = 0.015625f;  // 2^-6, the Gauss-Newton kernel's cell tie-break

__device__ __forceinline__ void gen4(int j, double G[4][4]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) G[r][c] = 0.0;
  if (j < 3) {
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    G[b][a] = 1.0;
    G[a][b] = -1.0;
  } else {
    G[j - 3][3] = 1.0;
  }
}

// Cholesky of the symmetric 6x6 M + mu I into L; false if a pivot is not positive
__device__ bool chol6(const double M[6][6], double mu, double L[6][6]) {
  for (int j = 0; j < 6; ++j) {
    double dsum = M[j][j] + mu;
    for (int k = 0; k < j; ++k) dsum -= L[j][k] * L[j][k];
    if (!(dsum > 0.0)) return false;
    L[j][j] = sqrt(dsum);
    for (int i = j + 1; i < 6; ++i) {
      double t = M[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  return true;
}

// x = (L L^T)^-1 rhs
__device__ void chol6_solve(const double L[6][6], const double* rhs, double* x) {
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double t = rhs[i];
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < 6; ++k) t -= L[k][i] * x[k];
    x[i] = t / L[i][i];
  }
}

__device__ __forceinline__ void mul4(const double A[4][4], const double B[4][4], double C[4][4]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[r][k] * B[k][c];
      C[r][c] = s;
    }
}

}  // namespace

__global__ void __launch_bounds__(kNThreads) k_icp_newton(Params p, Buffers b, int level, int flags) {
  pdl_enter();
  __shared__ HD sT[kPairs][12];
  __shared__ float sTr[12], sPi[12];
  __shared__ int sjk[kPairs][2];
  __shared__ float s_acc[kOut - 2][kNThreads];
  __shared__ float s_red[kNThreads / 32][kOut];
  __shared__ double s_sum[kOut];
  __shared__ int s_skip, s_last;
  const int tid = threadIdx.x;
  if (tid == 0) s_skip = b.status[0];
  if (tid < kPairs) {
    int q = tid, j = 0;
    while (q >= 6 - j) {
      q -= 6 - j;
      ++j;
    }
    const int k = j + q;
    sjk[tid][0] = j;
    sjk[tid][1] = k;
    double T[4][4], Gj[4][4], Gk[4][4], GjT[4][4], GkT[4][4], GjGk[4][4], GkGj[4][4], S[4][4], ST[4][4];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) T[r][c] = r < 3 ? b.pose[4 * r + c] : (c == 3 ? 1.0 : 0.0);
    gen4(j, Gj);
    gen4(k, Gk);
    mul4(Gj, T, GjT);
    mul4(Gk, T, GkT);
    mul4(Gj, Gk, GjGk);
    mul4(Gk, Gj, GkGj);
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) S[r][c] = 0.5 * (GjGk[r][c] + GkGj[r][c]);
    mul4(S, T, ST);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 4; ++c) sT[tid][4 * r + c] = {(float)T[r][c], (float)GjT[r][c], (float)GkT[r][c], (float)ST[r][c]};
  }
  if (tid >= 32 && tid < 44) sTr[tid - 32] = (float)b.pose[tid - 32];
  if (tid == 64) {
    const double* P = b.pose_prev;  // T_prev^-1 = [R^T | -R^T t]
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) sPi[4 * r + c] = (float)P[4 * c + r];
      sPi[4 * r + 3] = (float)(-(P[r] * P[3] + P[4 + r] * P[7] + P[8 + r] * P[11]));
    }
  }
  for (int q = 0; q < kOut - 2; ++q) s_acc[q][tid] = 0.f;
  __syncthreads();

  const int W = p.W >> level, H = p.H >> level, s = 1 << level;
  const float fx = p.fx / s, fy = p.fy / s, cx = p.cx / s, cy = p.cy / s;
  const float* D = level == 0 ? b.pyr[0] : (level == 1 ? b.pyr[1] : b.pyr[2]);
  const size_t hw0 = (size_t)p.W * p.H;
  const float* mdep = b.model;
  const float* mV = b.model + hw0;
  const float* mN = b.model + hw0 * (1 + 3 * p.L);
  float cnt = 0.f, E = 0.f;
  const int npx = W * H;
  for (int px = s_skip ? npx : blockIdx.x * blockDim.x + tid; px < npx; px += gridDim.x * blockDim.x) {
    const int u = px % W, v = px / W;
    if (u >= W - 1 || v >= H - 1) continue;
    const float d0 = D[px], dxp = D[px + 1], dyp = D[px + W];
    if (!(d0 > 0.f && dxp > 0.f && dyp > 0.f)) continue;
    const float rx = (u - cx) / fx, ry = (v - cy) / fy, rx1 = (u + 1 - cx) / fx, ry1 = (v + 1 - cy) / fy;
    const float V[3] = {d0 * rx, d0 * ry, d0};
    const float ex[3] = {dxp * rx1 - V[0], dxp * ry - V[1], dxp - V[2]};
    const float ey[3] = {dyp * rx - V[0], dyp * ry1 - V[1], dyp - V[2]};
    const float c3[3] = {ex[1] * ey[2] - ex[2] * ey[1], ex[2] * ey[0] - ex[0] * ey[2], ex[0] * ey[1] - ex[1] * ey[0]};
    const float n2m = c3[0] * c3[0] + c3[1] * c3[1] + c3[2] * c3[2];
    if (!(n2m > 0.f)) continue;
    const float inm = 1.f / sqrtf(n2m);
    float pp[3], pc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) pp[r] = sTr[4 * r] * V[0] + sTr[4 * r + 1] * V[1] + sTr[4 * r + 2] * V[2] + sTr[4 * r + 3];
#pragma unroll
    for (int r = 0; r < 3; ++r) pc[r] = sPi[4 * r] * pp[0] + sPi[4 * r + 1] * pp[1] + sPi[4 * r + 2] * pp[2] + sPi[4 * r + 3];
    if (!(pc[2] > 0.f)) continue;
    const float ux = fx * (pc[0] / pc[2]) + cx, uy = fy * (pc[1] / pc[2]) + cy;
    const float ci = floorf(ux + kCellBiasN), cj = floorf(uy + kCellBiasN);
    if (!(ci >= 0.f && ci <= (float)(W - 2) && cj >= 0.f && cj <= (float)(H - 2))) continue;
    const size_t t00 = (size_t)((int)cj * s) * p.W + (size_t)((int)ci * s);
    const size_t tk[4] = {t00, t00 + s, t00 + (size_t)s * p.W, t00 + (size_t)s * p.W + s};
    const float g00 = mdep[tk[0]], g10 = mdep[tk[1]], g01 = mdep[tk[2]], g11 = mdep[tk[3]];
    if (!(g00 > 0.f && g10 > 0.f && g01 > 0.f && g11 > 0.f)) continue;
    if (!(fabsf(g10 - g00) + fabsf(g01 - g00) + fabsf(g11 - g00) < p.disc_gate)) continue;
    float mv[4][3], mn[4][3];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        mv[t][r] = mV[(size_t)r * hw0 + tk[t]];
        mn[t][r] = mN[(size_t)r * hw0 + tk[t]];
      }
    const float a = ux - ci, bb = uy - cj;
    const float w[4] = {(1.f - a) * (1.f - bb), a * (1.f - bb), (1.f - a) * bb, a * bb};
    float q[3], n[3], d2 = 0.f, nl2 = 0.f, dot = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      q[r] = w[0] * mv[0][r] + w[1] * mv[1][r] + w[2] * mv[2][r] + w[3] * mv[3][r];
      n[r] = w[0] * mn[0][r] + w[1] * mn[1][r] + w[2] * mn[2][r] + w[3] * mn[3][r];
      d2 += (pp[r] - q[r]) * (pp[r] - q[r]);
      nl2 += n[r] * n[r];
    }
    if (!(d2 <= p.dist_gate2)) continue;
#pragma unroll
    for (int r = 0; r < 3; ++r)
      dot += (sTr[4 * r] * c3[0] + sTr[4 * r + 1] * c3[1] + sTr[4 * r + 2] * c3[2]) * inm * n[r];
    if (!(fabsf(dot) >= p.cos_normal_gate * sqrtf(nl2))) continue;
    // ---- accepted: the 21 second-order directions ----
    cnt += 1.f;
    {
      const float r0 = (pp[0] - q[0]) * n[0] + (pp[1] - q[1]) * n[1] + (pp[2] - q[2]) * n[2];
      E += r0 * r0;
      // the point-to-plane Gauss-Newton system of this correspondence
      const float J[6] = {pp[1] * n[2] - pp[2] * n[1], pp[2] * n[0] - pp[0] * n[2], pp[0] * n[1] - pp[1] * n[0],
                          n[0], n[1], n[2]};
      int e = 0;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int k = i; k < 6; ++k) s_acc[27 + e++][tid] += J[i] * J[k];
        s_acc[48 + i][tid] -= J[i] * r0;
      }
    }
    for (int qq = 0; qq < kPairs; ++qq) {
      const HD* T = sT[qq];
      HD P[3], C[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) P[r] = V[0] * T[4 * r] + V[1] * T[4 * r + 1] + V[2] * T[4 * r + 2] + T[4 * r + 3];
#pragma unroll
      for (int r = 0; r < 3; ++r) C[r] = sPi[4 * r] * P[0] + sPi[4 * r + 1] * P[1] + sPi[4 * r + 2] * P[2] + sPi[4 * r + 3];
      const HD iz = inv(C[2]);
      const HD A = (fx * (C[0] * iz)) + (cx - ci), B = (fy * (C[1] * iz)) + (cy - cj);
      const HD oA = hd(1.f) - A, oB = hd(1.f) - B;
      const HD wq[4] = {oA * oB, A * oB, oA * B, A * B};
      HD res = hd(0.f);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const HD qh = mv[0][r] * wq[0] + mv[1][r] * wq[1] + mv[2][r] * wq[2] + mv[3][r] * wq[3];
        const HD nh = mn[0][r] * wq[0] + mn[1][r] * wq[1] + mn[2][r] * wq[2] + mn[3][r] * wq[3];
        res = res + (P[r] - qh) * nh;
      }
      s_acc[6 + qq][tid] += 2.f * (res.a * res.d + res.b * res.c);
      if (sjk[qq][0] == sjk[qq][1]) s_acc[sjk[qq][0]][tid] += 2.f * res.a * res.b;
    }
  }
  // ---- block sums, then the last block ----
  const int lane = tid & 31, warp = tid >> 5;
  float acc[kOut];
  acc[0] = cnt;
  acc[1] = E;
#pragma unroll
  for (int q = 2; q < kOut; ++q) acc[q] = s_acc[q - 2][tid];
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    float x = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_red[warp][q] = x;
  }
  __syncthreads();
  if (tid < kOut) {
    float t = 0.f;
    for (int w = 0; w < kNThreads / 32; ++w) t += s_red[w][tid];
    b.partial[(size_t)tid * gridDim.x + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(b.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = warp; q < kOut; q += kNThreads / 32) {
    double t = 0.0;
    for (int k = lane; k < (int)gridDim.x; k += 32) t += (double)__ldcg(&b.partial[(size_t)q * gridDim.x + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_sum[q] = t;
  }
  __syncthreads();
  if (tid != 0) return;
  int fail = s_skip;
  const double ncorr = s_sum[0];
  if (!fail && ncorr < (double)p.min_corr_frac * npx) fail = 1;
  double x[6] = {0, 0, 0, 0, 0, 0};
  if (!fail) {
    double Hm[6][6], Am[6][6], g[6], bv[6], L[6][6];
    int e = 0;
    for (int i = 0; i < 6; ++i)
      for (int k = i; k < 6; ++k) {
        Hm[i][k] = Hm[k][i] = s_sum[8 + e];
        Am[i][k] = Am[k][i] = s_sum[29 + e];
        ++e;
      }
    for (int i = 0; i < 6; ++i) {
      g[i] = -s_sum[2 + i];  // the Newton right-hand side -g
      bv[i] = s_sum[50 + i];
    }
    if (isinf(p.icp_newton_eta)) {
      const double tr = (Hm[0][0] + Hm[1][1] + Hm[2][2] + Hm[3][3] + Hm[4][4] + Hm[5][5]) / 6.0;
      bool solved = false;
      for (int kk = 0; kk < 7 && !solved; ++kk)
        if (chol6(Hm, kk == 0 ? 0.0 : pow(10.0, kk - 4) * tr, L)) {
          chol6_solve(L, g, x);
          solved = true;
        }
      if (!solved) fail = 1;
    } else if (s_sum[1] <= (double)p.icp_newton_eta * ncorr && chol6(Hm, 0.0, L)) {
      chol6_solve(L, g, x);
    } else if (chol6(Am, 0.0, L)) {
      chol6_solve(L, bv, x);
    } else {
      fail = 1;
    }
  }
  if (!fail) {
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    SeCoef kc;
    se3_coef_lane(x, zero, kc);
    double Ex[12], Tn[12];
    for (int el = 0; el < 12; ++el) Ex[el] = se3_exp_element(x, zero, kc, false, el);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 4; ++c)
        Tn[4 * r + c] = Ex[4 * r] * b.pose[c] + Ex[4 * r + 1] * b.pose[4 + c] + Ex[4 * r + 2] * b.pose[8 + c] +
                        (c == 3 ? Ex[4 * r + 3] : 0.0);
    for (int el = 0; el < 12; ++el) b.pose[el] = Tn[el];
  } else if (!s_skip) {
    b.status[0] = 1;
  }
  if (flags & kIcpLast) {
    const int failed = b.status[0];
    if (failed)
      for (int el = 0; el < 12; ++el) b.pose[el] = b.pose_prev[el];
    b.status[1] += failed;
    b.status[0] = 0;
    b.status[2] = (int)ncorr;
  }
  *b.ticket = 0u;
}

cudaError_t launch_icp_newton(const Params& p, const Buffers& b, int level, int flags, int nblk, cudaStream_t s) {
  return launch_pdl(k_icp_newton, dim3(nblk), dim3(kNThreads), 0, s, p, b, level, flags);
}

int icp_newton_blocks(int level_pixels, int sms) {
  const int n = (level_pixels + kNThreads - 1) / kNThreads;
  return n < 4 * sms ? (n < 1 ? 1 : n) : 4 * sms;
}

}  // namespace xslam
