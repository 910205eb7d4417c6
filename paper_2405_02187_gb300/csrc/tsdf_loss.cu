// The paper's relocalisation loss (X-SLAM Sec. 5.2): the query frame D_q fused into the reference
// volume at the query pose T gives (F_q, W_q) = surface_update(M_r, T, D_q), and
//   E(T) = sum_p (F_r(p) - F_q(p))^2 = sum over the observed voxels the query updates of
//          ((F_r - F_D) / (W_r + 1))^2,
// since F_q = (W_r F_r + F_D) / (W_r + 1) there and F_q = F_r elsewhere. The sum runs over the voxels the
// reference has observed (W_r > 0): an unobserved voxel has no TSDF value to compare, and counting it
// would reward poses that see less of the map. Its gradient and Hessian with respect to a left twist of T come from
// the truncated-bicomplex step (Sec. 3, simplified arithmetic): for each of the 21 pairs j <= k the
// update's arithmetic runs on numbers a + b e1 + c e2 + d e1 e2 from T = exp(e1 G_j + e2 G_k) T_q,
// with the real pose's decisions (which voxels are updated, which are clamped at F_D = 1, the pixel
// cells). A clamped voxel has no derivative.
//
// The voxels are those of the fusion tile list built for the query pose. A 256-thread block takes two
// 8 x 8 x 8 tiles (four voxels per thread) at a time from the list, by work stealing; each thread takes
// the real decisions of its voxels, and the observed, updated, unclamped ones are pushed to a stack in
// shared memory, which the block drains 256 voxels at a time, so that the derivative work runs on full
// warps whatever the mix of clamped and free voxels in a tile. Order 1 computes the 6 tangents only.
// Per-thread sums of E, g and H in registers, then block sums, FP64 cross-block sums in the last block.
#include "bc.cuh"
#include "internal.cuh"

namespace xslam {

namespace {

constexpr int kPairs = 21;
constexpr int kOut = 29;  // count, E, g[6], H[21]
constexpr int kThreads = 256;

}  // namespace

// The truncated-bicomplex pass, factored. Along pair (j, k) every intermediate u of the update is a
// number u + u_j e1 + u_k e2 + u_jk e1 e2 whose e1 part is the same for every pair with that j (the
// first-order tangent along generator j) and whose e2 part is the tangent along k. So a voxel computes
// its real values and its 6 tangents once and, per pair, only the e1 e2 parts. The start poses are
// affine in the voxel centre p: p_c = R^T (p - t) has tangent A_j (p - t) + a_j and mixed part
// A_jk (p - t) + a_jk, with the pose-only constants a_j = -R^T dt_j, a_jk = -R^T dt_jk - dR_j^T dt_k -
// dR_k^T dt_j taken once per launch. The arithmetic is that of the per-pair numbers up to rounding order.
struct TsdfEntry {  // an observed, updated, unclamped voxel waiting for its 21 directions
  float dv[3];      // p - t
  float pc[3];      // R^T (p - t)
  float a, b;       // bilinear fractions of the pixel cell
  float d00, dx, d01, dy;  // taps: D00, D10 - D00, D01, D11 - D01
  float e;          // (F_r - F_D) / (W_r + 1), as the loss sums it
  float s;          // 1 / ((W_r + 1) mu)
};
constexpr int kEntryFloats = 14;
constexpr int kTilesPerRound = 2;               // tiles a block takes from the list at a time
constexpr int kVox = 2 * kTilesPerRound;        // voxels per thread per round (a tile is 2 x kThreads voxels)
constexpr int kStack = kThreads * (1 + kVox);  // entries pending: < kThreads after a drain, + kVox kThreads
constexpr size_t kTsdfSmem = sizeof(float) * kEntryFloats * kStack;

__global__ void __launch_bounds__(kThreads, 2) k_tsdf_hess(Params p, const float* __restrict__ D,
                                                          const float* __restrict__ F, const float* __restrict__ Wt,
                                                          const float* __restrict__ poses, int order,
                                                          const int* __restrict__ tiles, unsigned* __restrict__ ctr,
                                                          float* __restrict__ partial, unsigned* __restrict__ ticket,
                                                          double* __restrict__ out) {
  pdl_enter();
  extern __shared__ float s_stack[];  // [kEntryFloats][kStack], field-major
  __shared__ float sAt[6][12];        // tangent of p_c along generator j: 9 matrix entries [3c + r], 3 constants
  __shared__ float sAm[kPairs][12];   // mixed part of p_c for pair q: same layout
  __shared__ float s_red[kThreads / 32][kOut];
  __shared__ unsigned s_cnt, s_tile;
  __shared__ int s_last;
  const int tid = threadIdx.x;
  // pose tables from the 21 start poses [pair][element][a, e1, e2, e1 e2]
  auto P = [&](int q, int e, int part) { return poses[4 * (12 * q + e) + part]; };
  if (tid < 6 * 12) {  // tangents from the diagonal pairs' e1 parts
    const int j = tid / 12, f = tid % 12;
    const int qd = j * 6 - j * (j - 1) / 2;  // pair (j, j)
    if (f < 9) {
      sAt[j][f] = P(qd, 4 * (f % 3) + f / 3, 1);
    } else {
      const int c = f - 9;
      float v = 0.f;
      for (int r = 0; r < 3; ++r) v -= P(0, 4 * r + c, 0) * P(qd, 4 * r + 3, 1);
      sAt[j][f] = v;
    }
  }
  for (int i = tid; i < kPairs * 12; i += blockDim.x) {
    const int q = i / 12, f = i % 12;
    if (f < 9) {
      sAm[q][f] = P(q, 4 * (f % 3) + f / 3, 3);
    } else {
      const int c = f - 9;
      float v = 0.f;
      for (int r = 0; r < 3; ++r)
        v -= P(0, 4 * r + c, 0) * P(q, 4 * r + 3, 3) + P(q, 4 * r + c, 1) * P(q, 4 * r + 3, 2) +
             P(q, 4 * r + c, 2) * P(q, 4 * r + 3, 1);
      sAm[q][f] = v;
    }
  }
  if (tid == 0) s_cnt = 0u;
  float T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = P(0, e, 0);
  float acc[kOut];  // count, E, g[6], H[21]
#pragma unroll
  for (int q = 0; q < kOut; ++q) acc[q] = 0.f;
  const unsigned count = ctr[0];
  const int ntx = (p.nx + 7) / 8, nty = (p.ny + 7) / 8;
  const float fx = p.fx, fy = p.fy;

  // the 6 tangents and 21 mixed parts of one pending voxel, added to acc
  auto directions = [&](int m) {
    float dv[3], pc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dv[c] = s_stack[c * kStack + m];
      pc[c] = s_stack[(3 + c) * kStack + m];
    }
    const float a = s_stack[6 * kStack + m], b = s_stack[7 * kStack + m];
    const float d00 = s_stack[8 * kStack + m], dx = s_stack[9 * kStack + m];
    const float d01 = s_stack[10 * kStack + m], dy = s_stack[11 * kStack + m];
    const float e = s_stack[12 * kStack + m], sc = s_stack[13 * kStack + m];
    const float r = 1.f / pc[2], r2 = r * r;
    const float dw = dy - dx;                    // slope of x1 - x0 in a
    const float w = dw * a + (d01 - d00);        // x1 - x0
    // tangents: p_c, 1/z, the cell coordinates A, B, x1 - x0 and the residual e
    float tpc[6][3], tiz[6], tA[6], tB[6], tw[6], te[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        tpc[j][c] = sAt[j][9 + c] + sAt[j][3 * c] * dv[0] + sAt[j][3 * c + 1] * dv[1] + sAt[j][3 * c + 2] * dv[2];
      tiz[j] = -r2 * tpc[j][2];
      tA[j] = fx * (tpc[j][0] * r + pc[0] * tiz[j]);
      tB[j] = fy * (tpc[j][1] * r + pc[1] * tiz[j]);
      tw[j] = dw * tA[j];
      const float tL = dx * tA[j] + b * tw[j] + tB[j] * w;
      te[j] = -sc * (tL - tpc[j][2]);
      acc[2 + j] += 2.f * e * te[j];
    }
    if (order == 1) return;
#pragma unroll
    for (int j = 0, q = 0; j < 6; ++j) {
#pragma unroll
      for (int k = j; k < 6; ++k, ++q) {
        const float* Am = sAm[q];
        float mpc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) mpc[c] = Am[9 + c] + Am[3 * c] * dv[0] + Am[3 * c + 1] * dv[1] + Am[3 * c + 2] * dv[2];
        const float miz = -r2 * mpc[2] + 2.f * r2 * r * tpc[j][2] * tpc[k][2];
        const float mA = fx * (pc[0] * miz + mpc[0] * r + tpc[j][0] * tiz[k] + tpc[k][0] * tiz[j]);
        const float mB = fy * (pc[1] * miz + mpc[1] * r + tpc[j][1] * tiz[k] + tpc[k][1] * tiz[j]);
        const float mw = dw * mA;
        const float mL = dx * mA + b * mw + mB * w + tB[j] * tw[k] + tB[k] * tw[j];
        const float me = -sc * (mL - mpc[2]);
        acc[8 + q] += 2.f * (e * me + te[j] * te[k]);
      }
    }
  };

  __syncthreads();
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(ctr + 1, (unsigned)kTilesPerRound);
    __syncthreads();
    const unsigned q0 = s_tile;
    if (q0 < count) {
      // a round takes kTilesPerRound tiles, kVox voxels per thread; every load of a voxel is issued
      // before any decision that needs it, for all kVox voxels at once
      int tt[kTilesPerRound];
#pragma unroll
      for (int r = 0; r < kTilesPerRound; ++r) tt[r] = q0 + r < count ? tiles[q0 + r] : -1;
      float dv[kVox][3], pc[kVox][3], fa[kVox], fb[kVox];
      int cell[kVox];  // j0 W + i0, or -1: behind the camera, outside the image or the volume
#pragma unroll
      for (int u = 0; u < kVox; ++u) {
        const int t = tt[u >> 1], lv = tid + (u & 1) * kThreads;
        const int i = (t % ntx) * 8 + (lv & 7), j = ((t / ntx) % nty) * 8 + ((lv >> 3) & 7),
                  k = (t / (ntx * nty)) * 8 + (lv >> 6);
        cell[u] = -1;
        fa[u] = fb[u] = 0.f;
        // ---- the surface update's decisions at the real pose (the fusion kernel's arithmetic) ----
        const float px = p.ox + (i + 0.5f) * p.voxel, py = p.oy + (j + 0.5f) * p.voxel,
                    pz = p.oz + (k + 0.5f) * p.voxel;
        dv[u][0] = px - T0[3];
        dv[u][1] = py - T0[7];
        dv[u][2] = pz - T0[11];
#pragma unroll
        for (int c = 0; c < 3; ++c) pc[u][c] = T0[c] * dv[u][0] + T0[4 + c] * dv[u][1] + T0[8 + c] * dv[u][2];
        if (t >= 0 && i < p.nx && j < p.ny && k < p.nz && pc[u][2] > 0.f) {
          const float invz = 1.f / pc[u][2];
          const float x = fx * (pc[u][0] * invz) + p.cx, y = fy * (pc[u][1] * invz) + p.cy;
          if (x >= 0.f && x < (float)(p.W - 1) && y >= 0.f && y < (float)(p.H - 1)) {
            const int i0 = (int)x, j0 = (int)y;
            fa[u] = x - i0;
            fb[u] = y - j0;
            cell[u] = j0 * p.W + i0;
          }
        }
      }
      float tap[kVox][4], wv[kVox], fv[kVox];
#pragma unroll
      for (int u = 0; u < kVox; ++u) {
        tap[u][0] = tap[u][1] = tap[u][2] = tap[u][3] = 0.f;
        wv[u] = fv[u] = 0.f;
        if (cell[u] >= 0) {
          const float* row0 = D + cell[u];
          tap[u][0] = __ldg(row0);
          tap[u][1] = __ldg(row0 + 1);
          tap[u][2] = __ldg(row0 + p.W);
          tap[u][3] = __ldg(row0 + p.W + 1);
          const size_t v = ((size_t)tt[u >> 1] << 9) + tid + (u & 1) * kThreads;
          wv[u] = Wt[v];
          fv[u] = F[v];
        }
      }
#pragma unroll
      for (int u = 0; u < kVox; ++u) {
        const float d00 = tap[u][0], d10 = tap[u][1], d01 = tap[u][2], d11 = tap[u][3];
        const float a = fa[u], bb = fb[u];
        bool push = false;
        float e = 0.f, sc = 0.f;
        if (cell[u] >= 0 && d00 > 0.f && d10 > 0.f && d01 > 0.f && d11 > 0.f &&
            fabsf(d10 - d00) + fabsf(d01 - d00) + fabsf(d11 - d00) < p.disc_gate) {
          const float L = (1.f - a) * (1.f - bb) * d00 + a * (1.f - bb) * d10 + (1.f - a) * bb * d01 + a * bb * d11;
          const float sdf = L - pc[u][2];
          const float w = wv[u];
          if (!(sdf < -p.mu) && w > 0.f) {  // updated, and observed by the reference
            const bool clamp = sdf >= p.mu;
            const float iw = 1.f / (w + 1.f);
            e = (fv[u] - (clamp ? 1.f : sdf / p.mu)) * iw;  // F_D rounded as the surface update rounds it
            acc[0] += 1.f;
            acc[1] += e * e;
            push = !clamp;
            sc = iw / p.mu;
          }
        }
        // warp-aggregated append to the pending stack
        const unsigned bal = __ballot_sync(0xffffffffu, push);
        unsigned base = 0;
        if ((tid & 31) == 0 && bal) base = atomicAdd(&s_cnt, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (push) {
          const unsigned m = base + __popc(bal & ((1u << (tid & 31)) - 1u));
          const float vals[kEntryFloats] = {dv[u][0], dv[u][1], dv[u][2], pc[u][0], pc[u][1], pc[u][2], a, bb,
                                            d00, d10 - d00, d01, d11 - d01, e, sc};
#pragma unroll
          for (int f = 0; f < kEntryFloats; ++f) s_stack[f * kStack + m] = vals[f];
        }
      }
    }
    __syncthreads();
    // drain full rounds from the top of the stack; after the last tiles, drain the rest (a later grab
    // returns at least q0 + kTilesPerRound)
    const bool last = q0 + kTilesPerRound >= count;
    unsigned n = s_cnt;
    while (n >= (unsigned)kThreads || (last && n > 0u)) {
      const unsigned take = n >= (unsigned)kThreads ? (unsigned)kThreads : n;
      if ((unsigned)tid < take) directions((int)(n - take + tid));
      n -= take;
      __syncthreads();
    }
    if (tid == 0) s_cnt = n;
    if (last) break;
    // s_cnt is read again only after the next round's first barrier
  }

  // block sums
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    float xs = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
    if (lane == 0) s_red[warp][q] = xs;
  }
  __syncthreads();
  if (tid < kOut) {
    float sum = 0.f;
    for (int wv = 0; wv < kThreads / 32; ++wv) sum += s_red[wv][tid];
    partial[(size_t)tid * gridDim.x + blockIdx.x] = sum;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_sum[kOut];
  for (int q = warp; q < kOut; q += kThreads / 32) {
    double sum = 0.0;
    for (int kk = lane; kk < (int)gridDim.x; kk += 32) sum += (double)__ldcg(&partial[(size_t)q * gridDim.x + kk]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) s_sum[q] = sum;
  }
  __syncthreads();
  if (tid == 0) {
    out[0] = s_sum[1];
    for (int q = 0; q < 6; ++q) out[1 + q] = s_sum[2 + q];
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_sum[8 + q];
    out[28] = s_sum[0];
    *ticket = 0u;
    ctr[0] = 0u;  // the tile list is consumed: ready for the next fusion or loss
    ctr[1] = 0u;
  }
}

// ---- the plain FP64 path: Sec. 3's bicomplex step as printed ----
// Numbers a + b i1 + c i2 + d i1 i2 with i1^2 = i2^2 = -1 (i1 i2 = i2 i1), every product kept, in FP64,
// with the step h folded into the start poses (b, c scaled by h, d by h^2): g = Im_1 E / h and
// H = Im_12 E / h^2. The update's decisions are taken in FP64 too. This is the comparison path of the
// truncated FP32 kernel above: same loss, same voxels, the paper's arithmetic.
__global__ void __launch_bounds__(kThreads) k_tsdf_hess64(Params p, const float* __restrict__ D,
                                                         const float* __restrict__ F, const float* __restrict__ Wt,
                                                         const double* __restrict__ poses, double inv_h,
                                                         const int* __restrict__ tiles, unsigned* __restrict__ ctr,
                                                         double* __restrict__ partial, unsigned* __restrict__ ticket,
                                                         double* __restrict__ out) {
  pdl_enter();
  constexpr int kJ[kPairs] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
  constexpr int kK[kPairs] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};
  __shared__ BC sT[kPairs][12];
  __shared__ double s_red[kThreads / 32][kOut];
  __shared__ int s_last;
  for (int i = threadIdx.x; i < kPairs * 12; i += blockDim.x) {
    const double* q = poses + 4 * i;
    sT[i / 12][i % 12] = {q[0], q[1], q[2], q[3]};
  }
  __syncthreads();
  double T0[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) T0[e] = sT[0][e].a;
  double acc[kOut];
#pragma unroll
  for (int q = 0; q < kOut; ++q) acc[q] = 0.0;
  const unsigned count = ctr[0];
  const int ntx = (p.nx + 7) / 8, nty = (p.ny + 7) / 8;
  const double mu = p.mu, vox = p.voxel, fx = p.fx, fy = p.fy, cx = p.cx, cy = p.cy;
  for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
    const int t = tiles[q];
    for (int half = 0; half < 2; ++half) {
      const int lv = threadIdx.x + half * kThreads;
      const int i = (t % ntx) * 8 + (lv & 7), j = ((t / ntx) % nty) * 8 + ((lv >> 3) & 7),
                k = (t / (ntx * nty)) * 8 + (lv >> 6);
      if (i >= p.nx || j >= p.ny || k >= p.nz) continue;
      const double px = p.ox + (i + 0.5) * vox, py = p.oy + (j + 0.5) * vox, pz = p.oz + (k + 0.5) * vox;
      const double dx = px - T0[3], dy = py - T0[7], dz = pz - T0[11];
      const double pcx = T0[0] * dx + T0[4] * dy + T0[8] * dz;
      const double pcy = T0[1] * dx + T0[5] * dy + T0[9] * dz;
      const double pcz = T0[2] * dx + T0[6] * dy + T0[10] * dz;
      if (!(pcz > 0.0)) continue;
      const double x = fx * (pcx / pcz) + cx, y = fy * (pcy / pcz) + cy;
      if (!(x >= 0.0 && x < (double)(p.W - 1) && y >= 0.0 && y < (double)(p.H - 1))) continue;
      const int i0 = (int)x, j0 = (int)y;
      const double a = x - i0, bb = y - j0;
      const float* row0 = D + (size_t)j0 * p.W + i0;
      const double d00 = __ldg(row0), d10 = __ldg(row0 + 1), d01 = __ldg(row0 + p.W), d11 = __ldg(row0 + p.W + 1);
      if (!(d00 > 0.0 && d10 > 0.0 && d01 > 0.0 && d11 > 0.0)) continue;
      if (!(fabs(d10 - d00) + fabs(d01 - d00) + fabs(d11 - d00) < (double)p.disc_gate)) continue;
      const double L = (1.0 - a) * (1.0 - bb) * d00 + a * (1.0 - bb) * d10 + (1.0 - a) * bb * d01 + a * bb * d11;
      const double sdf = L - pcz;
      if (sdf < -mu) continue;
      const bool clamp = sdf >= mu;
      const size_t v = ((size_t)t << 9) + lv;
      const double w = Wt[v];
      if (!(w > 0.0)) continue;
      const double Fr = F[v];
      const double iw = 1.0 / (w + 1.0);
      const double e = (Fr - (clamp ? 1.0 : sdf / mu)) * iw;
      acc[0] += 1.0;
      acc[1] += e * e;
      if (clamp) continue;
#pragma unroll
      for (int qq = 0; qq < kPairs; ++qq) {
        const BC* T = sT[qq];
        const BC dv[3] = {bc(px) - T[3], bc(py) - T[7], bc(pz) - T[11]};
        BC pc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) pc[c] = T[c] * dv[0] + T[4 + c] * dv[1] + T[8 + c] * dv[2];
        const BC iz = binv(pc[2]);
        const BC A = fx * (pc[0] * iz) + (cx - (double)i0);
        const BC B = fy * (pc[1] * iz) + (cy - (double)j0);
        const BC x0 = (d10 - d00) * A + d00, x1 = (d11 - d01) * A + d01;
        const BC Lh = x0 + B * (x1 - x0);
        const BC eh = iw * (bc(Fr) - (1.0 / mu) * (Lh - pc[2]));
        const BC e2 = eh * eh;
        acc[8 + qq] += e2.d;
        if (kJ[qq] == kK[qq]) acc[2 + kJ[qq]] += e2.b;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kOut; ++q) {
    double xs = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
    if (lane == 0) s_red[warp][q] = xs;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int wv = 0; wv < kThreads / 32; ++wv) s += s_red[wv][threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_sum[kOut];
  for (int q = warp; q < kOut; q += kThreads / 32) {
    double s = 0.0;
    for (int kk = lane; kk < (int)gridDim.x; kk += 32) s += __ldcg(&partial[(size_t)q * gridDim.x + kk]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) s_sum[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = s_sum[1];
    for (int q = 0; q < 6; ++q) out[1 + q] = s_sum[2 + q] * inv_h;
    for (int q = 0; q < kPairs; ++q) out[7 + q] = s_sum[8 + q] * inv_h * inv_h;
    out[28] = s_sum[0];
    *ticket = 0u;
    ctr[0] = 0u;
    ctr[1] = 0u;
  }
}

cudaError_t launch_tsdf_hess64(const Params& p, const Buffers& b, const float* depth, const double* pose,
                               const double* poses, double h, double* out, int nblk, cudaStream_t s) {
  cudaError_t e = launch_fuse_tiles(p, b, pose, s);
  if (e != cudaSuccess) return e;
  // the float partial buffer holds (blocks + 4) x 27 x 16 floats: room for 29 doubles per block
  return launch_pdl(k_tsdf_hess64, dim3(nblk), dim3(kThreads), 0, s, p, depth, (const float*)b.F, (const float*)b.Wt,
                    poses, 1.0 / h, (const int*)b.tiles, b.tile_ctr, reinterpret_cast<double*>(b.partial), b.ticket,
                    out);
}

cudaError_t launch_tsdf_hess(const Params& p, const Buffers& b, const float* depth, const double* pose,
                             const float* poses, int order, double* out, int nblk, cudaStream_t s) {
  cudaError_t e = launch_fuse_tiles(p, b, pose, s);
  if (e != cudaSuccess) return e;
  // per device, so set on every call (a host-side attribute write)
  e = cudaFuncSetAttribute(k_tsdf_hess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTsdfSmem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_tsdf_hess, dim3(nblk), dim3(kThreads), kTsdfSmem, s, p, depth, (const float*)b.F,
                    (const float*)b.Wt, poses, order, (const int*)b.tiles, b.tile_ctr, b.partial, b.ticket, out);
}

}  // namespace xslam
