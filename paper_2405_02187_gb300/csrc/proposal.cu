// ICP start poses and the judge of the learned proposal.
//
// X-SLAM starts the ICP of frame k at the previous pose T_{k-1} (Sec. 4.1). Two other starts are
// built here, both carried on every CSFD lane (dual-number products: a lane's part of a product is
// the lane part of one factor times the real parts of the others):
//   constant velocity  T_1 T_2^-1 T_1, with T_1 = T_{k-1}, T_2 = T_{k-2} (T_2 = T_0 at k = 1);
//   learned proposal   T_1 exp(xi), xi = scale * y the network's output (real: no lanes).
// With a proposal, two ICP runs go from the coarsest level down to the judge level: run A from the
// constant-velocity (or previous) pose, run B from the proposal. The judge J of each run's pose is
// the mean over the level's pixels with a depth of min(r_u^2, g^2), r_u the point-to-plane residual
// against the model point at the nearest pixel of the projection into the model's camera (g^2 for a
// pixel without one, or farther than the distance gate g). Run B is kept if it did not fail and
// J_B <= J_A, else run A; the kept run goes on to the finer levels.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace xslam {

namespace {

struct Scale6 {
  float v[6];
};

// ---------------------------------------------------------------------------------------------------
// features: one thread per 80 x 60 block (mean of in-range depths / 4 m, 0 if none), frame = blockIdx.y
// ---------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_features(const float* __restrict__ D, int W, int H, float dmin, float dmax,
                                                  __nv_bfloat16* __restrict__ out, size_t out_stride,
                                                  __nv_bfloat16* __restrict__ prev) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kFeat) return;
  const int f = blockIdx.y;
  const int by = H / kFeatH, bx = W / kFeatW;
  const int i0 = (j / kFeatW) * by, c0 = (j % kFeatW) * bx;
  const float* Df = D + (size_t)f * W * H;
  float s = 0.f;
  int n = 0;
  for (int y = i0; y < i0 + by; ++y) {
    const float* row = Df + (size_t)y * W + c0;
    for (int x = 0; x < bx; ++x) {
      const float d = row[x];
      if (d >= dmin && d <= dmax) {
        s += d;
        ++n;
      }
    }
  }
  const __nv_bfloat16 q = __float2bfloat16(n ? s / (float)n * 0.25f : 0.f);
  __nv_bfloat16* o = out + (size_t)f * out_stride;
  if (prev) {
    o[j] = prev[j];
    o[kFeat + j] = q;
    prev[j] = q;
  } else {
    o[j] = q;
  }
}

// ---------------------------------------------------------------------------------------------------
// start poses (one thread per lane, FP64)
// ---------------------------------------------------------------------------------------------------
struct Rig {
  double R[9], t[3];
};

__device__ Rig load_rig(const double* T) {
  Rig r;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) r.R[3 * i + j] = T[4 * i + j];
    r.t[i] = T[4 * i + 3];
  }
  return r;
}

__device__ void store_rig(const Rig& r, double* T) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T[4 * i + j] = r.R[3 * i + j];
    T[4 * i + 3] = r.t[i];
  }
}

// real part of a b
__device__ Rig mul0(const Rig& a, const Rig& b) {
  Rig c;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      c.R[3 * i + j] = a.R[3 * i] * b.R[j] + a.R[3 * i + 1] * b.R[3 + j] + a.R[3 * i + 2] * b.R[6 + j];
    c.t[i] = a.R[3 * i] * b.t[0] + a.R[3 * i + 1] * b.t[1] + a.R[3 * i + 2] * b.t[2] + a.t[i];
  }
  return c;
}

// lane part of a b: a_l b_0 + a_0 b_l (the translation of a_l enters once)
__device__ Rig mul_l(const Rig& a0, const Rig& al, const Rig& b0, const Rig& bl) {
  Rig c = mul0(al, b0);  // includes al.t
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      c.R[3 * i + j] += a0.R[3 * i] * bl.R[j] + a0.R[3 * i + 1] * bl.R[3 + j] + a0.R[3 * i + 2] * bl.R[6 + j];
    c.t[i] += a0.R[3 * i] * bl.t[0] + a0.R[3 * i + 1] * bl.t[1] + a0.R[3 * i + 2] * bl.t[2];
  }
  return c;
}

// inverse [R^T | -R^T t] (plain transpose): real part and lane part
__device__ Rig inv0(const Rig& a) {
  Rig c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.R[3 * i + j] = a.R[3 * j + i];
  for (int i = 0; i < 3; ++i) c.t[i] = -(c.R[3 * i] * a.t[0] + c.R[3 * i + 1] * a.t[1] + c.R[3 * i + 2] * a.t[2]);
  return c;
}

// 3x3 products of row-major blocks: c = a b, c = a^T b, c = a b^T
__device__ void mm3(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
__device__ void mtm3(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c[3 * i + j] = a[i] * b[j] + a[3 + i] * b[3 + j] + a[6 + i] * b[6 + j];
}

// One Newton step of the polar decomposition, P(R) = 1.5 R - 0.5 R R^T R, on the rotation block: it
// takes R to the nearest rotation up to the square of its deviation from one. The constant-velocity
// start T_1 T_2^-1 T_1 otherwise amplifies the rotation's deviation (from the FP32 ICP increments)
// about 2.4 times per frame. Real part and lane part (the derivative of P: a valid tangent R_l, with
// R_0^T R_l skew, is kept as it is).
__device__ void polar0(const Rig& a0, Rig& out) {
  double G[9], RG[9];
  mtm3(a0.R, a0.R, G);  // R^T R
  mm3(a0.R, G, RG);
  for (int k = 0; k < 9; ++k) out.R[k] = 1.5 * a0.R[k] - 0.5 * RG[k];
}

__device__ void polar_l(const Rig& a0, const Rig& al, Rig& out) {
  double G[9], Gl[9], H[9], t1[9], t2[9], t3[9];
  mtm3(a0.R, a0.R, G);   // R0^T R0
  mtm3(al.R, a0.R, Gl);  // Rl^T R0
  mtm3(a0.R, al.R, H);   // R0^T Rl
  mm3(al.R, G, t1);      // Rl R0^T R0
  mm3(a0.R, Gl, t2);     // R0 Rl^T R0
  mm3(a0.R, H, t3);      // R0 R0^T Rl
  for (int k = 0; k < 9; ++k) out.R[k] = 1.5 * al.R[k] - 0.5 * (t1[k] + t2[k] + t3[k]);
}

__device__ Rig inv_l(const Rig& a0, const Rig& al) {
  Rig c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.R[3 * i + j] = al.R[3 * j + i];
  for (int i = 0; i < 3; ++i)
    c.t[i] = -(al.R[i] * a0.t[0] + al.R[3 + i] * a0.t[1] + al.R[6 + i] * a0.t[2]) -
             (a0.R[i] * al.t[0] + a0.R[3 + i] * al.t[1] + a0.R[6 + i] * al.t[2]);
  return c;
}

// exp of a twist (phi, rho): R = I + a W + b W^2, t = (I + b W + c W^2) rho, W = [phi]x
__device__ Rig se3_exp_d(const double* xi) {
  const double p0 = xi[0], p1 = xi[1], p2 = xi[2];
  const double th2 = p0 * p0 + p1 * p1 + p2 * p2, th = sqrt(th2);
  double a, b, c;
  if (th < 1e-4) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
    c = 1.0 / 6.0 - th2 / 120.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
    c = (th - sin(th)) / (th2 * th);
  }
  const double Wm[9] = {0.0, -p2, p1, p2, 0.0, -p0, -p1, p0, 0.0};
  double W2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W2[3 * i + j] = Wm[3 * i] * Wm[j] + Wm[3 * i + 1] * Wm[3 + j] + Wm[3 * i + 2] * Wm[6 + j];
  Rig r;
  double V[9];
  for (int k = 0; k < 9; ++k) {
    const double I = (k % 4 == 0) ? 1.0 : 0.0;
    r.R[k] = I + a * Wm[k] + b * W2[k];
    V[k] = I + b * Wm[k] + c * W2[k];
  }
  for (int i = 0; i < 3; ++i) r.t[i] = V[3 * i] * xi[3] + V[3 * i + 1] * xi[4] + V[3 * i + 2] * xi[5];
  return r;
}

__global__ void __launch_bounds__(32) k_prop_seed(Params p, Buffers b, PropBuffers q, Scale6 sc, int mode) {
  pdl_enter();
  const int l = threadIdx.x;
  const bool act = l < p.L;
  const int lr = act ? l : 0;
  // every lane reads T_{k-1} before any lane writes the new start (one warp)
  const Rig T10 = load_rig(b.pose), T1l = load_rig(b.pose + 12 * lr);
  const Rig T20 = load_rig(q.pose_pp), T2l = load_rig(q.pose_pp + 12 * lr);
  Rig A = lr == 0 ? T10 : T1l;
  if (mode & 1) {
    const Rig I0 = inv0(T20);
    const Rig M0 = mul0(I0, T10);  // T_2^-1 T_1
    const Rig A0 = mul0(T10, M0);
    if (lr == 0) {
      polar0(A0, A);
      A.t[0] = A0.t[0], A.t[1] = A0.t[1], A.t[2] = A0.t[2];
    } else {
      const Rig Ml = mul_l(I0, inv_l(T20, T2l), T10, T1l);
      const Rig Al = mul_l(T10, T1l, M0, Ml);
      polar_l(A0, Al, A);
      A.t[0] = Al.t[0], A.t[1] = Al.t[1], A.t[2] = Al.t[2];
    }
  }
  Rig B = A;
  if (mode & 2) {
    double xi[6];
    for (int k = 0; k < 6; ++k) xi[k] = (double)(sc.v[k] * q.y[k]);
    // T_1 exp(xi); exp(xi) is real, so a lane's part is T1_l exp(xi) (its translation enters once)
    B = mul0(lr == 0 ? T10 : T1l, se3_exp_d(xi));
  }
  __syncwarp();
  if (!act) return;
  store_rig(lr == 0 ? T10 : T1l, q.pose_pp + 12 * l);
  if (mode & 4) return;  // frame 0: T_{k-2} of frame 1 is T_0
  store_rig(A, b.pose + 12 * l);
  if (mode & 2) store_rig(B, q.candB + 12 * l);
}

// ---------------------------------------------------------------------------------------------------
// judge (grid-stride over the level's pixels; last block reduces in block order)
// ---------------------------------------------------------------------------------------------------
struct JLvl {
  int W, H, s;
  float fx, fy, cx, cy;
};

__global__ void __launch_bounds__(256) k_prop_judge(Params p, Buffers b, PropBuffers q, JLvl lv, int phase, int final_) {
  pdl_enter();
  __shared__ float sT[12], sP[12];
  __shared__ double s_red[8][2];
  __shared__ int s_last;
  if (threadIdx.x < 12) {
    sT[threadIdx.x] = (float)b.pose[threadIdx.x];
    sP[threadIdx.x] = (float)b.pose_prev[threadIdx.x];
  }
  __syncthreads();
  const float g2 = p.dist_gate2;
  const float* D = lv.s == 1 ? b.pyr[0] : (lv.s == 2 ? b.pyr[1] : b.pyr[2]);
  const size_t hw0 = (size_t)p.W * p.H;
  const float* mdep = b.model;
  const float* mV = b.model + hw0;
  const float* mN = b.model + hw0 * (1 + 3 * p.L);
  float acc = 0.f, cnt = 0.f;
  const int npx = lv.W * lv.H;
  for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < npx; px += gridDim.x * blockDim.x) {
    const float d = D[px];
    if (!(d > 0.f)) continue;
    cnt += 1.f;
    const int u = px % lv.W, v = px / lv.W;
    const float V[3] = {d * ((u - lv.cx) / lv.fx), d * ((v - lv.cy) / lv.fy), d};
    float pp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) pp[r] = sT[4 * r] * V[0] + sT[4 * r + 1] * V[1] + sT[4 * r + 2] * V[2] + sT[4 * r + 3];
    const float e0 = pp[0] - sP[3], e1 = pp[1] - sP[7], e2 = pp[2] - sP[11];
    const float pcx = sP[0] * e0 + sP[4] * e1 + sP[8] * e2;
    const float pcy = sP[1] * e0 + sP[5] * e1 + sP[9] * e2;
    const float pcz = sP[2] * e0 + sP[6] * e1 + sP[10] * e2;
    float c = g2;
    if (pcz > 0.f) {
      const float ui = floorf(lv.fx * (pcx / pcz) + lv.cx + 0.5f), vi = floorf(lv.fy * (pcy / pcz) + lv.cy + 0.5f);
      if (ui >= 0.f && ui <= (float)(lv.W - 1) && vi >= 0.f && vi <= (float)(lv.H - 1)) {
        const size_t t = (size_t)((int)vi * lv.s) * p.W + (size_t)((int)ui * lv.s);
        if (mdep[t] > 0.f) {
          const float df[3] = {pp[0] - mV[t], pp[1] - mV[hw0 + t], pp[2] - mV[2 * hw0 + t]};
          if (df[0] * df[0] + df[1] * df[1] + df[2] * df[2] <= g2) {
            const float r = df[0] * mN[t] + df[1] * mN[hw0 + t] + df[2] * mN[2 * hw0 + t];
            c = fminf(r * r, g2);
          }
        }
      }
    }
    acc += c;
  }
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  double a = acc, n = cnt;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if (lid == 0) {
    s_red[warp][0] = a;
    s_red[warp][1] = n;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w][threadIdx.x];
    q.partial[2 * blockIdx.x + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(q.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ int s_keep;  // 1: the pose lanes in b.pose stay, 0: run A's lanes come back
  if (threadIdx.x == 0) {
    double tot = 0.0, num = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) {
      tot += __ldcg(&q.partial[2 * k]);
      num += __ldcg(&q.partial[2 * k + 1]);
    }
    *q.ticket = 0u;
    const double J = num > 0.0 ? tot / num : (double)g2;
    if (phase == 0) {
      q.judge[0] = J;
      *q.failA = b.status[0];
      s_keep = 1;
    } else {
      q.judge[1] = J;
      const int failB = b.status[0], failA = *q.failA;
      const int accept = !failB && (failA || J <= q.judge[0]);
      s_keep = accept;
      if (!accept) b.status[0] = failA;
      if (b.stats) {
        b.stats[kStatJudged] += 1;
        b.stats[kStatAccepted] += accept;
      }
    }
  }
  __syncthreads();
  const int n12 = 12 * p.L;
  if (phase == 0) {
    // keep run A, start run B from the proposal
    for (int i = threadIdx.x; i < n12; i += blockDim.x) {
      q.candA[i] = b.pose[i];
      b.pose[i] = q.candB[i];
    }
    if (threadIdx.x == 0) {
      b.status[0] = 0;
      b.status[3] = 0;
    }
    return;
  }
  if (!s_keep)
    for (int i = threadIdx.x; i < n12; i += blockDim.x) b.pose[i] = q.candA[i];
  __syncthreads();
  if (final_) {
    const int failed = b.status[0];
    if (failed)
      for (int i = threadIdx.x; i < n12; i += blockDim.x) b.pose[i] = b.pose_prev[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (failed) {
        b.status[1] += 1;
        b.status[2] = 0;
      }
      b.status[0] = 0;
    }
  }
  if (threadIdx.x == 0) b.status[3] = 0;
}

}  // namespace

cudaError_t launch_features(const float* D, int n, int W, int H, float dmin, float dmax, void* out, size_t out_stride,
                            void* prev, cudaStream_t s) {
  return launch_pdl(k_features, dim3((kFeat + 255) / 256, n), dim3(256), 0, s, D, W, H, dmin, dmax,
                    (__nv_bfloat16*)out, out_stride, (__nv_bfloat16*)prev);
}

cudaError_t launch_prop_seed(const Params& p, const Buffers& b, const PropBuffers& q, const float* scale, int mode,
                             cudaStream_t s) {
  Scale6 sc;
  for (int k = 0; k < 6; ++k) sc.v[k] = scale ? scale[k] : 0.f;
  return launch_pdl(k_prop_seed, dim3(1), dim3(32), 0, s, p, b, q, sc, mode);
}

cudaError_t launch_prop_judge(const Params& p, const Buffers& b, const PropBuffers& q, int level, int phase, int final_,
                              int nblk, cudaStream_t s) {
  JLvl lv;
  lv.s = 1 << level;
  lv.W = p.W >> level;
  lv.H = p.H >> level;
  lv.fx = p.fx / lv.s;
  lv.fy = p.fy / lv.s;
  lv.cx = p.cx / lv.s;
  lv.cy = p.cy / lv.s;
  return launch_pdl(k_prop_judge, dim3(nblk), dim3(256), 0, s, p, b, q, lv, phase, final_);
}

}  // namespace xslam
