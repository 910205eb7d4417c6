// Small kernels of the frame step: pose-lane seeding (X-SLAM Sec. 4.1, Eq. lie: T_0* = exp(h i e_j) T_0),
// derivative read-out (Eq. csfd / eq. pvnpxi: dT = Im T* / h, as a left twist), and the reduction of the
// relocalisation loss used by xslam_grad (Sec. 5.2, point-to-plane reading).
#include "internal.cuh"

namespace xslam {

// seed kinds (xslam_seed_kind)
enum : int { kSeedPose0 = 0, kSeedPose = 1, kSeedTrunc = 2, kSeedDepth = 3, kSeedPoseTracked = 4 };

// Tl = Im exp(h i e_idx) T0 = h G_idx T0 (exact to O(h^3)); G_idx the generator of the left twist
// (phi then rho)
__device__ void generator_times(int e, double h, const double* __restrict__ T0, double* __restrict__ Tl) {
  for (int i = 0; i < 12; ++i) Tl[i] = 0.0;
  if (e < 3) {
    // [e] T0: rows of the generator applied to every column of [R | t]
    for (int q = 0; q < 4; ++q) {
      const double c0 = T0[q], c1 = T0[4 + q], c2 = T0[8 + q];
      double r0 = 0, r1 = 0, r2 = 0;  // [w] c = w x c with w the unit vector e
      if (e == 0) { r1 = -c2; r2 = c1; }
      if (e == 1) { r0 = c2; r2 = -c0; }
      if (e == 2) { r0 = -c1; r1 = c0; }
      Tl[q] = h * r0;
      Tl[4 + q] = h * r1;
      Tl[8 + q] = h * r2;
    }
  } else {
    Tl[4 * (e - 3) + 3] = h;
  }
}

// Frame 0: lanes of the pose kinds (POSE0, and the per-frame kinds, whose start and tracked pose are
// T_0 itself at frame 0) get h G_idx T_0; every other lane is zero. Lane 0 untouched.
__device__ __forceinline__ void seed_pose_body(double* pose, int L, const int* kinds, const int* index,
                                               const Params& p) {
  const int l = threadIdx.x;
  if (l < 1 || l >= L) return;
  const int k = kinds[l];
  double* Tl = pose + 12 * l;
  if (k == kSeedPose0 || k == kSeedPose || k == kSeedPoseTracked) {
    generator_times(index[l], p.h[l], pose, Tl);
  } else {
    for (int i = 0; i < 12; ++i) Tl[i] = 0.0;
  }
}

__global__ void k_seed_pose(double* pose, int L, const int* kinds, const int* index, Params p) {
  pdl_enter();
  seed_pose_body(pose, L, kinds, index, p);
}

// Per-frame pose lanes of a tracked frame (X-SLAM Sec. 4.1, Eq. lie promoting frame k's own pose):
// mode bit 0 restarts them (the imaginary parts earlier frames left in the pose, the previous pose and
// T_{k-2} are dropped), bit 1 perturbs ICP's start (kind POSE; also the proposal's start candB), bit 2
// the tracked pose (kind POSE_TRACKED). One thread per lane.
__global__ void k_seed_frame(Params p, double* __restrict__ pose, double* __restrict__ pose_prev,
                             double* __restrict__ pose_pp, double* __restrict__ candB, const int* __restrict__ kinds,
                             const int* __restrict__ index, int mode) {
  pdl_enter();
  const int l = threadIdx.x;
  if (l < 1 || l >= p.L || !((p.fresh >> l) & 1u)) return;
  const int k = kinds[l];
  if (mode & 1) {
    for (int i = 0; i < 12; ++i) {
      pose[12 * l + i] = 0.0;
      pose_prev[12 * l + i] = 0.0;
      if (pose_pp) pose_pp[12 * l + i] = 0.0;
    }
  }
  if ((mode & 2) && k == kSeedPose) {
    generator_times(index[l], p.h[l], pose, pose + 12 * l);
    if (candB) generator_times(index[l], p.h[l], candB, candB + 12 * l);
  }
  if ((mode & 4) && k == kSeedPoseTracked) generator_times(index[l], p.h[l], pose, pose + 12 * l);
}

__device__ __forceinline__ void readout_body(const double* __restrict__ pose, int L, const Params& p,
                                             double* __restrict__ out) {
  const int l = threadIdx.x;
  if (l == 0)
    for (int i = 0; i < 12; ++i) out[i] = pose[i];
  if (l < 1 || l >= L) return;
  const double* T = pose;
  const double* Tl = pose + 12 * l;
  const double inv_h = 1.0 / p.h[l];
  double dT[12];
  for (int i = 0; i < 12; ++i) {
    dT[i] = Tl[i] * inv_h;
    out[12 + 12 * (l - 1) + i] = dT[i];
  }
  // W = dR R^T; omega = vee of its skew part; v = dt - omega x t
  double W[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) W[3 * r + c] = dT[4 * r] * T[4 * c] + dT[4 * r + 1] * T[4 * c + 1] + dT[4 * r + 2] * T[4 * c + 2];
  const double w0 = 0.5 * (W[7] - W[5]), w1 = 0.5 * (W[2] - W[6]), w2 = 0.5 * (W[3] - W[1]);
  const double t0 = T[3], t1 = T[7], t2 = T[11];
  double* tw = out + 12 + 12 * (kMaxLanes - 1) + 6 * (l - 1);
  tw[0] = w0;
  tw[1] = w1;
  tw[2] = w2;
  tw[3] = dT[3] - (w1 * t2 - w2 * t1);
  tw[4] = dT[7] - (w2 * t0 - w0 * t2);
  tw[5] = dT[11] - (w0 * t1 - w1 * t0);
}

__global__ void k_readout(const double* __restrict__ pose, int L, Params p, double* __restrict__ out) {
  pdl_enter();
  readout_body(pose, L, p, out);
}

// one 32-thread block per segment: mode 0 seeds frame 0's pose lanes, mode 1 reads the frame out
__global__ void __launch_bounds__(32) k_lanes_seg(SegTable st, int mode) {
  pdl_enter();
  const TrajDesc& d = st.desc[st.seg[blockIdx.x].traj];
  if (mode == 0) seed_pose_body(d.b.pose, d.p.L, d.kinds, d.index, d.p);
  else readout_body(d.b.pose, d.p.L, d.p, d.b.result);
}

cudaError_t launch_lanes_seg(const SegTable& t, int mode, cudaStream_t s) {
  return launch_pdl(k_lanes_seg, dim3(t.nseg), dim3(32), 0, s, t, mode);
}

// Relocalisation loss E = mean_u r_u^2, r_u = (T V_q(u) - V_g(u)) . N_g(u), model ray cast at T itself
// (so the correspondence of u is u); lanes carry d r / d xi. Accepts the pixels whose query depth and
// model are valid and |T V_q - V_g| <= dist_gate. Per-block FP32 partials, FP64 sum in the last block:
// out[0] = loss, out[1 + j] = d loss / d xi_j (divided by h_j), out[7] = pixel count.
__global__ void __launch_bounds__(256) k_loss(Params p, const float* __restrict__ D, const float* __restrict__ model,
                                              const double* __restrict__ pose, float* __restrict__ partial,
                                              unsigned* __restrict__ ticket, double* __restrict__ out) {
  pdl_enter();
  __shared__ float sT[kMaxLanes][12];
  __shared__ float s_red[8][kMaxLanes + 1];
  __shared__ int s_last;
  const int L = p.L;
  for (int i = threadIdx.x; i < L * 12; i += blockDim.x) sT[i / 12][i % 12] = (float)pose[i];
  __syncthreads();
  float acc[kMaxLanes + 1];
  for (int i = 0; i <= L; ++i) acc[i] = 0.f;  // [0] sum r^2, [1..L-1] sum 2 r r_l, [L] count
  const size_t hw = (size_t)p.W * p.H;
  const float* T = sT[0];
  for (size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x; pix < hw; pix += (size_t)gridDim.x * blockDim.x) {
    const float d = D[pix];
    const float g = model[pix];
    if (!(d > 0.f && g > 0.f)) continue;
    const int u = (int)(pix % p.W), v = (int)(pix / p.W);
    const float V[3] = {d * (u - p.cx) / p.fx, d * (v - p.cy) / p.fy, d};
    float df[3], nn[3];
    for (int r = 0; r < 3; ++r) {
      const float pr = T[4 * r] * V[0] + T[4 * r + 1] * V[1] + T[4 * r + 2] * V[2] + T[4 * r + 3];
      df[r] = pr - model[(1 + r) * hw + pix];
      nn[r] = model[(1 + 3 * L + r) * hw + pix];
    }
    if (!(df[0] * df[0] + df[1] * df[1] + df[2] * df[2] <= p.dist_gate2)) continue;
    const float res = df[0] * nn[0] + df[1] * nn[1] + df[2] * nn[2];
    acc[0] += res * res;
    acc[L] += 1.f;
    for (int l = 1; l < L; ++l) {
      const float* Tl = sT[l];
      float rl = 0.f;
      for (int r = 0; r < 3; ++r) {
        const float pl = Tl[4 * r] * V[0] + Tl[4 * r + 1] * V[1] + Tl[4 * r + 2] * V[2] + Tl[4 * r + 3];
        rl += (pl - model[(1 + 3 * l + r) * hw + pix]) * nn[r] + df[r] * model[(1 + 3 * L + 3 * l + r) * hw + pix];
      }
      acc[l] += 2.f * res * rl;
    }
  }
  const int warp = threadIdx.x >> 5, lid = threadIdx.x & 31;
  for (int i = 0; i <= L; ++i) {
    float x = acc[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lid == 0) s_red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x <= L) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * (kMaxLanes + 1) + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x <= L) {
    double s = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) s += (double)__ldcg(&partial[(size_t)k * (kMaxLanes + 1) + threadIdx.x]);
    s_red[0][threadIdx.x] = 0.f;
    if (threadIdx.x == 0) out[0] = s;
    else if (threadIdx.x == L) out[7] = s;
    else out[threadIdx.x] = s / p.h[threadIdx.x];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double n = out[7];
    for (int i = 0; i < L; ++i) out[i] = n > 0 ? out[i] / n : 0.0;
    *ticket = 0u;
  }
}

cudaError_t launch_seed_pose(const Params& p, const Buffers& b, const int* kinds, const int* index, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_seed_pose, dim3(1), dim3(32), 0, s, b.pose, p.L, kinds, index, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_seed_frame(const Params& p, const Buffers& b, double* pose_pp, double* candB, const int* kinds,
                              const int* index, int mode, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_seed_frame, dim3(1), dim3(32), 0, s, p, b.pose, b.pose_prev, pose_pp, candB, kinds,
                                   index, mode);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_readout(const Params& p, const Buffers& b, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_readout, dim3(1), dim3(32), 0, s, b.pose, p.L, p, b.result);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_loss(const Params& p, const Buffers& b, const float* depth, const float* model, const double* pose,
                        double* out, int nblk, cudaStream_t s) {
  const cudaError_t e = launch_pdl(k_loss, dim3(nblk), dim3(256), 0, s, p, depth, model, pose, b.partial, b.ticket, out);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace xslam
