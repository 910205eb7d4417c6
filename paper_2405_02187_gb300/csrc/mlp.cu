// The learned pose proposal's network (include/xslam_mlp.h): parameters, the forward and backward
// passes as tcgen05 GEMMs (gemm.cu) with split-K reduction epilogues, the loss, Adam, and the
// training loop (one CUDA graph per step, replayed once per batch).
//
// Shapes of one training step with batch B (widths padded to multiples of 64, np[l]):
//   forward  layer l:  Z = a_l W_l^T        GEMM M = B,       N = np[l+1], K = np[l]
//   weights  layer l:  dW_l = dz^T a_l      GEMM M = np[l+1], N = np[l],   K = B   (operands dz^T, a_l^T)
//   inputs   layer l:  da_l = dz W_l        GEMM M = B,       N = np[l],   K = np[l+1] (operand W_l^T)
// Every GEMM writes FP32 partial products of its K ranges; the reduction kernel adds them in a fixed
// order and applies the epilogue (bias and ReLU; or the ReLU mask of the backward pass), writing FP32
// and/or BF16 and the BF16 transpose the next GEMM reads as a K-major operand.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"
#include "mlp.cuh"

using namespace xslam;

namespace {

std::string g_mlp_err;
__device__ int g_gemm_err;  // timeout flag of xslam_gemm_bf16

xslam_status mfail(xslam_mlp_t m, xslam_status st, const std::string& msg) {
  if (m)
    m->msg = msg;
  else
    g_mlp_err = msg;
  return st;
}

#define MCU(x)                                                                                \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return mfail(m, XSLAM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define KCU(x)                         \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)

int pad64(int n) { return (n + 63) / 64 * 64; }

// ---------------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------------

// The element-wise kernels work on 32 x 32 tiles with 32 x 8 threads: a row of a tile is read and
// written with coalesced accesses, and a transposed copy goes through shared memory so that it is
// written coalesced too.

// sum of the split-K partials (in range order), then the epilogue, over the M x N product: one element
// per thread (32 x 32 threads per tile), so that every partial load of the tile is in flight at once
__global__ void __launch_bounds__(1024) k_reduce(const float* __restrict__ P, int splits, int M, int N,
                                                 const float* __restrict__ bias, int relu,
                                                 const __nv_bfloat16* __restrict__ mask, float* __restrict__ out32,
                                                 int ld32, int n32, __nv_bfloat16* __restrict__ out16,
                                                 __nv_bfloat16* __restrict__ out16T) {
  pdl_enter();
  __shared__ __nv_bfloat16 tile[32][34];
  const size_t MN = (size_t)M * N;
  const int c = blockIdx.x * 32 + threadIdx.x;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = blockIdx.y * 32 + k;
    __nv_bfloat16 q = __float2bfloat16(0.f);
    if (r < M && c < N) {
      const size_t i = (size_t)r * N + c;
      float v = 0.f;
      for (int z = 0; z < splits; ++z) v += P[(size_t)z * MN + i];
      if (bias) v += bias[c];
      if (relu) v = fmaxf(v, 0.f);
      if (mask && !(__bfloat162float(mask[i]) > 0.f)) v = 0.f;
      if (out32 && c < n32) out32[(size_t)r * ld32 + c] = v;
      q = __float2bfloat16(v);
      if (out16) out16[i] = q;
    }
    tile[k][threadIdx.x] = q;
  }
  if (!out16T) return;
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int rt = blockIdx.x * 32 + k, ct = blockIdx.y * 32 + threadIdx.x;  // row of the transpose = column
    if (rt < N && ct < M) out16T[(size_t)rt * M + ct] = tile[threadIdx.x][k];
  }
}

// dz_L = (y - t) / B on the first nL columns (0 on the padding), its BF16 copy and transpose, and the
// batch loss sum |y - t|^2 / (2B) added to *loss (atomically: the loss is a report); block 0 advances the
// Adam step and the batch index
__global__ void __launch_bounds__(256) k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, int B,
                                                   int np, int nL, float* __restrict__ dz32,
                                                   __nv_bfloat16* __restrict__ dzq, __nv_bfloat16* __restrict__ dzqT,
                                                   double* loss, int* ctr) {
  pdl_enter();
  __shared__ double s_red[8];
  double acc = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * np) {
    const int r = i / np, c = i % np;
    const float d = c < nL ? y[i] - t[i] : 0.f;
    acc = (double)d * (double)d;
    const float g = d / (float)B;
    dz32[i] = g;
    const __nv_bfloat16 q = __float2bfloat16(g);
    dzq[i] = q;
    dzqT[(size_t)c * B + r] = q;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_red[w];
    atomicAdd(loss, sum / (2.0 * B));
    if (ctr && blockIdx.x == 0) {
      ctr[0] += 1;
      ctr[1] += 1;
    }
  }
}

// db = column sums of dz [B x N] (rows y, y + 8, ... per thread, then the 8 partial sums in order)
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ dz, int B, int N, float* __restrict__ out) {
  pdl_enter();
  __shared__ float part[8][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < N)
    for (int r = threadIdx.y; r < B; r += 8) s += dz[(size_t)r * N + c];
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < N) {
    float t = 0.f;
    for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
    out[c] = t;
  }
}

// training batch: rows [f_i, f_j] of the pairs idx[k B .. k B + B) with k = ctr[1], the step's batch
// index (0 at the start of an epoch; the loss kernel of each step advances it), with the transposed
// copy and the zero-padded targets. An entry of idx is (pair << 2) | mirror: mirror bit 0 reflects
// both feature maps left-right (camera x -> -x), bit 1 top-bottom (y -> -y); a reflection M maps the
// motion twist (phi, rho) to (-M phi, M rho), i.e. negates phi_y, phi_z, rho_x (left-right) or phi_x,
// phi_z, rho_y (top-bottom). Tile (blockIdx.y, blockIdx.x) = 32 rows x 32 input columns; the blocks of
// the first tile column also write the rows' targets.
__global__ void __launch_bounds__(256) k_gather(const __nv_bfloat16* __restrict__ feat, const int* __restrict__ pairs,
                                                const float* __restrict__ targets, const int* __restrict__ idx,
                                                const int* __restrict__ ctr, int B, int nL, int npL, int n_feat,
                                                __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ XT,
                                                float* __restrict__ tgt, int* __restrict__ err) {
  pdl_enter();
  __shared__ __nv_bfloat16 tile[32][34];
  const int* ib = idx + (size_t)ctr[1] * B;
  const int n0 = 2 * kFeat;
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int second = j >= kFeat;
  const int jj = j - second * kFeat;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int b = blockIdx.y * 32 + k;
    const int code = ib[b], mir = code & 3;
    const int f = pairs[2 * (code >> 2) + second];
    const bool ok = f >= 0 && f < n_feat;  // a frame index outside the feature table reads zeros
    if (!ok) atomicOr(err, 2);
    int r = jj / kFeatW, c = jj % kFeatW;
    if (mir & 1) c = kFeatW - 1 - c;
    if (mir & 2) r = kFeatH - 1 - r;
    const __nv_bfloat16 v = ok ? feat[(size_t)f * kFeat + r * kFeatW + c] : __float2bfloat16(0.f);
    X[(size_t)b * n0 + j] = v;
    tile[k][threadIdx.x] = v;
    if (blockIdx.x == 0)
      for (int cc = threadIdx.x; cc < npL; cc += 32) {
        const int neg = (((mir & 1) ? 0x0E : 0) ^ ((mir & 2) ? 0x15 : 0)) >> cc & 1;
        const float tv = cc < nL ? targets[(size_t)(code >> 2) * nL + cc] : 0.f;
        tgt[(size_t)b * npL + cc] = neg ? -tv : tv;
      }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8)
    XT[(size_t)(blockIdx.x * 32 + k) * B + blockIdx.y * 32 + threadIdx.x] = tile[threadIdx.x][k];
}

// an explicit batch: x [B x n0] and targets [B x nL] into the batch buffers (tiles as k_gather)
__global__ void __launch_bounds__(256) k_load(const __nv_bfloat16* __restrict__ x, const float* __restrict__ targets,
                                              int B, int n0, int nL, int npL, __nv_bfloat16* __restrict__ X,
                                              __nv_bfloat16* __restrict__ XT, float* __restrict__ tgt) {
  pdl_enter();
  __shared__ __nv_bfloat16 tile[32][34];
  const int j = blockIdx.x * 32 + threadIdx.x;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int b = blockIdx.y * 32 + k;
    const __nv_bfloat16 v = x[(size_t)b * n0 + j];
    X[(size_t)b * n0 + j] = v;
    tile[k][threadIdx.x] = v;
    if (blockIdx.x == 0)
      for (int cc = threadIdx.x; cc < npL; cc += 32) tgt[(size_t)b * npL + cc] = cc < nL ? targets[(size_t)b * nL + cc] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8)
    XT[(size_t)(blockIdx.x * 32 + k) * B + blockIdx.y * 32 + threadIdx.x] = tile[threadIdx.x][k];
}

struct LayerTab {
  int L;
  int ntiles;                            // 32 x 32 weight tiles of all layers
  int tile_off[kMlpMaxLayers + 1];       // first tile of each layer
  int bias_off[kMlpMaxLayers + 1];       // first bias of each layer in the biases' concatenation
  unsigned long long offW[kMlpMaxLayers], offb[kMlpMaxLayers];
  int rows[kMlpMaxLayers], cols[kMlpMaxLayers];
  __nv_bfloat16* Wq[kMlpMaxLayers];
  __nv_bfloat16* WqT[kMlpMaxLayers];
};

__device__ __forceinline__ float adam_update(float* p, const float* g, float* m1, float* m2, size_t i, float lr,
                                             float bc1, float bc2, int update) {
  float w = p[i];
  if (update) {
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w -= lr * (a / bc1) / (sqrtf(b / bc2) + 1e-8f);
    p[i] = w;
  }
  return w;
}

// Adam on the FP32 masters (update = 1; step t = ctr[0]) and the BF16 copies of the weights and their
// transposes: blocks [0, ntiles) take a 32 x 32 weight tile each, the rest 256 biases each
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                                              float* __restrict__ m2, const int* __restrict__ ctr, float lr,
                                              LayerTab tab, int update) {
  pdl_enter();
  __shared__ __nv_bfloat16 tile[32][34];
  float bc1 = 1.f, bc2 = 1.f;
  if (update) {
    const float t = (float)ctr[0];
    bc1 = 1.f - powf(0.9f, t);
    bc2 = 1.f - powf(0.999f, t);
  }
  const int bid = blockIdx.x;
  if (bid < tab.ntiles) {
    int l = 0;
    while (l + 1 < tab.L && bid >= tab.tile_off[l + 1]) ++l;
    const int rows = tab.rows[l], cols = tab.cols[l];
    const int local = bid - tab.tile_off[l], tcn = cols / 32;
    const int r0 = (local / tcn) * 32, c0 = (local % tcn) * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
      const size_t e = (size_t)(r0 + k) * cols + c0 + threadIdx.x;
      const float w = adam_update(p, g, m1, m2, tab.offW[l] + e, lr, bc1, bc2, update);
      const __nv_bfloat16 q = __float2bfloat16(w);
      tab.Wq[l][e] = q;
      tile[k][threadIdx.x] = q;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8)
      tab.WqT[l][(size_t)(c0 + k) * rows + r0 + threadIdx.x] = tile[threadIdx.x][k];
    return;
  }
  const int j = (bid - tab.ntiles) * 256 + threadIdx.y * 32 + threadIdx.x;
  if (j >= tab.bias_off[tab.L]) return;
  int l = 0;
  while (l + 1 < tab.L && j >= tab.bias_off[l + 1]) ++l;
  adam_update(p, g, m1, m2, tab.offb[l] + (j - tab.bias_off[l]), lr, bc1, bc2, update);
}

cudaError_t launch_reduce(const xslam_mlp_s* m, const float* P, int splits, int M, int N, const float* bias, int relu,
                          const __nv_bfloat16* mask, float* out32, int ld32, int n32, __nv_bfloat16* out16,
                          __nv_bfloat16* out16T, cudaStream_t s) {
  (void)m;
  // one row of threads per output row of the tile (a single-row product, the proposal's inference, uses one)
  const int ty = M >= 32 ? 32 : M;
  return launch_pdl(k_reduce, dim3((N + 31) / 32, (M + 31) / 32), dim3(32, ty), 0, s, P, splits, M, N, bias, relu, mask,
                    out32, ld32, n32, out16, out16T);
}

LayerTab layer_tab(const xslam_mlp_s* m) {
  LayerTab t = {};
  t.L = m->L;
  int nt = 0, nb = 0;
  for (int l = 0; l < m->L; ++l) {
    t.tile_off[l] = nt;
    t.bias_off[l] = nb;
    t.offW[l] = m->offW[l];
    t.offb[l] = m->offb[l];
    t.rows[l] = m->np[l + 1];
    t.cols[l] = m->np[l];
    t.Wq[l] = m->Wq[l];
    t.WqT[l] = m->WqT[l];
    nt += (m->np[l + 1] / 32) * (m->np[l] / 32);
    nb += m->np[l + 1];
  }
  t.tile_off[m->L] = nt;
  t.bias_off[m->L] = nb;
  t.ntiles = nt;
  return t;
}

cudaError_t enqueue_train_forward(xslam_mlp_s* m, int B, cudaStream_t s) {
  const void* in = m->act[0];
  for (int l = 0; l < m->L; ++l) {
    const int N = m->np[l + 1], K = m->np[l];
    const GemmPlan g = gemm_plan(B, N, K, m->nsm);
    KCU(launch_gemm_bf16(in, m->Wq[l], B, N, K, g, m->ws, m->err, s));
    const bool last = l == m->L - 1;
    KCU(launch_reduce(m, m->ws, g.splits, B, N, m->master + m->offb[l], last ? 0 : 1, nullptr, last ? m->y : nullptr, N,
                      N, last ? nullptr : m->act[l + 1], last ? nullptr : m->actT[l + 1], s));
    in = m->act[l + 1];
  }
  return cudaSuccess;
}

// count: the loss kernel advances the Adam step and the batch index (a training step)
cudaError_t enqueue_backward(xslam_mlp_s* m, int B, bool count, cudaStream_t s) {
  const int npL = m->np[m->L];
  KCU(launch_pdl(k_loss_grad, dim3((B * npL + 255) / 256), dim3(256), 0, s, (const float*)m->y, (const float*)m->tgt, B,
                 npL, m->n[m->L], m->dz32, m->dzq, m->dzqT, m->loss, count ? m->ctr : nullptr));
  for (int l = m->L - 1; l >= 0; --l) {
    const int No = m->np[l + 1], Ni = m->np[l];
    KCU(launch_pdl(k_colsum, dim3((No + 31) / 32), dim3(32, 8), 0, s, (const float*)m->dz32, B, No,
                   m->grad + m->offb[l]));
    GemmPlan g = gemm_plan(No, Ni, B, m->nsm);
    if (g.splits == 1) {  // the weight gradient [No x Ni] is the GEMM's own output: no reduction pass
      KCU(launch_gemm_bf16(m->dzqT, m->actT[l], No, Ni, B, g, m->grad + m->offW[l], m->err, s));
    } else {
      KCU(launch_gemm_bf16(m->dzqT, m->actT[l], No, Ni, B, g, m->ws, m->err, s));
      KCU(launch_reduce(m, m->ws, g.splits, No, Ni, nullptr, 0, nullptr, m->grad + m->offW[l], Ni, Ni, nullptr, nullptr,
                        s));
    }
    if (l > 0) {
      g = gemm_plan(B, Ni, No, m->nsm);
      KCU(launch_gemm_bf16(m->dzq, m->WqT[l], B, Ni, No, g, m->ws, m->err, s));
      KCU(launch_reduce(m, m->ws, g.splits, B, Ni, nullptr, 0, m->act[l], m->dz32, Ni, Ni, m->dzq, m->dzqT, s));
    }
  }
  return cudaSuccess;
}

cudaError_t enqueue_adam(xslam_mlp_s* m, float lr, int update, cudaStream_t s) {
  const LayerTab t = layer_tab(m);
  const int blocks = t.ntiles + (t.bias_off[m->L] + 255) / 256;
  return launch_pdl(k_adam, dim3(blocks), dim3(32, 8), 0, s, m->master, (const float*)m->grad, m->m1, m->m2,
                    (const int*)m->ctr, lr, t, update);
}

size_t gemm_ws(int M, int N, int K, int nsm) {
  const GemmPlan g = gemm_plan(M, N, K, nsm);
  return (size_t)g.splits * M * N;
}

xslam_status enter(xslam_mlp_t m) {
  MCU(cudaEventRecord(m->ev_in, m->user));
  MCU(cudaStreamWaitEvent(m->s, m->ev_in, 0));
  return XSLAM_OK;
}

xslam_status leave_sync(xslam_mlp_t m) {
  MCU(cudaEventRecord(m->ev_out, m->s));
  MCU(cudaStreamWaitEvent(m->user, m->ev_out, 0));
  MCU(cudaStreamSynchronize(m->s));
  int e = 0;
  MCU(cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    MCU(cudaMemset(m->err, 0, sizeof(int)));
    if (e & 1) return mfail(m, XSLAM_ETIMEOUT, "a tensor-core wait of the GEMM kernel ran out");
    return mfail(m, XSLAM_EINVAL, "a training pair names a frame outside the feature table");
  }
  return XSLAM_OK;
}

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void free_all(xslam_mlp_t m) {
  cudaFree(m->master);
  cudaFree(m->grad);
  cudaFree(m->m1);
  cudaFree(m->m2);
  for (int l = 0; l < kMlpMaxLayers; ++l) {
    cudaFree(m->Wq[l]);
    cudaFree(m->WqT[l]);
    cudaFree(m->act[l]);
    cudaFree(m->actT[l]);
  }
  cudaFree(m->dzq);
  cudaFree(m->dzqT);
  cudaFree(m->dz32);
  cudaFree(m->y);
  cudaFree(m->tgt);
  cudaFree(m->ws);
  cudaFree(m->loss);
  cudaFree(m->ctr);
  cudaFree(m->err);
  cudaFree(m->idx);
  if (m->ev_in) cudaEventDestroy(m->ev_in);
  if (m->ev_out) cudaEventDestroy(m->ev_out);
  if (m->s) cudaStreamDestroy(m->s);
}

}  // namespace

// ---------------------------------------------------------------------------------------------------
// shared with the proposal path of the frame chain
// ---------------------------------------------------------------------------------------------------
size_t xslam::mlp_ws_floats(const xslam_mlp_s* m, int B) {
  size_t w = 0;
  for (int l = 0; l < m->L; ++l) w = std::max(w, gemm_ws(B, m->np[l + 1], m->np[l], m->nsm));
  return w;
}

cudaError_t xslam::mlp_enqueue_forward(const xslam_mlp_s* m, const void* X, int B, __nv_bfloat16* const* act, float* ws,
                                       float* y, int ld_y, int ny, int* err, cudaStream_t s) {
  const void* in = X;
  for (int l = 0; l < m->L; ++l) {
    const int N = m->np[l + 1], K = m->np[l];
    const GemmPlan g = gemm_plan(B, N, K, m->nsm);
    KCU(launch_gemm_bf16(in, m->Wq[l], B, N, K, g, ws, err, s));
    const bool last = l == m->L - 1;
    KCU(launch_reduce(m, ws, g.splits, B, N, m->master + m->offb[l], last ? 0 : 1, nullptr, last ? y : nullptr, ld_y,
                      ny, last ? nullptr : act[l + 1], nullptr, s));
    if (!last) in = act[l + 1];
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------------
extern "C" xslam_status xslam_mlp_create(xslam_mlp_t* out, int n_layers, const int* sizes, int max_batch,
                                         void* cuda_stream) {
  xslam_mlp_t m = nullptr;
  if (!out) return mfail(nullptr, XSLAM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_layers < 1 || n_layers > kMlpMaxLayers || !sizes)
    return mfail(nullptr, XSLAM_EINVAL, "n_layers must be 1..6 with sizes given");
  for (int l = 0; l <= n_layers; ++l)
    if (sizes[l] < 1 || sizes[l] > 16384) return mfail(nullptr, XSLAM_EINVAL, "every width must be 1..16384");
  if (sizes[0] % 64) return mfail(nullptr, XSLAM_EINVAL, "sizes[0] must be a multiple of 64");
  if (max_batch < 1 || max_batch > 4096) return mfail(nullptr, XSLAM_EINVAL, "max_batch must be 1..4096");
  m = new xslam_mlp_s();
  m->L = n_layers;
  m->max_batch = max_batch;
  m->user = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int l = 0; l <= n_layers; ++l) {
    m->n[l] = sizes[l];
    m->np[l] = l == 0 ? sizes[0] : pad64(sizes[l]);
    if (l > 0) m->npmax = std::max(m->npmax, m->np[l]);
  }
  size_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->offW[l] = off;
    off += (size_t)m->np[l + 1] * m->np[l];
    m->offb[l] = off;
    off += (size_t)m->np[l + 1];
    m->n_params += (size_t)m->n[l + 1] * m->n[l] + m->n[l + 1];
  }
  m->n_master = off;
  const int B = max_batch;
  size_t ws = 0;
  for (int b = 1; b <= B; ++b) ws = std::max(ws, mlp_ws_floats(m, b));
  for (int Bt = 64; Bt <= B; Bt += 64)  // training and gradient batches are multiples of 64
    for (int l = 0; l < n_layers; ++l) {
      ws = std::max(ws, gemm_ws(m->np[l + 1], m->np[l], Bt, m->nsm));
      ws = std::max(ws, gemm_ws(Bt, m->np[l], m->np[l + 1], m->nsm));
    }
  m->ws_floats = ws;
  bool ok = cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming) == cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) { ok &= cudaMalloc(p, bytes < 16 ? 16 : bytes) == cudaSuccess; };
  alloc((void**)&m->master, sizeof(float) * off);
  alloc((void**)&m->grad, sizeof(float) * off);
  alloc((void**)&m->m1, sizeof(float) * off);
  alloc((void**)&m->m2, sizeof(float) * off);
  for (int l = 0; l < n_layers; ++l) {
    alloc((void**)&m->Wq[l], sizeof(__nv_bfloat16) * m->np[l + 1] * m->np[l]);
    alloc((void**)&m->WqT[l], sizeof(__nv_bfloat16) * m->np[l + 1] * m->np[l]);
    alloc((void**)&m->act[l], sizeof(__nv_bfloat16) * (size_t)B * m->np[l]);
    alloc((void**)&m->actT[l], sizeof(__nv_bfloat16) * (size_t)B * m->np[l]);
  }
  alloc((void**)&m->dzq, sizeof(__nv_bfloat16) * (size_t)B * m->npmax);
  alloc((void**)&m->dzqT, sizeof(__nv_bfloat16) * (size_t)B * m->npmax);
  alloc((void**)&m->dz32, sizeof(float) * (size_t)B * m->npmax);
  alloc((void**)&m->y, sizeof(float) * (size_t)B * m->np[n_layers]);
  alloc((void**)&m->tgt, sizeof(float) * (size_t)B * m->np[n_layers]);
  alloc((void**)&m->ws, sizeof(float) * ws);
  alloc((void**)&m->loss, sizeof(double));
  alloc((void**)&m->ctr, sizeof(int) * 2);
  alloc((void**)&m->err, sizeof(int));
  if (!ok) {
    free_all(m);
    delete m;
    cudaGetLastError();
    return mfail(nullptr, XSLAM_ENOMEM, "device allocation failed");
  }
  cudaError_t e = gemm_configure();
  if (e == cudaSuccess) e = cudaMemsetAsync(m->master, 0, sizeof(float) * off, m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, sizeof(float) * off, m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, sizeof(float) * off, m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * off, m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->ctr, 0, sizeof(int) * 2, m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int), m->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->s);
  for (int l = 0; l < n_layers && e == cudaSuccess; ++l) {
    e = cudaMemsetAsync(m->Wq[l], 0, sizeof(__nv_bfloat16) * m->np[l + 1] * m->np[l], m->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->WqT[l], 0, sizeof(__nv_bfloat16) * m->np[l + 1] * m->np[l], m->s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->s);
  if (e != cudaSuccess) {
    const std::string msg = std::string("initialisation: ") + cudaGetErrorString(e);
    free_all(m);
    delete m;
    return mfail(nullptr, XSLAM_ECUDA, msg);
  }
  *out = m;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_mlp_destroy(xslam_mlp_t m) {
  if (!m) return XSLAM_OK;
  if (m->s) cudaStreamSynchronize(m->s);
  free_all(m);
  delete m;
  return XSLAM_OK;
}

extern "C" size_t xslam_mlp_param_count(xslam_mlp_t m) { return m ? m->n_params : 0; }

extern "C" xslam_status xslam_mlp_set_params(xslam_mlp_t m, const float* params) {
  if (!m || !params) return mfail(m, XSLAM_EINVAL, "NULL argument");
  std::vector<float> pad(m->n_master, 0.f);
  size_t k = 0;
  for (int l = 0; l < m->L; ++l) {
    for (int r = 0; r < m->n[l + 1]; ++r)
      for (int c = 0; c < m->n[l]; ++c) pad[m->offW[l] + (size_t)r * m->np[l] + c] = params[k++];
    for (int r = 0; r < m->n[l + 1]; ++r) pad[m->offb[l] + r] = params[k++];
  }
  xslam_status st = enter(m);
  if (st != XSLAM_OK) return st;
  MCU(cudaMemcpyAsync(m->master, pad.data(), sizeof(float) * m->n_master, cudaMemcpyHostToDevice, m->s));
  MCU(cudaMemsetAsync(m->m1, 0, sizeof(float) * m->n_master, m->s));
  MCU(cudaMemsetAsync(m->m2, 0, sizeof(float) * m->n_master, m->s));
  MCU(cudaMemsetAsync(m->ctr, 0, sizeof(int) * 2, m->s));
  MCU(enqueue_adam(m, 0.f, 0, m->s));
  return leave_sync(m);
}

extern "C" xslam_status xslam_mlp_get_params(xslam_mlp_t m, float* params) {
  if (!m || !params) return mfail(m, XSLAM_EINVAL, "NULL argument");
  std::vector<float> pad(m->n_master);
  MCU(cudaStreamSynchronize(m->s));
  MCU(cudaMemcpy(pad.data(), m->master, sizeof(float) * m->n_master, cudaMemcpyDeviceToHost));
  size_t k = 0;
  for (int l = 0; l < m->L; ++l) {
    for (int r = 0; r < m->n[l + 1]; ++r)
      for (int c = 0; c < m->n[l]; ++c) params[k++] = pad[m->offW[l] + (size_t)r * m->np[l] + c];
    for (int r = 0; r < m->n[l + 1]; ++r) params[k++] = pad[m->offb[l] + r];
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_mlp_forward(xslam_mlp_t m, const void* x, int B, float* y) {
  if (!m || !x || !y) return mfail(m, XSLAM_EINVAL, "NULL argument");
  if (B < 1 || B > m->max_batch) return mfail(m, XSLAM_EINVAL, "B must be 1..max_batch");
  if (((uintptr_t)x) % 16) return mfail(m, XSLAM_EINVAL, "x must be 16-byte aligned");
  xslam_status st = enter(m);
  if (st != XSLAM_OK) return st;
  MCU(mlp_enqueue_forward(m, x, B, m->act, m->ws, y, m->n[m->L], m->n[m->L], m->err, m->s));
  return leave_sync(m);
}

extern "C" xslam_status xslam_mlp_gradient(xslam_mlp_t m, const void* x, const float* targets, int B, float* grad,
                                           double* loss) {
  if (!m || !x || !targets) return mfail(m, XSLAM_EINVAL, "NULL argument");
  if (B < 64 || B % 64 || B > m->max_batch) return mfail(m, XSLAM_EINVAL, "B must be a multiple of 64 up to max_batch");
  xslam_status st = enter(m);
  if (st != XSLAM_OK) return st;
  MCU(cudaMemsetAsync(m->loss, 0, sizeof(double), m->s));
  MCU(launch_pdl(k_load, dim3(m->np[0] / 32, B / 32), dim3(32, 8), 0, m->s, (const __nv_bfloat16*)x, targets, B,
                 m->np[0], m->n[m->L], m->np[m->L], m->act[0], m->actT[0], m->tgt));
  MCU(enqueue_train_forward(m, B, m->s));
  MCU(enqueue_backward(m, B, false, m->s));
  if ((st = leave_sync(m)) != XSLAM_OK) return st;
  if (loss) MCU(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
  if (grad) {
    std::vector<float> pad(m->n_master);
    MCU(cudaMemcpy(pad.data(), m->grad, sizeof(float) * m->n_master, cudaMemcpyDeviceToHost));
    size_t k = 0;
    for (int l = 0; l < m->L; ++l) {
      for (int r = 0; r < m->n[l + 1]; ++r)
        for (int c = 0; c < m->n[l]; ++c) grad[k++] = pad[m->offW[l] + (size_t)r * m->np[l] + c];
      for (int r = 0; r < m->n[l + 1]; ++r) grad[k++] = pad[m->offb[l] + r];
    }
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_mlp_features(const float* depth, int n, int W, int H, float depth_min, float depth_max,
                                           void* out, void* cuda_stream) {
  xslam_mlp_t m = nullptr;
  if (!depth || !out || n < 1) return mfail(m, XSLAM_EINVAL, "NULL argument or n < 1");
  if (W < kFeatW || H < kFeatH || W % kFeatW || H % kFeatH)
    return mfail(m, XSLAM_EINVAL, "the image size must be a multiple of 80 x 60");
  MCU(launch_features(depth, n, W, H, depth_min, depth_max, out, kFeat, nullptr, (cudaStream_t)cuda_stream));
  return XSLAM_OK;
}

extern "C" xslam_status xslam_mlp_pair_targets(const double* poses, int n_poses, const int* pairs, int n_pairs,
                                               const float* scale, float* out) {
  xslam_mlp_t m = nullptr;
  if (!poses || !pairs || !scale || !out || n_poses < 1 || n_pairs < 0) return mfail(m, XSLAM_EINVAL, "bad argument");
  for (int p = 0; p < n_pairs; ++p) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    if (i < 0 || j < 0 || i >= n_poses || j >= n_poses) return mfail(m, XSLAM_EINVAL, "pair index out of range");
    const double* A = poses + 12 * i;
    const double* Bm = poses + 12 * j;
    // D = T_i^-1 T_j = [Ri^T Rj | Ri^T (tj - ti)]
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) R[3 * r + c] = A[r] * Bm[c] + A[4 + r] * Bm[4 + c] + A[8 + r] * Bm[8 + c];
      t[r] = A[r] * (Bm[3] - A[3]) + A[4 + r] * (Bm[7] - A[7]) + A[8 + r] * (Bm[11] - A[11]);
    }
    // rotation: angle from the trace, axis from the skew part
    const double cth = std::min(1.0, std::max(-1.0, (R[0] + R[4] + R[8] - 1.0) / 2.0));
    const double th = std::acos(cth);
    double w[3] = {(R[7] - R[5]) / 2.0, (R[2] - R[6]) / 2.0, (R[3] - R[1]) / 2.0};
    const double f = th < 1e-8 ? 1.0 : th / std::sin(th);
    double phi[3] = {w[0] * f, w[1] * f, w[2] * f};
    // rho = J(phi)^-1 t with J = I + (1 - cos)/th^2 P + (th - sin)/th^3 P^2, solved by Gaussian elimination
    const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], tn = std::sqrt(t2);
    double a, b;
    if (tn < 1e-8) {
      a = 0.5;
      b = 1.0 / 6.0;
    } else {
      a = (1.0 - std::cos(tn)) / t2;
      b = (tn - std::sin(tn)) / (t2 * tn);
    }
    const double P[9] = {0.0, -phi[2], phi[1], phi[2], 0.0, -phi[0], -phi[1], phi[0], 0.0};
    double J[3][4];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) {
        double p2 = P[3 * r] * P[c] + P[3 * r + 1] * P[3 + c] + P[3 * r + 2] * P[6 + c];
        J[r][c] = (r == c ? 1.0 : 0.0) + a * P[3 * r + c] + b * p2;
      }
      J[r][3] = t[r];
    }
    for (int c = 0; c < 3; ++c) {
      int piv = c;
      for (int r = c + 1; r < 3; ++r)
        if (std::fabs(J[r][c]) > std::fabs(J[piv][c])) piv = r;
      for (int k = 0; k < 4; ++k) std::swap(J[c][k], J[piv][k]);
      for (int r = 0; r < 3; ++r) {
        if (r == c) continue;
        const double q = J[r][c] / J[c][c];
        for (int k = c; k < 4; ++k) J[r][k] -= q * J[c][k];
      }
    }
    const double xi[6] = {phi[0], phi[1], phi[2], J[0][3] / J[0][0], J[1][3] / J[1][1], J[2][3] / J[2][2]};
    for (int k = 0; k < 6; ++k) out[6 * p + k] = (float)(xi[k] / (double)scale[k]);
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_mlp_train(xslam_mlp_t m, const void* feat, int n_feat, const int* pairs,
                                        const float* targets, int n_pairs, int batch, int epochs, float lr,
                                        unsigned long long seed, int mirror, float* epoch_loss) {
  if (!m || !feat || !pairs || !targets) return mfail(m, XSLAM_EINVAL, "NULL argument");
  if (m->n[0] != 2 * kFeat) return mfail(m, XSLAM_EINVAL, "training from frame pairs needs sizes[0] = 9600");
  if (mirror != 0 && mirror != 1) return mfail(m, XSLAM_EINVAL, "mirror must be 0 or 1");
  if (mirror && m->n[m->L] != 6) return mfail(m, XSLAM_EINVAL, "mirroring needs 6 twist outputs");
  if (n_pairs > (1 << 28)) return mfail(m, XSLAM_EINVAL, "too many pairs");
  if (batch < 64 || batch % 64 || batch > m->max_batch)
    return mfail(m, XSLAM_EINVAL, "batch must be a multiple of 64 up to max_batch");
  if (n_pairs < batch || epochs < 1 || n_feat < 1 || !(lr > 0.f)) return mfail(m, XSLAM_EINVAL, "bad sizes or lr");
  if (n_pairs > m->idx_cap) {
    MCU(cudaStreamSynchronize(m->s));
    cudaFree(m->idx);
    m->idx = nullptr;
    m->idx_cap = 0;
    if (cudaMalloc(&m->idx, sizeof(int) * (size_t)n_pairs) != cudaSuccess) {
      cudaGetLastError();
      return mfail(m, XSLAM_ENOMEM, "permutation allocation failed");
    }
    m->idx_cap = n_pairs;
  }
  xslam_status st = enter(m);
  if (st != XSLAM_OK) return st;
  // one step as a graph: gather, forward, loss, backward, Adam
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  MCU(cudaStreamBeginCapture(m->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_pdl(k_gather, dim3(m->np[0] / 32, batch / 32), dim3(32, 8), 0, m->s,
                             (const __nv_bfloat16*)feat, pairs, targets, (const int*)m->idx, (const int*)m->ctr, batch,
                             m->n[m->L], m->np[m->L], n_feat, m->act[0], m->actT[0], m->tgt, m->err);
  if (e == cudaSuccess) e = enqueue_train_forward(m, batch, m->s);
  if (e == cudaSuccess) e = enqueue_backward(m, batch, true, m->s);
  if (e == cudaSuccess) e = enqueue_adam(m, lr, 1, m->s);
  cudaError_t e2 = cudaStreamEndCapture(m->s, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    return mfail(m, XSLAM_ECUDA, std::string("training graph: ") + cudaGetErrorString(e));
  }
  std::vector<int> perm(n_pairs);
  const int nb = n_pairs / batch;
  uint64_t rs = seed;
  for (int ep = 0; ep < epochs && st == XSLAM_OK; ++ep) {
    for (int i = 0; i < n_pairs; ++i) perm[i] = i << 2;
    for (int i = n_pairs - 1; i > 0; --i) {
      const int j = (int)(splitmix64(rs) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    if (mirror)
      for (int i = 0; i < n_pairs; ++i) perm[i] |= (int)(splitmix64(rs) & 3u);
    e = cudaMemcpyAsync(m->idx, perm.data(), sizeof(int) * (size_t)n_pairs, cudaMemcpyHostToDevice, m->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->ctr + 1, 0, sizeof(int), m->s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->s);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaGraphLaunch(exec, m->s);
    double ls = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ls, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->s);  // the host permutation is reused next epoch
    if (e != cudaSuccess) {
      st = mfail(m, XSLAM_ECUDA, std::string("training step: ") + cudaGetErrorString(e));
      break;
    }
    if (epoch_loss) epoch_loss[ep] = (float)(ls / nb);
  }
  cudaGraphExecDestroy(exec);
  if (st != XSLAM_OK) return st;
  return leave_sync(m);
}

extern "C" xslam_status xslam_gemm_bf16(const void* A, const void* B, int M, int N, int K, float* C, int splits,
                                        float* workspace, void* cuda_stream) {
  xslam_mlp_t m = nullptr;
  if (!A || !B || !C) return mfail(m, XSLAM_EINVAL, "NULL argument");
  if (!gemm_shape_ok(M, N, K)) return mfail(m, XSLAM_EINVAL, "need M, N >= 1 and K a positive multiple of 64");
  if (splits < 1 || splits > K / 64) return mfail(m, XSLAM_EINVAL, "splits must be 1..K/64");
  if (splits > 1 && !workspace) return mfail(m, XSLAM_EINVAL, "splits > 1 needs a workspace");
  if (((uintptr_t)A) % 16 || ((uintptr_t)B) % 16) return mfail(m, XSLAM_EINVAL, "A and B must be 16-byte aligned");
  int* err = nullptr;
  MCU(cudaGetSymbolAddress((void**)&err, g_gemm_err));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  GemmPlan g;
  g.kb_per_split = (K / 64 + splits - 1) / splits;
  g.splits = (K / 64 + g.kb_per_split - 1) / g.kb_per_split;
  if (e == cudaSuccess) e = gemm_configure();
  if (e == cudaSuccess) e = launch_gemm_bf16(A, B, M, N, K, g, g.splits == 1 ? C : workspace, err, s);
  if (e == cudaSuccess && g.splits > 1)
    e = launch_pdl(k_reduce, dim3((N + 31) / 32, (M + 31) / 32), dim3(32, M >= 32 ? 32 : M), 0, s, (const float*)workspace, g.splits, M,
                   N, (const float*)nullptr, 0, (const __nv_bfloat16*)nullptr, C, N, N, (__nv_bfloat16*)nullptr,
                   (__nv_bfloat16*)nullptr);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mfail(m, XSLAM_ECUDA, std::string("gemm: ") + cudaGetErrorString(e));
  if (h_err) return mfail(m, XSLAM_ETIMEOUT, "a tensor-core wait of the GEMM kernel ran out");
  return XSLAM_OK;
}

extern "C" const char* xslam_mlp_last_error(xslam_mlp_t m) { return m ? m->msg.c_str() : g_mlp_err.c_str(); }
