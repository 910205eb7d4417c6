// The network object behind xslam_mlp_t (include/xslam_mlp.h), shared by its C ABI (mlp.cu) and the
// proposal path of the frame chain (api.cu).
#pragma once

#include <cuda_bf16.h>

#include <string>

#include "../../include/xslam_mlp.h"
#include "internal.cuh"

constexpr int kMlpMaxLayers = 6;

struct xslam_mlp_s {
  int L = 0;
  int n[kMlpMaxLayers + 1] = {};   // layer widths
  int np[kMlpMaxLayers + 1] = {};  // widths padded to multiples of 64 (np[0] = n[0])
  int npmax = 0;                   // max of np[1..L]
  int max_batch = 0;
  int nsm = 148;
  cudaStream_t s = nullptr, user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // FP32 parameters in the padded layout: per layer W_l [np[l+1] x np[l]] at offW[l], b_l at offb[l]
  size_t n_master = 0, n_params = 0;
  size_t offW[kMlpMaxLayers] = {}, offb[kMlpMaxLayers] = {};
  float* master = nullptr;
  float* grad = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  __nv_bfloat16* Wq[kMlpMaxLayers] = {};   // BF16 W_l [np[l+1] x np[l]]
  __nv_bfloat16* WqT[kMlpMaxLayers] = {};  // BF16 W_l^T [np[l] x np[l+1]]
  // batch scratch (max_batch rows): act[l] = a_l [B x np[l]] (act[0] the input), actT[l] its transpose
  __nv_bfloat16* act[kMlpMaxLayers] = {};
  __nv_bfloat16* actT[kMlpMaxLayers] = {};
  __nv_bfloat16* dzq = nullptr;   // q(dz) [B x npmax]
  __nv_bfloat16* dzqT = nullptr;  // its transpose [npmax x B]
  float* dz32 = nullptr;          // dz [B x npmax]
  float* y = nullptr;             // output [B x np[L]]
  float* tgt = nullptr;           // targets [B x np[L]] (zero padded)
  float* ws = nullptr;            // split-K partial products
  size_t ws_floats = 0;
  double* loss = nullptr;  // summed batch losses since the last clear
  int* ctr = nullptr;      // [0] Adam step, [1] batch index within the epoch
  int* err = nullptr;      // tensor-core wait timed out
  int* idx = nullptr;      // training permutation
  int idx_cap = 0;
  std::string msg;
};

namespace xslam {
// split-K workspace (floats) the forward pass of B rows needs
size_t mlp_ws_floats(const xslam_mlp_s* m, int B);
// forward pass of B rows X (BF16 [B x np[0]]) into y (FP32, row stride ld_y, first ny columns), on
// stream s: act[1..L-1] the hidden activations ([B x np[l]] BF16 each), ws the split-K workspace
cudaError_t mlp_enqueue_forward(const xslam_mlp_s* m, const void* X, int B, __nv_bfloat16* const* act, float* ws,
                                float* y, int ld_y, int ny, int* err, cudaStream_t s);
}  // namespace xslam
