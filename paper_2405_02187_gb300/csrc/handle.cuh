// The handle behind xslam_t (include/xslam.h), shared by the C ABI (api.cu) and the batch driver
// (batch.cu).
#pragma once

#include <string>

#include "../../include/xslam.h"
#include "internal.cuh"

constexpr int kProfRing = 256;

struct xslam_s {
  xslam::Params p;
  xslam::Buffers b;
  xslam_config cfg;
  int max_lanes = 0;
  int nsm = 148;
  cudaStream_t s = nullptr;     // internal stream
  cudaStream_t user = nullptr;  // caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int frame = 0;
  int K = 0;
  xslam_seed seeds[xslam::kMaxLanes];
  int* d_kinds = nullptr;   // device copies of lane kinds / indices
  int* d_index = nullptr;
  double* pose_tmp = nullptr;  // scratch pose lanes (raycast / grad)
  float* hess_poses = nullptr;  // the 21 truncated-bicomplex start poses of xslam_grad order 2
  double* hess_poses64 = nullptr;  // the 21 bicomplex start poses (h = 1e-20) of the plain FP64 TSDF Hessian
  float* model_q = nullptr;    // scratch model maps of xslam_grad (7 lanes)
  double* h_result = nullptr;  // pinned host staging
  int* h_status = nullptr;
  // pipelined frames (xslam_frame_submit / xslam_frame_wait), allocated by the first submit
  cudaStream_t cs = nullptr;                  // copy stream of host depth maps
  float* stage[2] = {};                       // device staging buffers of host depth maps, used in turn
  cudaEvent_t ev_h2d[2] = {}, ev_used[2] = {};  // staging buffer filled / consumed by its frame
  int stage_next = 0;
  double* h_ring = nullptr;                   // pinned outputs: XSLAM_PIPELINE slots of kResSys doubles
  int* h_sring = nullptr;                     // pinned status words: XSLAM_PIPELINE slots of 8
  cudaEvent_t ev_res[XSLAM_PIPELINE] = {};    // a slot's outputs are on the host
  int ring_K[XSLAM_PIPELINE] = {};            // lane count of each slot's frame
  long long t_next = 0, t_done = 0;           // next ticket handed out, oldest not waited for
  // constant-velocity start and learned proposal (proposal.cu); the network is the caller's
  xslam::PropBuffers q = {};
  struct xslam_mlp_s* mlp = nullptr;
  float prop_scale[6] = {};
  int judge_level = 0;
  int judge_nblk = 1;
  void* prop_act[8] = {};   // BF16 hidden activations of the network's forward pass (1 row each)
  float* prop_ws = nullptr; // its split-K workspace
  int nblk[3] = {1, 1, 1};
  bool in_batch = false;      // grouped by a live xslam_batch (which may change nblk until it is destroyed)
  int nblk_max = 1;
  cudaGraphExec_t g_first = nullptr, g_track = nullptr;
  bool use_graphs = true;
  // stage profiling (xslam_profile): one event pair per stage and frame, accumulated on read
  bool profiling = false;
  cudaEvent_t pev[XSLAM_NSTAGE][kProfRing][2] = {};
  int pcount[XSLAM_NSTAGE] = {};      // pairs recorded and not yet accumulated
  double pms[XSLAM_NSTAGE] = {};      // accumulated milliseconds
  long long plaunch[XSLAM_NSTAGE] = {};
  long long pframes = 0;
  std::string err;
};

namespace xslam {
// enqueues one frame chain (frame 0 when first, else a tracking frame) on the handle's stream
cudaError_t enqueue_chain(xslam_t h, bool first);
// drops the handle's captured frame graphs (after a change of lanes or grid sizes)
void handle_drop_graphs(xslam_t h);
}  // namespace xslam
