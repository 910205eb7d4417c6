// Batch driver (include/xslam_batch.h): many trajectories advanced by one CUDA graph per step.
//
// The graph of a step is captured from the handles' own frame chains: on the batch stream, a start
// event and one gather kernel that copies every active trajectory's depth frame (through a device
// table of source pointers, refreshed before each launch) into its handle's input buffer; then a
// fork to every active handle's stream, where that handle's chain is enqueued exactly as xslam_frame
// does, and a join back. The kernels of different trajectories therefore run concurrently, while
// each trajectory's own kernels keep their order. A captured graph is reused as long as the set of
// active trajectories (and which of them are at frame 0) does not change.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/xslam_batch.h"
#include "handle.cuh"

using namespace xslam;

namespace {

// dst[t][0..cnt[t]) = src[t][...] for every trajectory t with a source this step
__global__ void k_gather_frames(const float* const* __restrict__ src, float* const* __restrict__ dst,
                                const int* __restrict__ cnt, int n) {
  const int t = blockIdx.y;
  if (t >= n) return;
  const float* s = src[t];
  if (!s) return;
  float* d = dst[t];
  const int c = cnt[t];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) d[i] = s[i];
}

std::string g_batch_err;
constexpr int kRing = 8;        // pinned source tables in flight
constexpr int kMaxBatch = 256;  // trajectories per batch
constexpr int kDivisors[5] = {1, 2, 4, 8, 16};

}  // namespace

struct xslam_batch_s {
  int n = 0;
  std::vector<xslam_t> hs;
  std::vector<std::vector<xslam_seed>> seeds;      // lanes recorded at create
  std::vector<std::array<double, 12>> pose0;       // frame-0 pose recorded at create
  std::vector<std::array<int, 3>> nblk0;           // default ICP grids
  std::vector<char> persistent0;                   // the handles' ICP kernel choice, restored at destroy
  cudaStream_t s = nullptr, user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_start = nullptr;
  std::vector<cudaEvent_t> ev_join;                // per trajectory, end of its chain (join edge)
  std::vector<cudaEvent_t> ev_done;                // per trajectory, end of its chain (timing node)
  const float** h_src[kRing] = {};                 // pinned source tables
  cudaEvent_t ev_slot[kRing] = {};
  int slot = 0;
  const float** d_src = nullptr;                   // device source table read by the gather kernel
  float** d_dst = nullptr;
  int* d_cnt = nullptr;
  int max_hw = 1;
  std::vector<int> key;                            // per trajectory: 0 idle, 1 frame 0, 2 tracking
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> last;                           // trajectories that advanced in the last step
  std::string err;
};

static xslam_status bfail(xslam_batch_t b, xslam_status st, const std::string& m) {
  if (b) b->err = m;
  else g_batch_err = m;
  return st;
}

#define BCU(call)                                                                                        \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return bfail(b, XSLAM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

static void drop_graph(xslam_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key.clear();
}

static void free_batch(xslam_batch_t b) {
  if (b->s) cudaStreamSynchronize(b->s);
  drop_graph(b);
  for (size_t i = 0; i < b->persistent0.size(); ++i) {
    b->hs[i]->icp_persistent = b->persistent0[i] != 0;
    handle_drop_graphs(b->hs[i]);
  }
  for (int r = 0; r < kRing; ++r) {
    if (b->h_src[r]) cudaFreeHost(b->h_src[r]);
    if (b->ev_slot[r]) cudaEventDestroy(b->ev_slot[r]);
  }
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_done)
    if (e) cudaEventDestroy(e);
  cudaFree(b->d_src);
  cudaFree(b->d_dst);
  cudaFree(b->d_cnt);
  for (cudaEvent_t e : {b->ev_in, b->ev_out, b->ev_fork, b->ev_start})
    if (e) cudaEventDestroy(e);
  if (b->s) cudaStreamDestroy(b->s);
}

extern "C" xslam_status xslam_batch_create(xslam_batch_t* out, int n, xslam_t const* handles, void* cuda_stream) {
  xslam_batch_t b = nullptr;
  if (!out || !handles) return bfail(b, XSLAM_EINVAL, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > kMaxBatch) return bfail(b, XSLAM_EINVAL, "n must be in 1..256");
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return bfail(b, XSLAM_EINVAL, "a handle is NULL");
    if (handles[i]->frame != 0) return bfail(b, XSLAM_EINVAL, "every handle must be before its first frame");
    if (handles[i]->profiling) return bfail(b, XSLAM_EINVAL, "stage profiling must be off in a batch");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return bfail(b, XSLAM_EINVAL, "a handle is listed twice");
  }
  b = new xslam_batch_s();
  b->n = n;
  b->user = (cudaStream_t)cuda_stream;
  b->hs.assign(handles, handles + n);
  auto cleanup = [&](xslam_status st, const std::string& m) {
    free_batch(b);
    delete b;
    return bfail(nullptr, st, m);
  };
  bool ok = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreate(&b->ev_start) == cudaSuccess;
  b->ev_join.assign(n, nullptr);
  b->ev_done.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i) {
    ok &= cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
    ok &= cudaEventCreate(&b->ev_done[i]) == cudaSuccess;
  }
  for (int r = 0; r < kRing && ok; ++r) {
    ok &= cudaMallocHost(&b->h_src[r], sizeof(float*) * n) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&b->ev_slot[r], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&b->d_src, sizeof(float*) * n) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_dst, sizeof(float*) * n) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_cnt, sizeof(int) * n) == cudaSuccess;
  if (!ok) return cleanup(XSLAM_ENOMEM, "stream, event or allocation failed");
  std::vector<float*> dst(n);
  std::vector<int> cnt(n);
  for (int i = 0; i < n; ++i) {
    xslam_t h = b->hs[i];
    dst[i] = h->b.depth_in;
    cnt[i] = h->p.W * h->p.H;
    b->max_hw = std::max(b->max_hw, cnt[i]);
    b->seeds.emplace_back(h->seeds, h->seeds + h->K);
    b->nblk0.push_back({h->nblk[0], h->nblk[1], h->nblk[2]});
    // the trajectories' chains run as concurrent graph branches: each ICP iteration is its own launch
    // sized to its level (a cooperative launch holds a block on every SM for the whole ICP range)
    b->persistent0.push_back(h->icp_persistent ? 1 : 0);
    h->icp_persistent = false;
    handle_drop_graphs(h);
    std::array<double, 12> T{};
    cudaStreamSynchronize(h->s);
    if (cudaMemcpy(T.data(), h->b.pose, sizeof(double) * 12, cudaMemcpyDeviceToHost) != cudaSuccess)
      return cleanup(XSLAM_ECUDA, "cannot read a handle's pose");
    b->pose0.push_back(T);
  }
  if (cudaMemcpy(b->d_dst, dst.data(), sizeof(float*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_cnt, cnt.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_src, 0, sizeof(float*) * n) != cudaSuccess)
    return cleanup(XSLAM_ECUDA, "cannot initialise the gather tables");
  *out = b;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_destroy(xslam_batch_t b) {
  if (!b) return XSLAM_OK;
  free_batch(b);
  delete b;
  return XSLAM_OK;
}

static xslam_status build_graph(xslam_batch_t b, const std::vector<int>& key) {
  drop_graph(b);
  const int n = b->n;
  BCU(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
  // timing events become event-record nodes of the graph (external records); the fork and join events
  // only carry dependencies
  cudaError_t e = cudaEventRecordWithFlags(b->ev_start, b->s, cudaEventRecordExternal);
  if (e == cudaSuccess) {
    const int gx = std::max(1, std::min(64, (b->max_hw + 255) / 256));
    k_gather_frames<<<dim3(gx, n), 256, 0, b->s>>>(b->d_src, b->d_dst, b->d_cnt, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (!key[i]) continue;
    xslam_t h = b->hs[i];
    e = cudaStreamWaitEvent(h->s, b->ev_fork, 0);
    if (e == cudaSuccess) e = enqueue_chain(h, key[i] == 1);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_done[i], h->s, cudaEventRecordExternal);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[i], h->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, b->ev_join[i], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->s, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, XSLAM_ECUDA, std::string("batch graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  const cudaError_t e3 = cudaGraphInstantiate(&b->exec, g, 0);
  if (e3 != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    return bfail(b, XSLAM_ECUDA, std::string("batch graph instantiation failed: ") + cudaGetErrorString(e3));
  }
  b->graph = g;
  b->key = key;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_step(xslam_batch_t b, const float* const* depths) {
  if (!b) return XSLAM_EINVAL;
  if (!depths) return bfail(b, XSLAM_EINVAL, "depths is NULL");
  std::vector<int> key(b->n, 0);
  int active = 0;
  for (int i = 0; i < b->n; ++i)
    if (depths[i]) {
      key[i] = b->hs[i]->frame == 0 ? 1 : 2;
      ++active;
    }
  if (!active) return bfail(b, XSLAM_EINVAL, "no trajectory has a frame this step");
  if (key != b->key) {
    xslam_status st = build_graph(b, key);
    if (st != XSLAM_OK) return st;
  }
  // the source table of this step: a pinned slot that no earlier copy still reads
  const int r = b->slot;
  b->slot = (b->slot + 1) % kRing;
  BCU(cudaEventSynchronize(b->ev_slot[r]));
  for (int i = 0; i < b->n; ++i) b->h_src[r][i] = depths[i];
  BCU(cudaEventRecord(b->ev_in, b->user));
  BCU(cudaStreamWaitEvent(b->s, b->ev_in, 0));
  BCU(cudaMemcpyAsync(b->d_src, b->h_src[r], sizeof(float*) * b->n, cudaMemcpyHostToDevice, b->s));
  BCU(cudaEventRecord(b->ev_slot[r], b->s));
  BCU(cudaGraphLaunch(b->exec, b->s));
  BCU(cudaEventRecord(b->ev_out, b->s));
  BCU(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  b->last.clear();
  for (int i = 0; i < b->n; ++i)
    if (key[i]) {
      b->hs[i]->frame += 1;
      b->last.push_back(i);
    }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_sync(xslam_batch_t b, int* n_failed) {
  if (!b) return XSLAM_EINVAL;
  BCU(cudaStreamSynchronize(b->s));
  if (n_failed)
    for (int i = 0; i < b->n; ++i) {
      int st[4];
      BCU(cudaMemcpy(st, b->hs[i]->b.status, sizeof(st), cudaMemcpyDeviceToHost));
      n_failed[i] = st[1];
    }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_read(xslam_batch_t b, int i, double* pose_out, double* dpose_out,
                                         double* dtwist_out) {
  if (!b) return XSLAM_EINVAL;
  if (i < 0 || i >= b->n) return bfail(b, XSLAM_EINVAL, "trajectory index out of range");
  BCU(cudaStreamSynchronize(b->s));
  xslam_t h = b->hs[i];
  std::vector<double> r(kResSys);
  BCU(cudaMemcpy(r.data(), h->b.result, sizeof(double) * kResSys, cudaMemcpyDeviceToHost));
  if (pose_out) memcpy(pose_out, r.data(), sizeof(double) * 12);
  for (int j = 0; j < h->K; ++j) {
    if (dpose_out) memcpy(dpose_out + 12 * j, r.data() + 12 + 12 * j, sizeof(double) * 12);
    if (dtwist_out) memcpy(dtwist_out + 6 * j, r.data() + 12 + 12 * (kMaxLanes - 1) + 6 * j, sizeof(double) * 6);
  }
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_latency(xslam_batch_t b, float* ms) {
  if (!b || !ms) return bfail(b, XSLAM_EINVAL, "NULL argument");
  BCU(cudaStreamSynchronize(b->s));
  for (int i = 0; i < b->n; ++i) ms[i] = 0.f;
  for (int i : b->last) BCU(cudaEventElapsedTime(&ms[i], b->ev_start, b->ev_done[i]));
  return XSLAM_OK;
}

// every handle back to frame 0: empty volume, the lanes and the pose recorded at create
static xslam_status restore_all(xslam_batch_t b) {
  BCU(cudaStreamSynchronize(b->s));
  for (int i = 0; i < b->n; ++i) {
    xslam_t h = b->hs[i];
    xslam_status st = xslam_reset(h);
    if (st == XSLAM_OK) st = xslam_set_lanes(h, b->seeds[i].data(), (int)b->seeds[i].size());
    if (st == XSLAM_OK) st = xslam_set_pose(h, b->pose0[i].data());
    if (st != XSLAM_OK) return bfail(b, st, std::string("restoring a handle failed: ") + h->err);
  }
  drop_graph(b);
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_autotune(xslam_batch_t b, const float* const* frames, int steps, int* divisor,
                                             float* ms_per_step) {
  if (!b) return XSLAM_EINVAL;
  if (!frames || !divisor) return bfail(b, XSLAM_EINVAL, "NULL argument");
  if (steps < 3) return bfail(b, XSLAM_EINVAL, "steps must be >= 3 (two untimed steps, then timed tracking steps)");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  BCU(cudaEventCreate(&t0));
  BCU(cudaEventCreate(&t1));
  float best = 0.f;
  int best_d = 1;
  xslam_status st = XSLAM_OK;
  for (int c = 0; c < 5 && st == XSLAM_OK; ++c) {
    const int d = kDivisors[c];
    for (int i = 0; i < b->n; ++i) {
      for (int l = 0; l < 3; ++l) b->hs[i]->nblk[l] = std::max(1, b->nblk0[i][l] / d);
      handle_drop_graphs(b->hs[i]);
    }
    if ((st = restore_all(b)) != XSLAM_OK) break;
    // steps 0 and 1 are untimed: they capture the frame-0 and the tracking graphs (host work); the
    // tracking steps 2.. are timed
    for (int s = 0; s < 2 && st == XSLAM_OK; ++s) st = xslam_batch_step(b, frames + (size_t)s * b->n);
    if (st != XSLAM_OK) break;
    cudaEventRecord(t0, b->s);
    for (int s = 2; s < steps && st == XSLAM_OK; ++s) st = xslam_batch_step(b, frames + (size_t)s * b->n);
    cudaEventRecord(t1, b->s);
    if (st != XSLAM_OK) break;
    if (cudaEventSynchronize(t1) != cudaSuccess) {
      st = bfail(b, XSLAM_ECUDA, "autotune timing failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    ms /= (steps - 2);
    if (ms_per_step) ms_per_step[c] = ms;
    if (c == 0 || ms < best) {
      best = ms;
      best_d = d;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != XSLAM_OK) return st;
  for (int i = 0; i < b->n; ++i) {
    for (int l = 0; l < 3; ++l) b->hs[i]->nblk[l] = std::max(1, b->nblk0[i][l] / best_d);
    handle_drop_graphs(b->hs[i]);
  }
  if ((st = restore_all(b)) != XSLAM_OK) return st;
  *divisor = best_d;
  return XSLAM_OK;
}

extern "C" const char* xslam_batch_last_error(xslam_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
