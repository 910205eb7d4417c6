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
constexpr int kTuneMax = 15;    // autotuner candidates at most: 2 modes, 6 ICP divisors, 4 fusion grids, 3 tiles

}  // namespace

struct xslam_batch_s {
  int n = 0;
  std::vector<xslam_t> hs;
  std::vector<std::vector<xslam_seed>> seeds;      // lanes recorded at create
  std::vector<std::array<double, 12>> pose0;       // frame-0 pose recorded at create
  std::vector<std::array<int, 3>> nblk0;           // default ICP grids
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
  // segmented mode: every stage is one launch over all active trajectories (see build_graph_seg);
  // possible when every handle runs the plain frame chain (seg_ok), chosen by the autotuner
  bool segmented = false, seg_ok = false;
  TrajDesc* d_desc = nullptr;                      // the trajectories' parameters and buffers (device)
  Seg* d_seg = nullptr;                            // the segment tables of the current graph (device)
  size_t seg_cap = 0;
  int fuse_per_sm = 0;                             // fusion blocks per SM of each trajectory (0: default)
  int ray_tile = 0;                                // ray-cast block: 0 = 32 x 8, 1 = 16 x 16, 2 = 64 x 4
  // launch profile of the segmented step (xslam_batch_profile): an event after every launch
  bool prof = false;
  std::vector<cudaEvent_t> ev_plan;
  std::vector<std::array<int, 3>> plan_info;       // kind, argument, blocks of every launch of the graph
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
  for (int r = 0; r < kRing; ++r) {
    if (b->h_src[r]) cudaFreeHost(b->h_src[r]);
    if (b->ev_slot[r]) cudaEventDestroy(b->ev_slot[r]);
  }
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_done)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_plan)
    if (e) cudaEventDestroy(e);
  cudaFree(b->d_src);
  cudaFree(b->d_dst);
  cudaFree(b->d_cnt);
  cudaFree(b->d_desc);
  cudaFree(b->d_seg);
  for (cudaEvent_t e : {b->ev_in, b->ev_out, b->ev_fork, b->ev_start})
    if (e) cudaEventDestroy(e);
  if (b->s) cudaStreamDestroy(b->s);
}

static bool plain_chain(xslam_t h);
static void apply_shapes(xslam_batch_t b, int div, int fuse_per_sm, int tile, int mode);

extern "C" xslam_status xslam_batch_create(xslam_batch_t* out, int n, xslam_t const* handles, void* cuda_stream) {
  xslam_batch_t b = nullptr;
  if (!out || !handles) return bfail(b, XSLAM_EINVAL, "NULL argument");
  *out = nullptr;
  if (n < 1 || n > kMaxBatch) return bfail(b, XSLAM_EINVAL, "n must be in 1..256");
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return bfail(b, XSLAM_EINVAL, "a handle is NULL");
    if (handles[i]->frame != 0) return bfail(b, XSLAM_EINVAL, "every handle must be before its first frame");
    if (handles[i]->profiling) return bfail(b, XSLAM_EINVAL, "stage profiling must be off in a batch");
    if (handles[i]->in_batch) return bfail(b, XSLAM_EINVAL, "a handle is already in a batch");
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
  ok = ok && cudaMalloc(&b->d_desc, sizeof(TrajDesc) * n) == cudaSuccess;
  if (!ok) return cleanup(XSLAM_ENOMEM, "stream, event or allocation failed");
  // one launch per stage for the whole batch when every handle runs the plain frame chain
  b->seg_ok = true;
  for (int i = 0; i < n; ++i) b->seg_ok = b->seg_ok && plain_chain(handles[i]);
  b->segmented = b->seg_ok;
  std::vector<float*> dst(n);
  std::vector<int> cnt(n);
  for (int i = 0; i < n; ++i) {
    xslam_t h = b->hs[i];
    dst[i] = h->b.depth_in;
    cnt[i] = h->p.W * h->p.H;
    b->max_hw = std::max(b->max_hw, cnt[i]);
    b->seeds.emplace_back(h->seeds, h->seeds + h->K);
    b->nblk0.push_back({h->nblk[0], h->nblk[1], h->nblk[2]});
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
  for (xslam_t h : b->hs) h->in_batch = true;
  *out = b;
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_destroy(xslam_batch_t b) {
  if (!b) return XSLAM_OK;
  free_batch(b);
  // the handles get back their own ICP grids (the autotuner may have changed them)
  for (int i = 0; i < b->n; ++i) {
    xslam_t h = b->hs[i];
    for (int l = 0; l < 3; ++l) h->nblk[l] = b->nblk0[i][l];
    handle_drop_graphs(h);
    h->in_batch = false;
  }
  delete b;
  return XSLAM_OK;
}

// The frame chain the segmented launches reproduce: Gauss-Newton ICP with fixed iteration counts from
// the previous pose, and lanes that need no per-frame kernels of their own (POSE0, TRUNC, DEPTH on every
// pixel). Other handles (learned proposal, Newton ICP, a stop tolerance, a constant-velocity start,
// per-frame pose or single-pixel DEPTH seeds) run their own chains as graph branches.
static bool plain_chain(xslam_t h) {
  if (h->mlp || h->cfg.icp_newton || h->cfg.icp_stop > 0.f || h->cfg.icp_seed != 0 || h->p.fresh) return false;
  for (int l = 1; l < h->p.L; ++l)
    if (h->p.dpix[l] >= 0) return false;
  return true;
}

// one segmented launch of the step: its kind, stage argument and its segments [off, off + cnt)
struct SegPlan {
  enum Kind { kPrepare, kSeed, kIcp, kFuseTiles, kIntegrate, kRaycast, kReadout } kind;
  int arg;  // prepare: stage; ICP: the largest lane count; integrate: lane count; raycast: tile
  size_t off, cnt;
  int nblocks;
};

static xslam_status build_graph_seg(xslam_batch_t b, const std::vector<int>& key) {
  drop_graph(b);
  const int n = b->n;
  std::vector<TrajDesc> desc(n);
  for (int i = 0; i < n; ++i) desc[i] = {b->hs[i]->p, b->hs[i]->b, b->hs[i]->d_kinds, b->hs[i]->d_index};
  BCU(cudaMemcpy(b->d_desc, desc.data(), sizeof(TrajDesc) * n, cudaMemcpyHostToDevice));
  std::vector<Seg> segs;
  std::vector<SegPlan> plans;
  int sms = 148, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // a launch over the trajectories `who` with grid(i) blocks each (and a per-segment argument)
  auto plan = [&](SegPlan::Kind k, int arg, const std::vector<int>& who, auto grid, auto sarg) {
    if (who.empty()) return;
    SegPlan pl{k, arg, segs.size(), who.size(), 0};
    for (int i : who) {
      const int g = grid(i);
      segs.push_back(Seg{i, pl.nblocks, g, sarg(i)});
      pl.nblocks += g;
    }
    plans.push_back(pl);
  };
  auto zero = [](int) { return 0; };
  std::vector<int> all, first, track;
  int max_levels = 1;
  for (int i = 0; i < n; ++i) {
    if (!key[i]) continue;
    all.push_back(i);
    (key[i] == 1 ? first : track).push_back(i);
    if (key[i] == 2) max_levels = std::max(max_levels, b->hs[i]->cfg.icp_levels);
  }
  // measurement: range gate, bilateral filter, pyramid levels (tracking trajectories)
  plan(SegPlan::kPrepare, 0, all, [&](int i) { return (b->hs[i]->p.W * b->hs[i]->p.H + 255) / 256; }, zero);
  std::vector<int> filt;
  for (int i : all)
    if (b->hs[i]->p.bilateral) filt.push_back(i);
  auto gx2 = [&](int i, int l) { return ((b->hs[i]->p.W >> l) + 31) / 32; };
  auto gy2 = [&](int i, int l) { return ((b->hs[i]->p.H >> l) + 7) / 8; };
  plan(SegPlan::kPrepare, 1, filt, [&](int i) { return gx2(i, 0) * gy2(i, 0); }, [&](int i) { return gx2(i, 0); });
  for (int l = 1; l < max_levels; ++l) {
    std::vector<int> who;
    for (int i : track)
      if (b->hs[i]->cfg.icp_levels > l) who.push_back(i);
    plan(SegPlan::kPrepare, 1 + l, who, [&](int i) { return gx2(i, l) * gy2(i, l); }, [&](int i) { return gx2(i, l); });
  }
  plan(SegPlan::kSeed, 0, first, [](int) { return 1; }, zero);
  // ICP: iteration g of every tracking trajectory that has one (each with its own level and flags)
  std::vector<std::vector<int>> sched(n);
  size_t max_it = 0;
  for (int i : track) {
    const xslam_config& c = b->hs[i]->cfg;
    int last_level = -1;
    for (int l = c.icp_levels - 1; l >= 0; --l)
      if (c.icp_iters[l] > 0) last_level = l;
    for (int l = c.icp_levels - 1; l >= 0; --l)
      for (int it = 0; it < c.icp_iters[l]; ++it) {
        int flags = it == 0 ? kIcpFirst : 0;
        if (l == last_level && it == c.icp_iters[l] - 1) flags |= kIcpLast;
        sched[i].push_back(l | (flags << 4));
      }
    max_it = std::max(max_it, sched[i].size());
  }
  for (size_t g = 0; g < max_it; ++g) {
    std::vector<int> who;
    for (int i : track)
      if (sched[i].size() > g) who.push_back(i);
    int max_lanes = 1;  // sizes the launch's dynamic shared memory
    for (int i : who) max_lanes = std::max(max_lanes, b->hs[i]->p.L);
    plan(SegPlan::kIcp, max_lanes, who, [&](int i) { return b->hs[i]->nblk[sched[i][g] & 15]; },
         [&](int i) { return sched[i][g]; });
  }
  // fusion: the tile lists, then the update grouped by lane count
  plan(SegPlan::kFuseTiles, 0, all, [&](int i) { return fuse_tiles_grid(b->hs[i]->p); }, zero);
  for (int L = 1; L <= kMaxLanes; ++L) {
    std::vector<int> who;
    for (int i : all)
      if (b->hs[i]->p.L == L) who.push_back(i);
    plan(SegPlan::kIntegrate, L, who,
         [&](int i) {
           const int def = integrate_grid(b->hs[i]->p);
           return b->fuse_per_sm > 0 ? std::max(1, std::min(fuse_tile_count(b->hs[i]->p), b->fuse_per_sm * sms)) : def;
         },
         zero);
  }
  // ray cast and read-out
  const int tw = b->ray_tile == 1 ? 16 : (b->ray_tile == 2 ? 64 : 32), th = 256 / tw;
  plan(SegPlan::kRaycast, b->ray_tile, all,
       [&](int i) { return ((b->hs[i]->p.W + tw - 1) / tw) * ((b->hs[i]->p.H + th - 1) / th); },
       [&](int i) { return (b->hs[i]->p.W + tw - 1) / tw; });
  plan(SegPlan::kReadout, 1, all, [](int) { return 1; }, zero);
  if (segs.size() > b->seg_cap) {
    cudaFree(b->d_seg);
    b->d_seg = nullptr;
    b->seg_cap = 0;
    BCU(cudaMalloc(&b->d_seg, sizeof(Seg) * segs.size()));
    b->seg_cap = segs.size();
  }
  BCU(cudaMemcpy(b->d_seg, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice));
  b->plan_info.clear();
  for (const SegPlan& pl : plans) b->plan_info.push_back({(int)pl.kind, pl.arg, pl.nblocks});
  if (b->prof)
    while (b->ev_plan.size() < plans.size()) {
      cudaEvent_t ev = nullptr;
      BCU(cudaEventCreate(&ev));
      b->ev_plan.push_back(ev);
    }

  BCU(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecordWithFlags(b->ev_start, b->s, cudaEventRecordExternal);
  if (e == cudaSuccess) {
    const int gx = std::max(1, std::min(64, (b->max_hw + 255) / 256));
    k_gather_frames<<<dim3(gx, n), 256, 0, b->s>>>(b->d_src, b->d_dst, b->d_cnt, n);
    e = cudaGetLastError();
  }
  for (size_t q = 0; q < plans.size() && e == cudaSuccess; ++q) {
    const SegPlan& pl = plans[q];
    const SegTable t{b->d_desc, b->d_seg + pl.off, (int)pl.cnt};
    switch (pl.kind) {
      case SegPlan::kPrepare: e = launch_prepare_seg(t, pl.nblocks, pl.arg, b->s); break;
      case SegPlan::kSeed: e = launch_lanes_seg(t, 0, b->s); break;
      case SegPlan::kIcp: e = launch_icp_seg(t, pl.nblocks, pl.arg, b->s); break;
      case SegPlan::kFuseTiles: e = launch_fuse_tiles_seg(t, pl.nblocks, b->s); break;
      case SegPlan::kIntegrate: e = launch_integrate_seg(t, pl.nblocks, pl.arg, b->s); break;
      case SegPlan::kRaycast: e = launch_raycast_seg(t, pl.nblocks, tw, b->s); break;
      case SegPlan::kReadout: e = launch_lanes_seg(t, 1, b->s); break;
    }
    if (e == cudaSuccess && b->prof) e = cudaEventRecordWithFlags(b->ev_plan[q], b->s, cudaEventRecordExternal);
  }
  // every trajectory's frame ends with the read-out launch
  for (int i : all)
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev_done[i], b->s, cudaEventRecordExternal);
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

static xslam_status build_graph(xslam_batch_t b, const std::vector<int>& key) {
  if (b->segmented) return build_graph_seg(b, key);
  drop_graph(b);
  b->plan_info.clear();
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

extern "C" xslam_status xslam_batch_set_shapes(xslam_batch_t b, const int* choice) {
  if (!b) return XSLAM_EINVAL;
  if (!choice) return bfail(b, XSLAM_EINVAL, "NULL argument");
  const int div = choice[0], fps = choice[1], tile = choice[2], mode = choice[3];
  if (div < 1 || fps < 0 || fps > 32 || tile < 0 || tile > 2 || mode < 0 || mode > 1)
    return bfail(b, XSLAM_EINVAL, "shape out of range");
  BCU(cudaStreamSynchronize(b->s));
  apply_shapes(b, div, fps, tile, mode);
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_profile(xslam_batch_t b, int enable) {
  if (!b) return XSLAM_EINVAL;
  BCU(cudaStreamSynchronize(b->s));
  b->prof = enable != 0;
  drop_graph(b);
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_profile_read(xslam_batch_t b, int cap, int* kind, int* arg, int* blocks,
                                                 float* ms, int* n) {
  if (!b || !n || cap < 0) return bfail(b, XSLAM_EINVAL, "NULL argument or negative capacity");
  BCU(cudaStreamSynchronize(b->s));
  *n = 0;
  if (!b->prof || !b->exec || b->last.empty()) return XSLAM_OK;
  const int np = (int)b->plan_info.size();
  *n = np;
  for (int q = 0; q < np && q < cap; ++q) {
    if (kind) kind[q] = b->plan_info[q][0];
    if (arg) arg[q] = b->plan_info[q][1];
    if (blocks) blocks[q] = b->plan_info[q][2];
    if (ms) BCU(cudaEventElapsedTime(&ms[q], q ? b->ev_plan[q - 1] : b->ev_start, b->ev_plan[q]));
  }
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

// the launch shapes of a tuning candidate: ICP grids divided by div, fusion blocks per SM (0 = the
// default grid), ray-cast tile (0 = 32 x 8, 1 = 16 x 16, 2 = 64 x 4), mode (0 = segmented launches where
// possible, 1 = every trajectory's own chain as a graph branch)
static void apply_shapes(xslam_batch_t b, int div, int fuse_per_sm, int tile, int mode) {
  for (int i = 0; i < b->n; ++i) {
    for (int l = 0; l < 3; ++l) b->hs[i]->nblk[l] = std::max(1, b->nblk0[i][l] / div);
    handle_drop_graphs(b->hs[i]);
  }
  b->fuse_per_sm = fuse_per_sm;
  b->ray_tile = tile;
  b->segmented = b->seg_ok && mode == 0;
  drop_graph(b);
}

// steps 0 and 1 from frame 0 untimed (they build the graphs), steps 2.. timed: milliseconds per step
static xslam_status time_candidate(xslam_batch_t b, const float* const* frames, int steps, cudaEvent_t t0,
                                   cudaEvent_t t1, float* ms) {
  xslam_status st = restore_all(b);
  for (int s = 0; s < 2 && st == XSLAM_OK; ++s) st = xslam_batch_step(b, frames + (size_t)s * b->n);
  if (st != XSLAM_OK) return st;
  BCU(cudaEventRecord(t0, b->s));
  for (int s = 2; s < steps && st == XSLAM_OK; ++s) st = xslam_batch_step(b, frames + (size_t)s * b->n);
  if (st != XSLAM_OK) return st;
  BCU(cudaEventRecord(t1, b->s));
  BCU(cudaEventSynchronize(t1));
  BCU(cudaEventElapsedTime(ms, t0, t1));
  *ms /= (float)(steps - 2);
  return XSLAM_OK;
}

extern "C" xslam_status xslam_batch_autotune(xslam_batch_t b, const float* const* frames, int steps, int* choice,
                                             float* ms_per_step) {
  if (!b) return XSLAM_EINVAL;
  if (!frames || !choice) return bfail(b, XSLAM_EINVAL, "NULL argument");
  if (steps < 3) return bfail(b, XSLAM_EINVAL, "steps must be >= 3 (two untimed steps, then timed tracking steps)");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  BCU(cudaEventCreate(&t0));
  BCU(cudaEventCreate(&t1));
  // one coordinate at a time, each with the best choices of the coordinates before it: the mode, the ICP
  // divisor, then (segmented mode only) the fusion grid and the ray-cast tile
  int best[4] = {1, 0, 0, b->seg_ok ? 0 : 1};  // divisor, fusion blocks per SM, tile, mode
  const int order[4] = {3, 0, 1, 2};
  constexpr int kCands = 6;
  const int cands[4][kCands] = {{1, 2, 4, 8, 16, 32}, {0, 1, 2, 4, -1, -1}, {0, 1, 2, -1, -1, -1}, {0, 1, -1, -1, -1, -1}};
  xslam_status st = XSLAM_OK;
  int k = 0;
  for (int o = 0; o < 4 && st == XSLAM_OK; ++o) {
    const int coord = order[o];
    if (coord == 3 && !b->seg_ok) continue;        // branches only
    if ((coord == 1 || coord == 2) && best[3] != 0) continue;  // shapes of the segmented launches
    float best_ms = 0.f;
    for (int c = 0; c < kCands && st == XSLAM_OK; ++c) {
      const int v = cands[coord][c];
      if (v < 0) continue;
      int shape[4] = {best[0], best[1], best[2], best[3]};
      shape[coord] = v;
      apply_shapes(b, shape[0], shape[1], shape[2], shape[3]);
      float ms = 0.f;
      st = time_candidate(b, frames, steps, t0, t1, &ms);
      if (st != XSLAM_OK) break;
      if (ms_per_step) ms_per_step[k] = ms;
      ++k;
      if (c == 0 || ms < best_ms) {
        best_ms = ms;
        best[coord] = v;
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != XSLAM_OK) return st;
  apply_shapes(b, best[0], best[1], best[2], best[3]);
  if ((st = restore_all(b)) != XSLAM_OK) return st;
  for (int q = 0; q < 4; ++q) choice[q] = best[q];
  if (ms_per_step)
    for (int q = k; q < kTuneMax; ++q) ms_per_step[q] = 0.f;
  return XSLAM_OK;
}

extern "C" const char* xslam_batch_last_error(xslam_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
