// Serving loop: continuous batching of contact requests (ccm_submit / ccm_poll).
//
// Requests reference resident geometry and bring their own device poses,
// outputs and (for the gradient) cotangents.  A native scheduler thread packs
// the queued requests, first come first served, into waves bounded by a
// capacity fixed at start (pairs, groups, requests) that the context's HBM
// budget must hold.  Each wave runs one graph:
//   gather  (every request's poses / cotangents into the wave buffers),
//   forward (all units of the wave, heaviest first),
//   reverse (units of the requests that asked for the gradient) + reduction,
//   scatter (outputs back into every request's buffers).
// The kernels read the wave's counts from device memory, so the graph of each
// of the two buffer sets is captured once and replayed for every wave; while
// one wave runs on its stream, the scheduler forms and launches the next one on
// the other, so requests that arrive during a wave join the next one and the
// two waves overlap on the device.  The launch shape is fixed at start from the
// resident geometry, so a request's result does not depend on its wave mates.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ccm_host.h"
#include "ccm_launch.h"

namespace ccm {

struct ReqDesc {
  const float* pose_a;
  const float* pose_b;
  float* y;
  const float* ybar;   // NULL: forward only
  float* grad;
  int64_t pair0, n, goff0, G;
  int64_t e_in, e_out;   // first element of this request in the wave's gather / scatter
};

struct WaveCounts {
  int64_t n_pairs, n_items_f, n_items_b, n_req;
  int64_t e_in, e_out;   // elements gathered / scattered in total
  int64_t n_pairs_b;     // pairs of the gradient requests (per-pair reverse pass)
};

// Cost class of a work item: four classes per octave of its estimated cost.
constexpr int kCostClasses = 256;
static inline uint8_t cost_class(int64_t cost) {
  if (cost < 1) return 0;
  const int e = 63 - __builtin_clzll((unsigned long long)cost);
  const int frac = e >= 2 ? (int)((cost >> (e - 2)) & 3) : (int)((cost << (2 - e)) & 3);
  return (uint8_t)std::min(kCostClasses - 1, 4 * e + frac);
}

struct Pending {
  uint64_t ticket;
  std::vector<PairRec> pairs;     // goff relative to the request
  std::vector<WorkItem> items;    // units relative to the request's first pair
  std::vector<uint8_t> cls;       // cost class per item (see cost_class)
  std::vector<uint8_t> pcls;      // cost class per pair (sum of its items' costs)
  std::vector<int64_t> item_off;  // [n + 1], from 0
  ReqDesc d;
  double t_submit = 0.0;
};

enum TicketState { kQueued = 0, kRunning = 1, kDone = 2 };

struct TicketInfo {
  TicketState state;
  double t_submit, t_done;
};

struct Serving;

struct WaveSet {
  Serving* owner = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;            // end of the wave's graph
  cudaEvent_t t0 = nullptr;              // start of the wave's graph
  cudaGraphExec_t graph_f = nullptr;    // gather, forward, scatter
  cudaGraphExec_t graph_fb = nullptr;   // gather, forward, reverse pass, scatter
  DevBuf d_pairs, d_items, d_order_f, d_order_b, d_item_off, d_porder, d_reqs, d_counts, d_pose_a,
      d_pose_b, d_y, d_ybar, d_part, d_grad, d_saved, d_sched;
  PairRec* h_pairs = nullptr;
  WorkItem* h_items = nullptr;
  int32_t* h_order_f = nullptr;
  int32_t* h_order_b = nullptr;
  int64_t* h_item_off = nullptr;
  int32_t* h_porder = nullptr;
  ReqDesc* h_reqs = nullptr;
  WaveCounts* h_counts = nullptr;
  std::vector<uint64_t> tickets;
  bool busy = false;       // a wave is in flight
  bool finished = false;   // its completion callback ran (Serving::mu)
};

struct Serving {
  Context* ctx = nullptr;
  ccm_serve_config cfg{};
  KParams kp{};
  UnitShape us{};
  int fwd_grid = 1, bwd_grid = 1, bwd_pair_grid = 1;
  int64_t cap_pairs = 0, cap_groups = 0, cap_req = 0, cap_items = 0;
  BatchMaxima mx;                  // largest pieces the launch shape holds
  bool per_pair = false;           // per-pair reverse pass (every body <= kHitS pieces)
  std::vector<int8_t> fit_cache;   // per body: -1 unknown, 0 no, 1 yes (ctx->mu held)
  std::vector<std::vector<PieceChunk>> chunk_cache;   // per body, under `us` (ctx->mu held)
  WaveSet sets[2];
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  bool held = false;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, TicketInfo> tickets;
  std::deque<uint64_t> completed;   // done, in completion order, until retired
  uint64_t next_ticket = 1;
  int64_t queued_pairs = 0;         // body pairs of the queued requests
  ccm_serve_counters counters{};
  cudaError_t async_error = cudaSuccess;

  // A body fits when no piece of it exceeds the per-piece budgets; larger
  // bodies (more pieces or planes) are chunked by the kernels as usual.
  bool fits(const Context& c, int32_t b) {
    if ((size_t)b >= fit_cache.size()) fit_cache.resize(c.bodies.size(), -1);
    if (fit_cache[b] < 0) {
      const BatchMaxima m = body_maxima(c, b);
      fit_cache[b] = m.vmax <= mx.vmax && m.fmax <= mx.fmax && m.emax <= mx.emax &&
                     (!per_pair || m.s_pieces <= kHitS);
    }
    return fit_cache[b] == 1;
  }

  // A body's feature-piece chunks under the serving shape, computed once: a
  // submission then builds its items from a few chunks per pair side instead
  // of walking every piece.
  const std::vector<PieceChunk>& chunks(const Context& c, int32_t b) {
    if ((size_t)b >= chunk_cache.size()) chunk_cache.resize(c.bodies.size());
    std::vector<PieceChunk>& v = chunk_cache[b];
    if (v.empty()) body_chunks(c, b, us, &v);
    return v;
  }
};

// Longest wait of a queued request for a running wave before a second,
// overlapping wave is launched for it (seconds).
constexpr double kSecondWaveWait = 0.25e-3;

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// gather / scatter kernels (counts read on device)
// ---------------------------------------------------------------------------
// Request owning element i of a wave's flattened copy (offsets ascending).
__device__ __forceinline__ int64_t owner_of(const ReqDesc* __restrict__ reqs, int64_t nr,
                                            int64_t i, bool in) {
  int64_t lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if ((in ? reqs[mid].e_in : reqs[mid].e_out) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Copies every request's poses (24 floats per pair) and, for gradient
// requests, cotangents (8 per group) into the wave buffers: one element per
// thread over the whole wave, so large and small requests copy alike.
__global__ void serve_gather(const ReqDesc* __restrict__ reqs, const WaveCounts* __restrict__ wc,
                             float* __restrict__ pose_a, float* __restrict__ pose_b,
                             float* __restrict__ ybar) {
  const int64_t nr = wc->n_req, total = wc->e_in;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ReqDesc& d = reqs[owner_of(reqs, nr, i, true)];
    int64_t j = i - d.e_in;
    if (j < 12 * d.n) { pose_a[12 * d.pair0 + j] = d.pose_a[j]; continue; }
    j -= 12 * d.n;
    if (j < 12 * d.n) { pose_b[12 * d.pair0 + j] = d.pose_b[j]; continue; }
    j -= 12 * d.n;
    ybar[8 * d.goff0 + j] = d.ybar[j];
  }
}

// Copies the outputs (8 floats per group) and, for gradient requests, the
// gradients (12 per pair) back into every request's buffers.
__global__ void serve_scatter(const ReqDesc* __restrict__ reqs, const WaveCounts* __restrict__ wc,
                              const float* __restrict__ y, const float* __restrict__ grad) {
  const int64_t nr = wc->n_req, total = wc->e_out;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ReqDesc& d = reqs[owner_of(reqs, nr, i, false)];
    int64_t j = i - d.e_out;
    if (j < 8 * d.G) { d.y[j] = y[8 * d.goff0 + j]; continue; }
    j -= 8 * d.G;
    d.grad[j] = grad[12 * d.pair0 + j];
  }
}

// ---------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------
template <class T>
static ccm_status alloc_buf(DevBuf& b, int64_t count, const char* what) {
  const size_t bytes = (size_t)std::max<int64_t>(1, count) * sizeof(T);
  cudaError_t e = cudaMalloc(&b.ptr, bytes);
  if (e != cudaSuccess) return fail(CCM_ERR_OOM, "%s: cudaMalloc(%zu): %s", what, bytes,
                                    cudaGetErrorString(e));
  b.bytes = bytes;
  return CCM_OK;
}

// Device bytes of one wave buffer set (setup_set allocates exactly these):
// per pair the pair record, item offset, two poses and the gradient; per work
// item its record, two order entries and its reverse-pass slot; per group the
// outputs and cotangents.
constexpr int64_t kBytesPerPair = (int64_t)sizeof(PairRec) + 8 + 4 + 2 * 12 * 4 + 12 * 4;
constexpr int64_t kBytesPerItem = (int64_t)sizeof(WorkItem) + 2 * 4 + 24 * 4;
constexpr int64_t kBytesPerGroup = 2 * 8 * 4 + CCM_SAVED_FLOATS * 4;

static int64_t set_bytes(int64_t P, int64_t G, int64_t R, int64_t I) {
  return P * kBytesPerPair + 8 + I * kBytesPerItem + G * kBytesPerGroup +
         R * (int64_t)sizeof(ReqDesc) + (int64_t)sizeof(WaveCounts);
}

static void launch_wave_graph(Serving* sv, WaveSet& s, bool reverse) {
  const WaveCounts* wc = static_cast<const WaveCounts*>(s.d_counts.ptr);
  const ReqDesc* reqs = static_cast<const ReqDesc*>(s.d_reqs.ptr);
  serve_gather<<<sv->ctx->n_sm * 4, 256, 0, s.stream>>>(
      reqs, wc, static_cast<float*>(s.d_pose_a.ptr), static_cast<float*>(s.d_pose_b.ptr),
      static_cast<float*>(s.d_ybar.ptr));
  count_launch();
  FwdLaunch F;
  F.g = sv->ctx->dev_geom();
  F.pairs = static_cast<const PairRec*>(s.d_pairs.ptr);
  F.items = static_cast<const WorkItem*>(s.d_items.ptr);
  F.order = static_cast<const int32_t*>(s.d_order_f.ptr);
  F.n_items = sv->cap_items;
  F.dev_items = &static_cast<const int64_t*>(s.d_counts.ptr)[1];
  F.pose_a = static_cast<const float*>(s.d_pose_a.ptr);
  F.pose_b = static_cast<const float*>(s.d_pose_b.ptr);
  F.kp = sv->kp;
  F.us = sv->us;
  F.y = static_cast<float*>(s.d_y.ptr);
  F.saved = reverse ? static_cast<float*>(s.d_saved.ptr) : nullptr;
  F.counters = nullptr;
  F.sched = static_cast<int*>(s.d_sched.ptr);
  F.grid = sv->fwd_grid;
  launch_forward(F, s.stream);
  BwdLaunch B;
  B.g = F.g;
  B.pairs = F.pairs;
  B.items = F.items;
  B.order = static_cast<const int32_t*>(s.d_order_b.ptr);
  B.n_items = sv->cap_items;
  B.item_off = static_cast<const int64_t*>(s.d_item_off.ptr);
  B.n_pairs = sv->cap_pairs;
  B.dev_items = &static_cast<const int64_t*>(s.d_counts.ptr)[2];
  B.dev_pairs = &static_cast<const int64_t*>(s.d_counts.ptr)[sv->per_pair ? 6 : 0];
  B.pair_order = sv->per_pair ? static_cast<const int32_t*>(s.d_porder.ptr) : nullptr;
  B.pose_a = F.pose_a;
  B.pose_b = F.pose_b;
  B.ybar = static_cast<const float*>(s.d_ybar.ptr);
  B.dir = nullptr;
  B.saved = static_cast<const float*>(s.d_saved.ptr);
  B.kp = sv->kp;
  B.us = sv->us;
  B.part = static_cast<float*>(s.d_part.ptr);
  B.grad = static_cast<float*>(s.d_grad.ptr);
  B.hvp = nullptr;
  B.jvp = nullptr;
  B.counters = nullptr;
  B.sched = static_cast<int*>(s.d_sched.ptr) + 1;
  B.grid = sv->bwd_grid;
  B.pair_grid = sv->bwd_pair_grid;
  if (reverse) launch_backward(B, s.stream);
  serve_scatter<<<sv->ctx->n_sm * 4, 256, 0, s.stream>>>(
      reqs, wc, static_cast<const float*>(s.d_y.ptr), static_cast<const float*>(s.d_grad.ptr));
  count_launch();
}

static ccm_status setup_set(Serving* sv, WaveSet& s) {
  const int64_t P = sv->cap_pairs, G = sv->cap_groups, R = sv->cap_req, I = sv->cap_items;
  ccm_status st;
  if ((st = alloc_buf<PairRec>(s.d_pairs, P, "wave pairs")) != CCM_OK) return st;
  if ((st = alloc_buf<WorkItem>(s.d_items, I, "wave items")) != CCM_OK) return st;
  if ((st = alloc_buf<int32_t>(s.d_order_f, I, "wave order")) != CCM_OK) return st;
  if ((st = alloc_buf<int32_t>(s.d_order_b, I, "wave order")) != CCM_OK) return st;
  if ((st = alloc_buf<int64_t>(s.d_item_off, P + 1, "wave item offsets")) != CCM_OK) return st;
  if ((st = alloc_buf<int32_t>(s.d_porder, P, "wave pair order")) != CCM_OK) return st;
  if ((st = alloc_buf<ReqDesc>(s.d_reqs, R, "wave requests")) != CCM_OK) return st;
  if ((st = alloc_buf<WaveCounts>(s.d_counts, 1, "wave counts")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_pose_a, 12 * P, "wave poses")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_pose_b, 12 * P, "wave poses")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_y, 8 * G, "wave outputs")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_ybar, 8 * G, "wave cotangents")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_saved, CCM_SAVED_FLOATS * G, "wave records")) != CCM_OK) return st;
  if ((st = alloc_buf<int32_t>(s.d_sched, 2, "wave work counters")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_part, 24 * I, "wave slots")) != CCM_OK) return st;
  if ((st = alloc_buf<float>(s.d_grad, 12 * P, "wave gradients")) != CCM_OK) return st;
  if (cudaMallocHost(&s.h_pairs, sizeof(PairRec) * P) != cudaSuccess ||
      cudaMallocHost(&s.h_items, sizeof(WorkItem) * I) != cudaSuccess ||
      cudaMallocHost(&s.h_order_f, 4 * I) != cudaSuccess ||
      cudaMallocHost(&s.h_order_b, 4 * I) != cudaSuccess ||
      cudaMallocHost(&s.h_item_off, 8 * (P + 1)) != cudaSuccess ||
      cudaMallocHost(&s.h_porder, 4 * P) != cudaSuccess ||
      cudaMallocHost(&s.h_reqs, sizeof(ReqDesc) * R) != cudaSuccess ||
      cudaMallocHost(&s.h_counts, sizeof(WaveCounts)) != cudaSuccess)
    return fail(CCM_ERR_OOM, "pinned staging buffers");
  CCM_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "cudaStreamCreate");
  CCM_CUDA(cudaEventCreate(&s.done), "cudaEventCreate");
  CCM_CUDA(cudaEventCreate(&s.t0), "cudaEventCreate");
  // capture the wave once (with and without the reverse pass); every wave
  // replays one of them after uploading its tables
  for (int reverse = 0; reverse < 2; ++reverse) {
    cudaGraph_t g = nullptr;
    CCM_CUDA(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    launch_wave_graph(sv, s, reverse != 0);
    CCM_CUDA(cudaStreamEndCapture(s.stream, &g), "end capture");
    const cudaError_t e = cudaGraphInstantiate(reverse ? &s.graph_fb : &s.graph_f, g, 0);
    cudaGraphDestroy(g);
    CCM_CUDA(e, "graph instantiate");
  }
  s.owner = sv;
  return CCM_OK;
}

static void release_set(WaveSet& s) {
  if (s.stream) cudaStreamSynchronize(s.stream);   // no completion callback pending
  if (s.graph_f) cudaGraphExecDestroy(s.graph_f);
  if (s.graph_fb) cudaGraphExecDestroy(s.graph_fb);
  if (s.done) cudaEventDestroy(s.done);
  if (s.t0) cudaEventDestroy(s.t0);
  if (s.stream) cudaStreamDestroy(s.stream);
  for (DevBuf* b : {&s.d_pairs, &s.d_items, &s.d_order_f, &s.d_order_b, &s.d_item_off, &s.d_porder,
                    &s.d_reqs, &s.d_counts, &s.d_pose_a, &s.d_pose_b, &s.d_y, &s.d_ybar,
                    &s.d_part, &s.d_grad, &s.d_saved, &s.d_sched})
    b->release();
  for (void* p : {(void*)s.h_pairs, (void*)s.h_items, (void*)s.h_order_f, (void*)s.h_order_b,
                  (void*)s.h_item_off, (void*)s.h_porder, (void*)s.h_reqs, (void*)s.h_counts})
    if (p) cudaFreeHost(p);
  s = WaveSet();
}

// ---------------------------------------------------------------------------
// the scheduler
// ---------------------------------------------------------------------------
// Runs on a CUDA callback thread once a wave's graph has finished: flags the
// set and wakes the scheduler (no CUDA calls are allowed here).
static void CUDART_CB wave_finished(void* arg) {
  WaveSet* s = static_cast<WaveSet*>(arg);
  Serving* sv = s->owner;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    s->finished = true;
  }
  sv->cv.notify_all();
}

// Takes the queued requests that fit set `s` (mu held), then fills the set's
// tables and launches its graph with mu released, so that submissions and
// polls are not held up while a wave is formed.
static void launch_wave(Serving* sv, WaveSet& s, std::unique_lock<std::mutex>& lk) {
  std::vector<Pending> take;
  {
    int64_t P = 0, G = 0, I = 0;
    while (!sv->queue.empty()) {
      const Pending& q = sv->queue.front();
      const int64_t ni = (int64_t)q.items.size();
      if ((int64_t)take.size() + 1 > sv->cap_req || P + q.d.n > sv->cap_pairs ||
          G + q.d.G > sv->cap_groups || I + ni > sv->cap_items)
        break;
      P += q.d.n;
      G += q.d.G;
      I += ni;
      sv->tickets[q.ticket].state = kRunning;
      sv->queued_pairs -= q.d.n;
      take.push_back(std::move(sv->queue.front()));
      sv->queue.pop_front();
    }
  }
  if (take.empty()) return;
  const double t_form = now_s();
  s.busy = true;
  s.tickets.clear();
  for (const Pending& q : take) s.tickets.push_back(q.ticket);
  lk.unlock();

  // tables of the wave, and a counting sort of its items by cost class,
  // heaviest class first, index order within a class (two linear passes; a
  // request's results do not depend on this order)
  int64_t P = 0, G = 0, R = 0, I = 0, EI = 0, EO = 0;
  int64_t cnt_f[kCostClasses] = {0}, cnt_b[kCostClasses] = {0};
  s.h_item_off[0] = 0;
  for (const Pending& q : take) {
    const int64_t ni = (int64_t)q.items.size();
    ReqDesc d = q.d;
    d.pair0 = P;
    d.goff0 = G;
    d.e_in = EI;
    d.e_out = EO;
    EI += 24 * d.n + (d.ybar ? 8 * d.G : 0);
    EO += 8 * d.G + (d.ybar ? 12 * d.n : 0);
    s.h_reqs[R] = d;
    for (int64_t i = 0; i < q.d.n; ++i) {
      PairRec pr = q.pairs[i];
      pr.goff += G;
      s.h_pairs[P + i] = pr;
      s.h_item_off[P + i + 1] = I + q.item_off[i + 1];
    }
    const int32_t du = (int32_t)(2 * P);
    for (int64_t j = 0; j < ni; ++j) {
      WorkItem it = q.items[j];
      it.unit += du;
      s.h_items[I + j] = it;
      ++cnt_f[q.cls[j]];
      if (q.d.ybar) ++cnt_b[q.cls[j]];
    }
    P += q.d.n;
    G += q.d.G;
    I += ni;
    ++R;
  }
  int64_t nf = 0, nb = 0;
  for (int c = kCostClasses - 1; c >= 0; --c) {   // first slot of each class
    const int64_t a = cnt_f[c], b = cnt_b[c];
    cnt_f[c] = nf;
    cnt_b[c] = nb;
    nf += a;
    nb += b;
  }
  {
    int64_t base = 0;
    for (const Pending& q : take) {
      const int64_t ni = (int64_t)q.items.size();
      for (int64_t j = 0; j < ni; ++j) {
        const int c = q.cls[j];
        s.h_order_f[cnt_f[c]++] = (int32_t)(base + j);
        if (q.d.ybar) s.h_order_b[cnt_b[c]++] = (int32_t)(base + j);
      }
      base += ni;
    }
  }
  // the gradient requests' pairs by cost class, heaviest first
  int64_t npb = 0;
  {
    int64_t cnt_p[kCostClasses] = {0};
    for (const Pending& q : take)
      if (q.d.ybar)
        for (uint8_t c : q.pcls) ++cnt_p[c];
    for (int c = kCostClasses - 1; c >= 0; --c) {
      const int64_t a = cnt_p[c];
      cnt_p[c] = npb;
      npb += a;
    }
    int64_t base = 0;
    for (const Pending& q : take) {
      if (q.d.ybar)
        for (int64_t i = 0; i < q.d.n; ++i) s.h_porder[cnt_p[q.pcls[i]]++] = (int32_t)(base + i);
      base += q.d.n;
    }
  }
  *s.h_counts = WaveCounts{P, nf, nb, R, EI, EO, npb};
  cudaError_t e = cudaSuccess;
  auto copy = [&](void* dst, const void* src, size_t bytes) {
    if (bytes && e == cudaSuccess)
      e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s.stream);
  };
  copy(s.d_pairs.ptr, s.h_pairs, sizeof(PairRec) * P);
  copy(s.d_items.ptr, s.h_items, sizeof(WorkItem) * I);
  copy(s.d_item_off.ptr, s.h_item_off, 8 * (P + 1));
  copy(s.d_porder.ptr, s.h_porder, 4 * npb);
  copy(s.d_order_f.ptr, s.h_order_f, 4 * nf);
  copy(s.d_order_b.ptr, s.h_order_b, 4 * nb);
  copy(s.d_reqs.ptr, s.h_reqs, sizeof(ReqDesc) * R);
  copy(s.d_counts.ptr, s.h_counts, sizeof(WaveCounts));
  if (e == cudaSuccess) e = cudaEventRecord(s.t0, s.stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(nb == 0 ? s.graph_f : s.graph_fb, s.stream);
  if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, wave_finished, &s);
  lk.lock();
  if (e != cudaSuccess) {
    // nothing will call back: fail the wave's requests now
    if (sv->async_error == cudaSuccess) sv->async_error = e;
    s.finished = true;
  }
  sv->counters.waves += 1;
  sv->counters.wave_pairs += P;
  sv->counters.wave_items += I;
  sv->counters.form_s += now_s() - t_form;
}

static void worker_main(Serving* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    bool progressed = false;
    for (WaveSet& s : sv->sets) {
      if (!s.busy || !s.finished) continue;
      const cudaError_t q = cudaEventQuery(s.done);   // complete; reports async errors
      if (q != cudaSuccess && q != cudaErrorNotReady && sv->async_error == cudaSuccess)
        sv->async_error = q;
      const double t = now_s();
      for (uint64_t tk : s.tickets) {
        auto it = sv->tickets.find(tk);
        if (it != sv->tickets.end()) {
          it->second.state = kDone;
          it->second.t_done = t;
          sv->completed.push_back(tk);
        }
      }
      sv->counters.served += (int64_t)s.tickets.size();
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s.t0, s.done) == cudaSuccess) sv->counters.gpu_s += 1e-3 * ms;
      s.tickets.clear();
      s.busy = false;
      s.finished = false;
      progressed = true;
    }
    if (sv->stop) sv->held = false;   // stopping runs what is queued
    for (WaveSet& s : sv->sets) {
      if (s.busy || sv->held || sv->queue.empty()) continue;
      // With the other set's wave still running, a second wave goes out only
      // for a queue that fills half a wave, or whose oldest request has
      // waited kSecondWaveWait: otherwise the queue waits for the running
      // wave and leaves as one larger wave (fewer, larger waves under load,
      // no added wait on an idle loop).
      const bool other_busy = sv->sets[0].busy || sv->sets[1].busy;
      if (other_busy && !sv->stop && 2 * sv->queued_pairs < sv->cap_pairs &&
          now_s() - sv->queue.front().t_submit < kSecondWaveWait)
        continue;
      launch_wave(sv, s, lk);
      progressed = true;
    }
    const bool any_busy = sv->sets[0].busy || sv->sets[1].busy;
    if (sv->stop && sv->queue.empty() && !any_busy) break;
    // woken by a submit, a hold change, a stop or a wave's completion
    // callback; a queue held back for a running wave is looked at again
    // when its oldest request has waited kSecondWaveWait
    if (!progressed) {
      const bool waiting = !sv->queue.empty() && !sv->held;
      sv->cv.wait_for(lk, waiting ? std::chrono::microseconds(100)
                                  : std::chrono::microseconds(50000));
    }
  }
}

void Context::shutdown_serving() {
  if (!serving) return;
  {
    std::lock_guard<std::mutex> lk(serving->mu);
    serving->stop = true;
  }
  serving->cv.notify_all();
  if (serving->worker.joinable()) serving->worker.join();
  for (WaveSet& s : serving->sets) release_set(s);
  delete serving;
  serving = nullptr;
}

}  // namespace ccm

using namespace ccm;

extern "C" {

void ccm_default_serve_config(ccm_serve_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->max_wave_pairs = 1 << 14;
  c->max_wave_requests = 1024;
  c->max_queued = 1 << 16;
  ccm_default_params(&c->params);
  default_tuning(&c->tuning);
}

ccm_status ccm_serve_start(ccm_ctx ctx, const ccm_serve_config* cfg) {
  if (!ctx || !cfg) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  if (c->serving) return fail(CCM_ERR_INVALID, "serving already started");
  if (cfg->max_wave_pairs < 0 || cfg->max_wave_requests < 1 || cfg->max_queued < 1 ||
      cfg->max_wave_pairs > ((int64_t)1 << 26) || (cfg->max_wave_pairs == 0 && c->budget == 0))
    return fail(CCM_ERR_INVALID, "bad serving capacities");
  KParams kp;
  ccm_status st = make_kparams(&cfg->params, &kp);
  if (st != CCM_OK) return st;
  if (kp.flags & (CCM_FLAG_NO_CULL | CCM_FLAG_BODY_UNION | CCM_FLAG_PROJECT | CCM_FLAG_SPLINE))
    return fail(CCM_ERR_INVALID, "the serving loop runs the default method (no flags)");
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  // launch shape from every resident body, independent of any wave's mix
  std::vector<ccm_geom> all;
  int64_t max_np = 1;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (size_t b = 0; b < c->bodies.size(); ++b)
      if (c->alive[b]) {
        all.push_back((ccm_geom)(b + 1));
        max_np = std::max<int64_t>(max_np, c->bodies[b].np);
      }
  }
  if (all.empty()) return fail(CCM_ERR_INVALID, "no resident geometry");
  Serving* sv = new Serving();
  sv->ctx = c;
  sv->cfg = *cfg;
  sv->kp = kp;
  sv->cap_req = cfg->max_wave_requests;
  int64_t max_items = 1;   // most work items of one pair of resident bodies
  {
    Batch probe;   // one (b, b) pair per resident body: the maxima of all of them
    probe.ctx = c;
    probe.n = (int64_t)all.size();
    st = build_batch(c, probe.n, all.data(), all.data(), &probe);
    if (st == CCM_OK) st = apply_tuning(c, &probe, cfg->tuning);
    if (st != CCM_OK) {
      probe.release();
      delete sv;
      return st;
    }
    sv->mx = probe.mx;
    sv->us = probe.us;
    sv->per_pair = probe.mx.s_pieces <= kHitS;
    std::vector<WorkItem> items;
    std::vector<int64_t> cost, off(1, 0);
    {
      std::lock_guard<std::mutex> lk(c->mu);
      make_items(*c, probe.pairs.data(), probe.n, 0, sv->us, &items, &cost, &off);
    }
    for (int64_t k = 0; k < probe.n; ++k) max_items = std::max(max_items, off[k + 1] - off[k]);
    probe.release();
    // persistent grids: every resident warp slot of the device
    int per_sm = 1;
    BwdOccupancy occ{};
    cudaError_t e = configure_forward(sv->us, c->smem_optin, &per_sm);
    if (e == cudaSuccess) e = configure_backward(sv->us, c->smem_optin, &occ);
    if (e != cudaSuccess) {
      delete sv;
      return cuda_fail(e, "configure serving kernels");
    }
    sv->fwd_grid = c->n_sm * std::max(1, per_sm);
    const int k = sv->kp.trace_iters == 3 ? 1 : 0;   // waves run gradients only
    sv->bwd_grid = c->n_sm * std::max(1, occ.unit[0][k]);
    sv->bwd_pair_grid = c->n_sm * std::max(1, occ.pair[0][k]);
  }
  // per pair of the largest resident bodies: its record, items and groups
  const int64_t per_pair = kBytesPerPair + max_items * kBytesPerItem + 2 * max_np * kBytesPerGroup;
  if (cfg->max_wave_pairs > 0) {
    sv->cap_pairs = cfg->max_wave_pairs;
  } else {   // the largest wave whose two buffer sets fit the budget
    const int64_t fixed = set_bytes(0, 0, sv->cap_req, 0);
    sv->cap_pairs = std::min<int64_t>((int64_t)1 << 20, ((int64_t)c->budget / 2 - fixed) / per_pair);
    if (sv->cap_pairs < 1) {
      delete sv;
      return fail(CCM_ERR_OOM, "budget %zu holds no wave", c->budget);
    }
  }
  sv->cap_groups = sv->cap_pairs * 2 * max_np;
  sv->cap_items = sv->cap_pairs * max_items;
  if (sv->cap_items >= ((int64_t)1 << 31)) {
    delete sv;
    return fail(CCM_ERR_INVALID, "wave of %lld work items is too large", (long long)sv->cap_items);
  }
  const int64_t need = 2 * set_bytes(sv->cap_pairs, sv->cap_groups, sv->cap_req, sv->cap_items);
  if (c->budget && (size_t)need > c->budget) {
    delete sv;
    return fail(CCM_ERR_OOM, "serving buffers need %lld bytes, budget %zu", (long long)need,
                c->budget);
  }
  for (WaveSet& s : sv->sets) {
    if ((st = setup_set(sv, s)) != CCM_OK) {
      for (WaveSet& r : sv->sets) release_set(r);
      delete sv;
      return st;
    }
  }
  c->serving = sv;
  sv->worker = std::thread(worker_main, sv);
  return CCM_OK;
}

ccm_status ccm_serve_stop(ccm_ctx ctx) {
  if (!ctx) return fail(CCM_ERR_INVALID, "ctx is NULL");
  Context* c = reinterpret_cast<Context*>(ctx);
  if (!c->serving) return fail(CCM_ERR_INVALID, "serving not started");
  c->shutdown_serving();
  return CCM_OK;
}

ccm_status ccm_submit(ccm_ctx ctx, const ccm_request* req, ccm_ticket* out) {
  if (!ctx || !req || !out) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  Serving* sv = c->serving;
  if (!sv) return fail(CCM_ERR_INVALID, "serving not started");
  if (req->n_pairs < 1 || !req->A || !req->B || !req->pose_a || !req->pose_b || !req->y)
    return fail(CCM_ERR_INVALID, "bad request");
  if (req->ybar && !req->grad) return fail(CCM_ERR_INVALID, "ybar without grad");
  Pending p;
  p.pairs.resize(req->n_pairs);
  int64_t G = 0;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (int64_t i = 0; i < req->n_pairs; ++i) {
      int32_t a, b;
      ccm_status s;
      if ((s = c->body_of(req->A[i], &a)) != CCM_OK || (s = c->body_of(req->B[i], &b)) != CCM_OK)
        return s;
      if (!sv->fits(*c, a) || !sv->fits(*c, b))
        return fail(CCM_ERR_INVALID, "body %d or %d has a piece larger than the serving shape", a, b);
      p.pairs[i] = PairRec{a, b, G};
      G += c->bodies[a].np + c->bodies[b].np;
    }
    p.item_off.assign(1, 0);
    std::vector<int64_t> cost;
    p.items.reserve(2 * req->n_pairs);
    cost.reserve(2 * req->n_pairs);
    p.item_off.reserve(req->n_pairs + 1);
    for (int64_t i = 0; i < req->n_pairs; ++i) {   // make_items, from the cached chunks
      const int32_t a = p.pairs[i].bodyA, b = p.pairs[i].bodyB;
      push_items(sv->chunks(*c, a), (int32_t)(2 * i), c->bodies[b].np, &p.items, &cost);
      push_items(sv->chunks(*c, b), (int32_t)(2 * i + 1), c->bodies[a].np, &p.items, &cost);
      p.item_off.push_back((int64_t)p.items.size());
    }
    p.pcls.resize(req->n_pairs);
    for (int64_t i = 0; i < req->n_pairs; ++i) {
      int64_t pc = 0;
      for (int64_t j = p.item_off[i]; j < p.item_off[i + 1]; ++j) pc += cost[j];
      p.pcls[i] = cost_class(pc);
    }
    p.cls.resize(cost.size());
    for (size_t j = 0; j < cost.size(); ++j) p.cls[j] = cost_class(cost[j]);
  }
  p.d = ReqDesc{req->pose_a, req->pose_b, req->y, req->ybar, req->grad, 0, req->n_pairs, 0, G,
                0, 0};
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->async_error != cudaSuccess) return cuda_fail(sv->async_error, "serving");
  if (req->n_pairs > sv->cap_pairs || G > sv->cap_groups ||
      (int64_t)p.items.size() > sv->cap_items)
    return fail(CCM_ERR_OOM, "request of %lld pairs exceeds the wave capacity of %lld",
                (long long)req->n_pairs, (long long)sv->cap_pairs);
  if ((int64_t)sv->queue.size() >= sv->cfg.max_queued)
    return fail(CCM_ERR_BUSY, "request queue full (%lld)", (long long)sv->cfg.max_queued);
  p.ticket = sv->next_ticket++;
  p.t_submit = now_s();
  sv->tickets[p.ticket] = TicketInfo{kQueued, p.t_submit, 0.0};
  *out = p.ticket;
  sv->queued_pairs += p.d.n;
  sv->queue.push_back(std::move(p));
  // Wake the scheduler when it has something new to decide: a queue that was
  // empty (an idle loop launches at once) or one that now fills half a wave
  // (a second wave may go out).  Otherwise it wakes on a wave's completion or
  // its own 100 us re-check; waking it on every submission made the
  // submitting thread and the scheduler trade the lock at the arrival rate.
  if (sv->queue.size() == 1 || 2 * sv->queued_pairs >= sv->cap_pairs) sv->cv.notify_one();
  return CCM_OK;
}

ccm_status ccm_poll(ccm_ctx ctx, ccm_ticket ticket, int* done, double* latency_s) {
  if (!ctx || !done) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  Serving* sv = c->serving;
  if (!sv) return fail(CCM_ERR_INVALID, "serving not started");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->async_error != cudaSuccess) return cuda_fail(sv->async_error, "serving");
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return fail(CCM_ERR_UNKNOWN_TICKET, "unknown ticket %llu",
                                          (unsigned long long)ticket);
  *done = it->second.state == kDone;
  if (*done) {
    if (latency_s) *latency_s = it->second.t_done - it->second.t_submit;
    sv->tickets.erase(it);
  }
  return CCM_OK;
}

ccm_status ccm_poll_completed(ccm_ctx ctx, ccm_ticket* tickets, double* latency_s,
                              int64_t capacity, int64_t* n_out) {
  if (!ctx || !n_out || capacity < 0 || (capacity > 0 && !tickets))
    return fail(CCM_ERR_INVALID, "bad arguments");
  Serving* sv = reinterpret_cast<Context*>(ctx)->serving;
  if (!sv) return fail(CCM_ERR_INVALID, "serving not started");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->async_error != cudaSuccess) return cuda_fail(sv->async_error, "serving");
  int64_t n = 0;
  while (n < capacity && !sv->completed.empty()) {
    const uint64_t tk = sv->completed.front();
    sv->completed.pop_front();
    auto it = sv->tickets.find(tk);
    if (it == sv->tickets.end()) continue;   // already retired by ccm_poll
    tickets[n] = tk;
    if (latency_s) latency_s[n] = it->second.t_done - it->second.t_submit;
    sv->tickets.erase(it);
    ++n;
  }
  *n_out = n;
  return CCM_OK;
}

ccm_status ccm_serve_hold(ccm_ctx ctx, int hold) {
  if (!ctx) return fail(CCM_ERR_INVALID, "ctx is NULL");
  Serving* sv = reinterpret_cast<Context*>(ctx)->serving;
  if (!sv) return fail(CCM_ERR_INVALID, "serving not started");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->held = hold != 0;
  }
  sv->cv.notify_one();
  return CCM_OK;
}

ccm_status ccm_serve_stats(ccm_ctx ctx, ccm_serve_counters* out) {
  if (!ctx || !out) return fail(CCM_ERR_INVALID, "bad arguments");
  Serving* sv = reinterpret_cast<Context*>(ctx)->serving;
  if (!sv) return fail(CCM_ERR_INVALID, "serving not started");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->counters;
  return CCM_OK;
}

}  // extern "C"
