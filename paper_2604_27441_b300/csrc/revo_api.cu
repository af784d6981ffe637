// Runtime behind revo_recover_create / submit / flush / poll / destroy.
//
// A context owns, on one device: the RGB and depth networks, per-lane work
// arenas (a lane = a pair of CUDA streams, one per modality, so the two models
// run concurrently as in Section 3.1), per-conference-stream rings of the last
// k clean frames (Section 3.4.1 reuses the clean references across a GoP),
// staging buffers for host inputs/outputs, and the request queue.
//
// Scheduling (continuous batching): submitted frames wait in a pending queue;
// a batch of up to max_batch pending frames is launched on a lane whenever a
// lane has room (at most one batch running on it), when max_batch frames are
// waiting, on flush, or on a waiting poll.  Frames that arrive while both
// batches of every lane run are admitted together into the next batch as lanes
// and staging slots free up.  All device work is ordered with events: a batch waits
// for the copy stream (input uploads, reference pushes); a reference push
// waits for every lane's last batch.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "model.h"

namespace revo {

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxLanes = 8;
// FP8 precision, layers in E4M3 per model unless the config names others.  RGB:
// all four LayerNorm-fed layers (encoder and decoder qkv and fc1; 64 dB against
// the FP64 forward at 640x480).  Depth: none -- its millimetre gate is the
// binding one: the encoder fc1 alone gave 5.9 mm at 640x480 (500-4000 mm) but
// 17.6 mm on the 640x576 stream of 300-5000 mm, above the 8 mm gate, and every
// larger set measured worse.
constexpr int kDefaultFp8Layers[2] = {0xF, 0x0};

struct Ring {
  int H = 0, W = 0;
  int count = 0;       // valid frames
  int next = 0;        // slot the next push writes
  std::vector<int64_t> index;
  uint8_t* frames = nullptr;  // k slots of slot_bytes
  float* stats = nullptr;     // k x (mu, sigma) for depth
  size_t slot_bytes = 0;
};

struct Slot {  // staging for one request
  uint8_t* in[2] = {nullptr, nullptr};     // current frame rgb / depth
  uint32_t* mask[2] = {nullptr, nullptr};
  uint8_t* out[2] = {nullptr, nullptr};
  float* values[2] = {nullptr, nullptr};
  bool busy = false;
};

struct Pending {
  uint64_t ticket;
  revo_request req;
  int slot;  // staging slot or -1
  PlaneJob job[2];
  bool has[2];
  Clock::time_point t_submit;
};

struct Batch {
  uint64_t id;
  int lane;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  std::vector<uint64_t> tickets;
  std::vector<int> slots;
  int size = 0;
  int* err_host = nullptr;  // pinned, 2 words (rgb, depth)
  bool done = false;
  revo_status status = REVO_OK;
  double device_ms = 0;
  int launches = 0;
};

// A retired batch's events and pinned error words, kept for the next batch:
// creating events and pinned memory per frame costs host time, and freeing
// pinned memory can synchronise the device.
struct BatchRes {
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  int* err_host = nullptr;
};

struct TicketInfo {
  uint64_t batch = 0;  // 0 = still pending
  uint32_t stream_id = 0;
  int64_t frame_index = 0;
  Clock::time_point t_submit;
};

constexpr int kArgRing = 4;     // pinned host copies of a batch's per-request arguments
constexpr int kMaxGraphs = 64;  // captured forwards kept per lane and modality

struct GraphEntry {
  int seen = 0;
  bool failed = false;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

struct Lane {
  cudaStream_t st[2] = {nullptr, nullptr};
  bool own_main = true;
  Workspace* ws[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join = nullptr, last_end = nullptr;
  bool used = false;
  // Graph replay: per modality, the device table the per-request kernels read,
  // a ring of pinned host tables it is uploaded from (an event per entry marks
  // the upload done), and the captured forwards keyed by the request sizes.
  JobArgs* dev_args[2] = {nullptr, nullptr};
  JobArgs* host_args[2][kArgRing] = {};
  cudaEvent_t args_ev[2][kArgRing] = {};
  int args_next[2] = {0, 0};
  std::map<std::vector<int>, GraphEntry> graphs[2];
};

}  // namespace

}  // namespace revo

struct revo_ctx {
  revo_config cfg{};
  int device = 0;
  int sms = 148;
  revo::NetShape shape[2]{};
  revo::Net* net[2] = {nullptr, nullptr};
  revo::Lane lanes[revo::kMaxLanes];
  int n_lanes = 1;
  int next_lane = 0;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev = nullptr;
  bool copy_ev_valid = false;
  std::vector<revo::Ring> rings[2];
  std::vector<revo::Slot> slots;
  void* stats_scratch = nullptr;
  std::deque<revo::Pending> pending;
  std::map<uint64_t, revo::TicketInfo> tickets;
  std::map<uint64_t, revo::Batch> batches;
  uint64_t next_ticket = 1, next_batch = 1;
  uint64_t n_batches = 0, graph_replays = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<revo::BatchRes> batch_pool;  // resources of retired batches
};

namespace revo {

namespace {

revo_status fail(revo_status s, const char* fmt, const char* what = "") {
  set_last_error(fmt, what);
  return s;
}

size_t frame_bytes(int m, int H, int W) { return static_cast<size_t>(H) * W * (m == 0 ? 3 : 2); }
size_t mask_words(int H, int W) { return static_cast<size_t>(H) * ((W + 31) / 32); }

cudaError_t ctx_alloc(revo_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    c->allocs.push_back(*p);
    c->bytes += bytes;
  }
  return e;
}

void release_batch(revo_ctx* c, Batch& b) {
  for (int s : b.slots) c->slots[s].busy = false;
  b.slots.clear();
}

// Marks the batch done if its end event completed; returns true if done.
bool batch_check(revo_ctx* c, Batch& b, bool block) {
  if (b.done) return true;
  cudaError_t e = block ? cudaEventSynchronize(b.ev_end) : cudaEventQuery(b.ev_end);
  if (e == cudaErrorNotReady) return false;
  b.done = true;
  if (e != cudaSuccess) {
    b.status = REVO_ECUDA;
    set_last_error("batch failed: %s", cudaGetErrorString(e));
  } else {
    float ms = 0.f;
    if (b.lane >= 0 && b.ev_start) cudaEventElapsedTime(&ms, b.ev_start, b.ev_end);  // copy-only batches: 0
    b.device_ms = ms;
    if (b.err_host && (b.err_host[0] || b.err_host[1])) b.status = REVO_ETIMEDOUT;
  }
  release_batch(c, b);
  return true;
}

void free_batch_res(const BatchRes& r) {
  if (r.ev_start) cudaEventDestroy(r.ev_start);
  if (r.ev_end) cudaEventDestroy(r.ev_end);
  if (r.err_host) cudaFreeHost(r.err_host);
}

// Events and pinned error words for a new batch: a retired batch's, else new ones.
cudaError_t acquire_batch_res(revo_ctx* c, Batch& b) {
  BatchRes r;
  if (!c->batch_pool.empty()) {
    r = c->batch_pool.back();
    c->batch_pool.pop_back();
  } else {
    cudaError_t e;
    if ((e = cudaEventCreate(&r.ev_start)) != cudaSuccess || (e = cudaEventCreate(&r.ev_end)) != cudaSuccess ||
        (e = cudaMallocHost(&r.err_host, 2 * sizeof(int))) != cudaSuccess) {
      free_batch_res(r);
      return e;
    }
  }
  b.ev_start = r.ev_start;
  b.ev_end = r.ev_end;
  b.err_host = r.err_host;
  b.err_host[0] = b.err_host[1] = 0;
  return cudaSuccess;
}

void retire_if_empty(revo_ctx* c, uint64_t bid) {
  auto it = c->batches.find(bid);
  if (it == c->batches.end() || !it->second.tickets.empty() || !it->second.done) return;
  Batch& b = it->second;
  const BatchRes r{b.ev_start, b.ev_end, b.err_host};
  if (r.ev_start && r.ev_end && r.err_host)
    c->batch_pool.push_back(r);
  else
    free_batch_res(r);
  c->batches.erase(it);
}

bool lane_idle(revo_ctx* c, int l) {
  Lane& L = c->lanes[l];
  return !L.used || cudaEventQuery(L.last_end) == cudaSuccess;
}

// A lane with room runs at most one batch: a new batch queued behind it starts
// on the device as soon as the running one ends, with no host round trip in
// between.  Lanes with two batches in flight leave new arrivals pending, to be
// launched together.
bool lane_room(revo_ctx* c, int l) {
  if (lane_idle(c, l)) return true;
  int in_flight = 0;
  for (auto& kv : c->batches)
    if (kv.second.lane == l && !batch_check(c, kv.second, false)) ++in_flight;
  return in_flight < 2;
}

// Enqueues the forward of `jobs` (modality m) on lane L.  Without graphs: plain
// launches.  With graphs: the per-request arguments are uploaded to the lane's
// device table (one copy from pinned memory), then the graph captured for these
// request sizes is replayed.  A size pattern runs eagerly (reading the same
// table) the first time it is seen, so every kernel's one-time set-up happens
// outside a capture, and is captured the second time.
cudaError_t lane_forward(revo_ctx* c, Lane& L, int m, const std::vector<PlaneJob>& jobs, int* launches) {
  Net* net = c->net[m];
  Workspace* ws = L.ws[m];
  cudaStream_t s = L.st[m];
  const int n = static_cast<int>(jobs.size());
  if (!c->cfg.use_graphs || !L.dev_args[m])
    return net_forward(net, ws, jobs.data(), n, s, c->sms, launches, nullptr);

  const int r = L.args_next[m];
  L.args_next[m] = (r + 1) % kArgRing;
  cudaError_t e = cudaEventSynchronize(L.args_ev[m][r]);  // that copy's last upload has been read
  if (e != cudaSuccess) return e;
  if ((e = prepare_job_args(net, ws, jobs.data(), n, L.host_args[m][r])) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.dev_args[m], L.host_args[m][r], n * sizeof(JobArgs), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaEventRecord(L.args_ev[m][r], s)) != cudaSuccess) return e;

  std::vector<int> key;
  for (const PlaneJob& j : jobs) {
    key.push_back(j.H);
    key.push_back(j.W);
  }
  auto it = L.graphs[m].find(key);
  if (it == L.graphs[m].end()) {
    if (static_cast<int>(L.graphs[m].size()) >= kMaxGraphs)
      return net_forward(net, ws, jobs.data(), n, s, c->sms, launches, L.dev_args[m]);
    it = L.graphs[m].emplace(key, GraphEntry{}).first;
  }
  GraphEntry& g = it->second;
  if (!g.exec) {
    if (g.failed || g.seen++ == 0)
      return net_forward(net, ws, jobs.data(), n, s, c->sms, launches, L.dev_args[m]);
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    int nl = 0;
    const cudaError_t ef = net_forward(net, ws, jobs.data(), n, s, c->sms, &nl, L.dev_args[m]);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    cudaError_t ei = cudaErrorUnknown;
    if (ef == cudaSuccess && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ef != cudaSuccess) return ef;  // an argument error, not a capture problem
    if (ei != cudaSuccess) {
      // The capture did not take: run this size pattern with plain launches from now on.
      (void)cudaGetLastError();
      g.exec = nullptr;
      g.failed = true;
      return net_forward(net, ws, jobs.data(), n, s, c->sms, launches, L.dev_args[m]);
    }
    g.launches = nl;
  }
  if (launches) *launches = g.launches;
  ++c->graph_replays;
  return cudaGraphLaunch(g.exec, s);
}

revo_status launch_batch(revo_ctx* c, int count) {
  if (count <= 0 || c->pending.empty()) return REVO_OK;
  if (count > static_cast<int>(c->pending.size())) count = static_cast<int>(c->pending.size());
  // Prefer an idle lane, then one with room; otherwise round-robin (stream
  // order queues the work).
  int lane = -1;
  for (int i = 0; i < c->n_lanes && lane < 0; ++i) {
    const int l = (c->next_lane + i) % c->n_lanes;
    if (lane_idle(c, l)) lane = l;
  }
  for (int i = 0; i < c->n_lanes && lane < 0; ++i) {
    const int l = (c->next_lane + i) % c->n_lanes;
    if (lane_room(c, l)) lane = l;
  }
  if (lane < 0) lane = c->next_lane;
  c->next_lane = (lane + 1) % c->n_lanes;
  Lane& L = c->lanes[lane];

  Batch b;
  b.id = c->next_batch++;
  b.lane = lane;
  cudaError_t e;
  if ((e = acquire_batch_res(c, b)) != cudaSuccess) return cuda_status(e, "batch setup");

  std::vector<PlaneJob> jobs[2];
  std::vector<Pending> taken;
  for (int i = 0; i < count; ++i) {
    taken.push_back(c->pending.front());
    c->pending.pop_front();
  }
  for (const Pending& p : taken)
    for (int m = 0; m < 2; ++m)
      if (p.has[m]) jobs[m].push_back(p.job[m]);
  // Jobs in size order: the same mix of sizes maps to one captured graph
  // whatever the arrival order (each job carries its own output pointers).
  for (int m = 0; m < 2; ++m)
    std::stable_sort(jobs[m].begin(), jobs[m].end(), [](const PlaneJob& a, const PlaneJob& b) {
      return a.H != b.H ? a.H < b.H : a.W < b.W;
    });

  cudaStream_t main = L.st[0];
  cudaEventRecord(b.ev_start, main);
  if (c->copy_ev_valid) cudaStreamWaitEvent(main, c->copy_ev, 0);
  cudaEventRecord(L.fork, main);
  cudaStreamWaitEvent(L.st[1], L.fork, 0);
  revo_status st = REVO_OK;
  for (int m = 0; m < 2 && st == REVO_OK; ++m) {
    if (jobs[m].empty()) continue;
    cudaStream_t s = L.st[m];
    cudaMemsetAsync(L.ws[m]->err, 0, sizeof(int), s);
    int nl = 0;
    e = lane_forward(c, L, m, jobs[m], &nl);
    b.launches += nl;
    if (e != cudaSuccess) st = cuda_status(e, "forward launch");
    cudaMemcpyAsync(b.err_host + m, L.ws[m]->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (m == 0 && c->cfg.serial_models && !jobs[1].empty()) {
      // The depth forward starts once the RGB forward has finished.
      cudaEventRecord(L.fork, main);
      cudaStreamWaitEvent(L.st[1], L.fork, 0);
    }
  }
  cudaEventRecord(L.join, L.st[1]);
  cudaStreamWaitEvent(main, L.join, 0);
  // Host outputs: copy back from staging.
  for (const Pending& p : taken) {
    if (p.req.outputs_on_device || p.slot < 0) continue;
    const Slot& sl = c->slots[p.slot];
    for (int m = 0; m < 2; ++m) {
      if (!p.has[m]) continue;
      const revo_plane& pl = m == 0 ? p.req.rgb : p.req.depth;
      const size_t row = static_cast<size_t>(pl.width) * (m == 0 ? 3 : 2);
      void* dst = m == 0 ? p.req.rgb_out : p.req.depth_out;
      const size_t dp = m == 0 ? p.req.rgb_out_pitch : p.req.depth_out_pitch;
      if (dst) cudaMemcpy2DAsync(dst, dp, sl.out[m], row, row, pl.height, cudaMemcpyDeviceToHost, main);
      float* vals = m == 0 ? p.req.rgb_values : p.req.depth_values;
      if (vals)
        cudaMemcpyAsync(vals, sl.values[m], static_cast<size_t>(pl.height) * pl.width * (m == 0 ? 3 : 1) * 4,
                        cudaMemcpyDeviceToHost, main);
    }
  }
  cudaEventRecord(b.ev_end, main);
  cudaEventRecord(L.last_end, main);
  L.used = true;
  for (const Pending& p : taken) {
    b.tickets.push_back(p.ticket);
    if (p.slot >= 0) b.slots.push_back(p.slot);
    auto it = c->tickets.find(p.ticket);
    if (it != c->tickets.end()) it->second.batch = b.id;
  }
  b.size = count;
  ++c->n_batches;
  if (st != REVO_OK) b.status = st;
  c->batches.emplace(b.id, b);
  return st;
}

// Launches batches while a lane has room (see lane_room) and frames are
// waiting, or while max_batch are pending, or all of them when forced.
void dispatch(revo_ctx* c, bool force) {
  while (!c->pending.empty()) {
    bool room = false;
    for (int l = 0; l < c->n_lanes; ++l) room = room || lane_room(c, l);
    const bool full = static_cast<int>(c->pending.size()) >= c->cfg.max_batch;
    if (!(room || full || force)) break;
    launch_batch(c, c->cfg.max_batch);
  }
}

int find_free_slot(revo_ctx* c) {
  for (size_t i = 0; i < c->slots.size(); ++i)
    if (!c->slots[i].busy) return static_cast<int>(i);
  return -1;
}

// Frees staging by waiting for the oldest running batch (launching pending work first).
int acquire_slot(revo_ctx* c) {
  int s = find_free_slot(c);
  if (s >= 0) return s;
  for (auto& kv : c->batches) batch_check(c, kv.second, false);
  if ((s = find_free_slot(c)) >= 0) return s;
  dispatch(c, true);
  for (auto& kv : c->batches) {
    if (kv.second.done) continue;
    batch_check(c, kv.second, true);
    if ((s = find_free_slot(c)) >= 0) return s;
  }
  return -1;
}

revo_status push_clean(revo_ctx* c, const revo_request* r, int m, uint64_t* ticket) {
  const revo_plane& pl = m == 0 ? r->rgb : r->depth;
  Ring& ring = c->rings[m][r->stream_id];
  if (ring.count > 0 && (ring.H != pl.height || ring.W != pl.width))
    return fail(REVO_EINVAL, "clean frame size differs from the stream's history%s");
  // Work that reads this ring must be launched (and ordered) before the slot is
  // overwritten: pending requests of this stream hold pointers into it.  Other
  // streams' pending requests stay pending (to be batched with later arrivals).
  bool reads_ring = false;
  for (const Pending& p : c->pending) reads_ring = reads_ring || p.req.stream_id == r->stream_id;
  dispatch(c, reads_ring);
  for (int l = 0; l < c->n_lanes; ++l)
    if (c->lanes[l].used) cudaStreamWaitEvent(c->copy_st, c->lanes[l].last_end, 0);
  ring.H = pl.height;
  ring.W = pl.width;
  const int slot = ring.next;
  uint8_t* dst = ring.frames + slot * ring.slot_bytes;
  const size_t row = static_cast<size_t>(pl.width) * (m == 0 ? 3 : 2);
  cudaError_t e = cudaMemcpy2DAsync(dst, row, pl.data, pl.pitch_bytes, row, pl.height,
                                    r->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c->copy_st);
  if (e != cudaSuccess) return cuda_status(e, "reference upload");
  if (m == 1) {
    e = launch_depth_stats(reinterpret_cast<const uint16_t*>(dst), pl.height, pl.width, row, ring.stats + 2 * slot,
                           c->stats_scratch, c->copy_st);
    if (e != cudaSuccess) return cuda_status(e, "depth statistics");
  }
  ring.index[slot] = r->frame_index;
  ring.next = (slot + 1) % c->cfg.k;
  if (ring.count < c->cfg.k) ++ring.count;
  (void)ticket;
  return REVO_OK;
}

revo_status validate_plane(revo_ctx* c, const revo_plane& pl, const uint32_t* mask, size_t mask_pitch, bool clean) {
  if (!pl.data) return fail(REVO_EINVAL, "null plane data%s");
  if (pl.height <= 0 || pl.width <= 0 || pl.height % c->cfg.patch || pl.width % c->cfg.patch)
    return fail(REVO_EINVAL, "plane size must be a positive multiple of the patch size%s");
  if (pl.height > c->cfg.max_height || pl.width > c->cfg.max_width)
    return fail(REVO_EINVAL, "plane larger than max_height x max_width%s");
  if (!clean && (!mask || mask_pitch < static_cast<size_t>((pl.width + 31) / 32)))
    return fail(REVO_EINVAL, "missing loss mask or mask pitch too small%s");
  return REVO_OK;
}

}  // namespace

}  // namespace revo

using namespace revo;

extern "C" {

void revo_config_default(revo_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->k = 5;
  cfg->tubelet = 2;
  cfg->patch = 16;
  cfg->enc_dim = 768;
  cfg->enc_depth = 12;
  cfg->enc_heads = 12;
  cfg->dec_dim = 384;
  cfg->dec_depth = 4;
  cfg->dec_heads = 6;
  cfg->mlp_ratio = 4;
  cfg->precision = REVO_BF16;
  cfg->hbm_budget_bytes = 40ull << 30;
  cfg->max_streams = 16;
  cfg->max_height = 720;
  cfg->max_width = 1280;
  cfg->max_batch = 1;
  cfg->lanes = 1;
}

void revo_recover_destroy(revo_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (auto& kv : c->batches) batch_check(c, kv.second, true);
  for (auto& kv : c->batches) free_batch_res(BatchRes{kv.second.ev_start, kv.second.ev_end, kv.second.err_host});
  for (const BatchRes& r : c->batch_pool) free_batch_res(r);
  if (c->copy_st) cudaStreamSynchronize(c->copy_st);
  for (int l = 0; l < c->n_lanes; ++l) {
    Lane& L = c->lanes[l];
    for (int m = 0; m < 2; ++m) {
      if (L.st[m]) cudaStreamSynchronize(L.st[m]);
      workspace_destroy(L.ws[m]);
      for (auto& kv : L.graphs[m])
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      for (int r = 0; r < kArgRing; ++r) {
        if (L.host_args[m][r]) cudaFreeHost(L.host_args[m][r]);
        if (L.args_ev[m][r]) cudaEventDestroy(L.args_ev[m][r]);
      }
    }
    if (L.st[0] && L.own_main) cudaStreamDestroy(L.st[0]);
    if (L.st[1]) cudaStreamDestroy(L.st[1]);
    if (L.fork) cudaEventDestroy(L.fork);
    if (L.join) cudaEventDestroy(L.join);
    if (L.last_end) cudaEventDestroy(L.last_end);
  }
  if (c->copy_st) cudaStreamDestroy(c->copy_st);
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  for (void* p : c->allocs) cudaFree(p);
  for (int m = 0; m < 2; ++m) net_destroy(c->net[m]);
  delete c;
}

// Autotune cache file: a header line naming the GPU it was timed on, then one
// line per choice: modality, shape key (tune_key, hex), tile choice.
std::string autotune_tag(const cudaDeviceProp& p) {
  char buf[320];
  snprintf(buf, sizeof(buf), "revo-autotune 1 sm_%d%d sms=%d %s", p.major, p.minor, p.multiProcessorCount, p.name);
  for (char* q = buf; *q; ++q)
    if (*q == '\n') *q = ' ';
  return buf;
}

void load_autotune_cache(revo_ctx* c, const char* path, const std::string& tag) {
  FILE* f = fopen(path, "r");
  if (!f) return;  // no file yet: everything is timed and the file written
  char line[512];
  if (fgets(line, sizeof(line), f) && std::string(line).substr(0, tag.size()) == tag) {
    int m = 0, choice = 0;
    unsigned long long key = 0;
    while (fgets(line, sizeof(line), f))
      if (sscanf(line, "%d %llx %d", &m, &key, &choice) == 3 && m >= 0 && m < 2 && c->net[m] &&
          ((choice & ~kTilePair) == 128 || (choice & ~kTilePair) == 256))
        c->net[m]->tuned_bn[key] = choice;
  }
  fclose(f);
}

bool save_autotune_cache(revo_ctx* c, const char* path, const std::string& tag) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return false;
  fprintf(f, "%s\n", tag.c_str());
  for (int m = 0; m < 2; ++m)
    if (c->net[m])
      for (const auto& kv : c->net[m]->tuned_bn)
        fprintf(f, "%d %llx %d\n", m, static_cast<unsigned long long>(kv.first), kv.second);
  const bool ok = fclose(f) == 0;
  return ok && rename(tmp.c_str(), path) == 0;
}

revo_status revo_recover_create(const revo_config* cfg, revo_ctx** out) {
  if (!out) return fail(REVO_EINVAL, "null out%s");
  *out = nullptr;
  if (!cfg) return fail(REVO_EINVAL, "null config%s");
  if (cfg->max_batch < 1 || cfg->max_batch > kMaxSegments || cfg->lanes < 1 || cfg->lanes > kMaxLanes ||
      cfg->max_streams < 1 || cfg->max_height <= 0 || cfg->max_width <= 0)
    return fail(REVO_EINVAL, "max_batch must be 1..64, lanes 1..8, max_streams and max size positive%s");
  if (static_cast<long long>(cfg->max_height) * cfg->max_width > kDepthStatsMaxPixels)
    return fail(REVO_EINVAL, "max_height x max_width above 2^24 pixels%s");
  if (cfg->precision != REVO_FP32 && cfg->precision != REVO_BF16 && cfg->precision != REVO_FP8)
    return fail(REVO_ENOTSUP, "precision not supported%s");
  if (cfg->precision == REVO_FP8 && (cfg->enc_dim % 128 || cfg->dec_dim % 128))
    return fail(REVO_EINVAL, "the FP8 path needs widths that are multiples of 128%s");
  if (!cfg->rgb_weights && !cfg->depth_weights && !cfg->rgb_weights_path && !cfg->depth_weights_path &&
      !(cfg->random_init & 3))
    return fail(REVO_EINVAL, "no model weights given%s");
  if (cudaSetDevice(cfg->device) != cudaSuccess) return fail(REVO_EINVAL, "bad device ordinal%s");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg->device) != cudaSuccess) return fail(REVO_ECUDA, "device query failed%s");
  if (cfg->precision != REVO_FP32 && prop.major != 10)
    return fail(REVO_ENOTSUP, "the tensor-core path needs an sm_100-class GPU%s");

  std::unique_ptr<revo_ctx, void (*)(revo_ctx*)> c(new revo_ctx(), revo_recover_destroy);
  c->cfg = *cfg;
  c->device = cfg->device;
  c->sms = prop.multiProcessorCount;
  c->n_lanes = cfg->lanes;
  const size_t budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (40ull << 30);
  const float* w[2] = {cfg->rgb_weights, cfg->depth_weights};
  size_t wn[2] = {cfg->rgb_weights_count, cfg->depth_weights_count};
  // Models without an array: from their file, or the seeded random initialisation.
  std::vector<float> host_w[2];
  const char* wpath[2] = {cfg->rgb_weights_path, cfg->depth_weights_path};
  for (int m = 0; m < 2; ++m) {
    if (w[m] || (!wpath[m] && !((cfg->random_init >> m) & 1))) continue;
    NetShape s{m == 0 ? 3 : 1, cfg->k, cfg->tubelet, cfg->patch, cfg->enc_dim, cfg->enc_depth, cfg->enc_heads,
               cfg->dec_dim, cfg->dec_depth, cfg->dec_heads, cfg->mlp_ratio};
    std::string why = check_shape(s);
    if (!why.empty()) return fail(REVO_EINVAL, "unsupported network shape: %s", why.c_str());
    host_w[m].resize(param_count(s));
    if (wpath[m]) {
      if (!load_weights_file(wpath[m], 0, host_w[m].size(), host_w[m].data(), &why))
        return fail(REVO_EINVAL, "%s", why.c_str());
    } else {
      init_weights_random(s, cfg->seed + static_cast<uint64_t>(m), host_w[m].data());
    }
    w[m] = host_w[m].data();
    wn[m] = host_w[m].size();
  }
  int cap_tok[2] = {0, 0}, cap_p[2] = {0, 0};
  size_t need = 0;
  for (int m = 0; m < 2; ++m) {
    NetShape s{m == 0 ? 3 : 1, cfg->k, cfg->tubelet, cfg->patch, cfg->enc_dim, cfg->enc_depth, cfg->enc_heads,
               cfg->dec_dim, cfg->dec_depth, cfg->dec_heads, cfg->mlp_ratio};
    c->shape[m] = s;
    if (!w[m]) continue;
    std::string why = check_shape(s);
    if (!why.empty()) return fail(REVO_EINVAL, "unsupported network shape: %s", why.c_str());
    if (wn[m] != param_count(s)) return fail(REVO_EINVAL, "weight count does not match the network shape%s");
    cap_p[m] = cfg->max_batch * request_patches(s, cfg->max_height, cfg->max_width);
    cap_tok[m] = cfg->max_batch * request_tokens(s, cfg->max_height, cfg->max_width);
    need += net_bytes(s, cfg->precision) + cfg->lanes * workspace_bytes(s, cfg->precision, cap_tok[m], cap_p[m], cfg->max_batch,
                                                  std::max(cfg->max_width, cfg->max_height) / cfg->patch);
    need += static_cast<size_t>(cfg->max_streams) * cfg->k * frame_bytes(m, cfg->max_height, cfg->max_width);
    need += static_cast<size_t>(2 * cfg->max_batch * cfg->lanes) *
            (frame_bytes(m, cfg->max_height, cfg->max_width) * 2 + mask_words(cfg->max_height, cfg->max_width) * 4 +
             static_cast<size_t>(cfg->max_height) * cfg->max_width * (m == 0 ? 3 : 1) * 4);
  }
  if (need > budget) return fail(REVO_ENOMEM, "the configuration needs more device memory than hbm_budget_bytes%s");

  std::string err;
  for (int m = 0; m < 2; ++m) {
    if (!w[m]) continue;
    c->net[m] = net_create(c->shape[m], cfg->precision, w[m], &err);
    if (!c->net[m]) return fail(REVO_ENOMEM, "network upload: %s", err.c_str());
    c->net[m]->autotune = cfg->autotune != 0 && cfg->precision != REVO_FP32;
    c->net[m]->fp8_mask = cfg->fp8_layers ? ((cfg->fp8_layers >> (4 * m)) & 15) : kDefaultFp8Layers[m];
    c->bytes += net_bytes(c->shape[m], cfg->precision);
  }
  cudaError_t e;
  for (int l = 0; l < c->n_lanes; ++l) {
    Lane& L = c->lanes[l];
    if (l == 0 && cfg->cuda_stream) {
      L.st[0] = static_cast<cudaStream_t>(cfg->cuda_stream);
      L.own_main = false;
    } else if ((e = cudaStreamCreateWithFlags(&L.st[0], cudaStreamNonBlocking)) != cudaSuccess) {
      return cuda_status(e, "stream create");
    }
    if ((e = cudaStreamCreateWithFlags(&L.st[1], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&L.last_end, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_status(e, "lane setup");
    for (int m = 0; m < 2; ++m) {
      if (!c->net[m]) continue;
      L.ws[m] = workspace_create(c->shape[m], cfg->precision, cap_tok[m], cap_p[m], cfg->max_batch,
                                 std::max(cfg->max_width, cfg->max_height) / cfg->patch, &err);
      if (!L.ws[m]) return fail(REVO_ENOMEM, "workspace: %s", err.c_str());
      c->bytes += L.ws[m]->bytes;
      if (!cfg->use_graphs) continue;
      const size_t tb = static_cast<size_t>(cfg->max_batch) * sizeof(JobArgs);
      if (ctx_alloc(c.get(), reinterpret_cast<void**>(&L.dev_args[m]), tb) != cudaSuccess)
        return fail(REVO_ENOMEM, "argument table allocation failed%s");
      for (int r = 0; r < kArgRing; ++r)
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&L.host_args[m][r]), tb)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&L.args_ev[m][r], cudaEventDisableTiming)) != cudaSuccess)
          return cuda_status(e, "argument table setup");
    }
  }
  if ((e = cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_status(e, "copy stream");
  for (int m = 0; m < 2; ++m) {
    if (!c->net[m]) continue;
    c->rings[m].resize(cfg->max_streams);
    for (Ring& r : c->rings[m]) {
      r.slot_bytes = frame_bytes(m, cfg->max_height, cfg->max_width);
      r.index.assign(cfg->k, 0);
      if ((e = ctx_alloc(c.get(), reinterpret_cast<void**>(&r.frames), r.slot_bytes * cfg->k)) != cudaSuccess)
        return fail(REVO_ENOMEM, "reference ring allocation failed%s");
      if (m == 1 &&
          (e = ctx_alloc(c.get(), reinterpret_cast<void**>(&r.stats), sizeof(float) * 2 * cfg->k)) != cudaSuccess)
        return fail(REVO_ENOMEM, "reference statistics allocation failed%s");
    }
  }
  if (c->net[1] && (e = ctx_alloc(c.get(), &c->stats_scratch, depth_stats_scratch_bytes())) != cudaSuccess)
    return fail(REVO_ENOMEM, "statistics scratch allocation failed%s");
  c->slots.resize(static_cast<size_t>(2 * cfg->max_batch * cfg->lanes));
  for (Slot& s : c->slots) {
    for (int m = 0; m < 2; ++m) {
      if (!c->net[m]) continue;
      const size_t fb = frame_bytes(m, cfg->max_height, cfg->max_width);
      const size_t vb = static_cast<size_t>(cfg->max_height) * cfg->max_width * (m == 0 ? 3 : 1) * 4;
      if (ctx_alloc(c.get(), reinterpret_cast<void**>(&s.in[m]), fb) != cudaSuccess ||
          ctx_alloc(c.get(), reinterpret_cast<void**>(&s.out[m]), fb) != cudaSuccess ||
          ctx_alloc(c.get(), reinterpret_cast<void**>(&s.mask[m]),
                    mask_words(cfg->max_height, cfg->max_width) * 4) != cudaSuccess ||
          ctx_alloc(c.get(), reinterpret_cast<void**>(&s.values[m]), vb) != cudaSuccess)
        return fail(REVO_ENOMEM, "staging allocation failed%s");
    }
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_status(e, "create");
  if (cfg->autotune && cfg->precision != REVO_FP32) {
    // Tile choices: from the cache file where it has them, timed here for the rest.
    const std::string tag = autotune_tag(prop);
    if (cfg->autotune_cache) load_autotune_cache(c.get(), cfg->autotune_cache, tag);
    size_t before = 0, after = 0;
    for (int m = 0; m < 2; ++m) before += c->net[m] ? c->net[m]->tuned_bn.size() : 0;
    for (int m = 0; m < 2; ++m) {
      if (!c->net[m]) continue;
      if ((e = net_autotune(c->net[m], c->lanes[0].ws[m], cap_tok[m], cap_p[m], c->lanes[0].st[m], c->sms)) !=
          cudaSuccess)
        return cuda_status(e, "autotune");
      after += c->net[m]->tuned_bn.size();
    }
    if (cfg->autotune_cache && after != before && !save_autotune_cache(c.get(), cfg->autotune_cache, tag))
      return fail(REVO_EINVAL, "cannot write the autotune cache file %s", cfg->autotune_cache);
  }
  *out = c.release();
  return REVO_OK;
}

revo_status revo_init_weights(const revo_config* cfg, int channels, uint64_t seed, float* out, size_t count) {
  if (!cfg || !out || (channels != 1 && channels != 3)) return fail(REVO_EINVAL, "bad argument%s");
  NetShape s{channels, cfg->k, cfg->tubelet, cfg->patch, cfg->enc_dim, cfg->enc_depth, cfg->enc_heads,
             cfg->dec_dim, cfg->dec_depth, cfg->dec_heads, cfg->mlp_ratio};
  const std::string why = check_shape(s);
  if (!why.empty()) return fail(REVO_EINVAL, "unsupported network shape: %s", why.c_str());
  if (count != param_count(s)) return fail(REVO_EINVAL, "count differs from the model's parameter count%s");
  init_weights_random(s, seed, out);
  return REVO_OK;
}

revo_status revo_recover_submit(revo_ctx* c, const revo_request* r, uint64_t* ticket) {
  if (!c || !r || !ticket) return fail(REVO_EINVAL, "null argument%s");
  cudaSetDevice(c->device);
  const bool clean = (r->flags & REVO_CLEAN) != 0;
  const bool has[2] = {(r->flags & REVO_RGB) != 0, (r->flags & REVO_DEPTH) != 0};
  if (!has[0] && !has[1]) return fail(REVO_EINVAL, "request carries neither REVO_RGB nor REVO_DEPTH%s");
  if (r->stream_id >= static_cast<uint32_t>(c->cfg.max_streams)) return fail(REVO_EINVAL, "stream_id out of range%s");
  for (int m = 0; m < 2; ++m) {
    if (!has[m]) continue;
    if (!c->net[m]) return fail(REVO_EINVAL, "no model was loaded for this modality%s");
    const revo_plane& pl = m == 0 ? r->rgb : r->depth;
    revo_status s = validate_plane(c, pl, m == 0 ? r->rgb_lost_mask : r->depth_lost_mask,
                                   m == 0 ? r->rgb_mask_pitch_words : r->depth_mask_pitch_words, clean);
    if (s != REVO_OK) return s;
    const size_t row = static_cast<size_t>(pl.width) * (m == 0 ? 3 : 2);
    if (pl.pitch_bytes < row) return fail(REVO_EINVAL, "plane pitch smaller than a row%s");
    if (!clean) {
      const Ring& ring = c->rings[m][r->stream_id];
      if (ring.count < c->cfg.k) return fail(REVO_ENOREF, "the stream has fewer than k clean reference frames%s");
      if (ring.H != pl.height || ring.W != pl.width)
        return fail(REVO_EINVAL, "frame size differs from the stream's references%s");
      if (!(m == 0 ? r->rgb_out : r->depth_out)) return fail(REVO_EINVAL, "missing output buffer%s");
    }
  }
  const uint64_t t = c->next_ticket++;
  TicketInfo ti;
  ti.stream_id = r->stream_id;
  ti.frame_index = r->frame_index;
  ti.t_submit = Clock::now();

  if (clean) {
    for (int m = 0; m < 2; ++m)
      if (has[m]) {
        revo_status s = push_clean(c, r, m, ticket);
        if (s != REVO_OK) return s;
      }
    // A push completes as a batch of its own on the copy stream.
    Batch b;
    b.id = c->next_batch++;
    b.lane = -1;
    cudaError_t e = acquire_batch_res(c, b);
    if (e != cudaSuccess) return cuda_status(e, "clean frame batch");
    cudaEventRecord(b.ev_end, c->copy_st);
    cudaEventRecord(c->copy_ev, c->copy_st);
    c->copy_ev_valid = true;
    b.tickets.push_back(t);
    b.size = 1;
    ti.batch = b.id;
    c->batches.emplace(b.id, b);
    c->tickets[t] = ti;
    *ticket = t;
    return REVO_OK;
  }

  Pending p{};
  p.ticket = t;
  p.req = *r;
  p.slot = -1;
  p.t_submit = ti.t_submit;
  if (!r->inputs_on_device || !r->outputs_on_device) {
    p.slot = acquire_slot(c);
    if (p.slot < 0) return fail(REVO_EAGAIN, "no staging slot free%s");
    c->slots[p.slot].busy = true;
  }
  for (int m = 0; m < 2; ++m) {
    p.has[m] = has[m];
    if (!has[m]) continue;
    const revo_plane& pl = m == 0 ? r->rgb : r->depth;
    const Ring& ring = c->rings[m][r->stream_id];
    PlaneJob& j = p.job[m];
    j.H = pl.height;
    j.W = pl.width;
    const int k = c->cfg.k;
    const size_t row = static_cast<size_t>(pl.width) * (m == 0 ? 3 : 2);
    for (int i = 0; i < k; ++i) {
      const int slot = (ring.next + i) % k;  // oldest first
      j.frames[i] = ring.frames + slot * ring.slot_bytes;
      j.pitch[i] = row;
    }
    const int newest = (ring.next + k - 1) % k;
    j.mu_sigma = m == 1 ? ring.stats + 2 * newest : nullptr;
    for (int s = 0; s < c->shape[m].slots(); ++s) {
      const int f = s * c->cfg.tubelet;
      const int64_t idx = f < k ? ring.index[(ring.next + f) % k] : r->frame_index;
      j.taus[s] = static_cast<int>(r->frame_index - idx);
    }
    const uint32_t* mask = m == 0 ? r->rgb_lost_mask : r->depth_lost_mask;
    const size_t mpitch = m == 0 ? r->rgb_mask_pitch_words : r->depth_mask_pitch_words;
    if (r->inputs_on_device) {
      j.frames[k] = pl.data;
      j.pitch[k] = pl.pitch_bytes;
      j.mask = mask;
      j.mask_pitch = mpitch;
    } else {
      Slot& sl = c->slots[p.slot];
      cudaError_t e = cudaMemcpy2DAsync(sl.in[m], row, pl.data, pl.pitch_bytes, row, pl.height,
                                        cudaMemcpyHostToDevice, c->copy_st);
      const size_t mw = (pl.width + 31) / 32;
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(sl.mask[m], mw * 4, mask, mpitch * 4, mw * 4, pl.height, cudaMemcpyHostToDevice,
                              c->copy_st);
      if (e != cudaSuccess) {
        sl.busy = false;
        return cuda_status(e, "input upload");
      }
      j.frames[k] = sl.in[m];
      j.pitch[k] = row;
      j.mask = sl.mask[m];
      j.mask_pitch = mw;
    }
    if (r->outputs_on_device) {
      j.out = m == 0 ? r->rgb_out : r->depth_out;
      j.out_pitch = m == 0 ? r->rgb_out_pitch : r->depth_out_pitch;
      j.values = m == 0 ? r->rgb_values : r->depth_values;
    } else {
      Slot& sl = c->slots[p.slot];
      j.out = sl.out[m];
      j.out_pitch = row;
      j.values = (m == 0 ? r->rgb_values : r->depth_values) ? sl.values[m] : nullptr;
    }
  }
  if (!r->inputs_on_device) {
    cudaEventRecord(c->copy_ev, c->copy_st);
    c->copy_ev_valid = true;
  }
  c->tickets[t] = ti;
  c->pending.push_back(p);
  *ticket = t;
  if (!(r->flags & REVO_HOLD) || static_cast<int>(c->pending.size()) >= c->cfg.max_batch) dispatch(c, false);
  return REVO_OK;
}

revo_status revo_recover_stats(revo_ctx* c, revo_stats* out) {
  if (!c || !out) return fail(REVO_EINVAL, "null argument%s");
  memset(out, 0, sizeof(*out));
  out->device_bytes = c->bytes;
  out->batches = c->n_batches;
  out->graph_replays = c->graph_replays;
  for (int l = 0; l < c->n_lanes; ++l)
    for (int m = 0; m < 2; ++m)
      for (const auto& kv : c->lanes[l].graphs[m]) out->graphs_captured += kv.second.exec != nullptr;
  for (int m = 0; m < 2; ++m)
    if (c->net[m]) {
      out->tuned_shapes += static_cast<int>(c->net[m]->tuned_bn.size());
      out->tuned_wide += c->net[m]->tuned_shapes_256;
      out->tuned_pair += c->net[m]->tuned_shapes_pair;
      out->tuned_timed += c->net[m]->tuned_shapes_128 + c->net[m]->tuned_shapes_256;
    }
  out->pending = static_cast<int>(c->pending.size());
  for (const auto& kv : c->batches) out->in_flight += kv.second.lane >= 0 && !kv.second.done;
  return REVO_OK;
}

revo_status revo_recover_flush(revo_ctx* c) {
  if (!c) return fail(REVO_EINVAL, "null context%s");
  cudaSetDevice(c->device);
  dispatch(c, true);
  return REVO_OK;
}

revo_status revo_recover_poll(revo_ctx* c, uint64_t ticket, int64_t timeout_us, revo_result* out) {
  if (!c) return fail(REVO_EINVAL, "null context%s");
  cudaSetDevice(c->device);
  auto it = c->tickets.find(ticket);
  if (it == c->tickets.end()) return fail(REVO_EINVAL, "unknown ticket%s");
  if (it->second.batch == 0) {
    // Still pending.  A caller that will wait launches it now; a non-blocking
    // poll leaves it to be batched with later arrivals (it starts as soon as a
    // lane is free or max_batch requests are pending).
    dispatch(c, timeout_us != 0);
    if (it->second.batch == 0) return REVO_EAGAIN;
  } else {
    dispatch(c, false);
  }
  Batch& b = c->batches.at(it->second.batch);
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  while (!batch_check(c, b, timeout_us < 0)) {
    if (timeout_us == 0) return REVO_EAGAIN;
    if (Clock::now() >= deadline) return fail(REVO_ETIMEDOUT, "poll timed out%s");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  if (out) {
    out->status = b.status;
    out->stream_id = it->second.stream_id;
    out->frame_index = it->second.frame_index;
    out->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - it->second.t_submit).count();
    out->device_ms = b.device_ms;
    out->batch_size = b.size;
    out->kernel_launches = b.launches;
  }
  const uint64_t bid = it->second.batch;
  auto& tv = b.tickets;
  for (size_t i = 0; i < tv.size(); ++i)
    if (tv[i] == ticket) {
      tv.erase(tv.begin() + i);
      break;
    }
  c->tickets.erase(it);
  retire_if_empty(c, bid);
  dispatch(c, false);
  return REVO_OK;
}

}  // extern "C"
