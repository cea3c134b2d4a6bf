// smcx_batch.cu -- batched execution of many independent lattices (the
// temperature parallelism of Sec. 2.2: simulations at different
// temperatures or compositions share nothing) behind the smcx_batch_* C ABI.
//
// The caller hands over one device arena.  Its head holds the control area
// (device job table, threshold and difference tables per job slot, per-job
// statistics, the work-item order, the persistent plan and per-job phase
// counters, two transfer buffers); the rest is a job heap from which every
// admitted lattice gets its occupancy (first-fit, coalescing free list).  Work items are 32 active
// link cells of one job and colour phase (kernels_cell.cuh), ordered within
// a phase with the jobs whose largest cells have the most trials first.  Two
// schedules run a chunk of S sweeps of every active job: the persistent
// schedule (one cooperative launch following a plan that gives every warp
// fixed ranges of items, the same in every phase; a per-job counter of
// finished items keeps each job's phases in sequence, so a job runs ahead of
// the others as far as its own items allow), or one launch per colour phase
// for all jobs.  With a stream the chunk is captured into a CUDA graph,
// replayed until the job set or the tuning changes.
//
// Tuning (results never depend on it): item shape, schedule and register
// budget are picked online.  While untuned, a run spends its first sweeps on
// short sub-chunks, one per candidate, each timed with CUDA events
// (attempted swaps per millisecond), and keeps the fastest; splitting a
// chunk into sub-chunks does not change any job's trajectory.  Tuning
// restarts when the number of items per phase has moved by more than 2x.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/smcx.h"
#include "kernels.h"
#include "kernels_cell.cuh"
#include "trace.h"

using namespace smcx;

namespace smcx {
// shared with smcx_capi.cu (host helpers of the plain path)
smcx_status batch_fail(smcx_status s, const std::string& msg);
bool host_build_tables(double T, Tables* tab, int* mode, int* s);
Geom host_geom(const smcx_lattice_desc& d, int M, const int m[3]);
void host_layout(const smcx_lattice_desc& d, int M, int* L, int m[3]);
bool host_dtable(const smcx_lattice_desc& d, int M, const int64_t* V, std::vector<uint8_t>* out);
size_t host_occ_bytes(const smcx_lattice_desc& d);
bool host_desc_ok(const smcx_lattice_desc* d, std::string* why);
}  // namespace smcx

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kTabBytes = 4 * kTabWords;
constexpr size_t kDtabBytes = 6 * 6 * 160;  // largest difference table (K = 6, M = 4)

// work items of 32 active cells: {-1, 0} = the next 32 cells of the colour in
// x-fastest order (rows wrap), else boxes (log2 x, log2 y), z = 5 - x - y
constexpr int kTiles[][2] = {{-1, 0}, {3, 2}, {2, 2}, {1, 2}};
constexpr int kTileCount = 4;
// register budgets: 3 or 4 resident blocks of 128 threads per SM
constexpr int kOccCount = 2;
// schedules: 0 = persistent plan (one launch per chunk), 1 = one launch per
// colour phase
constexpr int kSchedCount = 2;
constexpr int kDefaultTile = 0, kDefaultSched = 1, kDefaultOcc = 1;
constexpr uint32_t kTuneSweeps = 2;  // sweeps per timed candidate

using QueueLauncher = cudaError_t (*)(const void*, int, cudaStream_t);
constexpr QueueLauncher kLaunchers[] = {launch_sweep_queue_3, launch_sweep_queue_4};
using PhaseLauncher = cudaError_t (*)(const void*, uint32_t, cudaStream_t);
constexpr PhaseLauncher kPhaseLaunchers[] = {launch_sweep_phase_3, launch_sweep_phase_4};
using QueueBlocks = int (*)();
constexpr QueueBlocks kBlocks[] = {sweep_queue_blocks_3, sweep_queue_blocks_4};
// capacity of the persistent plan: warps of the grid (4 per block) and
// segments (at most two per warp plus one per job, see build_plan)
constexpr uint32_t kPlanWarps = 16384;

size_t aup(size_t v, size_t a) { return (v + a - 1) / a * a; }

// first-fit allocator with coalescing over [0, size)
class Heap {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    total_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = aup(bytes, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = aup(bytes, kAlign);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }
  size_t largest() const {
    size_t s = 0;
    for (auto& kv : free_) s = std::max(s, kv.second);
    return s;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0;
};

struct Job {
  bool used = false, done = false;
  smcx_lattice_desc desc{};
  uint32_t M = 0;
  std::vector<int64_t> V;
  double T = 0;
  uint32_t total = 0, done_sweeps = 0, t = 0;
  int64_t E0 = 0;
  size_t occ_off = 0, occ_bytes = 0;
  uint64_t sites = 0;
  uint32_t A[3] = {1, 1, 1};  // active cells of a colour per axis
  Geom g{};
  int mode = 0, sbin = 0;
};

struct ControlLayout {
  size_t jobs, tabs, dtabs, stats, order, first, seg, wfirst, ctr, qstats, pairs, flag, scratch;
  size_t pairs2, flag2, scratch2;  // the side stream's (admission and results during a chunk)
  size_t heap;
};

ControlLayout control_layout(uint32_t max_jobs, size_t transfer_bytes) {
  ControlLayout c;
  size_t o = 0;
  c.jobs = o;
  o += aup(sizeof(cell::JobDev) * max_jobs, kAlign);
  c.tabs = o;
  o += aup(kTabBytes * max_jobs, kAlign);
  c.dtabs = o;
  o += aup(kDtabBytes * max_jobs, kAlign);
  c.stats = o;
  o += aup(sizeof(unsigned long long) * 8 * max_jobs, kAlign);
  c.order = o;
  o += aup(sizeof(uint32_t) * max_jobs, kAlign);
  c.first = o;
  o += aup(sizeof(uint32_t) * (max_jobs + 1), kAlign);
  c.seg = o;
  o += aup(sizeof(uint4) * (2 * static_cast<size_t>(kPlanWarps) + max_jobs), kAlign);
  c.wfirst = o;
  o += aup(sizeof(uint32_t) * (kPlanWarps + 1), kAlign);
  c.ctr = o;
  o += aup(sizeof(unsigned long long) * (2 + max_jobs), kAlign);
  c.qstats = o;
  o += aup(sizeof(unsigned long long) * 4, kAlign);
  c.pairs = o;
  o += aup(sizeof(unsigned long long) * 4 * 6 * 6, kAlign);
  c.flag = o;
  o += kAlign;
  c.scratch = o;
  o += aup(transfer_bytes, kAlign);
  c.pairs2 = o;
  o += aup(sizeof(unsigned long long) * 4 * 6 * 6, kAlign);
  c.flag2 = o;
  o += kAlign;
  c.scratch2 = o;
  o += aup(transfer_bytes, kAlign);
  c.heap = o;
  return c;
}

uint32_t ceil_shift(uint32_t a, int s) { return (a + (1u << s) - 1) >> s; }

// items of one colour phase of a job for tile index `tile`
uint32_t job_items(const Job& j, int tile, uint32_t* ex, uint32_t* ey) {
  if (kTiles[tile][0] < 0) {
    if (ex) *ex = 0;
    if (ey) *ey = 0;
    return (j.A[0] * j.A[1] * j.A[2] + 31) / 32;
  }
  const int tx = kTiles[tile][0], ty = kTiles[tile][1], tz = 5 - tx - ty;
  const uint32_t x = ceil_shift(j.A[0], tx), y = ceil_shift(j.A[1], ty), z = ceil_shift(j.A[2], tz);
  if (ex) *ex = x;
  if (ey) *ey = y;
  return x * y * z;
}

// Online choice of (tile, schedule, register budget) by coordinate descent:
// every value of one knob with the others at their best so far, knob after
// knob, each configuration measured once; forced knobs are not searched.
struct Tuner {
  static constexpr int kDims = 3;
  static constexpr int kCount[kDims] = {kTileCount, kSchedCount, kOccCount};
  static constexpr int kDefault[kDims] = {kDefaultTile, kDefaultSched, kDefaultOcc};
  int forced[kDims] = {-1, -1, -1};
  int cand[kDims] = {kDefaultTile, kDefaultSched, kDefaultOcc};
  int best[kDims] = {kDefaultTile, kDefaultSched, kDefaultOcc};
  double best_rate = 0;
  bool tuned = false;
  int dim = 0, idx = 0;
  std::map<int, double> seen;  // measured configurations -> attempted swaps per ms
  uint32_t tuned_items = 0;

  int tile() const { return cand[0]; }
  int sched() const { return cand[1]; }
  int occ() const { return cand[2]; }
  static int enc(const int* c) { return (c[0] * 4 + c[1]) * 4 + c[2]; }

  void restart() {
    for (int d = 0; d < kDims; ++d) best[d] = forced[d] >= 0 ? forced[d] : kDefault[d];
    best_rate = 0;
    seen.clear();
    tuned = false;
    dim = idx = 0;
    advance();
  }
  // next configuration to measure, or the best one once all are measured
  void advance() {
    for (; dim < kDims; ++dim, idx = 0) {
      if (forced[dim] >= 0) continue;
      for (; idx < kCount[dim]; ++idx) {
        int c[kDims] = {best[0], best[1], best[2]};
        c[dim] = idx;
        if (seen.count(enc(c))) continue;
        for (int d = 0; d < kDims; ++d) cand[d] = c[d];
        return;
      }
    }
    for (int d = 0; d < kDims; ++d) cand[d] = best[d];
    tuned = true;
  }
  void record(double rate) {
    seen[enc(cand)] = rate;
    if (rate > best_rate) {
      best_rate = rate;
      for (int d = 0; d < kDims; ++d) best[d] = cand[d];
    }
    advance();
  }
};

}  // namespace

struct smcx_batch {
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t stream = nullptr;
  uint32_t max_jobs = 0;
  size_t transfer_bytes = 0;
  ControlLayout cl{};
  Heap heap;
  std::vector<Job> jobs;
  std::vector<uint32_t> done_queue;
  bool dirty = true;  // the job set changed: rebuild the queue order
  int n_sm = 0;
  int grid[kOccCount] = {};  // persistent grid of each register budget
  bool inject_wait_timeout = false;  // SMCX_BATCH_OPT_TEST_WAIT_TIMEOUT
  smcx_status sticky = SMCX_OK;
  std::vector<uint32_t> order;  // active slots (queue order)
  int queue_tile = -1;          // tile the device order/first arrays were built for
  int plan_tile = -1, plan_occ = -1;  // tile and register budget of the device plan
  uint32_t plan_warps = 0;      // warps of the device plan
  uint32_t n_items = 0;         // items of one phase over all active jobs
  Tuner tuner;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraphExec_t graph = nullptr;
  uint32_t graph_sweeps = 0;
  int graph_tile = -1, graph_sched = -1, graph_occ = -1;
  // a chunk launched by smcx_batch_launch and not yet completed: its sweeps,
  // the jobs it runs, the event after its status read-back, the status word
  // (pinned host memory) and the jobs finished by chunks already completed
  // but not yet reported by smcx_batch_wait
  bool in_flight = false;
  uint32_t flight_sweeps = 0;
  std::vector<uint32_t> flight_jobs;
  cudaEvent_t ev_chunk = nullptr;
  unsigned long long* h_status = nullptr;
  uint32_t unreported_fin = 0;
  // side stream: admission and result read-back while a chunk runs
  cudaStream_t side = nullptr;

  uint8_t* at(size_t off) { return arena + off; }
  uint8_t* scratch() { return at(cl.scratch); }
  unsigned int* flag() { return reinterpret_cast<unsigned int*>(at(cl.flag)); }
  unsigned long long* ctr() { return reinterpret_cast<unsigned long long*>(at(cl.ctr)); }
  unsigned long long* qstats() { return reinterpret_cast<unsigned long long*>(at(cl.qstats)); }
  unsigned long long* stats(uint32_t slot) {
    return reinterpret_cast<unsigned long long*>(at(cl.stats)) + 8 * slot;
  }
};

namespace {

smcx_status bcuda(smcx_batch* b, cudaError_t e, const char* what) {
  if (b) b->sticky = SMCX_ECUDA;
  return batch_fail(SMCX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BATCH_CUDA(b, call)                               \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);    \
  } while (0)

smcx_status bcheck(smcx_batch* b) {
  if (!b) return batch_fail(SMCX_EINVAL, "null batch");
  if (b->sticky != SMCX_OK) return batch_fail(SMCX_ESTATE, "batch is in an error state");
  return SMCX_OK;
}

void drop_graph(smcx_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_sweeps = 0;
  b->graph_tile = b->graph_sched = b->graph_occ = -1;
}

// trials of the largest link cell of a job: the length of its chain of
// dependent trials in one colour phase
uint32_t longest_cell(const Job& j) {
  uint32_t t = static_cast<uint32_t>(j.g.nb);
  for (int d = 0; d < 3; ++d) t *= (j.desc.n[d] + j.g.m[d] - 1) / j.g.m[d];
  return t;
}

// queue order and the first item of each job within a phase, for tile
// `tile`: jobs with the longest chains of dependent trials first (their
// phases bound the chunk), jobs of one kernel variant together (neighbouring
// blocks then run the same code), then the larger ones, then by slot
smcx_status build_queue(smcx_batch* b, int tile) {
  b->order.clear();
  for (uint32_t slot = 0; slot < b->max_jobs; ++slot) {
    const Job& j = b->jobs[slot];
    if (j.used && !j.done) b->order.push_back(slot);
  }
  std::stable_sort(b->order.begin(), b->order.end(), [&](uint32_t x, uint32_t y) {
    const Job& a = b->jobs[x];
    const Job& c = b->jobs[y];
    const uint32_t la = longest_cell(a), lc = longest_cell(c);
    if (la != lc) return la > lc;
    const int va = cell_variant(a.g), vc = cell_variant(c.g);  // neighbouring blocks, same code
    if (va != vc) return va < vc;
    return job_items(a, tile, nullptr, nullptr) > job_items(c, tile, nullptr, nullptr);
  });
  std::vector<uint32_t> first;
  uint64_t n = 0;
  for (uint32_t slot : b->order) {
    first.push_back(static_cast<uint32_t>(n));
    n += job_items(b->jobs[slot], tile, nullptr, nullptr);
  }
  first.push_back(static_cast<uint32_t>(n));
  if (n >= (1ull << 31)) return batch_fail(SMCX_EBUDGET, "too many work items per phase");
  b->n_items = static_cast<uint32_t>(n);
  if (!b->order.empty()) {
    BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.order), b->order.data(),
                                  sizeof(uint32_t) * b->order.size(), cudaMemcpyHostToDevice,
                                  b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.first), first.data(), sizeof(uint32_t) * first.size(),
                                  cudaMemcpyHostToDevice, b->stream));
  }
  b->queue_tile = tile;
  b->plan_tile = -1;
  b->dirty = false;
  drop_graph(b);
  return SMCX_OK;
}

// The persistent schedule's plan for tile `tile` on the grid of register
// budget `occ`: every active job's items of a phase cut into ranges and each
// range given to the warp with the least work so far (jobs in queue order,
// the longest chains first), work = items x the job's longest cell.  A range
// holds r = max(1, tau / c) items of a job whose largest cell has c trials,
// tau = max(largest c, total work / warps), so no warp's range outlasts the
// longest chain and there are at most 2 x warps + jobs ranges.  The same
// plan serves every phase, so a warp returns to the same cells.
smcx_status build_plan(smcx_batch* b, int tile, int occ) {
  const uint32_t W = std::min<uint32_t>(static_cast<uint32_t>(b->grid[occ]) * cell::kQueueWarps,
                                        kPlanWarps);
  uint64_t total = 0, tau = 1;
  for (uint32_t slot : b->order) {
    const Job& j = b->jobs[slot];
    const uint64_t c = longest_cell(j);
    total += c * job_items(j, tile, nullptr, nullptr);
    tau = std::max(tau, c);
  }
  tau = std::max<uint64_t>(tau, (total + W - 1) / W);
  std::vector<std::vector<uint4>> per(W);
  // least-loaded warp first (ties: lower index)
  std::vector<std::pair<uint64_t, uint32_t>> heap;
  heap.reserve(W);
  for (uint32_t w = 0; w < W; ++w) heap.emplace_back(0, w);
  auto later = [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) {
    return x > y;
  };
  size_t n_seg = 0;
  for (uint32_t slot : b->order) {
    const Job& j = b->jobs[slot];
    const uint64_t c = longest_cell(j);
    const uint32_t items = job_items(j, tile, nullptr, nullptr);
    const uint32_t r = static_cast<uint32_t>(std::max<uint64_t>(1, tau / c));
    for (uint32_t i0 = 0; i0 < items; i0 += r) {
      const uint32_t n = std::min(r, items - i0);
      std::pop_heap(heap.begin(), heap.end(), later);
      auto& h = heap.back();
      per[h.second].push_back(make_uint4(slot, i0, n, 0));
      h.first += c * n;
      std::push_heap(heap.begin(), heap.end(), later);
      ++n_seg;
    }
  }
  if (n_seg > 2 * static_cast<size_t>(kPlanWarps) + b->max_jobs)
    return batch_fail(SMCX_EBUDGET, "persistent plan larger than its capacity");
  std::vector<uint4> seg;
  std::vector<uint32_t> wfirst;
  seg.reserve(n_seg);
  wfirst.reserve(W + 1);
  for (uint32_t w = 0; w < W; ++w) {
    wfirst.push_back(static_cast<uint32_t>(seg.size()));
    seg.insert(seg.end(), per[w].begin(), per[w].end());
  }
  wfirst.push_back(static_cast<uint32_t>(seg.size()));
  if (!seg.empty())
    BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.seg), seg.data(), sizeof(uint4) * seg.size(),
                                  cudaMemcpyHostToDevice, b->stream));
  BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.wfirst), wfirst.data(),
                                sizeof(uint32_t) * wfirst.size(), cudaMemcpyHostToDevice,
                                b->stream));
  // the host vectors must outlive the copies
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  b->plan_tile = tile;
  b->plan_occ = occ;
  b->plan_warps = W;
  drop_graph(b);
  return SMCX_OK;
}

// `sweeps` sweeps of every active job: counter reset + one launch of the
// persistent kernel (sched 0), or one launch per colour phase (sched 1)
smcx_status enqueue_chunk(smcx_batch* b, uint32_t sweeps, int tile, int sched, int occ) {
  cell::QueueArgs q{};
  q.jobs = reinterpret_cast<const cell::JobDev*>(b->at(b->cl.jobs));
  q.order = reinterpret_cast<const uint32_t*>(b->at(b->cl.order));
  q.first = reinterpret_cast<const uint32_t*>(b->at(b->cl.first));
  q.n_active = static_cast<uint32_t>(b->order.size());
  q.n_items = b->n_items;
  q.seg = reinterpret_cast<const uint4*>(b->at(b->cl.seg));
  q.wfirst = reinterpret_cast<const uint32_t*>(b->at(b->cl.wfirst));
  q.n_warps = b->plan_warps;
  q.n_ph = 8 * sweeps;
  q.ctr = b->ctr();
  q.qstats = b->qstats();
  q.tx = kTiles[tile][0];
  q.ty = kTiles[tile][1];
  if (sched == 0) {
    BATCH_CUDA(b, cudaMemsetAsync(b->ctr(), 0, sizeof(unsigned long long) * (2 + b->max_jobs),
                                  b->stream));
    const int grid = static_cast<int>((b->plan_warps + cell::kQueueWarps - 1) / cell::kQueueWarps);
    BATCH_CUDA(b, kLaunchers[occ](&q, grid, b->stream));
  } else {
    for (uint32_t ph = 0; ph < 8 * sweeps; ++ph)
      BATCH_CUDA(b, kPhaseLaunchers[occ](&q, ph, b->stream));
  }
  return SMCX_OK;
}

// Advances the listed jobs by one completed chunk of `sweeps` sweeps and
// queues those that finished; returns how many finished.
uint32_t advance_jobs(smcx_batch* b, const std::vector<uint32_t>& slots, uint32_t sweeps) {
  uint32_t fin = 0;
  for (uint32_t slot : slots) {
    Job& j = b->jobs[slot];
    const uint32_t ran = std::min(sweeps, j.total - j.done_sweeps);
    j.done_sweeps += ran;
    j.t += ran;
    if (j.done_sweeps == j.total) {
      j.done = true;
      b->done_queue.push_back(slot);
      b->dirty = true;
      ++fin;
    }
  }
  return fin;
}

// Runs `sweeps` sweeps of every active job with (tile, sched, occ);
// graph-captured when `use_graph` and a stream is bound.  *trials =
// attempted swaps, *ms = device time (when ms != NULL, timed with events).
// async: enqueue only; complete_chunk finishes it.
smcx_status run_sweeps(smcx_batch* b, uint32_t sweeps, int tile, int sched, int occ,
                       bool use_graph, uint32_t* n_finished, uint64_t* trials, float* ms,
                       bool async = false) {
  TraceRange trace(sched == 0 ? "smcx_batch_chunk_persistent" : "smcx_batch_chunk_phases");
  smcx_status s;
  if (b->dirty || b->queue_tile != tile) {
    s = build_queue(b, tile);
    if (s != SMCX_OK) return s;
  }
  if (sched == 0 && (b->plan_tile != tile || b->plan_occ != occ)) {
    s = build_plan(b, tile, occ);
    if (s != SMCX_OK) return s;
  }
  std::vector<uint8_t> table(sizeof(cell::JobDev) * b->max_jobs, 0);
  uint32_t s_max = 0;
  uint64_t tr = 0;
  for (uint32_t slot : b->order) {
    const Job& j = b->jobs[slot];
    cell::JobDev jd{};
    jd.g = j.g;
    jd.occ = b->at(j.occ_off);
    jd.dtab = b->at(b->cl.dtabs) + kDtabBytes * slot;
    jd.tab = reinterpret_cast<const uint32_t*>(b->at(b->cl.tabs) + kTabBytes * slot);
    jd.stats = b->stats(slot);
    jd.t0 = j.t;
    jd.sweeps = std::min(sweeps, j.total - j.done_sweeps);
    jd.mode = j.mode;
    jd.sbin = j.sbin;
    jd.no_shift = (j.desc.flags & SMCX_NO_SHIFT) ? 1 : 0;
    jd.variant = cell_variant(j.g);
    jd.items = job_items(j, tile, &jd.ex, &jd.ey);
    for (int d = 0; d < 3; ++d) jd.A[d] = j.A[d];
    std::memcpy(table.data() + sizeof(cell::JobDev) * slot, &jd, sizeof(jd));
    s_max = std::max(s_max, jd.sweeps);
    tr += j.sites * jd.sweeps;
  }
  if (b->inject_wait_timeout && sched == 0 && !b->order.empty()) {
    // testing aid: the first job's phase counters now fall one item short of
    // what its next phases wait for, so those (bounded) waits give up
    reinterpret_cast<cell::JobDev*>(table.data() + sizeof(cell::JobDev) * b->order[0])->items += 1;
    b->inject_wait_timeout = false;
    use_graph = false;
  }
  if (n_finished) *n_finished = 0;
  if (trials) *trials = tr;
  if (ms) *ms = 0;
  if (s_max == 0) return SMCX_OK;
  BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.jobs), table.data(), table.size(),
                                cudaMemcpyHostToDevice, b->stream));
  if (ms) BATCH_CUDA(b, cudaEventRecord(b->ev[0], b->stream));
  if (use_graph && b->stream) {
    if (!b->graph || b->graph_sweeps != s_max || b->graph_tile != tile || b->graph_sched != sched ||
        b->graph_occ != occ) {
      drop_graph(b);
      cudaGraph_t gr = nullptr;
      BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      s = enqueue_chunk(b, s_max, tile, sched, occ);
      cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
      if (s != SMCX_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s;
      }
      if (e != cudaSuccess) return bcuda(b, e, "graph capture");
      e = cudaGraphInstantiate(&b->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
      b->graph_sweeps = s_max;
      b->graph_tile = tile;
      b->graph_sched = sched;
      b->graph_occ = occ;
    }
    BATCH_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
  } else {
    s = enqueue_chunk(b, s_max, tile, sched, occ);
    if (s != SMCX_OK) return s;
  }
  if (ms) BATCH_CUDA(b, cudaEventRecord(b->ev[1], b->stream));
  if (async) {
    // the status word comes back with the chunk; smcx_batch_wait reads it
    // and advances the jobs
    BATCH_CUDA(b, cudaMemcpyAsync(b->h_status, b->ctr() + 1, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaEventRecord(b->ev_chunk, b->stream));
    b->in_flight = true;
    b->flight_sweeps = sweeps;
    b->flight_jobs = b->order;
    return SMCX_OK;
  }
  unsigned long long status = 0;
  BATCH_CUDA(b, cudaMemcpyAsync(&status, b->ctr() + 1, sizeof(status), cudaMemcpyDeviceToHost,
                                b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  if (status != 0) {
    b->sticky = SMCX_ETIMEOUT;
    return batch_fail(SMCX_ETIMEOUT, "batched sweep: a wait for a job's previous phase gave up");
  }
  if (ms) BATCH_CUDA(b, cudaEventElapsedTime(ms, b->ev[0], b->ev[1]));
  const uint32_t fin = advance_jobs(b, b->order, sweeps);
  if (n_finished) *n_finished = fin;
  return SMCX_OK;
}

// Completes the chunk in flight (if any): waits for it, checks its status
// and advances its jobs; the jobs it finished are counted for the next
// smcx_batch_wait.
smcx_status complete_chunk(smcx_batch* b) {
  if (!b->in_flight) return SMCX_OK;
  b->in_flight = false;
  BATCH_CUDA(b, cudaEventSynchronize(b->ev_chunk));
  if (*b->h_status != 0) {
    b->sticky = SMCX_ETIMEOUT;
    return batch_fail(SMCX_ETIMEOUT, "batched sweep: a wait for a job's previous phase gave up");
  }
  b->unreported_fin += advance_jobs(b, b->flight_jobs, b->flight_sweeps);
  b->flight_jobs.clear();
  return SMCX_OK;
}

smcx_status job_energy(smcx_batch* b, Job& j, int64_t* e, cudaStream_t st, size_t pairs_off) {
  const Geom& g = j.g;
  const size_t kmax = g.K <= 5 ? 5 : 6;
  const size_t n_h = static_cast<size_t>(j.M) * kmax * kmax;
  unsigned long long* d_pairs = reinterpret_cast<unsigned long long*>(b->at(pairs_off));
  BATCH_CUDA(b, cudaMemsetAsync(d_pairs, 0, sizeof(uint64_t) * n_h, st));
  BATCH_CUDA(b, launch_pair_count_tiled(g, static_cast<int>(j.M), b->at(j.occ_off), d_pairs,
                                        b->n_sm, st, false));
  std::vector<uint64_t> h(n_h);
  BATCH_CUDA(b, cudaMemcpyAsync(h.data(), d_pairs, sizeof(uint64_t) * n_h, cudaMemcpyDeviceToHost,
                                st));
  BATCH_CUDA(b, cudaStreamSynchronize(st));
  const size_t K = g.K;
  __int128 acc = 0;
  for (size_t m = 0; m < j.M; ++m)
    for (size_t p = 0; p < K; ++p)
      for (size_t q = 0; q < K; ++q) {
        const uint64_t n = h[(m * kmax + p) * kmax + q] + h[(m * kmax + q) * kmax + p];
        acc += static_cast<__int128>(n) * j.V[(m * K + p) * K + q];
      }
  acc /= 2;
  if (acc > static_cast<__int128>(INT64_MAX) || acc < static_cast<__int128>(INT64_MIN))
    return batch_fail(SMCX_EOVERFLOW, "energy does not fit int64");
  *e = static_cast<int64_t>(acc);
  return SMCX_OK;
}

}  // namespace

extern "C" {

size_t smcx_batch_control_bytes(uint32_t max_jobs, size_t transfer_bytes) {
  if (max_jobs == 0) return 0;
  return control_layout(max_jobs, transfer_bytes).heap;
}

size_t smcx_batch_job_bytes(const smcx_lattice_desc* desc) {
  std::string why;
  if (!host_desc_ok(desc, &why)) return 0;
  return aup(host_occ_bytes(*desc), kAlign);
}

smcx_status smcx_batch_create(uint32_t max_jobs, void* d_arena, size_t arena_bytes,
                              size_t transfer_bytes, void* cuda_stream, smcx_batch** out) {
  if (!out) return batch_fail(SMCX_EINVAL, "null out pointer");
  *out = nullptr;
  if (max_jobs == 0 || !d_arena) return batch_fail(SMCX_EINVAL, "max_jobs and arena required");
  if (reinterpret_cast<uintptr_t>(d_arena) % kAlign)
    return batch_fail(SMCX_EINVAL, "arena must be 256-byte aligned");
  const ControlLayout cl = control_layout(max_jobs, transfer_bytes);
  if (arena_bytes < cl.heap) return batch_fail(SMCX_ENOMEM, "arena smaller than the control area");
  auto* b = new smcx_batch();
  b->arena = static_cast<uint8_t*>(d_arena);
  b->arena_bytes = arena_bytes;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->max_jobs = max_jobs;
  b->transfer_bytes = transfer_bytes;
  b->cl = cl;
  b->heap.reset(arena_bytes - cl.heap);
  b->jobs.resize(max_jobs);
  b->tuner.restart();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->at(cl.stats), 0, sizeof(unsigned long long) * 8 * max_jobs, b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->at(cl.qstats), 0, sizeof(unsigned long long) * 4, b->stream);
  if (e == cudaSuccess)  // status word and per-job counters (word 0 unused)
    e = cudaMemsetAsync(b->at(cl.ctr), 0, sizeof(unsigned long long) * (2 + max_jobs), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  for (int o = 0; o < kOccCount && e == cudaSuccess; ++o) {
    const int per_sm = kBlocks[o]();
    if (per_sm < 1) e = cudaErrorInvalidConfiguration;
    b->grid[o] = b->n_sm * per_sm;
  }
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_chunk, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_status),
                                          sizeof(unsigned long long), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    for (cudaEvent_t ev : b->ev)
      if (ev) cudaEventDestroy(ev);
    if (b->ev_chunk) cudaEventDestroy(b->ev_chunk);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
    return batch_fail(SMCX_ECUDA, std::string("batch create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return SMCX_OK;
}

smcx_status smcx_batch_add(smcx_batch* b, const smcx_lattice_desc* desc, const uint8_t* h_init,
                           uint32_t n_shells, const int64_t* v_q, double T, uint32_t n_sweeps,
                           uint32_t* job_id) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  std::string why;
  if (!host_desc_ok(desc, &why)) return batch_fail(SMCX_EINVAL, why);
  if (!h_init || !v_q || !job_id) return batch_fail(SMCX_EINVAL, "null argument");
  if (desc->pack_bits != 8) return batch_fail(SMCX_EINVAL, "batched jobs use 8-bit storage");
  if (desc->n_species > 6) return batch_fail(SMCX_EINVAL, "batched jobs need n_species <= 6");
  if (n_shells < 2 || n_shells > 4) return batch_fail(SMCX_EINVAL, "batched jobs need 2..4 shells");
  for (int d = 0; d < 3; ++d)
    if (desc->n[d] < 4) return batch_fail(SMCX_EINVAL, "batched jobs need n >= 4 in every dimension");
  if (std::isnan(T) || T < 0) return batch_fail(SMCX_EINVAL, "temperature must be >= 0");
  const size_t K = desc->n_species;
  for (size_t m = 0; m < n_shells; ++m)
    for (size_t p = 0; p < K; ++p)
      for (size_t q = 0; q < K; ++q)
        if (v_q[(m * K + p) * K + q] != v_q[(m * K + q) * K + p])
          return batch_fail(SMCX_EINVAL, "EPI table is not symmetric");
  const uint64_t N = static_cast<uint64_t>(desc->kind == SMCX_BCC ? 2 : 4) * desc->n[0] *
                     desc->n[1] * desc->n[2];
  if (N > b->transfer_bytes) return batch_fail(SMCX_EINVAL, "lattice larger than the transfer buffer");
  std::vector<uint8_t> dtab;
  if (!host_dtable(*desc, static_cast<int>(n_shells), v_q, &dtab))
    return batch_fail(SMCX_EINVAL, "EPI differences do not fit the batched kernel (|V| too large)");
  uint32_t slot = b->max_jobs;
  for (uint32_t i = 0; i < b->max_jobs; ++i)
    if (!b->jobs[i].used) {
      slot = i;
      break;
    }
  if (slot == b->max_jobs) return batch_fail(SMCX_EBUDGET, "no free job slot");
  const size_t ob = host_occ_bytes(*desc);
  size_t off = 0;
  if (!b->heap.alloc(ob, &off)) return batch_fail(SMCX_EBUDGET, "arena has no room for the lattice");
  Job j;
  j.used = true;
  j.desc = *desc;
  j.M = n_shells;
  j.V.assign(v_q, v_q + n_shells * K * K);
  j.T = T;
  j.total = n_sweeps;
  j.occ_off = b->cl.heap + off;
  j.occ_bytes = ob;
  int L = 0, m[3];
  host_layout(*desc, static_cast<int>(n_shells), &L, m);
  j.g = host_geom(*desc, static_cast<int>(n_shells), m);
  j.sites = N;
  for (int d = 0; d < 3; ++d) j.A[d] = m[d] == 1 ? 1u : static_cast<uint32_t>(m[d] / 2);
  Tables tab;
  host_build_tables(T, &tab, &j.mode, &j.sbin);
  auto fail_release = [&](smcx_status st) {
    b->heap.release(off, ob);
    return st;
  };
  // upload: canonical -> transfer buffer -> validated -> device layout.
  // While a chunk runs this goes through the side stream and its own
  // transfer buffer, flag and pair counts: the new job's heap block and slot
  // are not in the running chunk, so the two overlap on the device.
  const bool side = b->in_flight;
  cudaStream_t st = side ? b->side : b->stream;
  uint8_t* scr = b->at(side ? b->cl.scratch2 : b->cl.scratch);
  unsigned int* flg = reinterpret_cast<unsigned int*>(b->at(side ? b->cl.flag2 : b->cl.flag));
  cudaError_t e = cudaMemcpyAsync(scr, h_init, N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flg, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = launch_validate(scr, N, desc->n_species, flg, b->n_sm, st);
  unsigned int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flg, sizeof(bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch upload"));
  if (bad) return fail_release(batch_fail(SMCX_EINVAL, "species id >= n_species in occupancy"));
  e = launch_canon_to_dev(j.g, scr, b->at(j.occ_off), static_cast<uint32_t>(N / j.g.nb), b->n_sm,
                          st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->at(b->cl.tabs) + kTabBytes * slot, tab.w, kTabBytes,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->at(b->cl.dtabs) + kDtabBytes * slot, dtab.data(), dtab.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->stats(slot), 0, sizeof(unsigned long long) * 8, st);
  if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch add"));
  s = job_energy(b, j, &j.E0, st, side ? b->cl.pairs2 : b->cl.pairs);
  if (s != SMCX_OK) return fail_release(s);
  b->jobs[slot] = j;
  if (n_sweeps == 0) {
    b->jobs[slot].done = true;
    b->done_queue.push_back(slot);
  }
  b->dirty = true;
  *job_id = slot;
  return SMCX_OK;
}

smcx_status smcx_batch_run(smcx_batch* b, uint32_t chunk_sweeps, uint32_t* n_finished) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (chunk_sweeps == 0) return batch_fail(SMCX_EINVAL, "chunk_sweeps must be > 0");
  if (n_finished) *n_finished = 0;
  s = complete_chunk(b);
  if (s != SMCX_OK) return s;
  if (n_finished) *n_finished = b->unreported_fin;
  b->unreported_fin = 0;
  uint32_t left = chunk_sweeps;
  while (left > 0) {
    if (b->dirty) {
      // re-tune when the work per phase has moved by more than 2x
      uint64_t items = 0;
      for (const Job& j : b->jobs)
        if (j.used && !j.done) items += job_items(j, b->tuner.best[0], nullptr, nullptr);
      const uint64_t ref = b->tuner.tuned_items;
      if (b->tuner.tuned && items > 0 && (items > 2 * ref || 2 * items < ref)) b->tuner.restart();
    }
    uint32_t fin = 0;
    if (!b->tuner.tuned) {
      const uint32_t ts = std::min(left, kTuneSweeps);
      uint64_t trials = 0;
      float ms = 0;
      s = run_sweeps(b, ts, b->tuner.tile(), b->tuner.sched(), b->tuner.occ(), false, &fin, &trials,
                     &ms);
      if (s != SMCX_OK) return s;
      left -= ts;
      if (trials == 0) break;  // no active job
      b->tuner.record(ms > 0 ? static_cast<double>(trials) / ms : 0.0);
      if (b->tuner.tuned) {
        uint64_t items = 0;
        for (const Job& j : b->jobs)
          if (j.used && !j.done) items += job_items(j, b->tuner.tile(), nullptr, nullptr);
        b->tuner.tuned_items = static_cast<uint32_t>(std::min<uint64_t>(items, 0xFFFFFFFFu));
      }
    } else {
      uint64_t trials = 0;
      s = run_sweeps(b, left, b->tuner.tile(), b->tuner.sched(), b->tuner.occ(), true, &fin, &trials,
                     nullptr);
      if (s != SMCX_OK) return s;
      left = 0;
    }
    if (n_finished) *n_finished += fin;
  }
  return SMCX_OK;
}

smcx_status smcx_batch_launch(smcx_batch* b, uint32_t chunk_sweeps) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (chunk_sweeps == 0) return batch_fail(SMCX_EINVAL, "chunk_sweeps must be > 0");
  s = complete_chunk(b);
  if (s != SMCX_OK) return s;
  // the jobs admitted through the side stream are on the device
  if (b->side) BATCH_CUDA(b, cudaStreamSynchronize(b->side));
  bool retune = false;
  if (b->dirty && b->tuner.tuned) {
    uint64_t items = 0;
    for (const Job& j : b->jobs)
      if (j.used && !j.done) items += job_items(j, b->tuner.best[0], nullptr, nullptr);
    const uint64_t ref = b->tuner.tuned_items;
    retune = items > 0 && (items > 2 * ref || 2 * items < ref);
  }
  if (!b->tuner.tuned || retune || !b->stream) {
    // tuning times its candidates, which needs the chunk finished: run it
    // here (the finished jobs are reported by the next smcx_batch_wait)
    uint32_t fin = 0;
    s = smcx_batch_run(b, chunk_sweeps, &fin);
    b->unreported_fin += fin;
    return s;
  }
  uint64_t trials = 0;
  return run_sweeps(b, chunk_sweeps, b->tuner.tile(), b->tuner.sched(), b->tuner.occ(), true,
                    nullptr, &trials, nullptr, true);
}

smcx_status smcx_batch_wait(smcx_batch* b, uint32_t* n_finished) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  s = complete_chunk(b);
  if (s != SMCX_OK) return s;
  if (n_finished) *n_finished = b->unreported_fin;
  b->unreported_fin = 0;
  return SMCX_OK;
}

smcx_status smcx_batch_set_option(smcx_batch* b, uint32_t key, int64_t value) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (key == SMCX_BATCH_OPT_TEST_WAIT_TIMEOUT) {
    b->inject_wait_timeout = value != 0;
    return SMCX_OK;
  }
  int d = -1;
  if (key == SMCX_BATCH_OPT_TILE) d = 0;
  else if (key == SMCX_BATCH_OPT_SCHEDULE) d = 1;
  else if (key == SMCX_BATCH_OPT_OCCUPANCY) d = 2;
  if (d < 0) return batch_fail(SMCX_EINVAL, "unknown batch option");
  if (value < -1 || value >= Tuner::kCount[d])
    return batch_fail(SMCX_EINVAL, "batch option value out of range");
  b->tuner.forced[d] = static_cast<int>(value);
  b->tuner.restart();
  return SMCX_OK;
}

smcx_status smcx_batch_tuning(smcx_batch* b, int32_t* tile, int32_t* schedule, int32_t* occupancy,
                              uint32_t* tuned) {
  if (!b) return batch_fail(SMCX_EINVAL, "null batch");
  const bool t = b->tuner.tuned;
  if (tile) *tile = t ? b->tuner.tile() : -1;
  if (schedule) *schedule = t ? b->tuner.sched() : -1;
  if (occupancy) *occupancy = t ? b->tuner.occ() : -1;
  if (tuned) *tuned = t ? 1u : 0u;
  return SMCX_OK;
}

// Replica exchange (parallel tempering, Sec. 2.2, Eqs. 6-7) between jobs
// that simulate one system at different temperatures: ladder[k] is the job at
// the k-th temperature.  Round r attempts the neighbour pairs (k, k+1),
// k = r mod 2, r mod 2 + 2, ...; Delta = (beta_k - beta_{k+1}) (E_k -
// E_{k+1}) with beta = 1/(k_B T) and the jobs' exact running energies
// (difference in integers, scaled by 2^-32 to eV); a pair is accepted iff
// Delta >= 0 or u < exp(Delta), u from the 53 high bits of words 0, 1 of
// Philox(counter = (k, r, 0, 3), key = seed).  An accepted pair exchanges the
// two jobs' temperatures (tables included) and its ladder entries.
smcx_status smcx_batch_exchange(smcx_batch* b, uint32_t* ladder, uint32_t n, uint64_t seed,
                                uint32_t round, uint32_t* n_accepted) {
  TraceRange trace("smcx_batch_exchange");
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  s = complete_chunk(b);  // the energies and tables belong to completed sweeps
  if (s != SMCX_OK) return s;
  if (!ladder || n < 2) return batch_fail(SMCX_EINVAL, "exchange needs a ladder of >= 2 jobs");
  std::vector<bool> seen(b->max_jobs, false);
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t id = ladder[k];
    if (id >= b->max_jobs || !b->jobs[id].used || seen[id])
      return batch_fail(SMCX_EINVAL, "exchange: unknown or repeated job id");
    seen[id] = true;
    const Job& j = b->jobs[id];
    const Job& j0 = b->jobs[ladder[0]];
    if (!(j.T > 0) || std::isinf(j.T))
      return batch_fail(SMCX_EINVAL, "exchange: temperatures must be finite and > 0");
    if (j.desc.kind != j0.desc.kind || j.desc.n_species != j0.desc.n_species || j.M != j0.M ||
        j.desc.n[0] != j0.desc.n[0] || j.desc.n[1] != j0.desc.n[1] || j.desc.n[2] != j0.desc.n[2] ||
        j.V != j0.V)
      return batch_fail(SMCX_EINVAL, "exchange: the jobs do not simulate the same system");
  }
  std::vector<unsigned long long> st(8ull * b->max_jobs);
  BATCH_CUDA(b, cudaMemcpyAsync(st.data(), b->stats(0), sizeof(unsigned long long) * st.size(),
                                cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  auto energy = [&](uint32_t id) {
    return b->jobs[id].E0 + static_cast<int64_t>(st[8ull * id + kStatCum + 3]);
  };
  constexpr double kB = 8.617333262e-5;  // eV/K, as for the acceptance tables
  uint32_t acc = 0;
  for (uint32_t k = round % 2; k + 1 < n; k += 2) {
    Job& a = b->jobs[ladder[k]];
    Job& c = b->jobs[ladder[k + 1]];
    const double beta_a = 1.0 / (kB * a.T), beta_c = 1.0 / (kB * c.T);
    const __int128 diff = static_cast<__int128>(energy(ladder[k])) - energy(ladder[k + 1]);
    const double delta = (beta_a - beta_c) * std::ldexp(static_cast<double>(diff), -32);
    const U4 w = philox4x32_10(k, round, 0u, 3u, static_cast<uint32_t>(seed),
                               static_cast<uint32_t>(seed >> 32));
    const double u =
        std::ldexp(static_cast<double>(((static_cast<uint64_t>(w.x) << 32) | w.y) >> 11), -53);
    if (!(delta >= 0.0 || u < std::exp(delta))) continue;
    std::swap(a.T, c.T);
    for (uint32_t id : {ladder[k], ladder[k + 1]}) {
      Job& j = b->jobs[id];
      Tables tab;
      host_build_tables(j.T, &tab, &j.mode, &j.sbin);
      BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.tabs) + kTabBytes * id, tab.w, kTabBytes,
                                    cudaMemcpyHostToDevice, b->stream));
    }
    std::swap(ladder[k], ladder[k + 1]);
    ++acc;
  }
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));  // the tables' host copies go out of scope
  if (n_accepted) *n_accepted = acc;
  return SMCX_OK;
}

smcx_status smcx_batch_temperature(smcx_batch* b, uint32_t job_id, double* T) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (job_id >= b->max_jobs || !b->jobs[job_id].used || !T)
    return batch_fail(SMCX_EINVAL, "unknown job or null output");
  *T = b->jobs[job_id].T;
  return SMCX_OK;
}

smcx_status smcx_batch_queue_stats(smcx_batch* b, uint64_t* out) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  s = complete_chunk(b);
  if (s != SMCX_OK) return s;
  if (!out) return batch_fail(SMCX_EINVAL, "null output");
  unsigned long long h[3];
  BATCH_CUDA(b, cudaMemcpyAsync(h, b->qstats(), sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  for (int i = 0; i < 3; ++i) out[i] = h[i];
  return SMCX_OK;
}

smcx_status smcx_batch_tile_shape(uint32_t i, uint32_t* cells_xyz) {
  if (i >= static_cast<uint32_t>(kTileCount) || !cells_xyz)
    return batch_fail(SMCX_EINVAL, "bad batch tile request");
  if (kTiles[i][0] < 0) {  // 32 consecutive cells, x fastest
    cells_xyz[0] = 32;
    cells_xyz[1] = cells_xyz[2] = 1;
    return SMCX_OK;
  }
  cells_xyz[0] = 1u << kTiles[i][0];
  cells_xyz[1] = 1u << kTiles[i][1];
  cells_xyz[2] = 1u << (5 - kTiles[i][0] - kTiles[i][1]);
  return SMCX_OK;
}

smcx_status smcx_batch_poll(smcx_batch* b, uint32_t* ids, uint32_t cap, uint32_t* n) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (!n || (cap && !ids)) return batch_fail(SMCX_EINVAL, "null argument");
  const uint32_t k = std::min<uint32_t>(cap, static_cast<uint32_t>(b->done_queue.size()));
  for (uint32_t i = 0; i < k; ++i) ids[i] = b->done_queue[i];
  b->done_queue.erase(b->done_queue.begin(), b->done_queue.begin() + k);
  *n = k;
  return SMCX_OK;
}

smcx_status smcx_batch_result(smcx_batch* b, uint32_t job_id, uint8_t* h_occ,
                              smcx_sweep_stats* totals, int64_t* e_run, uint32_t* sweeps_done) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (job_id >= b->max_jobs || !b->jobs[job_id].used) return batch_fail(SMCX_EINVAL, "unknown job");
  Job& j = b->jobs[job_id];
  if (!j.done) {  // its occupancy and statistics may be those of a running chunk
    s = complete_chunk(b);
    if (s != SMCX_OK) return s;
  }
  // a finished job is in no chunk: while one runs, read it back through the
  // side stream and its own transfer buffer
  const bool side = b->in_flight;
  cudaStream_t rs = side ? b->side : b->stream;
  uint8_t* scr = b->at(side ? b->cl.scratch2 : b->cl.scratch);
  if (h_occ) {
    const uint64_t N = static_cast<uint64_t>(j.g.nb) * j.g.n[0] * j.g.n[1] * j.g.n[2];
    BATCH_CUDA(b, launch_dev_to_canon(j.g, b->at(j.occ_off), scr, static_cast<uint32_t>(N / j.g.nb),
                                      b->n_sm, rs));
    BATCH_CUDA(b, cudaMemcpyAsync(h_occ, scr, N, cudaMemcpyDeviceToHost, rs));
  }
  unsigned long long st[8];
  BATCH_CUDA(b, cudaMemcpyAsync(st, b->stats(job_id), sizeof(st), cudaMemcpyDeviceToHost, rs));
  BATCH_CUDA(b, cudaStreamSynchronize(rs));
  if (totals) {
    totals->attempts = st[4];
    totals->unlike = st[5];
    totals->accepted = st[6];
    totals->sum_dE_q = static_cast<int64_t>(st[7]);
  }
  if (e_run) *e_run = j.E0 + static_cast<int64_t>(st[7]);
  if (sweeps_done) *sweeps_done = j.done_sweeps;
  return SMCX_OK;
}

smcx_status smcx_batch_remove(smcx_batch* b, uint32_t job_id) {
  smcx_status s = bcheck(b);
  if (s != SMCX_OK) return s;
  if (job_id >= b->max_jobs || !b->jobs[job_id].used) return batch_fail(SMCX_EINVAL, "unknown job");
  Job& j = b->jobs[job_id];
  if (!j.done) {  // a job of the running chunk
    s = complete_chunk(b);
    if (s != SMCX_OK) return s;
  }
  b->heap.release(j.occ_off - b->cl.heap, j.occ_bytes);
  j = Job();
  b->done_queue.erase(std::remove(b->done_queue.begin(), b->done_queue.end(), job_id),
                      b->done_queue.end());
  b->dirty = true;
  return SMCX_OK;
}

smcx_status smcx_batch_info(smcx_batch* b, uint32_t* active, uint32_t* free_slots,
                            size_t* free_bytes, size_t* largest_free) {
  if (!b) return batch_fail(SMCX_EINVAL, "null batch");
  uint32_t a = 0, f = 0;
  for (const Job& j : b->jobs) {
    if (!j.used) ++f;
    else if (!j.done) ++a;
  }
  if (active) *active = a;
  if (free_slots) *free_slots = f;
  if (free_bytes) *free_bytes = b->heap.free_bytes();
  if (largest_free) *largest_free = b->heap.largest();
  return SMCX_OK;
}

smcx_status smcx_batch_destroy(smcx_batch* b) {
  if (!b) return batch_fail(SMCX_EINVAL, "null batch");
  if (b->in_flight) cudaEventSynchronize(b->ev_chunk);
  if (b->side) cudaStreamSynchronize(b->side);
  drop_graph(b);
  for (cudaEvent_t ev : b->ev)
    if (ev) cudaEventDestroy(ev);
  if (b->ev_chunk) cudaEventDestroy(b->ev_chunk);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
  return SMCX_OK;
}

}  // extern "C"
