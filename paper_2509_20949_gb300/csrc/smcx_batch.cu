// smcx_batch.cu -- batched execution of many independent lattices (the
// temperature parallelism of Sec. 2.2: simulations at different
// temperatures or compositions share nothing) behind the smcx_batch_* C ABI.
//
// The caller hands over one device arena.  Its head holds the control area
// (device job table, threshold and difference tables per job slot, per-job
// statistics, block tables, a transfer buffer); the rest is a job heap from
// which every admitted lattice gets its occupancy (first-fit, coalescing free
// list).  A chunk of S sweeps runs every active job: per sweep and colour one
// launch per kernel variant covers all jobs of that variant, blocks mapped to
// (job, first cell); jobs with fewer sweeps left simply stop.  With a stream
// the 8 * S * variants launches are captured once into a CUDA graph and
// replayed until the job set changes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/smcx.h"
#include "kernels.h"
#include "kernels_cell.cuh"

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
constexpr int kVariants = 12;

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
  int variant = 0;
  uint32_t cells = 0;  // active cells of a colour
  Geom g{};
  int mode = 0, sbin = 0;
};

struct ControlLayout {
  size_t jobs, tabs, dtabs, stats, blocks, pairs, flag, scratch, heap;
  uint32_t max_blocks;
};

ControlLayout control_layout(uint32_t max_jobs, size_t transfer_bytes, uint32_t max_blocks) {
  ControlLayout c;
  size_t o = 0;
  c.jobs = o;
  o += aup(cell_job_bytes() * max_jobs, kAlign);
  c.tabs = o;
  o += aup(kTabBytes * max_jobs, kAlign);
  c.dtabs = o;
  o += aup(kDtabBytes * max_jobs, kAlign);
  c.stats = o;
  o += aup(sizeof(unsigned long long) * 8 * max_jobs, kAlign);
  c.blocks = o;
  o += aup(sizeof(uint2) * max_blocks, kAlign);
  c.pairs = o;
  o += aup(sizeof(unsigned long long) * 4 * 6 * 6, kAlign);
  c.flag = o;
  o += kAlign;
  c.scratch = o;
  o += aup(transfer_bytes, kAlign);
  c.heap = o;
  c.max_blocks = max_blocks;
  return c;
}

uint32_t blocks_for(uint32_t max_jobs) { return std::max<uint32_t>(1u << 16, max_jobs * 64u); }

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
  bool dirty = true;
  int n_sm = 0;
  smcx_status sticky = SMCX_OK;
  // block tables per variant (offset into the device block array, count)
  uint32_t var_off[kVariants] = {}, var_cnt[kVariants] = {};
  cudaGraphExec_t graph = nullptr;
  uint32_t graph_chunk = 0;

  uint8_t* at(size_t off) { return arena + off; }
  uint8_t* scratch() { return at(cl.scratch); }
  unsigned int* flag() { return reinterpret_cast<unsigned int*>(at(cl.flag)); }
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
  b->graph_chunk = 0;
}

// rebuild the per-variant block tables of the active jobs
smcx_status rebuild_blocks(smcx_batch* b) {
  std::vector<uint2> all;
  for (int v = 0; v < kVariants; ++v) {
    b->var_off[v] = static_cast<uint32_t>(all.size());
    for (uint32_t slot = 0; slot < b->max_jobs; ++slot) {
      const Job& j = b->jobs[slot];
      if (!j.used || j.done || j.variant != v) continue;
      for (uint32_t c0 = 0; c0 < j.cells; c0 += 128) all.push_back(make_uint2(slot, c0));
    }
    b->var_cnt[v] = static_cast<uint32_t>(all.size()) - b->var_off[v];
  }
  if (all.size() > b->cl.max_blocks) return batch_fail(SMCX_EBUDGET, "block table full");
  if (!all.empty())
    BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.blocks), all.data(), sizeof(uint2) * all.size(),
                                  cudaMemcpyHostToDevice, b->stream));
  drop_graph(b);
  b->dirty = false;
  return SMCX_OK;
}

smcx_status enqueue_chunk(smcx_batch* b, uint32_t chunk) {
  const uint2* blocks = reinterpret_cast<const uint2*>(b->at(b->cl.blocks));
  for (uint32_t s = 0; s < chunk; ++s)
    for (int colour = 0; colour < 8; ++colour)
      for (int v = 0; v < kVariants; ++v) {
        if (!b->var_cnt[v]) continue;
        BATCH_CUDA(b, launch_sweep_cells_batch(v, b->at(b->cl.jobs), blocks + b->var_off[v],
                                               b->var_cnt[v], b->var_cnt[v], s, colour, b->stream));
      }
  return SMCX_OK;
}

smcx_status job_energy(smcx_batch* b, Job& j, int64_t* e) {
  const Geom& g = j.g;
  const size_t kmax = g.K <= 5 ? 5 : 6;
  const size_t n_h = static_cast<size_t>(j.M) * kmax * kmax;
  unsigned long long* d_pairs = reinterpret_cast<unsigned long long*>(b->at(b->cl.pairs));
  BATCH_CUDA(b, cudaMemsetAsync(d_pairs, 0, sizeof(uint64_t) * n_h, b->stream));
  BATCH_CUDA(b, launch_pair_count_tiled(g, static_cast<int>(j.M), b->at(j.occ_off), d_pairs,
                                        b->n_sm, b->stream, false));
  std::vector<uint64_t> h(n_h);
  BATCH_CUDA(b, cudaMemcpyAsync(h.data(), d_pairs, sizeof(uint64_t) * n_h, cudaMemcpyDeviceToHost,
                                b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
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
  return control_layout(max_jobs, transfer_bytes, blocks_for(max_jobs)).heap;
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
  const ControlLayout cl = control_layout(max_jobs, transfer_bytes, blocks_for(max_jobs));
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->at(cl.stats), 0, sizeof(unsigned long long) * 8 * max_jobs, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
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
  j.variant = cell_variant(j.g);
  j.cells = 1;
  for (int d = 0; d < 3; ++d) j.cells *= m[d] == 1 ? 1u : static_cast<uint32_t>(m[d] / 2);
  Tables tab;
  host_build_tables(T, &tab, &j.mode, &j.sbin);
  auto fail_release = [&](smcx_status st) {
    b->heap.release(off, ob);
    return st;
  };
  // upload: canonical -> transfer buffer -> validated -> device layout
  cudaError_t e = cudaMemcpyAsync(b->scratch(), h_init, N, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flag(), 0, sizeof(unsigned int), b->stream);
  if (e == cudaSuccess)
    e = launch_validate(b->scratch(), N, desc->n_species, b->flag(), b->n_sm, b->stream);
  unsigned int bad = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, b->flag(), sizeof(bad), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch upload"));
  if (bad) return fail_release(batch_fail(SMCX_EINVAL, "species id >= n_species in occupancy"));
  e = cudaMemsetAsync(b->at(j.occ_off), 0, ob, b->stream);
  if (e == cudaSuccess)
    e = launch_canon_to_dev(j.g, b->scratch(), b->at(j.occ_off), static_cast<uint32_t>(N / j.g.nb),
                            b->n_sm, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->at(b->cl.tabs) + kTabBytes * slot, tab.w, kTabBytes,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->at(b->cl.dtabs) + kDtabBytes * slot, dtab.data(), dtab.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->stats(slot), 0, sizeof(unsigned long long) * 8, b->stream);
  if (e != cudaSuccess) return fail_release(bcuda(b, e, "batch add"));
  s = job_energy(b, j, &j.E0);
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
  if (b->dirty) {
    s = rebuild_blocks(b);
    if (s != SMCX_OK) return s;
  }
  // per-job chunk parameters
  std::vector<uint8_t> table(cell_job_bytes() * b->max_jobs, 0);
  bool any = false;
  for (uint32_t slot = 0; slot < b->max_jobs; ++slot) {
    Job& j = b->jobs[slot];
    if (!j.used || j.done) continue;
    cell::JobDev jd{};
    jd.g = j.g;
    jd.occ = b->at(j.occ_off);
    jd.dtab = b->at(b->cl.dtabs) + kDtabBytes * slot;
    jd.tab = reinterpret_cast<const uint32_t*>(b->at(b->cl.tabs) + kTabBytes * slot);
    jd.stats = b->stats(slot);
    jd.t0 = j.t;
    jd.sweeps = std::min(chunk_sweeps, j.total - j.done_sweeps);
    jd.mode = j.mode;
    jd.sbin = j.sbin;
    jd.no_shift = (j.desc.flags & SMCX_NO_SHIFT) ? 1 : 0;
    std::memcpy(table.data() + cell_job_bytes() * slot, &jd, sizeof(jd));
    any = true;
  }
  if (n_finished) *n_finished = 0;
  if (!any) return SMCX_OK;
  BATCH_CUDA(b, cudaMemcpyAsync(b->at(b->cl.jobs), table.data(), table.size(),
                                cudaMemcpyHostToDevice, b->stream));
  if (b->stream) {
    if (!b->graph || b->graph_chunk != chunk_sweeps) {
      drop_graph(b);
      cudaGraph_t gr = nullptr;
      BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      s = enqueue_chunk(b, chunk_sweeps);
      cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
      if (s != SMCX_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s;
      }
      if (e != cudaSuccess) return bcuda(b, e, "graph capture");
      e = cudaGraphInstantiate(&b->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
      b->graph_chunk = chunk_sweeps;
    }
    BATCH_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
  } else {
    s = enqueue_chunk(b, chunk_sweeps);
    if (s != SMCX_OK) return s;
  }
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
  uint32_t fin = 0;
  for (uint32_t slot = 0; slot < b->max_jobs; ++slot) {
    Job& j = b->jobs[slot];
    if (!j.used || j.done) continue;
    const uint32_t ran = std::min(chunk_sweeps, j.total - j.done_sweeps);
    j.done_sweeps += ran;
    j.t += ran;
    if (j.done_sweeps == j.total) {
      j.done = true;
      b->done_queue.push_back(slot);
      b->dirty = true;
      ++fin;
    }
  }
  if (n_finished) *n_finished = fin;
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
  if (h_occ) {
    const uint64_t N = static_cast<uint64_t>(j.g.nb) * j.g.n[0] * j.g.n[1] * j.g.n[2];
    BATCH_CUDA(b, launch_dev_to_canon(j.g, b->at(j.occ_off), b->scratch(),
                                      static_cast<uint32_t>(N / j.g.nb), b->n_sm, b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(h_occ, b->scratch(), N, cudaMemcpyDeviceToHost, b->stream));
  }
  unsigned long long st[8];
  BATCH_CUDA(b, cudaMemcpyAsync(st, b->stats(job_id), sizeof(st), cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
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
  drop_graph(b);
  delete b;
  return SMCX_OK;
}

}  // extern "C"
