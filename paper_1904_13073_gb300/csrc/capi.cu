// C ABI of the SurfelWarp hot path: stream lifecycle, device memory under a
// process-wide budget, model set-up (skinning, node graph, the block-sparse
// pattern of JᵀJ), the per-frame calls and the inspection hooks.
//
// Model set-up sorts the surfels by their 4-node set on the GPU (the
// library's radix sort, k_sort.cu), so that surfels that contribute to the same ten JᵀJ blocks are
// adjacent; the node-level structure (pattern of 6x6 blocks, graph in-edges,
// the transposed-block lists of the SpMV) is O(nodes + node sets) and is
// built on the host once per model.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include <chrono>

#include <cuda.h>   // CUtensorMap and its encoder's signature; the encoder itself comes from the runtime's
                    // driver entry-point query, so the library does not link the driver library

#include "sw_internal.h"

using namespace sw;

// ------------------------------------------------------------------ errors / memory

namespace {

std::mutex g_err_mu;
std::string g_last_error;
std::atomic<size_t> g_budget{0};
std::atomic<size_t> g_in_use{0};
// highest PCG mode a launch plan may take: 3 the cluster PCG
// (k_pcg_cluster.cu) where a stream's system fits it, else the cooperative
// PCG's SpMV staging mode 2, 1 or 0 (k_pcg.cu: SpmvMode); lowered only by
// sw_debug_set_pcg_mode
std::atomic<int> g_pcg_mode_cap{3};

void set_global_error(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_last_error = s;
}

}  // namespace

namespace sw {
// process-wide error text for calls that take no stream handle
void set_process_error(const std::string& msg) { set_global_error(msg); }
}  // namespace sw

// A Runner launches the per-frame kernels over one stream or over a batch of
// streams: it owns the device tile tables, the descriptor array, the active
// mask, the grid barrier of the persistent PCG, the captured solve graphs and
// the profiling events.
enum ProfStage { kProfDepth = 0, kProfReg, kProfData, kProfPcg, kProfFuse, kProfVis, kProfStages };

struct ProfEvent {
  int stage;
  cudaEvent_t a, b;
};

struct Runner {
  std::vector<sw_stream*> members;
  std::vector<uint64_t> versions;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  BatchHost bh{};
  std::vector<std::pair<void*, size_t>> allocs;
  int* active_host = nullptr;    // current active flags (host copy)
  int* frames_dev = nullptr;
  // pinned staging slots for small host->device copies, reused round-robin;
  // each slot's event tells when its previous copy has been consumed
  static constexpr int kRing = 8;
  static constexpr int kSlotInts = 4096;
  int* ring = nullptr;
  cudaEvent_t ring_ev[kRing] = {};
  int ring_pos = 0;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  std::map<std::pair<int, int>, std::vector<ProfEvent>> graph_prof;
  std::pair<int, int> last_key{0, 0};
  bool profiling = false;
  std::vector<ProfEvent> eager_prof;   // events of the last upload / fusion
  std::vector<cudaEvent_t> event_pool;
  int pcg_rows_per_cta = 32;     // PCG granularity: a stream takes one CTA per this many rows (autotuned)
  int alloc_n = -1;              // member count the device tables in `allocs` were sized for
  std::vector<int> cluster_list; // members on the cluster PCG (their indices)
  std::string err;
};

struct sw_stream {
  sw_params p{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  bool has_model = false;
  bool has_depth = false;
  uint64_t version = 0;      // bumped whenever the device layout of the model changes
  std::string err;
  // device memory
  std::vector<std::pair<void*, size_t>> allocs;   // fixed arena pieces
  std::vector<std::pair<void*, size_t>> model_allocs;
  SwDev h{};                 // host mirror of the descriptor
  int4* knn_dist = nullptr;  // skinning in distance order, caller's order (inspection, checkpoint)
  float4* w_dist = nullptr;
  Runner* run = nullptr;     // the stream's own one-stream runner
  std::vector<int> rl_ptr_host;   // per block row, the start of its SpMV entries (PCG work sizing)
  int cplan_ctas = 0;             // cluster size of the stream's cluster-PCG plan (0: none)
  int last_sys = 0;               // the FP32 system buffer (0: A and g, 1: A2 and g2) assembled last
  int* corr_rec_buf = nullptr;    // sw_debug_record_correspondence: kMaxGn x max_surfels
  size_t cplan_smem = 0;          // shared memory per CTA that plan needs
  // ordering against batches this stream belongs to
  cudaEvent_t batch_done = nullptr;   // recorded by the last batch call (owned by the batch)
  cudaEvent_t own_ev = nullptr;       // recorded before a batch call when own work is pending
  bool own_pending = false;
  // appending (allocated on first use)
  bool fused = false;         // fusion ran since the last depth frame (its per-pixel results are current)
  bool app_ready = false;
  AppendBufs app{};
  int app_last_cand = 0;      // candidates of the last sw_append_frame
  int unsorted = 0;           // surfels appended after the set-sorted ones since the last full rebuild
  int sorted_sets = 0;        // sets in increasing key order; sets added by fast updates follow them
  // device blocks of earlier models and set-up scratch, kept for reuse (their
  // bytes stay counted against the budget until the stream is destroyed)
  std::multimap<size_t, void*> cache;
};

struct sw_batch {
  Runner run;
  cudaEvent_t done = nullptr;
};

namespace {


sw_status fail(sw_stream* s, sw_status code, const std::string& msg) {
  if (s) s->err = msg; else set_global_error(msg);
  return code;
}

#define SW_CUDA(s, call)                                                          \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail((s), SW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool reserve(size_t bytes) {
  const size_t budget = g_budget.load();
  size_t cur = g_in_use.load();
  do {
    if (budget && cur + bytes > budget) return false;
  } while (!g_in_use.compare_exchange_weak(cur, cur + bytes));
  return true;
}

sw_status dalloc(sw_stream* s, std::vector<std::pair<void*, size_t>>& list, void** out, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  if (!reserve(bytes)) return fail(s, SW_ERR_NO_MEMORY, "device memory budget exceeded");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    g_in_use -= bytes;
    return fail(s, e == cudaErrorMemoryAllocation ? SW_ERR_NO_MEMORY : SW_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  list.emplace_back(p, bytes);
  *out = p;
  return SW_OK;
}

void free_list(std::vector<std::pair<void*, size_t>>& list) {
  for (auto& a : list) {
    cudaFree(a.first);
    g_in_use -= a.second;
  }
  list.clear();
}

#define SW_TRY_(expr)                   \
  do {                                  \
    sw_status st_ = (expr);             \
    if (st_ != SW_OK) return st_;       \
  } while (0)

// Block sizes come in classes, eight per power of two (at most 12.5% over the
// request), so that arrays which grow a little with every appended frame keep
// fitting the blocks of the frame before.
size_t size_class(size_t bytes) {
  if (bytes <= 4096) return bytes <= 256 ? 256 : (bytes + 255) & ~size_t(255);
  int e = 63 - __builtin_clzll((unsigned long long)bytes);   // 2^e <= bytes < 2^(e+1)
  const size_t step = size_t(1) << (e - 3);
  return (bytes + step - 1) & ~(step - 1);
}

// A device block of at least `bytes` for stream s: a cached one of at most
// twice the size, else a new one of its size class.  *got is its size.
sw_status cached_alloc(sw_stream* s, void** out, size_t bytes, size_t* got) {
  bytes = size_class(bytes);
  auto it = s->cache.lower_bound(bytes);
  if (it != s->cache.end() && it->first <= 2 * bytes) {
    *out = it->second;
    *got = it->first;
    s->cache.erase(it);
    return SW_OK;
  }
  if (!reserve(bytes)) return fail(s, SW_ERR_NO_MEMORY, "device memory budget exceeded");
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    g_in_use -= bytes;
    return fail(s, e == cudaErrorMemoryAllocation ? SW_ERR_NO_MEMORY : SW_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  *out = p;
  *got = bytes;
  return SW_OK;
}

// The model's blocks go back to the stream's cache (work on the stream that
// uses them is ordered before any later use, which is on the same stream).
// Size of the model block that starts at p (0 if none).
size_t model_block_size(const sw_stream* s, const void* p) {
  for (const auto& a : s->model_allocs)
    if (a.first == p) return a.second;
  return 0;
}

// Make the model block *p hold `need` bytes, keeping its first `used` bytes:
// a larger block from the cache, the old one back into it (stream order keeps
// the copy ahead of any reuse).
sw_status grow_model_block(sw_stream* s, void** p, size_t used, size_t need) {
  if (model_block_size(s, *p) >= need) return SW_OK;
  void* q = nullptr;
  size_t got = 0;
  SW_TRY_(cached_alloc(s, &q, need, &got));
  if (used) {
    const cudaError_t e = cudaMemcpyAsync(q, *p, used, cudaMemcpyDeviceToDevice, s->st);
    if (e != cudaSuccess) return fail(s, SW_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  for (auto& a : s->model_allocs)
    if (a.first == *p) {
      s->cache.emplace(a.second, a.first);
      a = std::make_pair(q, got);
      break;
    }
  *p = q;
  return SW_OK;
}

// The given model blocks (null entries skipped) go back to the cache.
void recycle_blocks(sw_stream* s, std::initializer_list<const void*> blocks) {
  for (const void* p : blocks) {
    if (!p) continue;
    for (size_t k = 0; k < s->model_allocs.size(); ++k)
      if (s->model_allocs[k].first == p) {
        s->cache.emplace(s->model_allocs[k].second, s->model_allocs[k].first);
        s->model_allocs.erase(s->model_allocs.begin() + (long)k);
        break;
      }
  }
}

void recycle_model(sw_stream* s) {
  for (auto& a : s->model_allocs) s->cache.emplace(a.second, a.first);
  s->model_allocs.clear();
}

void release_cache(sw_stream* s) {
  for (auto& kv : s->cache) {
    cudaFree(kv.second);
    g_in_use -= kv.first;
  }
  s->cache.clear();
}

template <typename T>
sw_status A(sw_stream* s, T** out, size_t count, bool model = false) {
  if (!model) return dalloc(s, s->allocs, reinterpret_cast<void**>(out), count * sizeof(T));
  void* p = nullptr;
  size_t got = 0;
  SW_TRY_(cached_alloc(s, &p, count * sizeof(T), &got));
  s->model_allocs.emplace_back(p, got);
  *out = reinterpret_cast<T*>(p);
  return SW_OK;
}

#define SW_TRY(expr)                    \
  do {                                  \
    sw_status st_ = (expr);             \
    if (st_ != SW_OK) return st_;       \
  } while (0)

// Order a stream's own call after the batch work that touched it.
void enter(sw_stream* s) {
  if (s->batch_done) cudaStreamWaitEvent(s->st, s->batch_done, 0);
  s->own_pending = true;
}

void drop_graphs(Runner* r) {
  for (auto& kv : r->graphs) cudaGraphExecDestroy(kv.second);
  r->graphs.clear();
  for (auto& kv : r->graph_prof)
    for (auto& e : kv.second) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  r->graph_prof.clear();
}

void destroy_runner(Runner* r) {
  if (!r) return;
  if (r->st) cudaStreamSynchronize(r->st);
  drop_graphs(r);
  for (auto& e : r->eager_prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  r->eager_prof.clear();
  free_list(r->allocs);
  if (r->ring) cudaFreeHost(r->ring);
  for (auto& e : r->ring_ev) if (e) { cudaEventDestroy(e); e = nullptr; }
  delete[] r->active_host;
  if (r->own_stream && r->st) cudaStreamDestroy(r->st);
  r->active_host = nullptr;
  r->ring = nullptr;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// (Re)build the device tables of a runner for its members.
sw_status build_runner(Runner* r, sw_stream* err_to) {
  drop_graphs(r);
  const int n = (int)r->members.size();
  r->versions.clear();
  for (auto* m : r->members) r->versions.push_back(m->version);
  std::vector<SwDev> devs(n);
  for (int i = 0; i < n; ++i) devs[i] = r->members[i]->h;
  std::vector<int> tiles((size_t)kTileKinds * (n + 1), 0);
  for (int k = 0; k < kTileKinds; ++k) {
    int acc = 0;
    for (int i = 0; i < n; ++i) {
      tiles[(size_t)k * (n + 1) + i] = acc;
      acc += tiles_for(k, devs[i]);
    }
    tiles[(size_t)k * (n + 1) + n] = acc;
    r->bh.total_tiles[k] = acc;
  }
  // PCG: one cooperative grid (every CTA resident); each stream gets its own
  // CTAs
  {
    const int prec = n ? devs[0].precision : SW_PRECISION_MIXED;
    for (int i = 1; i < n; ++i)
      if (devs[i].precision != prec) return fail(err_to, SW_ERR_INVALID_ARG, "batch members differ in precision");
    r->bh.precision = prec;
    r->bh.any_visibility = 0;
    for (int i = 0; i < n; ++i) r->bh.any_visibility |= devs[i].visibility;
    // members whose system has a cluster plan run on the cluster PCG (one
    // cluster each, its own launch); the others share the cooperative grid
    std::vector<int> cl;
    size_t cl_smem = 0;
    int cl_ctas = 0;
    std::vector<char> in_cluster(n, 0);
    if (g_pcg_mode_cap.load() >= 3)
      for (int i = 0; i < n; ++i) {
        const sw_stream* m = r->members[i];
        if (!devs[i].cplan || m->cplan_ctas == 0 || (cl_ctas && m->cplan_ctas != cl_ctas)) continue;
        cl_ctas = m->cplan_ctas;
        cl_smem = std::max(cl_smem, m->cplan_smem);
        cl.push_back(i);
        in_cluster[i] = 1;
      }
    // clusters only when they take the whole batch in one wave: members left
    // to the cooperative kernel run in a second launch after them, and
    // clusters beyond those the device runs at once in further waves.  On
    // the 16-stream uneven batch (7 clusters resident at once) one
    // cooperative launch over every member took 407 us per Gauss-Newton
    // iteration, one wave of clusters and the rest cooperative 407 us,
    // clusters in waves 437 us.
    if (!cl.empty() && ((int)cl.size() != n || cluster_pcg_active(prec, cl_ctas, cl_smem) < (int)cl.size())) {
      cl.clear();
      cl_smem = 0;
      cl_ctas = 0;
      std::fill(in_cluster.begin(), in_cluster.end(), 0);
    }
    const int n_coop = n - (int)cl.size();
    const int per_sm = std::max(1, pcg_blocks_per_sm(prec));
    const int cap = sm_count() * per_sm;
    if (n_coop > cap) return fail(err_to, SW_ERR_INVALID_ARG, "too many streams for one persistent launch");
    // greedy: the next CTA goes to the stream with the most rows per CTA,
    // which minimises the largest share (the launch ends with the slowest
    // stream); a stream takes at most one CTA per pcg_rows_per_cta rows
    std::vector<int> want(n, 1);
    for (int i = 0; i < n; ++i)
      if (in_cluster[i]) want[i] = 0;
    int total = n_coop;
    {
      const int rows = std::max(8, r->pcg_rows_per_cta);
      auto limit = [&](int i) { return std::max(1, std::min(kMaxCtaPerStream, (devs[i].n_n + rows - 1) / rows)); };
      auto share = [&](int i) { return (devs[i].n_n + want[i] - 1) / want[i]; };
      std::priority_queue<std::pair<int, int>> pq;   // (rows per CTA, stream)
      for (int i = 0; i < n; ++i)
        if (!in_cluster[i] && want[i] < limit(i)) pq.push({share(i), i});
      while (total < cap && !pq.empty()) {
        const int i = pq.top().second;
        pq.pop();
        ++want[i];
        ++total;
        if (want[i] < limit(i)) pq.push({share(i), i});
      }
    }
    int acc = 0, rows_cap = 1;
    for (int i = 0; i < n; ++i) {
      tiles[(size_t)kTilePcg * (n + 1) + i] = acc;
      acc += want[i];
      if (want[i]) rows_cap = std::max(rows_cap, (devs[i].n_n + want[i] - 1) / want[i]);
    }
    r->cluster_list = cl;
    r->bh.n_cluster = (int)cl.size();
    r->bh.cluster_ctas = cl_ctas;
    r->bh.cluster_smem = cl_smem;
    tiles[(size_t)kTilePcg * (n + 1) + n] = acc;
    r->bh.total_tiles[kTilePcg] = acc;
    // the most SpMV entries one CTA owns (its rows are i = t + G a)
    int ent_cap = 1;
    for (int i = 0; i < n; ++i) {
      const std::vector<int>& rp = r->members[i]->rl_ptr_host;
      const int G = want[i], nn = devs[i].n_n;
      if (nn == 0 || G == 0) continue;   // a stream without a model yet, or on the cluster PCG
      if ((int)rp.size() != nn + 1) return fail(err_to, SW_ERR_INVALID_ARG, "batch member without a JᵀJ pattern");
      for (int t = 0; t < G; ++t) {
        int e = 0;
        for (int j = t; j < nn; j += G) e += rp[j + 1] - rp[j];
        ent_cap = std::max(ent_cap, e);
      }
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the SpMV stages as much in shared memory as fits: the rows' blocks and
    // the entries' outputs (2), the outputs only (1), or nothing (0)
    int mode = std::min(2, g_pcg_mode_cap.load());
    while (mode >= 0 && pcg_smem_bytes(rows_cap, ent_cap, prec, mode) > (size_t)optin) --mode;
    if (mode < 0) return fail(err_to, SW_ERR_INVALID_ARG, "a stream has too many nodes for the PCG's on-chip state");
    r->bh.pcg_rows_cap = rows_cap;
    r->bh.pcg_ent_cap = ent_cap;
    r->bh.pcg_mode = mode;
  }
  SwDev* devs_dev = nullptr;
  int* tile_dev = nullptr;
  int* active_dev = nullptr;
  int* cl_dev = nullptr;
  if (r->alloc_n == n && r->allocs.size() == 5) {   // same members: the tables are rewritten in stream order
    devs_dev = reinterpret_cast<SwDev*>(r->allocs[0].first);
    tile_dev = reinterpret_cast<int*>(r->allocs[1].first);
    active_dev = reinterpret_cast<int*>(r->allocs[2].first);
    r->frames_dev = reinterpret_cast<int*>(r->allocs[3].first);
    cl_dev = reinterpret_cast<int*>(r->allocs[4].first);
  } else {
    free_list(r->allocs);
    r->alloc_n = -1;
    SW_TRY(dalloc(err_to, r->allocs, reinterpret_cast<void**>(&devs_dev), sizeof(SwDev) * std::max(1, n)));
    SW_TRY(dalloc(err_to, r->allocs, reinterpret_cast<void**>(&tile_dev), sizeof(int) * tiles.size()));
    SW_TRY(dalloc(err_to, r->allocs, reinterpret_cast<void**>(&active_dev), sizeof(int) * std::max(1, n)));
    SW_TRY(dalloc(err_to, r->allocs, reinterpret_cast<void**>(&r->frames_dev), sizeof(int) * std::max(1, n)));
    SW_TRY(dalloc(err_to, r->allocs, reinterpret_cast<void**>(&cl_dev), sizeof(int) * std::max(1, n)));
    r->alloc_n = n;
  }
  if (!r->cluster_list.empty())
    SW_CUDA(err_to, cudaMemcpyAsync(cl_dev, r->cluster_list.data(), sizeof(int) * r->cluster_list.size(),
                                    cudaMemcpyHostToDevice, r->st));
  r->bh.cluster_members_dev = cl_dev;
  if (!r->ring) {
    if (cudaMallocHost(&r->ring, sizeof(int) * Runner::kRing * Runner::kSlotInts) != cudaSuccess)
      return fail(err_to, SW_ERR_NO_MEMORY, "pinned host allocation failed");
    for (auto& e : r->ring_ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    r->active_host = new int[Runner::kSlotInts];
  }
  for (int i = 0; i < n; ++i) r->active_host[i] = 1;
  std::vector<int> ones(std::max(1, n), 1);
  SW_CUDA(err_to, cudaMemcpyAsync(devs_dev, devs.data(), sizeof(SwDev) * n, cudaMemcpyHostToDevice, r->st));
  SW_CUDA(err_to, cudaMemcpyAsync(tile_dev, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, r->st));
  SW_CUDA(err_to, cudaMemcpyAsync(active_dev, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, r->st));
  SW_CUDA(err_to, cudaStreamSynchronize(r->st));
  r->bh.bt.devs = devs_dev;
  r->bh.bt.active = active_dev;
  r->bh.bt.n_streams = n;
  for (int k = 0; k < kTileKinds; ++k) r->bh.tile_base_dev[k] = tile_dev + (size_t)k * (n + 1);
  r->bh.spin_limit = 1 << 22;   // bounded polls (well under a second), then a timeout status
  return SW_OK;
}

// Copy n ints to device memory on the runner's stream through a pinned slot,
// without waiting for earlier work on the stream.
cudaError_t ring_copy(Runner* r, int* dst, const int* src, int n) {
  const int k = r->ring_pos;
  r->ring_pos = (k + 1) % Runner::kRing;
  cudaError_t e = cudaEventSynchronize(r->ring_ev[k]);   // the slot's last copy has run
  if (e != cudaSuccess) return e;
  int* slot = r->ring + (size_t)k * Runner::kSlotInts;
  std::memcpy(slot, src, sizeof(int) * n);
  e = cudaMemcpyAsync(dst, slot, sizeof(int) * n, cudaMemcpyHostToDevice, r->st);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(r->ring_ev[k], r->st);
}

bool runner_stale(const Runner* r) {
  for (size_t i = 0; i < r->members.size(); ++i)
    if (r->members[i]->version != r->versions[i]) return true;
  return false;
}

cudaEvent_t take_event(Runner* r) {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records a stage boundary.  During capture the record becomes a graph node.
void prof_mark(Runner* r, std::vector<ProfEvent>* list, int stage, bool begin, bool capturing) {
  if (!list) return;
  if (begin) {
    ProfEvent pe{stage, take_event(r), take_event(r)};
    list->push_back(pe);
    if (capturing) cudaEventRecordWithFlags(pe.a, r->st, cudaEventRecordExternal);
    else cudaEventRecord(pe.a, r->st);
  } else {
    const ProfEvent& pe = list->back();
    if (capturing) cudaEventRecordWithFlags(pe.b, r->st, cudaEventRecordExternal);
    else cudaEventRecord(pe.b, r->st);
  }
}

// A Gauss-Newton iteration's assembly in the batch's precision: FP64, the
// regulariser's launch (plain stores, which also initialise the system),
// then the data term's (profiled as two stages); FP32, one launch of both
// into the iteration's system buffer, cleared by the previous iteration's
// launch or, before the solve's first, by launch_system_clear (profiled as
// the data stage).
void launch_assembly_stage(Runner* r, int it, std::vector<ProfEvent>* prof) {
  const BatchHost& b = r->bh;
  cudaStream_t st = r->st;
  if (b.precision == SW_PRECISION_FP64) {
    prof_mark(r, prof, kProfReg, true, true);
    launch_reg_assemble64(b, it, st);
    prof_mark(r, prof, kProfReg, false, true);
    prof_mark(r, prof, kProfData, true, true);
    launch_data_assemble64(b, it, st);
    prof_mark(r, prof, kProfData, false, true);
  } else {
    prof_mark(r, prof, kProfData, true, true);
    if (it == 0) launch_system_clear(b, st);
    launch_assemble(b, it, st);
    prof_mark(r, prof, kProfData, false, true);
  }
}

sw_status enqueue_solve(Runner* r, sw_stream* err_to, int gn, int pcg, std::vector<ProfEvent>* prof) {
  cudaStream_t st = r->st;
  launch_solve_begin(r->bh, st);
  if (r->bh.any_visibility) {   // Sec. 7: visibility predicted once, under the warp the solve starts from
    prof_mark(r, prof, kProfVis, true, true);
    launch_vis_splat(r->bh, 0, st);
    launch_vis_mark(r->bh, 0, st);
    prof_mark(r, prof, kProfVis, false, true);
  }
  for (int it = 0; it < gn; ++it) {
    launch_assembly_stage(r, it, prof);
    prof_mark(r, prof, kProfPcg, true, true);
    launch_precond(r->bh, it, st);
    SW_CUDA(err_to, launch_pcg_cluster(r->bh, it, pcg, st));
    SW_CUDA(err_to, launch_pcg(r->bh, it, pcg, st));
    prof_mark(r, prof, kProfPcg, false, true);
  }
  SW_CUDA(err_to, cudaGetLastError());
  return SW_OK;
}

sw_status runner_solve(Runner* r, sw_stream* err_to, int gn, int pcg) {
  const auto key = std::make_pair(gn, pcg);
  auto itg = r->graphs.find(key);
  if (itg == r->graphs.end()) {
    std::vector<ProfEvent> prof;
    cudaGraph_t graph = nullptr;
    SW_CUDA(err_to, cudaStreamBeginCapture(r->st, cudaStreamCaptureModeThreadLocal));
    const sw_status e = enqueue_solve(r, err_to, gn, pcg, r->profiling ? &prof : nullptr);
    const cudaError_t ce = cudaStreamEndCapture(r->st, &graph);
    if (e != SW_OK) { if (graph) cudaGraphDestroy(graph); return e; }
    if (ce != cudaSuccess) return fail(err_to, SW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(err_to, SW_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    itg = r->graphs.emplace(key, exec).first;
    r->graph_prof[key] = prof;
  }
  r->last_key = key;
  SW_CUDA(err_to, cudaGraphLaunch(itg->second, r->st));
  for (size_t i = 0; i < r->members.size(); ++i)   // iteration gn - 1 assembled into buffer (gn - 1) mod 2
    if (!r->active_host || r->active_host[i]) r->members[i]->last_sys = (gn - 1) & 1;
  return SW_OK;
}

void reset_eager_prof(Runner* r) {
  for (auto& e : r->eager_prof) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  r->eager_prof.clear();
}

sw_status runner_fuse(Runner* r, sw_stream* err_to) {
  cudaStream_t st = r->st;
  std::vector<ProfEvent>* prof = r->profiling ? &r->eager_prof : nullptr;
  prof_mark(r, prof, kProfFuse, true, false);
  launch_warp_live(r->bh, st);
  launch_index_map(r->bh, st);
  launch_fuse(r->bh, 0, st);
  prof_mark(r, prof, kProfFuse, false, false);
  SW_CUDA(err_to, cudaGetLastError());
  return SW_OK;
}

sw_status runner_profile(Runner* r, sw_stream* err_to, double* ms, int* launches) {
  SW_CUDA(err_to, cudaStreamSynchronize(r->st));
  for (int k = 0; k < kProfStages; ++k) { if (ms) ms[k] = 0.0; if (launches) launches[k] = 0; }
  auto add = [&](const std::vector<ProfEvent>& v) -> sw_status {
    for (const auto& e : v) {
      float t = 0.f;
      const cudaError_t ce = cudaEventElapsedTime(&t, e.a, e.b);
      if (ce != cudaSuccess) return fail(err_to, SW_ERR_CUDA, std::string("profile events: ") + cudaGetErrorString(ce));
      if (ms) ms[e.stage] += t;
      if (launches) launches[e.stage] += 1;
    }
    return SW_OK;
  };
  auto it = r->graph_prof.find(r->last_key);
  if (it != r->graph_prof.end()) SW_TRY(add(it->second));
  SW_TRY(add(r->eager_prof));
  return SW_OK;
}

// Push the host descriptor of a stream to its own runner.
sw_status sync_desc(sw_stream* s) {
  if (!s->run) {
    s->run = new Runner();
    s->run->st = s->st;
  }
  s->run->members.assign(1, s);
  return build_runner(s->run, s);
}

bool params_ok(const sw_params* p, std::string& why) {
  if (!p) { why = "null params"; return false; }
  if (p->width < 3 || p->height < 3 || p->width > 16384 || p->height > 16384) { why = "image size out of range"; return false; }
  if (!(p->fx > 0 && p->fy > 0)) { why = "focal lengths must be positive"; return false; }
  if (p->max_surfels < 0 || p->max_surfels > (1 << 28)) { why = "max_surfels out of range"; return false; }
  if (p->max_nodes < 9 || p->max_nodes > SW_MAX_NODES) { why = "max_nodes must be in [9, 65535]"; return false; }
  if (!(p->lambda >= 0 && p->fuse_dist >= 0 && p->corr_dist >= 0)) { why = "negative threshold"; return false; }
  if (p->visibility != 0 && p->visibility != 1) { why = "visibility must be 0 or 1"; return false; }
  if (p->extend_nodes != 0 && p->extend_nodes != 1) { why = "extend_nodes must be 0 or 1"; return false; }
  if (!(p->eps > 0 && p->eps < 1 && p->delta_nn >= 0 && p->fd_step > 0)) {
    why = "appending parameters out of range (0 < eps < 1, delta_nn >= 0, fd_step > 0)";
    return false;
  }
  if (p->precision != SW_PRECISION_MIXED && p->precision != SW_PRECISION_FP64 &&
      p->precision != SW_PRECISION_MIXED_F64DOTS) {
    why = "precision must be one of SW_PRECISION_MIXED, SW_PRECISION_FP64, SW_PRECISION_MIXED_F64DOTS";
    return false;
  }
  return true;
}

}  // namespace

// ------------------------------------------------------------------ set-up kernels

namespace {

__global__ void k_set_keys(const int4* __restrict__ knn, int n, unsigned long long* keys, int* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 k = knn[i];
  int a[4] = {k.x, k.y, k.z, k.w};
  // sort 4 ids ascending
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3 - x; ++y)
      if (a[y] > a[y + 1]) { const int t = a[y]; a[y] = a[y + 1]; a[y + 1] = t; }
  keys[i] = ((unsigned long long)a[0] << 48) | ((unsigned long long)a[1] << 32) |
            ((unsigned long long)a[2] << 16) | (unsigned long long)a[3];
  vals[i] = i;
}

__global__ void k_gather_model(SwDev d, const unsigned long long* __restrict__ keys, const int* __restrict__ perm,
                               const float4* __restrict__ tv, const float4* __restrict__ tn,
                               const int2* __restrict__ tt, const int4* __restrict__ tknn,
                               const float4* __restrict__ tw, int* __restrict__ head) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_s) return;
  const int o = perm[i];
  d.v_ref[i] = tv[o];
  d.n_ref[i] = tn[o];
  d.tt[i] = tt[o];
  d.orig_id[i] = o;
  d.inv_perm[o] = i;
  const int4 k = tknn[o];
  const float4 w = tw[o];
  int id[4] = {k.x, k.y, k.z, k.w};
  float ww[4] = {w.x, w.y, w.z, w.w};
  int slot0 = 0;   // tracks where the nearest node (distance slot 0) goes
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3 - x; ++y)
      if (id[y] > id[y + 1]) {
        const int t = id[y]; id[y] = id[y + 1]; id[y + 1] = t;
        const float u = ww[y]; ww[y] = ww[y + 1]; ww[y + 1] = u;
        if (slot0 == y) slot0 = y + 1; else if (slot0 == y + 1) slot0 = y;
      }
  d.knn[i] = make_int4(id[0], id[1], id[2], id[3]);
  d.w[i] = make_float4(ww[0], ww[1], ww[2], ww[3]);
  d.ref_slot[i] = slot0;
  head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_set_nodes(SwDev d, const int* __restrict__ head, int4* __restrict__ set_nodes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_s) return;
  if (head[i]) set_nodes[d.set_id[i]] = d.knn[i];
}

__global__ void k_minus_one(int* a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] -= 1;
}

__global__ void k_identity_dq(float4* dq, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  dq[2 * j] = make_float4(1.f, 0.f, 0.f, 0.f);
  dq[2 * j + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// a depth frame arrives: its id, and the depth stage's wait status cleared
__global__ void k_frame_begin(int* t_now, int v, int* status) {
  *t_now = v;
  atomicAnd(status, ~kStatusDepthTimeout);
}

__global__ void k_set_frames(Batch bt, const int* __restrict__ frames) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < bt.n_streams && stream_active(bt, s)) {
    *bt.devs[s].t_now = frames[s];
    atomicAnd(bt.devs[s].status, ~kStatusDepthTimeout);
  }
}

}  // namespace

// ------------------------------------------------------------------ autotuning

// Choose the PCG's granularity (rows per CTA) for a runner by timing its
// persistent launch on the members' current systems: for each candidate the
// runner is rebuilt (CTA allocation and SpMV staging follow), the system is
// assembled again (which also starts a new PCG epoch) and the PCG launch
// alone is timed with events, six times after one untimed launch, in two
// sweeps over the candidates; the fastest launch is a candidate's figure.
// The node transforms are saved before and restored after every candidate, so
// the call leaves the streams' state as it found it.  Every member is made
// active.
sw_status runner_autotune(Runner* r, sw_stream* err_to, int pcg, int* best_rows, double* best_us) {
  static const int kCand[] = {16, 24, 32, 48, 64, 96};
  cudaStream_t st = r->st;
  struct Saved { void* dst; void* copy; size_t bytes; };
  std::vector<Saved> saved;
  auto release = [&] { for (auto& sv : saved) cudaFree(sv.copy); };
  for (sw_stream* m : r->members) {
    if (!m->has_model || !m->has_depth) { release(); return fail(err_to, SW_ERR_NOT_INITIALIZED, "a member has no model or depth frame"); }
    const size_t nb[2] = {(size_t)m->h.n_n * 32, m->h.dq64 ? (size_t)m->h.n_n * 64 : 0};
    void* src[2] = {m->h.dq, m->h.dq64};
    for (int k = 0; k < 2; ++k) {
      if (!nb[k]) continue;
      void* cp = nullptr;
      if (cudaMalloc(&cp, nb[k]) != cudaSuccess) { release(); return fail(err_to, SW_ERR_NO_MEMORY, "autotune scratch"); }
      saved.push_back({src[k], cp, nb[k]});
      SW_CUDA(err_to, cudaMemcpyAsync(cp, src[k], nb[k], cudaMemcpyDeviceToDevice, st));
    }
  }
  auto restore = [&]() -> cudaError_t {
    for (auto& sv : saved) {
      const cudaError_t e = cudaMemcpyAsync(sv.dst, sv.copy, sv.bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // two sweeps over the candidates, each timing a candidate's launch six
  // times after one untimed launch; a candidate's figure is its fastest
  // launch, which is robust to the run-to-run spread of the launches'
  // synchronisation waits
  constexpr int kSweeps = 2, kTimed = 6;
  const int n_cand = (int)(sizeof(kCand) / sizeof(kCand[0]));
  std::vector<double> cand_t(n_cand, 1e30);
  for (int sweep = 0; sweep < kSweeps; ++sweep)
    for (int c = 0; c < n_cand; ++c) {
      r->pcg_rows_per_cta = kCand[c];
      if (build_runner(r, nullptr) != SW_OK) continue;   // does not fit on chip: skip
      launch_solve_begin(r->bh, st);
      bool ok = true;
      for (int rep = 0; rep <= kTimed && ok; ++rep) {
        launch_assembly_stage(r, 0, nullptr);
        launch_precond(r->bh, 0, st);
        cudaEventRecord(e0, st);
        ok = launch_pcg_cluster(r->bh, 0, pcg, st) == cudaSuccess && launch_pcg(r->bh, 0, pcg, st) == cudaSuccess;
        cudaEventRecord(e1, st);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) cand_t[c] = std::min(cand_t[c], (double)ms);
      }
      ok = ok && restore() == cudaSuccess;
      if (!ok) cand_t[c] = 1e30;
    }
  int best = r->pcg_rows_per_cta;
  double best_t = 1e30;
  for (int c = 0; c < n_cand; ++c)
    if (cand_t[c] < best_t) {
      best_t = cand_t[c];
      best = kCand[c];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  r->pcg_rows_per_cta = best;
  const sw_status bs = build_runner(r, err_to);
  const cudaError_t re = restore();
  SW_CUDA(err_to, cudaStreamSynchronize(st));
  release();
  if (bs != SW_OK) return bs;
  if (re != cudaSuccess) return fail(err_to, SW_ERR_CUDA, "autotune restore failed");
  if (best_rows) *best_rows = best;
  if (best_us) *best_us = best_t * 1000.0;
  return SW_OK;
}

// ------------------------------------------------------------------ public API

// Definitions take C linkage from their declarations in surfelwarp.h.

sw_status sw_params_default(sw_params* p, int width, int height, float fx, float fy, float cx, float cy,
                            int max_surfels, int max_nodes) {
  if (!p || width <= 0 || height <= 0) return fail(nullptr, SW_ERR_INVALID_ARG, "bad sw_params_default arguments");
  std::memset(p, 0, sizeof(*p));
  p->width = width; p->height = height;
  p->fx = fx; p->fy = fy; p->cx = cx; p->cy = cy;
  p->max_surfels = max_surfels; p->max_nodes = max_nodes;
  p->lambda = 5.f;          // Table 1
  p->fuse_dist = 1e-3f;     // Table 1
  p->fuse_normal = 0.85f;   // Table 1
  p->corr_dist = 0.05f;
  p->corr_normal = 0.7f;
  p->stable_conf = 10.f;    // Table 1
  p->recent_frames = 2;     // Table 1
  p->precision = SW_PRECISION_MIXED;
  p->visibility = 0;
  p->extend_nodes = 1;
  p->eps = 0.2f;            // Table 1
  p->delta_nn = 0.3f;
  p->fd_step = 1e-3f;
  p->t_low_confid = 30;     // Table 1
  return SW_OK;
}

sw_status sw_set_memory_budget(size_t bytes) {
  g_budget = bytes;
  return SW_OK;
}

size_t sw_memory_in_use(void) { return g_in_use.load(); }

// A TMA descriptor of a stream's depth image for k_depth_maps: 2D FP32,
// width x height, rows width*4 bytes apart, a 40x10 box, zeros outside the
// image.  False (plain loads) if the rows are not 16-byte aligned or the
// encoder is unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_depth_tmap(float* depth, int width, int height, CUtensorMap* out) {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  if (!fn || width % 4 != 0 || (reinterpret_cast<uintptr_t>(depth) & 15) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
  const cuuint64_t strides[1] = {(cuuint64_t)width * sizeof(float)};
  const cuuint32_t box[2] = {40, 10};
  const cuuint32_t estr[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, depth, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

sw_status sw_create_stream(const sw_params* p, void* cuda_stream, sw_handle* out) {
  std::string why;
  if (!out) return fail(nullptr, SW_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (!params_ok(p, why)) return fail(nullptr, SW_ERR_INVALID_ARG, why);
  sw_stream* s = new sw_stream();
  s->p = *p;
  auto cleanup = [&](sw_status code) {
    const std::string msg = s->err;
    if (s->run) { destroy_runner(s->run); delete s->run; }
    free_list(s->allocs);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
    set_global_error(msg);
    return code;
  };
  if (cuda_stream) {
    s->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      s->err = "cudaStreamCreate failed";
      return cleanup(SW_ERR_CUDA);
    }
    s->own_stream = true;
  }
  SwDev& h = s->h;
  h.W = p->width; h.H = p->height;
  h.fx = p->fx; h.fy = p->fy; h.cx = p->cx; h.cy = p->cy;
  h.sqrt_lambda = std::sqrt(p->lambda);
  h.precision = p->precision;
  h.visibility = p->visibility;
  h.corr_dist = p->corr_dist; h.corr_normal = p->corr_normal;
  h.fuse_dist = p->fuse_dist; h.fuse_normal = p->fuse_normal;
  h.stable_conf = p->stable_conf; h.recent_frames = p->recent_frames;
  const size_t ns = std::max(1, p->max_surfels), nn = p->max_nodes, np = (size_t)p->width * p->height;
  sw_status st = SW_OK;
#define ALLOC(ptr, count) if (st == SW_OK) st = A(s, &(ptr), (count))
  ALLOC(h.v_ref, ns); ALLOC(h.n_ref, ns); ALLOC(h.tt, ns); ALLOC(h.knn, ns); ALLOC(h.w, ns);
  ALLOC(h.ref_slot, ns); ALLOC(h.set_id, ns); ALLOC(h.orig_id, ns); ALLOC(h.inv_perm, ns);
  ALLOC(h.v_live, ns); ALLOC(h.n_live, ns); ALLOC(h.corr_pix, ns);
  ALLOC(h.node_p, nn); ALLOC(h.dq, 2 * nn); ALLOC(h.graph, SW_K_GRAPH * nn);
  ALLOC(h.in_ptr, nn + 1); ALLOC(h.in_src, SW_K_GRAPH * nn);
  ALLOC(h.depth, np); ALLOC(h.vmap, np); ALLOC(h.nmap, np); ALLOC(h.imap, 16 * np); ALLOC(h.fuse_target, np);
  ALLOC(h.vis_map, np); ALLOC(h.visible, ns);
  ALLOC(h.row_ptr, nn + 1); ALLOC(h.rl_ptr, nn + 1); ALLOC(h.g, 6 * nn); ALLOC(h.g2, 6 * nn); ALLOC(h.minv, 21 * nn);
  ALLOC(h.part, 4 * kMaxCtaPerStream); ALLOC(h.pcg_epoch, 1);
  ALLOC(h.xp, 12 * nn);
  ALLOC(h.rigid, kRigidSlots); ALLOC(h.rigid_stats, 2 * kMaxRigid);
  ALLOC(h.rigid_part, (size_t)kRigidSums * ((ns + kSurfTile - 1) / kSurfTile));
  if (p->precision == SW_PRECISION_FP64) {
    ALLOC(h.g64, 6 * nn); ALLOC(h.v64, 18 * nn); ALLOC(h.dq64, 8 * nn); ALLOC(h.minv64, 21 * nn);
  }
  ALLOC(h.e_depth, kMaxGn); ALLOC(h.e_reg, kMaxGn); ALLOC(h.n_corr, kMaxGn); ALLOC(h.pcg_rz, kMaxGn);
  ALLOC(h.status, 1); ALLOC(h.t_now, 1);
#undef ALLOC
  if (st != SW_OK) return cleanup(st);
  {
    CUtensorMap tm;
    unsigned char* dev_tm = nullptr;
    h.depth_tmap = nullptr;
    if (encode_depth_tmap(h.depth, h.W, h.H, &tm)) {
      if ((st = A(s, &dev_tm, sizeof(CUtensorMap))) != SW_OK) return cleanup(st);
      if (cudaMemcpy(dev_tm, &tm, sizeof(tm), cudaMemcpyHostToDevice) != cudaSuccess) {
        s->err = "tensor map upload failed";
        return cleanup(SW_ERR_CUDA);
      }
      h.depth_tmap = dev_tm;
    }
  }
  // the index map is cleared here once; fusion leaves it empty after every frame
  if (cudaMemsetAsync(h.status, 0, sizeof(int), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.t_now, 0, sizeof(int), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.part, 0, 4 * kMaxCtaPerStream * sizeof(PartSlot), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.xp, 0, 12 * nn * sizeof(unsigned long long), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.pcg_epoch, 0, sizeof(unsigned long long), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.imap, 0xff, 16 * np * sizeof(unsigned long long), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.vis_map, 0xff, np * sizeof(unsigned long long), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.visible, 0, ns * sizeof(int), s->st) != cudaSuccess ||
      cudaMemsetAsync(h.vmap, 0, np * sizeof(float4), s->st) != cudaSuccess) {
    s->err = "cudaMemset failed";
    return cleanup(SW_ERR_CUDA);
  }
  {
    const sw_status e = sync_desc(s);
    if (e != SW_OK) return cleanup(e);
  }
  *out = s;
  return SW_OK;
}

sw_status sw_destroy_stream(sw_handle s) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  cudaStreamSynchronize(s->st);
  if (s->run) { destroy_runner(s->run); delete s->run; s->run = nullptr; }
  if (s->own_ev) cudaEventDestroy(s->own_ev);
  free_list(s->model_allocs);
  release_cache(s);
  free_list(s->allocs);
  if (s->own_stream) cudaStreamDestroy(s->st);
  delete s;
  return SW_OK;
}

namespace {

// temporary device buffer freed at scope exit (set-up only)
struct Tmp {
  sw_stream* s = nullptr;
  void* p = nullptr;
  size_t got = 0;
  explicit Tmp(sw_stream* st) : s(st) {}
  Tmp(sw_stream* st, size_t bytes) : s(st) { alloc(bytes); }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
  ~Tmp() { put(); }
  void put() {
    if (p) s->cache.emplace(got, p);
    p = nullptr;
  }
  bool alloc(size_t bytes) {
    put();
    if (cached_alloc(s, &p, bytes, &got) != SW_OK) p = nullptr;
    return p != nullptr;
  }
  template <typename T> T* as() { return reinterpret_cast<T*>(p); }
};

// In-edges of the node graph (m -> j for j in N_m), CSR by j, sources
// ascending; the graph comes from the library's own k-NN kernel.
bool build_in_edges(int n_n, const std::vector<int>& graph, std::vector<int>& in_ptr, std::vector<int>& in_src,
                    std::string& why) {
  std::vector<std::vector<int>> in(n_n);
  for (int j = 0; j < n_n; ++j)
    for (int e = 0; e < SW_K_GRAPH; ++e) {
      const int i = graph[(size_t)j * SW_K_GRAPH + e];
      if (i < 0 || i >= n_n || i == j) { why = "node graph index out of range"; return false; }
      in[i].push_back(j);
    }
  in_ptr.assign(n_n + 1, 0);
  in_src.clear();
  for (int j = 0; j < n_n; ++j) {
    std::sort(in[j].begin(), in[j].end());
    in_src.insert(in_src.end(), in[j].begin(), in[j].end());
    in_ptr[j + 1] = (int)in_src.size();
  }
  return true;
}


}  // namespace

namespace {
// The surfel half of the set-up, from caller-order device arrays (which may
// be scratch): the caller-order skinning is kept for inspection, the surfels
// are sorted by their 4-node set and gathered into the internal order, and the
// distinct sets are left in `sets` (device, *n_sets of them) for the pattern.
sw_status setup_surfels(sw_stream* s, const float4* tv, const float4* tn, const int2* tt, const int4* tknn,
                        const float4* tw, int n_s, Tmp& sets, int* n_sets) {
  SwDev& h = s->h;
  cudaStream_t st = s->st;
  const size_t n = n_s;
  *n_sets = 0;
  SW_TRY(A(s, &s->knn_dist, std::max<size_t>(1, n), true));
  SW_TRY(A(s, &s->w_dist, std::max<size_t>(1, n), true));
  if (n_s == 0) {
    if (!sets.alloc(16)) return fail(s, SW_ERR_NO_MEMORY, "set table allocation failed");
    return SW_OK;
  }
  Tmp keys(s, n * 8), keys2(s, n * 8), vals(s, n * 4), perm(s, n * 4), head(s, n * 4);
  if (!keys.p || !keys2.p || !vals.p || !perm.p || !head.p) return fail(s, SW_ERR_NO_MEMORY, "set-up scratch allocation failed");
  SW_CUDA(s, cudaMemcpyAsync(s->knn_dist, tknn, n * 16, cudaMemcpyDeviceToDevice, st));
  SW_CUDA(s, cudaMemcpyAsync(s->w_dist, tw, n * 16, cudaMemcpyDeviceToDevice, st));
  k_set_keys<<<(n_s + 255) / 256, 256, 0, st>>>(tknn, n_s, keys.as<unsigned long long>(), vals.as<int>());
  const size_t sort_bytes = sort_scratch_bytes_u64(n_s, true), scan_bytes = scan_scratch_bytes(n_s);
  Tmp sorttmp(s, std::max(sort_bytes, scan_bytes));
  if (!sorttmp.p) return fail(s, SW_ERR_NO_MEMORY, "sort scratch allocation failed");
  SW_CUDA(s, radix_sort_u64(keys.as<unsigned long long>(), keys2.as<unsigned long long>(), vals.as<int>(),
                            perm.as<int>(), n_s, 0, 64, sorttmp.p, sort_bytes, st));
  k_gather_model<<<(n_s + 255) / 256, 256, 0, st>>>(h, keys2.as<unsigned long long>(), perm.as<int>(), tv, tn, tt,
                                                    tknn, tw, head.as<int>());
  SW_CUDA(s, scan_sum(head.as<int>(), h.set_id, n_s, true, sorttmp.p, scan_bytes, st));
  k_minus_one<<<(n_s + 255) / 256, 256, 0, st>>>(h.set_id, n_s);
  int last = 0;
  SW_CUDA(s, cudaMemcpyAsync(&last, h.set_id + n_s - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  SW_CUDA(s, cudaStreamSynchronize(st));
  *n_sets = last + 1;
  if (!sets.alloc((size_t)*n_sets * 16)) return fail(s, SW_ERR_NO_MEMORY, "set table allocation failed");
  k_set_nodes<<<(n_s + 255) / 256, 256, 0, st>>>(h, head.as<int>(), sets.as<int4>());
  SW_CUDA(s, cudaGetLastError());
  return SW_OK;
}

// The cluster size of the cluster PCG on the current device (16 CTAs where
// the hardware runs such clusters, else 8, else 0: no cluster PCG), found
// once per device with a modest shared-memory request.
int device_cluster_ctas(int precision) {
  static std::mutex mu;
  static std::map<int, int> known;   // device -> cluster size
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find(dev);
  if (it != known.end()) return it->second;
  int C = 0;
  for (int c : {16, 8})
    if (cluster_pcg_fits(precision, c, 64 * 1024)) { C = c; break; }
  known[dev] = C;
  return C;
}

// The cluster PCG's plan for the stream's JᵀJ pattern (FP32 modes), built on
// the host from the pattern and the node positions, or none when the system
// does not fit one cluster's shared memory.
sw_status build_plan(sw_stream* s) {
  SwDev& h = s->h;
  h.cplan = nullptr;
  s->cplan_ctas = 0;
  s->cplan_smem = 0;
  if (h.precision == SW_PRECISION_FP64 || h.n_n < 1) return SW_OK;
  const int C = device_cluster_ctas(h.precision);
  if (C == 0) return SW_OK;
  const int n_n = h.n_n, nnzb = h.nnzb;
  std::vector<int> rp(n_n + 1), col(nnzb);
  std::vector<float> node4((size_t)n_n * 4);
  SW_CUDA(s, cudaMemcpyAsync(rp.data(), h.row_ptr, (n_n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaMemcpyAsync(col.data(), h.col, nnzb * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaMemcpyAsync(node4.data(), h.node_p, node4.size() * sizeof(float), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t limit = optin > 4096 ? (size_t)optin - 2048 : 0;   // the kernel's static shared memory
  std::vector<int> plan;
  size_t smem = 0;
  if (!build_cluster_plan(C, n_n, rp, col, node4, limit, plan, &smem)) return SW_OK;
  if (!cluster_pcg_fits(h.precision, C, smem)) return SW_OK;
  int* dp = nullptr;
  SW_TRY(A(s, &dp, plan.size(), true));
  SW_CUDA(s, cudaMemcpyAsync(dp, plan.data(), plan.size() * sizeof(int), cudaMemcpyHostToDevice, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  h.cplan = dp;
  s->cplan_ctas = C;
  s->cplan_smem = smem;
  return SW_OK;
}

// The JᵀJ pattern from the surfels' sets (device) and the node graph, built
// on the device; the system is cleared, the stream re-described to its runner
// and warped live.  `graph_changed`: the node graph's in-edge lists are
// rebuilt too (set-up), or kept (appending leaves the nodes alone).
sw_status install_pattern(sw_stream* s, const int4* sets, int n_sets, bool graph_changed) {
  SwDev& h = s->h;
  cudaStream_t st = s->st;
  const int n_n = h.n_n, n_s = h.n_s;
  if (graph_changed) {
    std::vector<int> graph((size_t)n_n * SW_K_GRAPH), in_ptr, in_src;
    SW_CUDA(s, cudaMemcpyAsync(graph.data(), h.graph, graph.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    SW_CUDA(s, cudaStreamSynchronize(st));
    std::string why;
    if (!build_in_edges(n_n, graph, in_ptr, in_src, why)) return fail(s, SW_ERR_INVALID_ARG, why);
    SW_CUDA(s, cudaMemcpyAsync(h.in_ptr, in_ptr.data(), (n_n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    SW_CUDA(s, cudaMemcpyAsync(h.in_src, in_src.data(), in_src.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  const int K = 10 * n_sets + (1 + SW_K_GRAPH) * n_n;
  Tmp keys(s, (size_t)K * 4), skeys(s, (size_t)K * 4), flag(s, (size_t)K * 4), pos(s, (size_t)K * 4), cnt(s, 16);
  Tmp tmp(s, pattern_scratch_bytes(K, 2 * K));
  if (!keys.p || !skeys.p || !flag.p || !pos.p || !cnt.p || !tmp.p)
    return fail(s, SW_ERR_NO_MEMORY, "pattern scratch allocation failed");
  PatternScratch w{keys.as<uint32_t>(), skeys.as<uint32_t>(), flag.as<int>(), pos.as<int>(), cnt.as<int>(), tmp.p,
                   pattern_scratch_bytes(K, 2 * K)};
  SW_CUDA(s, launch_pattern_blocks(sets, n_sets, h.graph, n_n, w, st));
  int nnzb = 0;
  SW_CUDA(s, cudaMemcpyAsync(&nnzb, w.count, sizeof(int), cudaMemcpyDeviceToHost, st));
  SW_CUDA(s, cudaStreamSynchronize(st));
  h.n_sets = n_sets;
  s->sorted_sets = n_sets;
  h.nnzb = nnzb;
  SW_TRY(A(s, &h.col, nnzb, true));
  SW_TRY(A(s, &h.blk_row, nnzb, true));
  SW_TRY(A(s, &h.blk_edge, nnzb, true));
  SW_TRY(A(s, &h.rl_ent, (size_t)2 * nnzb - n_n, true));
  SW_TRY(A(s, &h.set_slots, (size_t)std::max(1, n_sets) * 14, true));
  {
    Tmp rlk(s, (size_t)nnzb * 16), rlsk(s, (size_t)nnzb * 16);
    if (!rlk.p || !rlsk.p) return fail(s, SW_ERR_NO_MEMORY, "pattern scratch allocation failed");
    SW_CUDA(s, launch_pattern_fill(sets, n_sets, h.graph, n_n, nnzb, w, rlk.as<unsigned long long>(),
                                   rlsk.as<unsigned long long>(), h, st));
    s->rl_ptr_host.resize(n_n + 1);
    SW_CUDA(s, cudaMemcpyAsync(s->rl_ptr_host.data(), h.rl_ptr, (n_n + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    SW_CUDA(s, cudaStreamSynchronize(st));
  }
  SW_TRY(build_plan(s));
  SW_TRY(A(s, &h.A, (size_t)h.nnzb * 36, true));
  SW_TRY(A(s, &h.A2, (size_t)h.nnzb * 36, true));
  SW_CUDA(s, cudaMemsetAsync(h.A, 0, (size_t)h.nnzb * 36 * sizeof(float), st));
  SW_CUDA(s, cudaMemsetAsync(h.A2, 0, (size_t)h.nnzb * 36 * sizeof(float), st));
  if (h.precision == SW_PRECISION_FP64) {
    SW_TRY(A(s, &h.A64, (size_t)h.nnzb * 36, true));
    SW_CUDA(s, cudaMemsetAsync(h.A64, 0, (size_t)h.nnzb * 36 * sizeof(double), st));
  }
  SW_CUDA(s, cudaMemsetAsync(h.g, 0, (size_t)n_n * 6 * sizeof(float), st));
  SW_CUDA(s, cudaMemsetAsync(h.g2, 0, (size_t)n_n * 6 * sizeof(float), st));
  SW_CUDA(s, cudaMemsetAsync(h.corr_pix, 0xff, (size_t)std::max(1, n_s) * sizeof(int), st));
  SW_CUDA(s, cudaMemsetAsync(h.status, 0, sizeof(int), st));
  SW_TRY(sync_desc(s));
  launch_warp_live(s->run->bh, st);
  SW_CUDA(s, cudaGetLastError());
  SW_CUDA(s, cudaStreamSynchronize(st));
  s->has_model = true;
  return SW_OK;
}

sw_status set_model_impl(sw_handle s, const float* v4, const float* n4, const int* t2, int n_s, const float* node4,
                         int n_n, const int* knn_in, const float* w_in) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (n_s < 0 || n_s > s->p.max_surfels) return fail(s, SW_ERR_INVALID_ARG, "n_surfels out of range");
  if (n_n < SW_K_GRAPH + 1 || n_n > s->p.max_nodes) return fail(s, SW_ERR_INVALID_ARG, "n_nodes out of range");
  if ((n_s > 0 && (!v4 || !n4)) || !node4) return fail(s, SW_ERR_INVALID_ARG, "null model array");
  if (knn_in) {   // a restored skinning (distance order): node ids in range and distinct
    for (int i = 0; i < n_s; ++i) {
      const int* k = knn_in + (size_t)i * SW_K_SKIN;
      for (int a = 0; a < SW_K_SKIN; ++a) {
        bool ok = k[a] >= 0 && k[a] < n_n;
        for (int b = 0; b < a; ++b) ok = ok && k[b] != k[a];
        if (!ok) return fail(s, SW_ERR_INVALID_ARG, "restored skinning has a node id out of range or repeated");
      }
    }
  }
  enter(s);
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  if (s->run) drop_graphs(s->run);
  recycle_model(s);
  s->version++;
  s->fused = false;
  s->unsorted = 0;
  SwDev& h = s->h;
  h.n_s = n_s; h.n_n = n_n;
  cudaStream_t st = s->st;
  // nodes, identity transforms, graph
  SW_CUDA(s, cudaMemcpyAsync(h.node_p, node4, (size_t)n_n * sizeof(float4), cudaMemcpyHostToDevice, st));
  k_identity_dq<<<(n_n + 127) / 128, 128, 0, st>>>(h.dq, n_n);
  launch_dq_widen(h, st);
  launch_node_graph(h, st);

  Tmp sets(s);
  int n_sets = 0;
  if (n_s > 0) {
    const size_t n = n_s;
    Tmp tv(s, n * 16), tn(s, n * 16), tt(s, n * 8), tknn(s, n * 16), tw(s, n * 16), ids(s, n * 16), d2(s, n * 16);
    if (!tv.p || !tn.p || !tt.p || !tknn.p || !tw.p || !ids.p || !d2.p)
      return fail(s, SW_ERR_NO_MEMORY, "set-up scratch allocation failed");
    SW_CUDA(s, cudaMemcpyAsync(tv.p, v4, n * 16, cudaMemcpyHostToDevice, st));
    SW_CUDA(s, cudaMemcpyAsync(tn.p, n4, n * 16, cudaMemcpyHostToDevice, st));
    if (t2) SW_CUDA(s, cudaMemcpyAsync(tt.p, t2, n * 8, cudaMemcpyHostToDevice, st));
    else SW_CUDA(s, cudaMemsetAsync(tt.p, 0, n * 8, st));
    if (knn_in) {
      SW_CUDA(s, cudaMemcpyAsync(tknn.p, knn_in, n * 16, cudaMemcpyHostToDevice, st));
      SW_CUDA(s, cudaMemcpyAsync(tw.p, w_in, n * 16, cudaMemcpyHostToDevice, st));
    } else {
      launch_knn_skin(h, tv.as<float4>(), n_s, ids.as<int>(), d2.as<float>(), tknn.as<int4>(), tw.as<float4>(), st);
    }
    SW_TRY(setup_surfels(s, tv.as<float4>(), tn.as<float4>(), tt.as<int2>(), tknn.as<int4>(), tw.as<float4>(), n_s,
                         sets, &n_sets));
  } else {
    SW_TRY(setup_surfels(s, nullptr, nullptr, nullptr, nullptr, nullptr, 0, sets, &n_sets));
  }
  SW_TRY(install_pattern(s, sets.as<int4>(), n_sets, true));
  sets.put();
  release_cache(s);   // set-up scratch and the previous model: a new model starts lean
  return SW_OK;
}
}  // namespace

sw_status sw_set_model(sw_handle s, const float* v4, const float* n4, const int* t2, int n_s, const float* node4,
                       int n_n) {
  return set_model_impl(s, v4, n4, t2, n_s, node4, n_n, nullptr, nullptr);
}

sw_status sw_upload_depth(sw_handle s, const float* depth, int on_device, int frame_id) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!depth) return fail(s, SW_ERR_INVALID_ARG, "null depth");
  const size_t bytes = (size_t)s->h.W * s->h.H * sizeof(float);
  enter(s);
  if (on_device && s->own_stream) SW_CUDA(s, cudaStreamSynchronize(0));   // order after the caller's default-stream work
  SW_CUDA(s, cudaMemcpyAsync(s->h.depth, depth, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s->st));
  Runner* r = s->run;
  std::vector<ProfEvent>* prof = nullptr;
  if (r->profiling) { reset_eager_prof(r); prof = &r->eager_prof; }
  k_frame_begin<<<1, 1, 0, s->st>>>(s->h.t_now, frame_id, s->h.status);
  prof_mark(r, prof, kProfDepth, true, false);
  launch_depth_maps(r->bh, s->st);
  prof_mark(r, prof, kProfDepth, false, false);
  SW_CUDA(s, cudaGetLastError());
  s->has_depth = true;
  s->fused = false;
  return SW_OK;
}

namespace {

// The checked build (-DSW_BOUNDS_CHECK) waits for each per-frame call's
// kernels and reports an index that failed its range check; the status bit
// stays set until the next sw_set_model.  The normal build never sets it.
sw_status bounds_check(sw_stream* s) {
#ifdef SW_BOUNDS_CHECK
  int status = 0;
  SW_CUDA(s, cudaMemcpyAsync(&status, s->h.status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  if (status & kStatusBounds) return fail(s, SW_ERR_BOUNDS, "a device index was out of range (checked build)");
#else
  (void)s;
#endif
  return SW_OK;
}

sw_status read_stats(sw_stream* s, int gn, sw_solve_stats* out) {
  int status = 0;
  SW_CUDA(s, cudaMemcpyAsync(&status, s->h.status, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->gn_iters = gn;
    SW_CUDA(s, cudaMemcpyAsync(out->e_depth, s->h.e_depth, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaMemcpyAsync(out->e_reg, s->h.e_reg, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaMemcpyAsync(out->n_corr, s->h.n_corr, kMaxGn * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaMemcpyAsync(out->pcg_rz, s->h.pcg_rz, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  }
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  if (status & kStatusBounds) return fail(s, SW_ERR_BOUNDS, "a device index was out of range (checked build)");
  if (status & kStatusTimeout)
    return fail(s, SW_ERR_TIMEOUT, "a bounded wait of the PCG gave up (a reduction or a neighbour's vector); "
                                   "the node transforms were left as they were");
  if (status & kStatusDepthTimeout)
    return fail(s, SW_ERR_TIMEOUT, "the depth stage's bounded wait for a TMA tile gave up (the tile was read with "
                                   "plain loads instead)");
  if (status & kStatusBreakdown) return fail(s, SW_ERR_SOLVER_BREAKDOWN, "a diagonal block is not positive definite or pᵀAp <= 0");
  return SW_OK;
}

}  // namespace

sw_status sw_solve_frame(sw_handle s, int gn_iters, int pcg_iters, sw_solve_stats* stats) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "solve needs a model and a depth frame");
  if (gn_iters < 1 || gn_iters > kMaxGn || pcg_iters < 1 || pcg_iters > kMaxPcg)
    return fail(s, SW_ERR_INVALID_ARG, "iteration counts out of range");
  enter(s);
  SW_TRY(runner_solve(s->run, s, gn_iters, pcg_iters));
  if (stats) return read_stats(s, gn_iters, stats);
  return bounds_check(s);
}

sw_status sw_fuse_frame(sw_handle s) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "fusion needs a model and a depth frame");
  enter(s);
  SW_TRY(runner_fuse(s->run, s));
  s->fused = true;
  return bounds_check(s);
}

sw_status sw_read_nodes(sw_handle s, float* pos4, float* dq8, int cap, int* n_out) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  const int n = s->h.n_n;
  if (n_out) *n_out = n;
  enter(s);
  if ((pos4 || dq8) && cap < n) return fail(s, SW_ERR_INVALID_ARG, "capacity too small");
  if (pos4) SW_CUDA(s, cudaMemcpyAsync(pos4, s->h.node_p, (size_t)n * 16, cudaMemcpyDeviceToHost, s->st));
  if (dq8) SW_CUDA(s, cudaMemcpyAsync(dq8, s->h.dq, (size_t)n * 32, cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  int status = 0;
  SW_CUDA(s, cudaMemcpy(&status, s->h.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status & kStatusBounds) return fail(s, SW_ERR_BOUNDS, "a device index was out of range (checked build)");
  if (status & kStatusBreakdown) return fail(s, SW_ERR_SOLVER_BREAKDOWN, "the last solve broke down");
  return SW_OK;
}

// ------------------------------------------------------------------ inspection hooks

namespace {

template <typename T>
sw_status d2h_perm(sw_stream* s, const T* dev, T* host, int per, bool permute) {
  const int n = s->h.n_s;
  std::vector<T> buf((size_t)n * per);
  if (n) SW_CUDA(s, cudaMemcpyAsync(buf.data(), dev, buf.size() * sizeof(T), cudaMemcpyDeviceToHost, s->st));
  std::vector<int> orig(n);
  if (n && permute) SW_CUDA(s, cudaMemcpyAsync(orig.data(), s->h.orig_id, n * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  for (int i = 0; i < n; ++i) {
    const int o = permute ? orig[i] : i;
    std::memcpy(host + (size_t)o * per, buf.data() + (size_t)i * per, per * sizeof(T));
  }
  return SW_OK;
}

template <typename T>
sw_status h2d_perm(sw_stream* s, const T* host, T* dev, int per) {
  const int n = s->h.n_s;
  std::vector<int> orig(n);
  if (n) SW_CUDA(s, cudaMemcpy(orig.data(), s->h.orig_id, n * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<T> buf((size_t)n * per);
  for (int i = 0; i < n; ++i) std::memcpy(buf.data() + (size_t)i * per, host + (size_t)orig[i] * per, per * sizeof(T));
  if (n) SW_CUDA(s, cudaMemcpyAsync(dev, buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status need_model(sw_stream* s, int cap) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  enter(s);
  if (cap < s->h.n_s) return fail(s, SW_ERR_INVALID_ARG, "capacity too small");
  return SW_OK;
}

}  // namespace

sw_status sw_read_surfels(sw_handle s, float* v4, float* n4, int* t2, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  if (n_out) *n_out = s->h.n_s;
  if (v4) SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.v_ref), v4, 4, true));
  if (n4) SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.n_ref), n4, 4, true));
  if (t2) SW_TRY(d2h_perm(s, reinterpret_cast<const int*>(s->h.tt), t2, 2, true));
  return SW_OK;
}

sw_status sw_read_live_surfels(sw_handle s, float* v4, float* n4, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  if (n_out) *n_out = s->h.n_s;
  if (v4) SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.v_live), v4, 4, true));
  if (n4) SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.n_live), n4, 4, true));
  return SW_OK;
}

sw_status sw_read_skinning(sw_handle s, int* knn4, float* w4, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  const int n = s->h.n_s;
  if (n_out) *n_out = n;
  if (knn4 && n) SW_CUDA(s, cudaMemcpyAsync(knn4, s->knn_dist, (size_t)n * 16, cudaMemcpyDeviceToHost, s->st));
  if (w4 && n) SW_CUDA(s, cudaMemcpyAsync(w4, s->w_dist, (size_t)n * 16, cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_read_graph(sw_handle s, int* graph8, int cap) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  if (!graph8 || cap < s->h.n_n) return fail(s, SW_ERR_INVALID_ARG, "bad graph buffer");
  SW_CUDA(s, cudaMemcpyAsync(graph8, s->h.graph, (size_t)s->h.n_n * SW_K_GRAPH * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_read_maps(sw_handle s, float* V4, float* N4) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "no depth frame");
  enter(s);
  const size_t np = (size_t)s->h.W * s->h.H;
  if (V4) SW_CUDA(s, cudaMemcpyAsync(V4, s->h.vmap, np * 16, cudaMemcpyDeviceToHost, s->st));
  if (N4) SW_CUDA(s, cudaMemcpyAsync(N4, s->h.nmap, np * 16, cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_debug_set_maps(sw_handle s, const float* V4, const float* N4) {
  if (!s || !V4 || !N4) return fail(s, SW_ERR_INVALID_ARG, "null argument");
  const size_t np = (size_t)s->h.W * s->h.H;
  SW_CUDA(s, cudaMemcpyAsync(s->h.vmap, V4, np * 16, cudaMemcpyHostToDevice, s->st));
  SW_CUDA(s, cudaMemcpyAsync(s->h.nmap, N4, np * 16, cudaMemcpyHostToDevice, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  s->has_depth = true;
  s->fused = false;
  return SW_OK;
}

sw_status sw_set_node_dq(sw_handle s, const float* dq8, int n) {
  if (!s || !dq8) return fail(s, SW_ERR_INVALID_ARG, "null argument");
  if (!s->has_model || n != s->h.n_n) return fail(s, SW_ERR_INVALID_ARG, "node count mismatch");
  SW_CUDA(s, cudaMemcpyAsync(s->h.dq, dq8, (size_t)n * 32, cudaMemcpyHostToDevice, s->st));
  launch_dq_widen(s->h, s->st);
  SW_CUDA(s, cudaGetLastError());
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_debug_set_skin_node(sw_handle s, int surfel, int slot, int node) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  if (surfel < 0 || surfel >= s->h.n_s || slot < 0 || slot > 3)
    return fail(s, SW_ERR_INVALID_ARG, "surfel or slot out of range");
  // inside the node arrays' allocation (max_nodes), whatever n_nodes is
  if (node < 0 || node >= s->p.max_nodes) return fail(s, SW_ERR_INVALID_ARG, "node outside [0, max_nodes)");
  enter(s);
  SW_CUDA(s, cudaMemcpyAsync(reinterpret_cast<int*>(s->h.knn + surfel) + slot, &node, sizeof(int),
                             cudaMemcpyHostToDevice, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_debug_record_correspondence(sw_handle s, int enable) {
  if (!s || (enable != 0 && enable != 1)) return fail(s, SW_ERR_INVALID_ARG, "bad argument");
  if (enable && !s->corr_rec_buf)
    SW_TRY(A(s, &s->corr_rec_buf, (size_t)kMaxGn * std::max(1, s->p.max_surfels)));
  int* want = enable ? s->corr_rec_buf : nullptr;
  if (s->h.corr_rec != want) {
    SW_CUDA(s, cudaStreamSynchronize(s->st));
    s->h.corr_rec = want;
    // the runners' device tables carry the pointer: the stream's own is
    // rebuilt now, a batch's at its next call
    s->version++;
    if (s->has_model && s->run) SW_TRY(build_runner(s->run, s));
  }
  return SW_OK;
}

sw_status sw_read_correspondence_iter(sw_handle s, int gn_iter, int* pix, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  if (!s->h.corr_rec) return fail(s, SW_ERR_NOT_INITIALIZED, "recording is off (sw_debug_record_correspondence)");
  if (gn_iter < 0 || gn_iter >= kMaxGn) return fail(s, SW_ERR_INVALID_ARG, "gn_iter out of range");
  if (n_out) *n_out = s->h.n_s;
  if (pix) SW_TRY(d2h_perm(s, s->h.corr_rec + (size_t)gn_iter * s->h.n_s, pix, 1, true));
  return SW_OK;
}

sw_status sw_read_correspondence(sw_handle s, int* pix, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  if (n_out) *n_out = s->h.n_s;
  if (pix) SW_TRY(d2h_perm(s, s->h.corr_pix, pix, 1, true));
  return SW_OK;
}

sw_status sw_debug_set_live(sw_handle s, const float* v4, const float* n4, int n) {
  SW_TRY(need_model(s, n));
  if (n != s->h.n_s || !v4 || !n4) return fail(s, SW_ERR_INVALID_ARG, "surfel count mismatch");
  // keep each surfel's radius / confidence in .w
  std::vector<float> v((size_t)n * 4), nn((size_t)n * 4), vr((size_t)n * 4), nr((size_t)n * 4);
  SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.v_ref), vr.data(), 4, true));
  SW_TRY(d2h_perm(s, reinterpret_cast<const float*>(s->h.n_ref), nr.data(), 4, true));
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) { v[4 * i + k] = v4[4 * i + k]; nn[4 * i + k] = n4[4 * i + k]; }
    v[4 * i + 3] = vr[4 * i + 3];
    nn[4 * i + 3] = nr[4 * i + 3];
  }
  SW_TRY(h2d_perm(s, v.data(), reinterpret_cast<float*>(s->h.v_live), 4));
  SW_TRY(h2d_perm(s, nn.data(), reinterpret_cast<float*>(s->h.n_live), 4));
  return SW_OK;
}

sw_status sw_debug_associate(sw_handle s) {
  SW_TRY(need_model(s, s ? s->h.n_s : 0));
  if (!s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "no depth frame");
  launch_associate_only(s->run->bh, s->st);
  SW_CUDA(s, cudaGetLastError());
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_debug_fusion_targets(sw_handle s, int* target, int* imap) {
  SW_TRY(need_model(s, s ? s->h.n_s : 0));
  if (!s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "no depth frame");
  const size_t np = (size_t)s->h.W * s->h.H;
  SW_CUDA(s, cudaMemsetAsync(s->h.imap, 0xff, 16 * np * sizeof(unsigned long long), s->st));
  launch_index_map(s->run->bh, s->st);
  launch_fuse(s->run->bh, 1, s->st);
  SW_CUDA(s, cudaGetLastError());
  std::vector<int> t(np), orig(std::max(1, s->h.n_s));
  SW_CUDA(s, cudaMemcpyAsync(t.data(), s->h.fuse_target, np * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  if (s->h.n_s) SW_CUDA(s, cudaMemcpyAsync(orig.data(), s->h.orig_id, s->h.n_s * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  std::vector<unsigned long long> im;
  if (imap) {
    im.resize(16 * np);
    SW_CUDA(s, cudaMemcpyAsync(im.data(), s->h.imap, im.size() * 8, cudaMemcpyDeviceToHost, s->st));
  }
  SW_CUDA(s, cudaMemsetAsync(s->h.imap, 0xff, 16 * np * sizeof(unsigned long long), s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  s->fused = true;
  if (target)
    for (size_t p = 0; p < np; ++p) target[p] = t[p] < 0 ? -1 : orig[t[p]];
  if (imap)
    for (size_t p = 0; p < im.size(); ++p) imap[p] = im[p] == ~0ull ? -1 : (int)(im[p] & 0xffffffffu);
  return SW_OK;
}

namespace {
sw_status ensure_append_bufs(sw_stream* s) {
  if (s->app_ready) return SW_OK;
  AppendBufs& a = s->app;
  const size_t np = (size_t)s->h.W * s->h.H, nn = std::max(1, s->p.max_nodes);
  const size_t nmax = std::max(np, (size_t)std::max(1, s->p.max_surfels));
  SW_TRY(A(s, &a.live, nn)); SW_TRY(A(s, &a.cand, np)); SW_TRY(A(s, &a.query, np)); SW_TRY(A(s, &a.knn, 4 * np));
  SW_TRY(A(s, &a.flags, np)); SW_TRY(A(s, &a.wsum, np)); SW_TRY(A(s, &a.strain, 9 * np)); SW_TRY(A(s, &a.w, np));
  SW_TRY(A(s, &a.v, np)); SW_TRY(A(s, &a.n, np)); SW_TRY(A(s, &a.acc, np)); SW_TRY(A(s, &a.stay, nmax));
  SW_TRY(A(s, &a.pos, nmax)); SW_TRY(A(s, &a.counts, kAppCounts));
  a.scan_bytes = append_scan_bytes((int)np, (int)nmax);
  unsigned char* tmp = nullptr;
  SW_TRY(A(s, &tmp, std::max<size_t>(16, a.scan_bytes)));
  SW_CUDA(s, cudaMemsetAsync(tmp, 0, 16, s->st));   // the scans' ticket counter (each scan leaves it 0)
  a.scan_tmp = tmp;
  s->app_ready = true;
  return SW_OK;
}
}  // namespace

sw_status sw_append_frame(sw_handle s, sw_append_stats* stats) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "appending needs a model and a depth frame");
  if (!s->fused) return fail(s, SW_ERR_NOT_INITIALIZED, "no fusion since the last depth frame");
  enter(s);
  SW_TRY(ensure_append_bufs(s));
  const AppendBufs& a = s->app;
  SwDev& h = s->h;
  cudaStream_t st = s->st;
  const double eps = s->p.eps;
  AppendParams ap;
  ap.lo2 = (float)((1.0 - eps) * (1.0 - eps));
  ap.hi2 = (float)((1.0 + eps) * (1.0 + eps));
  ap.bound2 = (1.0 + eps) * (1.0 + eps);
  ap.delta_nn = s->p.delta_nn;
  ap.h = s->p.fd_step;
  ap.t_low = s->p.t_low_confid;
  int counts[kAppCounts];
  cudaEvent_t ev0 = take_event(s->run), ev1 = take_event(s->run);
  SW_CUDA(s, cudaEventRecord(ev0, st));
  SW_CUDA(s, launch_append_candidates(h, a, st));
  SW_CUDA(s, cudaMemcpyAsync(counts, a.counts, sizeof(counts), cudaMemcpyDeviceToHost, st));
  SW_CUDA(s, cudaStreamSynchronize(st));
  const int n_cand = counts[kAppNCand];
  SW_CUDA(s, launch_append_eval(h, a, ap, n_cand, st));
  SW_CUDA(s, launch_append_removal(h, a, ap.t_low, st));
  SW_CUDA(s, cudaMemcpyAsync(counts, a.counts, sizeof(counts), cudaMemcpyDeviceToHost, st));
  SW_CUDA(s, cudaStreamSynchronize(st));
  const int n_stay = counts[kAppNStay];
  const int n_app = std::min(counts[kAppNAcc], std::max(0, s->p.max_surfels - n_stay));
  const int n_new = n_stay + n_app, n_old = h.n_s;
  if (stats) {
    stats->candidates = n_cand;
    stats->rejected_nn = counts[kAppNLow];
    stats->rejected_strain = counts[kAppNComp];
    stats->appended = n_app;
    stats->removed = n_old - n_stay;
    stats->n_surfels = n_new;
    stats->kernel_ms = stats->rebuild_ms = 0.0;
    stats->new_nodes = 0;
    stats->resorted = 0;
  }
  s->app_last_cand = n_cand;
  if (n_app == 0 && n_stay == n_old) {   // nothing appended or removed: the model stands as it is
    SW_CUDA(s, cudaEventRecord(ev1, st));
    SW_CUDA(s, cudaEventSynchronize(ev1));
    float kms = 0.f;
    cudaEventElapsedTime(&kms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (stats) stats->kernel_ms = kms;
    s->fused = false;
    return bounds_check(s);
  }
  {
    const size_t n = std::max(1, n_new), m = std::max(1, n_app);
    Tmp tv(s, n * 16), tn(s, n * 16), tt(s, n * 8), tknn(s, n * 16), tw(s, n * 16), ids(s, m * 16), d2(s, m * 16);
    if (!tv.p || !tn.p || !tt.p || !tknn.p || !tw.p || !ids.p || !d2.p)
      return fail(s, SW_ERR_NO_MEMORY, "appending scratch allocation failed");
    launch_append_compose(h, a, s->knn_dist, s->w_dist, n_stay, n_app, tv.as<float4>(), tn.as<float4>(),
                          tt.as<int2>(), tknn.as<int4>(), tw.as<float4>(), st);
    launch_knn_skin(h, tv.as<float4>() + n_stay, n_app, ids.as<int>(), d2.as<float>(), tknn.as<int4>() + n_stay,
                    tw.as<float4>() + n_stay, st);
    // node-graph extension over the appended surfels (Sec. 6.4, last paragraph)
    int new_nodes = 0;
    const int n_old_nodes = h.n_n;
    if (s->p.extend_nodes && n_app > 0 && h.n_n < s->p.max_nodes) {
      Tmp unc(s, (size_t)n_app * 4), list(s, (size_t)n_app * 4), cnt(s, 16), sig(s, (size_t)n_app * 20 + 16), near(s, (size_t)n_app * 8);
      if (!unc.p || !list.p || !cnt.p || !sig.p || !near.p)
        return fail(s, SW_ERR_NO_MEMORY, "node extension scratch allocation failed");
      launch_node_cover(h, tv.as<float4>(), n_stay, n_app, unc.as<int>(), st);
      SW_CUDA(s, launch_node_subsample(h, a, tv.as<float4>(), n_stay, n_app, unc.as<int>(), list.as<int>(),
                                       cnt.as<int>(), sig.as<float>(), near.as<int>(), n_old_nodes,
                                       s->p.max_nodes - n_old_nodes, cnt.as<int>() + 1, st));
      SW_CUDA(s, cudaMemcpyAsync(&new_nodes, cnt.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      SW_CUDA(s, cudaStreamSynchronize(st));
      if (new_nodes > 0) {
        Tmp nid(s, (size_t)new_nodes * 16);
        if (!nid.p) return fail(s, SW_ERR_NO_MEMORY, "node extension scratch allocation failed");
        launch_knn4(h.node_p + n_old_nodes, new_nodes, h.node_p, n_old_nodes, nid.as<int>(), st);
        launch_new_node_dq(h, n_old_nodes, new_nodes, nid.as<int>(), st);
        h.n_n = n_old_nodes + new_nodes;
        launch_node_graph(h, st);
        launch_skin_merge(h, tv.as<float4>(), n_new, n_old_nodes, tknn.as<int4>(), tw.as<float4>(), st);
        SW_CUDA(s, cudaStreamSynchronize(st));
      }
    }
    if (stats) stats->new_nodes = new_nodes;
    SW_CUDA(s, cudaGetLastError());
    SW_CUDA(s, cudaEventRecord(ev1, st));
    const auto t0 = std::chrono::steady_clock::now();
    auto finish = [&](int resorted) -> sw_status {
      float kms = 0.f;
      cudaEventElapsedTime(&kms, ev0, ev1);   // both are complete: the caller synchronised
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      if (stats) {
        stats->kernel_ms = kms;
        stats->rebuild_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      }
      if (stats) stats->resorted = resorted;
      s->fused = false;
      return bounds_check(s);
    };
    // Fast update: nothing removed, no new node, and the surfels appended
    // since the last set sort a small share of the model.  Each appended
    // surfel takes its node set's id: a known set's, or a new one added after
    // the known sets.  The appended surfels follow the sorted ones in the
    // internal order (the data term sums runs of equal sets, so any order is
    // correct; the sort only keeps the runs long).  The JᵀJ pattern stays when
    // every new set's node pairs are blocks of it already, else it is rebuilt
    // from the extended set table (the surfels keep their order).
    if (n_stay == n_old && new_nodes == 0 && n_app > 0 && (s->unsorted + n_app) * 16 <= n_new) {
      Tmp set_of(s, (size_t)n_app * 4), keys(s, (size_t)n_app * 8), miss(s, 16);
      if (!set_of.p || !keys.p || !miss.p) return fail(s, SW_ERR_NO_MEMORY, "appending scratch allocation failed");
      SW_CUDA(s, cudaMemsetAsync(miss.p, 0, 4 * sizeof(int), st));
      launch_find_sets(h, s->sorted_sets, tknn.as<int4>(), n_stay, n_app, set_of.as<int>(),
                       keys.as<unsigned long long>(), miss.as<int>(), st);
      int cnt[4] = {0, 0, 0, 0};
      SW_CUDA(s, cudaMemcpyAsync(cnt, miss.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
      SW_CUDA(s, cudaStreamSynchronize(st));
      int n_sets_all = h.n_sets;
      bool new_pairs = false;
      // from here the model changes: a failure leaves the stream without one
      // (as a failed rebuild does) until the next sw_set_model or import
      s->has_model = false;
      if (cnt[0] > 0) {
        // the new sets' slots go after the known sets' (the table grows if needed)
        SW_TRY(grow_model_block(s, reinterpret_cast<void**>(&h.set_slots), (size_t)h.n_sets * 14 * sizeof(int),
                                (size_t)(h.n_sets + cnt[0]) * 14 * sizeof(int)));
        const size_t nb = new_sets_scratch_bytes(n_app);
        Tmp sorted(s, (size_t)n_app * 8), head(s, (size_t)n_app * 4), rank(s, (size_t)n_app * 4), tmp(s, nb);
        if (!sorted.p || !head.p || !rank.p || !tmp.p)
          return fail(s, SW_ERR_NO_MEMORY, "appending scratch allocation failed");
        SW_CUDA(s, launch_new_sets(h, keys.as<unsigned long long>(), sorted.as<unsigned long long>(), head.as<int>(),
                                   rank.as<int>(), n_app, cnt[0], set_of.as<int>(), miss.as<int>() + 1,
                                   miss.as<int>() + 2, tmp.p, nb, st));
        SW_CUDA(s, cudaMemcpyAsync(cnt, miss.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        SW_CUDA(s, cudaStreamSynchronize(st));
        n_sets_all = h.n_sets + cnt[1];
        if (cnt[2] == 0) h.n_sets = n_sets_all;   // the new sets' slots are complete
        else new_pairs = true;                    // a pair of nodes has no block yet
      }
      // the caller-order skinning copies grow into a larger block if needed
      SW_TRY(grow_model_block(s, reinterpret_cast<void**>(&s->knn_dist), (size_t)n_old * 16, (size_t)n_new * 16));
      SW_TRY(grow_model_block(s, reinterpret_cast<void**>(&s->w_dist), (size_t)n_old * 16, (size_t)n_new * 16));
      SW_CUDA(s, cudaMemcpyAsync(s->knn_dist + n_old, tknn.as<int4>() + n_stay, (size_t)n_app * 16,
                                 cudaMemcpyDeviceToDevice, st));
      SW_CUDA(s, cudaMemcpyAsync(s->w_dist + n_old, tw.as<float4>() + n_stay, (size_t)n_app * 16,
                                 cudaMemcpyDeviceToDevice, st));
      launch_append_internal(h, tv.as<float4>(), tn.as<float4>(), tt.as<int2>(), tknn.as<int4>(), tw.as<float4>(),
                             n_old, n_app, set_of.as<int>(), st);
      SW_CUDA(s, cudaGetLastError());
      if (s->run) drop_graphs(s->run);
      s->version++;
      h.n_s = n_new;
      s->unsorted += n_app;
      if (!new_pairs) {
        SW_TRY(sync_desc(s));
        launch_warp_live(s->run->bh, st);
        SW_CUDA(s, cudaGetLastError());
        SW_CUDA(s, cudaStreamSynchronize(st));
        s->has_model = true;
        return finish(0);
      }
      // the pattern gains the new sets' node pairs: rebuilt from the set
      // table (known sets first, in their order), the surfels untouched
      Tmp all_sets(s, (size_t)n_sets_all * 16);
      if (!all_sets.p) return fail(s, SW_ERR_NO_MEMORY, "appending scratch allocation failed");
      launch_slot_sets(h.set_slots, n_sets_all, all_sets.as<int4>(), st);
      SW_CUDA(s, cudaGetLastError());
      const int sorted_sets = s->sorted_sets;
      recycle_blocks(s, {h.col, h.blk_row, h.blk_edge, h.rl_ent, h.set_slots, h.A, h.A2, h.A64, h.cplan});
      SW_TRY(install_pattern(s, all_sets.as<int4>(), n_sets_all, false));
      s->sorted_sets = sorted_sets;
      return finish(2);
    }
    s->unsorted = 0;
    SW_TRY(bounds_check(s));   // checked build: before the rebuild clears the status
    // the model's layout changes: rebuild its structure (nodes and transforms
    // stay).  The old model's blocks go back to the cache while the kernels
    // above may still read them: anything that reuses them is later on the
    // same stream.
    s->has_model = false;
    if (s->run) drop_graphs(s->run);
    recycle_model(s);
    s->version++;
    h.n_s = n_new;
    Tmp sets(s);
    int n_sets = 0;
    SW_TRY(setup_surfels(s, tv.as<float4>(), tn.as<float4>(), tt.as<int2>(), tknn.as<int4>(), tw.as<float4>(),
                         n_new, sets, &n_sets));
    SW_TRY(install_pattern(s, sets.as<int4>(), n_sets, new_nodes > 0));
    return finish(1);
  }
}

sw_status sw_debug_read_append(sw_handle s, int* pix, int* knn4, int* flags, double* wsum, double* strain9,
                               float* w4, float* v4, float* n4, int cap, int* n_out) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->app_ready) return fail(s, SW_ERR_NOT_INITIALIZED, "no appending step has run");
  const int n = s->app_last_cand;
  if (n_out) *n_out = n;
  if (!pix && !knn4 && !flags && !wsum && !strain9 && !w4 && !v4 && !n4) return SW_OK;   // count only
  if (cap < n) return fail(s, SW_ERR_INVALID_ARG, "capacity too small");
  const AppendBufs& a = s->app;
  auto get = [&](void* dst, const void* src, size_t bytes) -> sw_status {
    if (dst && bytes) SW_CUDA(s, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->st));
    return SW_OK;
  };
  SW_TRY(get(pix, a.cand, (size_t)n * 4));
  SW_TRY(get(knn4, a.knn, (size_t)n * 16));
  SW_TRY(get(flags, a.flags, (size_t)n * 4));
  SW_TRY(get(wsum, a.wsum, (size_t)n * 8));
  SW_TRY(get(strain9, a.strain, (size_t)n * 72));
  SW_TRY(get(w4, a.w, (size_t)n * 16));
  SW_TRY(get(v4, a.v, (size_t)n * 16));
  SW_TRY(get(n4, a.n, (size_t)n * 16));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

sw_status sw_debug_visibility(sw_handle s, int* vis_map, int* visible) {
  SW_TRY(need_model(s, s ? s->h.n_s : 0));
  if (!s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "no depth frame");
  const size_t np = (size_t)s->h.W * s->h.H;
  const int n = s->h.n_s;
  launch_vis_splat(s->run->bh, 1, s->st);
  std::vector<unsigned long long> vm(np);
  SW_CUDA(s, cudaMemcpyAsync(vm.data(), s->h.vis_map, np * 8, cudaMemcpyDeviceToHost, s->st));
  launch_vis_mark(s->run->bh, 1, s->st);
  SW_CUDA(s, cudaGetLastError());
  std::vector<int> vis(std::max(1, n)), orig(std::max(1, n));
  if (n) {
    SW_CUDA(s, cudaMemcpyAsync(vis.data(), s->h.visible, n * sizeof(int), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaMemcpyAsync(orig.data(), s->h.orig_id, n * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  }
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  if (vis_map)
    for (size_t p = 0; p < np; ++p) vis_map[p] = vm[p] == ~0ull ? -1 : (int)(vm[p] & 0xffffffffu);
  if (visible)
    for (int i = 0; i < n; ++i) visible[orig[i]] = vis[i];
  return SW_OK;
}

sw_status sw_debug_assemble(sw_handle s, int* nnzb_out, int* n_corr_out) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "needs a model and a depth frame");
  launch_solve_begin(s->run->bh, s->st);
  if (s->h.precision == SW_PRECISION_FP64) {
    launch_reg_assemble64(s->run->bh, 0, s->st);
    launch_data_assemble64(s->run->bh, 0, s->st);
  } else {
    launch_system_clear(s->run->bh, s->st);
    launch_assemble(s->run->bh, 0, s->st);
    s->last_sys = 0;
  }
  SW_CUDA(s, cudaGetLastError());
  int nc = 0;
  SW_CUDA(s, cudaMemcpyAsync(&nc, s->h.n_corr, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  if (nnzb_out) *nnzb_out = s->h.nnzb;
  if (n_corr_out) *n_corr_out = nc;
  return SW_OK;
}

sw_status sw_debug_read_jtj(sw_handle s, int* rows, int* cols, float* vals, float* g, int cap_blocks) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  const int nb = s->h.nnzb;
  if (cap_blocks < nb) return fail(s, SW_ERR_INVALID_ARG, "capacity too small");
  if (rows) SW_CUDA(s, cudaMemcpyAsync(rows, s->h.blk_row, nb * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  if (cols) SW_CUDA(s, cudaMemcpyAsync(cols, s->h.col, nb * sizeof(int), cudaMemcpyDeviceToHost, s->st));
  if (s->h.precision == SW_PRECISION_FP64) {   // the FP64 system, rounded for the caller
    std::vector<double> va(vals ? (size_t)nb * 36 : 0), vg(g ? (size_t)s->h.n_n * 6 : 0);
    if (vals) SW_CUDA(s, cudaMemcpyAsync(va.data(), s->h.A64, va.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    if (g) SW_CUDA(s, cudaMemcpyAsync(vg.data(), s->h.g64, vg.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaStreamSynchronize(s->st));
    for (size_t k = 0; k < va.size(); ++k) vals[k] = (float)va[k];
    for (size_t k = 0; k < vg.size(); ++k) g[k] = (float)vg[k];
    return SW_OK;
  }
  const float* sa = s->last_sys ? s->h.A2 : s->h.A;
  const float* sg = s->last_sys ? s->h.g2 : s->h.g;
  if (vals) SW_CUDA(s, cudaMemcpyAsync(vals, sa, (size_t)nb * 36 * sizeof(float), cudaMemcpyDeviceToHost, s->st));
  if (g) SW_CUDA(s, cudaMemcpyAsync(g, sg, (size_t)s->h.n_n * 6 * sizeof(float), cudaMemcpyDeviceToHost, s->st));
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  return SW_OK;
}

// ------------------------------------------------------------------ checkpoint

namespace {
constexpr uint32_t kStateMagic = 0x53574731u;   // "SWG1"
struct StateHeader {
  uint32_t magic;
  int n_s, n_n, W, H, t_now;
};
}  // namespace

sw_status sw_export_state(sw_handle s, void* buf, size_t* bytes) {
  if (!s || !bytes) return fail(s, SW_ERR_INVALID_ARG, "null argument");
  if (!s->has_model) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  const int n = s->h.n_s, m = s->h.n_n;
  const size_t need = sizeof(StateHeader) + (size_t)n * (16 + 16 + 8 + 16 + 16) + (size_t)m * (16 + 32);
  if (!buf) { *bytes = need; return SW_OK; }
  if (*bytes < need) return fail(s, SW_ERR_INVALID_ARG, "state buffer too small");
  char* p = static_cast<char*>(buf);
  int t_now = 0;
  SW_CUDA(s, cudaMemcpy(&t_now, s->h.t_now, sizeof(int), cudaMemcpyDeviceToHost));
  StateHeader hd{kStateMagic, n, m, s->h.W, s->h.H, t_now};
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  SW_TRY(sw_read_surfels(s, reinterpret_cast<float*>(p), reinterpret_cast<float*>(p + (size_t)n * 16),
                         reinterpret_cast<int*>(p + (size_t)n * 32), n, nullptr));
  p += (size_t)n * 40;
  SW_TRY(sw_read_skinning(s, reinterpret_cast<int*>(p), reinterpret_cast<float*>(p + (size_t)n * 16), n, nullptr));
  p += (size_t)n * 32;
  SW_TRY(sw_read_nodes(s, reinterpret_cast<float*>(p), reinterpret_cast<float*>(p + (size_t)m * 16), m, nullptr));
  *bytes = need;
  return SW_OK;
}

sw_status sw_import_state(sw_handle s, const void* buf, size_t bytes) {
  if (!s || !buf || bytes < sizeof(StateHeader)) return fail(s, SW_ERR_INVALID_ARG, "bad state buffer");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.W != s->h.W || hd.H != s->h.H) return fail(s, SW_ERR_INVALID_ARG, "state does not match the stream");
  const int n = hd.n_s, m = hd.n_n;
  if (bytes < sizeof(StateHeader) + (size_t)n * 72 + (size_t)m * 48) return fail(s, SW_ERR_INVALID_ARG, "state truncated");
  if (n > s->p.max_surfels || m > s->p.max_nodes) return fail(s, SW_ERR_INVALID_ARG, "state exceeds the stream capacity");
  const char* p = static_cast<const char*>(buf) + sizeof(StateHeader);
  const float* v4 = reinterpret_cast<const float*>(p);
  const float* n4 = reinterpret_cast<const float*>(p + (size_t)n * 16);
  const int* t2 = reinterpret_cast<const int*>(p + (size_t)n * 32);
  const int* knn = reinterpret_cast<const int*>(p + (size_t)n * 40);
  const float* w = reinterpret_cast<const float*>(p + (size_t)n * 56);
  const float* node4 = reinterpret_cast<const float*>(p + (size_t)n * 72);
  const float* dq8 = node4 + (size_t)m * 4;
  SW_TRY(set_model_impl(s, v4, n4, t2, n, node4, m, knn, w));
  k_set_int<<<1, 1, 0, s->st>>>(s->h.t_now, hd.t_now);
  SW_TRY(sw_set_node_dq(s, dq8, m));
  return SW_OK;
}

const char* sw_last_error(sw_handle s) {
  if (s) return s->err.c_str();
  static thread_local std::string copy;
  std::lock_guard<std::mutex> lk(g_err_mu);
  copy = g_last_error;
  return copy.c_str();
}

const char* sw_status_string(sw_status s) {
  switch (s) {
    case SW_OK: return "ok";
    case SW_ERR_INVALID_ARG: return "invalid argument";
    case SW_ERR_NO_MEMORY: return "out of device memory budget";
    case SW_ERR_NOT_INITIALIZED: return "not initialized";
    case SW_ERR_SOLVER_BREAKDOWN: return "solver breakdown";
    case SW_ERR_TIMEOUT: return "device wait timed out";
    case SW_ERR_CUDA: return "CUDA error";
    case SW_ERR_BOUNDS: return "device index out of range (checked build)";
  }
  return "unknown status";
}



// ------------------------------------------------------------------ batches

namespace {

// A member's model changed since the batch's tables were built (sw_set_model,
// sw_append_frame): rebuild them, keeping the active flags.
sw_status batch_check(sw_batch* b) {
  if (!b) return fail(nullptr, SW_ERR_INVALID_ARG, "null batch");
  Runner* r = &b->run;
  if (!runner_stale(r)) return SW_OK;
  for (sw_stream* m : r->members)
    if (!m->has_model) return fail(nullptr, SW_ERR_NOT_INITIALIZED, "a batch member has no model");
  const int n = (int)r->members.size();
  std::vector<int> act(r->active_host, r->active_host + n);
  SW_CUDA(nullptr, cudaStreamSynchronize(r->st));
  SW_TRY(build_runner(r, nullptr));
  for (int i = 0; i < n; ++i) r->active_host[i] = act[i];
  SW_CUDA(nullptr, ring_copy(r, const_cast<int*>(r->bh.bt.active), r->active_host, n));
  return SW_OK;
}

// The batch stream waits for work that members enqueued on their own streams.
void batch_enter(sw_batch* b) {
  for (sw_stream* m : b->run.members) {
    if (!m->own_pending) continue;
    if (!m->own_ev) cudaEventCreateWithFlags(&m->own_ev, cudaEventDisableTiming);
    cudaEventRecord(m->own_ev, m->st);
    cudaStreamWaitEvent(b->run.st, m->own_ev, 0);
    m->own_pending = false;
  }
}

// Members' own streams will wait for this batch call's work.
void batch_leave(sw_batch* b) {
  cudaEventRecord(b->done, b->run.st);
  for (sw_stream* m : b->run.members) m->batch_done = b->done;
}

}  // namespace

sw_status sw_batch_create(const sw_handle* streams, int n, void* cuda_stream, sw_batch_handle* out) {
  if (!out || !streams || n < 1 || n > 4096) return fail(nullptr, SW_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  std::vector<sw_stream*> mem(streams, streams + n);
  for (int i = 0; i < n; ++i) {
    if (!mem[i] || !mem[i]->has_model) return fail(nullptr, SW_ERR_INVALID_ARG, "batch member without a model");
    for (int j = 0; j < i; ++j)
      if (mem[j] == mem[i]) return fail(nullptr, SW_ERR_INVALID_ARG, "a stream appears twice in a batch");
  }
  sw_batch* b = new sw_batch();
  Runner* r = &b->run;
  if (cuda_stream) {
    r->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) == cudaSuccess) {
    r->own_stream = true;
  } else {
    delete b;
    return fail(nullptr, SW_ERR_CUDA, "cudaStreamCreate failed");
  }
  cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  r->members = mem;
  for (sw_stream* m : mem) {   // the members' pending work comes first
    if (!m->own_ev) cudaEventCreateWithFlags(&m->own_ev, cudaEventDisableTiming);
    cudaEventRecord(m->own_ev, m->st);
    cudaStreamWaitEvent(r->st, m->own_ev, 0);
    m->own_pending = false;
  }
  const sw_status e = build_runner(r, nullptr);
  if (e != SW_OK) {
    destroy_runner(r);
    cudaEventDestroy(b->done);
    delete b;
    return e;
  }
  *out = b;
  return SW_OK;
}

sw_status sw_batch_destroy(sw_batch_handle b) {
  if (!b) return fail(nullptr, SW_ERR_INVALID_ARG, "null batch");
  cudaStreamSynchronize(b->run.st);
  for (sw_stream* m : b->run.members)
    if (m->batch_done == b->done) m->batch_done = nullptr;
  destroy_runner(&b->run);
  cudaEventDestroy(b->done);
  delete b;
  return SW_OK;
}

sw_status sw_batch_set_active(sw_batch_handle b, const int* active) {
  SW_TRY(batch_check(b));
  if (!active) return fail(nullptr, SW_ERR_INVALID_ARG, "null active array");
  Runner* r = &b->run;
  const int n = (int)r->members.size();
  for (int i = 0; i < n; ++i) r->active_host[i] = active[i] ? 1 : 0;
  SW_CUDA(nullptr, ring_copy(r, const_cast<int*>(r->bh.bt.active), r->active_host, n));
  return SW_OK;
}

sw_status sw_batch_upload_depth(sw_batch_handle b, const float* const* depths, int on_device, const int* frame_ids) {
  SW_TRY(batch_check(b));
  if (!depths || !frame_ids) return fail(nullptr, SW_ERR_INVALID_ARG, "null argument");
  Runner* r = &b->run;
  const int n = (int)r->members.size();
  batch_enter(b);
  if (on_device) SW_CUDA(nullptr, cudaStreamSynchronize(0));
  for (int i = 0; i < n; ++i) {
    sw_stream* m = r->members[i];
    if (!r->active_host[i] || !depths[i]) continue;
    const size_t bytes = (size_t)m->h.W * m->h.H * sizeof(float);
    SW_CUDA(nullptr, cudaMemcpyAsync(m->h.depth, depths[i], bytes,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, r->st));
    m->has_depth = true;
    m->fused = false;
  }
  SW_CUDA(nullptr, ring_copy(r, r->frames_dev, frame_ids, n));
  k_set_frames<<<(n + 127) / 128, 128, 0, r->st>>>(r->bh.bt, r->frames_dev);
  std::vector<ProfEvent>* prof = nullptr;
  if (r->profiling) { reset_eager_prof(r); prof = &r->eager_prof; }
  prof_mark(r, prof, kProfDepth, true, false);
  launch_depth_maps(r->bh, r->st);
  prof_mark(r, prof, kProfDepth, false, false);
  SW_CUDA(nullptr, cudaGetLastError());
  batch_leave(b);
  return SW_OK;
}

sw_status sw_batch_solve(sw_batch_handle b, int gn_iters, int pcg_iters, sw_solve_stats* stats) {
  SW_TRY(batch_check(b));
  if (gn_iters < 1 || gn_iters > kMaxGn || pcg_iters < 1 || pcg_iters > kMaxPcg)
    return fail(nullptr, SW_ERR_INVALID_ARG, "iteration counts out of range");
  Runner* r = &b->run;
  for (int i = 0; i < (int)r->members.size(); ++i)
    if (r->active_host[i] && !r->members[i]->has_depth)
      return fail(nullptr, SW_ERR_NOT_INITIALIZED, "an active member has no depth frame");
  batch_enter(b);
  SW_TRY(runner_solve(r, nullptr, gn_iters, pcg_iters));
  batch_leave(b);
  if (!stats) return SW_OK;
  sw_status worst = SW_OK;
  for (int i = 0; i < (int)r->members.size(); ++i) {
    sw_stream* m = r->members[i];
    std::memset(&stats[i], 0, sizeof(sw_solve_stats));
    if (!r->active_host[i]) continue;
    int status = 0;
    stats[i].gn_iters = gn_iters;
    SW_CUDA(nullptr, cudaMemcpyAsync(&status, m->h.status, sizeof(int), cudaMemcpyDeviceToHost, r->st));
    SW_CUDA(nullptr, cudaMemcpyAsync(stats[i].e_depth, m->h.e_depth, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, r->st));
    SW_CUDA(nullptr, cudaMemcpyAsync(stats[i].e_reg, m->h.e_reg, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, r->st));
    SW_CUDA(nullptr, cudaMemcpyAsync(stats[i].n_corr, m->h.n_corr, kMaxGn * sizeof(int), cudaMemcpyDeviceToHost, r->st));
    SW_CUDA(nullptr, cudaMemcpyAsync(stats[i].pcg_rz, m->h.pcg_rz, kMaxGn * sizeof(double), cudaMemcpyDeviceToHost, r->st));
    SW_CUDA(nullptr, cudaStreamSynchronize(r->st));
    if (status & kStatusBounds) worst = SW_ERR_BOUNDS;
    else if ((status & (kStatusTimeout | kStatusDepthTimeout)) && worst != SW_ERR_BOUNDS) worst = SW_ERR_TIMEOUT;
    else if ((status & kStatusBreakdown) && worst == SW_OK) worst = SW_ERR_SOLVER_BREAKDOWN;
  }
  if (worst != SW_OK) return fail(nullptr, worst, "a member's solve broke down or timed out (see its stats)");
  return SW_OK;
}

sw_status sw_batch_fuse(sw_batch_handle b) {
  SW_TRY(batch_check(b));
  batch_enter(b);
  SW_TRY(runner_fuse(&b->run, nullptr));
  for (size_t i = 0; i < b->run.members.size(); ++i)
    if (b->run.active_host[i]) b->run.members[i]->fused = true;
  batch_leave(b);
  return SW_OK;
}

namespace sw {
sw_status batch_member_status(sw_batch_handle b, int* status) {
  if (!b || !status) return SW_ERR_INVALID_ARG;
  Runner* r = &b->run;
  const int n = (int)r->members.size();
  std::vector<int> raw(n, 0);
  for (int i = 0; i < n; ++i)
    if (r->active_host[i])
      SW_CUDA(nullptr, cudaMemcpyAsync(&raw[i], r->members[i]->h.status, sizeof(int), cudaMemcpyDeviceToHost, r->st));
  SW_CUDA(nullptr, cudaStreamSynchronize(r->st));
  for (int i = 0; i < n; ++i)
    status[i] = (raw[i] & kStatusBounds)                          ? SW_ERR_BOUNDS
                : (raw[i] & (kStatusTimeout | kStatusDepthTimeout)) ? SW_ERR_TIMEOUT
                : (raw[i] & kStatusBreakdown)                       ? SW_ERR_SOLVER_BREAKDOWN
                                                                     : SW_OK;
  return SW_OK;
}
}  // namespace sw

sw_status sw_rigid_align(sw_handle s, int iters, int* n_corr, double* energy) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (iters < 0 || iters > kMaxRigid) return fail(s, SW_ERR_INVALID_ARG, "iters out of range");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "needs a model and a depth frame");
  if (iters == 0) return SW_OK;
  enter(s);
  if (runner_stale(s->run)) SW_TRY(build_runner(s->run, s));
  launch_rigid_align(s->run->bh, iters, s->st);
  SW_CUDA(s, cudaGetLastError());
  if (n_corr || energy) {
    std::vector<double> st(2 * iters);
    SW_CUDA(s, cudaMemcpyAsync(st.data(), s->h.rigid_stats, st.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    SW_CUDA(s, cudaStreamSynchronize(s->st));
    for (int k = 0; k < iters; ++k) {
      if (n_corr) n_corr[k] = (int)st[2 * k];
      if (energy) energy[k] = st[2 * k + 1];
    }
  }
  return bounds_check(s);
}

sw_status sw_batch_rigid_align(sw_batch_handle b, int iters) {
  SW_TRY(batch_check(b));
  if (iters < 0 || iters > kMaxRigid) return fail(nullptr, SW_ERR_INVALID_ARG, "iters out of range");
  Runner* r = &b->run;
  for (int i = 0; i < (int)r->members.size(); ++i)
    if (r->active_host[i] && !r->members[i]->has_depth)
      return fail(nullptr, SW_ERR_NOT_INITIALIZED, "an active member has no depth frame");
  if (iters == 0) return SW_OK;
  batch_enter(b);
  launch_rigid_align(r->bh, iters, r->st);
  SW_CUDA(nullptr, cudaGetLastError());
  batch_leave(b);
  return SW_OK;
}

sw_status sw_autotune(sw_handle s, int pcg_iters, int* rows_per_cta, double* pcg_us) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  if (pcg_iters < 1 || pcg_iters > kMaxPcg) return fail(s, SW_ERR_INVALID_ARG, "pcg_iters out of range");
  if (!s->has_model || !s->has_depth) return fail(s, SW_ERR_NOT_INITIALIZED, "needs a model and a depth frame");
  enter(s);
  return runner_autotune(s->run, s, pcg_iters, rows_per_cta, pcg_us);
}

sw_status sw_batch_autotune(sw_batch_handle b, int pcg_iters, int* rows_per_cta, double* pcg_us) {
  SW_TRY(batch_check(b));
  if (pcg_iters < 1 || pcg_iters > kMaxPcg) return fail(nullptr, SW_ERR_INVALID_ARG, "pcg_iters out of range");
  batch_enter(b);
  const sw_status st = runner_autotune(&b->run, nullptr, pcg_iters, rows_per_cta, pcg_us);
  batch_leave(b);
  return st;
}

sw_status sw_set_profiling(sw_handle s, int enable) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  SW_CUDA(s, cudaStreamSynchronize(s->st));
  s->run->profiling = enable != 0;
  drop_graphs(s->run);
  reset_eager_prof(s->run);
  return SW_OK;
}

sw_status sw_read_profile(sw_handle s, double* ms, int* launches) {
  if (!s) return fail(nullptr, SW_ERR_INVALID_ARG, "null handle");
  return runner_profile(s->run, s, ms, launches);
}

sw_status sw_batch_set_profiling(sw_batch_handle b, int enable) {
  if (!b) return fail(nullptr, SW_ERR_INVALID_ARG, "null batch");
  SW_CUDA(nullptr, cudaStreamSynchronize(b->run.st));
  b->run.profiling = enable != 0;
  drop_graphs(&b->run);
  reset_eager_prof(&b->run);
  return SW_OK;
}

sw_status sw_batch_read_profile(sw_batch_handle b, double* ms, int* launches) {
  if (!b) return fail(nullptr, SW_ERR_INVALID_ARG, "null batch");
  return runner_profile(&b->run, nullptr, ms, launches);
}

sw_status sw_debug_block_inverse(const void* blocks36, int n, int mode, void* inv21, int* ok) {
  if (n < 0 || n > (1 << 24)) return fail(nullptr, SW_ERR_INVALID_ARG, "n out of range");
  if (n > 0 && (!blocks36 || !inv21 || !ok)) return fail(nullptr, SW_ERR_INVALID_ARG, "null array");
  if (n == 0) return SW_OK;
  if (mode < 0 || mode > 2) return fail(nullptr, SW_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
  const size_t es = mode == 1 ? sizeof(double) : sizeof(float);
  void *db = nullptr, *dout = nullptr;
  int* dok = nullptr;
  cudaError_t e = cudaMalloc(&db, (size_t)n * 36 * es);
  if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * 21 * es);
  if (e == cudaSuccess) e = cudaMalloc(&dok, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(db, blocks36, (size_t)n * 36 * es, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_debug_block_inverse(db, n, mode, dout, dok, 0);
  if (e == cudaSuccess) e = cudaMemcpy(inv21, dout, (size_t)n * 21 * es, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ok, dok, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(db);
  cudaFree(dout);
  cudaFree(dok);
  if (e != cudaSuccess) return fail(nullptr, SW_ERR_CUDA, std::string("block inverse: ") + cudaGetErrorString(e));
  return SW_OK;
}

sw_status sw_debug_scan(const int32_t* in, int n, int inclusive, int32_t* out) {
  if (n < 0 || n > (1 << 28)) return fail(nullptr, SW_ERR_INVALID_ARG, "n out of range");
  if (n > 0 && (!in || !out)) return fail(nullptr, SW_ERR_INVALID_ARG, "null array");
  if (n == 0) return SW_OK;
  const size_t tb = scan_scratch_bytes(n);
  int *din = nullptr, *dout = nullptr;
  void* dtmp = nullptr;
  cudaError_t e = cudaMalloc(&din, (size_t)n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dtmp, tb);
  if (e == cudaSuccess) e = cudaMemcpy(din, in, (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = scan_sum(din, dout, n, inclusive != 0, dtmp, tb, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n * 4, cudaMemcpyDeviceToHost);
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dtmp);
  if (e != cudaSuccess) return fail(nullptr, SW_ERR_CUDA, std::string("scan: ") + cudaGetErrorString(e));
  return SW_OK;
}

sw_status sw_debug_radix_sort(int key_bytes, const void* keys, const int32_t* vals, int n, int begin_bit,
                              int end_bit, void* keys_out, int32_t* vals_out) {
  if (key_bytes != 4 && key_bytes != 8) return fail(nullptr, SW_ERR_INVALID_ARG, "key_bytes must be 4 or 8");
  if (n < 0 || n > (1 << 28)) return fail(nullptr, SW_ERR_INVALID_ARG, "n out of range");
  if (begin_bit < 0 || begin_bit > end_bit || end_bit > 8 * key_bytes)
    return fail(nullptr, SW_ERR_INVALID_ARG, "bit range out of range");
  if (n > 0 && (!keys || !keys_out || (vals && !vals_out))) return fail(nullptr, SW_ERR_INVALID_ARG, "null array");
  if (n == 0) return SW_OK;
  const bool wv = vals != nullptr;
  const size_t kb = (size_t)n * key_bytes, vb = (size_t)n * 4;
  const size_t tb = key_bytes == 4 ? sort_scratch_bytes_u32(n, wv) : sort_scratch_bytes_u64(n, wv);
  void *dk = nullptr, *dk2 = nullptr, *dtmp = nullptr;
  int *dv = nullptr, *dv2 = nullptr;
  cudaError_t e = cudaMalloc(&dk, kb);
  if (e == cudaSuccess) e = cudaMalloc(&dk2, kb);
  if (e == cudaSuccess) e = cudaMalloc(&dtmp, tb);
  if (e == cudaSuccess && wv) e = cudaMalloc(&dv, vb);
  if (e == cudaSuccess && wv) e = cudaMalloc(&dv2, vb);
  if (e == cudaSuccess) e = cudaMemcpy(dk, keys, kb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && wv) e = cudaMemcpy(dv, vals, vb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = key_bytes == 4 ? radix_sort_u32(static_cast<const uint32_t*>(dk), static_cast<uint32_t*>(dk2), dv, dv2, n,
                                        begin_bit, end_bit, dtmp, tb, 0)
                       : radix_sort_u64(static_cast<const unsigned long long*>(dk),
                                        static_cast<unsigned long long*>(dk2), dv, dv2, n, begin_bit, end_bit, dtmp,
                                        tb, 0);
  if (e == cudaSuccess) e = cudaMemcpy(keys_out, dk2, kb, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && wv) e = cudaMemcpy(vals_out, dv2, vb, cudaMemcpyDeviceToHost);
  cudaFree(dk);
  cudaFree(dk2);
  cudaFree(dtmp);
  cudaFree(dv);
  cudaFree(dv2);
  if (e != cudaSuccess) return fail(nullptr, SW_ERR_CUDA, std::string("radix sort: ") + cudaGetErrorString(e));
  return SW_OK;
}

sw_status sw_debug_set_pcg_mode(int max_mode) {
  if (max_mode < 0 || max_mode > 3) return fail(nullptr, SW_ERR_INVALID_ARG, "max_mode must be 0, 1, 2 or 3");
  g_pcg_mode_cap.store(max_mode);
  return SW_OK;
}

sw_status sw_debug_pcg_mode(sw_handle s, int* mode) {
  if (!s || !mode) return fail(s, SW_ERR_INVALID_ARG, "null argument");
  if (!s->has_model || !s->run) return fail(s, SW_ERR_NOT_INITIALIZED, "no model");
  *mode = s->run->bh.n_cluster ? 3 : s->run->bh.pcg_mode;
  return SW_OK;
}

sw_status sw_batch_debug_pcg_mode(sw_batch_handle b, int* mode) {
  SW_TRY(batch_check(b));
  if (!mode) return fail(nullptr, SW_ERR_INVALID_ARG, "null argument");
  *mode = b->run.bh.n_cluster == (int)b->run.members.size() ? 3 : b->run.bh.pcg_mode;
  return SW_OK;
}

sw_status sw_read_visibility(sw_handle s, int* visible, int cap, int* n_out) {
  SW_TRY(need_model(s, cap));
  if (n_out) *n_out = s->h.n_s;
  if (visible) SW_TRY(d2h_perm(s, s->h.visible, visible, 1, true));
  return SW_OK;
}

sw_status sw_debug_inject_wait_fault(int kind, int spin_limit) {
  if (kind < kFaultNone || kind > kFaultDepthTma) return fail(nullptr, SW_ERR_INVALID_ARG, "unknown fault kind");
  if (spin_limit < 0 || spin_limit > (1 << 22)) return fail(nullptr, SW_ERR_INVALID_ARG, "spin_limit out of range");
  SW_CUDA(nullptr, cudaDeviceSynchronize());   // no launch in flight sees a half-written setting
  set_pcg_wait_fault(kind == kFaultPcgPartial || kind == kFaultPcgVector ? kind : kFaultNone, spin_limit);
  set_depth_wait_fault(kind == kFaultDepthTma ? kind : kFaultNone);
  SW_CUDA(nullptr, cudaDeviceSynchronize());
  SW_CUDA(nullptr, cudaGetLastError());
  return SW_OK;
}

sw_status sw_debug_cluster_plan(int ctas, int n_nodes, const int* row_ptr, const int* col, const float* node4,
                                size_t smem_limit, int* plan, size_t cap, size_t* n_out, size_t* smem_out) {
  if (ctas < 1 || ctas > 16 || n_nodes < 1 || !row_ptr || !col || !node4)
    return fail(nullptr, SW_ERR_INVALID_ARG, "bad cluster-plan arguments");
  const int nnzb = row_ptr[n_nodes];
  if (nnzb < n_nodes) return fail(nullptr, SW_ERR_INVALID_ARG, "row_ptr does not describe a pattern");
  std::vector<int> rp(row_ptr, row_ptr + n_nodes + 1), cl(col, col + nnzb);
  for (int i = 0; i < n_nodes; ++i) {
    if (rp[i + 1] <= rp[i] || cl[rp[i]] != i) return fail(nullptr, SW_ERR_INVALID_ARG, "a row does not lead with its diagonal block");
    for (int b = rp[i]; b < rp[i + 1]; ++b)
      if (cl[b] < i || cl[b] >= n_nodes) return fail(nullptr, SW_ERR_INVALID_ARG, "a block outside the upper triangle");
  }
  std::vector<float> nd(node4, node4 + (size_t)n_nodes * 4);
  std::vector<int> out;
  size_t smem = 0;
  if (!build_cluster_plan(ctas, n_nodes, rp, cl, nd, smem_limit, out, &smem))
    return fail(nullptr, SW_ERR_INVALID_ARG, "the system does not fit the cluster's shared memory");
  if (n_out) *n_out = out.size();
  if (smem_out) *smem_out = smem;
  if (plan) {
    if (cap < out.size()) return fail(nullptr, SW_ERR_INVALID_ARG, "plan capacity too small");
    std::memcpy(plan, out.data(), out.size() * sizeof(int));
  }
  return SW_OK;
}

sw_status sw_debug_pcg_cluster(sw_handle s, int precision, int ctas, size_t smem, int* plan_ctas,
                               size_t* plan_smem, int* active_clusters) {
  if (active_clusters) {
    if (ctas < 1 || ctas > 16) return fail(s, SW_ERR_INVALID_ARG, "ctas out of range");
    *active_clusters = cluster_pcg_active(precision, ctas, smem);
  }
  if (s) {
    if (plan_ctas) *plan_ctas = s->cplan_ctas;
    if (plan_smem) *plan_smem = s->cplan_smem;
  }
  return SW_OK;
}

sw_status sw_debug_cluster_barrier_us(int ctas, double* us) {
  if (ctas < 1 || ctas > 16 || !us) return fail(nullptr, SW_ERR_INVALID_ARG, "ctas out of range or null output");
  SW_CUDA(nullptr, cluster_barrier_cost(ctas, us));
  return SW_OK;
}
