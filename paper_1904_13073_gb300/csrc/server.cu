// Serving runtime: a request loop over many independent streams with
// continuous batching (no counterpart in the paper, which processes one
// camera stream).
//
// Clients open streams (model + parameters) and submit depth frames as they
// arrive; one worker thread owns the GPU.  Each step it
//   * admits waiting streams whose device state fits the memory budget
//     (creating them and loading their models), and releases closed streams
//     once their queued frames are done;
//   * takes the oldest queued frame of every admitted stream that has one
//     and runs depth processing, the Gauss-Newton solve and fusion for all
//     of them together through one batch (one set of launches, the persistent
//     PCG shared), the other streams masked inactive;
//   * stamps every frame with its submit, start and completion times.
// Frames that arrive while a step is on the GPU join the next step, so the
// batch follows the load from step to step; the batch object is rebuilt
// only when streams join or leave.  An optional batching window lets a step
// wait, up to that long after its oldest frame arrived, for frames of the
// other admitted streams.  Every stream's surfels, node graph and
// warp field stay resident on the device between its frames.
//
// A batch step costs about the same whatever share of its members is active:
// the persistent PCG's CTAs are divided among all members when the batch is
// built, so a step is as long as its largest active member's PCG on its
// share.  Under light load that is slower than running the few queued frames
// one after another through their streams' own calls (each with the whole
// GPU).  The adaptive policy (sw_server_set_adaptive, on by default) takes,
// every step, the cheaper of the two by measured times: an average of the
// batch's step time per size class of the step (reset when the membership
// changes) against the sum of the queued streams' own frame times (a
// per-stream average; a stream not yet measured counts at the average of the
// measured ones, and while none is measured a step of one or two frames runs
// alone, which measures them).  A step that runs alone serves only the oldest
// queued frame, as the plain mode does, and the next step decides again; the
// batch is first tried only on a long queue (kExploreBatch frames).
//
// In the plain mode (sw_server_set_plain) each step instead takes the single
// oldest queued frame and runs it through its stream's own calls, one stream
// at a time: the reference that continuous batching is measured against.
//
// Each stream queues up to `queue_depth` frames in pinned host slots that the
// submit call fills; a full queue refuses further frames (SW_ERR_NO_MEMORY)
// until the worker drains it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sw_internal.h"

namespace {

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Frame {
  int frame_id;
  int slot;
  double submit_ms;
};

struct SrvStream {
  int id = 0;
  sw_params p{};
  std::vector<float> v4, n4, node4;
  std::vector<int> t2;
  int n_s = 0, n_n = 0;       // surfels (current, after appending) and nodes at opening
  sw_handle h = nullptr;      // null while waiting for admission
  bool closing = false;
  std::deque<Frame> queue;
  std::vector<float*> slots;  // pinned depth buffers
  std::vector<int> free_slots;
  int in_submit = 0;          // submit calls copying into a slot right now
  long long frames_done = 0;
};

}  // namespace

struct sw_server {
  std::mutex mu;                 // queues, stream table, results
  std::mutex gpu;                // the device state of the streams (worker steps, read-back)
  std::condition_variable cv;    // work arrived / work finished
  std::thread worker;
  bool stop = false;
  int device = 0;
  int gn = 10, pcg = 20, qdepth = 4;
  double window_ms = 0.0;        // how long a step may wait for more streams' frames
  bool appending = false;        // sw_append_frame after every served frame
  bool plain = false;            // one frame per step through its stream's own calls (no batching)
  bool adaptive = true;          // per step, the batch or the oldest frame alone, by measured times
  // measured costs for the adaptive policy (worker thread only), in ms
  static constexpr int kSizeClasses = 8;   // step sizes 1, 2, 3-4, 5-8, ..., 65+
  double tb[kSizeClasses] = {};  // batch step time by size class (0: not measured)
  std::map<int, double> tp;      // per stream: its frame through its own calls
  double tp_sum = 0.0;           // sum and count of the per-stream averages
  int tp_count = 0;
  std::chrono::steady_clock::time_point t0;
  int next_id = 1;
  std::map<int, SrvStream*> streams;    // every open stream, by id
  std::vector<int> order;               // admission order of the admitted streams
  std::vector<int> batch_ids;           // members of the current batch, in order
  sw_batch_handle batch = nullptr;
  bool composition_changed = false;
  std::vector<sw_frame_result> results;
  long long submitted = 0, completed = 0;
  sw_server_stats st{};
  std::string err;
};

namespace {

int size_class(int k) {
  int c = 0;
  while (c + 1 < sw_server::kSizeClasses && (1 << c) < k) ++c;
  return c;
}

double ema(double old, double x) { return old > 0.0 ? 0.7 * old + 0.3 * x : x; }

// The adaptive policy's choice for a step of these streams' frames: true
// when serving them one by one through their own calls takes less time than
// one batch step.  Until the batch has been measured, a step batches only
// from kExploreBatch queued frames on: a batch step lasts about as long as
// the batch's largest member's solve whatever the share of active members,
// so trying it on a short queue costs every frame in it that time.
constexpr int kExploreBatch = 16;
bool cheaper_alone(const sw_server* S, const std::vector<int>& ids) {
  const int k = (int)ids.size();
  double alone = 0.0;
  bool all_known = true;
  const double prior = S->tp_count ? S->tp_sum / S->tp_count : 0.0;
  for (int id : ids) {
    auto it = S->tp.find(id);
    if (it != S->tp.end()) alone += it->second;
    else { all_known = false; alone += prior; }
  }
  if (!all_known && S->tp_count == 0) return k <= 2;   // nothing measured alone yet
  // the batch's time at this size, else at the nearest measured size
  const int c = size_class(k);
  double batch = 0.0;
  for (int d = 0; d < sw_server::kSizeClasses && batch == 0.0; ++d) {
    if (c - d >= 0 && S->tb[c - d] > 0.0) batch = S->tb[c - d];
    else if (c + d < sw_server::kSizeClasses && S->tb[c + d] > 0.0) batch = S->tb[c + d];
  }
  if (batch == 0.0) return k < kExploreBatch;   // the batch not measured yet
  return alone < batch;
}

void release_stream(SrvStream* s) {
  if (s->h) sw_destroy_stream(s->h);
  s->h = nullptr;
  for (float* p : s->slots) cudaFreeHost(p);
  s->slots.clear();
}

// Release closed streams whose queues are empty (and that no submit call is
// filling).  Called by the worker with `mu` and `gpu` held.
void release_closed(sw_server* S) {
  std::vector<int> gone;
  for (auto& kv : S->streams) {
    SrvStream* s = kv.second;
    if (s->closing && s->queue.empty() && s->in_submit == 0) gone.push_back(kv.first);
  }
  if (!gone.empty() && S->batch) {   // the batch refers to its members: it goes first
    sw_batch_destroy(S->batch);
    S->batch = nullptr;
  }
  for (int id : gone) {
    SrvStream* s = S->streams[id];
    auto t = S->tp.find(id);
    if (t != S->tp.end()) {
      S->tp_sum -= t->second;
      S->tp_count--;
      S->tp.erase(t);
    }
    if (s->h) S->composition_changed = true;
    release_stream(s);
    S->order.erase(std::remove(S->order.begin(), S->order.end(), id), S->order.end());
    S->streams.erase(id);
    delete s;
  }
}

// Try to admit one waiting stream: its device state under the memory budget,
// its model, its pinned depth slots.  Runs under `gpu` only; false if it
// does not fit yet.
bool admit(sw_server* S, SrvStream* s) {
  sw_handle h = nullptr;
  if (sw_create_stream(&s->p, nullptr, &h) != SW_OK) return false;
  if (sw_set_model(h, s->v4.data(), s->n4.data(), s->t2.data(), s->n_s, s->node4.data(), s->n_n) != SW_OK) {
    sw_destroy_stream(h);
    return false;
  }
  const size_t bytes = (size_t)s->p.width * s->p.height * sizeof(float);
  std::vector<float*> slots;
  for (int k = 0; k < S->qdepth; ++k) {
    float* buf = nullptr;
    if (cudaMallocHost(&buf, bytes) != cudaSuccess) {
      for (float* q : slots) cudaFreeHost(q);
      sw_destroy_stream(h);
      return false;
    }
    slots.push_back(buf);
  }
  s->slots = slots;
  s->h = h;
  return true;
}

void worker_main(sw_server* S) {
  cudaSetDevice(S->device);
  std::vector<const float*> depths;
  std::vector<int> frame_ids, active;
  for (;;) {
    std::vector<int> members;
    std::vector<SrvStream*> member_ptrs, taken_ptrs;   // only this thread deletes streams
    std::vector<Frame> taken;
    std::vector<int> taken_ids;
    {
      std::vector<SrvStream*> waiting;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) break;
        for (auto& kv : S->streams)
          if (!kv.second->h && !kv.second->closing) waiting.push_back(kv.second);
      }
      // admissions outside the queue lock (model loading takes a while);
      // a waiting stream is only ever removed by this thread
      std::vector<SrvStream*> admitted;
      if (!waiting.empty()) {
        std::lock_guard<std::mutex> g(S->gpu);
        for (SrvStream* s : waiting)
          if (admit(S, s)) admitted.push_back(s);
      }
      std::unique_lock<std::mutex> lk(S->mu);
      for (SrvStream* s : admitted) {
        s->free_slots.clear();
        for (int k = 0; k < S->qdepth; ++k) s->free_slots.push_back(k);
        std::vector<float>().swap(s->v4);   // the model now lives on the device
        std::vector<float>().swap(s->n4);
        std::vector<float>().swap(s->node4);
        std::vector<int>().swap(s->t2);
        S->order.push_back(s->id);
        S->composition_changed = true;
      }
      {
        std::lock_guard<std::mutex> g(S->gpu);
        release_closed(S);
      }
      for (int id : S->order) {
        SrvStream* s = S->streams[id];
        member_ptrs.push_back(s);
        if (!s->queue.empty()) {
          taken.push_back(s->queue.front());
          taken_ids.push_back(id);
          taken_ptrs.push_back(s);
        }
      }
      S->st.admitted = (int)S->order.size();
      S->st.waiting = (int)S->streams.size() - (int)S->order.size();
      if (taken.empty()) {
        S->cv.wait_for(lk, std::chrono::milliseconds(1));
        continue;
      }
      if (S->plain && taken.size() > 1) {   // one frame at a time: the oldest queued one
        size_t best = 0;
        for (size_t k = 1; k < taken.size(); ++k)
          if (taken[k].submit_ms < taken[best].submit_ms) best = k;
        taken = {taken[best]};
        taken_ids = {taken_ids[best]};
        taken_ptrs = {taken_ptrs[best]};
      }
      if (!S->plain && S->window_ms > 0.0 && taken.size() < S->order.size()) {   // batching window
        double oldest = taken[0].submit_ms;
        for (const Frame& f : taken) oldest = std::min(oldest, f.submit_ms);
        const double left = oldest + S->window_ms - now_ms(S->t0);
        if (left > 0.0) {
          S->cv.wait_for(lk, std::chrono::microseconds((long long)(left * 1000.0) + 1));
          continue;
        }
      }
      members = S->order;
    }
    std::lock_guard<std::mutex> g(S->gpu);
    // alone, the frames run oldest first
    std::vector<size_t> by_age(taken.size());
    for (size_t k = 0; k < taken.size(); ++k) by_age[k] = k;
    std::sort(by_age.begin(), by_age.end(),
              [&](size_t a, size_t b) { return taken[a].submit_ms < taken[b].submit_ms; });
    bool alone = S->plain;
    if (!alone && S->adaptive) {
      alone = cheaper_alone(S, taken_ids);
      if (alone && taken.size() > 1) {   // the oldest frame now; the others are decided again next step
        const size_t o = by_age[0];
        taken = {taken[o]};
        taken_ids = {taken_ids[o]};
        taken_ptrs = {taken_ptrs[o]};
        by_age = {0};
      }
    }
    sw_status status = SW_OK;
    std::vector<sw_status> fstat(taken.size(), SW_OK);   // per taken frame
    std::vector<sw_append_stats> app(taken.size());
    std::vector<sw_status> app_status(taken.size(), SW_OK);
    std::vector<double> f_start(taken.size(), 0.0), f_done(taken.size(), 0.0);
    if (alone) {
      // each frame's stream alone, through its own calls, oldest frame first
      for (size_t k : by_age) {
        SrvStream* s = taken_ptrs[k];
        f_start[k] = now_ms(S->t0);
        sw_status st = sw_upload_depth(s->h, s->slots[taken[k].slot], 0, taken[k].frame_id);
        if (st == SW_OK) st = sw_solve_frame(s->h, S->gn, S->pcg, nullptr);
        if (st == SW_OK) st = sw_fuse_frame(s->h);
        int nn = 0;
        if (st == SW_OK) st = sw_read_nodes(s->h, nullptr, nullptr, 0, &nn);   // waits; reports a breakdown
        fstat[k] = st;
        const double t_fused = now_ms(S->t0);
        if (S->appending && st == SW_OK) app_status[k] = sw_append_frame(s->h, &app[k]);
        f_done[k] = now_ms(S->t0);
        if (st == SW_OK) {   // the stream's own frame time (appending apart: both paths append alike)
          double& t = S->tp[taken_ids[k]];
          const double old = t;
          t = ema(t, t_fused - f_start[k]);
          S->tp_sum += t - old;
          if (old == 0.0) S->tp_count++;
        }
      }
    } else {
    if (S->composition_changed || !S->batch) {
      if (S->batch) sw_batch_destroy(S->batch);
      S->batch = nullptr;
      std::vector<sw_handle> hs;
      for (SrvStream* m : member_ptrs) hs.push_back(m->h);
      status = sw_batch_create(hs.data(), (int)hs.size(), nullptr, &S->batch);
      S->batch_ids = members;
      S->composition_changed = false;
      for (double& t : S->tb) t = 0.0;   // a new batch: its step times are measured again
    }
    const int n = (int)S->batch_ids.size();
    depths.assign(n, nullptr);
    frame_ids.assign(n, 0);
    active.assign(n, 0);
    for (size_t k = 0; k < taken.size(); ++k) {
      const int pos = (int)(std::find(S->batch_ids.begin(), S->batch_ids.end(), taken_ids[k]) - S->batch_ids.begin());
      SrvStream* s = taken_ptrs[k];
      depths[pos] = s->slots[taken[k].slot];
      frame_ids[pos] = taken[k].frame_id;
      active[pos] = 1;
    }
    const double t_start = now_ms(S->t0);
    if (status == SW_OK) status = sw_batch_set_active(S->batch, active.data());
    if (status == SW_OK) status = sw_batch_upload_depth(S->batch, depths.data(), 0, frame_ids.data());
    if (status == SW_OK) status = sw_batch_solve(S->batch, S->gn, S->pcg, nullptr);
    if (status == SW_OK) status = sw_batch_fuse(S->batch);
    std::vector<int> member_status(n, 0);
    const sw_status sync = S->batch ? sw::batch_member_status(S->batch, member_status.data()) : status;
    const double t_fused = now_ms(S->t0);
    if (status == SW_OK && sync == SW_OK) {
      double& t = S->tb[size_class((int)taken.size())];
      t = ema(t, t_fused - t_start);
    }
    for (size_t k = 0; k < taken.size(); ++k) {
      const int pos = (int)(std::find(S->batch_ids.begin(), S->batch_ids.end(), taken_ids[k]) - S->batch_ids.begin());
      fstat[k] = status != SW_OK ? status : sync != SW_OK ? sync : (sw_status)member_status[pos];
    }
    if (S->appending && status == SW_OK && sync == SW_OK)
      for (size_t k = 0; k < taken.size(); ++k)
        if (fstat[k] == SW_OK) app_status[k] = sw_append_frame(taken_ptrs[k]->h, &app[k]);
    const double t_done = now_ms(S->t0);
    for (size_t k = 0; k < taken.size(); ++k) {
      f_start[k] = t_start;
      f_done[k] = t_done;
    }
    }
    double busy = 0.0;
    for (size_t k = 0; k < taken.size(); ++k)
      if (alone || k == 0) busy += f_done[k] - f_start[k];
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (size_t k = 0; k < taken.size(); ++k) {
        SrvStream* s = S->streams[taken_ids[k]];
        s->queue.pop_front();
        s->free_slots.push_back(taken[k].slot);
        s->frames_done++;
        sw_frame_result r{};
        r.stream = taken_ids[k];
        r.frame_id = taken[k].frame_id;
        r.status = fstat[k] != SW_OK ? fstat[k] : app_status[k];
        if (S->appending && app_status[k] == SW_OK && r.status == SW_OK) s->n_s = app[k].n_surfels;
        r.appended = S->appending && r.status == SW_OK ? app[k].appended : 0;
        r.n_surfels = s->n_s;
        r.submit_ms = taken[k].submit_ms;
        r.start_ms = f_start[k];
        r.done_ms = f_done[k];
        r.batch_size = alone ? 1 : (int)taken.size();
        S->results.push_back(r);
      }
      S->completed += (long long)taken.size();
      S->st.steps++;
      S->st.frames += (long long)taken.size();
      S->st.busy_ms += busy;
      if (alone && !S->plain) S->st.steps_alone++;
      S->st.memory_in_use = sw_memory_in_use();
    }
    S->cv.notify_all();
  }
}

}  // namespace

sw_status sw_server_create(size_t memory_budget, int gn_iters, int pcg_iters, int queue_depth, sw_server_handle* out) {
  if (!out) return SW_ERR_INVALID_ARG;
  *out = nullptr;
  if (gn_iters < 1 || gn_iters > SW_MAX_GN_ITERS || pcg_iters < 1 || pcg_iters > SW_MAX_PCG_ITERS || queue_depth < 1 ||
      queue_depth > 64)
    return SW_ERR_INVALID_ARG;
  sw_server* S = new sw_server();
  S->gn = gn_iters;
  S->pcg = pcg_iters;
  S->qdepth = queue_depth;
  S->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&S->device);
  sw_set_memory_budget(memory_budget);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return SW_OK;
}

sw_status sw_server_destroy(sw_server_handle S) {
  if (!S) return SW_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->batch) sw_batch_destroy(S->batch);
  for (auto& kv : S->streams) {
    release_stream(kv.second);
    delete kv.second;
  }
  delete S;
  return SW_OK;
}

sw_status sw_server_open(sw_server_handle S, const sw_params* p, const float* v4, const float* n4, const int* t2,
                         int n_s, const float* node4, int n_n, int* stream_id) {
  if (!S || !p || !v4 || !n4 || !node4 || !stream_id || n_s < 1 || n_n < 1) return SW_ERR_INVALID_ARG;
  if (n_s > p->max_surfels || n_n > p->max_nodes) return SW_ERR_INVALID_ARG;
  SrvStream* s = new SrvStream();
  s->p = *p;
  s->v4.assign(v4, v4 + (size_t)n_s * 4);
  s->n4.assign(n4, n4 + (size_t)n_s * 4);
  if (t2) s->t2.assign(t2, t2 + (size_t)n_s * 2);
  else s->t2.assign((size_t)n_s * 2, 0);
  s->node4.assign(node4, node4 + (size_t)n_n * 4);
  s->n_s = n_s;
  s->n_n = n_n;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    s->id = S->next_id++;
    S->streams[s->id] = s;
    *stream_id = s->id;
  }
  S->cv.notify_all();
  return SW_OK;
}

sw_status sw_server_close(sw_server_handle S, int stream_id) {
  if (!S) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->streams.find(stream_id);
  if (it == S->streams.end()) return SW_ERR_INVALID_ARG;
  it->second->closing = true;   // the worker releases it once its queued frames are done
  S->cv.notify_all();
  return SW_OK;
}

sw_status sw_server_submit(sw_server_handle S, int stream_id, const float* depth, int frame_id) {
  if (!S || !depth) return SW_ERR_INVALID_ARG;
  float* dst = nullptr;
  size_t bytes = 0;
  int slot = -1;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end() || it->second->closing) return SW_ERR_INVALID_ARG;
    SrvStream* s = it->second;
    if (!s->h) return SW_ERR_NOT_INITIALIZED;   // not admitted yet
    if (s->free_slots.empty()) return SW_ERR_NO_MEMORY;   // queue full
    slot = s->free_slots.back();
    s->free_slots.pop_back();
    dst = s->slots[slot];
    bytes = (size_t)s->p.width * s->p.height * sizeof(float);
    s->in_submit++;   // keeps the stream and its slots alive during the copy
  }
  std::memcpy(dst, depth, bytes);   // the slot is ours until the frame completes
  {
    std::lock_guard<std::mutex> lk(S->mu);
    SrvStream* s = S->streams[stream_id];
    s->in_submit--;
    s->queue.push_back(Frame{frame_id, slot, now_ms(S->t0)});
    S->submitted++;
  }
  S->cv.notify_all();
  return SW_OK;
}

sw_status sw_server_poll(sw_server_handle S, sw_frame_result* out, int cap, int* n_out) {
  if (!S || !n_out || (cap > 0 && !out)) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const int n = std::min(cap, (int)S->results.size());
  for (int k = 0; k < n; ++k) out[k] = S->results[k];
  S->results.erase(S->results.begin(), S->results.begin() + n);
  *n_out = n;
  return SW_OK;
}

sw_status sw_server_wait(sw_server_handle S, int timeout_ms) {
  if (!S) return SW_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  const bool done = S->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                   [&] { return S->completed >= S->submitted; });
  return done ? SW_OK : SW_ERR_TIMEOUT;
}

sw_status sw_server_is_admitted(sw_server_handle S, int stream_id, int* admitted) {
  if (!S || !admitted) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->streams.find(stream_id);
  if (it == S->streams.end()) return SW_ERR_INVALID_ARG;
  *admitted = it->second->h != nullptr;
  return SW_OK;
}

sw_status sw_server_read_nodes(sw_server_handle S, int stream_id, float* pos4, float* dq8, int cap, int* n_out) {
  if (!S) return SW_ERR_INVALID_ARG;
  sw_handle h = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->streams.find(stream_id);
    if (it == S->streams.end()) return SW_ERR_INVALID_ARG;
    h = it->second->h;
  }
  if (!h) return SW_ERR_NOT_INITIALIZED;
  std::lock_guard<std::mutex> g(S->gpu);
  return sw_read_nodes(h, pos4, dq8, cap, n_out);
}

sw_status sw_server_set_batch_window(sw_server_handle S, double window_ms) {
  if (!S || !(window_ms >= 0.0) || window_ms > 1000.0) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->window_ms = window_ms;
  return SW_OK;
}

sw_status sw_server_set_appending(sw_server_handle S, int enable) {
  if (!S || (enable != 0 && enable != 1)) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->appending = enable != 0;
  return SW_OK;
}

sw_status sw_server_read_stats(sw_server_handle S, sw_server_stats* out) {
  if (!S || !out) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->memory_in_use = sw_memory_in_use();
  return SW_OK;
}

sw_status sw_server_set_adaptive(sw_server_handle S, int enable) {
  if (!S || (enable != 0 && enable != 1)) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->adaptive = enable != 0;
  return SW_OK;
}

sw_status sw_server_set_plain(sw_server_handle S, int enable) {
  if (!S || (enable != 0 && enable != 1)) return SW_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->plain = enable != 0;
  return SW_OK;
}
