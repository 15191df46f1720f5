// server.cu -- continuous-batching request server (stark_server_*).
//
// Requests (C = A*B on device pointers, any n) are queued by stark_submit
// and served by one dispatcher thread:
//   * admission in arrival order: the head request is admitted when a
//     workspace for its (n_pad, depth, dtype) bucket is idle in the cache, or
//     a new one fits the device-memory budget (idle workspaces of other
//     buckets are evicted, least recently used first, to make room);
//   * a bucket whose breadth-first workspace (all 7^d leaves' operands) is
//     larger than the whole budget gets a depth-first one instead: the
//     operands of one subtree below the top 1 or 2 recursion levels, 1/7 or
//     1/49 of the bytes (the fewest levels that fit); its requests run alone,
//     subtree after subtree, instead of in the grouped launch.  When no
//     traversal fits at the chosen depth, the fitting depth that the cost
//     model ranks fastest serves the request;
//   * every free stream slot takes a micro-batch of the admitted requests:
//     their C zeroing and divides, then ONE grouped leaf launch over all
//     their leaf products (the same kernel as stark_batch_mul), then an
//     event; requests that arrive while others run are admitted as slots and
//     memory free up, so their work overlaps on the device;
//   * completion is observed by polling the slot events; the request's
//     latency runs from stark_submit to that observation.
// Workspaces are plans keyed by padded size, so one workspace serves every
// n that pads to the same n_pad; they stay resident until evicted.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"
#include "stark_internal.h"

namespace stark {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxMicroBatch = 16;

struct Request {
  uint64_t id;
  int64_t n;
  stark_dtype dt;
  const void* A;
  const void* B;
  void* C;
  Clock::time_point t_submit;
  stark_plan_s* ws = nullptr;  // workspace while running
  void* target = nullptr;      // combine target: C, or the workspace's staging copy
  int64_t ld = 0;              // its row pitch
  stark_status status = STARK_OK;
  bool deferred = false;       // admission waited at least once for device memory
};

struct Workspace {
  stark_plan_s* plan;
  bool busy;
  Clock::time_point last_used;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  GroupDesc* d_desc = nullptr;  // device descriptors of the running micro-batch
  GroupDesc* h_desc = nullptr;  // pinned host staging
  std::vector<Request*> running;
};

}  // namespace
}  // namespace stark

struct stark_server_s {
  int device = 0;
  size_t budget = 0;
  size_t owned = 0;  // bytes of all cached workspaces
  std::mutex mu;
  std::condition_variable cv;
  std::deque<stark::Request*> queue;
  std::unordered_map<uint64_t, stark::Request*> live;  // queued or running
  std::unordered_map<uint64_t, std::pair<stark_status, double>> finished;  // not yet reaped
  std::unordered_map<uint64_t, double> latency;                          // every finished request
  std::map<std::tuple<int64_t, int, int, int>, std::vector<stark::Workspace>> cache;  // (npad, depth, dt, dfs)
  std::vector<stark::Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  int* d_err = nullptr;
  int num_sms = 1;
  // load counters (stark_server_load)
  int64_t max_queued = 0;  // most requests waiting at once
  int64_t deferred = 0;    // requests whose admission waited for device memory
  int64_t done = 0;        // requests finished
};

using namespace stark;

namespace {

// Tensor-core dtypes: the measured autotuner (per size class, cached);
// fp64/int64: the cost model.
int depth_for(int64_t n, stark_dtype dt) {
  return is_split(dt) ? autotune_depth(n, dt) : choose_depth(n, dt);
}

// Device bytes of a workspace for side npad over `levels` depth-first levels
// (the quadrant tables and error word fit in the 1 MB margin).
size_t workspace_need(int64_t npad, int d, stark_dtype dt, int levels) {
  return (size_t)(operand_bytes(npad, d, dt) / pow7i(levels)) + (1u << 20);
}

// Split dtypes combine a C that TMA cannot address (n % 4 != 0) in the
// workspace's staging copy of side npad.
bool needs_stage(int64_t n, stark_dtype dt, const void* C) {
  return is_split(dt) && !c_is_tma_target(C, n);
}
size_t stage_bytes(int64_t npad) { return (size_t)npad * (size_t)staged_ld(npad) * sizeof(float); }

// Traversal of a bucket's workspace: breadth first when it (plus `extra`
// bytes) fits the budget, else the fewest depth-first levels that fit; -1
// when none does.
int admit_levels(int64_t npad, int d, stark_dtype dt, size_t extra, size_t budget) {
  for (int levels = 0; levels <= 2; ++levels)
    if (traversal_supported(d, dt, levels) && workspace_need(npad, d, dt, levels) + extra <= budget) return levels;
  return -1;
}

// Depth and traversal of a request of side n: `first` (the dispatcher's
// depth; -1 for none) with the fewest depth-first levels that fit the
// budget, else the fitting depth the cost model ranks fastest.  false when
// no depth fits.
bool admission(int64_t n, stark_dtype dt, bool staged, size_t budget, int first, int* depth, int* levels) {
  std::vector<std::pair<double, int>> order;
  for (int d = 0; d <= kMaxDepth; ++d) order.emplace_back(d == first ? -1.0 : model_seconds(n, d, dt), d);
  std::sort(order.begin(), order.end());
  for (const auto& c : order) {
    const int64_t npad = padded_side(n, c.second, dt);
    const int l = admit_levels(npad, c.second, dt, staged ? stage_bytes(npad) : 0, budget);
    if (l >= 0) {
      *depth = c.second;
      *levels = l;
      return true;
    }
  }
  return false;
}

// Evict idle workspaces, least recently used first, until `need` more bytes
// fit the budget; false when the busy ones alone leave no room.
bool make_room(stark_server_s* s, size_t need) {
  while (s->owned + need > s->budget) {
    Workspace* victim = nullptr;
    std::vector<Workspace>* vpool = nullptr;
    for (auto& kv : s->cache)
      for (auto& w : kv.second)
        if (!w.busy && (!victim || w.last_used < victim->last_used)) {
          victim = &w;
          vpool = &kv.second;
        }
    if (!victim) return false;
    s->owned -= (size_t)victim->plan->ws_bytes;
    plan_release(victim->plan);
    delete victim->plan;
    vpool->erase(vpool->begin() + (victim - vpool->data()));
  }
  return true;
}

void release_workspace(stark_server_s* s, stark_plan_s* p);

// Find or make an idle workspace for request r, with its staging copy of C
// where it needs one (server mutex held).  EBUSY: it fits the budget once
// running requests free their workspaces.
stark_plan_s* acquire_workspace(stark_server_s* s, const Request& r, stark_status* err) {
  const bool staged = needs_stage(r.n, r.dt, r.C);
  int d = 0, levels = 0;
  if (!admission(r.n, r.dt, staged, s->budget, depth_for(r.n, r.dt), &d, &levels)) {
    *err = STARK_ENOMEM;
    return nullptr;
  }
  const int64_t npad = padded_side(r.n, d, r.dt);
  const size_t stage = staged ? stage_bytes(npad) : 0;
  auto key = std::make_tuple(npad, d, (int)r.dt, levels);
  stark_plan_s* p = nullptr;
  for (auto& w : s->cache[key])
    if (!w.busy) {
      w.busy = true;
      w.last_used = Clock::now();
      p = w.plan;  // the entry itself may move while room is made below
      break;
    }
  if (p) {
    if (stage && !p->cstage) {
      const int64_t before = p->ws_bytes;
      if (!make_room(s, stage) || plan_ensure_cstage(p) != STARK_OK) {
        release_workspace(s, p);
        *err = STARK_EBUSY;
        return nullptr;
      }
      s->owned += (size_t)(p->ws_bytes - before);
    }
    return p;
  }
  // a new workspace: does it fit once idle ones are evicted?
  if (!make_room(s, workspace_need(npad, d, r.dt, levels) + stage)) {
    *err = STARK_EBUSY;  // wait for running requests to free memory
    return nullptr;
  }
  p = new (std::nothrow) stark_plan_s();
  if (!p) {
    *err = STARK_ENOMEM;
    return nullptr;
  }
  stark_status st = plan_init(p, npad, d, r.dt, false, levels);  // sized for the whole bucket
  if (st == STARK_OK && stage) st = plan_ensure_cstage(p);
  if (st != STARK_OK) {
    plan_release(p);
    delete p;
    *err = st;
    return nullptr;
  }
  s->owned += (size_t)p->ws_bytes;
  s->cache[key].push_back(Workspace{p, true, Clock::now()});
  return p;
}

void release_workspace(stark_server_s* s, stark_plan_s* p) {
  for (auto& kv : s->cache)
    for (auto& w : kv.second)
      if (w.plan == p) {
        w.busy = false;
        w.last_used = Clock::now();
        return;
      }
}

void finish(stark_server_s* s, Request* r, stark_status st) {
  const double lat = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  s->finished[r->id] = {st, lat};
  s->latency[r->id] = lat;
  ++s->done;
  s->live.erase(r->id);
  if (r->ws) release_workspace(s, r->ws);
  delete r;
}

// Enqueue one micro-batch on a slot (server mutex held).
stark_status launch_micro_batch(stark_server_s* s, Slot& slot, std::vector<Request*>& reqs) {
  cudaStream_t st = slot.stream;
  std::vector<Request*> tc;
  for (Request* r : reqs) {
    const bool split = is_split(r->dt);
    // C that TMA cannot address is combined in the workspace's staging copy
    // (allocated at admission, inside the budget)
    const bool staged = needs_stage(r->n, r->dt, r->C);
    if (staged && !r->ws->cstage) return STARK_ENOMEM;
    stark_plan_s view = *r->ws;  // the bucket workspace, bounds of this request
    view.n = r->n;
    view.ev.clear();
    view.timing_cap = 0;
    stark_status e;
    if (split && !r->ws->dfs) {
      r->target = staged ? r->ws->cstage : r->C;
      r->ld = staged ? staged_ld(r->n) : r->n;
      if (cudaMemsetAsync(r->target, 0, (size_t)r->n * r->ld * sizeof(float), st) != cudaSuccess) return STARK_ECUDA;
      e = plan_divide(&view, r->A, r->B, st);
      tc.push_back(r);
    } else {
      // plain dtypes, and depth-first workspaces (one subtree's operands at a
      // time): the plan's own sequence on this slot's stream
      e = plan_run(&view, r->A, r->B, r->C, 0, view.P, st);
    }
    if (e != STARK_OK) return e;
  }
  if (!tc.empty()) {
    // 256-wide members first (one grouped launch), then 128-wide ones
    std::stable_partition(tc.begin(), tc.end(), [](Request* r) { return r->ws->L % 256 == 0; });
    int split = 0;
    while (split < (int)tc.size() && tc[split]->ws->L % 256 == 0) ++split;
    const bool tf32 = tc[0]->dt == STARK_F32_SPLIT_TF32;
    int64_t items_wide = 0, items = 0;
    for (size_t k = 0; k < tc.size(); ++k) {
      if ((int)k == split) {
        items_wide = items;
        items = 0;
      }
      const int bn = (int)k < split ? 256 : 128;
      stark_plan_s* p = tc[k]->ws;
      GroupDesc& g = slot.h_desc[k];
      std::memset(&g, 0, sizeof(g));
      g.tmA = p->tmA;
      if (tf32 && !p->tf32_mn) {
        // K-major tf32 Y; 256-wide members run CTA pairs: each CTA loads 128 Y rows
        if (!make_tmap_planes(&g.tmB, p->Y, true, p->L, 2 * p->P, bn == 256 ? 128 : bn)) return STARK_EUNSUPPORTED;
      } else {
        g.tmB = p->tmB;
      }
      g.item_base = (int32_t)items;
      g.P = (int32_t)p->P;
      g.L = (int32_t)p->L;
      g.ctab = p->d_ctab;
      g.ccount = p->d_ccount;
      g.maxT = p->maxT;
      g.C = static_cast<float*>(tc[k]->target);
      g.n = tc[k]->n;
      g.ldc = tc[k]->ld;
      g.use_tma_c = make_tmap_c(&g.tmC, g.C, g.n, g.ldc) ? 1 : 0;
      items += bn == 256 ? p->P * (p->L / 256) * (p->L / 256) : p->P * (p->L / 128) * (p->L / 128);
    }
    if (split == (int)tc.size()) {
      items_wide = items;
      items = 0;
    }
    if (cudaMemcpyAsync(slot.d_desc, slot.h_desc, sizeof(GroupDesc) * tc.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return STARK_ECUDA;
    LeafTcArgs a{};
    a.b_mn = tf32 && tc[0]->ws->tf32_mn;  // every workspace has the plan default
    a.fp16 = tc[0]->dt == STARK_F32_SPLIT_FP16 ? 1 : 0;  // one dtype per micro-batch
    a.err = s->d_err;
    a.timeout_ns = kDefaultTimeoutNs;
    if (split > 0) {
      a.groups = slot.d_desc;
      a.ngroups = split;
      a.total_items = (int32_t)items_wide;
      if (launch_leaf_tc2_grouped(a, tf32, s->num_sms, st) != cudaSuccess) return STARK_ECUDA;
    }
    if (split < (int)tc.size()) {
      a.groups = slot.d_desc + split;
      a.ngroups = (int32_t)tc.size() - split;
      a.total_items = (int32_t)items;
      if (launch_leaf_tc_grouped(a, tf32, 128, s->num_sms, st) != cudaSuccess) return STARK_ECUDA;
    }
    for (Request* r : tc)
      if (r->target != r->C) {
        const size_t w = (size_t)r->n * sizeof(float);
        if (cudaMemcpy2DAsync(r->C, w, r->target, (size_t)r->ld * sizeof(float), w, (size_t)r->n,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          return STARK_ECUDA;
      }
  }
  if (cudaEventRecord(slot.done, st) != cudaSuccess) return STARK_ECUDA;
  return STARK_OK;
}

void worker_loop(stark_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // 1. completions
    bool any_running = false;
    for (Slot& slot : s->slots) {
      if (slot.running.empty()) continue;
      const cudaError_t q = cudaEventQuery(slot.done);
      if (q == cudaErrorNotReady) {
        any_running = true;
        continue;
      }
      stark_status st = q == cudaSuccess ? STARK_OK : STARK_ECUDA;
      int e = 0;
      if (st == STARK_OK && cudaMemcpy(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && e) {
        st = STARK_ETIMEOUT;
        cudaMemset(s->d_err, 0, sizeof(int));
      }
      cudaGetLastError();
      for (Request* r : slot.running) finish(s, r, st);
      slot.running.clear();
    }
    if (s->stop && s->queue.empty() && !any_running) {
      bool idle = true;
      for (Slot& slot : s->slots) idle = idle && slot.running.empty();
      if (idle) break;
    }
    // 2. admission into free slots, arrival order
    for (Slot& slot : s->slots) {
      if (!slot.running.empty() || s->queue.empty()) continue;
      std::vector<Request*> batch;
      while (!s->queue.empty() && (int)batch.size() < kMaxMicroBatch) {
        Request* r = s->queue.front();
        if (!batch.empty() && (r->dt != batch[0]->dt)) break;  // one dtype per grouped launch
        stark_status err = STARK_OK;
        r->ws = acquire_workspace(s, *r, &err);
        if (!r->ws) {
          if (err == STARK_EBUSY) {
            bool running = false;
            for (Slot& o : s->slots) running = running || !o.running.empty();
            if (running || !batch.empty()) {  // memory frees up when those finish
              if (!r->deferred) {
                r->deferred = true;
                ++s->deferred;
              }
              break;
            }
            err = STARK_ENOMEM;                    // cannot ever fit
          }
          s->queue.pop_front();
          finish(s, r, err);
          continue;
        }
        s->queue.pop_front();
        batch.push_back(r);
      }
      if (batch.empty()) continue;
      const stark_status st = launch_micro_batch(s, slot, batch);
      if (st != STARK_OK) {
        cudaStreamSynchronize(slot.stream);
        cudaGetLastError();
        for (Request* r : batch) finish(s, r, st);
      } else {
        slot.running = batch;
        any_running = true;
      }
    }
    // 3. wait: briefly while work runs (poll events), else for a submission
    if (any_running) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else if (!s->stop && s->queue.empty()) {
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
    } else if (!s->queue.empty()) {
      // queued but not admissible right now and nothing runs: retry shortly
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      lk.lock();
    }
  }
}

void server_free(stark_server_s* s) {
  for (auto& kv : s->cache)
    for (auto& w : kv.second) {
      plan_release(w.plan);
      delete w.plan;
    }
  for (Slot& slot : s->slots) {
    if (slot.stream) cudaStreamDestroy(slot.stream);
    if (slot.done) cudaEventDestroy(slot.done);
    cudaFree(slot.d_desc);
    cudaFreeHost(slot.h_desc);
  }
  for (auto& kv : s->live) delete kv.second;
  cudaFree(s->d_err);
  cudaGetLastError();
  delete s;
}

}  // namespace

extern "C" {

stark_status stark_server_create(size_t hbm_budget_bytes, int32_t slots, stark_server_t* out) {
  if (!out || hbm_budget_bytes == 0 || slots <= 0 || slots > 64) return STARK_EINVAL;
  *out = nullptr;
  if (!device_is_sm100_family()) return STARK_EUNSUPPORTED;
  auto* s = new (std::nothrow) stark_server_s();
  if (!s) return STARK_ENOMEM;
  cudaGetDevice(&s->device);
  s->budget = hbm_budget_bytes;
  s->num_sms = device_sm_count();
  s->slots.resize((size_t)slots);
  bool ok = cudaMalloc(&s->d_err, sizeof(int)) == cudaSuccess && cudaMemset(s->d_err, 0, sizeof(int)) == cudaSuccess;
  for (Slot& slot : s->slots) {
    ok = ok && cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&slot.d_desc, sizeof(GroupDesc) * kMaxMicroBatch) == cudaSuccess;
    ok = ok && cudaMallocHost(&slot.h_desc, sizeof(GroupDesc) * kMaxMicroBatch) == cudaSuccess;
  }
  if (!ok) {
    server_free(s);
    return STARK_ENOMEM;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return STARK_OK;
}

stark_status stark_server_admission(size_t hbm_budget_bytes, int64_t n, stark_dtype dt, int staged, int32_t* depth,
                                    int32_t* levels, int64_t* bytes) {
  if (n < 0 || n > (int64_t)1 << 20) return STARK_EINVAL;
  if (dt != STARK_F64 && dt != STARK_I64 && !is_split(dt)) return STARK_EINVAL;
  const bool split = is_split(dt);
  int d = 0, l = 0;
  if (!admission(n, dt, split && staged, hbm_budget_bytes, choose_depth(n, dt), &d, &l)) return STARK_ENOMEM;
  const int64_t npad = padded_side(n, d, dt);
  if (depth) *depth = d;
  if (levels) *levels = l;
  if (bytes) *bytes = (int64_t)(workspace_need(npad, d, dt, l) + (split && staged ? stage_bytes(npad) : 0));
  return STARK_OK;
}

stark_status stark_submit(stark_server_t s, int64_t n, stark_dtype dt, const void* A, const void* B, void* C,
                          uint64_t* req_id) {
  if (!s || !req_id || n < 0 || n > (int64_t)1 << 20) return STARK_EINVAL;
  if (dt != STARK_F64 && dt != STARK_I64 && !is_split(dt)) return STARK_EINVAL;
  if (n > 0 && (!A || !B || !C)) return STARK_EINVAL;
  int d = 0, levels = 0;
  if (!admission(n, dt, needs_stage(n, dt, C), s->budget, -1, &d, &levels)) return STARK_ENOMEM;  // no depth fits
  auto* r = new (std::nothrow) Request();
  if (!r) return STARK_ENOMEM;
  r->n = n;
  r->dt = dt;
  r->A = A;
  r->B = B;
  r->C = C;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return STARK_EINVAL;
    }
    r->id = s->next_id++;
    *req_id = r->id;
    if (n == 0) {
      s->live[r->id] = r;
      finish(s, r, STARK_OK);
      return STARK_OK;
    }
    s->live[r->id] = r;
    s->queue.push_back(r);
    s->max_queued = std::max<int64_t>(s->max_queued, (int64_t)s->queue.size());
  }
  s->cv.notify_one();
  return STARK_OK;
}

stark_status stark_poll(stark_server_t s, uint64_t id, int* done, stark_status* req_status) {
  if (!s || !done) return STARK_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto f = s->finished.find(id);
  if (f != s->finished.end()) {
    *done = 1;
    if (req_status) *req_status = f->second.first;
    s->finished.erase(f);
    return STARK_OK;
  }
  if (s->live.count(id)) {
    *done = 0;
    return STARK_OK;
  }
  return STARK_ENOTFOUND;
}

stark_status stark_server_drain(stark_server_t s) {
  if (!s) return STARK_EINVAL;
  while (true) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->live.empty()) return STARK_OK;
    }
    s->cv.notify_one();
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

stark_status stark_request_latency(stark_server_t s, uint64_t id, double* seconds) {
  if (!s || !seconds) return STARK_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->latency.find(id);
  if (it == s->latency.end()) return s->live.count(id) ? STARK_EBUSY : STARK_ENOTFOUND;
  *seconds = it->second;
  return STARK_OK;
}

stark_status stark_server_stats(stark_server_t s, int64_t* cached_workspaces, int64_t* owned_bytes,
                                int64_t* queued) {
  if (!s) return STARK_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t w = 0;
  for (auto& kv : s->cache) w += (int64_t)kv.second.size();
  if (cached_workspaces) *cached_workspaces = w;
  if (owned_bytes) *owned_bytes = (int64_t)s->owned;
  if (queued) *queued = (int64_t)s->queue.size();
  return STARK_OK;
}

stark_status stark_server_load(stark_server_t s, int64_t* max_queued, int64_t* deferred, int64_t* finished) {
  if (!s) return STARK_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (max_queued) *max_queued = s->max_queued;
  if (deferred) *deferred = s->deferred;
  if (finished) *finished = s->done;
  return STARK_OK;
}

stark_status stark_server_destroy(stark_server_t s) {
  if (!s) return STARK_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_one();
  if (s->worker.joinable()) s->worker.join();
  cudaDeviceSynchronize();
  server_free(s);
  return STARK_OK;
}

}  // extern "C"
