// Multi-tenant serving with continuous batching.
//
// Tenant maps stay resident on the device.  Requests (one operation on one
// tenant: insert, activate, find or erase of n keys) arrive through
// ash_server_submit, which copies the caller's keys and values into pinned
// staging and queues the request.  A worker thread repeatedly
//   1. releases the device staging of batches that finished,
//   2. admits queued requests in arrival order while their device staging
//      fits the HBM budget (a request larger than the whole budget is admitted
//      alone),
//   3. forms a batch of at most one admitted request per tenant (so each
//      tenant's requests run in arrival order), grows a tenant map x2 before
//      an insert would push its live/capacity ratio past max_load,
//   4. uploads the batch on a copy stream, runs it as ONE ash_batch_run graph
//      on the compute stream, downloads its outputs on a second copy stream
//      and marks the requests done from a host callback.
// The worker does not wait for a batch before launching the next one, so
// uploads, kernels and downloads of consecutive batches overlap, and requests
// that arrive while others are on the GPU join the next batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ash.h"
#include "ash_internal.h"

using namespace ash::host;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kMaxTenants = 256;

int64_t align256(int64_t x) { return (x + 255) & ~int64_t{255}; }

// Pinned host staging.  One pinned arena is allocated when the server is
// created (pinning pages during serving is slow and stalls the caller), and
// carved first-fit in 4 KiB units with coalescing frees.  When the arena is
// full a block comes from cudaMallocHost and is cached by size for reuse.
class PinnedPool {
 public:
  void reserve(int64_t bytes) {
    bytes = (bytes + kUnit - 1) / kUnit * kUnit;
    if (bytes <= 0) return;
    void* p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    base_ = static_cast<char*>(p);
    size_ = bytes;
    free_.emplace(0, bytes);
  }
  void* take(int64_t bytes, int64_t* cls_bytes) {
    if (bytes <= 0) {
      *cls_bytes = 0;
      return nullptr;
    }
    const int64_t need = (bytes + kUnit - 1) / kUnit * kUnit;
    {
      std::lock_guard<std::mutex> lk(mu_);
      for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < need) continue;
        const int64_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > need) free_.emplace(off + need, len - need);
        *cls_bytes = need;  // arena block: its size
        return base_ + off;
      }
      // spill blocks come in power-of-two sizes, so that the few classes
      // are reused instead of pinning a new block of every request size
      auto& v = spill_[spill_class(need)];
      if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        *cls_bytes = -spill_class(need);  // spill block
        return p;
      }
    }
    const int64_t cls = spill_class(need);
    void* p = nullptr;
    if (cudaMallocHost(&p, cls) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    spills_.fetch_add(1, std::memory_order_relaxed);
    *cls_bytes = -cls;
    return p;
  }
  static int64_t spill_class(int64_t need) {
    int64_t c = kUnit;
    while (c < need) c *= 2;
    return c;
  }
  int64_t spills() const { return spills_.load(std::memory_order_relaxed); }
  void give(void* p, int64_t cls_bytes) {
    if (!p || cls_bytes == 0) return;
    std::lock_guard<std::mutex> lk(mu_);
    if (cls_bytes < 0) {
      spill_[-cls_bytes].push_back(p);
      return;
    }
    int64_t off = static_cast<char*>(p) - base_, len = cls_bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + len == next->first) {  // merge with the following block
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the preceding block
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        off = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_.emplace(off, len);
  }
  ~PinnedPool() {
    if (base_) cudaFreeHost(base_);
    for (auto& kv : spill_)
      for (void* p : kv.second) cudaFreeHost(p);
  }

 private:
  static constexpr int64_t kUnit = 4096;
  std::atomic<int64_t> spills_{0};
  std::mutex mu_;
  char* base_ = nullptr;
  int64_t size_ = 0;
  std::map<int64_t, int64_t> free_;                 // arena offset -> length
  std::map<int64_t, std::vector<void*>> spill_;     // cudaMallocHost blocks by size
};

// Device staging carved from one allocation made when the server is created
// (staging_bytes, the admission budget), first-fit in 256-byte units with
// coalescing frees: serving then calls no allocator per request.  A request
// that does not fit (one larger than the budget is admitted alone, or the
// free space is fragmented) gets a stream-ordered allocation instead.  Only
// the worker thread uses it.
class DeviceArena {
 public:
  void reserve(int64_t bytes) {
    bytes = (bytes + kUnit - 1) / kUnit * kUnit;
    if (bytes <= 0) return;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    base_ = static_cast<char*>(p);
    size_ = bytes;
    free_.emplace(0, bytes);
  }
  // nullptr when no free block is large enough
  char* take(int64_t bytes, int64_t* taken) {
    const int64_t need = (bytes + kUnit - 1) / kUnit * kUnit;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_.emplace(off + need, len - need);
      *taken = need;
      return base_ + off;
    }
    return nullptr;
  }
  void give(char* p, int64_t taken) {
    int64_t off = p - base_, len = taken;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + len == next->first) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        off = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_.emplace(off, len);
  }
  ~DeviceArena() {
    if (base_) cudaFree(base_);
  }

 private:
  static constexpr int64_t kUnit = 256;
  char* base_ = nullptr;
  int64_t size_ = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
};

// Page-locked (pinned or registered) host memory, which copy engines read
// directly.
bool is_pinned(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

struct Request {
  uint64_t id = 0;
  int tenant = 0;
  int op = 0;
  int64_t n = 0;
  int32_t* idx_user = nullptr;
  uint8_t* mask_user = nullptr;
  const int32_t* keys_user = nullptr;  // zero-copy: the caller's arrays, used in place
  const void* vals_user = nullptr;
  bool zero_copy = false;
  bool direct_in = false;    // inputs uploaded by DMA from the caller's pinned arrays
  bool direct_out = false;   // outputs downloaded by DMA into the caller's pinned arrays
  int64_t host_out_off = 0;  // offset of the outputs in the host staging block
  // staging: [keys | values | idx | mask], each 256-byte aligned
  int64_t off_keys = 0, off_vals = 0, off_idx = 0, off_mask = 0, bytes = 0;
  void* host = nullptr;
  int64_t host_cls = 0;
  char* dev = nullptr;
  int64_t dev_taken = 0;     // bytes carved from the device arena; 0: a stream-ordered allocation
  Clock::time_point t_submit, t_done;
  bool gpu_done = false;
  bool delivered = false;
};

// A launched batch.  It owns copies of what the worker must release after the
// batch finishes (device staging and its byte count), because once the
// completion callback publishes the requests as done, ash_server_wait may
// free them at any time; only the callback touches `reqs`, before that point.
struct Batch {
  std::vector<Request*> reqs;
  std::vector<std::pair<char*, int64_t>> dev;  // device staging and its arena bytes (0: allocated)
  int64_t staged = 0;
  struct ash_server* server = nullptr;
  bool done = false;
};

}  // namespace

struct ash_server {
  ash_server_config cfg{};
  std::vector<ash_map*> maps;
  ash_batch* batch = nullptr;
  cudaStream_t s_comp = nullptr, s_h2d = nullptr, s_d2h = nullptr;
  // Tenant growth runs on its own stream; the worker leaves the growing
  // tenant out of batches until grow_done[t] has completed, so the other
  // tenants' batches keep running.
  cudaStream_t s_grow = nullptr;
  cudaEvent_t comp_mark = nullptr;
  std::vector<cudaEvent_t> grow_done;
  std::vector<char> growing;
  PinnedPool pinned;
  DeviceArena arena;
  int64_t value_bytes = 0;

  std::mutex mu;
  std::condition_variable cv_work;
  std::condition_variable cv_done;
  std::deque<Request*> pending;   // submitted, not yet admitted
  std::deque<Request*> admitted;  // device staging granted, not yet launched
  std::deque<Batch*> inflight;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  int64_t staged_bytes = 0;       // device staging held by admitted / in-flight requests
  uint64_t next_id = 1;
  bool stop = false;
  ash_status worker_error = ASH_OK;
  std::string worker_msg;
  std::thread worker;
  ash_server_stats stats{};
};

namespace {

void CUDART_CB on_batch_done(void* arg) {
  Batch* b = static_cast<Batch*>(arg);
  ash_server* s = b->server;
  const auto now = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request* r : b->reqs) {
      r->t_done = now;
      r->gpu_done = true;
    }
    b->done = true;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_one();
}

// Worker-side: before an insert of n keys, grow the tenant map (x2 until it
// fits) when the host's upper bound on its live entries would pass max_load
// of the capacity.  The growth runs on the device with no host
// synchronisation (grow_async), on the growth stream after the compute
// stream's work so far (which may still read the old table); the worker
// leaves the tenant out of batches until it has finished, while other
// tenants' batches keep running.
ash_status grow_for_insert(ash_server* s, int t, int64_t n) {
  ash_map* m = s->maps[t];
  const double lim = s->cfg.max_load;
  const int64_t max_used = static_cast<int64_t>(m->tuning.max_used_fraction * static_cast<double>(m->n_slots));
  if (static_cast<double>(m->size_ub + n) > lim * static_cast<double>(m->capacity) || m->used_ub + n > max_used)
    tighten_bounds(m);
  const double need = static_cast<double>(m->size_ub + n);
  // a table whose live + erased slots could pass max_used_fraction is rebuilt
  // here too (at the same capacity when the live entries still fit), so the
  // batch's own growth check never has to synchronise the compute stream
  if (!(m->used_ub + n > max_used)) tighten_bounds(m);  // a landed snapshot may report new tombstones
  const bool grow = need > lim * static_cast<double>(m->capacity);
  const bool rebuild = m->used_ub + n > max_used || tombstones_need_rebuild(m);
  if (!grow && !rebuild) return ASH_OK;
  // the new capacity holds the live entries and this insert under both
  // limits, so a rebuild is never followed by another one for the same batch
  const double used_frac = m->tuning.max_used_fraction * m->tuning.slots_per_capacity;
  int64_t c = m->capacity;
  while (need > lim * static_cast<double>(c) || need > used_frac * static_cast<double>(c)) c *= 2;
  if (cudaEventRecord(s->comp_mark, s->s_comp) != cudaSuccess ||
      cudaStreamWaitEvent(s->s_grow, s->comp_mark, 0) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "server growth ordering");
  ash_status st = grow_async(m, c, s->s_grow);
  if (st != ASH_OK) return st;
  if (cudaEventRecord(s->grow_done[t], s->s_grow) != cudaSuccess) return cuda_fail(cudaGetLastError(), "grow event");
  s->growing[t] = 1;  // the caller counts the growth in the stats
  return ASH_OK;
}

}  // namespace

namespace ash {
namespace host {
void server_layout(const ash_server* s, int* key_dim, int* value_row_bytes, int* n_tenants) {
  *key_dim = s->cfg.key_dim;
  *value_row_bytes = s->cfg.value_row_bytes;
  *n_tenants = s->cfg.n_tenants;
}
}  // namespace host
}  // namespace ash

namespace {

void worker_loop(ash_server* s) {
  DeviceGuard g(s->cfg.device);
  // No CUDA call is made while holding s->mu: the completion callback of a
  // batch takes that mutex on the driver's callback thread.  growing[] and
  // the growth events belong to this thread alone.
  std::vector<Batch*> finished;
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // 1) batches that finished: their device staging is released below
    while (!s->inflight.empty() && s->inflight.front()->done) {
      finished.push_back(s->inflight.front());
      s->inflight.pop_front();
      s->staged_bytes -= finished.back()->staged;
    }
    if (s->stop && s->pending.empty() && s->admitted.empty() && s->inflight.empty() && finished.empty()) break;
    // 2) admission under the HBM staging budget, in arrival order
    while (!s->pending.empty()) {
      Request* r = s->pending.front();
      const bool alone = s->staged_bytes == 0;
      if (!alone && s->staged_bytes + r->bytes > s->cfg.staging_bytes) break;
      s->pending.pop_front();
      s->staged_bytes += r->bytes;
      s->admitted.push_back(r);
    }
    // 3) a batch: the oldest admitted request of each tenant.  A tenant whose
    //    map is growing (or rebuilding) on the growth stream is left out
    //    until that finishes, so its growth holds up no other tenant's batch.
    std::vector<Request*> pick;
    bool any_growing = false;
    {
      bool used[kMaxTenants] = {};
      for (int t = 0; t < s->cfg.n_tenants; ++t)
        if (s->growing[t]) used[t] = any_growing = true;
      for (auto it = s->admitted.begin(); it != s->admitted.end() && static_cast<int>(pick.size()) < s->cfg.max_batch_requests;) {
        Request* r = *it;
        if (used[r->tenant]) {
          ++it;
          continue;
        }
        used[r->tenant] = true;
        pick.push_back(r);
        it = s->admitted.erase(it);
      }
    }
    if (pick.empty() && finished.empty()) {
      if (any_growing) {
        s->cv_work.wait_for(lk, std::chrono::microseconds(50));
        lk.unlock();
        for (int t = 0; t < s->cfg.n_tenants; ++t) {  // poll the growth events
          if (!s->growing[t]) continue;
          if (cudaEventQuery(s->grow_done[t]) == cudaSuccess) s->growing[t] = 0;
          else cudaGetLastError();  // cudaErrorNotReady is not an error here
        }
        lk.lock();
      } else {
        s->cv_work.wait(lk);
      }
      continue;
    }
    lk.unlock();
    for (Batch* b : finished) {
      for (auto& d : b->dev) {
        if (d.second > 0) s->arena.give(d.first, d.second);  // the batch is done: the block is free at once
        else cudaFreeAsync(d.first, s->s_d2h);
      }
      delete b;
    }
    finished.clear();
    for (int t = 0; t < s->cfg.n_tenants; ++t) {  // growths that finished
      if (!s->growing[t]) continue;
      if (cudaEventQuery(s->grow_done[t]) == cudaSuccess) s->growing[t] = 0;
      else cudaGetLastError();
    }
    // an insert that needs its tenant to grow starts the growth and goes back
    // to the front of the queue (still the oldest of its tenant)
    ash_status st = ASH_OK;
    std::vector<Request*> deferred;
    for (size_t j = 0; j < pick.size() && st == ASH_OK;) {
      Request* r = pick[j];
      if (r->op == ASH_OP_INSERT || r->op == ASH_OP_ACTIVATE) {
        st = grow_for_insert(s, r->tenant, r->n);
        if (st == ASH_OK && s->growing[r->tenant]) {
          deferred.push_back(r);
          pick.erase(pick.begin() + static_cast<std::ptrdiff_t>(j));
          continue;
        }
      }
      ++j;
    }
    if (!deferred.empty()) {
      lk.lock();
      s->admitted.insert(s->admitted.begin(), deferred.begin(), deferred.end());
      s->stats.rehashes += static_cast<int64_t>(deferred.size());  // one growth started per deferred request
      lk.unlock();
    }
    if (pick.empty() && st == ASH_OK) {
      lk.lock();
      continue;
    }
    // 4) launch: upload, one batched graph, download, host callback
    std::vector<ash_batch_op> ops;
    if (st == ASH_OK) {
      for (Request* r : pick) {
        if (r->zero_copy) {
          ash_batch_op o{};
          o.map = s->maps[r->tenant];
          o.op = r->op;
          o.keys = r->keys_user;
          o.values = (r->op == ASH_OP_INSERT && s->value_bytes > 0) ? r->vals_user : nullptr;
          o.n = r->n;
          o.buf_indices = r->idx_user;
          o.masks = r->mask_user;
          ops.push_back(o);
          continue;
        }
        r->dev = s->arena.take(r->bytes, &r->dev_taken);
        if (!r->dev) {
          r->dev_taken = 0;
          if (cudaMallocAsync(reinterpret_cast<void**>(&r->dev), r->bytes, s->s_h2d) != cudaSuccess) {
            cudaGetLastError();
            r->dev = nullptr;
            st = ASH_ERR_OOM;
            break;
          }
        }
        if (r->direct_in) {
          const int64_t kb = r->n * s->cfg.key_dim * 4;
          cudaMemcpyAsync(r->dev + r->off_keys, r->keys_user, kb, cudaMemcpyHostToDevice, s->s_h2d);
          if (r->vals_user)
            cudaMemcpyAsync(r->dev + r->off_vals, r->vals_user, r->n * s->value_bytes, cudaMemcpyHostToDevice,
                            s->s_h2d);
        } else {
          const int64_t in_bytes = r->off_idx;  // keys and values precede the outputs
          cudaMemcpyAsync(r->dev, r->host, in_bytes, cudaMemcpyHostToDevice, s->s_h2d);
        }
        ash_batch_op o{};
        o.map = s->maps[r->tenant];
        o.op = r->op;
        o.keys = reinterpret_cast<const int32_t*>(r->dev + r->off_keys);
        o.values = (r->op == ASH_OP_INSERT && s->value_bytes > 0) ? r->dev + r->off_vals : nullptr;
        o.n = r->n;
        o.buf_indices = reinterpret_cast<int32_t*>(r->dev + r->off_idx);
        o.masks = reinterpret_cast<uint8_t*>(r->dev + r->off_mask);
        ops.push_back(o);
      }
    }
    if (st == ASH_OK) {
      cudaEvent_t up = nullptr, comp = nullptr;
      cudaEventCreateWithFlags(&up, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&comp, cudaEventDisableTiming);
      cudaEventRecord(up, s->s_h2d);
      cudaStreamWaitEvent(s->s_comp, up, 0);
      st = ash_batch_run(s->batch, ops.data(), static_cast<int>(ops.size()), reinterpret_cast<ash_stream>(s->s_comp));
      if (st == ASH_OK) {
        cudaEventRecord(comp, s->s_comp);
        cudaStreamWaitEvent(s->s_d2h, comp, 0);
        for (Request* r : pick) {
          if (r->zero_copy) continue;  // the kernels wrote the caller's arrays
          if (r->direct_out) {
            if (r->op != ASH_OP_ERASE)
              cudaMemcpyAsync(r->idx_user, r->dev + r->off_idx, r->n * 4, cudaMemcpyDeviceToHost, s->s_d2h);
            cudaMemcpyAsync(r->mask_user, r->dev + r->off_mask, r->n, cudaMemcpyDeviceToHost, s->s_d2h);
            continue;
          }
          const int64_t out_bytes = r->bytes - r->off_idx;
          cudaMemcpyAsync(static_cast<char*>(r->host) + r->host_out_off, r->dev + r->off_idx, out_bytes,
                          cudaMemcpyDeviceToHost, s->s_d2h);
        }
      }
      cudaEventDestroy(up);
      cudaEventDestroy(comp);
      if (st == ASH_OK) {
        Batch* b = new Batch();
        b->reqs = pick;
        for (Request* r : pick) {
          if (r->dev) b->dev.emplace_back(r->dev, r->dev_taken);
          b->staged += r->bytes;
        }
        b->server = s;
        lk.lock();
        s->inflight.push_back(b);
        s->stats.batches += 1;
        s->stats.batched_requests += static_cast<int64_t>(pick.size());
        lk.unlock();
        if (cudaLaunchHostFunc(s->s_d2h, on_batch_done, b) != cudaSuccess) {
          st = cuda_fail(cudaGetLastError(), "cudaLaunchHostFunc");
          lk.lock();
          s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), b));
          lk.unlock();
          delete b;
        }
      }
    }
    if (st != ASH_OK) {
      if (cudaStreamSynchronize(s->s_h2d) != cudaSuccess) cudaGetLastError();  // uploads issued for the failed batch
      for (Request* r : pick) {
        if (r->dev && r->dev_taken > 0) s->arena.give(r->dev, r->dev_taken);
        else if (r->dev) cudaFreeAsync(r->dev, s->s_h2d);
        r->dev = nullptr;
      }
    }
    lk.lock();
    if (st != ASH_OK) {
      // fail the picked requests so no waiter hangs, and give back their staging
      s->worker_error = st;
      s->worker_msg = ash_last_error();
      for (Request* r : pick) {
        s->staged_bytes -= r->bytes;
        r->gpu_done = true;
        r->t_done = Clock::now();
      }
      s->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

void ash_server_default_config(ash_server_config* c) {
  if (!c) return;
  c->n_tenants = 16;
  c->key_dim = 3;
  c->initial_capacity = 1 << 20;
  c->value_row_bytes = 0;
  c->device = 0;
  c->staging_bytes = int64_t{2} << 30;
  c->max_load = 0.7f;
  c->max_batch_requests = 256;
  c->zero_copy = 0;
}

ash_status ash_server_create(const ash_server_config* cfg, ash_server** out_host) {
  if (!cfg || !out_host) return fail(ASH_ERR_INVALID, "config and out are required");
  *out_host = nullptr;
  if (cfg->n_tenants < 1 || cfg->n_tenants > kMaxTenants) return fail(ASH_ERR_INVALID, "n_tenants must be in 1..256");
  if (cfg->key_dim < 1 || cfg->key_dim > 4) return fail(ASH_ERR_INVALID, "key_dim must be in 1..4");
  if (!(cfg->value_row_bytes == 0 || cfg->value_row_bytes == 4 || cfg->value_row_bytes == 8 || cfg->value_row_bytes == 16))
    return fail(ASH_ERR_INVALID, "value_row_bytes must be 0, 4, 8 or 16");
  if (cfg->initial_capacity < 1 || cfg->staging_bytes < (1 << 20)) return fail(ASH_ERR_INVALID, "bad capacity or budget");
  if (!(cfg->max_load > 0.05f && cfg->max_load <= 1.0f)) return fail(ASH_ERR_INVALID, "max_load must be in (0.05, 1]");
  if (cfg->max_batch_requests < 1 || cfg->max_batch_requests > 256) return fail(ASH_ERR_INVALID, "max_batch_requests in 1..256");
  if (cfg->zero_copy < 0 || cfg->zero_copy > 2) return fail(ASH_ERR_INVALID, "zero_copy must be 0, 1 or 2");
  if (cfg->zero_copy == 1) {
    ash_device_info info{};
    ash_status ds = ash_get_device_info(cfg->device, &info);
    if (ds != ASH_OK) return ds;
    if (info.pageable_memory_access != 1)
      return fail(ASH_ERR_INVALID, "zero_copy needs a device with pageable host memory access");
  }
  std::unique_ptr<ash_server> s(new ash_server());
  s->cfg = *cfg;
  s->value_bytes = cfg->value_row_bytes;
  if (cfg->zero_copy != 1) s->pinned.reserve(cfg->staging_bytes);  // host staging as large as the device budget
  DeviceGuard g(cfg->device);
  if (cfg->zero_copy != 1) s->arena.reserve(cfg->staging_bytes);     // device staging: the admission budget
  if (cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_grow, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->comp_mark, cudaEventDisableTiming) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "server streams");
  s->grow_done.assign(cfg->n_tenants, nullptr);
  s->growing.assign(cfg->n_tenants, 0);
  for (int t = 0; t < cfg->n_tenants; ++t)
    if (cudaEventCreateWithFlags(&s->grow_done[t], cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "server events");
  ash_status st = ash_batch_create(cfg->device, &s->batch);
  if (st != ASH_OK) return st;
  const int64_t numel = cfg->value_row_bytes / 4;
  const int32_t dt = ASH_I32;
  for (int t = 0; t < cfg->n_tenants; ++t) {
    ash_map* m = nullptr;
    st = ash_create(cfg->key_dim, cfg->initial_capacity, cfg->value_row_bytes ? 1 : 0, &numel, &dt, cfg->device, nullptr,
                    reinterpret_cast<ash_stream>(s->s_comp), &m);
    if (st != ASH_OK) {
      for (ash_map* x : s->maps) ash_destroy(x);
      ash_batch_destroy(s->batch);
      return st;
    }
    s->maps.push_back(m);
  }
  cudaStreamSynchronize(s->s_comp);
  ash_server* raw = s.release();
  raw->worker = std::thread(worker_loop, raw);
  *out_host = raw;
  return ASH_OK;
}

ash_status ash_server_submit(ash_server* s, int32_t tenant, int32_t op, const int32_t* keys_host,
                             const void* values_host, int64_t n, int32_t* buf_indices_host, uint8_t* masks_host,
                             uint64_t* request_id_host) {
  if (!s || !request_id_host) return fail(ASH_ERR_INVALID, "server and request_id are required");
  if (tenant < 0 || tenant >= s->cfg.n_tenants) return fail(ASH_ERR_INVALID, "tenant out of range");
  if (op < ASH_OP_INSERT || op > ASH_OP_ERASE) return fail(ASH_ERR_INVALID, "unknown op");
  if (n < 1 || n >= 0x7FFFFFFF) return fail(ASH_ERR_INVALID, "n must be in [1, 2^31 - 1)");
  if (!keys_host || !masks_host) return fail(ASH_ERR_INVALID, "keys and masks are required");
  if (op != ASH_OP_ERASE && !buf_indices_host) return fail(ASH_ERR_INVALID, "buf_indices is required");
  if (op == ASH_OP_INSERT && s->value_bytes > 0 && !values_host) return fail(ASH_ERR_INVALID, "values are required");
  auto r = std::make_unique<Request>();
  r->tenant = tenant;
  r->op = op;
  r->n = n;
  r->idx_user = buf_indices_host;
  r->mask_user = masks_host;
  const int64_t kb = n * s->cfg.key_dim * 4;
  const int64_t vb = (op == ASH_OP_INSERT) ? n * s->value_bytes : 0;
  if (s->cfg.zero_copy == 1) {
    r->zero_copy = true;
    r->keys_user = keys_host;
    r->vals_user = vb ? values_host : nullptr;
    r->bytes = 0;  // no device staging
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(ASH_ERR_INVALID, "server is stopping");
    r->id = s->next_id++;
    *request_id_host = r->id;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->stats.submitted += 1;
    s->cv_work.notify_one();
    return ASH_OK;
  }
  r->off_keys = 0;
  r->off_vals = align256(kb);
  r->off_idx = r->off_vals + align256(vb);
  r->off_mask = r->off_idx + align256(n * 4);
  r->bytes = r->off_mask + align256(n);
  // mode 2: pinned input arrays are uploaded by DMA straight from the caller.
  // Any mode: pinned output arrays receive the outputs by DMA (the caller
  // may not read them before wait returns, so no staging is needed).
  r->direct_in = s->cfg.zero_copy == 2 && is_pinned(keys_host) && (!vb || is_pinned(values_host));
  r->direct_out = is_pinned(masks_host) && (op == ASH_OP_ERASE || is_pinned(buf_indices_host));
  const int64_t in_bytes = r->direct_in ? 0 : r->off_idx;
  const int64_t out_bytes = r->direct_out ? 0 : r->bytes - r->off_idx;
  r->host_out_off = in_bytes;  // the host block holds the staged inputs, then the staged outputs
  r->host = nullptr;
  r->host_cls = 0;
  if (in_bytes + out_bytes > 0) {
    r->host = s->pinned.take(in_bytes + out_bytes, &r->host_cls);
    if (!r->host) return fail(ASH_ERR_OOM, "pinned staging allocation failed");
  }
  if (r->direct_in) {
    r->keys_user = keys_host;
    r->vals_user = vb ? values_host : nullptr;
  } else {
    std::memcpy(static_cast<char*>(r->host) + r->off_keys, keys_host, kb);
    if (vb) std::memcpy(static_cast<char*>(r->host) + r->off_vals, values_host, vb);
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      s->pinned.give(r->host, r->host_cls);
      return fail(ASH_ERR_INVALID, "server is stopping");
    }
    r->id = s->next_id++;
    *request_id_host = r->id;
    s->pending.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->stats.submitted += 1;
  }
  s->cv_work.notify_one();
  return ASH_OK;
}

ash_status ash_server_wait(ash_server* s, uint64_t request_id, int64_t timeout_ms, double* latency_ms_host) {
  if (!s) return fail(ASH_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return fail(ASH_ERR_INVALID, "unknown or already collected request id");
  Request* r = it->second.get();
  auto ready = [&] { return r->gpu_done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return fail(ASH_ERR_TIMEOUT, "request not finished within the timeout");
  std::unique_ptr<Request> owned = std::move(it->second);
  s->reqs.erase(it);
  const ash_status werr = s->worker_error;
  const std::string wmsg = s->worker_msg;
  lk.unlock();
  if (werr != ASH_OK) {
    s->pinned.give(r->host, r->host_cls);
    return fail(werr, "the serving worker failed a batch: " + wmsg);
  }
  if (!r->zero_copy) {
    if (!r->direct_out) {
      const char* out = static_cast<char*>(r->host) + r->host_out_off;
      if (r->op != ASH_OP_ERASE) std::memcpy(r->idx_user, out, r->n * 4);
      std::memcpy(r->mask_user, out + (r->off_mask - r->off_idx), r->n);
    }
    s->pinned.give(r->host, r->host_cls);
  }
  if (latency_ms_host)
    *latency_ms_host = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  std::lock_guard<std::mutex> lk2(s->mu);
  s->stats.completed += 1;
  return ASH_OK;
}

ash_status ash_server_stats_get(ash_server* s, ash_server_stats* out_host) {
  if (!s || !out_host) return fail(ASH_ERR_INVALID, "server and out are required");
  std::lock_guard<std::mutex> lk(s->mu);
  *out_host = s->stats;
  out_host->host_syncs = 0;
  for (ash_map* m : s->maps) out_host->host_syncs += __atomic_load_n(&m->host_syncs, __ATOMIC_RELAXED);
  out_host->pinned_spills = s->pinned.spills();
  return ASH_OK;
}

ash_status ash_server_map(ash_server* s, int32_t tenant, ash_map** out_host) {
  if (!s || !out_host || tenant < 0 || tenant >= s->cfg.n_tenants) return fail(ASH_ERR_INVALID, "bad arguments");
  *out_host = s->maps[tenant];
  return ASH_OK;
}

ash_status ash_server_stream(ash_server* s, ash_stream* out_host) {
  if (!s || !out_host) return fail(ASH_ERR_INVALID, "bad arguments");
  *out_host = reinterpret_cast<ash_stream>(s->s_comp);
  return ASH_OK;
}

ash_status ash_server_destroy(ash_server* s) {
  if (!s) return ASH_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  DeviceGuard g(s->cfg.device);
  cudaStream_t all[4] = {s->s_comp, s->s_h2d, s->s_d2h, s->s_grow};
  for (cudaStream_t x : all)
    if (x) cudaStreamSynchronize(x);
  for (auto& kv : s->reqs) s->pinned.give(kv.second->host, kv.second->host_cls);
  for (ash_map* m : s->maps) ash_destroy(m);  // frees on each map's last stream
  for (cudaStream_t x : all)
    if (x) cudaStreamSynchronize(x);
  ash_batch_destroy(s->batch);
  for (cudaEvent_t e : s->grow_done)
    if (e) cudaEventDestroy(e);
  if (s->comp_mark) cudaEventDestroy(s->comp_mark);
  for (cudaStream_t x : all)
    if (x) cudaStreamDestroy(x);
  delete s;
  return ASH_OK;
}

}  // extern "C"
