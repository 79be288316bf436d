// Native replay of a serving trace (measurement support, not part of the map).
//
// A trace is a list of requests (tenant, op, key rows, arrival time).  The
// replays below submit them at their arrival times from native threads and
// record, per request, the time from its scheduled arrival until its outputs
// are in the caller's host arrays.  Keeping the load generator native means
// the measured latency and throughput are the server's (or the sequential
// calls'), not those of a scripting-language client.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ash.h"
#include "ash_internal.h"

using namespace ash::host;
using Clock = std::chrono::steady_clock;

namespace {

// Host output arrays (indices, then masks) for every request of a trace, in
// one page-locked arena laid out before the replay starts, as a serving
// frontend with pinned buffers would hold them: the server downloads
// outputs into them by DMA, and no allocation falls inside the measured
// time.  The arena is kept for the next replay of the process (grown when a
// trace needs more) and is never freed: the CUDA runtime may be gone at
// exit.
struct OutArena {
  std::mutex mu;
  char* base = nullptr;
  int64_t bytes = 0;
};

OutArena& out_arena() {
  static OutArena* a = new OutArena();
  return *a;
}

// Offsets of each request's outputs (16-byte aligned: n int32 indices, then
// n mask bytes) and the arena holding them, or nullptr when pinning failed.
char* layout_outputs(const ash_replay_trace* t, std::vector<int64_t>& off) {
  off.resize(static_cast<size_t>(t->n_requests));
  int64_t at = 0;
  for (int64_t r = 0; r < t->n_requests; ++r) {
    off[static_cast<size_t>(r)] = at;
    at += (t->n[r] * 5 + 15) / 16 * 16;
  }
  OutArena& a = out_arena();
  if (a.bytes < at) {
    if (a.base) cudaFreeHost(a.base);
    a.base = nullptr;
    a.bytes = 0;
    const int64_t want = at + at / 4;  // headroom: traces of one workload differ a little in size
    void* p = nullptr;
    if (cudaMallocHost(&p, static_cast<size_t>(want)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    a.base = static_cast<char*>(p);
    a.bytes = want;
  }
  return a.base;
}

ash_status check_trace(const ash_replay_trace* t, int n_tenants) {
  if (!t || t->n_requests < 0) return fail(ASH_ERR_INVALID, "trace is required");
  if (t->n_requests == 0) return ASH_OK;
  if (!t->arrival_s || !t->tenant || !t->op || !t->n || !t->row || !t->keys_host)
    return fail(ASH_ERR_INVALID, "trace arrays are required");
  for (int64_t r = 0; r < t->n_requests; ++r) {
    if (t->n[r] < 1 || t->row[r] < 0) return fail(ASH_ERR_INVALID, "trace: request sizes must be >= 1, rows >= 0");
    if (t->row[r] + t->n[r] > t->rows) return fail(ASH_ERR_INVALID, "trace: a request reads past the key rows");
    if (t->tenant[r] < 0 || t->tenant[r] >= n_tenants) return fail(ASH_ERR_INVALID, "trace: tenant out of range");
    if (t->op[r] < ASH_OP_INSERT || t->op[r] > ASH_OP_ERASE) return fail(ASH_ERR_INVALID, "trace: unknown op");
    if (r > 0 && t->arrival_s[r] < t->arrival_s[r - 1]) return fail(ASH_ERR_INVALID, "trace: arrivals must not decrease");
  }
  return ASH_OK;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

ash_status ash_server_replay(ash_server* server, const ash_replay_trace* trace, int32_t threads,
                             double* latency_ms_host, double* span_s_host) {
  if (!server || !latency_ms_host || !span_s_host) return fail(ASH_ERR_INVALID, "server and outputs are required");
  if (threads < 1 || threads > 64) return fail(ASH_ERR_INVALID, "threads must be in 1..64");
  int key_dim = 0, value_row_bytes = 0, n_tenants = 0;
  server_layout(server, &key_dim, &value_row_bytes, &n_tenants);
  ash_status s = check_trace(trace, n_tenants);
  if (s != ASH_OK) return s;
  const int64_t R = trace->n_requests;
  *span_s_host = 0.0;
  if (R == 0) return ASH_OK;
  for (int64_t r = 0; r < R; ++r)
    if (trace->op[r] == ASH_OP_INSERT && value_row_bytes > 0 && !trace->values_host)
      return fail(ASH_ERR_INVALID, "trace: inserts need values");

  // requests of one tenant are submitted in trace order (the server applies
  // each tenant's requests in submission order); other tenants' requests
  // are submitted concurrently
  std::vector<int64_t> prev_same(static_cast<size_t>(R), -1);
  {
    std::vector<int64_t> last(static_cast<size_t>(n_tenants), -1);
    for (int64_t r = 0; r < R; ++r) {
      prev_same[static_cast<size_t>(r)] = last[static_cast<size_t>(trace->tenant[r])];
      last[static_cast<size_t>(trace->tenant[r])] = r;
    }
  }
  std::lock_guard<std::mutex> arena_lock(out_arena().mu);  // one replay at a time uses the arena
  std::vector<int64_t> out_off;
  char* arena = layout_outputs(trace, out_off);
  if (!arena) return fail(ASH_ERR_OOM, "replay: pinned output arena allocation failed");
  std::vector<std::atomic<uint64_t>> rid(static_cast<size_t>(R));
  for (auto& x : rid) x.store(0, std::memory_order_relaxed);
  std::atomic<int> error{ASH_OK};
  std::atomic<int64_t> last_done_ns{0};
  const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(20);
  const char* vals = static_cast<const char*>(trace->values_host);
  constexpr uint64_t kFailed = ~0ull;

  auto submitter = [&](int c) {
    for (int64_t r = c; r < R; r += threads) {
      const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(trace->arrival_s[r]));
      std::this_thread::sleep_until(due);
      const int64_t p = prev_same[static_cast<size_t>(r)];
      if (p >= 0)
        while (rid[static_cast<size_t>(p)].load(std::memory_order_acquire) == 0)
          std::this_thread::sleep_for(std::chrono::microseconds(2));
      const int64_t n = trace->n[r];
      char* o = arena + out_off[static_cast<size_t>(r)];
      uint64_t id = 0;
      ash_status st = static_cast<ash_status>(error.load());
      if (st == ASH_OK) {
        const int32_t* k = trace->keys_host + trace->row[r] * key_dim;
        const void* v = (trace->op[r] == ASH_OP_INSERT && value_row_bytes > 0) ? vals + trace->row[r] * value_row_bytes
                                                                                : nullptr;
        st = ash_server_submit(server, trace->tenant[r], trace->op[r], k, v, n, reinterpret_cast<int32_t*>(o),
                               reinterpret_cast<uint8_t*>(o + 4 * n), &id);
      }
      if (st != ASH_OK) {
        int ok = ASH_OK;
        error.compare_exchange_strong(ok, st);
        rid[static_cast<size_t>(r)].store(kFailed, std::memory_order_release);
      } else {
        rid[static_cast<size_t>(r)].store(id, std::memory_order_release);
      }
    }
  };
  auto waiter = [&](int w) {
    for (int64_t r = w; r < R; r += threads) {
      uint64_t id;
      while ((id = rid[static_cast<size_t>(r)].load(std::memory_order_acquire)) == 0)
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      if (id == kFailed) {
        latency_ms_host[r] = -1.0;
        continue;
      }
      double lat = 0.0;
      ash_status st = ash_server_wait(server, id, -1, &lat);
      const auto now = Clock::now();
      if (st != ASH_OK) {
        int ok = ASH_OK;
        error.compare_exchange_strong(ok, st);
      }
      const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(trace->arrival_s[r]));
      latency_ms_host[r] = ms_between(due, now);
      const int64_t ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - t0).count();
      int64_t prev = last_done_ns.load();
      while (ns > prev && !last_done_ns.compare_exchange_weak(prev, ns)) {
      }
    }
  };
  std::vector<std::thread> th;
  for (int c = 0; c < threads; ++c) th.emplace_back(submitter, c);
  for (int w = 0; w < threads; ++w) th.emplace_back(waiter, w);
  for (auto& t : th) t.join();
  *span_s_host = static_cast<double>(last_done_ns.load()) * 1e-9;
  if (error.load() != ASH_OK) return fail(static_cast<ash_status>(error.load()), "replay: a request failed");
  return ASH_OK;
}

ash_status ash_replay_sequential(ash_map* const* maps, int32_t n_maps, const ash_replay_trace* trace,
                                 double* latency_ms_host, double* span_s_host) {
  if (!maps || n_maps < 1 || !latency_ms_host || !span_s_host) return fail(ASH_ERR_INVALID, "maps and outputs are required");
  ash_status s = check_trace(trace, n_maps);
  if (s != ASH_OK) return s;
  const int64_t R = trace->n_requests;
  *span_s_host = 0.0;
  if (R == 0) return ASH_OK;
  if (!maps[0]) return fail(ASH_ERR_INVALID, "maps must not be NULL");
  const int key_dim = maps[0]->key_dim;
  const int device = maps[0]->device;
  int64_t value_bytes = maps[0]->n_values == 1 ? maps[0]->row_bytes[0] : 0;
  for (int i = 0; i < n_maps; ++i) {
    if (!maps[i] || maps[i]->key_dim != key_dim || maps[i]->device != device || maps[i]->n_values > 1 ||
        (maps[i]->n_values == 1 ? maps[i]->row_bytes[0] : 0) != value_bytes)
      return fail(ASH_ERR_INVALID, "maps must share device, key_dim and value layout (at most one value buffer)");
  }
  int64_t n_max = 0;
  for (int64_t r = 0; r < R; ++r) {
    n_max = std::max(n_max, trace->n[r]);
    if (trace->op[r] == ASH_OP_INSERT && value_bytes > 0 && !trace->values_host)
      return fail(ASH_ERR_INVALID, "trace: inserts need values");
  }
  DeviceGuard g(device);
  // the maps' own streams, restored at the end: destroy frees on them
  std::vector<cudaStream_t> prev_stream(static_cast<size_t>(n_maps));
  for (int i = 0; i < n_maps; ++i) prev_stream[static_cast<size_t>(i)] = maps[i]->last_stream;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaGetLastError(), "stream");
  char* dev = nullptr;
  char* host_out = nullptr;
  const int64_t kbytes = n_max * key_dim * 4, vbytes = n_max * value_bytes;
  const int64_t off_v = (kbytes + 255) / 256 * 256, off_i = off_v + (vbytes + 255) / 256 * 256;
  const int64_t off_m = off_i + (n_max * 4 + 255) / 256 * 256, total = off_m + n_max;
  if (cudaMalloc(&dev, total) != cudaSuccess || cudaMallocHost(&host_out, n_max * 5) != cudaSuccess) {
    cudaGetLastError();
    if (dev) cudaFree(dev);
    cudaStreamDestroy(st);
    return fail(ASH_ERR_OOM, "replay staging");
  }
  const char* vals = static_cast<const char*>(trace->values_host);
  const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(20);
  Clock::time_point last = t0;
  ash_status err = ASH_OK;
  for (int64_t r = 0; r < R && err == ASH_OK; ++r) {
    const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(trace->arrival_s[r]));
    std::this_thread::sleep_until(due);
    const int64_t n = trace->n[r];
    ash_map* m = maps[trace->tenant[r]];
    const int32_t* k = trace->keys_host + trace->row[r] * key_dim;
    int32_t* d_idx = reinterpret_cast<int32_t*>(dev + off_i);
    uint8_t* d_mask = reinterpret_cast<uint8_t*>(dev + off_m);
    const ash_stream as = reinterpret_cast<ash_stream>(st);
    cudaMemcpyAsync(dev, k, n * key_dim * 4, cudaMemcpyHostToDevice, st);
    const int op = trace->op[r];
    if (op == ASH_OP_INSERT) {
      const void* vp[1] = {dev + off_v};
      if (value_bytes > 0)
        cudaMemcpyAsync(dev + off_v, vals + trace->row[r] * value_bytes, n * value_bytes, cudaMemcpyHostToDevice, st);
      err = ash_insert(m, reinterpret_cast<const int32_t*>(dev), value_bytes > 0 ? vp : nullptr, n, d_idx, d_mask, as);
    } else if (op == ASH_OP_ACTIVATE) {
      err = ash_activate(m, reinterpret_cast<const int32_t*>(dev), n, d_idx, d_mask, as);
    } else if (op == ASH_OP_FIND) {
      err = ash_find(m, reinterpret_cast<const int32_t*>(dev), n, d_idx, d_mask, as);
    } else {
      err = ash_erase(m, reinterpret_cast<const int32_t*>(dev), n, d_mask, as);
    }
    if (err != ASH_OK) break;
    if (op != ASH_OP_ERASE) cudaMemcpyAsync(host_out, d_idx, n * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(host_out + 4 * n_max, d_mask, n, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      err = cuda_fail(cudaGetLastError(), "replay_sequential");
      break;
    }
    last = Clock::now();
    latency_ms_host[r] = ms_between(due, last);
  }
  cudaStreamSynchronize(st);
  for (int i = 0; i < n_maps; ++i) maps[i]->last_stream = prev_stream[static_cast<size_t>(i)];
  cudaFree(dev);
  cudaFreeHost(host_out);
  cudaStreamDestroy(st);
  *span_s_host = std::chrono::duration<double>(last - t0).count();
  return err;
}

}  // extern "C"
