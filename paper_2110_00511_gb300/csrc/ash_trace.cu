// Kernel launch counting and optional per-kernel CUDA-event timing.
//
// Every launcher of the library opens a TraceScope around its kernel launch.
// The scope always counts the launch; when tracing is on it also records a
// CUDA event before and after the launch on the launching stream.  Collecting
// waits for the recorded events and accumulates the elapsed time per kernel
// kind.  Used for measurement (the per-kernel roofline figures), never by the
// map logic itself.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ash.h"
#include "ash_trace.h"

namespace ash {
namespace {

std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_launches_by[kKernelKinds];
std::atomic<int> g_on{0};
std::mutex g_mu;

struct Rec {
  int kind;
  cudaEvent_t start;
  cudaEvent_t stop;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
double g_ms[kKernelKinds] = {};
long long g_count[kKernelKinds] = {};

const char* const kNames[kKernelKinds] = {
    "find", "insert_claim", "insert_commit", "erase_mark", "erase_resolve", "rebuild", "list_active",
    "heap_iota", "scatter_rows", "gather_rows", "gather_keys", "quantize", "probe_random_read", "set_ctrl",
    "batch_graph", "synth_keys", "find_neighbors", "gather_values", "depth_to_block_keys", "compact_new_keys",
    "tsdf_integrate", "tsdf_raycast", "tsdf_ray_range", "partition_keys", "unpermute_outputs"};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

TraceScope::TraceScope(int kind, cudaStream_t stream, int launches) : kind_(kind), stream_(stream), rec_(-1) {
  g_launches.fetch_add(static_cast<unsigned long long>(launches), std::memory_order_relaxed);
  if (kind >= 0 && kind < kKernelKinds)
    g_launches_by[kind].fetch_add(static_cast<unsigned long long>(launches), std::memory_order_relaxed);
  if (g_on.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{kind, take_event(), take_event()};
    if (r.start && r.stop) {
      cudaEventRecord(r.start, stream);
      g_recs.push_back(r);
      rec_ = static_cast<int>(g_recs.size()) - 1;
    }
  }
}

TraceScope::~TraceScope() {
  if (rec_ >= 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (rec_ < static_cast<int>(g_recs.size())) cudaEventRecord(g_recs[rec_].stop, stream_);
  }
}

}  // namespace ash

extern "C" {

int ash_trace_kernel_kinds(void) { return ash::kKernelKinds; }

const char* ash_trace_kernel_name(int kind) {
  if (kind < 0 || kind >= ash::kKernelKinds) return "";
  return ash::kNames[kind];
}

ash_status ash_trace_enable(int on) {
  ash::g_on.store(on ? 1 : 0);
  return ASH_OK;
}

ash_status ash_trace_collect(void) {
  std::lock_guard<std::mutex> lk(ash::g_mu);
  for (auto& r : ash::g_recs) {
    if (cudaEventSynchronize(r.stop) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      ash::g_ms[r.kind] += ms;
      ash::g_count[r.kind] += 1;
    } else {
      cudaGetLastError();
    }
    ash::g_pool.push_back(r.start);
    ash::g_pool.push_back(r.stop);
  }
  ash::g_recs.clear();
  return ASH_OK;
}

ash_status ash_trace_read(int kind, double* total_ms_host, int64_t* launches_host) {
  if (kind < 0 || kind >= ash::kKernelKinds) return ASH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ash::g_mu);
  if (total_ms_host) *total_ms_host = ash::g_ms[kind];
  if (launches_host) *launches_host = ash::g_count[kind];
  return ASH_OK;
}

ash_status ash_trace_reset(void) {
  std::lock_guard<std::mutex> lk(ash::g_mu);
  for (int k = 0; k < ash::kKernelKinds; ++k) {
    ash::g_ms[k] = 0.0;
    ash::g_count[k] = 0;
  }
  return ASH_OK;
}

uint64_t ash_kernel_launch_count(void) { return ash::g_launches.load(); }

}  // extern "C"
