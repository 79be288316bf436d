// Autotuner for the layout and launch knobs of a map.
//
// For a (key dimension, capacity, uniqueness) class it builds maps with each
// candidate tuning, activates and finds the same synthetic keys, times the two
// operations with CUDA events, and keeps the fastest candidate.  Synthetic
// keys are generated on the device: row r is derived from (r mod U), U =
// rho * n, with a splitmix64 mix, so a fraction rho of the rows is distinct.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "ash.h"
#include "ash_internal.h"
#include "ash_trace.h"

namespace ash {

__global__ void synth_keys_kernel(int32_t* __restrict__ keys, int64_t n, int d, int64_t distinct, uint64_t seed) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    const uint64_t id = static_cast<uint64_t>(r % distinct);
    for (int c = 0; c < d; ++c) {
      const uint64_t x = mix64(seed + id * 8u + static_cast<uint64_t>(c) + 1u);
      keys[r * d + c] = static_cast<int32_t>(static_cast<uint32_t>(x >> 40)) - (1 << 23);  // 24-bit coordinates
    }
  }
}

}  // namespace ash

using namespace ash;
using namespace ash::host;

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, ash_tuning> g_tune_cache;

}  // namespace

extern "C" ash_status ash_autotune(int key_dim, int64_t capacity, float rho, int device, ash_stream stream,
                                   ash_tuning* out_host) {
  if (!out_host) return fail(ASH_ERR_INVALID, "out is NULL");
  if (key_dim < 1 || key_dim > 8 || capacity < 1) return fail(ASH_ERR_INVALID, "bad key_dim or capacity");
  if (!(rho > 0.0f && rho <= 1.0f)) return fail(ASH_ERR_INVALID, "rho must be in (0, 1]");
  const int cap_class = static_cast<int>(std::ceil(std::log2(static_cast<double>(capacity))));
  const int rho_class = static_cast<int>(std::lround(rho * 10.0f));
  const auto key = std::make_tuple(device, key_dim, cap_class, rho_class);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out_host = it->second;
      return ASH_OK;
    }
  }
  DeviceGuard g(device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = std::min<int64_t>(capacity, int64_t{1} << 20);
  const int64_t distinct = std::max<int64_t>(1, static_cast<int64_t>(rho * static_cast<double>(n)));
  int32_t* keys = nullptr;
  int32_t* idx = nullptr;
  uint8_t* mask = nullptr;
  if (cudaMallocAsync(&keys, n * key_dim * 4, st) != cudaSuccess || cudaMallocAsync(&idx, n * 4, st) != cudaSuccess ||
      cudaMallocAsync(&mask, n, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(ASH_ERR_OOM, "autotune buffers");
  }
  {
    TraceScope ts(kKSynthKeys, st);
    synth_keys_kernel<<<sm_count(device) * 4, 256, 0, st>>>(keys, n, key_dim, distinct, 0x5EEDull + cap_class);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ash_tuning best{};
  float best_ms = 1e30f;
  ash_status status = ASH_OK;
  const int buckets[3] = {4, 8, 16};
  const float spcs[3] = {1.5f, 2.0f, 3.0f};
  // (keys per thread, find keys per thread, warp-cooperative find):
  // thread-per-key variants, and warp-cooperative probing
  const int modes[4][3] = {{1, 1, 0}, {2, 1, 0}, {2, 2, 0}, {2, 1, 1}};
  for (int S : buckets) {
    for (float spc : spcs) {
      for (const auto& md : modes) {
        ash_tuning t;
        ash_default_tuning(&t);
        t.slots_per_bucket = S;
        t.slots_per_capacity = spc;
        t.keys_per_thread = md[0];
        t.find_keys_per_thread = md[1];
        t.warp_probe = md[2];
        float total = 0.0f;
        for (int rep = 0; rep < 2 && status == ASH_OK; ++rep) {
          ash_map* m = nullptr;
          status = ash_create(key_dim, capacity, 0, nullptr, nullptr, device, &t, stream, &m);
          if (status != ASH_OK) break;
          cudaEventRecord(e0, st);
          status = ash_activate(m, keys, n, idx, mask, stream);
          if (status == ASH_OK) status = ash_find(m, keys, n, idx, mask, stream);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep == 1) total = ms;  // second run: warm code and pool
          ash_destroy(m);
        }
        if (status != ASH_OK) break;
        if (total < best_ms) {
          best_ms = total;
          best = t;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(keys, st);
  cudaFreeAsync(idx, st);
  cudaFreeAsync(mask, st);
  cudaStreamSynchronize(st);
  if (status != ASH_OK) return status;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  *out_host = best;
  return ASH_OK;
}
