// Host-side launchers of the dimension-independent kernels (ash_aux.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ash_device.cuh"

namespace ash {

struct Launch;

// Lists live buffer indices in ascending order (the complement of the free
// part of the heap).  scratch: list_scratch_bytes(capacity) bytes of device
// memory.  Writes at most out_cap indices; the live count goes to ctrl->count.
int64_t list_scratch_bytes(int64_t capacity);
// count_out (optional): device int64 receiving the live count.  The scratch
// bitmap must be zero on entry; the listing leaves it zero.  heap_identity:
// the heap's free part is h[j] = j (no erase since create, clear or a
// compacting rehash), so the live indices are 0..t-1 and are written directly.
void launch_list_active(bool heap_identity, const int32_t* heap, int64_t capacity, Ctrl* ctrl, void* scratch,
                        int32_t* out, int64_t out_cap, long long* count_out, const Launch& L);
void launch_set_top_used(Ctrl* ctrl, int64_t top, int64_t used, const Launch& L);
void launch_set_used_from_count(Ctrl* ctrl, const Launch& L);
// L2 prefetch of a byte range (a hint; plain stream order, no programmatic
// overlap, so it never runs beside the kernel before it).
void launch_prefetch_l2(const void* base, int64_t bytes, const Launch& L);
// Publishes the control block to a host-visible snapshot (publish_snapshot).
void launch_snapshot(Ctrl* ctrl, Snap* snap, uint32_t seq, const Launch& L);
void launch_iota(int32_t* h, int64_t from, int64_t to, const Launch& L);
void launch_scatter_rows(const ValueCopy& vc, const int32_t* idx, const uint8_t* mask, int64_t n, const Launch& L);
void launch_gather_rows(const ValueCopy& vc, const int32_t* list, int64_t n, const Launch& L);
void launch_gather_keys(const int32_t* kb, int ks, int d, int64_t capacity, const int32_t* indices, int64_t n,
                        const long long* n_dev, int32_t* out, const Launch& L);
void launch_gather_values(const void* src, int64_t row_bytes, int vec, int64_t capacity, const int32_t* indices,
                          int64_t n, const long long* n_dev, void* out, const Launch& L);
void launch_quantize(const float* pts, int64_t n, float cell, int32_t* keys, const Launch& L);
void launch_probe_atomic(void* buf, int64_t buf_bytes, int64_t n_ops, int mode, uint32_t seed, uint32_t* sink,
                         int64_t sink_len, const Launch& L);
void launch_probe(const void* buf, int64_t buf_bytes, int64_t n_reads, int sector, int loads_per_thread,
                  uint32_t seed, uint32_t* sink, int64_t sink_len, const Launch& L);

}  // namespace ash
