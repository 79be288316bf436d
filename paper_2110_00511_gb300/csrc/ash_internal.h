// Internal host-side view of a map, shared by the translation units of the
// library (map operations, batched execution, tuning, serving).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ash.h"
#include "ash_kernels.cuh"

namespace ash {
namespace host {

struct Allocator {
  ash_alloc_fn alloc = nullptr;
  ash_free_fn free = nullptr;
  void* ctx = nullptr;
};

}  // namespace host
}  // namespace ash

struct ash_map {
  int device = 0;
  int key_dim = 0;
  int ks = 0;  // key stride in kB
  int n_values = 0;
  int64_t capacity = 0;
  int64_t n_slots = 0;
  uint32_t n_buckets = 0;
  int S = 4;
  std::vector<int64_t> numel;
  std::vector<int32_t> dtype;
  std::vector<int64_t> row_bytes;
  uint64_t* slots = nullptr;
  int32_t* kb = nullptr;
  int32_t* heap = nullptr;
  std::vector<void*> vb;
  ash::Ctrl* ctrl = nullptr;
  ash::Ctrl* ctrl_host = nullptr;  // pinned mirror for synchronising reads
  int32_t* scratch = nullptr;      // erase: one slot index per key
  int64_t scratch_bytes = 0;
  uint32_t* win_bits = nullptr;    // insert: winner flags, one bit per key
  int64_t win_bits_bytes = 0;
  bool win_bits_clean = true;      // every winner flag is clear (the commit clears what it read)
  void* list_scratch = nullptr;    // listing: free-index bitmap + block counts
  int64_t list_scratch_bytes = 0;
  int64_t size_ub = 0;  // upper bound of live entries since the last sync
  int64_t used_ub = 0;  // upper bound of used slots since the last sync
  // Non-blocking snapshot of the control block: written by the device to
  // snap_host (mapped pinned memory, snap_dev on the device) after a batch
  // once the bounds pass half the limits, and read once its sequence number
  // shows snap_seq, to tighten the bounds without synchronising.
  ash::Snap* snap_host = nullptr;
  ash::Snap* snap_dev = nullptr;
  uint32_t snap_seq = 0;           // number of the last snapshot requested
  int snap_state = 0;              // 0 idle, 1 in flight, 2 in flight but stale
  int64_t added_since_snap = 0;    // insert/activate keys issued after the snapshot's copy
  // Lower bound on tombstones (used - live of the last landed snapshot):
  // inserts never reuse a tombstone, so the count only grows until a rebuild
  // (which resets it).  Drives the clean-up rebuilds (tombstones_need_rebuild).
  int64_t tomb_lb = 0;
  int64_t erased_since_snap = 0;   // erase keys issued after the last snapshot (tombstones may have formed)
  // Snapshots are taken only while every insert/activate of the map has come
  // on one stream (then stream order makes "snapshot + keys issued since" an
  // upper bound); a second stream turns them off for the map's life.
  cudaStream_t insert_stream = nullptr;
  bool insert_streams_mixed = false;
  bool any_insert = false;
  // Every key of the table sits in its preferred slot or that slot is
  // occupied (the preferred-slot invariant), so an insert may CAS the
  // preferred slot blindly.  Set by create, clear and every table rebuild;
  // cleared by batched inserts, which place keys in slot order.
  bool pref_placed = true;
  // The free part of the heap is the identity (h[j] = j for j >= t), so the
  // live indices are exactly 0..t-1: true from create, clear or a compacting
  // rehash until the first erase (growth keeps it).  Commit skips the heap
  // read and the listing writes 0..t-1.
  bool heap_identity = true;
  int64_t host_syncs = 0;          // growth checks that synchronised a stream (refresh)
  int64_t rebuilds = 0;            // table rebuilds (rebuild_to, grow_async)
  ash_tuning tuning{};
  ash::DimKernels K{};
  ash::host::Allocator alloc;
  cudaStream_t last_stream = nullptr;
};

namespace ash {
namespace host {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

ash_status fail(ash_status s, const std::string& msg);
ash_status cuda_fail(cudaError_t e, const char* where);
ash_status check_launch(const char* where);
int sm_count(int device);
int64_t l2_bytes(int device);
int vec_width(int64_t row_bytes, const void* a, const void* b);
void* dev_alloc(ash_map* m, size_t bytes, cudaStream_t st);
void dev_free(ash_map* m, void* p, cudaStream_t st);
Launch launch_of(const ash_map* m, cudaStream_t st);
TableView view_of(const ash_map* m);
ash_status check_keys(const ash_map* m, const void* keys, int64_t n);
// x2 growth / table rebuild so that a batch of n insert keys fits (may synchronise st).
ash_status ensure_room(ash_map* m, int64_t n, cudaStream_t st);
// Growth to new_capacity >= capacity, enqueued on st with no host synchronisation.
ash_status grow_async(ash_map* m, int64_t new_capacity, cudaStream_t st);
// Tightens size_ub / used_ub from a completed control-block snapshot (never blocks).
void tighten_bounds(ash_map* m);
// Marks an in-flight snapshot stale (after clear / rebuild change the count).
void invalidate_snapshot(ash_map* m);
// Whether to snapshot the control block after the batch being issued on st
// (`added` insert keys not yet on the bounds): once a bound passes half its
// limit, or after erases on a table of some size.  True takes the next
// sequence number (m->snap_seq); the caller has the device publish it and
// then calls snapshot_issued.
bool snapshot_wanted(ash_map* m, cudaStream_t st, int64_t added);
void snapshot_issued(ash_map* m);
// snapshot_wanted(m, st, 0), published by snapshot_kernel.
void maybe_snapshot(ash_map* m, cudaStream_t st);
// Records the stream of an insert/activate (snapshots need a single one).
void note_insert_stream(ash_map* m, cudaStream_t st);
// True when the map's known tombstones call for a table rebuild.
bool tombstones_need_rebuild(const ash_map* m);
// Key dimension, value row bytes and tenant count of a server.
void server_layout(const ash_server* s, int* key_dim, int* value_row_bytes, int* n_tenants);

}  // namespace host
}  // namespace ash
