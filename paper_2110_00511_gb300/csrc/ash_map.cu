// Host side of the hash map and the C ABI declared in include/ash.h.
//
// The map object owns the table, the key buffer kB, the value buffers vB_j,
// the index heap h and a small control block (heap top t, used slots, error
// bits) in device memory.  Every operation is a short sequence of kernel
// launches on the caller's stream; the host synchronises only where the
// answer is needed on the host (size, listing, rehash) or when the host-side
// upper bounds on the live and used counts say that the batch might not fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ash.h"
#include "ash_aux.h"
#include "ash_internal.h"
#include "ash_kernels.cuh"

namespace ash {
namespace host {

thread_local std::string g_last_error;

ash_status fail(ash_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ash_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ASH_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ASH_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)



std::mutex g_mu;
Allocator g_alloc;
bool g_pool_ready[64] = {};

// Pinned host mirrors of the maps' control blocks come from pinned pages
// allocated once and recycled, so creating and destroying maps does not pay
// for cudaMallocHost / cudaFreeHost each time.
std::mutex g_pin_mu;
std::vector<ash::Ctrl*> g_pin_free;

ash::Ctrl* pinned_ctrl_take() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr int kPerPage = 128;
    void* page = nullptr;
    if (cudaMallocHost(&page, sizeof(ash::Ctrl) * kPerPage) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = kPerPage - 1; i >= 0; --i) g_pin_free.push_back(static_cast<ash::Ctrl*>(page) + i);
  }
  ash::Ctrl* c = g_pin_free.back();
  g_pin_free.pop_back();
  return c;
}

void pinned_ctrl_give(ash::Ctrl* c) {
  if (!c) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(c);
}

// Snapshot records: mapped pinned memory that kernels write.  seq is the
// last number given to the record.  A record given back while its last
// snapshot may still land waits in g_snap_wait until that write shows.
struct SnapRec {
  ash::Snap* host;
  ash::Snap* dev;
  uint32_t seq;
};
std::vector<SnapRec> g_snap_free;
std::vector<SnapRec> g_snap_wait;

// The record's top_used if snapshot number seq has landed in it.
bool snap_read(const ash::Snap* s, uint32_t seq, unsigned long long* top_used) {
  const unsigned long long tu = __atomic_load_n(&s->top_used, __ATOMIC_ACQUIRE);
  const unsigned long long check = __atomic_load_n(&s->check, __ATOMIC_ACQUIRE);
  if ((tu ^ check) != ash::snap_tag(seq)) return false;
  *top_used = tu;
  return true;
}

bool snap_take(SnapRec* out) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  for (size_t i = 0; i < g_snap_wait.size();) {
    unsigned long long tu;
    if (snap_read(g_snap_wait[i].host, g_snap_wait[i].seq, &tu)) {
      g_snap_free.push_back(g_snap_wait[i]);
      g_snap_wait[i] = g_snap_wait.back();
      g_snap_wait.pop_back();
    } else {
      ++i;
    }
  }
  if (g_snap_free.empty()) {
    constexpr int kPerPage = 128;
    void* page = nullptr;
    void* dpage = nullptr;
    if (cudaHostAlloc(&page, sizeof(ash::Snap) * kPerPage, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaHostGetDevicePointer(&dpage, page, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(page);
      return false;
    }
    std::memset(page, 0, sizeof(ash::Snap) * kPerPage);
    for (int i = kPerPage - 1; i >= 0; --i)
      g_snap_free.push_back({static_cast<ash::Snap*>(page) + i, static_cast<ash::Snap*>(dpage) + i, 0u});
  }
  *out = g_snap_free.back();
  g_snap_free.pop_back();
  return true;
}

// pending: snapshot number r.seq was requested and may not have landed.
void snap_give(const SnapRec& r, bool pending) {
  if (!r.host) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  unsigned long long tu;
  if (pending && !snap_read(r.host, r.seq, &tu)) g_snap_wait.push_back(r);
  else g_snap_free.push_back(r);
}

int64_t dtype_bytes(int32_t dt) {
  switch (dt) {
    case ASH_F32: case ASH_I32: return 4;
    case ASH_F16: case ASH_BF16: return 2;
    case ASH_I64: case ASH_F64: return 8;
    case ASH_U8: return 1;
    default: return 0;
  }
}

int64_t l2_bytes(int device) {
  static int64_t cache[64] = {};
  if (device < 0 || device >= 64) return 0;
  if (cache[device] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device);
    cache[device] = v > 0 ? v : 1;
  }
  return cache[device];
}

int sm_count(int device) {
  static int cache[64] = {};
  if (device < 0 || device >= 64) return 1;
  if (cache[device] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    cache[device] = v > 0 ? v : 1;
  }
  return cache[device];
}



int vec_width(int64_t row_bytes, const void* a, const void* b) {
  const uintptr_t al = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b);
  for (int v : {16, 8, 4, 2}) {
    if (row_bytes % v == 0 && (al % v) == 0) return v;
  }
  return 1;
}


void* dev_alloc(ash_map* m, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 256;
  if (m->alloc.alloc) return m->alloc.alloc(bytes, m->device, reinterpret_cast<ash_stream>(st), m->alloc.ctx);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (m->device >= 0 && m->device < 64 && !g_pool_ready[m->device]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, m->device) == cudaSuccess) {
        uint64_t keep = ~0ull;  // cache freed blocks in this process's pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      g_pool_ready[m->device] = true;
    }
  }
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(ash_map* m, void* p, cudaStream_t st) {
  if (!p) return;
  if (m->alloc.free) {
    m->alloc.free(p, m->device, reinterpret_cast<ash_stream>(st), m->alloc.ctx);
    return;
  }
  cudaFreeAsync(p, st);
}

ash::DimKernels kernels_for(int d) {
  switch (d) {
    case 1: return ash::dim_kernels_1();
    case 2: return ash::dim_kernels_2();
    case 3: return ash::dim_kernels_3();
    case 4: return ash::dim_kernels_4();
    case 5: return ash::dim_kernels_5();
    case 6: return ash::dim_kernels_6();
    case 7: return ash::dim_kernels_7();
    default: return ash::dim_kernels_8();
  }
}

// Claim protocol of an insert: the preferred-slot CAS first while the table
// takes at most two thirds of L2 (a CAS that misses L2 waits on DRAM in the
// atomic unit), else the bucket load first.  On GB300 (L2 135.5 MB) the
// preferred-slot path is 6-25 % faster up to 80 MB tables, even at 96 MB and
// 19 % slower at 128 MB.  It needs the preferred-slot invariant, which a
// bucket-first or batched insert gives up until the next clear or rebuild.
// The preferred-slot claim pays off while the table is in L2: its CAS has
// no load before it, and a CAS that misses L2 waits on DRAM in the atomic
// unit.  (Keys in home-bucket range order do not change this: a range's
// lines are not in L2 when its keys arrive, and the bucket-first claim ran
// 3.6 against 5.1 ms on 10^8 ranged keys.)
int claim_prefers_slot(const ash_map* m) {
  if (m->tuning.claim_mode == 1 || !m->pref_placed) return 0;
  if (m->tuning.claim_mode == 2) return 1;
  return m->n_slots * 8 * 3 <= l2_bytes(m->device) * 2 ? 1 : 0;
}

// log2 of the number of home-bucket ranges a call on n keys is partitioned
// into, 0 for input order (tuning.partition_keys): 2 to 256 ranges of at
// most L2/2 bytes of table (8 at least when forced).  By default, calls of
// 2^20 keys or more on a table larger than twice L2.  The pay-off needs
// both sides: a ranged find reads kB in range order only if the inserts
// handed out indices in the same ranges.  Measured on GB300 (uniform keys,
// uniqueness 0.5, capacity n, queries in a fresh random order), ranged
// against input order: at 10^8 keys activate 5.6 / 7.9 ms and find 3.1 /
// 5.1 ms; at 2x10^7 activate 1.12 / 1.23 ms and find 0.58 / 0.80 ms.  Before
// the calls worked range by range (one launch over all ranged keys), a
// ranged activate of 10^7 keys (table 1.2x L2) took 0.59 against 0.53 ms,
// and ranges of L2/4 ran level with L2/2 at 10^8.
int partition_log(const ash_map* m, int64_t n) {
  const int mode = m->tuning.partition_keys;
  if (mode == 1 || n <= 0) return 0;
  const int64_t table = m->n_slots * 8;
  const int64_t l2 = l2_bytes(m->device);
  if (mode == 0 && (table <= 2 * l2 || n < (int64_t{1} << 20))) return 0;
  int lg = 1;
  while (lg < ash::kPartMaxLog && (table >> lg) > l2 / 2) ++lg;
  return mode == 2 ? std::max(lg, 3) : lg;
}

// Stream-ordered scratch of one partitioned call, freed on the same stream
// after its last kernel (concurrent finds on one map each have their own).
struct PartBufs {
  void* mem = nullptr;
  int32_t* keys = nullptr;  // key rows in range order
  int32_t* dest = nullptr;  // place of input row pos in that order
  int32_t* idx = nullptr;   // outputs in range order
  uint8_t* mask = nullptr;
};

// False (nothing enqueued) when the scratch cannot be had: the call then
// uses its keys in input order.
bool partition_call(ash_map* m, const int32_t* keys, int64_t n, int log_p, cudaStream_t st, PartBufs* pb) {
  auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t words = up(ash::partition_count_words(n, log_p, launch_of(m, st)) * 4);
  const int64_t rows = up(n * m->key_dim * 4);
  const int64_t ints = up(n * 4);
  char* base = static_cast<char*>(dev_alloc(m, words + rows + 2 * ints + up(n), st));
  if (!base) {
    cudaGetLastError();
    return false;
  }
  pb->mem = base;
  pb->keys = reinterpret_cast<int32_t*>(base + words);
  pb->dest = reinterpret_cast<int32_t*>(base + words + rows);
  pb->idx = reinterpret_cast<int32_t*>(base + words + rows + ints);
  pb->mask = reinterpret_cast<uint8_t*>(base + words + rows + 2 * ints);
  m->K.partition(keys, n, log_p, reinterpret_cast<uint32_t*>(base), pb->keys, pb->dest, launch_of(m, st));
  return true;
}

// The table buckets of range p of P (and a bucket past it, for probes
// that run on), asked into L2 before the range's keys are worked on.
void prefetch_table_range(const ash_map* m, int p, int P, const ash::Launch& L) {
  const int64_t b0 = static_cast<int64_t>(m->n_buckets) * p / P;
  int64_t b1 = static_cast<int64_t>(m->n_buckets) * (p + 1) / P + 1;
  if (b1 > m->n_buckets) b1 = m->n_buckets;
  ash::launch_prefetch_l2(m->slots + b0 * m->S, (b1 - b0) * m->S * 8, L);
}

// The partitioned call's outputs back in input order; its scratch freed.
void partition_finish(ash_map* m, const PartBufs& pb, int64_t n, int32_t* idx, uint8_t* mask, cudaStream_t st) {
  ash::launch_unpermute(pb.dest, n, pb.idx, pb.mask, idx, mask, launch_of(m, st));
  dev_free(m, pb.mem, st);
}

ash::Launch launch_of(const ash_map* m, cudaStream_t st) {
  ash::Launch L;
  L.stream = st;
  L.block = m->tuning.block_threads;
  L.grid_cap = sm_count(m->device) * m->tuning.blocks_per_sm;
  L.sms = sm_count(m->device);
  return L;
}

ash::TableView view_of(const ash_map* m) {
  ash::TableView t;
  t.slots = m->slots;
  t.kb = m->kb;
  t.heap = m->heap;
  t.ctrl = m->ctrl;
  t.n_buckets = m->n_buckets;
  t.max_probes = (m->tuning.max_probes > 0 && static_cast<uint32_t>(m->tuning.max_probes) < m->n_buckets)
                     ? static_cast<uint32_t>(m->tuning.max_probes)
                     : m->n_buckets;
  t.capacity = static_cast<int32_t>(m->capacity);
  t.flags = (m->heap_identity ? ash::kViewHeapIdentity : 0) | (m->pref_placed ? ash::kViewPrefPlaced : 0);
  t.lost = nullptr;
  t.snap = nullptr;
  t.snap_seq = 0;
  return t;
}

ash_status validate_tuning(const ash_tuning& t) {
  if (t.slots_per_bucket != 4 && t.slots_per_bucket != 8 && t.slots_per_bucket != 16)
    return fail(ASH_ERR_INVALID, "slots_per_bucket must be 4, 8 or 16");
  if (!(t.slots_per_capacity >= 1.05f && t.slots_per_capacity <= 64.0f))
    return fail(ASH_ERR_INVALID, "slots_per_capacity must be in [1.05, 64]");
  if (t.block_threads < 32 || t.block_threads > 256 || t.block_threads % 32 != 0)
    return fail(ASH_ERR_INVALID, "block_threads must be a multiple of 32 in [32, 256]");
  if (t.blocks_per_sm < 1 || t.blocks_per_sm > 64) return fail(ASH_ERR_INVALID, "blocks_per_sm must be in [1, 64]");
  if (t.max_probes < 0) return fail(ASH_ERR_INVALID, "max_probes must be >= 0");
  if (!(t.max_used_fraction > 0.1f && t.max_used_fraction < 0.99f))
    return fail(ASH_ERR_INVALID, "max_used_fraction must be in (0.1, 0.99)");
  if (t.inline_value_bytes < 0) return fail(ASH_ERR_INVALID, "inline_value_bytes must be >= 0");
  if (t.keys_per_thread != 1 && t.keys_per_thread != 2 && t.keys_per_thread != 4)
    return fail(ASH_ERR_INVALID, "keys_per_thread must be 1, 2 or 4");
  if (t.warp_probe != 0 && t.warp_probe != 1) return fail(ASH_ERR_INVALID, "warp_probe must be 0 or 1");
  if (t.find_keys_per_thread != 0 && t.find_keys_per_thread != 1 && t.find_keys_per_thread != 2 &&
      t.find_keys_per_thread != 4)
    return fail(ASH_ERR_INVALID, "find_keys_per_thread must be 0, 1, 2 or 4");
  if (t.claim_mode < 0 || t.claim_mode > 2) return fail(ASH_ERR_INVALID, "claim_mode must be 0, 1 or 2");
  if (t.commit_keys_per_thread != 0 && t.commit_keys_per_thread != 1 && t.commit_keys_per_thread != 2 &&
      t.commit_keys_per_thread != 4)
    return fail(ASH_ERR_INVALID, "commit_keys_per_thread must be 0, 1, 2 or 4");
  if (t.partition_keys < 0 || t.partition_keys > 2) return fail(ASH_ERR_INVALID, "partition_keys must be 0, 1 or 2");
  return ASH_OK;
}

int64_t slots_for(int64_t capacity, const ash_tuning& t) {
  const int S = t.slots_per_bucket;
  int64_t n = static_cast<int64_t>(std::ceil(static_cast<double>(capacity) * t.slots_per_capacity));
  n = std::max<int64_t>(n, capacity + 1);
  n = (n + S - 1) / S * S;
  return n;
}

// Reads the control block (synchronises `st`).
ash_status refresh(ash_map* m, cudaStream_t st, int64_t* top, int64_t* used, int* status) {
  __atomic_fetch_add(&m->host_syncs, 1, __ATOMIC_RELAXED);  // read by other threads as a statistic
  ASH_CUDA(cudaMemcpyAsync(m->ctrl_host, m->ctrl, sizeof(ash::Ctrl), cudaMemcpyDeviceToHost, st));
  ASH_CUDA(cudaStreamSynchronize(st));
  const unsigned long long tu = m->ctrl_host->top_used;
  *top = static_cast<int64_t>(tu & 0xFFFFFFFFull);
  *used = static_cast<int64_t>(tu >> 32);
  if (status) *status = m->ctrl_host->status;
  m->size_ub = *top;
  m->used_ub = *used;
  tighten_bounds(m);  // folds in a snapshot that has landed
  m->size_ub = *top;
  m->used_ub = *used;
  if (*used - *top > m->tomb_lb) m->tomb_lb = *used - *top;  // exact now
  return ASH_OK;
}

void tighten_bounds(ash_map* m) {
  unsigned long long tu = 0;
  if (m->snap_state == 0 || !snap_read(m->snap_host, m->snap_seq, &tu)) return;
  if (m->snap_state == 1) {
    const int64_t snap_top = static_cast<int64_t>(tu & 0xFFFFFFFFull);
    const int64_t snap_used = static_cast<int64_t>(tu >> 32);
    const int64_t top = snap_top + m->added_since_snap;
    const int64_t used = snap_used + m->added_since_snap;
    if (top < m->size_ub) m->size_ub = top;
    if (used < m->used_ub) m->used_ub = used;
    if (snap_used - snap_top > m->tomb_lb) m->tomb_lb = snap_used - snap_top;
  }
  m->snap_state = 0;
}

// Erased slots whose bucket has no EMPTY slot stay tombstones, and inserts
// claim only EMPTY slots, so under insert/erase churn the runs of full
// buckets lengthen: measured on a 2^24-capacity map, a find of 1M keys took
// 3x as long as on a rebuilt table with tombstones at 0.3 of the live count,
// 14x at 1.3 and 27x at 2.0, with the used slots (0.29-0.55 of the table)
// still below max_used_fraction.  A table whose known tombstones pass a
// quarter of its live entries (and 1/64 of its slots) is rebuilt.
bool tombstones_need_rebuild(const ash_map* m) {
  const int64_t live = m->size_ub;
  return m->tomb_lb > m->n_slots / 64 && 4 * m->tomb_lb > live;
}

void invalidate_snapshot(ash_map* m) {
  if (m->snap_state == 1) m->snap_state = 2;
}

void note_insert_stream(ash_map* m, cudaStream_t st) {
  if (m->any_insert && m->insert_stream != st) m->insert_streams_mixed = true;
  m->insert_stream = st;
  m->any_insert = true;
}

// Snapshots are taken once a bound passes half its limit, so that a later
// growth check can tighten it without a synchronisation, and after erases on
// a table of some size (the tombstone count).  One is in flight at a time.
bool snapshot_wanted(ash_map* m, cudaStream_t st, int64_t added) {
  // a snapshot that has landed is folded into the bounds first, so a fresh
  // one can be taken: the bounds then lag the device by the batches issued
  // since the last snapshot landed, not since the first one was taken
  if (m->snap_state != 0) tighten_bounds(m);
  if (m->snap_state != 0 || !m->snap_host || m->insert_streams_mixed || st != m->insert_stream) return false;
  const int64_t max_used = static_cast<int64_t>(m->tuning.max_used_fraction * static_cast<double>(m->n_slots));
  const bool churn = m->erased_since_snap > 0 && m->n_slots >= (int64_t{1} << 16);
  if (2 * (m->size_ub + added) <= m->capacity && 2 * (m->used_ub + added) <= max_used && !churn) return false;
  // Never inside a stream capture: a replayed graph would write the pinned
  // record long after this map (and its record) are gone.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cs != cudaStreamCaptureStatusNone) return false;
  ++m->snap_seq;
  return true;
}

// The snapshot numbered m->snap_seq follows every batch issued so far.
void snapshot_issued(ash_map* m) {
  m->snap_state = 1;
  m->added_since_snap = 0;
  m->erased_since_snap = 0;
}

void maybe_snapshot(ash_map* m, cudaStream_t st) {
  if (!snapshot_wanted(m, st, 0)) return;
  ash::launch_snapshot(m->ctrl, m->snap_dev, m->snap_seq, launch_of(m, st));
  snapshot_issued(m);
}

ash_status status_from_bits(int bits) {
  if (bits & ash::kStatusTableFull) return fail(ASH_ERR_TABLE_FULL, "a key found no free slot within max_probes buckets");
  if (bits & ash::kStatusCapacity) return fail(ASH_ERR_CAPACITY, "the index heap ran out (capacity exceeded)");
  return ASH_OK;
}

ash_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, where);
  return ASH_OK;
}

// Allocates and initialises table, buffers and heap for `capacity`.
ash_status alloc_storage(ash_map* m, int64_t capacity, cudaStream_t st) {
  const int64_t n_slots = slots_for(capacity, m->tuning);
  if (n_slots >= (int64_t{1} << 31)) return fail(ASH_ERR_INVALID, "capacity too large for 31-bit slot indices");
  const ash::Launch L = launch_of(m, st);
  m->slots = static_cast<uint64_t*>(dev_alloc(m, n_slots * 8, st));
  m->kb = static_cast<int32_t*>(dev_alloc(m, capacity * m->ks * 4, st));
  m->heap = static_cast<int32_t*>(dev_alloc(m, capacity * 4, st));
  m->vb.assign(m->n_values, nullptr);
  bool ok = m->slots && m->kb && m->heap;
  for (int j = 0; j < m->n_values && ok; ++j) {
    m->vb[j] = dev_alloc(m, capacity * m->row_bytes[j], st);
    ok = m->vb[j] != nullptr;
  }
  if (!ok) return fail(ASH_ERR_OOM, "device allocation failed");
  m->capacity = capacity;
  m->n_slots = n_slots;
  m->S = m->tuning.slots_per_bucket;
  m->n_buckets = static_cast<uint32_t>(n_slots / m->S);
  m->pref_placed = true;
  m->heap_identity = true;
  ASH_CUDA(cudaMemsetAsync(m->slots, 0xFF, n_slots * 8, st));
  for (int j = 0; j < m->n_values; ++j) ASH_CUDA(cudaMemsetAsync(m->vb[j], 0, capacity * m->row_bytes[j], st));
  ash::launch_iota(m->heap, 0, capacity, L);
  return check_launch("alloc_storage");
}

void free_storage(ash_map* m, cudaStream_t st) {
  dev_free(m, m->slots, st);
  dev_free(m, m->kb, st);
  dev_free(m, m->heap, st);
  for (void* p : m->vb) dev_free(m, p, st);
  m->slots = nullptr;
  m->kb = nullptr;
  m->heap = nullptr;
  m->vb.assign(m->n_values, nullptr);
}

ash_status ensure_scratch(ash_map* m, int64_t bytes, cudaStream_t st) {
  if (m->scratch_bytes >= bytes) return ASH_OK;
  dev_free(m, m->scratch, st);
  const int64_t want = std::max<int64_t>(bytes, m->scratch_bytes * 2);
  m->scratch = static_cast<int32_t*>(dev_alloc(m, want, st));
  if (!m->scratch) {
    m->scratch_bytes = 0;
    return fail(ASH_ERR_OOM, "scratch allocation failed");
  }
  m->scratch_bytes = want;
  return ASH_OK;
}

// Winner flags of an insert of n keys: one bit per input position.
ash_status ensure_win_bits(ash_map* m, int64_t n, cudaStream_t st) {
  const int64_t bytes = (n + 31) / 32 * 4;
  if (m->win_bits_bytes >= bytes) return ASH_OK;
  dev_free(m, m->win_bits, st);
  const int64_t want = std::max<int64_t>(bytes, m->win_bits_bytes * 2);
  m->win_bits = static_cast<uint32_t*>(dev_alloc(m, want, st));
  if (!m->win_bits) {
    m->win_bits_bytes = 0;
    return fail(ASH_ERR_OOM, "winner-flag allocation failed");
  }
  m->win_bits_bytes = want;
  // all bits start clear; every insert's commit clears the words it read
  ASH_CUDA(cudaMemsetAsync(m->win_bits, 0, want, st));
  m->win_bits_clean = true;
  return ASH_OK;
}

ash_status ensure_list_scratch(ash_map* m, cudaStream_t st) {
  const int64_t need = ash::list_scratch_bytes(m->capacity);
  if (m->list_scratch_bytes >= need) return ASH_OK;
  dev_free(m, m->list_scratch, st);
  m->list_scratch = dev_alloc(m, need, st);
  if (!m->list_scratch) {
    m->list_scratch_bytes = 0;
    return fail(ASH_ERR_OOM, "listing scratch allocation failed");
  }
  m->list_scratch_bytes = need;
  ASH_CUDA(cudaMemsetAsync(m->list_scratch, 0, need, st));  // each listing leaves it zero again
  return ASH_OK;
}

// Rebuilds the table for new_capacity from the live entries (Sec. 4.5).
// size: the exact live count (caller synchronised).
ash_status rebuild_to(ash_map* m, int64_t new_capacity, int64_t size, cudaStream_t st) {
  __atomic_fetch_add(&m->rebuilds, 1, __ATOMIC_RELAXED);
  const ash::Launch L = launch_of(m, st);
  // 1) collect the active indices
  int32_t* list = static_cast<int32_t*>(dev_alloc(m, std::max<int64_t>(size, 1) * 4, st));
  if (!list) return fail(ASH_ERR_OOM, "rehash list allocation failed");
  ash_status s = ensure_list_scratch(m, st);
  if (s != ASH_OK) {
    dev_free(m, list, st);
    return s;
  }
  ash::launch_list_active(m->heap_identity, m->heap, m->capacity, m->ctrl, m->list_scratch, list, size, nullptr, L);
  s = check_launch("rehash listing");
  if (s != ASH_OK) return s;

  ash_map old = *m;  // shallow copy of the old storage pointers
  const bool preserve = new_capacity >= m->capacity;
  const int64_t n_slots = slots_for(new_capacity, m->tuning);
  if (n_slots >= (int64_t{1} << 31)) {
    dev_free(m, list, st);
    return fail(ASH_ERR_INVALID, "capacity too large for 31-bit slot indices");
  }
  uint64_t* slots = static_cast<uint64_t*>(dev_alloc(m, n_slots * 8, st));
  if (!slots) {
    dev_free(m, list, st);
    return fail(ASH_ERR_OOM, "rehash table allocation failed");
  }
  ASH_CUDA(cudaMemsetAsync(slots, 0xFF, n_slots * 8, st));

  int32_t* kb = m->kb;
  int32_t* heap = m->heap;
  std::vector<void*> vb = m->vb;
  const bool grow = new_capacity != m->capacity;
  if (grow) {
    kb = static_cast<int32_t*>(dev_alloc(m, new_capacity * m->ks * 4, st));
    heap = static_cast<int32_t*>(dev_alloc(m, new_capacity * 4, st));
    bool ok = kb && heap;
    for (int j = 0; j < m->n_values && ok; ++j) {
      vb[j] = dev_alloc(m, new_capacity * m->row_bytes[j], st);
      ok = vb[j] != nullptr;
    }
    if (!ok) {
      dev_free(m, list, st);
      dev_free(m, slots, st);
      return fail(ASH_ERR_OOM, "rehash buffer allocation failed");
    }
    if (preserve) {
      // indices are kept: copy buffers, extend the heap with the new indices
      ASH_CUDA(cudaMemcpyAsync(kb, m->kb, m->capacity * m->ks * 4, cudaMemcpyDeviceToDevice, st));
      ASH_CUDA(cudaMemcpyAsync(heap, m->heap, m->capacity * 4, cudaMemcpyDeviceToDevice, st));
      ash::launch_iota(heap, m->capacity, new_capacity, L);
      for (int j = 0; j < m->n_values; ++j) {
        const int64_t rb = m->row_bytes[j];
        ASH_CUDA(cudaMemcpyAsync(vb[j], m->vb[j], m->capacity * rb, cudaMemcpyDeviceToDevice, st));
        ASH_CUDA(cudaMemsetAsync(static_cast<char*>(vb[j]) + m->capacity * rb, 0, (new_capacity - m->capacity) * rb, st));
      }
    } else {
      // compaction: entry j of the list becomes index j
      ash::launch_iota(heap, 0, new_capacity, L);
      m->heap_identity = true;
      ash::ValueCopy vc{};
      vc.n = m->n_values;
      for (int j = 0; j < m->n_values; ++j) {
        ASH_CUDA(cudaMemsetAsync(vb[j], 0, new_capacity * m->row_bytes[j], st));
        vc.dst[j] = vb[j];
        vc.src[j] = m->vb[j];
        vc.row_bytes[j] = m->row_bytes[j];
        vc.vec[j] = vec_width(m->row_bytes[j], vb[j], m->vb[j]);
      }
      ash::launch_gather_rows(vc, list, size, L);
    }
  }
  // 2) re-insert the live keys into the new table (preferred slots first)
  m->S = m->tuning.slots_per_bucket;
  m->slots = slots;
  m->n_slots = n_slots;
  m->pref_placed = true;
  m->n_buckets = static_cast<uint32_t>(n_slots / m->S);
  m->capacity = new_capacity;
  m->kb = kb;
  m->heap = heap;
  m->vb = vb;
  ash::TableView tv = view_of(m);
  m->K.rebuild(m->S, tv, old.kb, list, size, nullptr, preserve ? 1 : 0, (!preserve) ? 1 : 0, L);
  s = check_launch("rehash rebuild");
  if (s != ASH_OK) return s;
  ash::launch_set_top_used(m->ctrl, size, size, L);
  // 3) release the old storage
  dev_free(m, old.slots, st);
  if (grow) {
    dev_free(m, old.kb, st);
    dev_free(m, old.heap, st);
    for (void* p : old.vb) dev_free(m, p, st);
  }
  dev_free(m, list, st);
  m->size_ub = size;
  m->used_ub = size;
  m->tomb_lb = 0;
  invalidate_snapshot(m);
  return check_launch("rehash");
}

// Grows the capacity to new_capacity (>= capacity) without any host
// synchronisation: the live count never leaves the device.  The listing
// writes it to the control block, the rebuild kernel reads it there, and the
// used-slot count is set from it.  Buffer indices are kept.
ash_status grow_async(ash_map* m, int64_t new_capacity, cudaStream_t st) {
  if (new_capacity < m->capacity) return fail(ASH_ERR_INVALID, "grow_async cannot shrink");
  __atomic_fetch_add(&m->rebuilds, 1, __ATOMIC_RELAXED);
  const ash::Launch L = launch_of(m, st);
  const int64_t c = m->capacity;
  int32_t* list = static_cast<int32_t*>(dev_alloc(m, c * 4, st));
  if (!list) return fail(ASH_ERR_OOM, "growth list allocation failed");
  ash_status s = ensure_list_scratch(m, st);
  if (s != ASH_OK) {
    dev_free(m, list, st);
    return s;
  }
  ash::launch_list_active(m->heap_identity, m->heap, c, m->ctrl, m->list_scratch, list, c, nullptr, L);
  const int64_t n_slots = slots_for(new_capacity, m->tuning);
  if (n_slots >= (int64_t{1} << 31)) {
    dev_free(m, list, st);
    return fail(ASH_ERR_INVALID, "capacity too large for 31-bit slot indices");
  }
  uint64_t* slots = static_cast<uint64_t*>(dev_alloc(m, n_slots * 8, st));
  int32_t* kb = m->kb;
  int32_t* heap = m->heap;
  std::vector<void*> vb = m->vb;
  const bool grow = new_capacity != c;
  bool ok = slots != nullptr;
  if (grow && ok) {
    kb = static_cast<int32_t*>(dev_alloc(m, new_capacity * m->ks * 4, st));
    heap = static_cast<int32_t*>(dev_alloc(m, new_capacity * 4, st));
    ok = kb && heap;
    for (int j = 0; j < m->n_values && ok; ++j) {
      vb[j] = dev_alloc(m, new_capacity * m->row_bytes[j], st);
      ok = vb[j] != nullptr;
    }
  }
  if (!ok) {
    dev_free(m, list, st);
    dev_free(m, slots, st);
    if (grow) {
      if (kb != m->kb) dev_free(m, kb, st);
      if (heap != m->heap) dev_free(m, heap, st);
      for (int j = 0; j < m->n_values; ++j)
        if (vb[j] != m->vb[j]) dev_free(m, vb[j], st);
    }
    return fail(ASH_ERR_OOM, "growth allocation failed");
  }
  ASH_CUDA(cudaMemsetAsync(slots, 0xFF, n_slots * 8, st));
  if (grow) {
    ASH_CUDA(cudaMemcpyAsync(kb, m->kb, c * m->ks * 4, cudaMemcpyDeviceToDevice, st));
    ASH_CUDA(cudaMemcpyAsync(heap, m->heap, c * 4, cudaMemcpyDeviceToDevice, st));
    ash::launch_iota(heap, c, new_capacity, L);
    for (int j = 0; j < m->n_values; ++j) {
      const int64_t rb = m->row_bytes[j];
      ASH_CUDA(cudaMemcpyAsync(vb[j], m->vb[j], c * rb, cudaMemcpyDeviceToDevice, st));
      ASH_CUDA(cudaMemsetAsync(static_cast<char*>(vb[j]) + c * rb, 0, (new_capacity - c) * rb, st));
    }
  }
  ash_map old = *m;
  m->S = m->tuning.slots_per_bucket;
  m->slots = slots;
  m->n_slots = n_slots;
  m->pref_placed = true;  // the rebuild below places keys preferred-first
  m->n_buckets = static_cast<uint32_t>(n_slots / m->S);
  m->capacity = new_capacity;
  m->kb = kb;
  m->heap = heap;
  m->vb = vb;
  m->K.rebuild(m->S, view_of(m), old.kb, list, c, &m->ctrl->count, 1, 0, L);
  ash::launch_set_used_from_count(m->ctrl, L);
  dev_free(m, old.slots, st);
  if (grow) {
    dev_free(m, old.kb, st);
    dev_free(m, old.heap, st);
    for (void* p : old.vb) dev_free(m, p, st);
  }
  dev_free(m, list, st);
  m->used_ub = m->size_ub;
  m->tomb_lb = 0;
  invalidate_snapshot(m);  // a snapshot taken before the rebuild would report its tombstones
  return check_launch("grow_async");
}

// Makes room for a batch of n insert/activate keys: x2 growth when the live
// count could pass the capacity (Sec. 4.5), and a table rebuild when used
// slots (live + tombstones) could pass max_used_fraction.
ash_status ensure_room(ash_map* m, int64_t n, cudaStream_t st) {
  const int64_t max_used = static_cast<int64_t>(m->tuning.max_used_fraction * static_cast<double>(m->n_slots));
  tighten_bounds(m);  // folds in a landed snapshot (never blocks)
  const bool size_risk = m->size_ub + n > m->capacity;
  const bool used_risk = m->used_ub + n > max_used;
  if (!size_risk && !used_risk) {
    // a clean-up rebuild at the same capacity, enqueued with no host sync
    if (tombstones_need_rebuild(m)) return grow_async(m, m->capacity, st);
    return ASH_OK;
  }
  int64_t top, used;
  ash_status s = refresh(m, st, &top, &used, nullptr);
  if (s != ASH_OK) return s;
  int64_t new_c = m->capacity;
  if (top + n > m->capacity && m->tuning.auto_grow) {
    new_c = std::max<int64_t>(m->capacity, 1);
    while (top + n > new_c) new_c *= 2;
  }
  const int64_t max_used_new = static_cast<int64_t>(m->tuning.max_used_fraction * static_cast<double>(slots_for(new_c, m->tuning)));
  if (new_c != m->capacity || used + n > max_used_new) return rebuild_to(m, new_c, top, st);
  return ASH_OK;
}

ash_status check_keys(const ash_map* m, const void* keys, int64_t n) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (n < 0 || n >= 0x7FFFFFFF) return fail(ASH_ERR_INVALID, "n must be in [0, 2^31 - 1)");
  if (n > 0 && !keys) return fail(ASH_ERR_INVALID, "keys is NULL");
  return ASH_OK;
}

// pts != nullptr: the input rows are float32 points quantised in the kernels
// (keys == pts->p then); otherwise int32 key rows.
ash_status insert_impl(ash_map* m, const int32_t* keys, const void* const* values_host, int64_t n, int32_t* idx,
                       uint8_t* mask, cudaStream_t st, const ash::PointRows* pts = nullptr) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (n == 0) return ASH_OK;
  if (!idx || !mask) return fail(ASH_ERR_INVALID, "buf_indices and masks are required");
  if (values_host && m->n_values > 0) {
    for (int j = 0; j < m->n_values; ++j)
      if (!values_host[j]) return fail(ASH_ERR_INVALID, "a value pointer is NULL");
  }
  DeviceGuard g(m->device);
  m->last_stream = st;
  s = ensure_room(m, n, st);
  if (s != ASH_OK) return s;
  s = ensure_win_bits(m, n, st);
  if (s != ASH_OK) return s;
  // int32 keys and no value rows to copy: the keys may go in home-bucket
  // range order (the claim and commit then see positions in that order, and
  // equal keys keep their input order)
  int log_p = (pts || (values_host && m->n_values > 0)) ? 0 : partition_log(m, n);
  PartBufs pb;
  if (log_p > 0 && !partition_call(m, keys, n, log_p, st, &pb)) log_p = 0;
  const int32_t* ckeys = log_p > 0 ? pb.keys : keys;
  int32_t* cidx = log_p > 0 ? pb.idx : idx;
  uint8_t* cmask = log_p > 0 ? pb.mask : mask;
  // an insert that stopped between its claim and its commit left flags set
  if (!m->win_bits_clean) ASH_CUDA(cudaMemsetAsync(m->win_bits, 0, m->win_bits_bytes, st));
  m->win_bits_clean = false;  // until every commit of this insert is enqueued
  const ash::Launch L = launch_of(m, st);
  ash::TableView tv = view_of(m);
  const int kpt = m->tuning.keys_per_thread;
  const int pref = claim_prefers_slot(m);
  const int ckpt = m->tuning.commit_keys_per_thread ? m->tuning.commit_keys_per_thread : kpt;
  // one value buffer with small rows: copied by the committing thread;
  // anything else: warp-per-row scatter after the commit
  bool inline_value = false;
  ash::ValueRow vr{};
  ash::ValueCopy vc{};
  if (values_host && m->n_values > 0) {
    const int64_t rb0 = m->row_bytes[0];
    if (m->n_values == 1 && rb0 <= m->tuning.inline_value_bytes && (rb0 == 4 || rb0 == 8 || rb0 == 16) &&
        vec_width(rb0, m->vb[0], values_host[0]) == rb0) {
      inline_value = true;
      vr.dst = m->vb[0];
      vr.src = values_host[0];
      vr.row_bytes = m->row_bytes[0];
      vr.vec = vec_width(m->row_bytes[0], m->vb[0], values_host[0]);
    } else {
      vc.n = m->n_values;
      for (int j = 0; j < m->n_values; ++j) {
        vc.dst[j] = m->vb[j];
        vc.src[j] = values_host[j];
        vc.row_bytes[j] = m->row_bytes[j];
        vc.vec[j] = vec_width(m->row_bytes[j], m->vb[j], values_host[j]);
      }
    }
  }
  tv.lost = m->win_bits;
  // the commit's last block publishes the control block when a snapshot is due
  note_insert_stream(m, st);
  const bool snap = snapshot_wanted(m, st, n);
  if (snap) {
    tv.snap = m->snap_dev;
    tv.snap_seq = m->snap_seq;
  }
  if (pts) {
    m->K.claim_pts(m->S, kpt, pref, tv, *pts, n, idx, L);
    m->K.commit_pts(ckpt, tv, *pts, n, idx, mask, inline_value ? &vr : nullptr, L);
  } else if (log_p > 0) {
    // One range after the other: its table buckets are asked into L2, then
    // its keys claimed and committed.  The slices are the ranged order cut
    // at n p / P (about the ranges' bounds, which only the device knows).
    // Cutting claims and commits by position keeps the results: a slice's
    // keys equal to a key committed by an earlier slice report it present,
    // as losers of a join would, and the lowest position wins either way.
    const int P = 1 << log_p;
    for (int p = 0; p < P; ++p) {
      const int64_t a = n * p / P;
      const int64_t b = n * (p + 1) / P;  // the last slice is never empty
      if (b == a) continue;
      prefetch_table_range(m, p, P, L);
      ash::TableView tvp = tv;
      if (p != P - 1) tvp.snap = nullptr;  // the last commit publishes the control block
      const int32_t* sk = ckeys + a * m->key_dim;
      m->K.claim(m->S, kpt, pref, tvp, sk, b - a, cidx + a, L);
      m->K.commit(ckpt, tvp, sk, b - a, cidx + a, cmask + a, inline_value ? &vr : nullptr, L);
    }
  } else {
    m->K.claim(m->S, kpt, pref, tv, ckeys, n, cidx, L);
    m->K.commit(ckpt, tv, ckeys, n, cidx, cmask, inline_value ? &vr : nullptr, L);
  }
  if (log_p > 0) partition_finish(m, pb, n, idx, mask, st);
  if (vc.n > 0) ash::launch_scatter_rows(vc, idx, mask, n, L);
  if (!pref) m->pref_placed = false;  // the bucket-first claim places keys in slot order
  m->win_bits_clean = true;  // the commits clear every winner-flag word they read
  m->size_ub += n;
  m->used_ub += n;
  m->added_since_snap += n;
  if (snap) snapshot_issued(m);
  return check_launch("insert");
}

}  // namespace host
}  // namespace ash

using namespace ash::host;

extern "C" {

void ash_default_tuning(ash_tuning* out) {
  if (!out) return;
  out->slots_per_bucket = 4;
  out->slots_per_capacity = 2.0f;
  out->block_threads = 256;
  out->blocks_per_sm = 8;
  out->max_probes = 0;
  out->auto_grow = 1;
  out->max_used_fraction = 0.65f;
  out->inline_value_bytes = 16;
  out->keys_per_thread = 2;
  out->warp_probe = 0;
  out->find_keys_per_thread = 1;
  out->claim_mode = 0;
  out->commit_keys_per_thread = 1;
  out->partition_keys = 0;
}

ash_status ash_set_allocator(ash_alloc_fn alloc_fn, ash_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return fail(ASH_ERR_INVALID, "alloc and free must both be set or both NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  g_alloc.alloc = alloc_fn;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return ASH_OK;
}

ash_status ash_create(int key_dim, int64_t capacity, int n_values, const int64_t* value_numel_host,
                      const int32_t* value_dtypes_host, int device, const ash_tuning* tuning, ash_stream stream,
                      ash_map** out_host) {
  if (!out_host) return fail(ASH_ERR_INVALID, "out is NULL");
  *out_host = nullptr;
  if (key_dim < 1 || key_dim > 8) return fail(ASH_ERR_INVALID, "key_dim must be in 1..8");
  if (capacity < 1) return fail(ASH_ERR_INVALID, "capacity must be >= 1");
  if (n_values < 0 || n_values > ash::kMaxValues) return fail(ASH_ERR_INVALID, "n_values must be in 0..8");
  if (n_values > 0 && (!value_numel_host || !value_dtypes_host)) return fail(ASH_ERR_INVALID, "value shapes/dtypes missing");
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return fail(ASH_ERR_INVALID, "no such CUDA device");
  }
  ash_map* m = new ash_map();
  if (tuning) m->tuning = *tuning; else ash_default_tuning(&m->tuning);
  ash_status s = validate_tuning(m->tuning);
  if (s != ASH_OK) { delete m; return s; }
  m->device = device;
  m->key_dim = key_dim;
  m->ks = key_dim <= 1 ? 1 : (key_dim <= 2 ? 2 : (key_dim <= 4 ? 4 : 8));
  m->n_values = n_values;
  for (int j = 0; j < n_values; ++j) {
    const int64_t eb = dtype_bytes(value_dtypes_host[j]);
    if (eb == 0 || value_numel_host[j] < 1) { delete m; return fail(ASH_ERR_INVALID, "bad value dtype or shape"); }
    m->numel.push_back(value_numel_host[j]);
    m->dtype.push_back(value_dtypes_host[j]);
    m->row_bytes.push_back(eb * value_numel_host[j]);
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    m->alloc = g_alloc;
  }
  m->K = kernels_for(key_dim);
  DeviceGuard g(device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  m->ctrl_host = pinned_ctrl_take();
  SnapRec rec{nullptr, nullptr, 0u};
  if (!m->ctrl_host || !snap_take(&rec)) {
    pinned_ctrl_give(m->ctrl_host);
    delete m;
    return fail(ASH_ERR_OOM, "pinned host allocation failed");
  }
  m->snap_host = rec.host;
  m->snap_dev = rec.dev;
  m->snap_seq = rec.seq;
  m->ctrl = static_cast<ash::Ctrl*>(dev_alloc(m, sizeof(ash::Ctrl), st));
  if (!m->ctrl) { ash_destroy(m); return fail(ASH_ERR_OOM, "device allocation failed"); }
  if (cudaMemsetAsync(m->ctrl, 0, sizeof(ash::Ctrl), st) != cudaSuccess) {
    ash_destroy(m);
    return cuda_fail(cudaGetLastError(), "ash_create");
  }
  s = alloc_storage(m, capacity, st);
  // winner flags for a first insert of up to `capacity` keys, allocated here
  // so that the insert itself allocates nothing
  if (s == ASH_OK) s = ensure_win_bits(m, capacity, st);
  if (s != ASH_OK) {
    std::string msg = g_last_error;
    ash_destroy(m);
    return fail(s, msg);
  }
  *out_host = m;
  return ASH_OK;
}

ash_status ash_destroy(ash_map* m) {
  if (!m) return ASH_OK;
  DeviceGuard g(m->device);
  cudaStream_t st = m->last_stream;
  free_storage(m, st);
  dev_free(m, m->scratch, st);
  dev_free(m, m->win_bits, st);
  dev_free(m, m->list_scratch, st);
  dev_free(m, m->ctrl, st);
  pinned_ctrl_give(m->ctrl_host);
  // a snapshot still in flight keeps its record out of the pool until it lands
  snap_give({m->snap_host, m->snap_dev, m->snap_seq}, m->snap_state != 0);
  delete m;
  return ASH_OK;
}

ash_status ash_insert(ash_map* m, const int32_t* keys, const void* const* values_host, int64_t n,
                      int32_t* buf_indices, uint8_t* masks, ash_stream stream) {
  if (m && m->n_values > 0 && n > 0 && !values_host) return fail(ASH_ERR_INVALID, "values are required for insert");
  return insert_impl(m, keys, values_host, n, buf_indices, masks, reinterpret_cast<cudaStream_t>(stream));
}

ash_status ash_activate(ash_map* m, const int32_t* keys, int64_t n, int32_t* buf_indices, uint8_t* masks,
                        ash_stream stream) {
  return insert_impl(m, keys, nullptr, n, buf_indices, masks, reinterpret_cast<cudaStream_t>(stream));
}

ash_status ash_find(ash_map* m, const int32_t* keys, int64_t n, int32_t* buf_indices, uint8_t* masks,
                    ash_stream stream) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (n == 0) return ASH_OK;
  if (!buf_indices || !masks) return fail(ASH_ERR_INVALID, "buf_indices and masks are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  int log_p = partition_log(m, n);
  PartBufs pb;
  if (log_p > 0 && !partition_call(m, keys, n, log_p, st, &pb)) log_p = 0;
  const int32_t* fkeys = log_p > 0 ? pb.keys : keys;
  int32_t* fidx = log_p > 0 ? pb.idx : buf_indices;
  uint8_t* fmask = log_p > 0 ? pb.mask : masks;
  const ash::Launch L = launch_of(m, st);
  const int fkpt = m->tuning.find_keys_per_thread ? m->tuning.find_keys_per_thread : m->tuning.keys_per_thread;
  const int P = log_p > 0 ? 1 << log_p : 1;
  for (int p = 0; p < P; ++p) {
    // ranged: one range after the other, its table buckets asked into L2
    // first (slices cut at n p / P, as for inserts)
    const int64_t a = n * p / P;
    const int64_t b = n * (p + 1) / P;
    if (b == a) continue;
    if (log_p > 0) prefetch_table_range(m, p, P, L);
    const int32_t* sk = fkeys + a * m->key_dim;
    if (m->tuning.warp_probe == 1)
      m->K.find_group(m->S, view_of(m), sk, b - a, fidx + a, fmask + a, L);
    else
      m->K.find(m->S, fkpt, view_of(m), sk, b - a, fidx + a, fmask + a, L);
  }
  if (log_p > 0) partition_finish(m, pb, n, buf_indices, masks, st);
  return check_launch("find");
}

ash_status ash_insert_points(ash_map* m, const float* points, float cell, const void* const* values_host, int64_t n,
                             int32_t* buf_indices, uint8_t* masks, ash_stream stream) {
  if (m && m->n_values > 0 && n > 0 && !values_host) return fail(ASH_ERR_INVALID, "values are required for insert");
  if (!(cell > 0.0f)) return fail(ASH_ERR_INVALID, "cell must be > 0");
  const ash::PointRows p{points, cell};
  return insert_impl(m, reinterpret_cast<const int32_t*>(points), values_host, n, buf_indices, masks,
                     reinterpret_cast<cudaStream_t>(stream), &p);
}

ash_status ash_activate_points(ash_map* m, const float* points, float cell, int64_t n, int32_t* buf_indices,
                               uint8_t* masks, ash_stream stream) {
  if (!(cell > 0.0f)) return fail(ASH_ERR_INVALID, "cell must be > 0");
  const ash::PointRows p{points, cell};
  return insert_impl(m, reinterpret_cast<const int32_t*>(points), nullptr, n, buf_indices, masks,
                     reinterpret_cast<cudaStream_t>(stream), &p);
}

ash_status ash_find_points(ash_map* m, const float* points, float cell, int64_t n, int32_t* buf_indices,
                           uint8_t* masks, ash_stream stream) {
  ash_status s = check_keys(m, points, n);
  if (s != ASH_OK) return s;
  if (!(cell > 0.0f)) return fail(ASH_ERR_INVALID, "cell must be > 0");
  if (n == 0) return ASH_OK;
  if (!buf_indices || !masks) return fail(ASH_ERR_INVALID, "buf_indices and masks are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  const int kpt = m->tuning.find_keys_per_thread ? m->tuning.find_keys_per_thread : m->tuning.keys_per_thread;
  m->K.find_pts(m->S, kpt, view_of(m), ash::PointRows{points, cell}, n, buf_indices, masks, launch_of(m, st));
  return check_launch("find_points");
}

ash_status ash_erase(ash_map* m, const int32_t* keys, int64_t n, uint8_t* masks, ash_stream stream) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (n == 0) return ASH_OK;
  if (!masks) return fail(ASH_ERR_INVALID, "masks is required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  s = ensure_scratch(m, n * 4, st);
  if (s != ASH_OK) return s;
  const ash::Launch L = launch_of(m, st);
  const ash::TableView tv = view_of(m);
  m->K.erase_mark(m->S, tv, keys, n, m->scratch, L);
  ash::launch_erase_resolve(m->S, tv, n, m->scratch, masks, L);
  m->heap_identity = false;
  m->erased_since_snap += n;
  maybe_snapshot(m, st);
  return check_launch("erase");
}

ash_status ash_get_active_indices(ash_map* m, int32_t* out, int64_t out_capacity, int64_t* count_host,
                                  ash_stream stream) {
  if (!m || !count_host) return fail(ASH_ERR_INVALID, "map and count_host are required");
  if (out_capacity > 0 && !out) return fail(ASH_ERR_INVALID, "out is NULL");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  ash_status s = ensure_list_scratch(m, st);
  if (s != ASH_OK) return s;
  ash::launch_list_active(m->heap_identity, m->heap, m->capacity, m->ctrl, m->list_scratch, out, std::max<int64_t>(out_capacity, 0),
                          nullptr, launch_of(m, st));
  s = check_launch("get_active_indices");
  if (s != ASH_OK) return s;
  int64_t top, used;
  s = refresh(m, st, &top, &used, nullptr);
  if (s != ASH_OK) return s;
  *count_host = static_cast<int64_t>(m->ctrl_host->count);
  return ASH_OK;
}

ash_status ash_get_active_indices_async(ash_map* m, int32_t* out, int64_t out_capacity, int64_t* count_dev,
                                        ash_stream stream) {
  if (!m || !count_dev) return fail(ASH_ERR_INVALID, "map and count_dev are required");
  if (out_capacity > 0 && !out) return fail(ASH_ERR_INVALID, "out is NULL");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  ash_status s = ensure_list_scratch(m, st);
  if (s != ASH_OK) return s;
  const ash::Launch L = launch_of(m, st);
  ash::launch_list_active(m->heap_identity, m->heap, m->capacity, m->ctrl, m->list_scratch, out, std::max<int64_t>(out_capacity, 0),
                          reinterpret_cast<long long*>(count_dev), L);
  return check_launch("get_active_indices_async");
}

ash_status ash_gather_keys_count(ash_map* m, const int32_t* indices, int64_t n_max, const int64_t* n_dev,
                                 int32_t* out, ash_stream stream) {
  if (!m || !n_dev) return fail(ASH_ERR_INVALID, "map and n_dev are required");
  if (n_max < 0) return fail(ASH_ERR_INVALID, "n_max must be >= 0");
  if (n_max == 0) return ASH_OK;
  if (!indices || !out) return fail(ASH_ERR_INVALID, "indices and out are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ash::launch_gather_keys(m->kb, m->ks, m->key_dim, m->capacity, indices, n_max,
                          reinterpret_cast<const long long*>(n_dev), out, launch_of(m, st));
  return check_launch("gather_keys_count");
}

ash_status ash_gather_values_count(ash_map* m, int j, const int32_t* indices, int64_t n_max, const int64_t* n_dev,
                                   void* out, ash_stream stream) {
  if (!m || !n_dev) return fail(ASH_ERR_INVALID, "map and n_dev are required");
  if (j < 0 || j >= m->n_values) return fail(ASH_ERR_INVALID, "value buffer index out of range");
  if (n_max < 0) return fail(ASH_ERR_INVALID, "n_max must be >= 0");
  if (n_max == 0) return ASH_OK;
  if (!indices || !out) return fail(ASH_ERR_INVALID, "indices and out are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t rb = m->row_bytes[j];
  ash::launch_gather_values(m->vb[j], rb, vec_width(rb, m->vb[j], out), m->capacity, indices, n_max,
                            reinterpret_cast<const long long*>(n_dev), out, launch_of(m, st));
  return check_launch("gather_values_count");
}

ash_status ash_size(ash_map* m, int64_t* size_host, ash_stream stream) {
  if (!m || !size_host) return fail(ASH_ERR_INVALID, "map and size_host are required");
  DeviceGuard g(m->device);
  int64_t top, used;
  ash_status s = refresh(m, reinterpret_cast<cudaStream_t>(stream), &top, &used, nullptr);
  if (s != ASH_OK) return s;
  *size_host = top;
  return ASH_OK;
}

ash_status ash_get_map_stats(ash_map* m, ash_map_stats* out, ash_stream stream) {
  if (!m || !out) return fail(ASH_ERR_INVALID, "map and out are required");
  DeviceGuard g(m->device);
  int64_t top, used;
  ash_status s = refresh(m, reinterpret_cast<cudaStream_t>(stream), &top, &used, nullptr);
  if (s != ASH_OK) return s;
  out->capacity = m->capacity;
  out->table_slots = m->n_slots;
  out->live = top;
  out->used_slots = used;
  out->host_syncs = __atomic_load_n(&m->host_syncs, __ATOMIC_RELAXED);
  out->rebuilds = __atomic_load_n(&m->rebuilds, __ATOMIC_RELAXED);
  return ASH_OK;
}

int64_t ash_capacity(const ash_map* m) { return m ? m->capacity : 0; }
int ash_key_dim(const ash_map* m) { return m ? m->key_dim : 0; }
int ash_n_values(const ash_map* m) { return m ? m->n_values : 0; }

ash_status ash_rehash(ash_map* m, int64_t new_capacity, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (new_capacity < 0) return fail(ASH_ERR_INVALID, "new_capacity must be >= 0");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  int64_t top, used;
  ash_status s = refresh(m, st, &top, &used, nullptr);
  if (s != ASH_OK) return s;
  if (new_capacity == 0) new_capacity = 2 * m->capacity;
  if (new_capacity < top) return fail(ASH_ERR_INVALID, "new_capacity is below the live count");
  s = rebuild_to(m, new_capacity, top, st);
  if (s != ASH_OK) return s;
  ASH_CUDA(cudaStreamSynchronize(st));
  return ASH_OK;
}

ash_status ash_reserve(ash_map* m, int64_t new_capacity, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (new_capacity <= m->capacity) return ASH_OK;
  return ash_rehash(m, new_capacity, stream);
}

ash_status ash_reserve_async(ash_map* m, int64_t new_capacity, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (new_capacity <= m->capacity) return ASH_OK;
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  return grow_async(m, new_capacity, st);
}

ash_status ash_clear(ash_map* m, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  const ash::Launch L = launch_of(m, st);
  ASH_CUDA(cudaMemsetAsync(m->slots, 0xFF, m->n_slots * 8, st));
  ash::launch_iota(m->heap, 0, m->capacity, L);
  ash::launch_set_top_used(m->ctrl, 0, 0, L);
  m->size_ub = 0;
  m->used_ub = 0;
  m->tomb_lb = 0;
  m->pref_placed = true;
  m->heap_identity = true;
  invalidate_snapshot(m);
  return check_launch("clear");
}

ash_status ash_key_buffer(ash_map* m, int32_t** ptr_host, int64_t* row_stride_host) {
  if (!m || !ptr_host) return fail(ASH_ERR_INVALID, "map and ptr are required");
  *ptr_host = m->kb;
  if (row_stride_host) *row_stride_host = m->ks;
  return ASH_OK;
}

ash_status ash_value_buffer(ash_map* m, int j, void** ptr_host, int64_t* row_bytes_host) {
  if (!m || !ptr_host) return fail(ASH_ERR_INVALID, "map and ptr are required");
  if (j < 0 || j >= m->n_values) return fail(ASH_ERR_INVALID, "value buffer index out of range");
  *ptr_host = m->vb[j];
  if (row_bytes_host) *row_bytes_host = m->row_bytes[j];
  return ASH_OK;
}

ash_status ash_heap_buffer(ash_map* m, int32_t** heap_host, int32_t** top_host) {
  if (!m || !heap_host) return fail(ASH_ERR_INVALID, "map and heap are required");
  *heap_host = m->heap;
  if (top_host) *top_host = reinterpret_cast<int32_t*>(&m->ctrl->top_used);  // low word (little endian)
  return ASH_OK;
}

ash_status ash_gather_keys(ash_map* m, const int32_t* indices, int64_t n, int32_t* out, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (n < 0) return fail(ASH_ERR_INVALID, "n must be >= 0");
  if (n == 0) return ASH_OK;
  if (!indices || !out) return fail(ASH_ERR_INVALID, "indices and out are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ash::launch_gather_keys(m->kb, m->ks, m->key_dim, m->capacity, indices, n, nullptr, out, launch_of(m, st));
  return check_launch("gather_keys");
}

ash_status ash_gather_values(ash_map* m, int j, const int32_t* indices, int64_t n, void* out, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  if (j < 0 || j >= m->n_values) return fail(ASH_ERR_INVALID, "value buffer index out of range");
  if (n < 0) return fail(ASH_ERR_INVALID, "n must be >= 0");
  if (n == 0) return ASH_OK;
  if (!indices || !out) return fail(ASH_ERR_INVALID, "indices and out are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t rb = m->row_bytes[j];
  ash::launch_gather_values(m->vb[j], rb, vec_width(rb, m->vb[j], out), m->capacity, indices, n, nullptr, out,
                            launch_of(m, st));
  return check_launch("gather_values");
}

ash_status ash_find_neighbors(ash_map* m, const int32_t* keys, int64_t n, int32_t radius, int32_t* buf_indices,
                              uint8_t* masks, ash_stream stream) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (radius < 0 || radius > 8) return fail(ASH_ERR_INVALID, "radius must be in 0..8");
  int64_t n_off = 1;
  for (int j = 0; j < m->key_dim; ++j) n_off *= 2 * radius + 1;
  if (n_off > (int64_t{1} << 20) || n * n_off >= (int64_t{1} << 40))
    return fail(ASH_ERR_INVALID, "too many neighbour queries");
  if (n == 0) return ASH_OK;
  if (!buf_indices || !masks) return fail(ASH_ERR_INVALID, "buf_indices and masks are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  m->K.neighbors(m->S, view_of(m), keys, n, radius, n_off, buf_indices, masks, launch_of(m, st));
  return check_launch("find_neighbors");
}

ash_status ash_find_offsets(ash_map* m, const int32_t* keys, int64_t n, const int32_t* offsets, int64_t n_offsets,
                            int32_t* buf_indices, uint8_t* masks, ash_stream stream) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (n_offsets < 1 || n_offsets > 4096) return fail(ASH_ERR_INVALID, "n_offsets must be in 1..4096");
  if (!offsets) return fail(ASH_ERR_INVALID, "offsets is NULL");
  if (n * n_offsets >= (int64_t{1} << 40)) return fail(ASH_ERR_INVALID, "too many neighbour queries");
  if (n == 0) return ASH_OK;
  if (!buf_indices || !masks) return fail(ASH_ERR_INVALID, "buf_indices and masks are required");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  m->K.offsets(m->S, view_of(m), keys, n, offsets, n_offsets, buf_indices, masks, launch_of(m, st));
  return check_launch("find_offsets");
}

ash_status ash_get_tuning(const ash_map* m, ash_tuning* out_host) {
  if (!m || !out_host) return fail(ASH_ERR_INVALID, "map and out are required");
  *out_host = m->tuning;
  return ASH_OK;
}

ash_status ash_set_tuning(ash_map* m, const ash_tuning* t) {
  if (!m || !t) return fail(ASH_ERR_INVALID, "map and tuning are required");
  ash_status s = validate_tuning(*t);
  if (s != ASH_OK) return s;
  m->tuning = *t;  // S and slots_per_capacity apply at the next rebuild
  m->tuning.slots_per_bucket = t->slots_per_bucket;
  return ASH_OK;
}

ash_status ash_sync_status(ash_map* m, ash_stream stream) {
  if (!m) return fail(ASH_ERR_INVALID, "map is NULL");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int64_t top, used;
  int bits = 0;
  ash_status s = refresh(m, st, &top, &used, &bits);
  if (s != ASH_OK) return s;
  if (bits) {
    ASH_CUDA(cudaMemsetAsync(&m->ctrl->status, 0, sizeof(int), st));
    ASH_CUDA(cudaStreamSynchronize(st));
  }
  return status_from_bits(bits);
}

ash_status ash_quantize(const float* points, int64_t n_coords, float cell, int32_t* keys, ash_stream stream) {
  if (n_coords < 0) return fail(ASH_ERR_INVALID, "n_coords must be >= 0");
  if (n_coords == 0) return ASH_OK;
  if (!points || !keys) return fail(ASH_ERR_INVALID, "points and keys are required");
  if (!(cell > 0.0f) || !std::isfinite(cell)) return fail(ASH_ERR_INVALID, "cell must be finite and > 0");
  int dev = 0;
  cudaGetDevice(&dev);
  ash::Launch L;
  L.stream = reinterpret_cast<cudaStream_t>(stream);
  L.block = 256;
  L.grid_cap = sm_count(dev) * 8;
  ash::launch_quantize(points, n_coords, cell, keys, L);
  return check_launch("quantize");
}

ash_status ash_probe_random_read(const void* buf, int64_t buf_bytes, int64_t n_reads, int sector_bytes,
                                 int loads_per_thread, uint32_t seed, uint32_t* sink, int64_t sink_len,
                                 ash_stream stream) {
  if (!buf || !sink || sink_len < 1 || n_reads < 0) return fail(ASH_ERR_INVALID, "bad probe arguments");
  if (sector_bytes != 32 && sector_bytes != 64) return fail(ASH_ERR_INVALID, "sector_bytes must be 32 or 64");
  if (loads_per_thread != 4 && loads_per_thread != 8 && loads_per_thread != 16)
    return fail(ASH_ERR_INVALID, "loads_per_thread must be 4, 8 or 16");
  if (buf_bytes < 64 || buf_bytes % 64 != 0) return fail(ASH_ERR_INVALID, "buf_bytes must be a positive multiple of 64");
  if ((reinterpret_cast<uintptr_t>(buf) & 63u) != 0) return fail(ASH_ERR_INVALID, "buf must be 64-byte aligned");
  int dev = 0;
  cudaGetDevice(&dev);
  ash::Launch L;
  L.stream = reinterpret_cast<cudaStream_t>(stream);
  L.block = 256;
  L.grid_cap = sm_count(dev) * 8;
  ash::launch_probe(buf, buf_bytes, n_reads, sector_bytes, loads_per_thread, seed, sink, sink_len, L);
  return check_launch("probe");
}

ash_status ash_probe_random_atomic(void* buf, int64_t buf_bytes, int64_t n_ops, int mode, uint32_t seed,
                                   uint32_t* sink, int64_t sink_len, ash_stream stream) {
  if (!buf || !sink || sink_len < 1 || n_ops < 0) return fail(ASH_ERR_INVALID, "bad probe arguments");
  if (mode != 0 && mode != 1) return fail(ASH_ERR_INVALID, "mode must be 0 or 1");
  if (buf_bytes < 32 || buf_bytes % 32 != 0) return fail(ASH_ERR_INVALID, "buf_bytes must be a positive multiple of 32");
  if ((reinterpret_cast<uintptr_t>(buf) & 31u) != 0) return fail(ASH_ERR_INVALID, "buf must be 32-byte aligned");
  int dev = 0;
  cudaGetDevice(&dev);
  ash::Launch L;
  L.stream = reinterpret_cast<cudaStream_t>(stream);
  L.block = 256;
  L.grid_cap = sm_count(dev) * 8;
  ash::launch_probe_atomic(buf, buf_bytes, n_ops, mode, seed, sink, sink_len, L);
  return check_launch("probe_atomic");
}

ash_status ash_get_device_info(int device, ash_device_info* out) {
  if (!out) return fail(ASH_ERR_INVALID, "out is NULL");
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return fail(ASH_ERR_INVALID, "no such CUDA device");
  }
  int v = 0;
  out->sm_count = sm_count(device);
  ASH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device));
  out->l2_bytes = v;
  ASH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, device));
  out->pageable_memory_access = v;
  ASH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device));
  out->pageable_uses_host_page_tables = v;
  return ASH_OK;
}

const char* ash_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ------------------------------------------------ allocation-free erase
//
// Some callers cannot let a library allocate device memory: a host whose
// device memory is fully budgeted by its own allocator, or a latency-bound
// loop where a first-time cudaMalloc (which can synchronise the device) is
// not acceptable.  ash_erase may grow map-owned scratch; this variant
// instead uses the fixed array below, so it allocates nothing.
//
// The array lives in device global memory for the life of the process on
// every GPU that loads this library (ASH_ERASE_NOALLOC_MAX_KEYS int32 =
// 4 MiB).  Host code must not use the symbol's name as a pointer (it is a
// host-side stand-in); the device address is obtained once per device with
// cudaGetSymbolAddress, with that device current, on the first call that
// runs on it.  All calls share the array: two calls whose kernels overlap
// on the GPU (different streams, or different maps on the same device)
// race on it and must be ordered by the caller.  Nothing in it needs to
// start at zero: the mark kernel writes every entry that the resolve kernel
// reads.
namespace {

static __device__ __align__(256) int32_t g_erase_noalloc_scratch[ASH_ERASE_NOALLOC_MAX_KEYS];

std::mutex g_noalloc_mu;
int32_t* g_noalloc_ptr[64] = {};

ash_status noalloc_scratch(int device, int32_t** out) {
  if (device < 0 || device >= 64) return fail(ASH_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_erase_noalloc_scratch);  // device is current here
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(ASH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_noalloc_ptr[device] = static_cast<int32_t*>(p);
  }
  *out = g_noalloc_ptr[device];
  return ASH_OK;
}

}  // namespace

extern "C" ash_status ash_erase_noalloc(ash_map* m, const int32_t* keys, int64_t n, uint8_t* masks,
                                        ash_stream stream) {
  ash_status s = check_keys(m, keys, n);
  if (s != ASH_OK) return s;
  if (n > ASH_ERASE_NOALLOC_MAX_KEYS)
    return fail(ASH_ERR_INVALID, "ash_erase_noalloc: n exceeds ASH_ERASE_NOALLOC_MAX_KEYS (1048576)");
  if (n == 0) return ASH_OK;
  if (!masks) return fail(ASH_ERR_INVALID, "masks is required");
  DeviceGuard g(m->device);
  int32_t* scratch = nullptr;
  s = noalloc_scratch(m->device, &scratch);
  if (s != ASH_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  m->last_stream = st;
  const ash::Launch L = launch_of(m, st);
  const ash::TableView tv = view_of(m);
  m->K.erase_mark(m->S, tv, keys, n, scratch, L);
  ash::launch_erase_resolve(m->S, tv, n, scratch, masks, L);
  m->heap_identity = false;
  m->erased_since_snap += n;  // the map's next snapshot counts this call's tombstones
  return check_launch("erase_noalloc");
}
