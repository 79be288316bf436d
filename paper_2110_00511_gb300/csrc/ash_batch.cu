// Batched execution: one CUDA-graph launch services many maps.
//
// A batch is a list of operations, at most one per (map, phase), on maps of
// key dimension 1..4.  Phases run in the order insert/activate -> find ->
// erase (per map, the order the serving and batched workloads apply), each as
// one persistent kernel over ALL maps of that phase: claim, commit, find,
// erase-mark and erase-resolve.  Work is cut into tiles of blockDim.x keys that
// never straddle two operations, so a commit or erase-resolve tile still
// aggregates its heap atomic over one map.  The five kernels plus the upload of
// the descriptor table form one CUDA graph, built once per ring slot and
// replayed: the kernels read everything (maps, pointers, tile counts) from the
// device copy of the table, so a new batch only rewrites the pinned table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ash.h"
#include "ash_internal.h"
#include "ash_kernels.cuh"
#include "ash_trace.h"

namespace ash {

constexpr int kBatchMaxOps = 256;
constexpr int kBatchThreads = 256;
constexpr int kBatchRing = 4;
enum { kPhaseInsert = 0, kPhaseFind = 1, kPhaseErase = 2, kPhases = 3 };

struct BatchOp {
  TableView t;
  const int32_t* keys;
  int32_t* idx;    // insert/activate/find: outputs (claim scratch too); erase: slot scratch
  uint8_t* mask;
  ValueRow v;      // v.row_bytes == 0: no value copy
  int64_t n;
  int64_t tile0;   // first tile of this op within its phase
  int32_t key_dim;
  int32_t S;
};

struct BatchPhase {
  int32_t first;
  int32_t count;
  int64_t tiles;
};

struct BatchTable {
  BatchPhase ph[kPhases];
  int32_t n_ops;
  int32_t pad;
  BatchOp ops[kBatchMaxOps];
};

// Loads the tile starts of one phase into shared memory and maps a tile to
// its operation (binary search over at most kBatchMaxOps entries).
__device__ __forceinline__ void load_tile_starts(const BatchTable* tb, int phase, int64_t* s_tile0) {
  const BatchPhase ph = tb->ph[phase];
  for (int i = threadIdx.x; i < ph.count; i += blockDim.x) s_tile0[i] = tb->ops[ph.first + i].tile0;
  __syncthreads();
}

__device__ __forceinline__ int op_of_tile(const int64_t* s_tile0, int count, int64_t tile) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_tile0[mid] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

#define ASH_DS_CASES(FN, ...)                                       \
  switch (op.key_dim * 100 + op.S) {                                \
    case 104: FN<1, 4>(__VA_ARGS__); break;                         \
    case 108: FN<1, 8>(__VA_ARGS__); break;                         \
    case 116: FN<1, 16>(__VA_ARGS__); break;                        \
    case 204: FN<2, 4>(__VA_ARGS__); break;                         \
    case 208: FN<2, 8>(__VA_ARGS__); break;                         \
    case 216: FN<2, 16>(__VA_ARGS__); break;                        \
    case 304: FN<3, 4>(__VA_ARGS__); break;                         \
    case 308: FN<3, 8>(__VA_ARGS__); break;                         \
    case 316: FN<3, 16>(__VA_ARGS__); break;                        \
    case 404: FN<4, 4>(__VA_ARGS__); break;                         \
    case 408: FN<4, 8>(__VA_ARGS__); break;                         \
    default: FN<4, 16>(__VA_ARGS__); break;                         \
  }

// In the batched kernels the full per-key protocols are the main path, so
// they are inlined (the single-map kernels keep them out of line as their
// rare slow path).
template <int D, int S>
__device__ __forceinline__ void batch_claim_one(const BatchOp& op, int64_t pos) {
  // slot order (measured 7 % faster here than preferred-first placement);
  // the host clears the map's pref_placed flag
  op.idx[pos] = claim_key<D, S, const int32_t*, kClaimSlotMask, false>(op.t, op.keys, pos);
}

template <int D, int S>
__device__ __forceinline__ void batch_find_one(const BatchOp& op, int64_t pos) {
  int32_t k[D];
  load_input_key<D>(op.keys, pos, k);
  const int32_t r = find_key<D, S>(op.t, k);
  op.idx[pos] = r;
  op.mask[pos] = r >= 0 ? 1 : 0;
}

template <int D, int S>
__device__ __forceinline__ void batch_mark_one(const BatchOp& op, int64_t pos) {
  op.idx[pos] = erase_mark_one<D, S>(op.t, op.keys, pos);
}

__global__ void __launch_bounds__(kBatchThreads) batch_claim_kernel(const BatchTable* __restrict__ tb) {
  __shared__ int64_t s_tile0[kBatchMaxOps];
  load_tile_starts(tb, kPhaseInsert, s_tile0);
  const BatchPhase ph = tb->ph[kPhaseInsert];
  for (int64_t tile = blockIdx.x; tile < ph.tiles; tile += gridDim.x) {
    const BatchOp& op = tb->ops[ph.first + op_of_tile(s_tile0, ph.count, tile)];
    const int64_t pos = (tile - op.tile0) * blockDim.x + threadIdx.x;
    if (pos < op.n) { ASH_DS_CASES(batch_claim_one, op, pos) }
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_commit_kernel(const BatchTable* __restrict__ tb) {
  __shared__ int64_t s_tile0[kBatchMaxOps];
  __shared__ int s_warp[33];
  __shared__ int s_base;
  __shared__ int s_got;
  load_tile_starts(tb, kPhaseInsert, s_tile0);
  const BatchPhase ph = tb->ph[kPhaseInsert];
  for (int64_t tile = blockIdx.x; tile < ph.tiles; tile += gridDim.x) {
    const BatchOp& op = tb->ops[ph.first + op_of_tile(s_tile0, ph.count, tile)];
    const int64_t base0 = (tile - op.tile0) * blockDim.x;
    const bool val = op.v.row_bytes > 0;  // uniform over the block
    switch (op.key_dim * 2 + (val ? 1 : 0)) {
      case 2: commit_tile<1, 1, false>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 3: commit_tile<1, 1, true>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 4: commit_tile<2, 1, false>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 5: commit_tile<2, 1, true>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 6: commit_tile<3, 1, false>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 7: commit_tile<3, 1, true>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      case 8: commit_tile<4, 1, false>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
      default: commit_tile<4, 1, true>(op.t, op.keys, op.n, base0, op.idx, op.mask, op.v, s_warp, &s_base, &s_got); break;
    }
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_find_kernel(const BatchTable* __restrict__ tb) {
  __shared__ int64_t s_tile0[kBatchMaxOps];
  load_tile_starts(tb, kPhaseFind, s_tile0);
  const BatchPhase ph = tb->ph[kPhaseFind];
  for (int64_t tile = blockIdx.x; tile < ph.tiles; tile += gridDim.x) {
    const BatchOp& op = tb->ops[ph.first + op_of_tile(s_tile0, ph.count, tile)];
    const int64_t pos = (tile - op.tile0) * blockDim.x + threadIdx.x;
    if (pos < op.n) { ASH_DS_CASES(batch_find_one, op, pos) }
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_erase_mark_kernel(const BatchTable* __restrict__ tb) {
  __shared__ int64_t s_tile0[kBatchMaxOps];
  load_tile_starts(tb, kPhaseErase, s_tile0);
  const BatchPhase ph = tb->ph[kPhaseErase];
  for (int64_t tile = blockIdx.x; tile < ph.tiles; tile += gridDim.x) {
    const BatchOp& op = tb->ops[ph.first + op_of_tile(s_tile0, ph.count, tile)];
    const int64_t pos = (tile - op.tile0) * blockDim.x + threadIdx.x;
    if (pos < op.n) { ASH_DS_CASES(batch_mark_one, op, pos) }
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_erase_resolve_kernel(const BatchTable* __restrict__ tb) {
  __shared__ int64_t s_tile0[kBatchMaxOps];
  __shared__ int s_warp[33];
  __shared__ int s_cnt;
  __shared__ int s_base;
  load_tile_starts(tb, kPhaseErase, s_tile0);
  const BatchPhase ph = tb->ph[kPhaseErase];
  for (int64_t tile = blockIdx.x; tile < ph.tiles; tile += gridDim.x) {
    const BatchOp& op = tb->ops[ph.first + op_of_tile(s_tile0, ph.count, tile)];
    const int64_t base0 = (tile - op.tile0) * blockDim.x;
    if (op.S == 4) erase_resolve_tile<4>(op.t, op.n, base0, op.idx, op.mask, s_warp, &s_cnt, &s_base);
    else if (op.S == 8) erase_resolve_tile<8>(op.t, op.n, base0, op.idx, op.mask, s_warp, &s_cnt, &s_base);
    else erase_resolve_tile<16>(op.t, op.n, base0, op.idx, op.mask, s_warp, &s_cnt, &s_base);
  }
}

}  // namespace ash

using namespace ash;
using namespace ash::host;

struct ash_batch {
  int device = 0;
  int grid = 0;
  Allocator alloc;
  struct Slot {
    BatchTable* h = nullptr;  // pinned
    BatchTable* d = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
    int32_t* scratch = nullptr;  // erase slot indices
    int64_t scratch_n = 0;
  } slot[kBatchRing];
  int next = 0;
  std::mutex mu;
};

namespace {

ash_status build_graph(ash_batch* b, ash_batch::Slot& s) {
  if (cudaGraphCreate(&s.graph, 0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGraphCreate");
  cudaGraphNode_t copy = nullptr;
  if (cudaGraphAddMemcpyNode1D(&copy, s.graph, nullptr, 0, s.d, s.h, sizeof(BatchTable), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return cuda_fail(cudaGetLastError(), "cudaGraphAddMemcpyNode1D");
  void* kernels[5] = {reinterpret_cast<void*>(batch_claim_kernel), reinterpret_cast<void*>(batch_commit_kernel),
                      reinterpret_cast<void*>(batch_find_kernel), reinterpret_cast<void*>(batch_erase_mark_kernel),
                      reinterpret_cast<void*>(batch_erase_resolve_kernel)};
  cudaGraphNode_t prev = copy;
  const BatchTable* arg = s.d;
  void* args[1] = {&arg};
  for (void* k : kernels) {
    cudaKernelNodeParams p{};
    p.func = k;
    p.gridDim = dim3(b->grid);
    p.blockDim = dim3(kBatchThreads);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    p.extra = nullptr;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddKernelNode(&node, s.graph, &prev, 1, &p) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "cudaGraphAddKernelNode");
    prev = node;
  }
  if (cudaGraphInstantiate(&s.exec, s.graph, 0) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "cudaGraphInstantiate");
  return ASH_OK;
}

void* batch_alloc(ash_batch* b, size_t bytes, cudaStream_t st) {
  if (b->alloc.alloc) return b->alloc.alloc(bytes, b->device, reinterpret_cast<ash_stream>(st), b->alloc.ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void batch_free(ash_batch* b, void* p, cudaStream_t st) {
  if (!p) return;
  if (b->alloc.free) b->alloc.free(p, b->device, reinterpret_cast<ash_stream>(st), b->alloc.ctx);
  else cudaFreeAsync(p, st);
}

int phase_of(int32_t op) {
  switch (op) {
    case ASH_OP_INSERT: case ASH_OP_ACTIVATE: return kPhaseInsert;
    case ASH_OP_FIND: return kPhaseFind;
    case ASH_OP_ERASE: return kPhaseErase;
    default: return -1;
  }
}

}  // namespace

extern "C" {

ash_status ash_batch_create(int device, ash_batch** out_host) {
  if (!out_host) return fail(ASH_ERR_INVALID, "out is NULL");
  *out_host = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return fail(ASH_ERR_INVALID, "no such CUDA device");
  }
  DeviceGuard g(device);
  ash_batch* b = new ash_batch();
  b->device = device;
  b->grid = sm_count(device) * 8;
  for (auto& s : b->slot) {
    if (cudaMallocHost(&s.h, sizeof(BatchTable)) != cudaSuccess || cudaMalloc(&s.d, sizeof(BatchTable)) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ash_batch_destroy(b);
      return fail(ASH_ERR_OOM, "batch context allocation failed");
    }
    std::memset(s.h, 0, sizeof(BatchTable));
  }
  *out_host = b;
  return ASH_OK;
}

ash_status ash_batch_destroy(ash_batch* b) {
  if (!b) return ASH_OK;
  DeviceGuard g(b->device);
  for (auto& s : b->slot) {
    if (s.done) cudaEventSynchronize(s.done);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    if (s.h) cudaFreeHost(s.h);
    if (s.d) cudaFree(s.d);
    if (s.done) cudaEventDestroy(s.done);
    batch_free(b, s.scratch, nullptr);
  }
  cudaDeviceSynchronize();
  delete b;
  return ASH_OK;
}

ash_status ash_batch_run(ash_batch* b, const ash_batch_op* ops, int n_ops, ash_stream stream) {
  if (!b) return fail(ASH_ERR_INVALID, "batch is NULL");
  if (n_ops < 0 || n_ops > kBatchMaxOps) return fail(ASH_ERR_INVALID, "n_ops must be in [0, 256]");
  if (n_ops > 0 && !ops) return fail(ASH_ERR_INVALID, "ops is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // ---- validate
  std::vector<std::pair<const ash_map*, int>> seen;
  int64_t erase_total = 0;
  for (int i = 0; i < n_ops; ++i) {
    const ash_batch_op& o = ops[i];
    const int ph = phase_of(o.op);
    if (ph < 0) return fail(ASH_ERR_INVALID, "unknown batch op code");
    ash_status s = check_keys(o.map, o.keys, o.n);
    if (s != ASH_OK) return s;
    if (o.map->device != b->device) return fail(ASH_ERR_INVALID, "map is on another device than the batch");
    if (o.map->key_dim > 4) return fail(ASH_ERR_INVALID, "batched maps support key_dim 1..4");
    if (o.n > 0 && !o.masks) return fail(ASH_ERR_INVALID, "masks is required");
    if (o.n > 0 && ph != kPhaseErase && !o.buf_indices) return fail(ASH_ERR_INVALID, "buf_indices is required");
    if (o.op == ASH_OP_INSERT && o.map->n_values > 0) {
      const int64_t rb = o.map->row_bytes[0];
      if (o.map->n_values != 1 || !(rb == 4 || rb == 8 || rb == 16) || !o.values ||
          vec_width(rb, o.map->vb[0], o.values) != rb)
        return fail(ASH_ERR_INVALID,
                    "batched insert needs one value buffer of 4, 8 or 16-byte rows with aligned values");
    }
    for (auto& p : seen)
      if (p.first == o.map && p.second == ph) return fail(ASH_ERR_INVALID, "two ops on one map in the same phase");
    seen.emplace_back(o.map, ph);
    if (ph == kPhaseErase) erase_total += o.n;
  }
  DeviceGuard g(b->device);
  std::lock_guard<std::mutex> lk(b->mu);
  // ---- growth for the insert phase (may synchronise)
  for (int i = 0; i < n_ops; ++i) {
    if (phase_of(ops[i].op) == kPhaseInsert && ops[i].n > 0) {
      ash_status s = ensure_room(ops[i].map, ops[i].n, st);
      if (s != ASH_OK) return s;
    }
  }
  ash_batch::Slot& sl = b->slot[b->next];
  b->next = (b->next + 1) % kBatchRing;
  if (sl.used && cudaEventSynchronize(sl.done) != cudaSuccess) return cuda_fail(cudaGetLastError(), "batch slot wait");
  if (sl.scratch_n < erase_total) {
    batch_free(b, sl.scratch, st);
    sl.scratch_n = std::max<int64_t>(erase_total, 2 * sl.scratch_n);
    sl.scratch = static_cast<int32_t*>(batch_alloc(b, sl.scratch_n * 4, st));
    if (!sl.scratch) {
      sl.scratch_n = 0;
      return fail(ASH_ERR_OOM, "batch scratch allocation failed");
    }
  }
  // ---- descriptor table, grouped by phase
  BatchTable* tb = sl.h;
  int k = 0;
  int64_t scratch_off = 0;
  for (int ph = 0; ph < kPhases; ++ph) {
    tb->ph[ph].first = k;
    int64_t tiles = 0;
    for (int i = 0; i < n_ops; ++i) {
      const ash_batch_op& o = ops[i];
      if (phase_of(o.op) != ph || o.n == 0) continue;
      BatchOp& d = tb->ops[k++];
      d.t = view_of(o.map);
      d.keys = o.keys;
      d.mask = o.masks;
      d.n = o.n;
      d.key_dim = o.map->key_dim;
      d.S = o.map->S;
      d.tile0 = tiles;
      d.v = ValueRow{};
      if (ph == kPhaseErase) {
        d.idx = sl.scratch + scratch_off;
        scratch_off += o.n;
      } else {
        d.idx = o.buf_indices;
      }
      if (o.op == ASH_OP_INSERT && o.map->n_values == 1) {
        d.v.dst = o.map->vb[0];
        d.v.src = o.values;
        d.v.row_bytes = o.map->row_bytes[0];
        d.v.vec = static_cast<int>(o.map->row_bytes[0]);
      }
      tiles += (o.n + kBatchThreads - 1) / kBatchThreads;
      o.map->last_stream = st;
      if (ph == kPhaseInsert) {
        o.map->size_ub += o.n;
        o.map->used_ub += o.n;
        o.map->added_since_snap += o.n;
        note_insert_stream(o.map, st);
      }
    }
    tb->ph[ph].count = k - tb->ph[ph].first;
    tb->ph[ph].tiles = tiles;
  }
  tb->n_ops = k;
  if (!sl.exec) {
    ash_status s = build_graph(b, sl);
    if (s != ASH_OK) return s;
  }
  {
    TraceScope ts(kKBatch, st, 5);
    if (cudaGraphLaunch(sl.exec, st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGraphLaunch");
  }
  for (int i = 0; i < n_ops; ++i)
    if (ops[i].op == ASH_OP_INSERT || ops[i].op == ASH_OP_ACTIVATE) {
      ops[i].map->pref_placed = false;  // keys placed in slot order
      maybe_snapshot(ops[i].map, st);
    } else if (ops[i].op == ASH_OP_ERASE) {
      ops[i].map->heap_identity = false;
      ops[i].map->erased_since_snap += ops[i].n;
      maybe_snapshot(ops[i].map, st);
    }
  if (cudaEventRecord(sl.done, st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventRecord");
  sl.used = true;
  return ASH_OK;
}

}  // extern "C"
