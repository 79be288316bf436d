// Map kernels that do not depend on the key dimension: erase resolve, the
// active-index listing, heap initialisation, value-row scatter/gather, key
// gather, voxel quantisation and the random-read roofline probe.
#include "ash_aux.h"
#include "ash_kernels.cuh"
#include "ash_trace.h"

namespace ash {

// ------------------------------------------------------------ erase resolve
template <int S>
static void erase_resolve_s(const TableView& t, int64_t n, const int32_t* slot_in, uint8_t* mask, const Launch& L) {
  TraceScope ts(kKEraseResolve, L.stream);
  erase_resolve_kernel<S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, n, slot_in, mask);
}

void launch_erase_resolve(int S, const TableView& t, int64_t n, const int32_t* slot_in, uint8_t* mask, const Launch& L) {
  if (S == 4) erase_resolve_s<4>(t, n, slot_in, mask, L);
  else if (S == 8) erase_resolve_s<8>(t, n, slot_in, mask, L);
  else erase_resolve_s<16>(t, n, slot_in, mask, L);
}

// ------------------------------------------------------- key partitioning
// One block per range: its row of per-block counts (G <= a few thousand
// words) becomes the row's exclusive scan, and the row total is kept.
__global__ void __launch_bounds__(256) partition_scan_kernel(uint32_t* __restrict__ counts, int G,
                                                             uint32_t* __restrict__ range_totals) {
  __shared__ int s_warp[33];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  uint32_t* row = counts + static_cast<int64_t>(blockIdx.x) * G;
  const int per = (G + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per;
  const int hi = lo + per < G ? lo + per : G;
  uint32_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += row[i];
  int total;
  uint32_t at = static_cast<uint32_t>(block_exclusive_scan(static_cast<int>(sum), total, s_warp));
  for (int i = lo; i < hi; ++i) {
    const uint32_t c = row[i];
    row[i] = at;
    at += c;
  }
  if (threadIdx.x == 0) range_totals[blockIdx.x] = static_cast<uint32_t>(total);
}

void launch_partition_scan(uint32_t* counts, int G, int P, uint32_t* range_totals, const Launch& L) {
  launch_dependent(partition_scan_kernel, P, 256, L.stream, counts, G, range_totals);
}

// Asks the L2 to fetch [base, base + bytes) (one prefetch per 128-byte
// line); the loads that follow find the lines there instead of missing at
// random.  A hint: nothing waits for it.
__global__ void __launch_bounds__(256) prefetch_l2_kernel(const char* __restrict__ base, int64_t bytes) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * 128;
  for (int64_t off = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 128; off < bytes; off += stride)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
}

void launch_prefetch_l2(const void* base, int64_t bytes, const Launch& L) {
  if (bytes <= 0) return;
  const int64_t lines = (bytes + 127) / 128;
  const int64_t want = (lines + 255) / 256;
  const int grid = static_cast<int>(want < L.grid_cap ? (want < 1 ? 1 : want) : L.grid_cap);
  prefetch_l2_kernel<<<grid, 256, 0, L.stream>>>(static_cast<const char*>(base), bytes);
}

// Four positions per thread: the dest loads, then the gathers, then the
// stores.  A gather follows one of P runs that each advance in order.
__global__ void __launch_bounds__(256) unpermute_kernel(const int32_t* __restrict__ dest, int64_t n,
                                                        const int32_t* __restrict__ idx_p,
                                                        const uint8_t* __restrict__ mask_p, int32_t* __restrict__ idx,
                                                        uint8_t* __restrict__ mask) {
  constexpr int U = 4;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * U;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x * U + threadIdx.x; base < n; base += step) {
    int32_t d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t pos = base + static_cast<int64_t>(u) * blockDim.x;
      d[u] = pos < n ? dest[pos] : 0;
    }
    int32_t i[U];
    uint8_t m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t pos = base + static_cast<int64_t>(u) * blockDim.x;
      i[u] = pos < n ? idx_p[d[u]] : 0;
      m[u] = pos < n ? mask_p[d[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t pos = base + static_cast<int64_t>(u) * blockDim.x;
      if (pos < n) {
        idx[pos] = i[u];
        mask[pos] = m[u];
      }
    }
  }
}

void launch_unpermute(const int32_t* dest, int64_t n, const int32_t* idx_p, const uint8_t* mask_p, int32_t* idx,
                      uint8_t* mask, const Launch& L) {
  TraceScope ts(kKUnpermute, L.stream);
  launch_dependent(unpermute_kernel, grid_for((n + 3) / 4, L), L.block, L.stream, dest, n, idx_p, mask_p, idx, mask);
}

// ----------------------------------------------------------- active listing
// Live indices are the complement of the heap's free part h[t..c) (the heap
// keeps active + free a permutation of 0..c-1).  Free indices are marked in a
// bitmap; one kernel then compacts the unmarked bits: each block owns 8192
// consecutive indices (one bitmap word per thread), ranks its live ones with a
// block scan and reserves its output range with one atomic.  Each block's output is an ascending run, so
// gathers over the list read the key and value buffers in long sequential
// runs.  No table scan is needed.
constexpr int kListThreads = 256;
constexpr int kListWordsPerBlock = kListThreads;  // one bitmap word (32 indices) per thread

// Also resets the listing counters that compact_live_kernel accumulates into.
__global__ void mark_free_kernel(const int32_t* __restrict__ heap, int64_t capacity, Ctrl* __restrict__ ctrl,
                                 uint32_t* __restrict__ words) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->count = 0;
    ctrl->list_done = 0;
  }
  const int64_t t = static_cast<int64_t>(static_cast<uint32_t>(ctrl->top_used));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = t + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < capacity; j += stride) {
    const uint32_t i = static_cast<uint32_t>(heap[j]);
    atomicOr(words + (i >> 5), 1u << (i & 31));
  }
}

// Reads and re-zeroes its bitmap words (so the next listing needs no
// clearing pass).  The last block to finish copies the total to *count_out
// when given (the live count, left on the device for asynchronous callers).
__global__ void __launch_bounds__(kListThreads) compact_live_kernel(uint32_t* __restrict__ words, int64_t capacity,
                                                                    Ctrl* ctrl, int32_t* __restrict__ out,
                                                                    int64_t out_cap, long long* count_out) {
  __shared__ int s_warp[33];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31;
  const int64_t wi = static_cast<int64_t>(blockIdx.x) * kListThreads + threadIdx.x;
  uint32_t live = ~words[wi];
  words[wi] = 0u;
  const int64_t lo = wi * 32;
  if (lo >= capacity) live = 0;
  else if (lo + 32 > capacity) live &= (1u << (capacity - lo)) - 1u;
  int total;
  const int off = block_exclusive_scan(__popc(live), total, s_warp);
  if (threadIdx.x == 0) s_base = total ? atomicAdd(&ctrl->count, static_cast<unsigned long long>(total)) : 0ull;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(s_base);
  const int64_t w0 = wi - lane;  // first word of this warp
  // the warp writes its 32 words one after another, one bit per lane, so each
  // store instruction covers a contiguous run of the output
  for (int w = 0; w < 32; ++w) {
    const uint32_t word = __shfl_sync(0xFFFFFFFFu, live, w);
    const int o = __shfl_sync(0xFFFFFFFFu, off, w);
    if ((word >> lane) & 1u) {
      const int64_t dst = base + o + __popc(word & ((1u << lane) - 1u));
      if (dst < out_cap) out[dst] = static_cast<int32_t>((w0 + w) * 32 + lane);
    }
  }
  if (count_out != nullptr && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long done = atomicAdd(&ctrl->list_done, 1ull);
    if (done == gridDim.x - 1) {
      __threadfence();
      *count_out = static_cast<long long>(atomicAdd(&ctrl->count, 0ull));
    }
  }
}

int64_t list_scratch_words(int64_t capacity) {
  const int64_t words = (capacity + 31) / 32;
  return (words + kListWordsPerBlock - 1) / kListWordsPerBlock * kListWordsPerBlock;
}

int64_t list_scratch_bytes(int64_t capacity) { return list_scratch_words(capacity) * 4; }

// Listing of a map whose heap's free part is the identity: the live indices
// are exactly 0..t-1 (the complement of h[t..c) = t..c-1), written in order
// with 16-byte stores, and the count is t.
__global__ void list_prefix_kernel(Ctrl* __restrict__ ctrl, int32_t* __restrict__ out, int64_t out_cap,
                                   long long* count_out) {
  const int64_t t = static_cast<int64_t>(static_cast<uint32_t>(ctrl->top_used));
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (tid == 0) {
    ctrl->count = static_cast<unsigned long long>(t);
    if (count_out) *count_out = static_cast<long long>(t);
  }
  const int64_t n = min(t, out_cap);
  const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  const int64_t n4 = vec ? n / 4 : 0;
  for (int64_t q = tid; q < n4; q += stride) {
    const int32_t v = static_cast<int32_t>(4 * q);
    reinterpret_cast<int4*>(out)[q] = make_int4(v, v + 1, v + 2, v + 3);
  }
  for (int64_t j = 4 * n4 + tid; j < n; j += stride) out[j] = static_cast<int32_t>(j);
}

void launch_list_active(bool heap_identity, const int32_t* heap, int64_t capacity, Ctrl* ctrl, void* scratch,
                        int32_t* out, int64_t out_cap, long long* count_out, const Launch& L) {
  if (heap_identity) {
    TraceScope ts(kKListActive, L.stream);
    const int64_t n = std::min(capacity, out_cap);
    list_prefix_kernel<<<grid_for((n + 3) / 4, L), L.block, 0, L.stream>>>(ctrl, out, out_cap, count_out);
    return;
  }
  const int64_t words = list_scratch_words(capacity);
  const int n_blocks = static_cast<int>(words / kListWordsPerBlock);
  uint32_t* bitmap = static_cast<uint32_t*>(scratch);  // all zero between listings
  TraceScope ts(kKListActive, L.stream, 2);
  const int64_t free_max = capacity;  // the kernel starts at the device-side heap top
  mark_free_kernel<<<grid_for(free_max, L), L.block, 0, L.stream>>>(heap, capacity, ctrl, bitmap);
  compact_live_kernel<<<n_blocks, kListThreads, 0, L.stream>>>(bitmap, capacity, ctrl, out, out_cap, count_out);
}

// ------------------------------------------------------------------- heap
// h[i] = i for i in [from, to): scalar head and tail, int4 stores between.
__global__ void iota_kernel(int32_t* __restrict__ h, int64_t from, int64_t to) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t a = min(to, (from + 3) & ~int64_t{3});  // first multiple of 4
  const int64_t b = max(a, to & ~int64_t{3});
  for (int64_t i = from + tid; i < a; i += stride) h[i] = static_cast<int32_t>(i);
  for (int64_t q = a / 4 + tid; q < b / 4; q += stride) {
    const int32_t v = static_cast<int32_t>(4 * q);
    reinterpret_cast<int4*>(h)[q] = make_int4(v, v + 1, v + 2, v + 3);
  }
  for (int64_t i = b + tid; i < to; i += stride) h[i] = static_cast<int32_t>(i);
}

void launch_iota(int32_t* h, int64_t from, int64_t to, const Launch& L) {
  if (to <= from) return;
  TraceScope ts(kKIota, L.stream);
  iota_kernel<<<grid_for((to - from + 3) / 4, L), L.block, 0, L.stream>>>(h, from, to);
}

__global__ void set_top_used_kernel(Ctrl* ctrl, unsigned long long top_used) { ctrl->top_used = top_used; }

// used slots := the listed live count (heap top unchanged), after a rebuild
// whose count only the device knows.
__global__ void set_used_from_count_kernel(Ctrl* ctrl) {
  const unsigned long long top = ctrl->top_used & 0xFFFFFFFFull;
  ctrl->top_used = (ctrl->count << 32) | top;
}

void launch_set_used_from_count(Ctrl* ctrl, const Launch& L) {
  TraceScope ts(kKSetCtrl, L.stream);
  set_used_from_count_kernel<<<1, 1, 0, L.stream>>>(ctrl);
}

__global__ void snapshot_kernel(Ctrl* ctrl, Snap* snap, uint32_t seq) {
  if (threadIdx.x == 0) publish_snapshot(ctrl, snap, seq);
}

void launch_snapshot(Ctrl* ctrl, Snap* snap, uint32_t seq, const Launch& L) {
  TraceScope ts(kKSetCtrl, L.stream);
  snapshot_kernel<<<1, 32, 0, L.stream>>>(ctrl, snap, seq);
}

void launch_set_top_used(Ctrl* ctrl, int64_t top, int64_t used, const Launch& L) {
  const unsigned long long v = (static_cast<unsigned long long>(used) << 32) | static_cast<unsigned long long>(top);
  TraceScope ts(kKSetCtrl, L.stream);
  set_top_used_kernel<<<1, 1, 0, L.stream>>>(ctrl, v);
}

// -------------------------------------------------------------- value rows
// Warp per input position: rows of winners (mask[p] == 1) are copied from
// src_j + p*row to dst_j + idx[p]*row, 32 lanes x vec bytes per step.
__global__ void __launch_bounds__(256) scatter_rows_kernel(ValueCopy vc, const int32_t* __restrict__ idx,
                                                           const uint8_t* __restrict__ mask, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    if (!mask[p]) continue;
    const int64_t i = idx[p];
#pragma unroll
    for (int j = 0; j < kMaxValues; ++j) {
      if (j < vc.n)
        copy_row(static_cast<char*>(vc.dst[j]) + i * vc.row_bytes[j],
                 static_cast<const char*>(vc.src[j]) + p * vc.row_bytes[j], vc.row_bytes[j], vc.vec[j], lane, 32);
    }
  }
}

void launch_scatter_rows(const ValueCopy& vc, const int32_t* idx, const uint8_t* mask, int64_t n, const Launch& L) {
  if (vc.n == 0 || n == 0) return;
  int64_t g = (n * 32 + L.block - 1) / L.block;
  if (g > L.grid_cap) g = L.grid_cap;
  TraceScope ts(kKScatterRows, L.stream);
  scatter_rows_kernel<<<static_cast<int>(g < 1 ? 1 : g), L.block, 0, L.stream>>>(vc, idx, mask, n);
}

// Warp per row: dst_j row r <- src_j row list[r] (compacting rehash).
__global__ void __launch_bounds__(256) gather_rows_kernel(ValueCopy vc, const int32_t* __restrict__ list, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int64_t a = list[r];
#pragma unroll
    for (int j = 0; j < kMaxValues; ++j) {
      if (j < vc.n)
        copy_row(static_cast<char*>(vc.dst[j]) + r * vc.row_bytes[j],
                 static_cast<const char*>(vc.src[j]) + a * vc.row_bytes[j], vc.row_bytes[j], vc.vec[j], lane, 32);
    }
  }
}

void launch_gather_rows(const ValueCopy& vc, const int32_t* list, int64_t n, const Launch& L) {
  if (vc.n == 0 || n == 0) return;
  int64_t g = (n * 32 + L.block - 1) / L.block;
  if (g > L.grid_cap) g = L.grid_cap;
  TraceScope ts(kKGatherRows, L.stream);
  gather_rows_kernel<<<static_cast<int>(g < 1 ? 1 : g), L.block, 0, L.stream>>>(vc, list, n);
}

// --------------------------------------------------------------- key gather
// Thread per output row: out[r, 0:d] = kB(indices[r]) (zeros for indices
// outside [0, capacity)).
// n_dev (optional): the number of rows on the device; the kernel gathers
// min(n, *n_dev) rows, so a gather can follow an asynchronous listing.
__global__ void gather_keys_kernel(const int32_t* __restrict__ kb, int ks, int d, int64_t capacity,
                                   const int32_t* __restrict__ indices, int64_t n,
                                   const long long* __restrict__ n_dev, int32_t* __restrict__ out) {
  if (n_dev) n = min(n, static_cast<int64_t>(*n_dev));
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int32_t i = __ldg(indices + r);
    const bool ok = i >= 0 && i < capacity;
    const int32_t* src = kb + static_cast<int64_t>(ok ? i : 0) * ks;
    int32_t* dst = out + r * d;
    if (ks == 4) {
      const int4 v = ok ? __ldg(reinterpret_cast<const int4*>(src)) : make_int4(0, 0, 0, 0);
      const int32_t a[4] = {v.x, v.y, v.z, v.w};
      for (int c = 0; c < d; ++c) dst[c] = a[c];
    } else {
      for (int c = 0; c < d; ++c) dst[c] = ok ? __ldg(src + c) : 0;
    }
  }
}

void launch_gather_keys(const int32_t* kb, int ks, int d, int64_t capacity, const int32_t* indices, int64_t n,
                        const long long* n_dev, int32_t* out, const Launch& L) {
  if (n == 0) return;
  TraceScope ts(kKGatherKeys, L.stream);
  gather_keys_kernel<<<grid_for(n, L), L.block, 0, L.stream>>>(kb, ks, d, capacity, indices, n, n_dev, out);
}

// Warp per output row: out row r <- value buffer row indices[r] (zeros for
// indices outside [0, capacity)).
__global__ void __launch_bounds__(256) gather_values_kernel(const char* __restrict__ src, int64_t row_bytes, int vec,
                                                            int64_t capacity, const int32_t* __restrict__ indices,
                                                            int64_t n, const long long* __restrict__ n_dev,
                                                            char* __restrict__ out) {
  if (n_dev) n = min(n, static_cast<int64_t>(*n_dev));
  const int lane = threadIdx.x & 31;
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int32_t i = indices[r];
    char* dst = out + r * row_bytes;
    if (i >= 0 && i < capacity) {
      copy_row(dst, src + static_cast<int64_t>(i) * row_bytes, row_bytes, vec, lane, 32);
    } else {
      for (int64_t b = lane; b < row_bytes; b += 32) dst[b] = 0;
    }
  }
}

void launch_gather_values(const void* src, int64_t row_bytes, int vec, int64_t capacity, const int32_t* indices,
                          int64_t n, const long long* n_dev, void* out, const Launch& L) {
  if (n == 0) return;
  TraceScope ts(kKGatherValues, L.stream);
  int64_t g = (n * 32 + L.block - 1) / L.block;
  if (g > L.grid_cap) g = L.grid_cap;
  gather_values_kernel<<<static_cast<int>(g < 1 ? 1 : g), L.block, 0, L.stream>>>(
      static_cast<const char*>(src), row_bytes, vec, capacity, indices, n, n_dev, static_cast<char*>(out));
}

// ------------------------------------------------------------- quantisation
// floor(p / cell) in float32 with IEEE division (this file is compiled without
// fast-math), then float -> int32 conversion rounding toward minus infinity
// (saturating outside the int32 range).
__global__ void quantize_kernel(const float* __restrict__ pts, int64_t n, int64_t n4, float cell,
                                int32_t* __restrict__ keys) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const float4* p4 = reinterpret_cast<const float4*>(pts);
  int4* k4 = reinterpret_cast<int4*>(keys);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = __ldcs(p4 + i);
    int4 o;
    o.x = __float2int_rd(__fdiv_rn(v.x, cell));
    o.y = __float2int_rd(__fdiv_rn(v.y, cell));
    o.z = __float2int_rd(__fdiv_rn(v.z, cell));
    o.w = __float2int_rd(__fdiv_rn(v.w, cell));
    __stcs(k4 + i, o);
  }
  for (int64_t i = 4 * n4 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    keys[i] = __float2int_rd(__fdiv_rn(pts[i], cell));
}

void launch_quantize(const float* pts, int64_t n, float cell, int32_t* keys, const Launch& L) {
  if (n == 0) return;
  // the float4 path needs both arrays 16-byte aligned
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(pts) | reinterpret_cast<uintptr_t>(keys)) & 15u) == 0;
  const int64_t n4 = vec_ok ? n / 4 : 0;
  TraceScope ts(kKQuantize, L.stream);
  quantize_kernel<<<grid_for((n + 3) / 4, L), L.block, 0, L.stream>>>(pts, n, n4, cell, keys);
}

// ----------------------------------------------------------- roofline probe
// Each thread performs reads at pseudo-random sector-aligned offsets (a
// splitmix64 sequence), XOR-folds them and writes one word per block, so the
// loads cannot be removed.  UNROLL independent reads are issued before any of
// them is used, so each thread keeps UNROLL requests in flight.
template <int SECTOR, int UNROLL>
__global__ void __launch_bounds__(256) probe_kernel(const uint64_t* __restrict__ buf, uint64_t n_sectors,
                                                    int64_t n_reads, uint32_t seed, uint32_t* __restrict__ sink,
                                                    int64_t sink_len) {
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint64_t acc = 0;
  for (int64_t r0 = tid * UNROLL; r0 < n_reads; r0 += nthreads * UNROLL) {
    uint64_t v[UNROLL][4];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t r = r0 + u;
      const uint64_t sec = __umul64hi(mix64(static_cast<uint64_t>(r) * 0x9E3779B97F4A7C15ull + seed), n_sectors);
      const uint64_t* p = buf + sec * (SECTOR / 8);
      if (r < n_reads) {
        load32<true>(p, v[u][0], v[u][1], v[u][2], v[u][3]);
        if constexpr (SECTOR == 64) {
          uint64_t a, b, c, d;
          load32<true>(p + 4, a, b, c, d);
          v[u][0] ^= a; v[u][1] ^= b; v[u][2] ^= c; v[u][3] ^= d;
        }
      } else {
        v[u][0] = v[u][1] = v[u][2] = v[u][3] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) acc ^= v[u][0] ^ v[u][1] ^ v[u][2] ^ v[u][3];
  }
  const uint32_t folded = static_cast<uint32_t>(acc ^ (acc >> 32));
  const int64_t slot = tid % sink_len;
  if (folded == 0x9E3779B9u) sink[slot] = folded;  // practically never taken; keeps the loads live
}

// Random 64-bit atomics on a table of 32-byte buckets (all slots start
// EMPTY = all ones).  mode 0: CAS EMPTY -> op id on a random slot;
// mode 1: the claim chain, a relaxed 32-byte bucket load then a CAS on the
// bucket's first EMPTY slot.  Each thread keeps one operation in flight.
template <int MODE>
__global__ void __launch_bounds__(256) probe_atomic_kernel(uint64_t* __restrict__ slots, uint64_t n_buckets,
                                                           int64_t n_ops, uint32_t seed, uint32_t* __restrict__ sink,
                                                           int64_t sink_len) {
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint64_t acc = 0;
  for (int64_t r = tid; r < n_ops; r += nthreads) {
    const uint64_t b = __umul64hi(mix64(static_cast<uint64_t>(r) * 0x9E3779B97F4A7C15ull + seed), n_buckets);
    uint64_t* bp = slots + 4 * b;
    if constexpr (MODE == 0) {
      const uint32_t s = static_cast<uint32_t>(mix64(static_cast<uint64_t>(r) + seed) & 3u);
      acc ^= atomicCAS(reinterpret_cast<unsigned long long*>(bp + s), ~0ull, static_cast<unsigned long long>(r));
    } else {
      uint64_t w0, w1, w2, w3;
      load32<false>(bp, w0, w1, w2, w3);
      int e = w3 == ~0ull ? 3 : 0;
      e = w2 == ~0ull ? 2 : e;
      e = w1 == ~0ull ? 1 : e;
      e = w0 == ~0ull ? 0 : e;
      acc ^= atomicCAS(reinterpret_cast<unsigned long long*>(bp + e), ~0ull, static_cast<unsigned long long>(r));
    }
  }
  const uint32_t folded = static_cast<uint32_t>(acc ^ (acc >> 32));
  if (folded == 0x9E3779B9u) sink[tid % sink_len] = folded;  // practically never taken; keeps the atomics live
}

void launch_probe_atomic(void* buf, int64_t buf_bytes, int64_t n_ops, int mode, uint32_t seed, uint32_t* sink,
                         int64_t sink_len, const Launch& L) {
  const uint64_t n_buckets = static_cast<uint64_t>(buf_bytes) / 32u;
  TraceScope ts(kKProbe, L.stream);
  if (mode == 0)
    probe_atomic_kernel<0><<<L.grid_cap, L.block, 0, L.stream>>>(static_cast<uint64_t*>(buf), n_buckets, n_ops, seed,
                                                                  sink, sink_len);
  else
    probe_atomic_kernel<1><<<L.grid_cap, L.block, 0, L.stream>>>(static_cast<uint64_t*>(buf), n_buckets, n_ops, seed,
                                                                  sink, sink_len);
}

void launch_probe(const void* buf, int64_t buf_bytes, int64_t n_reads, int sector, int loads_per_thread,
                  uint32_t seed, uint32_t* sink, int64_t sink_len, const Launch& L) {
  const uint64_t n_sectors = static_cast<uint64_t>(buf_bytes) / static_cast<uint64_t>(sector);
  const int grid = L.grid_cap;
  const uint64_t* b = static_cast<const uint64_t*>(buf);
  TraceScope ts(kKProbe, L.stream);
#define ASH_PROBE(SEC, U) probe_kernel<SEC, U><<<grid, L.block, 0, L.stream>>>(b, n_sectors, n_reads, seed, sink, sink_len)
  if (sector == 64) {
    if (loads_per_thread == 16) ASH_PROBE(64, 16);
    else if (loads_per_thread == 8) ASH_PROBE(64, 8);
    else ASH_PROBE(64, 4);
  } else {
    if (loads_per_thread == 16) ASH_PROBE(32, 16);
    else if (loads_per_thread == 8) ASH_PROBE(32, 8);
    else ASH_PROBE(32, 4);
  }
#undef ASH_PROBE
}

}  // namespace ash
