// Hash map kernels, templated on the key dimension D and the bucket size S.
//
// find            one thread per query key: hash, probe buckets from the home
//                 bucket, verify fingerprint matches against kB (Eq. (4)).
// insert/activate two kernels (Sec. 4.3.1 lazy insertion, redesigned):
//   claim         one thread per input key.  A key already committed is
//                 rejected.  Otherwise the thread claims the first EMPTY slot
//                 of its probe sequence with a CAS writing {fingerprint,
//                 kClaimBit | input position}.  A thread that meets a claimed
//                 slot compares its key with the READ-ONLY input row of the
//                 claimant (never with a half-written kB row, which removes the
//                 torn-copy race of Sec. 4.4.2) and, if equal, lowers the
//                 recorded position with atomicMin.  After the kernel each
//                 claimed slot names the lowest input position of its key.
//                 The slot index goes to buf_indices[p] as scratch.
//   commit        one thread per input key: the position named by its slot
//                 wins, takes a buffer index from the heap (one atomicAdd per
//                 block on t, Sec. 4.3), writes kB(i) and small value rows,
//                 then replaces the claim with {fingerprint, i}.  Only winners
//                 allocate ("allocate only on success", Sec. 4.3.1).
// erase           two kernels: mark (atomicMin of the input position into the
//                 slot's high word, keeping the buffer index) and resolve (the
//                 lowest position wins, frees the index with one atomic per
//                 block, and empties the slot, or leaves a tombstone when its
//                 bucket holds no EMPTY slot).  Allocation and free never run
//                 in the same kernel (the atomicAdd/atomicSub conflict that
//                 Sec. 4.3.1 warns about).
// rebuild         inserts already-unique keys (rehash, Sec. 4.5) into an empty
//                 table: first EMPTY slot wins, no key comparisons.
#pragma once

#include "ash_device.cuh"
#include "ash_trace.h"

namespace ash {

// ---------------------------------------------------------------------- find
template <int D, int S>
__global__ void __launch_bounds__(256) find_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                   int32_t* __restrict__ idx, uint8_t* __restrict__ mask) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t pos = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; pos < n; pos += stride) {
    int32_t k[D];
    load_input_key<D>(keys, pos, k);
    const uint64_t h = hash_key<D>(k);
    const uint32_t fp = fingerprint(h);
    uint32_t b = home_bucket(h, t.n_buckets);
    int32_t out = -1;
    for (uint32_t probe = 0; probe < t.max_probes; ++probe) {
      uint64_t w[S];
      load_bucket<S, true>(t.slots + static_cast<size_t>(b) * S, w);
      bool stop = false;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        stop |= (w[s] == kEmpty);
        if (out < 0 && hi32(w[s]) == fp && lo32(w[s]) < kClaimBit) {
          if (kb_equal<D>(t.kb, lo32(w[s]), k)) out = static_cast<int32_t>(lo32(w[s]));
        }
      }
      if (out >= 0 || stop) break;
      b = next_bucket(b, t.n_buckets);
    }
    idx[pos] = out;
    mask[pos] = out >= 0 ? 1 : 0;
  }
}

// ------------------------------------------------------------- insert: claim
// Result codes written to buf_indices[p] by the claim kernel.
constexpr int32_t kClaimExists = -2;  // key already committed
constexpr int32_t kClaimFailed = -1;  // no slot within max_probes

// 0: no match.  1: slot claimed by an equal key in this batch.  2: committed equal key.
template <int D>
__device__ __forceinline__ int claim_match(uint64_t w, uint32_t fp, const int32_t (&k)[D],
                                           const int32_t* __restrict__ keys, const int32_t* kb) {
  const uint32_t lo = lo32(w);
  if (lo == kNoIndex || hi32(w) != fp) return 0;
  if (lo & kClaimBit) return input_key_equal<D>(keys, lo & ~kClaimBit, k) ? 1 : 0;
  return kb_equal<D>(kb, lo, k) ? 2 : 0;
}

template <int D, int S>
__device__ __forceinline__ int32_t claim_one(const TableView& t, const int32_t* __restrict__ keys, int64_t pos) {
  int32_t k[D];
  load_input_key<D>(keys, pos, k);
  const uint64_t h = hash_key<D>(k);
  const uint32_t fp = fingerprint(h);
  const uint64_t mine = (static_cast<uint64_t>(fp) << 32) | (kClaimBit | static_cast<uint32_t>(pos));
  uint32_t b = home_bucket(h, t.n_buckets);
  for (uint32_t probe = 0; probe < t.max_probes; ++probe) {
    uint64_t* bp = t.slots + static_cast<size_t>(b) * S;
    uint64_t w[S];
    load_bucket<S, false>(bp, w);
    // 1) an equal key already in the bucket (claimed or committed)
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int m = claim_match<D>(w[s], fp, k, keys, t.kb);
      if (m == 2) return kClaimExists;
      if (m == 1) {
        if ((lo32(w[s]) & ~kClaimBit) > static_cast<uint32_t>(pos))
          atomicMin(reinterpret_cast<unsigned long long*>(bp + s), static_cast<unsigned long long>(mine));
        return static_cast<int32_t>(b * S + s);
      }
    }
    // 2) claim the EMPTY slots of the bucket in order; a lost CAS re-checks
    //    the winner's word for an equal key
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (w[s] == kEmpty) {
        const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(bp + s),
                                       static_cast<unsigned long long>(kEmpty),
                                       static_cast<unsigned long long>(mine));
        if (old == kEmpty) return static_cast<int32_t>(b * S + s);
        const int m = claim_match<D>(old, fp, k, keys, t.kb);
        if (m == 2) return kClaimExists;
        if (m == 1) {
          if ((lo32(old) & ~kClaimBit) > static_cast<uint32_t>(pos))
            atomicMin(reinterpret_cast<unsigned long long*>(bp + s), static_cast<unsigned long long>(mine));
          return static_cast<int32_t>(b * S + s);
        }
      }
    }
    b = next_bucket(b, t.n_buckets);
  }
  atomicOr(&t.ctrl->status, kStatusTableFull);
  return kClaimFailed;
}

template <int D, int S>
__global__ void __launch_bounds__(256) claim_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                    int32_t* __restrict__ slot_out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t pos = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; pos < n; pos += stride)
    slot_out[pos] = claim_one<D, S>(t, keys, pos);
}

// ------------------------------------------------------------ insert: commit
template <int D>
__global__ void __launch_bounds__(256, 4) commit_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                     int32_t* __restrict__ idx, uint8_t* __restrict__ mask,
                                                     ValueCopy vc) {
  __shared__ int s_warp[33];
  __shared__ int s_base;
  __shared__ int s_got;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t pos = base + threadIdx.x;
    const bool active = pos < n;
    const int32_t s = active ? idx[pos] : -1;
    uint64_t w = 0;
    bool win = false;
    if (s >= 0) {
      w = load_slot_relaxed(t.slots + s);
      win = (lo32(w) == (kClaimBit | static_cast<uint32_t>(pos)));
    }
    int rank, total;
    block_rank(win, rank, total, s_warp);
    if (threadIdx.x == 0) {
      int got = 0, top = 0;
      if (total > 0) {
        const unsigned long long add = (static_cast<unsigned long long>(total) << 32) | static_cast<unsigned long long>(total);
        const unsigned long long old = atomicAdd(&t.ctrl->top_used, add);
        top = static_cast<int>(static_cast<uint32_t>(old));
        got = t.capacity - top;
        got = got < 0 ? 0 : (got > total ? total : got);
        if (got < total) {
          // give back the part of t that the heap could not serve
          atomicAdd(&t.ctrl->top_used, 0ull - static_cast<unsigned long long>(total - got));
          atomicOr(&t.ctrl->status, kStatusCapacity);
        }
      }
      s_base = top;
      s_got = got;
    }
    __syncthreads();
    if (win) {
      if (rank < s_got) {
        const int32_t i = t.heap[s_base + rank];
        int32_t k[D];
        load_input_key<D>(keys, pos, k);
        store_kb<D>(t.kb, static_cast<uint32_t>(i), k);
#pragma unroll
        for (int j = 0; j < kMaxValues; ++j) {
          if (j < vc.n)
            copy_row(static_cast<char*>(vc.dst[j]) + static_cast<int64_t>(i) * vc.row_bytes[j],
                     static_cast<const char*>(vc.src[j]) + pos * vc.row_bytes[j], vc.row_bytes[j], vc.vec[j], 0, 1);
        }
        t.slots[s] = (static_cast<uint64_t>(hi32(w)) << 32) | static_cast<uint32_t>(i);
        idx[pos] = i;
        mask[pos] = 1;
      } else {
        t.slots[s] = kTombstone;
        idx[pos] = -1;
        mask[pos] = 0;
      }
    } else if (active) {
      idx[pos] = -1;
      mask[pos] = 0;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- erase: mark
template <int D, int S>
__global__ void __launch_bounds__(256) erase_mark_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                         int32_t* __restrict__ slot_out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t pos = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; pos < n; pos += stride) {
    int32_t k[D];
    load_input_key<D>(keys, pos, k);
    const uint64_t h = hash_key<D>(k);
    const uint32_t fp = fingerprint(h);
    uint32_t b = home_bucket(h, t.n_buckets);
    int32_t res = -1;
    for (uint32_t probe = 0; probe < t.max_probes && res < 0; ++probe) {
      uint64_t* bp = t.slots + static_cast<size_t>(b) * S;
      uint64_t w[S];
      load_bucket<S, false>(bp, w);
      bool stop = false;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        stop |= (w[s] == kEmpty);
        const uint32_t lo = lo32(w[s]), hi = hi32(w[s]);
        // committed with an equal fingerprint, or already marked (fingerprint gone)
        if (res < 0 && lo < kClaimBit && (hi == fp || hi < kFpBit) && kb_equal<D>(t.kb, lo, k)) {
          if (hi > static_cast<uint32_t>(pos))
            atomicMin(reinterpret_cast<unsigned long long*>(bp + s),
                      (static_cast<unsigned long long>(pos) << 32) | lo);
          res = static_cast<int32_t>(b * S + s);
        }
      }
      if (stop) break;
      b = next_bucket(b, t.n_buckets);
    }
    slot_out[pos] = res;
  }
}

// ------------------------------------------------------------ erase: resolve
template <int S>
__global__ void __launch_bounds__(256) erase_resolve_kernel(TableView t, int64_t n, const int32_t* __restrict__ slot_in,
                                                            uint8_t* __restrict__ mask) {
  __shared__ int s_warp[33];
  __shared__ int s_cnt;
  __shared__ int s_base;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
    const int64_t pos = base + threadIdx.x;
    const bool active = pos < n;
    const int32_t s = active ? slot_in[pos] : -1;
    uint64_t w = 0;
    bool win = false, to_empty = false;
    if (s >= 0) {
      w = load_slot_relaxed(t.slots + s);
      win = hi32(w) == static_cast<uint32_t>(pos);
      if (win) {
        uint64_t bw[S];
        load_bucket<S, false>(t.slots + static_cast<size_t>(s / S) * S, bw);
#pragma unroll
        for (int q = 0; q < S; ++q) to_empty |= (bw[q] == kEmpty);
      }
    }
    int rank, total;
    block_rank(win, rank, total, s_warp);
    const int n_empty = block_count(to_empty, &s_cnt);
    if (threadIdx.x == 0) {
      int top = 0;
      if (total > 0) {
        const unsigned long long sub = (static_cast<unsigned long long>(n_empty) << 32) + static_cast<unsigned long long>(total);
        const unsigned long long old = atomicAdd(&t.ctrl->top_used, 0ull - sub);
        top = static_cast<int>(static_cast<uint32_t>(old));
      }
      s_base = top - total;
    }
    __syncthreads();
    if (win) {
      t.heap[s_base + rank] = static_cast<int32_t>(lo32(w));
      t.slots[s] = to_empty ? kEmpty : kTombstone;
      mask[pos] = 1;
    } else if (active) {
      mask[pos] = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ rebuild
// Inserts n unique keys taken from kb_src rows list[j] into an empty table.
// preserve: the entry keeps buffer index list[j]; otherwise it becomes j.
// The key row is copied to kb_dst when kb_dst != kb_src or !preserve.
template <int D, int S>
__global__ void __launch_bounds__(256) rebuild_kernel(TableView t, const int32_t* __restrict__ kb_src,
                                                      const int32_t* __restrict__ list, int64_t n, int preserve,
                                                      int copy_keys) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
    const uint32_t a = static_cast<uint32_t>(list[j]);
    int32_t row[KeyStride<D>::value];
    load_kb<D>(kb_src, a, row);
    int32_t k[D];
#pragma unroll
    for (int c = 0; c < D; ++c) k[c] = row[c];
    const uint32_t i = preserve ? a : static_cast<uint32_t>(j);
    const uint64_t h = hash_key<D>(k);
    const uint64_t word = (static_cast<uint64_t>(fingerprint(h)) << 32) | i;
    uint32_t b = home_bucket(h, t.n_buckets);
    bool placed = false;
    for (uint32_t probe = 0; probe < t.max_probes && !placed; ++probe) {
      uint64_t* bp = t.slots + static_cast<size_t>(b) * S;
      uint64_t w[S];
      load_bucket<S, false>(bp, w);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (!placed && w[s] == kEmpty) {
          const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(bp + s),
                                         static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(word));
          placed = (old == kEmpty);
        }
      }
      b = next_bucket(b, t.n_buckets);
    }
    if (!placed) atomicOr(&t.ctrl->status, kStatusTableFull);
    if (copy_keys) store_kb<D>(t.kb, i, k);
  }
}

// ----------------------------------------------------------------- launchers
struct Launch {
  cudaStream_t stream;
  int grid_cap;  // SMs x blocks_per_sm
  int block;
};

inline int grid_for(int64_t n, const Launch& L) {
  int64_t g = (n + L.block - 1) / L.block;
  if (g > L.grid_cap) g = L.grid_cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

// Function table for one key dimension (filled in by ash_dim<D>.cu).
struct DimKernels {
  void (*find)(int S, const TableView&, const int32_t*, int64_t, int32_t*, uint8_t*, const Launch&);
  void (*claim)(int S, const TableView&, const int32_t*, int64_t, int32_t*, const Launch&);
  void (*commit)(const TableView&, const int32_t*, int64_t, int32_t*, uint8_t*, const ValueCopy&, const Launch&);
  void (*erase_mark)(int S, const TableView&, const int32_t*, int64_t, int32_t*, const Launch&);
  void (*rebuild)(int S, const TableView&, const int32_t*, const int32_t*, int64_t, int, int, const Launch&);
};

template <int D>
struct DimLaunchers {
  template <int S>
  static void find_s(const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask, const Launch& L) {
    TraceScope ts(kKFind, L.stream);
    find_kernel<D, S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, keys, n, idx, mask);
  }
  static void find(int S, const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask, const Launch& L) {
    if (S == 4) find_s<4>(t, keys, n, idx, mask, L);
    else if (S == 8) find_s<8>(t, keys, n, idx, mask, L);
    else find_s<16>(t, keys, n, idx, mask, L);
  }
  template <int S>
  static void claim_s(const TableView& t, const int32_t* keys, int64_t n, int32_t* slot_out, const Launch& L) {
    TraceScope ts(kKClaim, L.stream);
    claim_kernel<D, S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, keys, n, slot_out);
  }
  static void claim(int S, const TableView& t, const int32_t* keys, int64_t n, int32_t* slot_out, const Launch& L) {
    if (S == 4) claim_s<4>(t, keys, n, slot_out, L);
    else if (S == 8) claim_s<8>(t, keys, n, slot_out, L);
    else claim_s<16>(t, keys, n, slot_out, L);
  }
  static void commit(const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask,
                     const ValueCopy& vc, const Launch& L) {
    TraceScope ts(kKCommit, L.stream);
    commit_kernel<D><<<grid_for(n, L), L.block, 0, L.stream>>>(t, keys, n, idx, mask, vc);
  }
  template <int S>
  static void erase_mark_s(const TableView& t, const int32_t* keys, int64_t n, int32_t* slot_out, const Launch& L) {
    TraceScope ts(kKEraseMark, L.stream);
    erase_mark_kernel<D, S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, keys, n, slot_out);
  }
  static void erase_mark(int S, const TableView& t, const int32_t* keys, int64_t n, int32_t* slot_out, const Launch& L) {
    if (S == 4) erase_mark_s<4>(t, keys, n, slot_out, L);
    else if (S == 8) erase_mark_s<8>(t, keys, n, slot_out, L);
    else erase_mark_s<16>(t, keys, n, slot_out, L);
  }
  template <int S>
  static void rebuild_s(const TableView& t, const int32_t* kb_src, const int32_t* list, int64_t n, int preserve,
                        int copy_keys, const Launch& L) {
    TraceScope ts(kKRebuild, L.stream);
    rebuild_kernel<D, S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, kb_src, list, n, preserve, copy_keys);
  }
  static void rebuild(int S, const TableView& t, const int32_t* kb_src, const int32_t* list, int64_t n, int preserve,
                      int copy_keys, const Launch& L) {
    if (S == 4) rebuild_s<4>(t, kb_src, list, n, preserve, copy_keys, L);
    else if (S == 8) rebuild_s<8>(t, kb_src, list, n, preserve, copy_keys, L);
    else rebuild_s<16>(t, kb_src, list, n, preserve, copy_keys, L);
  }
  static DimKernels table() {
    DimKernels k;
    k.find = &find;
    k.claim = &claim;
    k.commit = &commit;
    k.erase_mark = &erase_mark;
    k.rebuild = &rebuild;
    return k;
  }
};

// Defined in ash_dim<D>.cu.
DimKernels dim_kernels_1();
DimKernels dim_kernels_2();
DimKernels dim_kernels_3();
DimKernels dim_kernels_4();
DimKernels dim_kernels_5();
DimKernels dim_kernels_6();
DimKernels dim_kernels_7();
DimKernels dim_kernels_8();

// Defined in ash_aux.cu.
void launch_erase_resolve(int S, const TableView& t, int64_t n, const int32_t* slot_in, uint8_t* mask, const Launch& L);

}  // namespace ash
