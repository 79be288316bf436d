// Device-side building blocks of the hash map: slot encoding, the key hash,
// key and bucket loads, and block-level aggregation of heap atomics.
//
// Table layout.  The table is an array of 64-bit slots grouped into buckets of
// S = 4, 8 or 16 slots (32, 64 or 128 bytes, aligned to the bucket size).
// A key hashes to a home bucket and probes buckets linearly from there.  A
// slot word is one of:
//   committed   hi = fingerprint (top bit set)   lo = buffer index (< 2^31)
//   claimed     hi = fingerprint                 lo = kClaimBit | input position
//               (only between the two insert kernels)
//   marked      hi = input position (< 2^31)     lo = buffer index
//               (only between the two erase kernels)
//   EMPTY       all ones
//   TOMBSTONE   hi = 0xFFFFFFFE, lo = all ones
// Keys themselves live only in the key buffer kB (Sec. 4.2 of the paper); the
// fingerprint filters slots so that a probe reads kB only on a likely match.
//
// Probe-chain invariant: a committed key stored in bucket b_j with home bucket
// b_0 leaves no EMPTY slot in any bucket b_0 .. b_{j-1} (linear order).  A
// lookup can therefore stop at the first bucket holding an EMPTY slot.
//
// Preferred slot.  Every key also names one slot of its home bucket, picked by
// the low fingerprint bits (pref_slot).  Placement tries that slot first and
// takes another EMPTY slot only once it is occupied.  Preferred-slot
// invariant: while a key is in the table (claimed or committed), the preferred
// slot of its home bucket is not EMPTY.  Inserts keep it because a slot only
// goes from EMPTY to occupied during an insert; erase keeps it by leaving a
// TOMBSTONE instead of EMPTY where another live key of the bucket prefers the
// freed slot; a rebuild places keys preferred-first into an empty table.  So
// an insert may CAS the preferred slot blindly, without loading the bucket:
// if the CAS finds EMPTY, the key was absent and is now claimed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ash {

constexpr uint64_t kEmpty = 0xFFFFFFFFFFFFFFFFull;
constexpr uint64_t kTombstone = 0xFFFFFFFEFFFFFFFFull;
constexpr uint32_t kNoIndex = 0xFFFFFFFFu;
constexpr uint32_t kClaimBit = 0x80000000u;
constexpr uint32_t kFpBit = 0x80000000u;

// Status bits raised by kernels (bit n = ash_status n).
constexpr int kStatusCapacity = 1 << 3;
constexpr int kStatusTableFull = 1 << 4;

// Control block of a map, in device memory.
struct Ctrl {
  // Low 32 bits: heap top t (live entries).  High 32 bits: used slots
  // (committed + tombstones).  One 64-bit atomic updates both.
  unsigned long long top_used;
  int status;
  unsigned int commit_done;   // blocks of a snapshotting commit that have finished
  unsigned long long count;   // listing counter
  unsigned long long list_done;  // blocks of a counting compaction that have finished
};

// Host-visible copy of a control block's counters, in mapped pinned memory:
// the device writes it after a batch (the last block of the insert's commit,
// or snapshot_kernel) so that the host can tighten its bounds on the live and
// used counts without synchronising.  One 16-byte store writes top_used and
// check = top_used ^ snap_tag(seq), seq being the number the host gave the
// write; the host takes the record once the two words agree for that number
// (a record not yet written, or half of a write, does not pass).  One 64-byte
// line per map.
struct Snap {
  unsigned long long top_used;
  unsigned long long check;
  unsigned long long pad[6];
};

// View of one map handed to kernels by value.
struct TableView {
  uint64_t* slots;
  int32_t* kb;          // key buffer, row stride ks (template parameter KS)
  int32_t* heap;        // index heap h
  Ctrl* ctrl;
  uint32_t n_buckets;
  uint32_t max_probes;
  int32_t capacity;
  int32_t flags;        // kViewHeapIdentity | kViewPrefPlaced
  // Winner flags of one insert (one bit per input position, zero before the
  // claim kernel), or null.  A position that displaces an equal key's claim
  // with a lower position sets the displaced position's bit, so after the
  // claim kernel a position holding a slot index wins unless its bit is set,
  // and the commit decides without reading the slot word.
  uint32_t* lost;
  // Where the insert's commit publishes the control block when it finishes
  // (null: no snapshot), and the sequence number of that write.
  Snap* snap;
  uint32_t snap_seq;
};

// TableView::flags: the free part of the heap is the identity (h[j] = j for
// j >= t), as it is from create or clear until the first erase.  Commit then
// takes index t + rank without reading h.
constexpr int32_t kViewHeapIdentity = 1;
// TableView::flags: the map keeps the preferred-slot invariant (no bucket-
// first or batched insert since create, clear or the last rebuild).  Erase
// must then keep it too; otherwise it may empty any slot of a bucket that
// has an EMPTY slot.
constexpr int32_t kViewPrefPlaced = 2;

constexpr int kMaxValues = 8;

// Value rows to copy from input position p to buffer index i.
struct ValueCopy {
  int n;
  int pad;
  void* dst[kMaxValues];
  const void* src[kMaxValues];
  int64_t row_bytes[kMaxValues];
  int vec[kMaxValues];  // widest of 16/8/4/2/1 bytes dividing row_bytes and both bases
};

__device__ __forceinline__ uint32_t lo32(uint64_t w) { return static_cast<uint32_t>(w); }
__device__ __forceinline__ uint32_t hi32(uint64_t w) { return static_cast<uint32_t>(w >> 32); }

// Key stride in kB: 1, 2, 4 or 8 int32 so that a key row is one aligned
// vector load (4, 8, 16 or 2x16 bytes).
template <int D>
struct KeyStride {
  static constexpr int value = D <= 1 ? 1 : (D <= 2 ? 2 : (D <= 4 ? 4 : 8));
};

// ------------------------------------------------------------------ hashing
// 64-bit hash of an int32 tuple: each coordinate times a distinct odd 64-bit
// constant, summed, then the splitmix64 finaliser (Steele et al. 2014) for
// avalanche.  The home bucket uses the high 32 bits (multiply-shift range
// reduction), the fingerprint the low 32 bits with the top bit forced on.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

// Check word of snapshot number seq (a bijection of seq, never 0).
__host__ __device__ __forceinline__ uint64_t snap_tag(uint32_t seq) {
  return mix64(static_cast<uint64_t>(seq) + 0x9E3779B97F4A7C15ull);
}

// Copies the control block's counters to a host-visible snapshot: top_used
// is read at L2 (the atomics of this kernel and earlier ones are all there),
// then one 16-byte store writes it with its check word.
__device__ __forceinline__ void publish_snapshot(Ctrl* ctrl, Snap* snap, uint32_t seq) {
  const unsigned long long tu = atomicAdd(&ctrl->top_used, 0ull);
  *reinterpret_cast<ulonglong2*>(snap) = make_ulonglong2(tu, tu ^ snap_tag(seq));
}

__device__ __forceinline__ uint64_t coord_mult(int j) {
  // distinct odd constants (fractional parts of golden ratio / sqrt primes)
  switch (j) {
    case 0: return 0x9E3779B97F4A7C15ull;
    case 1: return 0xC2B2AE3D27D4EB4Full;
    case 2: return 0x165667B19E3779F9ull;
    case 3: return 0xD6E8FEB86659FD93ull;
    case 4: return 0xFF51AFD7ED558CCDull;
    case 5: return 0xC4CEB9FE1A85EC53ull;
    case 6: return 0x2545F4914F6CDD1Dull;
    default: return 0x27D4EB2F165667C5ull;
  }
}

template <int D>
__device__ __forceinline__ uint64_t hash_key(const int32_t (&k)[D]) {
  uint64_t h = static_cast<uint64_t>(D);
#pragma unroll
  for (int j = 0; j < D; ++j) h += static_cast<uint64_t>(static_cast<uint32_t>(k[j])) * coord_mult(j);
  return mix64(h);
}

__device__ __forceinline__ uint32_t fingerprint(uint64_t h) { return lo32(h) | kFpBit; }

// Preferred slot of a key within its home bucket (S a power of two).  The
// home bucket uses the hash's high word, this the fingerprint's low bits.
template <int S>
__device__ __forceinline__ uint32_t pref_slot(uint32_t fp) { return fp & static_cast<uint32_t>(S - 1); }

// A committed slot word: the only kind with the top bit of hi set and the
// top bit of lo clear (claimed, EMPTY and TOMBSTONE words set lo's top bit,
// marked words clear hi's).
__device__ __forceinline__ bool is_committed(uint64_t w) {
  return (hi32(w) & kFpBit) && !(lo32(w) & kClaimBit);
}

__device__ __forceinline__ uint32_t home_bucket(uint64_t h, uint32_t n_buckets) {
  return __umulhi(hi32(h), n_buckets);
}

__device__ __forceinline__ uint32_t next_bucket(uint32_t b, uint32_t n_buckets) {
  return (b + 1 == n_buckets) ? 0u : b + 1;
}

// --------------------------------------------------------------------- keys
template <int D>
__device__ __forceinline__ void load_input_key(const int32_t* __restrict__ keys, int64_t pos, int32_t (&k)[D]) {
  const int32_t* p = keys + pos * D;
#pragma unroll
  for (int j = 0; j < D; ++j) k[j] = __ldg(p + j);
}

// Input rows given as float32 points [n, D], quantised where they are read:
// key = floor(p / cell) per coordinate with an IEEE float32 division and
// rounding toward minus infinity (the voxel key of Sec. 6.1, bit-identical to
// the quantisation kernel), so no key array is written or read.
struct PointRows {
  const float* p;
  float cell;
};

template <int D>
__device__ __forceinline__ void load_input_key(const PointRows& in, int64_t pos, int32_t (&k)[D]) {
  const float* q = in.p + pos * D;
#pragma unroll
  for (int j = 0; j < D; ++j) k[j] = __float2int_rd(__fdiv_rn(__ldg(q + j), in.cell));
}

template <int D, class In>
__device__ __forceinline__ bool input_key_equal(const In& keys, int64_t pos, const int32_t (&k)[D]) {
  int32_t o[D];
  load_input_key<D>(keys, pos, o);
  bool eq = true;
#pragma unroll
  for (int j = 0; j < D; ++j) eq &= (o[j] == k[j]);
  return eq;
}

// Loads row i of kB into o (KS values; the first D are the key).
template <int D>
__device__ __forceinline__ void load_kb(const int32_t* kb, uint32_t i, int32_t (&o)[KeyStride<D>::value]) {
  constexpr int KS = KeyStride<D>::value;
  const int32_t* p = kb + static_cast<size_t>(i) * KS;
  if constexpr (KS == 1) {
    o[0] = __ldg(p);
  } else if constexpr (KS == 2) {
    int2 v = __ldg(reinterpret_cast<const int2*>(p));
    o[0] = v.x; o[1] = v.y;
  } else if constexpr (KS == 4) {
    int4 v = __ldg(reinterpret_cast<const int4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    int4 v0 = __ldg(reinterpret_cast<const int4*>(p));
    int4 v1 = __ldg(reinterpret_cast<const int4*>(p) + 1);
    o[0] = v0.x; o[1] = v0.y; o[2] = v0.z; o[3] = v0.w;
    o[4] = v1.x; o[5] = v1.y; o[6] = v1.z; o[7] = v1.w;
  }
}

template <int D>
__device__ __forceinline__ bool kb_equal(const int32_t* kb, uint32_t i, const int32_t (&k)[D]) {
  int32_t o[KeyStride<D>::value];
  load_kb<D>(kb, i, o);
  bool eq = true;
#pragma unroll
  for (int j = 0; j < D; ++j) eq &= (o[j] == k[j]);
  return eq;
}

// Stores key k as row i of kB, padding coordinates set to zero.
template <int D>
__device__ __forceinline__ void store_kb(int32_t* kb, uint32_t i, const int32_t (&k)[D]) {
  constexpr int KS = KeyStride<D>::value;
  int32_t o[KS];
#pragma unroll
  for (int j = 0; j < KS; ++j) o[j] = j < D ? k[j] : 0;
  int32_t* p = kb + static_cast<size_t>(i) * KS;
  if constexpr (KS == 1) {
    p[0] = o[0];
  } else if constexpr (KS == 2) {
    *reinterpret_cast<int2*>(p) = make_int2(o[0], o[1]);
  } else if constexpr (KS == 4) {
    *reinterpret_cast<int4*>(p) = make_int4(o[0], o[1], o[2], o[3]);
  } else {
    reinterpret_cast<int4*>(p)[0] = make_int4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<int4*>(p)[1] = make_int4(o[4], o[5], o[6], o[7]);
  }
}

// ------------------------------------------------------------------ buckets
// 32-byte pieces of a bucket.  READ_ONLY loads (find, no writer in the same
// kernel) use the non-coherent path without L1 allocation; the others are
// relaxed GPU-scope loads that observe atomics of concurrent threads.
template <bool READ_ONLY>
__device__ __forceinline__ void load32(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
  if constexpr (READ_ONLY) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                 : "l"(p));
  } else {
    asm volatile("ld.relaxed.gpu.global.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                 : "l"(p)
                 : "memory");
  }
}

template <int S, bool READ_ONLY>
__device__ __forceinline__ void load_bucket(const uint64_t* bp, uint64_t (&w)[S]) {
#pragma unroll
  for (int q = 0; q < S / 4; ++q) load32<READ_ONLY>(bp + 4 * q, w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

__device__ __forceinline__ uint64_t load_slot_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// --------------------------------------------------------------- aggregation
// Block-wide exclusive rank of threads with `flag` set and the block total.
// Every thread of the block must call it (it contains __syncthreads).
// `s_warp` needs blockDim.x / 32 + 1 ints of shared memory.
__device__ __forceinline__ void block_rank(bool flag, int& rank, int& total, int* s_warp) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int n_warps = blockDim.x >> 5;
  const unsigned ballot = __ballot_sync(0xFFFFFFFFu, flag);
  if (lane == 0) s_warp[warp] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < n_warps; ++w) {
      int c = s_warp[w];
      s_warp[w] = acc;
      acc += c;
    }
    s_warp[n_warps] = acc;
  }
  __syncthreads();
  rank = s_warp[warp] + __popc(ballot & ((1u << lane) - 1u));
  total = s_warp[n_warps];
}

// Block-wide exclusive scan of a small per-thread count; returns this
// thread's offset and sets the block total.  Every thread of the block must
// call it (it contains __syncthreads).
__device__ __forceinline__ int block_exclusive_scan(int v, int& total, int* s_warp) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int n_warps = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < n_warps; ++w) {
      const int c = s_warp[w];
      s_warp[w] = acc;
      acc += c;
    }
    s_warp[n_warps] = acc;
  }
  __syncthreads();
  total = s_warp[n_warps];
  return s_warp[warp] + x - v;
}

__device__ __forceinline__ int block_count(bool flag, int* s_cnt) {
  const unsigned ballot = __ballot_sync(0xFFFFFFFFu, flag);
  if (threadIdx.x == 0) *s_cnt = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(s_cnt, __popc(ballot));
  __syncthreads();
  return *s_cnt;
}

// ---------------------------------------------------------------- value rows
template <typename T>
__device__ __forceinline__ void copy_elems(void* dst, const void* src, int64_t n_elems, int64_t start, int64_t step) {
  T* d = static_cast<T*>(dst);
  const T* s = static_cast<const T*>(src);
  for (int64_t e = start; e < n_elems; e += step) d[e] = s[e];
}

// Copies one row of `bytes` bytes with vector width `vec`, elements
// start, start+step, ... (step = 1 for one thread, 32 for a warp).
__device__ __forceinline__ void copy_row(void* dst, const void* src, int64_t bytes, int vec, int64_t start, int64_t step) {
  switch (vec) {
    case 16: copy_elems<uint4>(dst, src, bytes / 16, start, step); break;
    case 8: copy_elems<uint2>(dst, src, bytes / 8, start, step); break;
    case 4: copy_elems<uint32_t>(dst, src, bytes / 4, start, step); break;
    case 2: copy_elems<uint16_t>(dst, src, bytes / 2, start, step); break;
    default: copy_elems<uint8_t>(dst, src, bytes, start, step); break;
  }
}

}  // namespace ash
