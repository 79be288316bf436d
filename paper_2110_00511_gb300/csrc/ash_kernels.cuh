// Hash map kernels, templated on the key dimension D and the bucket size S.
//
// find            KPT query keys per thread: hash, load the home buckets of all
//                 KPT keys back to back, verify the fingerprint match of each
//                 against kB (Eq. (4)); keys that overflow their home bucket
//                 take the scalar probe loop.
// insert/activate two kernels (Sec. 4.3.1 lazy insertion, redesigned):
//   claim         a key already committed is rejected.  Otherwise the thread
//                 claims an EMPTY slot with a CAS writing {fingerprint,
//                 kClaimBit | input position}: either the key's preferred
//                 slot of its home bucket, CASed with no load before it
//                 (claim_pref_kernel, while the table fits in L2; keys that
//                 find it taken are queued per warp and claimed from their
//                 buckets in dense rounds), or the first EMPTY slot of the
//                 loaded home bucket (claim_bucket_kernel).  A thread that
//                 meets a claimed slot compares its key with the READ-ONLY
//                 input row of the claimant (never with a half-written kB
//                 row, which removes the torn-copy race of Sec. 4.4.2) and,
//                 if equal, lowers the recorded position with atomicMin,
//                 marking the position it displaced in the winner flags.
//                 After the kernel each claimed slot names the lowest input
//                 position of its key.  The slot index goes to
//                 buf_indices[p] as scratch.
//   commit        one thread per input key: a position holding a slot index
//                 whose winner flag is clear wins, takes a buffer index from
//                 the heap (one atomicAdd per block on t, Sec. 4.3), writes
//                 kB(i) and small value rows, then replaces the claim with
//                 {fingerprint, i}.  Only winners allocate ("allocate only on
//                 success", Sec. 4.3.1).
// erase           two kernels: mark (atomicMin of the input position into the
//                 slot's high word, keeping the buffer index) and resolve (the
//                 lowest position wins, frees the index with one atomic per
//                 block, and empties the slot, or leaves a tombstone when its
//                 bucket holds no EMPTY slot or, under the preferred-slot
//                 invariant, another live key prefers it).  Allocation and
//                 free never run in the same kernel (the atomicAdd/atomicSub
//                 conflict that Sec. 4.3.1 warns about).
// rebuild         inserts already-unique keys (rehash, Sec. 4.5) into an empty
//                 table: the preferred slot first, else the first EMPTY slot
//                 of the probe sequence, no key comparisons.
#pragma once

#include "ash_device.cuh"
#include "ash_trace.h"

namespace ash {

// ---------------------------------------------------------------------- find
// Scalar lookup of key k from its home bucket.
template <int D, int S>
__device__ __forceinline__ int32_t find_key(const TableView& t, const int32_t (&k)[D]) {
  const uint64_t h = hash_key<D>(k);
  const uint32_t fp = fingerprint(h);
  uint32_t b = home_bucket(h, t.n_buckets);
  for (uint32_t probe = 0; probe < t.max_probes; ++probe) {
    uint64_t w[S];
    load_bucket<S, true>(t.slots + static_cast<size_t>(b) * S, w);
    bool stop = false;
    int32_t out = -1;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      stop |= (w[s] == kEmpty);
      if (out < 0 && hi32(w[s]) == fp && lo32(w[s]) < kClaimBit && kb_equal<D>(t.kb, lo32(w[s]), k))
        out = static_cast<int32_t>(lo32(w[s]));
    }
    if (out >= 0) return out;
    if (stop) return -1;
    b = next_bucket(b, t.n_buckets);
  }
  return -1;
}

// Scalar lookup of input row pos (the slow path of find).
template <int D, int S, class In>
__device__ __noinline__ int32_t find_one(const TableView t, const In keys, int64_t pos) {
  int32_t k[D];
  load_input_key<D>(keys, pos, k);
  return find_key<D, S>(t, k);
}

// Radius neighbour query (the radius search of Sec. 6.2): thread per (query,
// offset) pair.  Offsets enumerate [-radius, radius]^D row-major (the last
// coordinate fastest) and are added with int32 wrap-around; the (2r+1)^D
// query keys are never materialised.  Outputs are [n, (2r+1)^D].
template <int D, int S>
__global__ void __launch_bounds__(256) neighbors_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                        int radius, int64_t n_off, int32_t* __restrict__ idx,
                                                        uint8_t* __restrict__ mask) {
  const int64_t total = n * n_off;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int width = 2 * radius + 1;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t r = e / n_off;
    int64_t o = e - r * n_off;
    int32_t k[D];
    load_input_key<D>(keys, r, k);
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
      const int digit = static_cast<int>(o % width);
      o /= width;
      k[j] = static_cast<int32_t>(static_cast<uint32_t>(k[j]) + static_cast<uint32_t>(digit - radius));
    }
    const int32_t out = find_key<D, S>(t, k);
    idx[e] = out;
    mask[e] = out >= 0 ? 1 : 0;
  }
}

// Neighbour query over an explicit offset table (the neighbour tables of
// Sec. 6.2-6.4: 1-radius 3^D, 1-cube 2^D, 1-ring): thread per (query, offset)
// pair; offsets is [n_off, D] int32 in device memory, added with int32
// wrap-around.  Outputs are [n, n_off].
template <int D, int S>
__global__ void __launch_bounds__(256) offsets_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                      const int32_t* __restrict__ offsets, int64_t n_off,
                                                      int32_t* __restrict__ idx, uint8_t* __restrict__ mask) {
  const int64_t total = n * n_off;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t r = e / n_off;
    const int64_t o = e - r * n_off;
    int32_t k[D];
    load_input_key<D>(keys, r, k);
#pragma unroll
    for (int j = 0; j < D; ++j)
      k[j] = static_cast<int32_t>(static_cast<uint32_t>(k[j]) + static_cast<uint32_t>(__ldg(offsets + o * D + j)));
    const int32_t out = find_key<D, S>(t, k);
    idx[e] = out;
    mask[e] = out >= 0 ? 1 : 0;
  }
}

// KPT keys per thread: positions base, base + blockDim.x, ... so every load
// instruction stays coalesced across the warp.  All home buckets are loaded
// before any is examined, and all verify loads are issued before any compare.
template <int D, int S, int KPT, class In = const int32_t*>
__global__ void __launch_bounds__(256) find_kernel(TableView t, const In keys, int64_t n,
                                                   int32_t* __restrict__ idx, uint8_t* __restrict__ mask) {
  // a programmatic dependent of the previous kernel: wait for its grid (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int KS = KeyStride<D>::value;
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * KPT;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x * KPT + threadIdx.x; base < n; base += step) {
    int32_t k[KPT][D];
    uint32_t fp[KPT], b[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      if (pos < n) {
        load_input_key<D>(keys, pos, k[q]);
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) k[q][j] = 0;
      }
      const uint64_t h = hash_key<D>(k[q]);
      fp[q] = fingerprint(h);
      b[q] = home_bucket(h, t.n_buckets);
    }
    uint64_t w[KPT][S];
#pragma unroll
    for (int q = 0; q < KPT; ++q) load_bucket<S, true>(t.slots + static_cast<size_t>(b[q]) * S, w[q]);
    uint32_t cand[KPT];
    int ncand[KPT];
    bool stop[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      cand[q] = kNoIndex;
      ncand[q] = 0;
      stop[q] = false;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        stop[q] |= (w[q][s] == kEmpty);
        const bool m = hi32(w[q][s]) == fp[q] && lo32(w[q][s]) < kClaimBit;
        if (m && ncand[q] == 0) cand[q] = lo32(w[q][s]);
        ncand[q] += m ? 1 : 0;
      }
    }
    int32_t row[KPT][KS];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      if (ncand[q] > 0) {
        load_kb<D>(t.kb, cand[q], row[q]);
      } else {
#pragma unroll
        for (int j = 0; j < KS; ++j) row[q][j] = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      if (pos < n) {
        bool eq = ncand[q] > 0;
#pragma unroll
        for (int j = 0; j < D; ++j) eq &= (row[q][j] == k[q][j]);
        int32_t out = -1;
        if (eq) out = static_cast<int32_t>(cand[q]);
        else if (ncand[q] > 0 || !stop[q]) out = find_one<D, S, In>(t, keys, pos);  // rare
        idx[pos] = out;
        mask[pos] = out >= 0 ? 1 : 0;
      }
    }
  }
}

// Warp-cooperative find: a group of G = S / 2 lanes takes one key, each lane
// loading two slots (one 16-byte load; the group reads the whole bucket in one
// coalesced request), so a warp has 32 / G keys in flight.  Fingerprint
// matches are verified by the lane that holds them with one 128-bit kB load;
// the group agrees through __ballot_sync and the result comes from the
// lowest verified lane (__shfl_sync).  Probing continues while no lane saw an
// EMPTY slot.  Groups of one warp proceed together (warp-wide ballots), a
// finished group voting false.  The alternative to find_kernel's thread per
// key; the tuning's warp_probe picks one.
template <int D, int S>
__global__ void __launch_bounds__(256) find_group_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                         int32_t* __restrict__ idx, uint8_t* __restrict__ mask) {
  constexpr int G = S / 2;
  constexpr int KEYS_PER_WARP = 32 / G;
  constexpr uint32_t kGroupBits = (G == 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
  const int lane = threadIdx.x & 31;
  const int sub = lane % G;               // lane within the group
  const int grp = lane / G;               // group within the warp
  const uint32_t gshift = static_cast<uint32_t>(grp * G);
  const int64_t warp_global = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp_global * KEYS_PER_WARP; base < n; base += n_warps * KEYS_PER_WARP) {
    const int64_t pos = base + grp;
    bool active = pos < n;
    int32_t k[D];
    if (active) {
      load_input_key<D>(keys, pos, k);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) k[j] = 0;
    }
    const uint64_t h = hash_key<D>(k);
    const uint32_t fp = fingerprint(h);
    uint32_t b = home_bucket(h, t.n_buckets);
    int32_t out = -1;
    for (uint32_t probe = 0; probe < t.max_probes; ++probe) {
      const bool live = active;
      bool found = false, empty = false;
      uint32_t my = kNoIndex;
      if (live) {
        const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2*>(t.slots + static_cast<size_t>(b) * S) + sub);
        empty = (w.x == kEmpty) || (w.y == kEmpty);
        const bool m0 = hi32(w.x) == fp && lo32(w.x) < kClaimBit;
        const bool m1 = hi32(w.y) == fp && lo32(w.y) < kClaimBit;
        if (m0 && kb_equal<D>(t.kb, lo32(w.x), k)) my = lo32(w.x);
        else if (m1 && kb_equal<D>(t.kb, lo32(w.y), k)) my = lo32(w.y);
        found = my != kNoIndex;
      }
      const uint32_t fb = (__ballot_sync(0xFFFFFFFFu, found) >> gshift) & kGroupBits;
      const uint32_t eb = (__ballot_sync(0xFFFFFFFFu, empty) >> gshift) & kGroupBits;
      const int src = fb ? static_cast<int>(gshift) + __ffs(fb) - 1 : lane;
      const uint32_t hit = __shfl_sync(0xFFFFFFFFu, my, src);
      if (live) {
        if (fb) {
          out = static_cast<int32_t>(hit);
          active = false;
        } else if (eb) {
          active = false;
        } else {
          b = next_bucket(b, t.n_buckets);
        }
      }
      if (!__any_sync(0xFFFFFFFFu, active)) break;
    }
    if (pos < n && sub == 0) {
      idx[pos] = out;
      mask[pos] = out >= 0 ? 1 : 0;
    }
  }
}

// ------------------------------------------------------------- insert: claim
// Result codes written to buf_indices[p] by the claim kernel.
constexpr int32_t kClaimExists = -2;  // key already committed
constexpr int32_t kClaimJoined = -3;  // an equal key of this batch with a lower position holds the claim
constexpr int32_t kClaimFailed = -1;  // no slot within max_probes

// 0: no match.  1: slot claimed by an equal key in this batch.  2: committed equal key.
template <int D, class In>
__device__ __forceinline__ int claim_match(uint64_t w, uint32_t fp, const int32_t (&k)[D], const In& keys,
                                           const int32_t* kb) {
  const uint32_t lo = lo32(w);
  if (lo == kNoIndex || hi32(w) != fp) return 0;
  if (lo & kClaimBit) return input_key_equal<D>(keys, lo & ~kClaimBit, k) ? 1 : 0;
  return kb_equal<D>(kb, lo, k) ? 2 : 0;
}

// This position meets an equal key's claim, with position seen_lo, at slot p:
// the lower position keeps the claim (atomicMin on the word, whose high half
// is the shared fingerprint).  Returns false when this position lost for
// sure (a lower one holds the claim); true when it holds the claim for now.
// With winner flags (FLAGS and t.lost) the position it displaced is marked
// lost.
template <bool FLAGS = true>
__device__ __forceinline__ bool join_claim(const TableView& t, uint64_t* p, uint32_t seen_lo, uint64_t mine,
                                           uint32_t pos) {
  if (!FLAGS) {
    // no winner flags: the commit reads the slot word to see who won
    if ((seen_lo & ~kClaimBit) > pos)
      atomicMin(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(mine));
    return true;
  }
  if ((seen_lo & ~kClaimBit) < pos) return false;
  if (!t.lost) {
    atomicMin(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(mine));
    return true;
  }
  const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(mine));
  const uint32_t op = lo32(old) & ~kClaimBit;
  if (op < pos) return false;
  atomicOr(t.lost + (op >> 5), 1u << (op & 31));
  return true;
}

// Order of the EMPTY slots a claim tries (claim_key):
//   kClaimSlotOrder  slot order, one CAS site per slot (unrolled): the
//                    fastest form, used out of line as a slow path
//   kClaimSlotMask   slot order, one CAS site for all slots (a bit-mask
//                    loop): fewer registers, for the batched kernel that
//                    inlines the protocol for every key dimension
//   kClaimPrefFirst  the key's preferred slot first in its home bucket, then
//                    slot order (keeps the preferred-slot invariant)
constexpr int kClaimSlotOrder = 0;
constexpr int kClaimSlotMask = 1;
constexpr int kClaimPrefFirst = 2;

// The full claim protocol for one key, from its home bucket: 1) any slot of
// the bucket holding an equal key ends the search; 2) otherwise the EMPTY
// slots are claimed in the order ORDER gives, and a lost CAS re-checks the
// winner's word for an equal key; 3) a bucket without EMPTY slots sends the
// key to the next bucket.  FLAGS: winner flags may be set (t.lost); the
// batched kernel, which has none, compiles without them.
template <int D, int S, class In, int ORDER, bool FLAGS = true>
__device__ __forceinline__ int32_t claim_key(const TableView& t, const In& keys, int64_t pos) {
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
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int m = claim_match<D, In>(w[s], fp, k, keys, t.kb);
      if (m == 2) return kClaimExists;
      if (m == 1)
        return join_claim<FLAGS>(t, bp + s, lo32(w[s]), mine, static_cast<uint32_t>(pos)) ? static_cast<int32_t>(b * S + s)
                                                                                    : kClaimJoined;
    }
    if constexpr (ORDER == kClaimSlotOrder) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (w[s] == kEmpty) {
          const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(bp + s),
                                         static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(mine));
          if (old == kEmpty) return static_cast<int32_t>(b * S + s);
          const int m = claim_match<D, In>(old, fp, k, keys, t.kb);
          if (m == 2) return kClaimExists;
          if (m == 1)
            return join_claim<FLAGS>(t, bp + s, lo32(old), mine, static_cast<uint32_t>(pos)) ? static_cast<int32_t>(b * S + s)
                                                                                      : kClaimJoined;
        }
      }
    } else {
      // EMPTY slots of the snapshot as a bit mask (one CAS site for all)
      uint32_t emask = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) emask |= (w[s] == kEmpty ? 1u : 0u) << s;
      const uint32_t pbit = ORDER == kClaimPrefFirst && probe == 0 ? 1u << pref_slot<S>(fp) : 0u;
      while (emask) {
        const int s = (emask & pbit) ? static_cast<int>(pref_slot<S>(fp)) : __ffs(emask) - 1;
        emask &= ~(1u << s);
        const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(bp + s),
                                       static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(mine));
        if (old == kEmpty) return static_cast<int32_t>(b * S + s);
        const int m = claim_match<D, In>(old, fp, k, keys, t.kb);
        if (m == 2) return kClaimExists;
        if (m == 1)
          return join_claim<FLAGS>(t, bp + s, lo32(old), mine, static_cast<uint32_t>(pos)) ? static_cast<int32_t>(b * S + s)
                                                                                    : kClaimJoined;
      }
    }
    b = next_bucket(b, t.n_buckets);
  }
  atomicOr(&t.ctrl->status, kStatusTableFull);
  return kClaimFailed;
}

// Out-of-line copy of the full protocol: the rare slow path of the claim
// kernels (kept out of line so it does not raise their register count).
template <int D, int S, class In, bool PrefFirst>
__device__ __noinline__ int32_t claim_one(const TableView t, const In keys, int64_t pos) {
  return claim_key<D, S, In, PrefFirst ? kClaimPrefFirst : kClaimSlotOrder>(t, keys, pos);
}

// Claim from the loaded home bucket, DK keys per lane (pos[q] valid where
// v[q]; an invalid lane hashes key 0 and loads that bucket, in bounds).  Per
// key: if the bucket holds exactly one slot with the key's fingerprint,
// compare once (claimant's input row or kB row); on no match, CAS the first
// EMPTY slot (PrefFirst: the preferred slot when it is EMPTY).  The loads,
// compares and CASes of the DK keys are issued back to back.  Anything else
// (several fingerprint matches, a lost CAS, a full bucket) runs claim_one,
// which is safe because this path changed nothing then.
template <int D, int S, int DK, class In, bool PrefFirst>
__device__ __forceinline__ void claim_from_bucket(const TableView& t, const In& keys, const int64_t (&pos)[DK],
                                                  const bool (&v)[DK], int32_t* __restrict__ slot_out) {
  constexpr int KS = KeyStride<D>::value;
  int32_t k[DK][D];
  uint32_t fp[DK], b[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    if (v[q]) {
      load_input_key<D>(keys, pos[q], k[q]);
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) k[q][j] = 0;
    }
    const uint64_t h = hash_key<D>(k[q]);
    fp[q] = fingerprint(h);
    b[q] = home_bucket(h, t.n_buckets);
  }
  uint64_t w[DK][S];
#pragma unroll
  for (int q = 0; q < DK; ++q) load_bucket<S, false>(t.slots + static_cast<size_t>(b[q]) * S, w[q]);
  int cs[DK], nc[DK], es[DK];
  uint32_t clo[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    cs[q] = -1;
    nc[q] = 0;
    es[q] = -1;
    clo[q] = kNoIndex;
    const uint32_t pref = pref_slot<S>(fp[q]);
    int pe = -1;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const bool m = lo32(w[q][s]) != kNoIndex && hi32(w[q][s]) == fp[q];
      if (m && nc[q] == 0) {
        cs[q] = s;
        clo[q] = lo32(w[q][s]);
      }
      nc[q] += m ? 1 : 0;
      if (es[q] < 0 && w[q][s] == kEmpty) es[q] = s;
      if (PrefFirst && static_cast<uint32_t>(s) == pref && w[q][s] == kEmpty) pe = s;
    }
    if (PrefFirst && pe >= 0) es[q] = pe;  // preferred slot first (preferred-slot invariant)
  }
  int32_t row[DK][KS];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    if (nc[q] > 0) {
      if (clo[q] & kClaimBit) {
        int32_t o[D];
        load_input_key<D>(keys, clo[q] & ~kClaimBit, o);
#pragma unroll
        for (int j = 0; j < KS; ++j) row[q][j] = j < D ? o[j] : 0;
      } else {
        load_kb<D>(t.kb, clo[q], row[q]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < KS; ++j) row[q][j] = 0;
    }
  }
  int32_t res[DK];
  bool cas[DK], slow[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    res[q] = kClaimFailed;
    cas[q] = false;
    slow[q] = false;
    if (v[q]) {
      bool eq = nc[q] > 0;
#pragma unroll
      for (int j = 0; j < D; ++j) eq &= (row[q][j] == k[q][j]);
      if (eq) {
        if (clo[q] & kClaimBit) {
          const uint64_t mine = (static_cast<uint64_t>(fp[q]) << 32) | (kClaimBit | static_cast<uint32_t>(pos[q]));
          res[q] = join_claim(t, t.slots + static_cast<size_t>(b[q]) * S + cs[q], clo[q], mine,
                              static_cast<uint32_t>(pos[q]))
                       ? static_cast<int32_t>(b[q] * S + cs[q])
                       : kClaimJoined;
        } else {
          res[q] = kClaimExists;
        }
      } else if (nc[q] > 1 || es[q] < 0) {
        slow[q] = true;
      } else {
        cas[q] = true;
      }
    }
  }
  uint64_t old[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    old[q] = 0;
    if (cas[q]) {
      const uint64_t mine = (static_cast<uint64_t>(fp[q]) << 32) | (kClaimBit | static_cast<uint32_t>(pos[q]));
      old[q] = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + static_cast<size_t>(b[q]) * S + es[q]),
                         static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(mine));
    }
  }
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    if (cas[q]) {
      if (old[q] == kEmpty) res[q] = static_cast<int32_t>(b[q] * S + es[q]);
      else slow[q] = true;
    }
    if (slow[q]) res[q] = claim_one<D, S, In, PrefFirst>(t, keys, pos[q]);  // rare
    if (v[q]) slot_out[pos[q]] = res[q];
  }
}

// Claim kernel, bucket load first: KPT keys per thread, each claimed from its
// loaded home bucket (two dependent accesses per key: bucket load, CAS) in
// slot order.  The better choice when the table does not stay in L2: the
// loads bring the buckets in with deep miss queues and the CASes then hit L2.
// Slot order does not keep the preferred-slot invariant (preferred-first
// placement measured 5-10 % slower here), so the host clears the map's flag.
template <int D, int S, int KPT, class In = const int32_t*>
__global__ void __launch_bounds__(256) claim_bucket_kernel(TableView t, const In keys, int64_t n,
                                                           int32_t* __restrict__ slot_out) {
  // a programmatic dependent of the previous kernel: wait for its grid (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * KPT;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x * KPT + threadIdx.x; base < n; base += step) {
    int64_t p[KPT];
    bool v[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      p[q] = base + static_cast<int64_t>(q) * blockDim.x;
      v[q] = p[q] < n;
    }
    claim_from_bucket<D, S, KPT, In, false>(t, keys, p, v, slot_out);
  }
}

// Claim kernel, preferred slot first.  Each warp takes 32 * KPT consecutive
// keys per iteration (KPT per lane; the launcher uses 1).  Fast path per key:
// CAS the preferred slot of the home bucket, with no bucket load before it.
// EMPTY there: claimed.  An occupant with the key's fingerprint: compare once
// (claimant's input row or kB row); an equal key joins the claim (lowest
// position wins) or reports the committed key.  Any other key (the preferred
// slot holds another key, a tombstone, or a fingerprint collision) is queued
// in the warp's shared-memory list; whenever the list holds 32 * kDL keys the
// warp claims them from their buckets together, kDL per lane
// (claim_from_bucket), so the slower path runs on dense warps instead of
// stalling every warp for a few lanes.  A CAS that misses L2 waits on DRAM
// inside the atomic unit, so this path pays off while the table stays in L2.
template <int D, int S, int KPT, class In = const int32_t*>
__global__ void __launch_bounds__(256) claim_pref_kernel(TableView t, const In keys, int64_t n,
                                                         int32_t* __restrict__ slot_out) {
  // a programmatic dependent of the previous kernel: wait for its grid (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  constexpr int KS = KeyStride<D>::value;
  constexpr int kDL = KPT == 1 ? 1 : 2;      // queued keys per lane in a dense round
  constexpr int kDrain = 32 * kDL;
  constexpr int kCap = kDrain + 32 * KPT;    // a round starts before a tile could overflow
  __shared__ int32_t s_queue[8][kCap];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int32_t* queue = s_queue[threadIdx.x >> 5];
  int qn = 0;  // warp-uniform
  const int64_t n_warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t warp_id = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t wbase = warp_id * 32 * KPT; wbase < n; wbase += n_warps * 32 * KPT) {
    int32_t k[KPT][D];
    uint32_t fp[KPT], ps[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = wbase + q * 32 + lane;
      if (pos < n) {
        load_input_key<D>(keys, pos, k[q]);
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) k[q][j] = 0;
      }
      const uint64_t h = hash_key<D>(k[q]);
      fp[q] = fingerprint(h);
      ps[q] = home_bucket(h, t.n_buckets) * S + pref_slot<S>(fp[q]);
    }
    uint64_t old[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = wbase + q * 32 + lane;
      old[q] = kTombstone;
      if (pos < n) {
        const uint64_t mine = (static_cast<uint64_t>(fp[q]) << 32) | (kClaimBit | static_cast<uint32_t>(pos));
        old[q] = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + ps[q]),
                           static_cast<unsigned long long>(kEmpty), static_cast<unsigned long long>(mine));
      }
    }
    bool fm[KPT];
    int32_t row[KPT][KS];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const uint32_t lo = lo32(old[q]);
      fm[q] = lo != kNoIndex && hi32(old[q]) == fp[q];
      if (fm[q]) {
        if (lo & kClaimBit) {
          int32_t o[D];
          load_input_key<D>(keys, lo & ~kClaimBit, o);
#pragma unroll
          for (int j = 0; j < KS; ++j) row[q][j] = j < D ? o[j] : 0;
        } else {
          load_kb<D>(t.kb, lo, row[q]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < KS; ++j) row[q][j] = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = wbase + q * 32 + lane;
      bool pending = false;
      if (pos < n) {
        const uint32_t lo = lo32(old[q]);
        bool eq = fm[q];
#pragma unroll
        for (int j = 0; j < D; ++j) eq &= (row[q][j] == k[q][j]);
        if (old[q] == kEmpty) {
          slot_out[pos] = static_cast<int32_t>(ps[q]);
        } else if (!eq) {
          pending = true;
        } else if (lo & kClaimBit) {
          const uint64_t mine = (static_cast<uint64_t>(fp[q]) << 32) | (kClaimBit | static_cast<uint32_t>(pos));
          slot_out[pos] = join_claim(t, t.slots + ps[q], lo, mine, static_cast<uint32_t>(pos))
                              ? static_cast<int32_t>(ps[q])
                              : kClaimJoined;
        } else {
          slot_out[pos] = kClaimExists;
        }
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, pending);
      if (pending) queue[qn + __popc(bal & lt)] = static_cast<int32_t>(pos);
      qn += __popc(bal);
    }
    __syncwarp();
    while (qn >= kDrain) {
      int64_t p[kDL];
      bool v[kDL];
#pragma unroll
      for (int r = 0; r < kDL; ++r) {
        v[r] = true;
        p[r] = queue[qn - kDrain + r * 32 + lane];
      }
      __syncwarp();
      qn -= kDrain;
      claim_from_bucket<D, S, kDL, In, true>(t, keys, p, v, slot_out);
    }
  }
  __syncwarp();
  if (qn > 0) {
    int64_t p[kDL];
    bool v[kDL];
#pragma unroll
    for (int r = 0; r < kDL; ++r) {
      v[r] = r * 32 + lane < qn;
      p[r] = v[r] ? queue[r * 32 + lane] : 0;
    }
    claim_from_bucket<D, S, kDL, In, true>(t, keys, p, v, slot_out);
  }
}

// ------------------------------------------------------------ insert: commit
// One value buffer whose rows are exactly 4, 8 or 16 bytes with both bases
// aligned to the row size: the committing thread copies its row as one
// vector.  Other layouts use the scatter kernel after the commit.
struct ValueRow {
  void* dst;
  const void* src;
  int64_t row_bytes;  // 4, 8 or 16
  int vec;
  int pad;
};

__device__ __forceinline__ void copy_small_row(const ValueRow& v, int32_t i, int64_t pos) {
  char* d = static_cast<char*>(v.dst) + static_cast<int64_t>(i) * v.row_bytes;
  const char* s = static_cast<const char*>(v.src) + pos * v.row_bytes;
  if (v.row_bytes == 16) *reinterpret_cast<uint4*>(d) = __ldg(reinterpret_cast<const uint4*>(s));
  else if (v.row_bytes == 8) *reinterpret_cast<uint2*>(d) = __ldg(reinterpret_cast<const uint2*>(s));
  else *reinterpret_cast<uint32_t*>(d) = __ldg(reinterpret_cast<const uint32_t*>(s));
}

// KPT keys per thread per block iteration (blockDim.x * KPT keys).  Who won
// each key: FLAGS, a position holding a slot index whose winner-flag bit
// (t.lost) is clear, from two streamed reads; otherwise the slot word, read
// at random, names the winning position.  One block-wide scan ranks the
// winners and ONE heap atomic serves the iteration (Sec. 4.3: t is raised by
// the number of indices taken).  Winners then write kB(i), the value row, the
// committed slot word and their outputs.
template <int D, int KPT, bool VAL, class In, bool FLAGS = false>
__device__ __forceinline__ void commit_tile(const TableView& t, const In& keys, int64_t n,
                                            int64_t base0, int32_t* __restrict__ idx, uint8_t* __restrict__ mask,
                                            const ValueRow& v, int* s_warp, int* s_base, int* s_got) {
  const int64_t base = base0 + threadIdx.x;
  int32_t s[KPT];
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
    s[q] = pos < n ? idx[pos] : -1;
  }
  uint64_t w[KPT];
  bool win[KPT];
  int cnt = 0;
  if constexpr (FLAGS) {
    uint32_t lw[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      lw[q] = pos < n ? t.lost[pos >> 5] : 0u;
    }
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      w[q] = 0;
      win[q] = s[q] >= 0 && !((lw[q] >> (pos & 31)) & 1u);
      cnt += win[q] ? 1 : 0;
    }
  } else {
#pragma unroll
    for (int q = 0; q < KPT; ++q) w[q] = s[q] >= 0 ? load_slot_relaxed(t.slots + s[q]) : 0ull;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      win[q] = s[q] >= 0 && lo32(w[q]) == (kClaimBit | static_cast<uint32_t>(pos));
      cnt += win[q] ? 1 : 0;
    }
  }
  int total;
  const int off = block_exclusive_scan(cnt, total, s_warp);  // a block barrier: every flag word was read
  if constexpr (FLAGS) {
    // leave the flags clear for the next insert (one lane per 32 positions;
    // blockDim and the tile base are multiples of 32, so a warp's 32
    // positions of one slice share one word)
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
      if (pos < n && (pos & 31) == 0) t.lost[pos >> 5] = 0u;
    }
  }
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
    *s_base = top;
    *s_got = got;
  }
  __syncthreads();
  const int got = *s_got;
  const int hbase = *s_base;
  int r = off;
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    const int64_t pos = base + static_cast<int64_t>(q) * blockDim.x;
    if (pos < n) {
      if (win[q]) {
        if (r < got) {
          const int32_t i = (t.flags & kViewHeapIdentity) ? hbase + r : t.heap[hbase + r];
          int32_t k[D];
          load_input_key<D>(keys, pos, k);
          store_kb<D>(t.kb, static_cast<uint32_t>(i), k);
          if constexpr (VAL) copy_small_row(v, i, pos);
          const uint32_t fp = FLAGS ? fingerprint(hash_key<D>(k)) : hi32(w[q]);
          t.slots[s[q]] = (static_cast<uint64_t>(fp) << 32) | static_cast<uint32_t>(i);
          idx[pos] = i;
          mask[pos] = 1;
        } else {
          t.slots[s[q]] = kTombstone;
          idx[pos] = -1;
          mask[pos] = 0;
        }
        ++r;
      } else {
        idx[pos] = -1;
        mask[pos] = 0;
      }
    }
  }
  __syncthreads();
}

template <int D, int KPT, bool VAL, class In = const int32_t*, bool FLAGS = false>
__global__ void __launch_bounds__(256) commit_kernel(TableView t, const In keys, int64_t n,
                                                     int32_t* __restrict__ idx, uint8_t* __restrict__ mask,
                                                     ValueRow v) {
  __shared__ int s_warp[33];
  __shared__ int s_base;
  __shared__ int s_got;
  // a programmatic dependent of the previous kernel: wait for its grid (a no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x * KPT;
  for (int64_t base0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * KPT; base0 < n; base0 += step)
    commit_tile<D, KPT, VAL, In, FLAGS>(t, keys, n, base0, idx, mask, v, s_warp, &s_base, &s_got);
  // The last block to finish publishes the control block for the host's
  // growth checks (every block's heap atomics were made by its thread 0).
  if (t.snap != nullptr && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&t.ctrl->commit_done, 1u) == gridDim.x - 1) {
      __threadfence();
      t.ctrl->commit_done = 0u;
      publish_snapshot(t.ctrl, t.snap, t.snap_seq);
    }
  }
}

// ------------------------------------------------------- key partitioning
// For tables larger than L2, a call's keys are first put in the order of
// their home buckets' ranges: P = 2^log_p ranges of consecutive buckets (the
// top log_p bits of the hash word the home bucket comes from), a stable
// partition, so that equal keys keep their input order and the lowest
// position still wins.  The claim, commit and find kernels walk their keys
// in order, so each then works on one range of the table at a time, and of
// kB too once the commit has handed out indices in the same order, and
// finds it in L2.
//
// Each of G blocks owns a contiguous span of whole tiles of kPartTile input
// keys.  A count pass histograms each block's span per range (counts[P][G]);
// a scan turns each range's row into the blocks' offsets within the range
// (and the range totals); the scatter pass sorts each tile by range in
// shared memory (stable: warp w holds tile positions [256 w, 256 w + 256) in
// steps of 32, ranked by __match_any_sync) and writes each range's part of
// the tile as one run after the block's previous tiles' runs.  dest[pos]
// records where input row pos went, for the outputs' way back.
constexpr int kPartTile = 2048;     // keys per tile: 256 threads x 8
constexpr int kPartSteps = kPartTile / 256;
constexpr int kPartMaxLog = 8;      // at most 256 ranges
constexpr uint32_t kNoRange = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t key_range(uint64_t h, int log_p) { return hi32(h) >> (32 - log_p); }

// The kPartSteps key rows of one lane in warp w's part of a tile (local
// positions 256 w + 32 j + lane); zeros past the tile.
template <int D>
__device__ __forceinline__ void load_tile_rows(const int32_t* __restrict__ keys, int64_t base, int tn,
                                               int32_t (&k)[kPartSteps][D]) {
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kPartSteps; ++j) {
    const int local = w * 256 + j * 32 + lane;
    if (local < tn) {
      load_input_key<D>(keys, base + local, k[j]);
    } else {
#pragma unroll
      for (int c = 0; c < D; ++c) k[j][c] = 0;
    }
  }
}

// Their ranges (kNoRange past the tile).
template <int D>
__device__ __forceinline__ void tile_ranges(const int32_t (&k)[kPartSteps][D], int tn, int log_p,
                                            uint32_t (&r)[kPartSteps]) {
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kPartSteps; ++j)
    r[j] = w * 256 + j * 32 + lane < tn ? key_range(hash_key<D>(k[j]), log_p) : kNoRange;
}

// Keys in tile at `base` of a span ending at t1.
__device__ __forceinline__ int tile_keys(int64_t base, int64_t t1) {
  return t1 - base < kPartTile ? static_cast<int>(t1 - base) : kPartTile;
}

// counts[p * G + b]: keys of range p in block b's span.
template <int D>
__global__ void __launch_bounds__(256) partition_count_kernel(const int32_t* __restrict__ keys, int64_t n, int log_p,
                                                              int tiles_per_block, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_hist[1 << kPartMaxLog];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int P = 1 << log_p;
  for (int p = threadIdx.x; p < P; p += blockDim.x) s_hist[p] = 0u;
  __syncthreads();
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * tiles_per_block * kPartTile;
  const int64_t t1 = t0 + static_cast<int64_t>(tiles_per_block) * kPartTile < n
                         ? t0 + static_cast<int64_t>(tiles_per_block) * kPartTile
                         : n;
  // each tile's rows are loaded while the tile before is being counted
  int32_t k[kPartSteps][D];
  if (t0 < t1) load_tile_rows<D>(keys, t0, tile_keys(t0, t1), k);
  for (int64_t base = t0; base < t1; base += kPartTile) {
    const int tn = tile_keys(base, t1);
    uint32_t r[kPartSteps];
    tile_ranges<D>(k, tn, log_p, r);
    if (base + kPartTile < t1) load_tile_rows<D>(keys, base + kPartTile, tile_keys(base + kPartTile, t1), k);
#pragma unroll
    for (int j = 0; j < kPartSteps; ++j)
      if (r[j] != kNoRange) atomicAdd(&s_hist[r[j]], 1u);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) counts[static_cast<int64_t>(p) * gridDim.x + blockIdx.x] = s_hist[p];
}

// Dynamic shared memory of the scatter kernel: the tile's key rows.
template <int D>
constexpr size_t partition_scatter_smem() {
  return sizeof(int32_t) * kPartTile * D;
}

// row_offsets: counts after the scan (block b's first place within range p);
// range_totals: keys per range.
template <int D>
__global__ void __launch_bounds__(256) partition_scatter_kernel(const int32_t* __restrict__ keys, int64_t n, int log_p,
                                                                int tiles_per_block,
                                                                const uint32_t* __restrict__ row_offsets,
                                                                const uint32_t* __restrict__ range_totals,
                                                                int32_t* __restrict__ keys_out,
                                                                int32_t* __restrict__ dest) {
  extern __shared__ int32_t s_keys[];  // [kPartTile][D], the tile in range order
  __shared__ uint32_t s_run[1 << kPartMaxLog];    // next place of each range for this block
  __shared__ uint32_t s_start[1 << kPartMaxLog];  // first tile slot of each range
  __shared__ uint32_t s_tcnt[1 << kPartMaxLog];   // the tile's keys of each range
  __shared__ uint32_t s_cnt[8][1 << kPartMaxLog]; // per warp: keys of each range, then its offset in the range
  __shared__ uint16_t s_pos[kPartTile];           // tile position of each slot
  __shared__ uint8_t s_r[kPartTile];              // range of each slot
  __shared__ int s_warp[33];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int P = 1 << log_p;
  const int tid = threadIdx.x;
  const int w = tid >> 5;
  const int lane = tid & 31;
  const unsigned lt = (1u << lane) - 1u;
  {
    int unused;
    const uint32_t tot = tid < P ? range_totals[tid] : 0u;
    const uint32_t start = static_cast<uint32_t>(block_exclusive_scan(static_cast<int>(tot), unused, s_warp));
    if (tid < P) s_run[tid] = start + row_offsets[static_cast<int64_t>(tid) * gridDim.x + blockIdx.x];
    __syncthreads();
  }
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * tiles_per_block * kPartTile;
  const int64_t t1 = t0 + static_cast<int64_t>(tiles_per_block) * kPartTile < n
                         ? t0 + static_cast<int64_t>(tiles_per_block) * kPartTile
                         : n;
  for (int64_t base = t0; base < t1; base += kPartTile) {
    const int tn = tile_keys(base, t1);
    for (int p = lane; p < P; p += 32) s_cnt[w][p] = 0u;
    __syncwarp();
    int32_t k[kPartSteps][D];
    uint32_t r[kPartSteps];
    load_tile_rows<D>(keys, base, tn, k);
    tile_ranges<D>(k, tn, log_p, r);
    uint32_t rank[kPartSteps];
#pragma unroll
    for (int j = 0; j < kPartSteps; ++j) {
      const bool valid = r[j] != kNoRange;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, r[j]);
      const uint32_t c = valid ? s_cnt[w][r[j]] : 0u;
      rank[j] = c + __popc(peers & lt);
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) s_cnt[w][r[j]] = c + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint32_t tc = 0;
    if (tid < P) {
      for (int ww = 0; ww < 8; ++ww) {
        const uint32_t c = s_cnt[ww][tid];
        s_cnt[ww][tid] = tc;
        tc += c;
      }
    }
    int tile_total;
    const uint32_t st = static_cast<uint32_t>(block_exclusive_scan(static_cast<int>(tc), tile_total, s_warp));
    if (tid < P) {
      s_start[tid] = st;
      s_tcnt[tid] = tc;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPartSteps; ++j) {
      if (r[j] != kNoRange) {
        const uint32_t slot = s_start[r[j]] + s_cnt[w][r[j]] + rank[j];
#pragma unroll
        for (int c = 0; c < D; ++c) s_keys[slot * D + c] = k[j][c];
        s_pos[slot] = static_cast<uint16_t>(w * 256 + j * 32 + lane);
        s_r[slot] = static_cast<uint8_t>(r[j]);
      }
    }
    __syncthreads();
    for (int slot = tid; slot < tn; slot += blockDim.x) {
      const uint32_t rr = s_r[slot];
      const uint32_t d = s_run[rr] + (slot - s_start[rr]);
      int32_t* row = keys_out + static_cast<int64_t>(d) * D;
#pragma unroll
      for (int c = 0; c < D; ++c) row[c] = s_keys[slot * D + c];
      dest[base + s_pos[slot]] = static_cast<int32_t>(d);
    }
    __syncthreads();
    if (tid < P) s_run[tid] += s_tcnt[tid];
    __syncthreads();
  }
}

// --------------------------------------------------------------- erase: mark
// Finds input row pos and marks its slot with the lowest position seen
// (atomicMin into the high word, the buffer index kept in the low word).
// Returns the slot index, or -1 if the key is absent.
template <int D, int S>
__device__ __forceinline__ int32_t erase_mark_one(const TableView& t, const int32_t* __restrict__ keys, int64_t pos) {
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
          atomicMin(reinterpret_cast<unsigned long long*>(bp + s), (static_cast<unsigned long long>(pos) << 32) | lo);
        res = static_cast<int32_t>(b * S + s);
      }
    }
    if (stop) break;
    b = next_bucket(b, t.n_buckets);
  }
  return res;
}

template <int D, int S>
__global__ void __launch_bounds__(256) erase_mark_kernel(TableView t, const int32_t* __restrict__ keys, int64_t n,
                                                         int32_t* __restrict__ slot_out) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t pos = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; pos < n; pos += stride)
    slot_out[pos] = erase_mark_one<D, S>(t, keys, pos);
}

// ------------------------------------------------------------ erase: resolve
// One tile of blockDim.x positions starting at base0.  Every thread of the
// block must call it (block-wide scan and barriers).
template <int S>
__device__ __forceinline__ void erase_resolve_tile(const TableView& t, int64_t n, int64_t base0,
                                                   const int32_t* __restrict__ slot_in, uint8_t* __restrict__ mask,
                                                   int* s_warp, int* s_cnt, int* s_base) {
  const int64_t pos = base0 + threadIdx.x;
  const bool active = pos < n;
  const int32_t s = active ? slot_in[pos] : -1;
  uint64_t w = 0;
  bool win = false, to_empty = false;
  if (s >= 0) {
    w = load_slot_relaxed(t.slots + s);
    win = hi32(w) == static_cast<uint32_t>(pos);
    if (win) {
      // EMPTY only when the bucket already has an EMPTY slot (no probe chain
      // passes through it) and, while the map keeps the preferred-slot
      // invariant, no other live key of the bucket prefers the freed slot; a
      // TOMBSTONE otherwise (the freed slot itself holds a marked word, which
      // never counts).  The bucket is read 32 bytes at a time to keep few
      // words live.
      const uint64_t* bp = t.slots + static_cast<size_t>(s / S) * S;
      const uint32_t own = static_cast<uint32_t>(s) & (S - 1);
      bool preferred = false;
#pragma unroll 1
      for (int c = 0; c < S / 4; ++c) {
        uint64_t cw[4];
        load32<false>(bp + 4 * c, cw[0], cw[1], cw[2], cw[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          to_empty |= (cw[j] == kEmpty);
          preferred |= is_committed(cw[j]) && pref_slot<S>(hi32(cw[j])) == own;
        }
      }
      to_empty &= !(preferred && (t.flags & kViewPrefPlaced));
    }
  }
  int rank, total;
  block_rank(win, rank, total, s_warp);
  const int n_empty = block_count(to_empty, s_cnt);
  if (threadIdx.x == 0) {
    int top = 0;
    if (total > 0) {
      const unsigned long long sub = (static_cast<unsigned long long>(n_empty) << 32) + static_cast<unsigned long long>(total);
      const unsigned long long old = atomicAdd(&t.ctrl->top_used, 0ull - sub);
      top = static_cast<int>(static_cast<uint32_t>(old));
    }
    *s_base = top - total;
  }
  __syncthreads();
  if (win) {
    t.heap[*s_base + rank] = static_cast<int32_t>(lo32(w));
    t.slots[s] = to_empty ? kEmpty : kTombstone;
    mask[pos] = 1;
  } else if (active) {
    mask[pos] = 0;
  }
  __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(256) erase_resolve_kernel(TableView t, int64_t n, const int32_t* __restrict__ slot_in,
                                                            uint8_t* __restrict__ mask) {
  __shared__ int s_warp[33];
  __shared__ int s_cnt;
  __shared__ int s_base;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride)
    erase_resolve_tile<S>(t, n, base, slot_in, mask, s_warp, &s_cnt, &s_base);
}

// ------------------------------------------------------------------ rebuild
// Inserts n unique keys taken from kb_src rows list[j] into an empty table.
// preserve: the entry keeps buffer index list[j]; otherwise it becomes j.
// The key row is copied to kb_dst when kb_dst != kb_src or !preserve.
template <int D, int S>
// n_dev (optional): the live count on the device (written by the listing);
// the kernel then processes min(n, *n_dev) entries, so a rebuild can be
// enqueued without the host knowing the count.
__global__ void __launch_bounds__(256) rebuild_kernel(TableView t, const int32_t* __restrict__ kb_src,
                                                      const int32_t* __restrict__ list, int64_t n,
                                                      const unsigned long long* __restrict__ n_dev, int preserve,
                                                      int copy_keys) {
  if (n_dev) n = min(n, static_cast<int64_t>(*n_dev));
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
    // the preferred slot first (preferred-slot invariant), then the full probe
    const uint32_t ps = b * S + pref_slot<S>(fingerprint(h));
    bool placed = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + ps), static_cast<unsigned long long>(kEmpty),
                            static_cast<unsigned long long>(word)) == kEmpty;
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
  int sms = 0;   // SM count (0: unknown)
};

// Launch with programmatic stream serialisation: the kernel's blocks may be
// scheduled while the previous kernel on the stream drains, hiding the
// launch latency between the two.  The kernel must execute
// griddepcontrol.wait before it touches memory the previous kernel writes.
template <class... P, class... A>
inline void launch_dependent_smem(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t st,
                                  A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(block));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

template <class... P, class... A>
inline void launch_dependent(void (*kernel)(P...), int grid, int block, cudaStream_t st, A... args) {
  launch_dependent_smem(kernel, grid, block, 0, st, args...);
}

// Blocks of `kernel` (block threads `block`, no dynamic shared memory) that
// fit on one SM, from the occupancy API, cached per kernel and block size.
template <class K>
inline int resident_blocks(K kernel, int block) {
  static int cache[9] = {};  // block / 32 in 1..8
  const int slot = block / 32;
  if (slot < 1 || slot > 8) return 1;
  if (cache[slot] == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess || nb < 1) nb = 1;
    cache[slot] = nb;
  }
  return cache[slot];
}

// Grid of a grid-stride kernel whose registers allow fewer resident blocks
// than the Launch's cap: no more blocks than fit at once, so no thin second
// wave runs at low occupancy.
template <class K>
inline int resident_grid(K kernel, int want, const Launch& L) {
  if (L.sms <= 0) return want;
  const int cap = L.sms * resident_blocks(kernel, L.block);
  return want < cap ? want : cap;
}

inline int grid_for(int64_t n, const Launch& L) {
  int64_t g = (n + L.block - 1) / L.block;
  if (g > L.grid_cap) g = L.grid_cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

// Defined in ash_aux.cu.  Per range (one block each): the row of per-block
// counts counts[p][0..G) becomes its exclusive scan, the row's total goes to
// range_totals[p].
void launch_partition_scan(uint32_t* counts, int G, int P, uint32_t* range_totals, const Launch& L);
// idx[pos] = idx_p[dest[pos]], mask[pos] = mask_p[dest[pos]]: a partitioned
// call's outputs back in input order.
void launch_unpermute(const int32_t* dest, int64_t n, const int32_t* idx_p, const uint8_t* mask_p, int32_t* idx,
                      uint8_t* mask, const Launch& L);

// Blocks of a partition pass over n keys (G) and whole tiles per block.
inline int partition_grid(int64_t n, const Launch& L, int* tiles_per_block) {
  const int64_t tiles = (n + kPartTile - 1) / kPartTile;
  const int64_t cap = L.sms > 0 ? static_cast<int64_t>(L.sms) * 4 : 512;
  const int64_t g0 = tiles < cap ? tiles : cap;
  const int64_t tpb = (tiles + g0 - 1) / g0;
  *tiles_per_block = static_cast<int>(tpb);
  const int64_t g = (tiles + tpb - 1) / tpb;
  return static_cast<int>(g < 1 ? 1 : g);
}

// Count words of a partitioned call on n keys (counts[P][G] and the P range
// totals).
inline int64_t partition_count_words(int64_t n, int log_p, const Launch& L) {
  int tpb = 0;
  const int64_t G = partition_grid(n, L, &tpb);
  return (G + 1) * (int64_t{1} << log_p);
}

// Function table for one key dimension (filled in by ash_dim.cu).  S: slots
// per bucket (4, 8, 16); kpt: keys per thread (1, 2, 4).
struct DimKernels {
  void (*find)(int S, int kpt, const TableView&, const int32_t*, int64_t, int32_t*, uint8_t*, const Launch&);
  void (*claim)(int S, int kpt, int pref, const TableView&, const int32_t*, int64_t, int32_t*, const Launch&);
  void (*commit)(int kpt, const TableView&, const int32_t*, int64_t, int32_t*, uint8_t*, const ValueRow*,
                 const Launch&);
  void (*erase_mark)(int S, const TableView&, const int32_t*, int64_t, int32_t*, const Launch&);
  void (*rebuild)(int S, const TableView&, const int32_t*, const int32_t*, int64_t, const unsigned long long*, int, int,
                  const Launch&);
  void (*neighbors)(int S, const TableView&, const int32_t*, int64_t, int, int64_t, int32_t*, uint8_t*, const Launch&);
  void (*offsets)(int S, const TableView&, const int32_t*, int64_t, const int32_t*, int64_t, int32_t*, uint8_t*,
                  const Launch&);
  void (*find_group)(int S, const TableView&, const int32_t*, int64_t, int32_t*, uint8_t*, const Launch&);
  // stable partition of n key rows by home-bucket range (scratch: see partition_bytes)
  void (*partition)(const int32_t*, int64_t, int, uint32_t*, int32_t*, int32_t*, const Launch&);
  // the same operations on float32 points quantised in the kernels
  void (*find_pts)(int S, int kpt, const TableView&, const PointRows&, int64_t, int32_t*, uint8_t*, const Launch&);
  void (*claim_pts)(int S, int kpt, int pref, const TableView&, const PointRows&, int64_t, int32_t*, const Launch&);
  void (*commit_pts)(int kpt, const TableView&, const PointRows&, int64_t, int32_t*, uint8_t*, const ValueRow*,
                     const Launch&);
};

template <int D>
struct DimLaunchers {
  template <int S, int KPT, class In>
  static void find_sk(const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask, const Launch& L) {
    TraceScope ts(kKFind, L.stream);
    launch_dependent(find_kernel<D, S, KPT, In>, grid_for((n + KPT - 1) / KPT, L), L.block, L.stream, t, keys, n, idx,
                     mask);
  }
  template <int S, class In>
  static void find_s(int kpt, const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask,
                     const Launch& L) {
    if (kpt >= 4) find_sk<S, 4>(t, keys, n, idx, mask, L);
    else if (kpt == 2) find_sk<S, 2>(t, keys, n, idx, mask, L);
    else find_sk<S, 1>(t, keys, n, idx, mask, L);
  }
  template <class In>
  static void find_in(int S, int kpt, const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask,
                      const Launch& L) {
    if (S == 4) find_s<4>(kpt, t, keys, n, idx, mask, L);
    else if (S == 8) find_s<8>(kpt, t, keys, n, idx, mask, L);
    else find_s<16>(kpt, t, keys, n, idx, mask, L);
  }
  static void find(int S, int kpt, const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask,
                   const Launch& L) {
    find_in(S, kpt, t, keys, n, idx, mask, L);
  }
  static void find_pts(int S, int kpt, const TableView& t, const PointRows& p, int64_t n, int32_t* idx,
                       uint8_t* mask, const Launch& L) {
    find_in(S, kpt, t, p, n, idx, mask, L);
  }
  // pref: 1 = preferred slot first (claim_pref_kernel), 0 = bucket load first.
  // The preferred-slot claim always takes one key per thread: with one
  // queued key per lane in its dense rounds it needs 32 registers and runs
  // at full occupancy, 4-8 % faster than two keys per thread on GB300.
  template <int S, int KPT, class In>
  static void claim_sk(int pref, const TableView& t, const In& keys, int64_t n, int32_t* slot_out,
                       const Launch& L) {
    TraceScope ts(kKClaim, L.stream);
    const int g = grid_for((n + KPT - 1) / KPT, L);
    if (pref) {
      auto* k = claim_pref_kernel<D, S, 1, In>;
      launch_dependent(k, resident_grid(k, grid_for(n, L), L), L.block, L.stream, t, keys, n, slot_out);
    } else {
      // (capping this grid at its 4 resident blocks per SM measured 10-15 %
      // slower on 1e7-key tables)
      launch_dependent(claim_bucket_kernel<D, S, KPT, In>, g, L.block, L.stream, t, keys, n, slot_out);
    }
  }
  template <int S, class In>
  static void claim_s(int kpt, int pref, const TableView& t, const In& keys, int64_t n, int32_t* slot_out,
                      const Launch& L) {
    if (kpt >= 4) claim_sk<S, 4>(pref, t, keys, n, slot_out, L);
    else if (kpt == 2) claim_sk<S, 2>(pref, t, keys, n, slot_out, L);
    else claim_sk<S, 1>(pref, t, keys, n, slot_out, L);
  }
  template <class In>
  static void claim_in(int S, int kpt, int pref, const TableView& t, const In& keys, int64_t n, int32_t* slot_out,
                       const Launch& L) {
    if (S == 4) claim_s<4>(kpt, pref, t, keys, n, slot_out, L);
    else if (S == 8) claim_s<8>(kpt, pref, t, keys, n, slot_out, L);
    else claim_s<16>(kpt, pref, t, keys, n, slot_out, L);
  }
  static void claim(int S, int kpt, int pref, const TableView& t, const int32_t* keys, int64_t n, int32_t* slot_out,
                    const Launch& L) {
    claim_in(S, kpt, pref, t, keys, n, slot_out, L);
  }
  static void claim_pts(int S, int kpt, int pref, const TableView& t, const PointRows& p, int64_t n,
                        int32_t* slot_out, const Launch& L) {
    claim_in(S, kpt, pref, t, p, n, slot_out, L);
  }
  template <int KPT, bool VAL, class In>
  static void commit_kv(const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask,
                        const ValueRow& v, const Launch& L) {
    TraceScope ts(kKCommit, L.stream);
    const int g = grid_for((n + KPT - 1) / KPT, L);
    if (t.lost) launch_dependent(commit_kernel<D, KPT, VAL, In, true>, g, L.block, L.stream, t, keys, n, idx, mask, v);
    else launch_dependent(commit_kernel<D, KPT, VAL, In, false>, g, L.block, L.stream, t, keys, n, idx, mask, v);
  }
  template <bool VAL, class In>
  static void commit_v(int kpt, const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask,
                       const ValueRow& v, const Launch& L) {
    if (kpt >= 4) commit_kv<4, VAL>(t, keys, n, idx, mask, v, L);
    else if (kpt == 2) commit_kv<2, VAL>(t, keys, n, idx, mask, v, L);
    else commit_kv<1, VAL>(t, keys, n, idx, mask, v, L);
  }
  // v == nullptr: no inline value copy.
  template <class In>
  static void commit_in(int kpt, const TableView& t, const In& keys, int64_t n, int32_t* idx, uint8_t* mask,
                        const ValueRow* v, const Launch& L) {
    if (v) commit_v<true>(kpt, t, keys, n, idx, mask, *v, L);
    else commit_v<false>(kpt, t, keys, n, idx, mask, ValueRow{}, L);
  }
  static void commit(int kpt, const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask,
                     const ValueRow* v, const Launch& L) {
    commit_in(kpt, t, keys, n, idx, mask, v, L);
  }
  static void commit_pts(int kpt, const TableView& t, const PointRows& p, int64_t n, int32_t* idx, uint8_t* mask,
                         const ValueRow* v, const Launch& L) {
    commit_in(kpt, t, p, n, idx, mask, v, L);
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
  static void rebuild_s(const TableView& t, const int32_t* kb_src, const int32_t* list, int64_t n,
                        const unsigned long long* n_dev, int preserve, int copy_keys, const Launch& L) {
    TraceScope ts(kKRebuild, L.stream);
    rebuild_kernel<D, S><<<grid_for(n, L), L.block, 0, L.stream>>>(t, kb_src, list, n, n_dev, preserve, copy_keys);
  }
  static void rebuild(int S, const TableView& t, const int32_t* kb_src, const int32_t* list, int64_t n,
                      const unsigned long long* n_dev, int preserve, int copy_keys, const Launch& L) {
    if (S == 4) rebuild_s<4>(t, kb_src, list, n, n_dev, preserve, copy_keys, L);
    else if (S == 8) rebuild_s<8>(t, kb_src, list, n, n_dev, preserve, copy_keys, L);
    else rebuild_s<16>(t, kb_src, list, n, n_dev, preserve, copy_keys, L);
  }
  template <int S>
  static void neighbors_s(const TableView& t, const int32_t* keys, int64_t n, int radius, int64_t n_off, int32_t* idx,
                          uint8_t* mask, const Launch& L) {
    TraceScope ts(kKNeighbors, L.stream);
    neighbors_kernel<D, S><<<grid_for(n * n_off, L), L.block, 0, L.stream>>>(t, keys, n, radius, n_off, idx, mask);
  }
  static void neighbors(int S, const TableView& t, const int32_t* keys, int64_t n, int radius, int64_t n_off,
                        int32_t* idx, uint8_t* mask, const Launch& L) {
    if (S == 4) neighbors_s<4>(t, keys, n, radius, n_off, idx, mask, L);
    else if (S == 8) neighbors_s<8>(t, keys, n, radius, n_off, idx, mask, L);
    else neighbors_s<16>(t, keys, n, radius, n_off, idx, mask, L);
  }
  template <int S>
  static void offsets_s(const TableView& t, const int32_t* keys, int64_t n, const int32_t* off, int64_t n_off,
                        int32_t* idx, uint8_t* mask, const Launch& L) {
    TraceScope ts(kKNeighbors, L.stream);
    offsets_kernel<D, S><<<grid_for(n * n_off, L), L.block, 0, L.stream>>>(t, keys, n, off, n_off, idx, mask);
  }
  static void offsets(int S, const TableView& t, const int32_t* keys, int64_t n, const int32_t* off, int64_t n_off,
                      int32_t* idx, uint8_t* mask, const Launch& L) {
    if (S == 4) offsets_s<4>(t, keys, n, off, n_off, idx, mask, L);
    else if (S == 8) offsets_s<8>(t, keys, n, off, n_off, idx, mask, L);
    else offsets_s<16>(t, keys, n, off, n_off, idx, mask, L);
  }
  template <int S>
  static void find_group_s(const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask,
                           const Launch& L) {
    TraceScope ts(kKFind, L.stream);
    constexpr int kKeysPerBlock = 256 / (S / 2);
    int64_t g = (n + kKeysPerBlock - 1) / kKeysPerBlock;
    if (g > L.grid_cap) g = L.grid_cap;
    find_group_kernel<D, S><<<static_cast<int>(g < 1 ? 1 : g), 256, 0, L.stream>>>(t, keys, n, idx, mask);
  }
  static void find_group(int S, const TableView& t, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask,
                         const Launch& L) {
    if (S == 4) find_group_s<4>(t, keys, n, idx, mask, L);
    else if (S == 8) find_group_s<8>(t, keys, n, idx, mask, L);
    else find_group_s<16>(t, keys, n, idx, mask, L);
  }
  // counts: partition_count_words(n, log_p, L) words; keys_out: n rows; dest: n.
  static void partition(const int32_t* keys, int64_t n, int log_p, uint32_t* counts, int32_t* keys_out, int32_t* dest,
                        const Launch& L) {
    TraceScope ts(kKPartition, L.stream, 3);
    int tpb = 0;
    const int G = partition_grid(n, L, &tpb);
    const int P = 1 << log_p;
    uint32_t* range_totals = counts + static_cast<int64_t>(P) * G;
    launch_dependent(partition_count_kernel<D>, G, 256, L.stream, keys, n, log_p, tpb, counts);
    launch_partition_scan(counts, G, P, range_totals, L);
    constexpr size_t smem = partition_scatter_smem<D>();
    static bool attr_set = false;  // per key dimension; above 48 KB the kernel must opt in
    if (!attr_set) {
      cudaFuncSetAttribute(partition_scatter_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
      attr_set = true;
    }
    launch_dependent_smem(partition_scatter_kernel<D>, G, 256, smem, L.stream, keys, n, log_p, tpb,
                          static_cast<const uint32_t*>(counts), static_cast<const uint32_t*>(range_totals), keys_out,
                          dest);
  }
  static DimKernels table() {
    DimKernels k;
    k.partition = &partition;
    k.neighbors = &neighbors;
    k.offsets = &offsets;
    k.find_group = &find_group;
    k.find_pts = &find_pts;
    k.claim_pts = &claim_pts;
    k.commit_pts = &commit_pts;
    k.find = &find;
    k.claim = &claim;
    k.commit = &commit;
    k.erase_mark = &erase_mark;
    k.rebuild = &rebuild;
    return k;
  }
};

// Defined in ash_dim.cu (one translation unit per key dimension).
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
