// ASH reference oracle: a plain, sequential CPU spatial hash map.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  The
// product (the CUDA path in paper_2110_00511_gb300/) never calls it and shares
// no code, header, table or constant with it.
//
// What it computes (Dong et al., "ASH: A Modern Framework for Parallel
// Spatial Hashing in 3D Perception", arXiv 2110.00511):
//   * the index-first SoA hash map of Sec. 4.2: a key k maps to a buffer index
//     i with kB(i) = k and vB_j(i) = v_j (the masked query of Eq. (4)/(6));
//   * the index heap of Sec. 4.3: h : I_c -> I_c with top t, starting at
//     t = 0, allocation reads h[t] and raises t, free lowers t and writes the
//     index back at the new top;
//   * lazy insertion of Sec. 4.3.1: a key that is already present makes the
//     insertion fail and "nothing needs to be done" (no overwrite, no index
//     allocated);
//   * activate of Sec. 5.1: insertion of keys only, value bytes untouched;
//   * erase (the "dynamic" footnote of Sec. 1): remove the key, return its
//     buffer index to the heap;
//   * rehash of Sec. 4.5: x2 growth, collect the active keys and values, batch
//     insert them into the enlarged buffers;
//   * the voxel quantisation of Sec. 6.1 / Eq. (11): floor(p / s) in float32.
//
// Readings of points the paper leaves open:
//   * within one batch, the FIRST occurrence (lowest input position) of a key
//     wins; later duplicates get mask 0;
//   * the index returned with mask 0 is -1 (the paper says "undefined");
//   * erase of duplicated keys in one batch: the first occurrence gets mask 1;
//   * auto-growth: before a batch of N insert/activate keys, if size + N > c,
//     the capacity doubles until size + N <= c (the "x2 strategy" of Sec. 4.5
//     applied to the all-keys bound of Sec. 4.4.2);
//   * active-index listing returns indices in ascending order (the paper does
//     not fix an order; the GPU comparison is order-free).
//
// The map itself is std::unordered_map over the full key tuple: the plain
// definition of a dictionary, with its own hash (FNV-1a over the key bytes),
// independent of any hash the GPU path uses.
//
// ORACLE_MUTANT: when compiled with -DORACLE_MUTANT=n (n >= 1) one plausible
// mistake is planted on purpose; tests/test_oracle_mutants.py builds each
// variant and checks that the oracle's pins reject it.  The default build
// (ORACLE_MUTANT undefined, i.e. 0) is the oracle.
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kMaxKeyDim = 8;
constexpr int kMaxValues = 8;

using Key = std::array<int32_t, kMaxKeyDim>;

struct KeyHash {
  size_t operator()(const Key& k) const {
    // FNV-1a over the bytes of the key tuple.
    uint64_t h = 1469598103934665603ull;
    const unsigned char* p = reinterpret_cast<const unsigned char*>(k.data());
    for (size_t b = 0; b < sizeof(Key); ++b) {
      h ^= p[b];
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h);
  }
};

struct OracleMap {
  int key_dim = 0;
  int64_t capacity = 0;
  int n_values = 0;
  int auto_grow = 1;
  std::vector<int64_t> row_bytes;                 // bytes of one value row, per buffer
  std::unordered_map<Key, int32_t, KeyHash> dict;  // key -> buffer index
  std::vector<int32_t> heap;                       // h, Sec. 4.3
  int64_t top = 0;                                 // t, Sec. 4.3
  std::vector<int32_t> key_buf;                    // kB, capacity x key_dim
  std::vector<std::vector<unsigned char>> val_buf; // vB_j, capacity x row_bytes[j]
};

Key make_key(const int32_t* src, int d) {
  Key k{};
  int used = (ORACLE_MUTANT == 3 && d > 1) ? d - 1 : d;
  for (int j = 0; j < used; ++j) k[j] = src[j];
  return k;
}

void reset_storage(OracleMap* m, int64_t capacity) {
  m->capacity = capacity;
  m->heap.resize(capacity);
  for (int64_t i = 0; i < capacity; ++i) m->heap[i] = static_cast<int32_t>(i);
  m->top = 0;
  m->key_buf.assign(capacity * m->key_dim, 0);
  for (int j = 0; j < m->n_values; ++j) m->val_buf[j].assign(capacity * m->row_bytes[j], 0);
  m->dict.clear();
}

// Heap allocation (Sec. 4.3): the free index sits at h[t]; t is raised.
int32_t heap_alloc(OracleMap* m) {
  int32_t i = m->heap[m->top];
  m->top += 1;
  return i;
}

// Heap free (Sec. 4.3): t is lowered and the freed index is stored at h[t].
void heap_free(OracleMap* m, int32_t i) {
  if (ORACLE_MUTANT == 2 && m->top < m->capacity) m->heap[m->top] = i;
  m->top -= 1;
  if (ORACLE_MUTANT != 2) m->heap[m->top] = i;
}

// Rehash (Sec. 4.5): collect all active keys and values, make buffers of the
// new capacity, and batch insert the collected entries into them.  Entries are
// re-inserted in ascending order of their old buffer index.
int rehash_to(OracleMap* m, int64_t new_capacity) {
  if (new_capacity < static_cast<int64_t>(m->dict.size())) return -1;
  std::vector<std::pair<int32_t, Key>> active;
  active.reserve(m->dict.size());
  for (const auto& kv : m->dict) active.emplace_back(kv.second, kv.first);
  std::sort(active.begin(), active.end(),
            [](const std::pair<int32_t, Key>& a, const std::pair<int32_t, Key>& b) {
              return a.first < b.first;
            });
  std::vector<std::vector<unsigned char>> old_vals(m->n_values);
  for (int j = 0; j < m->n_values; ++j) {
    old_vals[j].resize(active.size() * m->row_bytes[j]);
    for (size_t r = 0; r < active.size(); ++r)
      std::memcpy(&old_vals[j][r * m->row_bytes[j]],
                  &m->val_buf[j][static_cast<size_t>(active[r].first) * m->row_bytes[j]],
                  m->row_bytes[j]);
  }
  reset_storage(m, new_capacity);
  size_t n_back = active.size();
  if (ORACLE_MUTANT == 5 && n_back > 0) n_back -= 1;
  for (size_t r = 0; r < n_back; ++r) {
    int32_t i = heap_alloc(m);
    m->dict.emplace(active[r].second, i);
    for (int c = 0; c < m->key_dim; ++c) m->key_buf[static_cast<size_t>(i) * m->key_dim + c] = active[r].second[c];
    for (int j = 0; j < m->n_values; ++j)
      std::memcpy(&m->val_buf[j][static_cast<size_t>(i) * m->row_bytes[j]],
                  &old_vals[j][r * m->row_bytes[j]], m->row_bytes[j]);
  }
  return 0;
}

// Growth rule applied before a batch of n insert/activate keys.
int grow_for(OracleMap* m, int64_t n) {
  int64_t size = static_cast<int64_t>(m->dict.size());
  if (size + n <= m->capacity) return 0;
  if (!m->auto_grow) return 0;
  int64_t c = std::max<int64_t>(m->capacity, 1);
  while (size + n > c) c = (ORACLE_MUTANT == 7) ? c + 1 : c * 2;
  return rehash_to(m, c);
}

// Lazy insertion (Sec. 4.3.1) processed in input order.  values == nullptr
// means activate (Sec. 5.1): keys only, value rows untouched.
int64_t insert_impl(OracleMap* m, const int32_t* keys, int64_t n, const void* const* values,
                    int32_t* idx, uint8_t* mask) {
  if (grow_for(m, n) != 0) return -1;
  int64_t inserted = 0;
  for (int64_t p = 0; p < n; ++p) {
    Key k = make_key(keys + p * m->key_dim, m->key_dim);
    auto found = m->dict.find(k);
    if (ORACLE_MUTANT == 1 && found != m->dict.end() && values != nullptr) {
      for (int j = 0; j < m->n_values; ++j) {
        const unsigned char* src = static_cast<const unsigned char*>(values[j]) + p * m->row_bytes[j];
        std::memcpy(&m->val_buf[j][static_cast<size_t>(found->second) * m->row_bytes[j]], src,
                    m->row_bytes[j]);
      }
    }
    if (found != m->dict.end() || m->top >= m->capacity) {
      idx[p] = -1;
      mask[p] = 0;
      continue;
    }
    int32_t i = heap_alloc(m);
    m->dict.emplace(k, i);
    for (int c = 0; c < m->key_dim; ++c) m->key_buf[static_cast<size_t>(i) * m->key_dim + c] = k[c];
    if (values != nullptr) {
      for (int j = 0; j < m->n_values; ++j) {
        const unsigned char* src = static_cast<const unsigned char*>(values[j]) + p * m->row_bytes[j];
        std::memcpy(&m->val_buf[j][static_cast<size_t>(i) * m->row_bytes[j]], src, m->row_bytes[j]);
      }
    }
    idx[p] = i;
    mask[p] = 1;
    inserted += 1;
  }
  return inserted;
}

}  // namespace

extern "C" {

void* om_create(int key_dim, int64_t capacity, int n_values, const int64_t* value_row_bytes,
                int auto_grow) {
  if (key_dim < 1 || key_dim > kMaxKeyDim || capacity < 1 || n_values < 0 || n_values > kMaxValues)
    return nullptr;
  OracleMap* m = new OracleMap();
  m->key_dim = key_dim;
  m->n_values = n_values;
  m->auto_grow = auto_grow;
  for (int j = 0; j < n_values; ++j) m->row_bytes.push_back(value_row_bytes[j]);
  m->val_buf.resize(n_values);
  reset_storage(m, capacity);
  return m;
}

void om_destroy(void* h) { delete static_cast<OracleMap*>(h); }

// Returns the number of keys inserted, or -1 if growth failed.
int64_t om_insert(void* h, const int32_t* keys, int64_t n, const void* const* values,
                  int32_t* idx, uint8_t* mask) {
  return insert_impl(static_cast<OracleMap*>(h), keys, n, values, idx, mask);
}

int64_t om_activate(void* h, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask) {
  return insert_impl(static_cast<OracleMap*>(h), keys, n, nullptr, idx, mask);
}

// Masked query, Eq. (4): mask 1 and the buffer index when the key is stored,
// mask 0 and -1 otherwise.
int64_t om_find(void* h, const int32_t* keys, int64_t n, int32_t* idx, uint8_t* mask) {
  OracleMap* m = static_cast<OracleMap*>(h);
  int64_t hits = 0;
  for (int64_t p = 0; p < n; ++p) {
    auto it = m->dict.find(make_key(keys + p * m->key_dim, m->key_dim));
    if (it == m->dict.end()) {
      idx[p] = -1;
      mask[p] = 0;
    } else {
      idx[p] = it->second;
      mask[p] = 1;
      hits += 1;
    }
  }
  return hits;
}

// Erase in input order; the freed index returns to the heap.
int64_t om_erase(void* h, const int32_t* keys, int64_t n, uint8_t* mask) {
  OracleMap* m = static_cast<OracleMap*>(h);
  int64_t erased = 0;
  for (int64_t p = 0; p < n; ++p) {
    auto it = m->dict.find(make_key(keys + p * m->key_dim, m->key_dim));
    if (it == m->dict.end()) {
      mask[p] = 0;
      continue;
    }
    if (ORACLE_MUTANT != 6) heap_free(m, it->second);
    m->dict.erase(it);
    mask[p] = 1;
    erased += 1;
  }
  return erased;
}

int64_t om_size(void* h) { return static_cast<int64_t>(static_cast<OracleMap*>(h)->dict.size()); }
int64_t om_capacity(void* h) { return static_cast<OracleMap*>(h)->capacity; }
int64_t om_heap_top(void* h) { return static_cast<OracleMap*>(h)->top; }

// Active buffer indices in ascending order; returns the count.
int64_t om_active_indices(void* h, int32_t* out) {
  OracleMap* m = static_cast<OracleMap*>(h);
  std::vector<int32_t> v;
  v.reserve(m->dict.size());
  for (const auto& kv : m->dict) v.push_back(kv.second);
  std::sort(v.begin(), v.end());
  std::copy(v.begin(), v.end(), out);
  return static_cast<int64_t>(v.size());
}

int om_rehash(void* h, int64_t new_capacity) {
  OracleMap* m = static_cast<OracleMap*>(h);
  if (new_capacity <= 0) new_capacity = 2 * m->capacity;
  return rehash_to(m, new_capacity);
}

void om_clear(void* h) {
  OracleMap* m = static_cast<OracleMap*>(h);
  m->dict.clear();
  for (int64_t i = 0; i < m->capacity; ++i) m->heap[i] = static_cast<int32_t>(i);
  m->top = 0;
}

// Copies of the buffers (caller owns out arrays of the stated sizes).
void om_copy_keys(void* h, int32_t* out) {
  OracleMap* m = static_cast<OracleMap*>(h);
  std::copy(m->key_buf.begin(), m->key_buf.end(), out);
}
void om_copy_values(void* h, int j, void* out) {
  OracleMap* m = static_cast<OracleMap*>(h);
  std::memcpy(out, m->val_buf[j].data(), m->val_buf[j].size());
}
void om_copy_heap(void* h, int32_t* out) {
  OracleMap* m = static_cast<OracleMap*>(h);
  std::copy(m->heap.begin(), m->heap.end(), out);
}

// Voxel quantisation of Sec. 6.1 and Eq. (11) with l = 1: each coordinate is
// divided by the voxel size and rounded toward minus infinity, in float32.
void om_quantize(const float* points, int64_t n_coords, float voxel, int32_t* keys) {
  for (int64_t j = 0; j < n_coords; ++j) {
    float q = points[j] / voxel;
    keys[j] = (ORACLE_MUTANT == 4) ? static_cast<int32_t>(q) : static_cast<int32_t>(std::floor(q));
  }
}

}  // extern "C"
