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
//   * the voxel quantisation of Sec. 6.1 / Eq. (11): floor(p / s) in float32;
//   * the double hash map block allocation of Sec. 6.2 (local activate, the
//     distinct keys, global activate + find, local values := global indices);
//   * the block keys of a depth frame (unprojection, then Eq. (11));
//   * TSDF integration of Sec. 6.2: projection and signed distance (Eq. (7)),
//     truncation, and the incremental weighted mean of Eq. (9) over the voxels
//     of hashed blocks addressed by Eq. (11)-(12);
//   * ray casting of Sec. 6.2: rays marched through the hashed blocks, the
//     first positive-to-negative zero crossing located by linear
//     interpolation.
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
//     not fix an order; the GPU comparison is order-free);
//   * geometry (integration, ray casting): every step that decides something
//     discrete (a pixel, a skip, a voxel, a zero crossing) is taken in float32
//     with a fixed operation order and no fused multiply-add (the library
//     computes in float32); the running mean and the crossing position are
//     kept in float64.  A voxel is sampled at its lattice point g * s.
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


// Double hash map block allocation (Sec. 6.2, the double-hash-map listing):
//   1. activate the frame's keys in the local map;
//   2. keep the keys whose activation succeeded (their first occurrences, in
//      input order) with their local indices;
//   3. activate those keys in the global map, then find them there;
//   4. write each global index into the local map's value buffer 0 (int32
//      rows) at the key's local index.
// Returns the number of distinct new keys u (rows 0..u-1 of the outputs), or
// -1 if an activation failed.
int64_t om_double_map_activate(void* local, void* global, const int32_t* keys, int64_t n, int32_t* unique_keys,
                               int32_t* local_idx, int32_t* global_idx) {
  OracleMap* lm = static_cast<OracleMap*>(local);
  OracleMap* gm = static_cast<OracleMap*>(global);
  const int d = lm->key_dim;
  std::vector<int32_t> li(n);
  std::vector<uint8_t> lmask(n);
  if (n > 0 && om_activate(local, keys, n, li.data(), lmask.data()) < 0) return -1;
  int64_t u = 0;
  for (int64_t p = 0; p < n; ++p) {
    if (!lmask[p]) continue;
    for (int c = 0; c < d; ++c) unique_keys[u * d + c] = keys[p * d + c];
    local_idx[u] = li[p];
    u += 1;
  }
  if (u == 0) return 0;
  std::vector<int32_t> gi(u);
  std::vector<uint8_t> gmask(u);
  if (om_activate(global, unique_keys, u, gi.data(), gmask.data()) < 0) return -1;
  om_find(global, unique_keys, u, global_idx, gmask.data());
  for (int64_t r = 0; r < u; ++r) {
    const int32_t v = (ORACLE_MUTANT == 10) ? local_idx[r] : global_idx[r];
    std::memcpy(&lm->val_buf[0][static_cast<size_t>(local_idx[r]) * lm->row_bytes[0]], &v, sizeof(int32_t));
  }
  (void)gm;
  return u;
}

namespace {

// One float32 operation at a time: every product and sum is rounded before
// the next step (the build passes -ffp-contract=off as well).
inline float mul32(float a, float b) {
  volatile float r = a * b;
  return r;
}
inline float add32(float a, float b) {
  volatile float r = a + b;
  return r;
}
inline float sub32(float a, float b) {
  volatile float r = a - b;
  return r;
}
inline float div32(float a, float b) {
  volatile float r = a / b;
  return r;
}

// Rigid transform of a point by a 3x4 row-major matrix [R | t]:
// ((r0 x + r1 y) + r2 z) + t per row.
void transform32(const float* e, const float x[3], float out[3]) {
  for (int a = 0; a < 3; ++a)
    out[a] = add32(add32(add32(mul32(e[4 * a], x[0]), mul32(e[4 * a + 1], x[1])), mul32(e[4 * a + 2], x[2])),
                   e[4 * a + 3]);
}

// Index of voxel (vx, vy, vz) inside a block's value row: x fastest.
inline int64_t voxel_slot(int ell, int vx, int vy, int vz) {
  return (static_cast<int64_t>(vz) * ell + vy) * ell + vx;
}

}  // namespace

// Voxel-block keys of a depth frame (Sec. 6.2, Eq. (11)): every pixel with a
// depth D in (0, depth_max] is unprojected to the camera point
// [(px - cx) / fx * D, (py - cy) / fy * D, D], taken to the world by the pose
// (x_w = R^T x_c + c with c = -R^T t), and its block key is
// floor(x_w / (s * ell)) per coordinate.  Keys are written in pixel order
// (row-major), skipping pixels without depth; returns their number.
int64_t om_depth_to_block_keys(const float* depth, int width, int height, const float* intr, const float* extr,
                               float block_edge, float depth_max, int32_t* keys) {
  const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
  float c[3];
  for (int a = 0; a < 3; ++a)
    c[a] = -add32(add32(mul32(extr[a], extr[3]), mul32(extr[4 + a], extr[7])), mul32(extr[8 + a], extr[11]));
  int64_t n = 0;
  for (int py = 0; py < height; ++py)
    for (int px = 0; px < width; ++px) {
      const float dm = depth[static_cast<int64_t>(py) * width + px];
      if (!(dm > 0.0f && dm <= depth_max)) continue;
      const float xc[3] = {mul32(div32(sub32(static_cast<float>(px), cx), fx), dm),
                           mul32(div32(sub32(static_cast<float>(py), cy), fy), dm), dm};
      for (int a = 0; a < 3; ++a) {
        const float xw =
            add32(add32(add32(mul32(extr[a], xc[0]), mul32(extr[4 + a], xc[1])), mul32(extr[8 + a], xc[2])),
                  (ORACLE_MUTANT == 11) ? -c[a] : c[a]);
        keys[n * 3 + a] = static_cast<int32_t>(std::floor(div32(xw, block_edge)));
      }
      n += 1;
    }
  return n;
}

// TSDF integration of one depth frame (Sec. 6.2) into the blocks whose buffer
// indices are listed in block_idx.  The oracle's block map holds two float64
// value buffers of ell^3 entries: 0 = signed distance d, 1 = weight w.
//   For voxel v of block K, the lattice point is g = K * ell + v (Eq. (11)-(12)
//   read backwards) and its world position x = g * s.  The camera point
//   [xc, yc, zc] = E x (E = world-to-camera [R | t], the inverse pose of
//   Eq. (7)); pixel u = floor(fx * (xc / zc) + cx + 1/2), likewise v; the
//   measurement is d^j = D(u, v) - zc (Eq. (7)-(8)).  Voxels behind the
//   camera, outside the image, with no depth (D <= 0 or D > depth_max) or
//   with d^j < -mu are left alone.  Otherwise the truncated value
//   Psi(d^j) = clamp(d^j, -mu, mu) enters the running mean of Eq. (9) with
//   w^j = 1.
void om_tsdf_integrate(void* h, const int32_t* block_idx, int64_t n_blocks, int ell, const float* depth, int width,
                       int height, const float* intr, const float* extr, float voxel, float trunc, float depth_max) {
  OracleMap* m = static_cast<OracleMap*>(h);
  const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
  double* tsdf = reinterpret_cast<double*>(m->val_buf[0].data());
  double* weight = reinterpret_cast<double*>(m->val_buf[1].data());
  const int64_t row = static_cast<int64_t>(ell) * ell * ell;
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int32_t bi = block_idx[b];
    if (bi < 0 || bi >= m->capacity) continue;
    const int32_t* key = &m->key_buf[static_cast<size_t>(bi) * m->key_dim];
    for (int vz = 0; vz < ell; ++vz)
      for (int vy = 0; vy < ell; ++vy)
        for (int vx = 0; vx < ell; ++vx) {
          const int32_t g[3] = {key[0] * ell + vx, key[1] * ell + vy, key[2] * ell + vz};
          const float x[3] = {mul32(static_cast<float>(g[0]), voxel), mul32(static_cast<float>(g[1]), voxel),
                              mul32(static_cast<float>(g[2]), voxel)};
          float xc[3];
          transform32(extr, x, xc);
          if (!(xc[2] > 0.0f)) continue;
          const float uf = std::floor(add32(add32(mul32(fx, div32(xc[0], xc[2])), cx), 0.5f));
          const float vf = std::floor(add32(add32(mul32(fy, div32(xc[1], xc[2])), cy), 0.5f));
          if (!(uf >= 0.0f && uf < static_cast<float>(width) && vf >= 0.0f && vf < static_cast<float>(height)))
            continue;
          const float dm = depth[static_cast<int64_t>(vf) * width + static_cast<int64_t>(uf)];
          if (!(dm > 0.0f && dm <= depth_max)) continue;
          const float sdf = sub32(dm, xc[2]);
          if (sdf < -trunc) continue;
          const double psi = static_cast<double>(std::min(sdf, trunc));
          const int64_t at = static_cast<int64_t>(bi) * row + voxel_slot(ell, vx, vy, vz);
          const double w = weight[at];
          tsdf[at] = (ORACLE_MUTANT == 8) ? psi : (w * tsdf[at] + 1.0 * psi) / (w + 1.0);
          weight[at] = w + 1.0;
        }
  }
}

// Ray casting (Sec. 6.2) of the listed pixels (ids py * width + px).  The
// ray of pixel (px, py) leaves the camera centre c = -R^T t along
// R^T [(px - cx) / fx, (py - cy) / fy, 1], so its parameter is the depth along
// the optical axis.  Samples sit at depth t_i = depth_min + i * step,
// i = 0..n_steps-1; sample i at p reads the nearest lattice point
// g = floor(p / s + 1/2) (float32 division), in block K = floor(g / ell) at
// voxel v = g - K * ell, and is valid when K is in the map and the voxel's
// weight is positive.  The first pair of consecutive valid
// samples with d_{i-1} > 0 >= d_i is the surface; its depth is
// t_{i-1} + step * d_{i-1} / (d_{i-1} - d_i).  0 where no crossing is found.
// value_bytes (4 or 8) is the element size of value buffers 0 (d) and 1 (w).
void om_tsdf_raycast(void* h, int ell, int value_bytes, const float* intr, const float* extr, int width,
                     float voxel, float depth_min, float step, int64_t n_steps, const int64_t* pixels,
                     int64_t n_pixels, double* depth_out) {
  OracleMap* m = static_cast<OracleMap*>(h);
  const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
  const int64_t row = static_cast<int64_t>(ell) * ell * ell;
  auto value = [&](int buf, int64_t at) -> double {
    if (value_bytes == 8) return reinterpret_cast<const double*>(m->val_buf[buf].data())[at];
    return static_cast<double>(reinterpret_cast<const float*>(m->val_buf[buf].data())[at]);
  };
  // camera centre c = -R^T t, in float32
  float c[3];
  for (int a = 0; a < 3; ++a)
    c[a] = -add32(add32(mul32(extr[a], extr[3]), mul32(extr[4 + a], extr[7])), mul32(extr[8 + a], extr[11]));
  for (int64_t q = 0; q < n_pixels; ++q) {
    const int64_t pid = pixels[q];
    const float px = static_cast<float>(pid % width), py = static_cast<float>(pid / width);
    const float dc[3] = {div32(sub32(px, cx), fx), div32(sub32(py, cy), fy), 1.0f};
    float dw[3];
    for (int a = 0; a < 3; ++a)
      dw[a] = add32(add32(mul32(extr[a], dc[0]), mul32(extr[4 + a], dc[1])), mul32(extr[8 + a], dc[2]));
    double out = 0.0;
    bool prev_valid = false;
    double prev_d = 0.0;
    float prev_t = 0.0f;
    for (int64_t i = 0; i < n_steps; ++i) {
      const float t = add32(depth_min, mul32(static_cast<float>(i), step));
      bool valid = false;
      double dcur = 0.0;
      int32_t g[3];
      bool in_range = true;
      for (int a = 0; a < 3; ++a) {
        const float gf = std::floor(add32(div32(add32(c[a], mul32(t, dw[a])), voxel), 0.5f));
        if (!(gf > -1.0e9f && gf < 1.0e9f)) in_range = false;
        g[a] = in_range ? static_cast<int32_t>(gf) : 0;
      }
      if (in_range) {
        Key k{};
        int32_t v[3];
        for (int a = 0; a < 3; ++a) {
          const int32_t kb = (g[a] >= 0) ? g[a] / ell : -((-g[a] + ell - 1) / ell);
          k[a] = kb;
          v[a] = g[a] - kb * ell;
        }
        auto it = m->dict.find(k);
        if (it != m->dict.end()) {
          const int64_t at = static_cast<int64_t>(it->second) * row + voxel_slot(ell, v[0], v[1], v[2]);
          if (value(1, at) > 0.0) {
            valid = true;
            dcur = value(0, at);
          }
        }
      }
      if (valid && prev_valid && prev_d > 0.0 && dcur <= 0.0) {
        out = (ORACLE_MUTANT == 9) ? static_cast<double>(t)
                                   : static_cast<double>(prev_t) + static_cast<double>(step) * prev_d / (prev_d - dcur);
        break;
      }
      prev_valid = valid;
      prev_d = dcur;
      prev_t = t;
    }
    depth_out[q] = out;
  }
}

}  // extern "C"
