// Geometry consumers of the hash map (Sec. 6.2 of the ASH paper):
//   * block keys of a depth frame: pinhole unprojection, then Eq. (11);
//   * the double hash map block allocation (local activate -> the frame's
//     distinct new keys -> global activate + find -> local values := global
//     indices), with an ordered compaction between the two maps;
//   * TSDF integration over hashed voxel blocks: projection and signed
//     distance (Eq. (7)), truncation, the running mean of Eq. (9);
//   * ray casting through the hashed blocks, optionally through the frame's
//     local map (the speed-up described with the double hash map).
//
// Every step that decides something discrete (a pixel, a skip, a voxel, a
// zero crossing) is written with explicitly rounded float32 intrinsics
// (__fmul_rn / __fadd_rn / __fdiv_rn: no contraction into fused
// multiply-adds) in a fixed operation order, so the decisions are
// reproducible bit for bit by any IEEE float32 implementation of the same
// steps.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "ash.h"
#include "ash_internal.h"
#include "ash_trace.h"

namespace ash {
namespace vol {

constexpr int kThreads = 256;
constexpr int kItems = 2;
constexpr int kTile = kThreads * kItems;  // items per compaction tile
constexpr int kScanThreads = 1024;

// Pinhole intrinsics and a world-to-camera pose [R | t] (row-major 3x4).
struct Cam {
  float fx, fy, cx, cy;
  float e[12];
};

__device__ __forceinline__ float rot_t_row(const Cam& k, int a, float x, float y, float z) {
  // (R^T v)_a = ((R_0a x + R_1a y) + R_2a z)
  return __fadd_rn(__fadd_rn(__fmul_rn(k.e[a], x), __fmul_rn(k.e[4 + a], y)), __fmul_rn(k.e[8 + a], z));
}

// Camera centre c = -R^T t.
__device__ __forceinline__ void camera_centre(const Cam& k, float (&c)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = -rot_t_row(k, a, k.e[3], k.e[7], k.e[11]);
}

// x_c = R x + t, row by row: ((r0 x + r1 y) + r2 z) + t.
__device__ __forceinline__ float transform_row(const Cam& k, int a, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(k.e[4 * a], x), __fmul_rn(k.e[4 * a + 1], y)),
                             __fmul_rn(k.e[4 * a + 2], z)),
                   k.e[4 * a + 3]);
}

__device__ __forceinline__ bool depth_valid(float d, float depth_max) { return d > 0.0f && d <= depth_max; }

// ------------------------------------------------------ ordered compaction
// Three launches: per-tile counts, one-block scan of the tile counts, and a
// write pass in which every tile places its flagged items at its offset in
// input order.  Tiles are kTile consecutive items; item q * kThreads + tid of
// a tile belongs to thread tid, so loads stay coalesced and the rank order
// (q, then tid) is input order.

template <class Pred>
__global__ void __launch_bounds__(kThreads) tile_count_kernel(Pred pred, int64_t n, int32_t* __restrict__ tile_count) {
  __shared__ int s_warp[kThreads / 32 + 1];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  int c = 0;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    const int64_t i = base + q * kThreads + threadIdx.x;
    c += (i < n && pred(i)) ? 1 : 0;
  }
  int total = 0;
  block_exclusive_scan(c, total, s_warp);
  if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

// Exclusive scan of n_tiles counts in place; the grand total goes to *total.
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(int32_t* __restrict__ tile, int64_t n_tiles,
                                                                 int64_t* __restrict__ total) {
  __shared__ int s_warp[kScanThreads / 32 + 1];
  int64_t carry = 0;
  for (int64_t base = 0; base < n_tiles; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int v = i < n_tiles ? tile[i] : 0;
    int chunk = 0;
    const int off = block_exclusive_scan(v, chunk, s_warp);
    if (i < n_tiles) tile[i] = static_cast<int32_t>(carry + off);
    carry += chunk;
    __syncthreads();  // s_warp is reused by the next chunk
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class Pred, class Write>
__global__ void __launch_bounds__(kThreads) tile_write_kernel(Pred pred, Write write, int64_t n,
                                                              const int32_t* __restrict__ tile_off) {
  __shared__ int s_warp[kThreads / 32 + 1];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  int64_t out = tile_off[blockIdx.x];
#pragma unroll 1
  for (int q = 0; q < kItems; ++q) {
    const int64_t i = base + q * kThreads + threadIdx.x;
    const bool f = i < n && pred(i);
    int rank = 0, total = 0;
    block_rank(f, rank, total, s_warp);
    if (f) write(i, out + rank);
    out += total;
    __syncthreads();  // s_warp is reused by the next round
  }
}

// ------------------------------------------------------ depth -> block keys
struct DepthValid {
  const float* depth;
  float depth_max;
  __device__ bool operator()(int64_t i) const { return depth_valid(__ldg(depth + i), depth_max); }
};

// Pixel i = py * width + px with depth D: camera point
// [(px - cx) / fx * D, (py - cy) / fy * D, D], world point R^T x_c + c, block
// key floor(x_w / edge) (Eq. (11)).
struct DepthKeyWrite {
  const float* depth;
  Cam cam;
  int32_t width;
  float edge;
  int32_t* keys;
  __device__ void operator()(int64_t i, int64_t o) const {
    const float d = __ldg(depth + i);
    const int32_t py = static_cast<int32_t>(i / width);
    const int32_t px = static_cast<int32_t>(i - static_cast<int64_t>(py) * width);
    const float xc = __fmul_rn(__fdiv_rn(__fsub_rn(static_cast<float>(px), cam.cx), cam.fx), d);
    const float yc = __fmul_rn(__fdiv_rn(__fsub_rn(static_cast<float>(py), cam.cy), cam.fy), d);
    float c[3];
    camera_centre(cam, c);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float xw = __fadd_rn(rot_t_row(cam, a, xc, yc, d), c[a]);
      keys[o * 3 + a] = static_cast<int32_t>(floorf(__fdiv_rn(xw, edge)));
    }
  }
};

// ------------------------------------------------------ double hash map
struct MaskSet {
  const uint8_t* mask;
  __device__ bool operator()(int64_t i) const { return __ldg(mask + i) != 0; }
};

struct UniqueWrite {
  const int32_t* keys;
  const int32_t* idx;
  int key_dim;
  int32_t* unique_keys;
  int32_t* local_idx;
  __device__ void operator()(int64_t i, int64_t o) const {
    for (int j = 0; j < key_dim; ++j) unique_keys[o * key_dim + j] = __ldg(keys + i * key_dim + j);
    local_idx[o] = __ldg(idx + i);
  }
};

// local value row li[r] := global index gi[r] (int32 rows).
__global__ void __launch_bounds__(kThreads) scatter_index_kernel(int32_t* __restrict__ local_values,
                                                                 const int32_t* __restrict__ li,
                                                                 const int32_t* __restrict__ gi, int64_t u) {
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < u;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    local_values[__ldg(li + r)] = __ldg(gi + r);
}

// ------------------------------------------------------ TSDF integration
// One CTA per listed block.  Voxel slot v = (vz * ELL + vy) * ELL + vx (x
// fastest) is handled by thread v mod kThreads, so the value rows are read
// and written in coalesced runs (every row is read; only updated voxels are
// written).  For voxel g = K * ELL + v at x = g * s:
// x_c = R x + t; skipped when z_c <= 0, when the pixel
// (floor(fx * (x_c / z_c) + cx + 1/2), likewise v) is outside the image, when
// the depth there is missing or beyond depth_max, or when
// d^j = D - z_c < -mu.  Otherwise d := (w d + Psi) / (w + 1), w := w + 1 with
// Psi = min(d^j, mu) (Eq. (9) with w^j = 1).
template <int ELL>
__global__ void __launch_bounds__(kThreads) integrate_kernel(const int32_t* __restrict__ kb, int ks, int32_t capacity,
                                                             const int32_t* __restrict__ block_idx,
                                                             float* __restrict__ tsdf, float* __restrict__ weight,
                                                             const float* __restrict__ depth, int32_t width,
                                                             int32_t height, Cam cam, float voxel, float trunc,
                                                             float depth_max) {
  constexpr int kVox = ELL * ELL * ELL;
  constexpr int kPer = kVox / kThreads;  // voxels per thread (2 for 8^3, 16 for 16^3)
  const int32_t bi = __ldg(block_idx + blockIdx.x);
  if (bi < 0 || bi >= capacity) return;
  float* trow = tsdf + static_cast<int64_t>(bi) * kVox;
  float* wrow = weight + static_cast<int64_t>(bi) * kVox;
  // the rows' loads go out together with the key's; they do not depend on it
  float dv[kPer], wv[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    dv[q] = trow[threadIdx.x + q * kThreads];
    wv[q] = wrow[threadIdx.x + q * kThreads];
  }
  const int32_t* key = kb + static_cast<int64_t>(bi) * ks;
  const uint32_t k0 = static_cast<uint32_t>(__ldg(key)) * ELL;
  const uint32_t k1 = static_cast<uint32_t>(__ldg(key + 1)) * ELL;
  const uint32_t k2 = static_cast<uint32_t>(__ldg(key + 2)) * ELL;
  const float fw = static_cast<float>(width), fh = static_cast<float>(height);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int v = threadIdx.x + q * kThreads;
    const int vx = v % ELL, vy = (v / ELL) % ELL, vz = v / (ELL * ELL);
    const float x = __fmul_rn(static_cast<float>(static_cast<int32_t>(k0 + vx)), voxel);
    const float y = __fmul_rn(static_cast<float>(static_cast<int32_t>(k1 + vy)), voxel);
    const float z = __fmul_rn(static_cast<float>(static_cast<int32_t>(k2 + vz)), voxel);
    const float zc = transform_row(cam, 2, x, y, z);
    if (!(zc > 0.0f)) continue;
    const float xc = transform_row(cam, 0, x, y, z);
    const float yc = transform_row(cam, 1, x, y, z);
    const float uf = floorf(__fadd_rn(__fadd_rn(__fmul_rn(cam.fx, __fdiv_rn(xc, zc)), cam.cx), 0.5f));
    const float vf = floorf(__fadd_rn(__fadd_rn(__fmul_rn(cam.fy, __fdiv_rn(yc, zc)), cam.cy), 0.5f));
    if (!(uf >= 0.0f && uf < fw && vf >= 0.0f && vf < fh)) continue;
    // uf, vf are in [0, 2^31): 32-bit conversions (64-bit ones run on the FP64 pipe)
    const float dm = __ldg(depth + static_cast<int64_t>(static_cast<int32_t>(vf)) * width + static_cast<int32_t>(uf));
    if (!depth_valid(dm, depth_max)) continue;
    const float sdf = __fsub_rn(dm, zc);
    if (sdf < -trunc) continue;
    const float psi = fminf(sdf, trunc);
    const float den = __fadd_rn(wv[q], 1.0f);
    trow[v] = __fdiv_rn(__fadd_rn(__fmul_rn(wv[q], dv[q]), psi), den);
    wrow[v] = den;
  }
}

// ------------------------------------------------------ per-tile depth range
// The min-max range estimate of Sec. 6.2: the live blocks of the map a ray
// casting looks up are projected into tiles of kRangeTile x kRangeTile
// pixels, each tile keeping the least and greatest camera depth any of those
// blocks reaches over it.  A ray then samples only inside its tile's range.
// The estimate is conservative, so the result is unchanged: a block's cell of
// samples (the lattice points within half a voxel of it) is widened by half
// a voxel more, its corners' pixel rectangle by one pixel, and a cell that
// reaches the camera plane covers every tile from depth 0.  Samples outside
// every listed cell read missing blocks, which are invalid.
constexpr int kRangeTile = 8;

__global__ void range_reset_kernel(unsigned int* __restrict__ zmin, unsigned int* __restrict__ zmax, int n_tiles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_tiles) {
    zmin[i] = 0x7F800000u;  // +inf: no block over this tile yet
    zmax[i] = 0u;
  }
}

// Thread per live block (grid-stride over at most n_max entries of `live`,
// the first *count_dev of which are valid).  Depths are positive, so their
// float bit patterns order like the values and integer atomics keep the
// extremes.
__global__ void __launch_bounds__(kThreads) block_range_kernel(const int32_t* __restrict__ kb, int ks, int ell,
                                                               const int32_t* __restrict__ live, int64_t n_max,
                                                               const int64_t* __restrict__ count_dev, Cam cam,
                                                               float voxel, int32_t width, int32_t height,
                                                               int tiles_x, int tiles_y, unsigned int* __restrict__ zmin,
                                                               unsigned int* __restrict__ zmax) {
  int64_t n = *count_dev;
  if (n > n_max) n = n_max;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t* key = kb + static_cast<int64_t>(__ldg(live + r)) * ks;
    float lo[3], hi[3];
    bool far_out = false;  // beyond |g| < 2^18 the margins are not proven: cover everything
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int32_t kk = __ldg(key + a);
      far_out |= (kk >= (1 << 18) / ell || kk <= -(1 << 18) / ell);
      const float k = static_cast<float>(kk) * static_cast<float>(ell);
      lo[a] = (k - 1.0f) * voxel;
      hi[a] = (k + static_cast<float>(ell)) * voxel;
    }
    float z_lo = 3.0e38f, z_hi = -3.0e38f, u_lo = 3.0e38f, u_hi = -3.0e38f, v_lo = 3.0e38f, v_hi = -3.0e38f;
    bool behind = false;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      const float x = (corner & 1) ? hi[0] : lo[0];
      const float y = (corner & 2) ? hi[1] : lo[1];
      const float z = (corner & 4) ? hi[2] : lo[2];
      const float xc = cam.e[0] * x + cam.e[1] * y + cam.e[2] * z + cam.e[3];
      const float yc = cam.e[4] * x + cam.e[5] * y + cam.e[6] * z + cam.e[7];
      const float zc = cam.e[8] * x + cam.e[9] * y + cam.e[10] * z + cam.e[11];
      z_lo = fminf(z_lo, zc);
      z_hi = fmaxf(z_hi, zc);
      if (zc <= 1.0e-6f) {
        behind = true;
      } else {
        const float u = cam.fx * (xc / zc) + cam.cx;
        const float v = cam.fy * (yc / zc) + cam.cy;
        u_lo = fminf(u_lo, u);
        u_hi = fmaxf(u_hi, u);
        v_lo = fminf(v_lo, v);
        v_hi = fmaxf(v_hi, v);
      }
    }
    if (!far_out && !(z_hi > 0.0f)) continue;  // wholly behind the camera: no sample (t > 0) reaches it
    int tx0, tx1, ty0, ty1;
    unsigned int zl;
    if (far_out) z_hi = __uint_as_float(0x7F800000u);
    if (behind || far_out) {
      tx0 = 0;
      ty0 = 0;
      tx1 = tiles_x - 1;
      ty1 = tiles_y - 1;
      zl = 0u;
    } else {
      const float px0 = fmaxf(floorf(u_lo) - 1.0f, 0.0f), px1 = fminf(ceilf(u_hi) + 1.0f, width - 1.0f);
      const float py0 = fmaxf(floorf(v_lo) - 1.0f, 0.0f), py1 = fminf(ceilf(v_hi) + 1.0f, height - 1.0f);
      if (!(px0 <= px1 && py0 <= py1)) continue;  // outside the image (or not finite)
      tx0 = static_cast<int>(px0) / kRangeTile;
      tx1 = static_cast<int>(px1) / kRangeTile;
      ty0 = static_cast<int>(py0) / kRangeTile;
      ty1 = static_cast<int>(py1) / kRangeTile;
      zl = __float_as_uint(fmaxf(z_lo, 0.0f));
    }
    const unsigned int zh = __float_as_uint(z_hi);
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        atomicMin(zmin + ty * tiles_x + tx, zl);
        atomicMax(zmax + ty * tiles_x + tx, zh);
      }
  }
}

// ------------------------------------------------------ ray casting
// Thread per pixel.  The ray of pixel (px, py) leaves the camera centre along
// R^T [(px - cx) / fx, (py - cy) / fy, 1]; sample i sits at depth
// t_i = depth_min + i * step, at p = c + t_i * dir, and reads the nearest
// lattice point g = floor(p / s + 1/2) (IEEE float32 division) in block K = floor(g / ELL),
// voxel v = g - K * ELL.  A sample is valid when K is in the map and its
// weight is positive.  The first valid pair d_{i-1} > 0 >= d_i gives the depth
// t_{i-1} + step * d_{i-1} / (d_{i-1} - d_i); 0 when there is none.  With a
// local index map, K is looked up there and its int32 value row names the
// block's index in the volume's buffers.
//
// Two shortcuts leave the result unchanged.  The last block's lookup is kept,
// so consecutive samples in one block cost one probe.  And every rounding
// step of the sample arithmetic is monotone, so each coordinate of g, and of
// K, is monotone in i: if samples i and m > i fall in the same block, so do
// all samples between them.  When a block is missing, the kernel estimates
// the last sample m inside its cell from the ray's exit, recomputes sample m
// exactly as above, and when it still falls in the block jumps over the
// samples up to m (all invalid by definition).
struct RaySample {
  int32_t g[3];
  bool in_range;
};

// i < 2^24, so the conversion to float32 is exact (and int32 keeps it off the
// 64-bit conversion path).
__device__ __forceinline__ RaySample ray_sample(const float (&c)[3], const float (&dw)[3], float depth_min,
                                                float step, float voxel, int32_t i) {
  RaySample r;
  r.in_range = true;
  const float t = __fadd_rn(depth_min, __fmul_rn(__int2float_rn(i), step));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float gf = floorf(__fadd_rn(__fdiv_rn(__fadd_rn(c[a], __fmul_rn(t, dw[a])), voxel), 0.5f));
    r.in_range &= (gf > -1.0e9f && gf < 1.0e9f);
    r.g[a] = r.in_range ? static_cast<int32_t>(gf) : 0;
  }
  return r;
}

template <int ELL, int S>
__device__ __forceinline__ float cast_ray(const TableView& tv, const TableView& local_tv,
                                          const int32_t* __restrict__ local_values, int use_local,
                                          const float* __restrict__ tsdf, const float* __restrict__ weight,
                                          int32_t volume_capacity, const Cam& cam, int32_t width, int64_t pid,
                                          float voxel, float depth_min, float step, float inv_step,
                                          int32_t i_begin, int32_t n_steps) {
  constexpr int kVox = ELL * ELL * ELL;
  constexpr int kShift = ELL == 8 ? 3 : 4;
  const int32_t py = static_cast<int32_t>(pid / width);
  const int32_t px = static_cast<int32_t>(pid - static_cast<int64_t>(py) * width);
  float c[3];
  camera_centre(cam, c);
  const float dcx = __fdiv_rn(__fsub_rn(static_cast<float>(px), cam.cx), cam.fx);
  const float dcy = __fdiv_rn(__fsub_rn(static_cast<float>(py), cam.cy), cam.fy);
  float dw[3], inv_dw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dw[a] = rot_t_row(cam, a, dcx, dcy, 1.0f);
    inv_dw[a] = __fdividef(1.0f, dw[a]);  // only for the skip estimate
  }

  int32_t last[3] = {0, 0, 0};
  int32_t last_bi = -1;
  bool have_last = false;
  bool prev_valid = false;
  float prev_d = 0.0f, prev_t = 0.0f;
  float out = 0.0f;
  for (int32_t i = i_begin; i < n_steps; ++i) {
    const float t = __fadd_rn(depth_min, __fmul_rn(__int2float_rn(i), step));
    const RaySample r = ray_sample(c, dw, depth_min, step, voxel, i);
    bool valid = false;
    float dcur = 0.0f;
    if (r.in_range) {
      const int32_t K[3] = {r.g[0] >> kShift, r.g[1] >> kShift, r.g[2] >> kShift};
      if (!have_last || K[0] != last[0] || K[1] != last[1] || K[2] != last[2]) {
        if (use_local) {
          const int32_t li = find_key<3, S>(local_tv, K);
          last_bi = li >= 0 ? __ldg(local_values + li) : -1;
        } else {
          last_bi = find_key<3, S>(tv, K);
        }
        last[0] = K[0];
        last[1] = K[1];
        last[2] = K[2];
        have_last = true;
      }
      if (last_bi >= 0 && last_bi < volume_capacity) {
        const int v = ((r.g[2] & (ELL - 1)) * ELL + (r.g[1] & (ELL - 1))) * ELL + (r.g[0] & (ELL - 1));
        const int64_t at = static_cast<int64_t>(last_bi) * kVox + v;
        const float w = __ldg(weight + at);
        const float d = __ldg(tsdf + at);
        if (w > 0.0f) {
          valid = true;
          dcur = d;
        }
      } else {
        // missing block: the ray's exit from the cell of samples that map to K
        float t_exit = 3.0e38f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float lo = (static_cast<float>(K[a]) * ELL - 0.5f) * voxel;
          const float hi = (static_cast<float>(K[a]) * ELL + (ELL - 0.5f)) * voxel;
          if (dw[a] > 0.0f) t_exit = fminf(t_exit, (hi - c[a]) * inv_dw[a]);
          else if (dw[a] < 0.0f) t_exit = fminf(t_exit, (lo - c[a]) * inv_dw[a]);
        }
        const float est = floorf((t_exit - t) * inv_step);
        if (est >= 1.0f) {
          int32_t m = i + static_cast<int32_t>(fminf(est, static_cast<float>(n_steps)));
          if (m > n_steps - 1) m = n_steps - 1;
          // confirm with the exact sample arithmetic; one step back if the
          // estimate crossed the face
          for (int tries = 0; tries < 2 && m > i; ++tries, --m) {
            const RaySample rm = ray_sample(c, dw, depth_min, step, voxel, m);
            if (rm.in_range && (rm.g[0] >> kShift) == K[0] && (rm.g[1] >> kShift) == K[1] &&
                (rm.g[2] >> kShift) == K[2]) {
              i = m;  // samples i+1..m are in the missing block
              break;
            }
          }
        }
      }
    }
    if (valid && prev_valid && prev_d > 0.0f && dcur <= 0.0f) {
      out = __fadd_rn(prev_t, __fmul_rn(step, __fdiv_rn(prev_d, __fsub_rn(prev_d, dcur))));
      break;
    }
    prev_valid = valid;
    prev_d = dcur;
    prev_t = t;
  }
  return out;
}

// Persistent grid; each warp takes the next 32 pixels from a counter, so rays
// of uneven length do not leave the tail of the launch idle.  Each ray
// samples only i in [i_begin, i_end) from its tile's depth range, widened by
// two steps on either side; the sample before i_begin lies outside every
// listed cell, so starting there with no valid predecessor is the same as
// marching from 0.
template <int ELL, int S>
__global__ void __launch_bounds__(kThreads) raycast_kernel(TableView tv, TableView local_tv,
                                                           const int32_t* __restrict__ local_values, int use_local,
                                                           const float* __restrict__ tsdf,
                                                           const float* __restrict__ weight, int32_t volume_capacity,
                                                           Cam cam, int32_t width, int64_t n_pixels, float voxel,
                                                           float depth_min, float step,
                                                           float inv_step, int32_t n_steps,
                                                           const unsigned int* __restrict__ zmin,
                                                           const unsigned int* __restrict__ zmax, int tiles_x,
                                                           int use_range, unsigned long long* __restrict__ next_chunk,
                                                           float* __restrict__ depth_out) {
  const int lane = threadIdx.x & 31;
  const uint64_t n_chunks = static_cast<uint64_t>((n_pixels + 31) / 32);
  while (true) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(next_chunk, 1ull);
    chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t pid = static_cast<int64_t>(chunk) * 32 + lane;
    if (pid < n_pixels) {
      const int32_t py = static_cast<int32_t>(pid / width);
      const int32_t px = static_cast<int32_t>(pid - static_cast<int64_t>(py) * width);
      int32_t i0 = 0, i1 = n_steps;
      if (use_range) {
        const int tile = (py / kRangeTile) * tiles_x + px / kRangeTile;
        const float z0 = __uint_as_float(__ldg(zmin + tile));
        const float z1 = __uint_as_float(__ldg(zmax + tile));
        if (z0 <= z1) {
          const float f0 = floorf((z0 - depth_min) * inv_step) - 2.0f;
          const float f1 = ceilf((z1 - depth_min) * inv_step) + 2.0f;
          i0 = f0 <= 0.0f ? 0 : (f0 >= static_cast<float>(n_steps) ? n_steps : static_cast<int32_t>(f0));
          i1 = f1 >= static_cast<float>(n_steps) ? n_steps : (f1 <= 0.0f ? 0 : static_cast<int32_t>(f1));
        } else {
          i1 = 0;  // no listed block over this tile
        }
      }
      float out = 0.0f;
      {
        if (i0 < i1)
          out = cast_ray<ELL, S>(tv, local_tv, local_values, use_local, tsdf, weight, volume_capacity, cam, width, pid,
                                 voxel, depth_min, step, inv_step, i0, i1);
      }
      depth_out[pid] = out;
    }
  }
}

// ------------------------------------------------------ host side
using host::fail;

Cam cam_of(const float* intr, const float* extr) {
  Cam k;
  k.fx = intr[0];
  k.fy = intr[1];
  k.cx = intr[2];
  k.cy = intr[3];
  std::memcpy(k.e, extr, sizeof(k.e));
  return k;
}

void* scratch_alloc(size_t bytes, cudaStream_t st) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

// Ordered compaction with a caller-provided predicate and writer; the count
// lands in *count_dev.  tile scratch: n_tiles int32.
template <class Pred, class Write>
void compact(Pred pred, Write write, int64_t n, int32_t* tile, int64_t* count_dev, cudaStream_t st, int kind) {
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  if (n_tiles == 0) {
    cudaMemsetAsync(count_dev, 0, sizeof(int64_t), st);
    return;
  }
  TraceScope ts(kind, st, 3);
  tile_count_kernel<<<static_cast<unsigned>(n_tiles), kThreads, 0, st>>>(pred, n, tile);
  tile_scan_kernel<<<1, kScanThreads, 0, st>>>(tile, n_tiles, count_dev);
  tile_write_kernel<<<static_cast<unsigned>(n_tiles), kThreads, 0, st>>>(pred, write, n, tile);
}

int ell_of(const ash_map* m, int j) {
  if (j < 0 || j >= m->n_values) return 0;
  if (m->row_bytes[j] == 4 * 8 * 8 * 8) return 8;
  if (m->row_bytes[j] == 4 * 16 * 16 * 16) return 16;
  return 0;
}

thread_local int64_t* t_pinned_count = nullptr;

int64_t* pinned_count() {
  if (!t_pinned_count) {
    if (cudaMallocHost(&t_pinned_count, sizeof(int64_t)) != cudaSuccess) {
      cudaGetLastError();
      t_pinned_count = nullptr;
    }
  }
  return t_pinned_count;
}

}  // namespace vol
}  // namespace ash

using namespace ash::host;
using ash::vol::Cam;

extern "C" {

ash_status ash_depth_to_block_keys(const float* depth, int32_t width, int32_t height, const float* intrinsics_host,
                                   const float* extrinsic_host, float block_edge, float depth_max, int32_t* keys,
                                   int64_t* count_dev, int64_t* count_host, ash_stream stream) {
  if (width < 0 || height < 0) return fail(ASH_ERR_INVALID, "width and height must be >= 0");
  const int64_t n = static_cast<int64_t>(width) * height;
  if (n >= (int64_t{1} << 31)) return fail(ASH_ERR_INVALID, "image too large");
  if (!intrinsics_host || !extrinsic_host) return fail(ASH_ERR_INVALID, "camera arguments are required");
  if (n > 0 && (!depth || !keys)) return fail(ASH_ERR_INVALID, "depth and keys are required");
  if (!count_dev && !count_host) return fail(ASH_ERR_INVALID, "count_dev or count_host is required");
  if (!(block_edge > 0.0f)) return fail(ASH_ERR_INVALID, "block_edge must be > 0");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n_tiles = (n + ash::vol::kTile - 1) / ash::vol::kTile;
  char* scratch = static_cast<char*>(ash::vol::scratch_alloc(16 + 4 * (n_tiles + 1), st));
  if (!scratch) return fail(ASH_ERR_OOM, "scratch allocation failed");
  int64_t* cnt = count_dev ? count_dev : reinterpret_cast<int64_t*>(scratch);
  int32_t* tile = reinterpret_cast<int32_t*>(scratch + 16);
  const Cam cam = ash::vol::cam_of(intrinsics_host, extrinsic_host);
  ash::vol::compact(ash::vol::DepthValid{depth, depth_max},
                    ash::vol::DepthKeyWrite{depth, cam, width, block_edge, keys}, n, tile, cnt, st,
                    ash::kKDepthKeys);
  ash_status s = check_launch("depth_to_block_keys");
  if (s == ASH_OK && count_host) {
    int64_t* pin = ash::vol::pinned_count();
    if (!pin) s = fail(ASH_ERR_OOM, "pinned allocation failed");
    if (s == ASH_OK) {
      cudaMemcpyAsync(pin, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(e, "depth_to_block_keys");
      else *count_host = *pin;
    }
  }
  cudaFreeAsync(scratch, st);
  return s;
}

ash_status ash_double_map_activate(ash_map* local, ash_map* global, const int32_t* keys, int64_t n,
                                   int32_t* unique_keys, int32_t* local_indices, int32_t* global_indices,
                                   int64_t* n_unique_host, ash_stream stream) {
  if (!local || !global || local == global) return fail(ASH_ERR_INVALID, "two distinct maps are required");
  if (local->device != global->device) return fail(ASH_ERR_INVALID, "maps on different devices");
  if (local->key_dim != global->key_dim) return fail(ASH_ERR_INVALID, "maps with different key dimensions");
  if (local->n_values != 1 || local->row_bytes[0] != 4 || local->dtype[0] != ASH_I32)
    return fail(ASH_ERR_INVALID, "the local map needs exactly one int32 value buffer of one element");
  if (!n_unique_host) return fail(ASH_ERR_INVALID, "n_unique_host is required");
  ash_status s = check_keys(local, keys, n);
  if (s != ASH_OK) return s;
  *n_unique_host = 0;
  if (n == 0) return ASH_OK;
  if (!unique_keys || !local_indices || !global_indices) return fail(ASH_ERR_INVALID, "outputs are required");
  DeviceGuard g(local->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n_tiles = (n + ash::vol::kTile - 1) / ash::vol::kTile;
  // scratch: count (16 B) | tile counts | local indices (n) | masks (n)
  const size_t off_tile = 16, off_idx = off_tile + ((4 * n_tiles + 15) / 16) * 16, off_mask = off_idx + 4 * n;
  char* scratch = static_cast<char*>(ash::vol::scratch_alloc(off_mask + n, st));
  if (!scratch) return fail(ASH_ERR_OOM, "scratch allocation failed");
  int64_t* cnt = reinterpret_cast<int64_t*>(scratch);
  int32_t* tile = reinterpret_cast<int32_t*>(scratch + off_tile);
  int32_t* idx_all = reinterpret_cast<int32_t*>(scratch + off_idx);
  uint8_t* mask_all = reinterpret_cast<uint8_t*>(scratch + off_mask);
  int64_t u = 0;
  // 1. local activate
  s = ash_activate(local, keys, n, idx_all, mask_all, stream);
  // 2. the frame's distinct new keys, in input order
  if (s == ASH_OK) {
    ash::vol::compact(ash::vol::MaskSet{mask_all},
                      ash::vol::UniqueWrite{keys, idx_all, local->key_dim, unique_keys, local_indices}, n, tile, cnt,
                      st, ash::kKCompact);
    s = check_launch("double_map_activate");
  }
  if (s == ASH_OK) {
    int64_t* pin = ash::vol::pinned_count();
    if (!pin) s = fail(ASH_ERR_OOM, "pinned allocation failed");
    if (s == ASH_OK) {
      cudaMemcpyAsync(pin, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(e, "double_map_activate");
      else u = *pin;
    }
  }
  // 3. global activate + find; 4. local values := global indices
  if (s == ASH_OK && u > 0) {
    s = ash_activate(global, unique_keys, u, global_indices, mask_all, stream);
    if (s == ASH_OK) s = ash_find(global, unique_keys, u, global_indices, mask_all, stream);
    if (s == ASH_OK) {
      ash::TraceScope ts(ash::kKScatterRows, st);
      ash::vol::scatter_index_kernel<<<grid_for(u, launch_of(local, st)), ash::vol::kThreads, 0, st>>>(
          static_cast<int32_t*>(local->vb[0]), local_indices, global_indices, u);
      s = check_launch("double_map_activate");
    }
  }
  cudaFreeAsync(scratch, st);
  if (s == ASH_OK) *n_unique_host = u;
  return s;
}

ash_status ash_tsdf_integrate(ash_map* blocks, int tsdf_buffer, int weight_buffer, const int32_t* block_indices,
                              int64_t n_blocks, const float* depth, int32_t width, int32_t height,
                              const float* intrinsics_host, const float* extrinsic_host, float voxel_size,
                              float trunc, float depth_max, ash_stream stream) {
  if (!blocks) return fail(ASH_ERR_INVALID, "map is NULL");
  if (blocks->key_dim != 3) return fail(ASH_ERR_INVALID, "the block map needs key_dim 3");
  const int ell = ash::vol::ell_of(blocks, tsdf_buffer);
  if (ell == 0 || ash::vol::ell_of(blocks, weight_buffer) != ell || tsdf_buffer == weight_buffer ||
      blocks->dtype[tsdf_buffer] != ASH_F32 || blocks->dtype[weight_buffer] != ASH_F32)
    return fail(ASH_ERR_INVALID, "tsdf and weight buffers must be distinct float32 rows of 8^3 or 16^3");
  if (n_blocks < 0 || n_blocks >= (int64_t{1} << 31)) return fail(ASH_ERR_INVALID, "n_blocks out of range");
  if (width <= 0 || height <= 0 || !depth) return fail(ASH_ERR_INVALID, "a depth image is required");
  if (!intrinsics_host || !extrinsic_host) return fail(ASH_ERR_INVALID, "camera arguments are required");
  if (!(voxel_size > 0.0f) || !(trunc > 0.0f)) return fail(ASH_ERR_INVALID, "voxel_size and trunc must be > 0");
  if (n_blocks == 0) return ASH_OK;
  if (!block_indices) return fail(ASH_ERR_INVALID, "block_indices is NULL");
  DeviceGuard g(blocks->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  blocks->last_stream = st;
  const Cam cam = ash::vol::cam_of(intrinsics_host, extrinsic_host);
  float* tsdf = static_cast<float*>(blocks->vb[tsdf_buffer]);
  float* weight = static_cast<float*>(blocks->vb[weight_buffer]);
  const int32_t cap = static_cast<int32_t>(blocks->capacity);
  ash::TraceScope ts(ash::kKIntegrate, st);
  if (ell == 8)
    ash::vol::integrate_kernel<8><<<static_cast<unsigned>(n_blocks), ash::vol::kThreads, 0, st>>>(
        blocks->kb, blocks->ks, cap, block_indices, tsdf, weight, depth, width, height, cam, voxel_size, trunc,
        depth_max);
  else
    ash::vol::integrate_kernel<16><<<static_cast<unsigned>(n_blocks), ash::vol::kThreads, 0, st>>>(
        blocks->kb, blocks->ks, cap, block_indices, tsdf, weight, depth, width, height, cam, voxel_size, trunc,
        depth_max);
  return check_launch("tsdf_integrate");
}

ash_status ash_tsdf_raycast(ash_map* blocks, int tsdf_buffer, int weight_buffer, ash_map* local_index_map,
                            const float* intrinsics_host, const float* extrinsic_host, int32_t width, int32_t height,
                            float voxel_size, float depth_min, float step, int64_t n_steps, float* depth_out,
                            ash_stream stream) {
  if (!blocks) return fail(ASH_ERR_INVALID, "map is NULL");
  if (blocks->key_dim != 3) return fail(ASH_ERR_INVALID, "the block map needs key_dim 3");
  const int ell = ash::vol::ell_of(blocks, tsdf_buffer);
  if (ell == 0 || ash::vol::ell_of(blocks, weight_buffer) != ell || blocks->dtype[tsdf_buffer] != ASH_F32 ||
      blocks->dtype[weight_buffer] != ASH_F32)
    return fail(ASH_ERR_INVALID, "tsdf and weight buffers must be float32 rows of 8^3 or 16^3");
  if (local_index_map) {
    if (local_index_map->key_dim != 3 || local_index_map->n_values != 1 || local_index_map->row_bytes[0] != 4 ||
        local_index_map->dtype[0] != ASH_I32 || local_index_map->device != blocks->device ||
        local_index_map->S != blocks->S)
      return fail(ASH_ERR_INVALID, "the local index map needs key_dim 3, one int32 value and the same bucket size");
  }
  if (width <= 0 || height <= 0) return fail(ASH_ERR_INVALID, "width and height must be > 0");
  const int64_t n_pix = static_cast<int64_t>(width) * height;
  if (n_pix >= (int64_t{1} << 31)) return fail(ASH_ERR_INVALID, "image too large");
  if (!depth_out || !intrinsics_host || !extrinsic_host) return fail(ASH_ERR_INVALID, "outputs and camera required");
  if (!(voxel_size > 0.0f) || !(step > 0.0f) || n_steps < 0 || n_steps > (int64_t{1} << 24))
    return fail(ASH_ERR_INVALID, "voxel_size and step must be > 0, n_steps in [0, 2^24]");
  DeviceGuard g(blocks->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  blocks->last_stream = st;
  const Cam cam = ash::vol::cam_of(intrinsics_host, extrinsic_host);
  const ash::TableView tv = view_of(blocks);
  const ash::TableView ltv = local_index_map ? view_of(local_index_map) : tv;
  const int32_t* lvals = local_index_map ? static_cast<const int32_t*>(local_index_map->vb[0]) : nullptr;
  const float* tsdf = static_cast<const float*>(blocks->vb[tsdf_buffer]);
  const float* weight = static_cast<const float*>(blocks->vb[weight_buffer]);
  const int32_t cap = static_cast<int32_t>(blocks->capacity);
  const int use_local = local_index_map ? 1 : 0;
  const float inv_step = 1.0f / step;
  // scratch: chunk counter | live count | tile zmin | tile zmax | live indices
  ash_map* lookup = local_index_map ? local_index_map : blocks;
  const int tiles_x = (width + ash::vol::kRangeTile - 1) / ash::vol::kRangeTile;
  const int tiles_y = (height + ash::vol::kRangeTile - 1) / ash::vol::kRangeTile;
  const int n_tiles = tiles_x * tiles_y;
  const size_t off_tiles = 16, off_live = off_tiles + ((8 * static_cast<size_t>(n_tiles) + 15) / 16) * 16;
  char* scratch = static_cast<char*>(ash::vol::scratch_alloc(off_live + 4 * static_cast<size_t>(lookup->capacity), st));
  if (!scratch) return fail(ASH_ERR_OOM, "scratch allocation failed");
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch);
  int64_t* live_count = reinterpret_cast<int64_t*>(scratch + 8);
  unsigned int* zmin = reinterpret_cast<unsigned int*>(scratch + off_tiles);
  unsigned int* zmax = zmin + n_tiles;
  int32_t* live = reinterpret_cast<int32_t*>(scratch + off_live);
  cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
  // the per-tile depth range (Sec. 6.2's min-max estimate) needs samples at t > 0
  const int use_range = depth_min > 0.0f ? 1 : 0;
  if (use_range) {
    ash_status ls = ash_get_active_indices_async(lookup, live, lookup->capacity, live_count, stream);
    if (ls != ASH_OK) {
      cudaFreeAsync(scratch, st);
      return ls;
    }
    ash::TraceScope tr(ash::kKRayRange, st, 2);
    ash::vol::range_reset_kernel<<<(n_tiles + 255) / 256, 256, 0, st>>>(zmin, zmax, n_tiles);
    ash::vol::block_range_kernel<<<grid_for(lookup->capacity, launch_of(lookup, st)), ash::vol::kThreads, 0, st>>>(
        lookup->kb, lookup->ks, ell, live, lookup->capacity, live_count, cam, voxel_size, width, height, tiles_x,
        tiles_y, zmin, zmax);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t warps_needed = (n_pix + 31) / 32;
  // one wave of resident blocks (all variants use about the same registers)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ash::vol::raycast_kernel<8, 4>, ash::vol::kThreads, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 4;
  }
  int64_t grid64 = static_cast<int64_t>(sm_count(dev)) * per_sm;
  if (grid64 * (ash::vol::kThreads / 32) > warps_needed) grid64 = (warps_needed + 7) / 8;
  const unsigned grid = static_cast<unsigned>(grid64 < 1 ? 1 : grid64);
  ash::TraceScope ts(ash::kKRaycast, st);
#define ASH_RAYCAST(E, SB)                                                                                          \
  ash::vol::raycast_kernel<E, SB><<<grid, ash::vol::kThreads, 0, st>>>(tv, ltv, lvals, use_local, tsdf, weight, cap, \
                                                                       cam, width, n_pix, voxel_size, depth_min,     \
                                                                       step, inv_step,                               \
                                                                       static_cast<int32_t>(n_steps), zmin, zmax,   \
                                                                       tiles_x, use_range, counter, depth_out)
  if (ell == 8) {
    if (blocks->S == 4) ASH_RAYCAST(8, 4);
    else if (blocks->S == 8) ASH_RAYCAST(8, 8);
    else ASH_RAYCAST(8, 16);
  } else {
    if (blocks->S == 4) ASH_RAYCAST(16, 4);
    else if (blocks->S == 8) ASH_RAYCAST(16, 8);
    else ASH_RAYCAST(16, 16);
  }
#undef ASH_RAYCAST
  const ash_status s = check_launch("tsdf_raycast");
  cudaFreeAsync(scratch, st);
  return s;
}

}  // extern "C"
