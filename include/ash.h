/*
 * ash.h -- C ABI of a GB300 (sm_103a) parallel spatial hash map.
 *
 * The operations follow the problem statement of ASH (Dong et al., "ASH: A
 * Modern Framework for Parallel Spatial Hashing in 3D Perception", arXiv
 * 2110.00511):
 *   - Sec. 4.2: an index-first structure-of-arrays map.  A key k is stored at a
 *     buffer index i of a key buffer kB and of one or more value buffers vB_j
 *     (Sec. 4.7), and queries return (buffer indices, masks) instead of
 *     pointers to pairs (the masked query, Eq. (4)).
 *   - Sec. 4.3: buffer indices come from an index heap h with top t.
 *   - Sec. 4.3.1: insertion is lazy; a key already present is left untouched.
 *   - Sec. 5.1: activate inserts keys only and returns their indices.
 *   - Sec. 1 (footnote on "dynamic" maps): erase.
 *   - Sec. 4.5: rehash (x2 growth, re-insertion of the active entries).
 *   - Sec. 4.6: keys are int32 tuples of any dimension 1..8; float keys must be
 *     quantised first (see ash_quantize, Sec. 6.1).
 *   - Sec. 4.7: a hash set is a map with zero value buffers.
 *
 * Conventions for every call
 *   - Pointers are DEVICE pointers of the map's device unless the name ends in
 *     _host.  The caller owns every input and output array; the library owns
 *     the table, the heap and the key/value buffers.  Where the device can
 *     access pageable host memory (ash_get_device_info: a coherent CPU-GPU
 *     system), the key, value, index, mask and point arrays of the map calls,
 *     ash_quantize and the gathers may instead be ordinary host memory: the
 *     kernels read and write it in place, with no staging copy.  The call
 *     returns before the kernels finish, so such host arrays must stay valid
 *     and untouched until the stream has reached that point.
 *   - Keys are row-major int32 [n, key_dim] with no padding.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue their kernels on it and return without waiting unless the
 *     description says "synchronises".
 *   - Within one batch the FIRST occurrence (lowest position) of a key is the
 *     one that inserts or erases; later duplicates get mask 0.
 *   - An output index whose mask is 0 is -1 (the paper leaves it undefined).
 *   - n = 0 is a valid no-op.  n must be below 2^31 - 1.
 *   - Return value: ASH_OK or an error code; ash_last_error() gives a message
 *     for the calling thread.  Errors found by a kernel (a key that could not
 *     be placed) clear that key's mask, set its index to -1 and are also
 *     reported by the next synchronising call or by ash_sync_status.
 */
#ifndef ASH_H_
#define ASH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ash_map ash_map;
/* Same type as cudaStream_t; declared here so this header needs no CUDA headers. */
typedef struct CUstream_st* ash_stream;

typedef enum ash_status {
  ASH_OK = 0,
  ASH_ERR_INVALID = 1,    /* bad argument */
  ASH_ERR_OOM = 2,        /* device allocation failed */
  ASH_ERR_CAPACITY = 3,   /* auto-grow off and the index heap ran out */
  ASH_ERR_TABLE_FULL = 4, /* a key found no free slot within max_probes buckets */
  ASH_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
  ASH_ERR_CUDA = 6        /* any other CUDA error */
} ash_status;

typedef enum ash_dtype {
  ASH_F32 = 0, ASH_F16 = 1, ASH_BF16 = 2, ASH_I32 = 3, ASH_I64 = 4, ASH_U8 = 5, ASH_F64 = 6
} ash_dtype;

/* Layout and launch knobs.  Structural fields (slots_per_bucket,
 * slots_per_capacity) take effect at create and at the next rehash. */
typedef struct ash_tuning {
  int32_t slots_per_bucket;   /* 4, 8 or 16 eight-byte slots: 32, 64 or 128 B buckets */
  float slots_per_capacity;   /* table slots per unit of capacity (2.0: load <= 0.5) */
  int32_t block_threads;      /* threads per block of the map kernels (multiple of 32, <= 256) */
  int32_t blocks_per_sm;      /* grid = SM count x blocks_per_sm (grid-stride loops) */
  int32_t max_probes;         /* bucket probes before a key fails; 0 = every bucket */
  int32_t auto_grow;          /* 1: insert/activate double the capacity until size+n <= c (Sec. 4.5) */
  float max_used_fraction;    /* rebuild the table when live+erased slots would pass this fraction
                                 (0.65: erased slots stay as tombstones until a rebuild, and with
                                 linear bucket probing a lookup that misses walks 1.5 buckets on
                                 average at 0.6 of the slots used but 6 at 0.85) */
  int32_t inline_value_bytes; /* a map with ONE value buffer whose rows are 4, 8 or 16 bytes (at most
                                 this limit, both bases aligned to the row size) has them copied by
                                 the committing thread; other layouts use a warp-per-row scatter
                                 kernel after the commit */
  int32_t keys_per_thread;    /* 1, 2 or 4 keys handled together by each thread of the find,
                                 bucket-first claim and commit kernels (more independent memory
                                 requests in flight); the preferred-slot claim takes one key per
                                 thread */
  int32_t warp_probe;         /* find: 0 = one thread per key (keys_per_thread keys each);
                                 1 = warp-cooperative probing, a group of slots_per_bucket / 2 lanes
                                 per key, each lane comparing two slots from one 16-byte load and
                                 verifying its matches with a 128-bit kB load, the group agreeing
                                 by warp ballot */
  int32_t find_keys_per_thread; /* keys per thread of the thread-per-key find: 1, 2 or 4, or 0 to use
                                   keys_per_thread (the find's dependent reads favour one key per
                                   thread and full occupancy on mid-sized tables) */
  int32_t claim_mode;         /* insert/activate claim protocol: 1 = load the home bucket, then CAS
                                 its first EMPTY slot; 2 = CAS the key's preferred slot of its
                                 home bucket with no load before it, keys that find it taken are
                                 claimed from their buckets in dense warp rounds; 0 = 2 while the
                                 table takes at most two thirds of L2, else 1 (a CAS that misses
                                 L2 waits on DRAM).  2 needs every key placed preferred-first:
                                 after a call that ran 1, or a batched insert (ash_batch_run),
                                 the map uses 1 until its next clear or rebuild */
  int32_t commit_keys_per_thread; /* keys per thread of the insert commit kernel: 1, 2 or 4, or 0
                                     to use keys_per_thread (its reads are streamed, so one key
                                     per thread and full occupancy usually win) */
  int32_t partition_keys;     /* find, activate, and insert into a map without value buffers:
                                 1 = use the keys in input order; 2 = first put them in the order
                                 of their home buckets' ranges (a stable partition into ranges of
                                 about L2/2 bytes of table each, 8 ranges at least) and work range
                                 by range, each range's table buckets prefetched into L2 before its
                                 keys, so that the kernels find the table (and kB) in L2 instead of
                                 missing at random; the outputs come back in input order, and equal
                                 keys keep their input order (the first occurrence still wins);
                                 0 = 2 for calls of at least 2^20 keys on a table larger than twice
                                 L2, else 1 (a ranged find reads kB in range order only when the
                                 inserts were ranged too, so both switch together).  Takes about
                                 9 + 4d bytes of stream-ordered scratch per key during the call;
                                 if that cannot be had the call uses input order */
} ash_tuning;

/* Fills *out with the defaults. */
void ash_default_tuning(ash_tuning* out);

/* Optional device allocator used for every buffer the library owns (the table,
 * key/value buffers, heap, scratch).  alloc returns NULL on failure.  Without
 * one, the library uses cudaMallocAsync/cudaFreeAsync from the device's
 * default memory pool on the call's stream.  Applies to maps created after the
 * call.  Passing NULLs restores the default. */
typedef void* (*ash_alloc_fn)(size_t bytes, int device, ash_stream stream, void* ctx);
typedef void (*ash_free_fn)(void* ptr, int device, ash_stream stream, void* ctx);
ash_status ash_set_allocator(ash_alloc_fn alloc_fn, ash_free_fn free_fn, void* ctx);

/* Creates a map on `device` (Sec. 4.2 and 4.7; the constructor of the paper's
 * HashMap(capacity, key dtype/shape, value dtypes/shapes)).
 *   key_dim:           1..8 int32 coordinates per key.
 *   capacity:          c, the maximum number of live entries (heap size),
 *                      1 <= c and c * slots_per_capacity < 2^31.
 *   n_values:          0..8 value buffers; 0 makes a hash set.
 *   value_numel_host:  elements per value row of buffer j (e.g. 512 for 8^3).
 *   value_dtypes_host: ash_dtype per buffer.
 *   tuning:            NULL for the defaults.
 * The key buffer is int32 [c, key_stride] (key_stride = 1, 2, 4 or 8 >= key_dim;
 * a row is written whole, padding zeroed, when its index is handed out; rows
 * never handed out are unspecified), value buffer j is [c, numel_j] of its
 * dtype, zero-filled.
 * The table starts empty and the heap as the identity with t = 0. */
ash_status ash_create(int key_dim, int64_t capacity, int n_values, const int64_t* value_numel_host,
                      const int32_t* value_dtypes_host, int device, const ash_tuning* tuning,
                      ash_stream stream, ash_map** out_host);

/* Frees every buffer of the map, stream-ordered on the stream of its last
 * call.  Work that used the map on other streams must be ordered before that
 * stream first (e.g. make it wait on those streams). */
ash_status ash_destroy(ash_map* map);

/* Lazy insertion (Sec. 4.3.1) of n keys with their values.
 *   values_host: host array of n_values device pointers; pointer j addresses
 *                [n, numel_j] rows of buffer j's dtype.
 *   buf_indices: int32 [n] out; the new buffer index, or -1.
 *   masks:       uint8 [n] out; 1 where this position inserted a new key.
 * A key already in the map, or a later duplicate within the batch, gets mask
 * 0 and its stored value is not changed.  With auto_grow the capacity first
 * doubles until size + n <= c (may synchronise). */
ash_status ash_insert(ash_map* map, const int32_t* keys, const void* const* values_host, int64_t n,
                      int32_t* buf_indices, uint8_t* masks, ash_stream stream);

/* Activate (Sec. 5.1): insertion of keys only.  Value rows of new entries are
 * left as they are (zero for never-used indices, stale bytes for indices
 * re-used after erase).  Outputs as ash_insert. */
ash_status ash_activate(ash_map* map, const int32_t* keys, int64_t n, int32_t* buf_indices,
                        uint8_t* masks, ash_stream stream);

/* Masked query (Eq. (4)): mask 1 and the buffer index i with kB(i) = key where
 * the key is stored; mask 0 and -1 elsewhere. */
ash_status ash_find(ash_map* map, const int32_t* keys, int64_t n, int32_t* buf_indices,
                    uint8_t* masks, ash_stream stream);

/* The same operations on float32 points [n, key_dim]: each row's key is
 * floor(p / cell) per coordinate, computed where the row is read, with an
 * IEEE float32 division and rounding toward minus infinity (bit-identical to
 * ash_quantize, the voxel key of Sec. 6.1).  Results, growth and errors are
 * those of ash_insert / ash_activate / ash_find on the quantised keys; no key
 * array is written.  cell > 0; the quantised keys must fit int32. */
ash_status ash_insert_points(ash_map* map, const float* points, float cell, const void* const* values_host, int64_t n,
                             int32_t* buf_indices, uint8_t* masks, ash_stream stream);
ash_status ash_activate_points(ash_map* map, const float* points, float cell, int64_t n, int32_t* buf_indices,
                               uint8_t* masks, ash_stream stream);
ash_status ash_find_points(ash_map* map, const float* points, float cell, int64_t n, int32_t* buf_indices,
                           uint8_t* masks, ash_stream stream);

/* Erase: removes each stored key and returns its buffer index to the heap.
 *   masks: uint8 [n] out; 1 at the first position of each key that was
 *          stored, 0 elsewhere.
 * Uses n * 4 bytes of map-owned scratch, grown on demand (a device
 * allocation the first time a batch is larger than any before it; see
 * ash_erase_noalloc for the form that allocates nothing). */
ash_status ash_erase(ash_map* map, const int32_t* keys, int64_t n, uint8_t* masks, ash_stream stream);

/* Allocation-free erase.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library allocate device memory (a host
 * whose device memory is fully budgeted by its own allocator, or a
 * latency-bound loop where a first-time allocation, which may synchronise the
 * device, is not acceptable).  Same semantics and outputs as ash_erase, but
 * its per-key scratch is a fixed device array inside libash.so
 * (ASH_ERASE_NOALLOC_MAX_KEYS int32 = 4 MiB, held on every GPU that loads the
 * library until the process exits) instead of map-owned memory; it calls no
 * allocator.
 *   n > ASH_ERASE_NOALLOC_MAX_KEYS: returns ASH_ERR_INVALID, nothing runs.
 *   The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   All calls share the array, which keeps the previous call's contents:
 *   calls whose kernels can overlap on the GPU (other streams, other maps on
 *   the same device) race on it and must be ordered by the caller. */
#define ASH_ERASE_NOALLOC_MAX_KEYS (1 << 20)
ash_status ash_erase_noalloc(ash_map* map, const int32_t* keys, int64_t n, uint8_t* masks, ash_stream stream);

/* Lists the buffer indices of all live entries (the "active" entries that
 * Sec. 4.5 collects for rehash).  The order is unspecified; it is made of
 * ascending runs (each covering 8192 consecutive indices).  Writes at most
 * out_capacity indices to out and the live count to *count_host.  Uses
 * about c/8 bytes of library-owned scratch (grown on demand).
 * Synchronises the stream. */
ash_status ash_get_active_indices(ash_map* map, int32_t* out, int64_t out_capacity,
                                  int64_t* count_host, ash_stream stream);

/* Asynchronous listing: as ash_get_active_indices, but enqueued with no host
 * synchronisation; the live count is written to *count_dev (an int64 in
 * device memory) when the listing kernels finish.  Pair it with the *_count
 * gathers below to keep a whole pipeline free of host round trips. */
ash_status ash_get_active_indices_async(ash_map* map, int32_t* out, int64_t out_capacity, int64_t* count_dev,
                                        ash_stream stream);

/* Gathers of key rows / value rows (as ash_gather_keys / ash_gather_values)
 * over min(n_max, *n_dev) indices, n_dev being an int64 in device memory
 * (e.g. the count of ash_get_active_indices_async). */
ash_status ash_gather_keys_count(ash_map* map, const int32_t* indices, int64_t n_max, const int64_t* n_dev,
                                 int32_t* out, ash_stream stream);
ash_status ash_gather_values_count(ash_map* map, int j, const int32_t* indices, int64_t n_max, const int64_t* n_dev,
                                   void* out, ash_stream stream);

/* Number of live entries (the heap top t).  Synchronises the stream. */
ash_status ash_size(ash_map* map, int64_t* size_host, ash_stream stream);

/* Table health of a map: capacity, table slots, live entries (the heap top
 * t), used slots (live entries plus tombstones: erased slots stay
 * tombstones until a rebuild when their bucket has no EMPTY slot), growth
 * checks that had to synchronise a stream, and table rebuilds (growth,
 * rehash, reserve, and clean-ups of erased slots).  Synchronises the stream. */
typedef struct ash_map_stats {
  int64_t capacity;
  int64_t table_slots;
  int64_t live;
  int64_t used_slots;
  int64_t host_syncs;
  int64_t rebuilds;
} ash_map_stats;
ash_status ash_get_map_stats(ash_map* map, ash_map_stats* out_host, ash_stream stream);

/* Capacity c, key dimension, and value-buffer count. */
int64_t ash_capacity(const ash_map* map);
int ash_key_dim(const ash_map* map);
int ash_n_values(const ash_map* map);

/* Rehash (Sec. 4.5) to new_capacity (0 = 2c).  new_capacity must be >= the
 * live count.  When new_capacity >= c the live entries keep their buffer
 * indices (buffers grow, the table is rebuilt); below c they are renumbered
 * 0..size-1.  Invalidates pointers from ash_key_buffer / ash_value_buffer.
 * Synchronises the stream. */
ash_status ash_rehash(ash_map* map, int64_t new_capacity, ash_stream stream);

/* Grows the capacity to at least new_capacity (no-op if already there). */
ash_status ash_reserve(ash_map* map, int64_t new_capacity, ash_stream stream);

/* Like ash_reserve, but enqueued on the stream with no host synchronisation:
 * the live count stays on the device (the listing writes it, the rebuild
 * reads it).  Keeps buffer indices.  Pointers from ash_key_buffer /
 * ash_value_buffer are invalidated. */
ash_status ash_reserve_async(ash_map* map, int64_t new_capacity, ash_stream stream);

/* Removes every entry: empty table, identity heap, t = 0.  Value bytes stay. */
ash_status ash_clear(ash_map* map, ash_stream stream);

/* The key buffer kB (int32 [c, *row_stride]) and value buffer vB_j
 * ([c, numel_j], *row_bytes per row).  Device pointers owned by the map; valid
 * until the next rehash, reserve, growth or destroy. */
ash_status ash_key_buffer(ash_map* map, int32_t** ptr_host, int64_t* row_stride_host);
ash_status ash_value_buffer(ash_map* map, int j, void** ptr_host, int64_t* row_bytes_host);

/* The index heap h (int32 [c]) and a device pointer to its top t (int32, the
 * low word of the map's control word).  For invariant checks. */
ash_status ash_heap_buffer(ash_map* map, int32_t** heap_host, int32_t** top_host);

/* Gathers key rows: out[r, 0:key_dim] = kB(indices[r]); rows whose index is
 * outside [0, c) are written as zeros.  out is int32 [n, key_dim]. */
ash_status ash_gather_keys(ash_map* map, const int32_t* indices, int64_t n, int32_t* out,
                           ash_stream stream);

/* Gathers value rows: out row r = vB_j(indices[r]) (row_bytes of buffer j
 * each); rows whose index is outside [0, c) are written as zeros. */
ash_status ash_gather_values(ash_map* map, int j, const int32_t* indices, int64_t n, void* out, ash_stream stream);

/* Radius neighbour query (the radius search of Sec. 6.2): for every key
 * keys[r] and every integer offset o in [-radius, radius]^key_dim, enumerated
 * row-major (the first coordinate slowest), finds keys[r] + o (int32
 * wrap-around).  buf_indices and masks are [n, (2*radius+1)^key_dim]; entry
 * [r, m] is the masked query (Eq. (4)) of keys[r] + offset m.  The offset
 * keys are formed inside the kernel, never materialised.  radius <= 8. */
ash_status ash_find_neighbors(ash_map* map, const int32_t* keys, int64_t n, int32_t radius, int32_t* buf_indices,
                              uint8_t* masks, ash_stream stream);

/* Neighbour query over an explicit offset table: the 1-radius (3^d), 1-cube
 * (2^d, the grid points enclosing a cell) and 1-ring (the 2d face
 * neighbours) tables of Sec. 6.2 and Sec. 6.4, or any other.  offsets is
 * [n_offsets, key_dim] int32 in device memory (1 <= n_offsets <= 4096);
 * entry [r, m] of buf_indices / masks ([n, n_offsets]) is the masked query
 * (Eq. (4)) of keys[r] + offsets[m] (int32 wrap-around). */
ash_status ash_find_offsets(ash_map* map, const int32_t* keys, int64_t n, const int32_t* offsets, int64_t n_offsets,
                            int32_t* buf_indices, uint8_t* masks, ash_stream stream);

ash_status ash_get_tuning(const ash_map* map, ash_tuning* out_host);
ash_status ash_set_tuning(ash_map* map, const ash_tuning* tuning_host);

/* Synchronises the stream and returns (then clears) the first error that a
 * kernel of this map reported since the last check. */
ash_status ash_sync_status(ash_map* map, ash_stream stream);

/* ---------------------------------------------------------------------------
 * Batched execution: one CUDA-graph launch services many maps (the paper has
 * no batched form; it applies the per-map operations above to many maps at
 * once).  Phases run in the order insert/activate -> find -> erase, each as
 * one persistent kernel over all maps of the batch, so a map with an insert
 * and a find in one batch sees its insert first.
 *   ops_host: n_ops (<= 256) operations, at most one per (map, phase), on maps
 *             of the batch's device with key_dim 1..4.  An insert on a map
 *             with values needs exactly one value buffer of 4, 8 or 16-byte
 *             rows, `values` aligned to the row size; other maps use
 *             activate.  buf_indices is unused for erase.
 *   Outputs and growth are as for the single-map calls (may synchronise to
 *   grow a map).  The call returns after enqueueing; the batch context keeps
 *   a ring of 4 descriptor slots and waits only when it reuses a slot whose
 *   previous launch has not finished. */
typedef struct ash_batch ash_batch;
typedef enum ash_op { ASH_OP_INSERT = 0, ASH_OP_ACTIVATE = 1, ASH_OP_FIND = 2, ASH_OP_ERASE = 3 } ash_op;
typedef struct ash_batch_op {
  ash_map* map;
  int32_t op;                /* ash_op */
  int32_t pad;
  const int32_t* keys;       /* [n, key_dim] */
  const void* values;        /* insert only: [n] rows of the map's value buffer 0 */
  int64_t n;
  int32_t* buf_indices;      /* [n] out (insert, activate, find) */
  uint8_t* masks;            /* [n] out */
} ash_batch_op;
ash_status ash_batch_create(int device, ash_batch** out_host);
ash_status ash_batch_destroy(ash_batch* batch);
ash_status ash_batch_run(ash_batch* batch, const ash_batch_op* ops_host, int n_ops, ash_stream stream);

/* Autotuner: times activate + find on synthetic keys of this shape (n =
 * min(capacity, 2^20) keys, uniqueness `rho` in (0, 1]) for candidate bucket
 * sizes, table slots per unit of capacity, keys per thread and thread-per-key
 * vs warp-cooperative probing, and writes the
 * fastest tuning to *out_host.  Results are cached per (device, key_dim,
 * capacity class, rho class).  Synchronises the stream. */
ash_status ash_autotune(int key_dim, int64_t capacity, float rho, int device, ash_stream stream,
                        ash_tuning* out_host);

/* ---------------------------------------------------------------------------
 * Multi-tenant serving with continuous batching (no counterpart in the paper;
 * it serves the per-map operations above to many clients).  Tenant maps stay
 * resident.  ash_server_submit copies a request's keys (and values) from host
 * memory into pinned staging and queues it (with zero_copy the kernels use the
 * caller's arrays in place instead); a worker thread admits queued
 * requests in arrival order while their device staging fits staging_bytes,
 * batches at most one request per tenant (so each tenant's requests apply in
 * arrival order), grows a tenant map x2 before an insert would push its
 * live/capacity ratio past max_load (and rebuilds its table when erased
 * slots would pass the map's max_used_fraction) on a growth stream, leaving
 * that tenant out of batches until the growth finishes, and runs each batch
 * as one ash_batch_run graph between an upload and a download on separate
 * streams.
 * Requests that arrive while batches are on the GPU join the next batch.
 *   ash_server_wait: blocks until the request's outputs are on the host,
 *     in the caller's buf_indices/masks (given at submit; they must stay
 *     valid until then: page-locked output arrays receive the outputs by DMA,
 *     others by a copy from pinned staging here) and returns the latency from
 *     submit to outputs on the host.  timeout_ms < 0 waits forever; a timeout returns
 *     ASH_ERR_TIMEOUT and the request can be waited for again.
 *   ash_server_map / ash_server_stream: a tenant map and the stream its
 *     kernels run on, for inspection after all submitted requests were
 *     waited for.
 *   ash_server_destroy: finishes queued requests, then frees everything. */
typedef struct ash_server ash_server;
typedef struct ash_server_config {
  int32_t n_tenants;          /* 1..256 resident maps */
  int32_t key_dim;            /* 1..4 */
  int64_t initial_capacity;   /* per tenant */
  int32_t value_row_bytes;    /* 0 (hash sets) or 4, 8, 16: one value buffer */
  int32_t device;
  int64_t staging_bytes;      /* HBM budget for admitted requests' device buffers */
  float max_load;             /* grow before live/capacity would pass this (0.7) */
  int32_t max_batch_requests; /* requests per batch, 1..256 */
  int32_t zero_copy;          /* 0: keys and values are copied into pinned staging at submit (the
                                 caller may reuse its arrays at once).
                                 1: no staging.  The kernels read each request's keys and values from
                                 the caller's host arrays and write buf_indices / masks into the
                                 caller's arrays in place (devices with pageable memory access only,
                                 see ash_get_device_info); all four arrays must stay valid and
                                 unmodified from submit until wait returns.  Requests then take no
                                 device staging and are admitted at once.  Lowest latency below
                                 saturation.
                                 2: as 0, except that keys and values in page-locked (pinned) host
                                 memory are uploaded by DMA straight from the caller's arrays, with
                                 no CPU copy; those arrays must stay valid and unmodified until wait
                                 returns.  Other requests behave as in mode 0. */
} ash_server_config;
typedef struct ash_server_stats {
  int64_t submitted;
  int64_t completed;
  int64_t batches;
  int64_t batched_requests;
  int64_t rehashes;
  int64_t host_syncs;     /* growth checks of tenant maps that had to synchronise a stream */
  int64_t pinned_spills;  /* host staging blocks pinned during serving (the arena was full) */
} ash_server_stats;
void ash_server_default_config(ash_server_config* out);
ash_status ash_server_create(const ash_server_config* cfg_host, ash_server** out_host);
ash_status ash_server_destroy(ash_server* server);
ash_status ash_server_submit(ash_server* server, int32_t tenant, int32_t op, const int32_t* keys_host,
                             const void* values_host, int64_t n, int32_t* buf_indices_host, uint8_t* masks_host,
                             uint64_t* request_id_host);
ash_status ash_server_wait(ash_server* server, uint64_t request_id, int64_t timeout_ms, double* latency_ms_host);
ash_status ash_server_stats_get(ash_server* server, ash_server_stats* out_host);
ash_status ash_server_map(ash_server* server, int32_t tenant, ash_map** out_host);
ash_status ash_server_stream(ash_server* server, ash_stream* out_host);

/* Serving replay (measurement support, not part of the map): a request trace
 * replayed from native threads, so that the measured latencies are the
 * server's and not a scripting-language client's.  Request r is op[r] on
 * tenant[r] over the n[r] key rows starting at row[r] of keys_host
 * ([rows, key_dim] int32, host memory; pinned arrays let zero_copy mode 2
 * upload them by DMA) and, for inserts, the same rows of values_host
 * ([rows] value rows).  arrival_s[r] is its arrival time in seconds after
 * the start (non-decreasing).  ash_server_replay lays out every request's
 * outputs in one page-locked host arena before the replay starts (kept for
 * later replays until the process exits); one replay runs at a time.
 *   ash_server_replay: `threads` submitter threads submit request r (r mod
 *     threads) at its arrival time, one tenant's requests in trace order
 *     (a request waits for the submit of its tenant's previous one); as
 *     many waiter threads wait for them.
 *   ash_replay_sequential: the same trace as plain calls in arrival order on
 *     maps[tenant] (one value buffer at most, shared layout): upload, the
 *     operation, download, synchronise; the next request starts after.
 * latency_ms_host[r]: from arrival to outputs in the caller's arrays (-1 for
 * a request that failed).  *span_s_host: start to the last completion.
 * Both return after every request finished; errors: ASH_ERR_INVALID for a
 * bad trace (checked before anything runs), else the first failed call. */
typedef struct ash_replay_trace {
  int64_t n_requests;
  const double* arrival_s;
  const int32_t* tenant;
  const int32_t* op;          /* ash_op */
  const int64_t* n;
  const int64_t* row;
  int64_t rows;               /* rows of keys_host (and values_host) */
  const int32_t* keys_host;
  const void* values_host;
} ash_replay_trace;
ash_status ash_server_replay(ash_server* server, const ash_replay_trace* trace, int32_t threads,
                             double* latency_ms_host, double* span_s_host);
ash_status ash_replay_sequential(ash_map* const* maps, int32_t n_maps, const ash_replay_trace* trace,
                                 double* latency_ms_host, double* span_s_host);

/* Voxel quantisation (Sec. 6.1 listing; Eq. (10) with s*l as the cell edge):
 * keys[j] = floor(points[j] / cell) per coordinate, computed in float32 with
 * IEEE division and rounding toward minus infinity, for n_coords floats.
 * Quotients outside the int32 range saturate.  cell must be finite and > 0. */
ash_status ash_quantize(const float* points, int64_t n_coords, float cell, int32_t* keys,
                        ash_stream stream);

/* Random-sector read probe (measurement only, not part of the map): n_reads
 * reads of sector_bytes (32 or 64) at pseudo-random sector-aligned offsets of
 * buf (buf_bytes, multiple of 64, 64-byte aligned), XOR-folded into
 * sink[0..sink_len).  Each thread of a grid of 8 blocks of 256 threads per SM
 * keeps loads_per_thread (4, 8 or 16) independent reads in flight.  Run over
 * a buffer of a kernel's random-access footprint, it sets the random-access
 * roofline that kernel is compared with. */
ash_status ash_probe_random_read(const void* buf, int64_t buf_bytes, int64_t n_reads,
                                 int sector_bytes, int loads_per_thread, uint32_t seed, uint32_t* sink,
                                 int64_t sink_len, ash_stream stream);

/* Kernel tracing (measurement support, not part of the map).  The library
 * counts every kernel it launches; with tracing on it also records a CUDA
 * event pair around each launch on the launching stream.
 *   ash_trace_kernel_kinds / ash_trace_kernel_name: the kernel kinds.
 *   ash_trace_enable(1/0): start / stop recording events.
 *   ash_trace_collect: waits for the recorded events and adds their elapsed
 *     times to per-kind totals (synchronises on those events).
 *   ash_trace_read: total milliseconds and timed launches of one kind.
 *   ash_trace_reset: zeroes the totals.
 *   ash_kernel_launch_count: kernels launched by this library since load. */
int ash_trace_kernel_kinds(void);
const char* ash_trace_kernel_name(int kind);
ash_status ash_trace_enable(int on);
ash_status ash_trace_collect(void);
ash_status ash_trace_read(int kind, double* total_ms_host, int64_t* launches_host);
ash_status ash_trace_reset(void);
uint64_t ash_kernel_launch_count(void);

/* Random-atomic probe (measurement only, not part of the map): n_ops 64-bit
 * CAS operations on buf (buf_bytes, a multiple of 32, 32-byte aligned, read
 * as 32-byte buckets whose slots must start all ones).  mode 0: a CAS on a
 * random slot; mode 1: a relaxed 32-byte bucket load followed by a CAS on
 * the bucket's first all-ones slot (the dependent chain of an insert claim).
 * Sets the atomic roofline the claim kernel is compared with. */
ash_status ash_probe_random_atomic(void* buf, int64_t buf_bytes, int64_t n_ops, int mode, uint32_t seed,
                                   uint32_t* sink, int64_t sink_len, ash_stream stream);

/* ---------------------------------------------------------------------------
 * Geometry consumers of the map (Sec. 6.2): the voxel-block pipeline of a
 * volumetric reconstruction.  Cameras: intrinsics_host = {fx, fy, cx, cy};
 * extrinsic_host = the world-to-camera pose [R | t], row-major 3x4 float32
 * (the inverse of the frame pose T^j of Eq. (7)); both are host arrays read
 * during the call.  Depth images are float32 [height, width] in device
 * memory, in metres along the optical axis; a pixel has a measurement when
 * 0 < D <= depth_max.  Every discrete decision (a block key, a pixel, a skip,
 * a voxel, a zero crossing) is taken in float32 with explicitly rounded
 * operations in the order given below, so any IEEE float32 implementation of
 * the same steps reproduces it bit for bit.
 * ------------------------------------------------------------------------- */

/* Block keys of a depth frame (Sec. 6.2 unprojection, then Eq. (11)): pixel
 * (px, py) with depth D gives the camera point
 * x_c = [((px - cx) / fx) * D, ((py - cy) / fy) * D, D], the world point
 * x_w = R^T x_c + c with c = -R^T t (each R^T row summed left to right), and
 * the key floor(x_w / block_edge) per coordinate.  keys ([width * height, 3],
 * device) receives the keys of the pixels with a measurement, in pixel order
 * (row-major).  Their number goes to count_dev (a device int64, no host
 * synchronisation) and/or count_host (synchronises the stream); at least one
 * is required.  World coordinates must stay within |x_w / block_edge| < 2^31. */
ash_status ash_depth_to_block_keys(const float* depth, int32_t width, int32_t height, const float* intrinsics_host,
                                   const float* extrinsic_host, float block_edge, float depth_max, int32_t* keys,
                                   int64_t* count_dev, int64_t* count_host, ash_stream stream);

/* Double hash map block allocation (Sec. 6.2, the double-hash-map listing):
 *   1. activate keys ([n, key_dim]) in `local`;
 *   2. the keys whose activation succeeded (their first occurrences, in input
 *      order) go to unique_keys [u, key_dim] with their local indices
 *      local_indices [u];
 *   3. activate them in `global`, then find them there: global_indices [u];
 *   4. the local map's value buffer (one int32 element per entry) gets
 *      local_v[local_indices[r]] = global_indices[r].
 * The outputs need room for n rows; *n_unique_host = u.  Both maps grow by the
 * usual rule.  Synchronises the stream once (to learn u before the global
 * map's growth check).  The maps must be distinct, on one device, with the
 * same key_dim; `local` must have exactly one value buffer of one int32. */
ash_status ash_double_map_activate(ash_map* local, ash_map* global, const int32_t* keys, int64_t n,
                                   int32_t* unique_keys, int32_t* local_indices, int32_t* global_indices,
                                   int64_t* n_unique_host, ash_stream stream);

/* TSDF integration of one depth frame (Sec. 6.2, Eq. (7)-(9)) into the voxel
 * blocks at block_indices [n_blocks] (buffer indices of `blocks`, key_dim 3).
 * Value buffers tsdf_buffer (signed distance d) and weight_buffer (weight w)
 * are float32 rows of l^3 voxels, l = 8 or 16, voxel (vx, vy, vz) at slot
 * (vz * l + vy) * l + vx.  For voxel g = K * l + v (K the block's key), the
 * lattice point x = g * voxel_size goes to the camera, x_c = R x + t (rows
 * ((r0 x + r1 y) + r2 z) + t); the voxel is left alone when z_c <= 0, when its
 * pixel u = floor(fx * (x_c / z_c) + cx + 1/2), v = floor(fy * (y_c / z_c) +
 * cy + 1/2) is outside the image, when D(u, v) has no measurement, or when
 * d^j = D(u, v) - z_c < -trunc.  Otherwise, with Psi = min(d^j, trunc) and
 * w^j = 1: d := (w * d + Psi) / (w + 1), w := w + 1 (Eq. (9)).  Indices outside
 * [0, capacity) are skipped.  Block indices must be distinct within a call. */
ash_status ash_tsdf_integrate(ash_map* blocks, int tsdf_buffer, int weight_buffer, const int32_t* block_indices,
                              int64_t n_blocks, const float* depth, int32_t width, int32_t height,
                              const float* intrinsics_host, const float* extrinsic_host, float voxel_size,
                              float trunc, float depth_max, ash_stream stream);

/* Ray casting (Sec. 6.2) into depth_out (float32 [height, width], device).
 * The ray of pixel (px, py) leaves the camera centre c = -R^T t along
 * dir = R^T [(px - cx) / fx, (py - cy) / fy, 1], so its parameter is the depth
 * along the optical axis.  Sample i (0 <= i < n_steps) sits at
 * t_i = depth_min + i * step, p = c + t_i * dir, and reads the nearest lattice
 * point g = floor(p / voxel_size + 1/2) (IEEE float32 division): block K = floor(g / l), voxel
 * v = g - K * l.  It is valid when K is in the map and w > 0.  The first pair
 * of consecutive valid samples with d_{i-1} > 0 >= d_i gives the depth
 * t_{i-1} + step * d_{i-1} / (d_{i-1} - d_i); pixels without one get 0.
 * local_index_map (optional): look blocks up in this map instead (key_dim 3,
 * one int32 value per entry holding the block's index in `blocks`, same
 * bucket size), as with the double hash map's local map; blocks it lacks
 * read as empty.  n_steps <= 2^24.  When depth_min > 0 the call first lists
 * the lookup map's live blocks and projects them into per-tile depth ranges
 * (the min-max estimate of Sec. 6.2), conservatively, so that rays skip
 * only samples that no block can hold: the output is the same.  The maps are
 * not modified (the listing uses their internal scratch). */
ash_status ash_tsdf_raycast(ash_map* blocks, int tsdf_buffer, int weight_buffer, ash_map* local_index_map,
                            const float* intrinsics_host, const float* extrinsic_host, int32_t width, int32_t height,
                            float voxel_size, float depth_min, float step, int64_t n_steps, float* depth_out,
                            ash_stream stream);

/* Device facts the library and its callers use: SM count, L2 bytes, and
 * whether kernels may read and write ordinary (pageable) host memory
 * directly (cudaDevAttrPageableMemoryAccess; on coherent CPU-GPU systems the
 * key and output arrays of the map calls may then be host pointers). */
typedef struct ash_device_info {
  int32_t sm_count;
  int64_t l2_bytes;
  int32_t pageable_memory_access;
  int32_t pageable_uses_host_page_tables;
} ash_device_info;
ash_status ash_get_device_info(int device, ash_device_info* out_host);

/* Message for the last error on the calling thread ("" if none). */
const char* ash_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ASH_H_ */
