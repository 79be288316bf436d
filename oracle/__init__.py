"""CPU oracle for the ASH hot path (test infrastructure).

A plain sequential hash map written from the paper (arXiv 2110.00511): the
index-first SoA map of Sec. 4.2, the index heap of Sec. 4.3, lazy insertion of
Sec. 4.3.1, activate of Sec. 5.1, erase, rehash of Sec. 4.5 and the voxel
quantisation of Sec. 6.1.  It also covers the geometry consumers of
Sec. 6.2: the double hash map block allocation, TSDF integration (Eq. (7)-(9))
and ray casting.  The arithmetic lives in ash_oracle.cpp; this module only
marshals numpy arrays.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  It shares no code with the CUDA path and never
imports it.
"""
import ctypes
import numpy as np

from . import build as _build

_libs = {}

_i64 = ctypes.c_int64
_ptr = ctypes.c_void_p


def _lib(mutant: int = 0):
    if mutant not in _libs:
        path = _build.build(mutant)
        lib = ctypes.CDLL(path)
        lib.om_create.restype = _ptr
        lib.om_create.argtypes = [ctypes.c_int, _i64, ctypes.c_int, ctypes.POINTER(_i64), ctypes.c_int]
        lib.om_destroy.argtypes = [_ptr]
        lib.om_insert.restype = _i64
        lib.om_insert.argtypes = [_ptr, _ptr, _i64, ctypes.POINTER(_ptr), _ptr, _ptr]
        lib.om_activate.restype = _i64
        lib.om_activate.argtypes = [_ptr, _ptr, _i64, _ptr, _ptr]
        lib.om_find.restype = _i64
        lib.om_find.argtypes = [_ptr, _ptr, _i64, _ptr, _ptr]
        lib.om_erase.restype = _i64
        lib.om_erase.argtypes = [_ptr, _ptr, _i64, _ptr]
        for name in ("om_size", "om_capacity", "om_heap_top"):
            getattr(lib, name).restype = _i64
            getattr(lib, name).argtypes = [_ptr]
        lib.om_active_indices.restype = _i64
        lib.om_active_indices.argtypes = [_ptr, _ptr]
        lib.om_rehash.restype = ctypes.c_int
        lib.om_rehash.argtypes = [_ptr, _i64]
        lib.om_clear.argtypes = [_ptr]
        lib.om_copy_keys.argtypes = [_ptr, _ptr]
        lib.om_copy_values.argtypes = [_ptr, ctypes.c_int, _ptr]
        lib.om_copy_heap.argtypes = [_ptr, _ptr]
        lib.om_quantize.argtypes = [_ptr, _i64, ctypes.c_float, _ptr]
        lib.om_depth_to_block_keys.restype = _i64
        lib.om_depth_to_block_keys.argtypes = [_ptr, ctypes.c_int, ctypes.c_int, _ptr, _ptr, ctypes.c_float,
                                               ctypes.c_float, _ptr]
        lib.om_double_map_activate.restype = _i64
        lib.om_double_map_activate.argtypes = [_ptr, _ptr, _ptr, _i64, _ptr, _ptr, _ptr]
        _f = ctypes.c_float
        lib.om_tsdf_integrate.argtypes = [_ptr, _ptr, _i64, ctypes.c_int, _ptr, ctypes.c_int, ctypes.c_int, _ptr, _ptr,
                                          _f, _f, _f]
        lib.om_tsdf_raycast.argtypes = [_ptr, ctypes.c_int, ctypes.c_int, _ptr, _ptr, ctypes.c_int, _f, _f, _f, _i64,
                                        _ptr, _i64, _ptr]
        _libs[mutant] = lib
    return _libs[mutant]


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleMap:
    """Sequential reference map.  Keys are int32 [N, key_dim]; value buffer j
    holds rows of `value_row_bytes[j]` bytes, passed as numpy arrays whose
    rows are that many bytes."""

    def __init__(self, key_dim, capacity, value_row_bytes=(), auto_grow=True, mutant=0):
        self._lib = _lib(mutant)
        self.key_dim = int(key_dim)
        self.row_bytes = [int(b) for b in value_row_bytes]
        rb = (_i64 * max(1, len(self.row_bytes)))(*self.row_bytes)
        self._h = self._lib.om_create(self.key_dim, int(capacity), len(self.row_bytes), rb, int(bool(auto_grow)))
        if not self._h:
            raise ValueError("oracle: invalid map arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.om_destroy(h)
            self._h = None

    def _keys(self, keys):
        k = _c(keys, np.int32).reshape(-1, self.key_dim)
        return k, k.shape[0]

    def insert(self, keys, values):
        k, n = self._keys(keys)
        vals = [_c(v, None) for v in values]
        for v, rb in zip(vals, self.row_bytes):
            if v.nbytes != n * rb:
                raise ValueError("oracle: value array size does not match rows")
        arr = (_ptr * max(1, len(vals)))(*[v.ctypes.data for v in vals])
        idx = np.empty(n, np.int32)
        mask = np.empty(n, np.uint8)
        r = self._lib.om_insert(self._h, k.ctypes.data, n, arr, idx.ctypes.data, mask.ctypes.data)
        if r < 0:
            raise RuntimeError("oracle: growth failed")
        return idx, mask.astype(bool)

    def activate(self, keys):
        k, n = self._keys(keys)
        idx = np.empty(n, np.int32)
        mask = np.empty(n, np.uint8)
        r = self._lib.om_activate(self._h, k.ctypes.data, n, idx.ctypes.data, mask.ctypes.data)
        if r < 0:
            raise RuntimeError("oracle: growth failed")
        return idx, mask.astype(bool)

    def find(self, keys):
        k, n = self._keys(keys)
        idx = np.empty(n, np.int32)
        mask = np.empty(n, np.uint8)
        self._lib.om_find(self._h, k.ctypes.data, n, idx.ctypes.data, mask.ctypes.data)
        return idx, mask.astype(bool)

    def erase(self, keys):
        k, n = self._keys(keys)
        mask = np.empty(n, np.uint8)
        self._lib.om_erase(self._h, k.ctypes.data, n, mask.ctypes.data)
        return mask.astype(bool)

    def size(self):
        return int(self._lib.om_size(self._h))

    def capacity(self):
        return int(self._lib.om_capacity(self._h))

    def heap_top(self):
        return int(self._lib.om_heap_top(self._h))

    def active_indices(self):
        out = np.empty(self.size(), np.int32)
        n = self._lib.om_active_indices(self._h, out.ctypes.data)
        return out[:n]

    def rehash(self, new_capacity=0):
        if self._lib.om_rehash(self._h, int(new_capacity)) != 0:
            raise ValueError("oracle: rehash below the current size")

    def clear(self):
        self._lib.om_clear(self._h)

    def key_buffer(self):
        out = np.empty((self.capacity(), self.key_dim), np.int32)
        self._lib.om_copy_keys(self._h, out.ctypes.data)
        return out

    def value_buffer(self, j):
        out = np.empty((self.capacity(), self.row_bytes[j]), np.uint8)
        self._lib.om_copy_values(self._h, j, out.ctypes.data)
        return out

    def heap(self):
        out = np.empty(self.capacity(), np.int32)
        self._lib.om_copy_heap(self._h, out.ctypes.data)
        return out

    def as_dict(self):
        """{key tuple: tuple(value row bytes per buffer)} over the active set."""
        kb = self.key_buffer()
        vb = [self.value_buffer(j) for j in range(len(self.row_bytes))]
        out = {}
        for i in self.active_indices():
            out[tuple(int(x) for x in kb[i])] = tuple(v[i].tobytes() for v in vb)
        return out


def quantize(points, voxel, mutant=0):
    """floor(p / s) per coordinate in float32 (Sec. 6.1, Eq. (11))."""
    p = _c(points, np.float32)
    out = np.empty(p.shape, np.int32)
    _lib(mutant).om_quantize(p.ctypes.data, p.size, ctypes.c_float(voxel), out.ctypes.data)
    return out


def double_map_activate(local, glob, keys):
    """Double hash map block allocation (Sec. 6.2): local activate, the
    distinct new keys in input order, global activate + find, and the local
    map's int32 value rows := global indices.  Returns (unique_keys [u, d],
    local_indices [u], global_indices [u])."""
    k, n = local._keys(keys)
    uk = np.empty((n, local.key_dim), np.int32)
    li = np.empty(n, np.int32)
    gi = np.empty(n, np.int32)
    u = local._lib.om_double_map_activate(local._h, glob._h, k.ctypes.data, n, uk.ctypes.data, li.ctypes.data,
                                          gi.ctypes.data)
    if u < 0:
        raise RuntimeError("oracle activation failed")
    return uk[:u].copy(), li[:u].copy(), gi[:u].copy()


def _cam(intrinsics, extrinsic):
    intr = _c(np.asarray(intrinsics, np.float32).reshape(4), np.float32)
    extr = _c(np.asarray(extrinsic, np.float32).reshape(3, 4), np.float32)
    return intr, extr


def depth_to_block_keys(depth, intrinsics, extrinsic, block_edge, depth_max, mutant=0):
    """int32 [n, 3] block keys of the pixels with depth in (0, depth_max], in
    pixel order (Sec. 6.2 unprojection, Eq. (11))."""
    dep = _c(depth, np.float32)
    intr, extr = _cam(intrinsics, extrinsic)
    out = np.empty((dep.size, 3), np.int32)
    n = _lib(mutant).om_depth_to_block_keys(dep.ctypes.data, dep.shape[1], dep.shape[0], intr.ctypes.data,
                                            extr.ctypes.data, ctypes.c_float(block_edge), ctypes.c_float(depth_max),
                                            out.ctypes.data)
    return out[:n].copy()


def tsdf_integrate(om, block_indices, depth, intrinsics, extrinsic, voxel, trunc, depth_max, ell=8):
    """TSDF integration of one frame (Sec. 6.2, Eq. (7)-(9)) into the blocks at
    block_indices.  om holds float64 value buffers: 0 = d, 1 = w (ell^3 each).
    intrinsics = (fx, fy, cx, cy); extrinsic = world-to-camera [R | t] (3x4)."""
    bi = _c(block_indices, np.int32).reshape(-1)
    dep = _c(depth, np.float32)
    intr, extr = _cam(intrinsics, extrinsic)
    om._lib.om_tsdf_integrate(om._h, bi.ctypes.data, bi.size, int(ell), dep.ctypes.data, dep.shape[1], dep.shape[0],
                              intr.ctypes.data, extr.ctypes.data, ctypes.c_float(voxel), ctypes.c_float(trunc),
                              ctypes.c_float(depth_max))


def tsdf_raycast(om, intrinsics, extrinsic, width, height, voxel, depth_min, step, n_steps, pixels=None, ell=8,
                 value_bytes=8):
    """Ray casting (Sec. 6.2): depth of the first positive-to-negative zero
    crossing per pixel (0 if none), for the listed pixel ids (py * width + px;
    all pixels if None).  Returns float64 depths."""
    if pixels is None:
        pixels = np.arange(width * height, dtype=np.int64)
    px = _c(pixels, np.int64).reshape(-1)
    out = np.empty(px.size, np.float64)
    intr, extr = _cam(intrinsics, extrinsic)
    om._lib.om_tsdf_raycast(om._h, int(ell), int(value_bytes), intr.ctypes.data, extr.ctypes.data, int(width),
                            ctypes.c_float(voxel), ctypes.c_float(depth_min), ctypes.c_float(step), int(n_steps),
                            px.ctypes.data, px.size, out.ctypes.data)
    return out
