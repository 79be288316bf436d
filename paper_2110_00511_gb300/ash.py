"""Thin ctypes binding of libash.so (include/ash.h).

Functions named ash_* mirror the C ABI one to one and only marshal torch
tensors (device pointers, sizes, the current CUDA stream).  Every step of the
hash map runs in the library's CUDA kernels; there is no CPU fallback: if
libash.so is missing or no GPU is present, calls raise.

`HashMap` wraps one map with the interface of the paper's HashMap (Sec. 4.2,
listings of Sec. 6): insert / activate / find return (buf_indices, masks);
value and key buffers are exposed as zero-copy tensors.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libash.so")

ASH_OK, ASH_ERR_INVALID, ASH_ERR_OOM, ASH_ERR_CAPACITY, ASH_ERR_TABLE_FULL, ASH_ERR_TIMEOUT, ASH_ERR_CUDA = range(7)
_STATUS_NAMES = ["ASH_OK", "ASH_ERR_INVALID", "ASH_ERR_OOM", "ASH_ERR_CAPACITY", "ASH_ERR_TABLE_FULL",
                 "ASH_ERR_TIMEOUT", "ASH_ERR_CUDA"]

DTYPES = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2, torch.int32: 3, torch.int64: 4,
          torch.uint8: 5, torch.float64: 6}


class AshError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("slots_per_bucket", ctypes.c_int32), ("slots_per_capacity", ctypes.c_float),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("max_probes", ctypes.c_int32), ("auto_grow", ctypes.c_int32),
                ("max_used_fraction", ctypes.c_float), ("inline_value_bytes", ctypes.c_int32),
                ("keys_per_thread", ctypes.c_int32), ("warp_probe", ctypes.c_int32),
                ("find_keys_per_thread", ctypes.c_int32), ("claim_mode", ctypes.c_int32),
                ("commit_keys_per_thread", ctypes.c_int32), ("partition_keys", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_lib = None

ASH_OP_INSERT, ASH_OP_ACTIVATE, ASH_OP_FIND, ASH_OP_ERASE = range(4)


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_tenants", ctypes.c_int32), ("key_dim", ctypes.c_int32), ("initial_capacity", ctypes.c_int64),
                ("value_row_bytes", ctypes.c_int32), ("device", ctypes.c_int32), ("staging_bytes", ctypes.c_int64),
                ("max_load", ctypes.c_float), ("max_batch_requests", ctypes.c_int32), ("zero_copy", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64), ("rehashes", ctypes.c_int64), ("host_syncs", ctypes.c_int64),
                ("pinned_spills", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class DeviceInfo(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("l2_bytes", ctypes.c_int64), ("pageable_memory_access", ctypes.c_int32),
                ("pageable_uses_host_page_tables", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MapStats(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("table_slots", ctypes.c_int64), ("live", ctypes.c_int64),
                ("used_slots", ctypes.c_int64), ("host_syncs", ctypes.c_int64), ("rebuilds", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ReplayTrace(ctypes.Structure):
    _fields_ = [("n_requests", ctypes.c_int64), ("arrival_s", ctypes.c_void_p), ("tenant", ctypes.c_void_p),
                ("op", ctypes.c_void_p), ("n", ctypes.c_void_p), ("row", ctypes.c_void_p), ("rows", ctypes.c_int64),
                ("keys_host", ctypes.c_void_p), ("values_host", ctypes.c_void_p)]


class BatchOp(ctypes.Structure):
    _fields_ = [("map", ctypes.c_void_p), ("op", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("keys", ctypes.c_void_p), ("values", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("buf_indices", ctypes.c_void_p), ("masks", ctypes.c_void_p)]

# C signatures: name -> (restype, argtypes)
_SIGS = {
    "ash_default_tuning": (None, [ctypes.POINTER(Tuning)]),
    "ash_set_allocator": (_I32, [_P, _P, _P]),
    "ash_create": (_I32, [ctypes.c_int, _I64, ctypes.c_int, ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.c_int,
                          ctypes.POINTER(Tuning), _P, ctypes.POINTER(_P)]),
    "ash_destroy": (_I32, [_P]),
    "ash_insert": (_I32, [_P, _P, ctypes.POINTER(_P), _I64, _P, _P, _P]),
    "ash_activate": (_I32, [_P, _P, _I64, _P, _P, _P]),
    "ash_find": (_I32, [_P, _P, _I64, _P, _P, _P]),
    "ash_erase": (_I32, [_P, _P, _I64, _P, _P]),
    "ash_erase_noalloc": (_I32, [_P, _P, _I64, _P, _P]),
    "ash_get_active_indices": (_I32, [_P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "ash_size": (_I32, [_P, ctypes.POINTER(_I64), _P]),
    "ash_get_active_indices_async": (_I32, [_P, _P, _I64, _P, _P]),
    "ash_gather_keys_count": (_I32, [_P, _P, _I64, _P, _P, _P]),
    "ash_gather_values_count": (_I32, [_P, ctypes.c_int, _P, _I64, _P, _P, _P]),
    "ash_capacity": (_I64, [_P]),
    "ash_get_map_stats": (_I32, [_P, ctypes.POINTER(MapStats), _P]),
    "ash_key_dim": (ctypes.c_int, [_P]),
    "ash_n_values": (ctypes.c_int, [_P]),
    "ash_rehash": (_I32, [_P, _I64, _P]),
    "ash_reserve": (_I32, [_P, _I64, _P]),
    "ash_reserve_async": (_I32, [_P, _I64, _P]),
    "ash_clear": (_I32, [_P, _P]),
    "ash_key_buffer": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "ash_value_buffer": (_I32, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "ash_heap_buffer": (_I32, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "ash_gather_keys": (_I32, [_P, _P, _I64, _P, _P]),
    "ash_gather_values": (_I32, [_P, ctypes.c_int, _P, _I64, _P, _P]),
    "ash_find_neighbors": (_I32, [_P, _P, _I64, _I32, _P, _P, _P]),
    "ash_insert_points": (_I32, [_P, _P, ctypes.c_float, ctypes.POINTER(_P), _I64, _P, _P, _P]),
    "ash_activate_points": (_I32, [_P, _P, ctypes.c_float, _I64, _P, _P, _P]),
    "ash_find_points": (_I32, [_P, _P, ctypes.c_float, _I64, _P, _P, _P]),
    "ash_find_offsets": (_I32, [_P, _P, _I64, _P, _I64, _P, _P, _P]),
    "ash_get_tuning": (_I32, [_P, ctypes.POINTER(Tuning)]),
    "ash_set_tuning": (_I32, [_P, ctypes.POINTER(Tuning)]),
    "ash_sync_status": (_I32, [_P, _P]),
    "ash_quantize": (_I32, [_P, _I64, ctypes.c_float, _P, _P]),
    "ash_probe_random_read": (_I32, [_P, _I64, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, _P, _I64, _P]),
    "ash_probe_random_atomic": (_I32, [_P, _I64, _I64, ctypes.c_int, ctypes.c_uint32, _P, _I64, _P]),
    "ash_trace_kernel_kinds": (ctypes.c_int, []),
    "ash_trace_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "ash_trace_enable": (_I32, [ctypes.c_int]),
    "ash_trace_collect": (_I32, []),
    "ash_trace_read": (_I32, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "ash_trace_reset": (_I32, []),
    "ash_kernel_launch_count": (ctypes.c_uint64, []),
    "ash_batch_create": (_I32, [ctypes.c_int, ctypes.POINTER(_P)]),
    "ash_batch_destroy": (_I32, [_P]),
    "ash_batch_run": (_I32, [_P, ctypes.POINTER(BatchOp), ctypes.c_int, _P]),
    "ash_autotune": (_I32, [ctypes.c_int, _I64, ctypes.c_float, ctypes.c_int, _P, ctypes.POINTER(Tuning)]),
    "ash_server_default_config": (None, [ctypes.POINTER(ServerConfig)]),
    "ash_server_create": (_I32, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    "ash_server_destroy": (_I32, [_P]),
    "ash_server_submit": (_I32, [_P, _I32, _I32, _P, _P, _I64, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "ash_server_wait": (_I32, [_P, ctypes.c_uint64, _I64, ctypes.POINTER(ctypes.c_double)]),
    "ash_server_stats_get": (_I32, [_P, ctypes.POINTER(ServerStats)]),
    "ash_server_map": (_I32, [_P, _I32, ctypes.POINTER(_P)]),
    "ash_server_stream": (_I32, [_P, ctypes.POINTER(_P)]),
    "ash_server_replay": (_I32, [_P, ctypes.POINTER(ReplayTrace), _I32, _P, ctypes.POINTER(ctypes.c_double)]),
    "ash_replay_sequential": (_I32, [_P, _I32, ctypes.POINTER(ReplayTrace), _P, ctypes.POINTER(ctypes.c_double)]),
    "ash_depth_to_block_keys": (_I32, [_P, _I32, _I32, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P,
                                       ctypes.POINTER(_I64), _P]),
    "ash_double_map_activate": (_I32, [_P, _P, _P, _I64, _P, _P, _P, ctypes.POINTER(_I64), _P]),
    "ash_tsdf_integrate": (_I32, [_P, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _I32, _I32, _P, _P, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, _P]),
    "ash_tsdf_raycast": (_I32, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _I32, _I32, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, _I64, _P, _P]),
    "ash_get_device_info": (_I32, [ctypes.c_int, ctypes.POINTER(DeviceInfo)]),
    "ash_last_error": (ctypes.c_char_p, []),
}


def exported_symbols():
    """Names the binding expects libash.so to export."""
    return list(_SIGS)


def lib():
    """Loads libash.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libash.so is not built ({LIB_PATH}); run paper_2110_00511_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != ASH_OK:
        raise AshError(status, lib().ash_last_error().decode())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_of(device_index):
    """The current CUDA stream of a device as an integer handle (the fast
    route of the map methods; same stream as _stream)."""
    if _raw_stream is not None:
        return _raw_stream(device_index)
    return torch.cuda.current_stream(device_index).cuda_stream


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _need_cuda(t, name, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class _DeviceArray:
    """__cuda_array_interface__ shim for zero-copy tensor views of library buffers."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}
        self._owner = owner


_TYPESTR = {torch.float32: "<f4", torch.float16: "<f2", torch.int32: "<i4", torch.int64: "<i8",
            torch.uint8: "|u1", torch.float64: "<f8"}


def _view(ptr, shape, dtype, device, owner):
    if dtype == torch.bfloat16:
        raw = torch.as_tensor(_DeviceArray(ptr, shape, "<i2", owner), device=device)
        return raw.view(torch.bfloat16)
    return torch.as_tensor(_DeviceArray(ptr, shape, _TYPESTR[dtype], owner), device=device)


def default_tuning() -> Tuning:
    t = Tuning()
    lib().ash_default_tuning(ctypes.byref(t))
    return t


# ------------------------------------------------------------ allocator hook
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_alloc_keepalive = []


def use_torch_allocator(enable: bool = True):
    """Routes the library's device allocations through PyTorch's caching
    allocator (maps created afterwards).  Off: cudaMallocAsync pool."""
    if not enable:
        _check(lib().ash_set_allocator(None, None, None))
        _alloc_keepalive.clear()
        return

    def _alloc(nbytes, device, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:
            return 0

    def _free(ptr, device, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _alloc_keepalive[:] = [a, f]
    _check(lib().ash_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))


# ---------------------------------------------------------------- functions
def ash_create(key_dim, capacity, value_numel=(), value_dtypes=(), device=0, tuning=None, stream=None):
    n_values = len(value_numel)
    numel = (_I64 * max(1, n_values))(*[int(x) for x in value_numel])
    dts = (_I32 * max(1, n_values))(*[DTYPES[d] if isinstance(d, torch.dtype) else int(d) for d in value_dtypes])
    out = ctypes.c_void_p()
    _check(lib().ash_create(int(key_dim), int(capacity), n_values, numel, dts, int(device),
                            ctypes.byref(tuning) if tuning is not None else None,
                            stream if stream is not None else _stream(device), ctypes.byref(out)))
    return out


def ash_destroy(handle):
    _check(lib().ash_destroy(handle))


def ash_insert(handle, keys, values, buf_indices, masks, stream=None):
    arr = (ctypes.c_void_p * max(1, len(values)))(*[v.data_ptr() for v in values])
    _check(lib().ash_insert(handle, _ptr(keys), arr, keys.shape[0], _ptr(buf_indices), _ptr(masks),
                            stream if stream is not None else _stream(keys.device)))


def ash_activate(handle, keys, buf_indices, masks, stream=None):
    _check(lib().ash_activate(handle, _ptr(keys), keys.shape[0], _ptr(buf_indices), _ptr(masks),
                              stream if stream is not None else _stream(keys.device)))


def ash_find(handle, keys, buf_indices, masks, stream=None):
    _check(lib().ash_find(handle, _ptr(keys), keys.shape[0], _ptr(buf_indices), _ptr(masks),
                          stream if stream is not None else _stream(keys.device)))


def ash_erase(handle, keys, masks, stream=None):
    _check(lib().ash_erase(handle, _ptr(keys), keys.shape[0], _ptr(masks),
                           stream if stream is not None else _stream(keys.device)))


# Largest n accepted by ash_erase_noalloc (ASH_ERASE_NOALLOC_MAX_KEYS in ash.h).
ASH_ERASE_NOALLOC_MAX_KEYS = 1 << 20


def ash_erase_noalloc(handle, keys, masks, stream=None):
    """Erase without any device allocation by the library: for callers that
    cannot let a library allocate (fully budgeted device memory, or loops
    where a first-time allocation may synchronise the device).  Uses a fixed
    4 MiB device array shared by all calls; n <= ASH_ERASE_NOALLOC_MAX_KEYS;
    calls that can overlap on the GPU must be ordered by the caller.

    keys: contiguous int32 CUDA tensor [n, key_dim]; masks: contiguous bool or
    uint8 CUDA tensor on the same device with at least n elements.  Anything
    else raises ValueError before the library is called, so the kernels never
    see a short or mistyped array."""
    if not isinstance(keys, torch.Tensor) or not isinstance(masks, torch.Tensor):
        raise ValueError("keys and masks must be torch tensors")
    _need_cuda(keys, "keys", torch.int32)
    if keys.dim() != 2:
        raise ValueError("keys must be int32 [n, key_dim]")
    if handle is not None and keys.shape[1] != lib().ash_key_dim(handle):
        raise ValueError("keys must have the map's key_dim columns")
    if masks.dtype not in (torch.bool, torch.uint8):
        raise ValueError("masks must be bool or uint8")
    _need_cuda(masks, "masks")
    if masks.device != keys.device:
        raise ValueError("keys and masks must be on the same device")
    if masks.numel() < keys.shape[0]:
        raise ValueError("masks must hold at least n elements")
    _check(lib().ash_erase_noalloc(handle, _ptr(keys), keys.shape[0], _ptr(masks),
                                   stream if stream is not None else _stream(keys.device)))


def ash_get_active_indices(handle, out, stream=None):
    count = _I64()
    _check(lib().ash_get_active_indices(handle, _ptr(out), out.numel(), ctypes.byref(count),
                                        stream if stream is not None else _stream(out.device)))
    return int(count.value)


def ash_size(handle, stream=None):
    v = _I64()
    _check(lib().ash_size(handle, ctypes.byref(v), stream if stream is not None else _stream()))
    return int(v.value)


def ash_rehash(handle, new_capacity=0, stream=None):
    _check(lib().ash_rehash(handle, int(new_capacity), stream if stream is not None else _stream()))


def ash_reserve(handle, new_capacity, stream=None):
    _check(lib().ash_reserve(handle, int(new_capacity), stream if stream is not None else _stream()))


def ash_reserve_async(handle, new_capacity, stream=None):
    _check(lib().ash_reserve_async(handle, int(new_capacity), stream if stream is not None else _stream()))


def ash_clear(handle, stream=None):
    _check(lib().ash_clear(handle, stream if stream is not None else _stream()))


def ash_gather_keys(handle, indices, out, stream=None):
    _check(lib().ash_gather_keys(handle, _ptr(indices), indices.numel(), _ptr(out),
                                 stream if stream is not None else _stream(indices.device)))


def ash_sync_status(handle, stream=None):
    _check(lib().ash_sync_status(handle, stream if stream is not None else _stream()))


def ash_quantize(points, cell, out=None, stream=None):
    """int32 keys floor(points / cell) (Sec. 6.1), same shape as points."""
    _need_cuda(points, "points", torch.float32)
    if out is None:
        out = torch.empty(points.shape, dtype=torch.int32, device=points.device)
    _check(lib().ash_quantize(_ptr(points), points.numel(), ctypes.c_float(cell), _ptr(out),
                              stream if stream is not None else _stream(points.device)))
    return out


def ash_probe_random_atomic(buf, n_ops, mode, sink, seed=0, stream=None):
    _check(lib().ash_probe_random_atomic(_ptr(buf), buf.numel() * buf.element_size(), int(n_ops), int(mode),
                                         ctypes.c_uint32(seed), _ptr(sink), sink.numel(),
                                         stream if stream is not None else _stream(buf.device)))


def ash_probe_random_read(buf, n_reads, sector_bytes, sink, seed=0, loads_per_thread=8, stream=None):
    _check(lib().ash_probe_random_read(_ptr(buf), buf.numel() * buf.element_size(), int(n_reads), int(sector_bytes),
                                       int(loads_per_thread), ctypes.c_uint32(seed), _ptr(sink), sink.numel(),
                                       stream if stream is not None else _stream(buf.device)))


def ash_trace_enable(on=True):
    _check(lib().ash_trace_enable(1 if on else 0))


def ash_trace_reset():
    _check(lib().ash_trace_reset())


def ash_trace_collect():
    """{kernel kind: (total ms, timed launches)} after waiting for the events."""
    L = lib()
    _check(L.ash_trace_collect())
    out = {}
    for k in range(L.ash_trace_kernel_kinds()):
        ms, n = ctypes.c_double(), _I64()
        _check(L.ash_trace_read(k, ctypes.byref(ms), ctypes.byref(n)))
        out[L.ash_trace_kernel_name(k).decode()] = (ms.value, int(n.value))
    return out


def ash_kernel_launch_count():
    return int(lib().ash_kernel_launch_count())


def ash_autotune(key_dim, capacity, rho=1.0, device=0, stream=None) -> Tuning:
    """Fastest tuning for maps of this shape (cached per shape class)."""
    t = Tuning()
    _check(lib().ash_autotune(int(key_dim), int(capacity), ctypes.c_float(rho), int(device),
                              stream if stream is not None else _stream(device), ctypes.byref(t)))
    return t


def ash_batch_create(device=0):
    h = ctypes.c_void_p()
    _check(lib().ash_batch_create(int(device), ctypes.byref(h)))
    return h


def ash_batch_destroy(handle):
    _check(lib().ash_batch_destroy(handle))


def ash_batch_run(handle, ops, stream=None):
    """ops: sequence of BatchOp."""
    arr = (BatchOp * max(1, len(ops)))(*ops)
    _check(lib().ash_batch_run(handle, arr, len(ops), stream if stream is not None else _stream()))


class Batch:
    """One batched-execution context (a ring of CUDA graphs).  `run` takes
    (HashMap, op, keys, values) tuples and returns [(buf_indices, masks)]."""

    def __init__(self, device=0):
        self.device = device
        self._h = ash_batch_create(device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().ash_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    def run(self, items, outputs=None):
        ops, outs = [], []
        for j, (hm, op, keys, values) in enumerate(items):
            n = keys.shape[0]
            if outputs is not None:
                idx, mask = outputs[j]
            else:
                idx = torch.empty(n, dtype=torch.int32, device=keys.device) if op != ASH_OP_ERASE else None
                mask = torch.empty(n, dtype=torch.bool, device=keys.device)
            ops.append(BatchOp(hm.handle.value, op, 0, keys.data_ptr(), values.data_ptr() if values is not None else None,
                               n, idx.data_ptr() if idx is not None else None, mask.data_ptr()))
            outs.append((idx, mask))
        ash_batch_run(self._h, ops)
        return outs


def ash_server_default_config() -> ServerConfig:
    c = ServerConfig()
    lib().ash_server_default_config(ctypes.byref(c))
    return c


class Server:
    """Multi-tenant continuous-batching server (native worker thread).

    submit() takes host numpy arrays and returns a request id; wait(id)
    returns (buf_indices, masks, latency_ms) as numpy arrays."""

    def __init__(self, config=None, **kw):
        cfg = config or ash_server_default_config()
        for k, v in kw.items():
            setattr(cfg, k, v)
        self.config = cfg
        self._h = ctypes.c_void_p()
        _check(lib().ash_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self._live = {}

    def close(self):
        if self._h is not None and self._h.value:
            _check(lib().ash_server_destroy(self._h))
        self._h = None
        self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, tenant, op, keys, values=None):
        import numpy as np
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        n = keys.shape[0]
        vals = None if values is None else np.ascontiguousarray(values)
        idx = np.empty(n, np.int32)
        mask = np.empty(n, np.uint8)
        rid = ctypes.c_uint64()
        _check(lib().ash_server_submit(self._h, int(tenant), int(op), keys.ctypes.data,
                                       vals.ctypes.data if vals is not None else None, n,
                                       idx.ctypes.data, mask.ctypes.data, ctypes.byref(rid)))
        self._live[rid.value] = (keys, vals, idx, mask)
        return rid.value

    def wait(self, rid, timeout_ms=-1):
        lat = ctypes.c_double()
        _check(lib().ash_server_wait(self._h, ctypes.c_uint64(rid), int(timeout_ms), ctypes.byref(lat)))
        keys, vals, idx, mask = self._live.pop(rid)
        return idx, mask.astype(bool), lat.value

    def stats(self):
        st = ServerStats()
        _check(lib().ash_server_stats_get(self._h, ctypes.byref(st)))
        return st.as_dict()

    def replay(self, trace, threads=8):
        """Replays a request trace (see make_trace) from native threads:
        (latency_ms per request, span seconds)."""
        import numpy as np
        tr, keep = trace.as_struct()
        lat = np.empty(trace.n_requests, np.float64)
        span = ctypes.c_double()
        _check(lib().ash_server_replay(self._h, ctypes.byref(tr), int(threads), lat.ctypes.data, ctypes.byref(span)))
        return lat, span.value

    def map_handle(self, tenant):
        h = ctypes.c_void_p()
        _check(lib().ash_server_map(self._h, int(tenant), ctypes.byref(h)))
        return h


class Trace:
    """A serving trace for the native replays: request r is op[r] on
    tenant[r] over rows row[r]:row[r]+n[r] of keys (int32 [rows, key_dim],
    host) and values (host, inserts), arriving arrival_s[r] seconds after
    the start."""

    def __init__(self, arrival_s, tenant, op, n, row, keys, values=None):
        import numpy as np
        self.arrival_s = np.ascontiguousarray(arrival_s, np.float64)
        self.tenant = np.ascontiguousarray(tenant, np.int32)
        self.op = np.ascontiguousarray(op, np.int32)
        self.n = np.ascontiguousarray(n, np.int64)
        self.row = np.ascontiguousarray(row, np.int64)
        if not (len(self.arrival_s) == len(self.tenant) == len(self.op) == len(self.n) == len(self.row)):
            raise ValueError("trace arrays differ in length")
        if keys.ndim != 2 or keys.dtype != np.int32 or not keys.flags.c_contiguous:
            raise ValueError("keys must be contiguous int32 [rows, key_dim]")
        if values is not None and (values.shape[0] != keys.shape[0] or not values.flags.c_contiguous):
            raise ValueError("values must be contiguous with one row per key row")
        self.keys, self.values = keys, values
        self.n_requests = len(self.arrival_s)

    def as_struct(self):
        t = ReplayTrace(self.n_requests, self.arrival_s.ctypes.data, self.tenant.ctypes.data, self.op.ctypes.data,
                        self.n.ctypes.data, self.row.ctypes.data, self.keys.shape[0], self.keys.ctypes.data,
                        self.values.ctypes.data if self.values is not None else None)
        return t, self


def replay_sequential(maps, trace):
    """The trace as plain calls in arrival order on maps[tenant] (upload, op,
    download, synchronise): (latency_ms per request, span seconds)."""
    import numpy as np
    arr = (ctypes.c_void_p * len(maps))(*[m.handle.value for m in maps])
    tr, keep = trace.as_struct()
    lat = np.empty(trace.n_requests, np.float64)
    span = ctypes.c_double()
    _check(lib().ash_replay_sequential(arr, len(maps), ctypes.byref(tr), lat.ctypes.data, ctypes.byref(span)))
    return lat, span.value


# -------------------------------------------------------------------- class
class HashMap:
    """A GPU hash map with int32 keys of dimension key_dim and SoA value
    buffers (Sec. 4.2, 4.7).  value_shapes=() makes a hash set."""

    def __init__(self, key_dim, capacity, value_shapes=(), value_dtypes=(), device=None, tuning=None):
        if len(value_shapes) != len(value_dtypes):
            raise ValueError("value_shapes and value_dtypes differ in length")
        if not torch.cuda.is_available():
            raise RuntimeError("HashMap needs a CUDA device (there is no CPU fallback)")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        self.key_dim = int(key_dim)
        self.value_shapes = [tuple(int(x) for x in (s if isinstance(s, (tuple, list)) else (s,))) for s in value_shapes]
        self.value_dtypes = list(value_dtypes)
        numel = [int(torch.Size(s).numel()) for s in self.value_shapes]
        self._h = ash_create(self.key_dim, capacity, numel, self.value_dtypes, self.device.index, tuning,
                             _stream(self.device))

    @classmethod
    def wrap(cls, handle, key_dim, value_shapes=(), value_dtypes=(), device=0):
        """A non-owning view of a map created elsewhere (e.g. a server tenant)."""
        self = cls.__new__(cls)
        self.device = torch.device("cuda", device)
        self.key_dim = int(key_dim)
        self.value_shapes = [tuple(s if isinstance(s, (tuple, list)) else (s,)) for s in value_shapes]
        self.value_dtypes = list(value_dtypes)
        self._h = handle
        self._owned = False
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and getattr(self, "_owned", True):
            try:
                lib().ash_destroy(h)
            except Exception:
                pass
            self._h = None

    def _keys(self, keys):
        # one combined test on the common path; the detailed checks name the problem
        if (keys.dtype is not torch.int32 or keys.dim() != 2 or keys.shape[1] != self.key_dim
                or keys.get_device() != self.device.index or not keys.is_contiguous()):
            _need_cuda(keys, "keys", torch.int32)
            if keys.dim() != 2 or keys.shape[1] != self.key_dim:
                raise ValueError(f"keys must be int32 [N, {self.key_dim}]")
            raise ValueError("keys must be on the map's device")
        return keys

    def _outputs(self, n):
        return (torch.empty(n, dtype=torch.int32, device=self.device),
                torch.empty(n, dtype=torch.bool, device=self.device))

    def insert(self, keys, values):
        keys = self._keys(keys)
        values = list(values) if isinstance(values, (list, tuple)) else [values]
        if len(values) != len(self.value_shapes):
            raise ValueError("one value tensor per value buffer is required")
        for v, shp, dt in zip(values, self.value_shapes, self.value_dtypes):
            _need_cuda(v, "values", dt)
            if v.numel() != keys.shape[0] * torch.Size(shp).numel():
                raise ValueError("value tensor does not match [N, *shape]")
            if v.get_device() != self.device.index:
                raise ValueError("values must be on the map's device")
        n = keys.shape[0]
        idx, mask = self._outputs(n)
        arr = (ctypes.c_void_p * max(1, len(values)))(*[v.data_ptr() for v in values])
        st = lib().ash_insert(self._h, keys.data_ptr(), arr, n, idx.data_ptr(), mask.data_ptr(),
                              _stream_of(self.device.index))
        if st:
            _check(st)
        return idx, mask

    def activate(self, keys):
        keys = self._keys(keys)
        n = keys.shape[0]
        idx, mask = self._outputs(n)
        st = lib().ash_activate(self._h, keys.data_ptr(), n, idx.data_ptr(), mask.data_ptr(),
                                _stream_of(self.device.index))
        if st:
            _check(st)
        return idx, mask

    def find(self, keys):
        keys = self._keys(keys)
        n = keys.shape[0]
        idx, mask = self._outputs(n)
        st = lib().ash_find(self._h, keys.data_ptr(), n, idx.data_ptr(), mask.data_ptr(),
                            _stream_of(self.device.index))
        if st:
            _check(st)
        return idx, mask

    def erase(self, keys):
        keys = self._keys(keys)
        n = keys.shape[0]
        mask = torch.empty(n, dtype=torch.bool, device=self.device)
        st = lib().ash_erase(self._h, keys.data_ptr(), n, mask.data_ptr(), _stream_of(self.device.index))
        if st:
            _check(st)
        return mask

    def erase_noalloc(self, keys, masks=None):
        """Erase through ash_erase_noalloc: the library allocates nothing (its
        per-key scratch is a fixed device array); n <= ASH_ERASE_NOALLOC_MAX_KEYS.
        `masks` (bool [n] on the map's device) may be given to avoid the output
        allocation too."""
        keys = self._keys(keys)
        if keys.device != self.device:
            raise ValueError("keys must be on the map's device")
        if masks is None:
            masks = torch.empty(keys.shape[0], dtype=torch.bool, device=self.device)
        ash_erase_noalloc(self._h, keys, masks)
        return masks

    def active_indices(self):
        out = torch.empty(max(1, self.capacity()), dtype=torch.int32, device=self.device)
        n = ash_get_active_indices(self._h, out)
        return out[:n]

    def active_indices_async(self):
        """(indices [capacity] int32, count [1] int64), both on the device, with
        no host synchronisation; indices[:count] are the live entries."""
        out = torch.empty(max(1, self.capacity()), dtype=torch.int32, device=self.device)
        count = torch.empty(1, dtype=torch.int64, device=self.device)
        _check(lib().ash_get_active_indices_async(self._h, _ptr(out), out.numel(), _ptr(count), _stream(self.device)))
        return out, count

    def gather_keys_count(self, indices, count):
        """[len(indices), key_dim] key rows; only the first *count (device) rows are written."""
        out = torch.empty((indices.numel(), self.key_dim), dtype=torch.int32, device=self.device)
        _check(lib().ash_gather_keys_count(self._h, _ptr(indices), indices.numel(), _ptr(count), _ptr(out),
                                           _stream(self.device)))
        return out

    def size(self):
        return ash_size(self._h, _stream(self.device))

    def capacity(self):
        return int(lib().ash_capacity(self._h))

    def stats(self):
        """Table health (synchronises): capacity, table_slots, live, used_slots
        (live + tombstones), host_syncs, rebuilds."""
        st = MapStats()
        _check(lib().ash_get_map_stats(self._h, ctypes.byref(st), _stream(self.device)))
        return st.as_dict()

    def rehash(self, new_capacity=0):
        ash_rehash(self._h, new_capacity, _stream(self.device))

    def reserve(self, new_capacity):
        ash_reserve(self._h, new_capacity, _stream(self.device))

    def reserve_async(self, new_capacity):
        ash_reserve_async(self._h, new_capacity, _stream(self.device))

    def clear(self):
        ash_clear(self._h, _stream(self.device))

    def sync_status(self):
        ash_sync_status(self._h, _stream(self.device))

    def gather_keys(self, indices):
        out = torch.empty((indices.numel(), self.key_dim), dtype=torch.int32, device=self.device)
        ash_gather_keys(self._h, indices.to(torch.int32).contiguous(), out)
        return out

    def gather_values(self, indices, j=0):
        """[n, *shape_j] rows of value buffer j at `indices` (zeros outside [0, c))."""
        idx = indices.to(torch.int32).contiguous()
        out = torch.empty((idx.numel(), *self.value_shapes[j]), dtype=self.value_dtypes[j], device=self.device)
        _check(lib().ash_gather_values(self._h, j, _ptr(idx), idx.numel(), _ptr(out), _stream(self.device)))
        return out

    def _points(self, points):
        _need_cuda(points, "points", torch.float32)
        if points.dim() != 2 or points.shape[1] != self.key_dim:
            raise ValueError(f"points must be float32 [N, {self.key_dim}]")
        return points

    def insert_points(self, points, cell, values):
        """insert() on the keys floor(points / cell), quantised in the kernels."""
        points = self._points(points)
        values = list(values) if isinstance(values, (list, tuple)) else [values]
        if len(values) != len(self.value_shapes):
            raise ValueError("one value tensor per value buffer is required")
        for v, dt in zip(values, self.value_dtypes):
            _need_cuda(v, "values", dt)
        idx, mask = self._outputs(points.shape[0])
        arr = (ctypes.c_void_p * max(1, len(values)))(*[v.data_ptr() for v in values])
        _check(lib().ash_insert_points(self._h, _ptr(points), ctypes.c_float(cell), arr, points.shape[0], _ptr(idx),
                                       _ptr(mask), _stream(self.device)))
        return idx, mask

    def activate_points(self, points, cell):
        points = self._points(points)
        idx, mask = self._outputs(points.shape[0])
        _check(lib().ash_activate_points(self._h, _ptr(points), ctypes.c_float(cell), points.shape[0], _ptr(idx),
                                         _ptr(mask), _stream(self.device)))
        return idx, mask

    def find_points(self, points, cell):
        points = self._points(points)
        idx, mask = self._outputs(points.shape[0])
        _check(lib().ash_find_points(self._h, _ptr(points), ctypes.c_float(cell), points.shape[0], _ptr(idx),
                                     _ptr(mask), _stream(self.device)))
        return idx, mask

    def find_neighbors(self, keys, radius=1):
        """Masked queries of keys[r] + every offset in [-radius, radius]^d:
        (buf_indices, masks), each [n, (2*radius+1)^d]."""
        keys = self._keys(keys)
        k = (2 * radius + 1) ** self.key_dim
        idx = torch.empty((keys.shape[0], k), dtype=torch.int32, device=self.device)
        mask = torch.empty((keys.shape[0], k), dtype=torch.bool, device=self.device)
        _check(lib().ash_find_neighbors(self._h, _ptr(keys), keys.shape[0], int(radius), _ptr(idx), _ptr(mask),
                                        _stream(self.device)))
        return idx, mask

    def find_offsets(self, keys, offsets):
        """Masked queries of keys[r] + offsets[m] for an explicit [n_off, d]
        offset table: (buf_indices, masks), each [n, n_off]."""
        keys = self._keys(keys)
        off = self._keys(offsets)
        idx = torch.empty((keys.shape[0], off.shape[0]), dtype=torch.int32, device=self.device)
        mask = torch.empty((keys.shape[0], off.shape[0]), dtype=torch.bool, device=self.device)
        _check(lib().ash_find_offsets(self._h, _ptr(keys), keys.shape[0], _ptr(off), off.shape[0], _ptr(idx),
                                      _ptr(mask), _stream(self.device)))
        return idx, mask

    def export(self):
        """Checkpoint of the live entries: {"keys": [n, d], "values": [..],
        "capacity": c} (device tensors; save with torch.save)."""
        act = self.active_indices()
        return {"keys": self.gather_keys(act), "values": [self.gather_values(act, j) for j in range(len(self.value_shapes))],
                "capacity": self.capacity(), "key_dim": self.key_dim,
                "value_shapes": self.value_shapes, "value_dtypes": [str(d) for d in self.value_dtypes]}

    @classmethod
    def from_export(cls, state, device=None, tuning=None):
        """Re-creates a map from export(): a bulk insert of the saved entries."""
        dts = [getattr(torch, d.replace("torch.", "")) for d in state["value_dtypes"]]
        hm = cls(state["key_dim"], state["capacity"], state["value_shapes"], dts, device=device, tuning=tuning)
        keys = state["keys"].to(hm.device).contiguous()
        if len(dts):
            hm.insert(keys, [v.to(hm.device).contiguous() for v in state["values"]])
        else:
            hm.activate(keys)
        return hm

    def key_buffer(self):
        """int32 [capacity, key_dim] view of kB (valid until the next rehash)."""
        p, stride = ctypes.c_void_p(), _I64()
        _check(lib().ash_key_buffer(self._h, ctypes.byref(p), ctypes.byref(stride)))
        full = _view(p.value, (self.capacity(), stride.value), torch.int32, self.device, self)
        return full[:, : self.key_dim]

    def value_buffer(self, j=0):
        """[capacity, *shape_j] view of vB_j (valid until the next rehash)."""
        p, rb = ctypes.c_void_p(), _I64()
        _check(lib().ash_value_buffer(self._h, j, ctypes.byref(p), ctypes.byref(rb)))
        return _view(p.value, (self.capacity(), *self.value_shapes[j]), self.value_dtypes[j], self.device, self)

    def heap(self):
        """(h as int32 [capacity] view, heap top t)."""
        hp, tp = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().ash_heap_buffer(self._h, ctypes.byref(hp), ctypes.byref(tp)))
        h = _view(hp.value, (self.capacity(),), torch.int32, self.device, self)
        t = _view(tp.value, (1,), torch.int32, self.device, self)
        return h, int(t.item())

    def tuning(self):
        t = Tuning()
        _check(lib().ash_get_tuning(self._h, ctypes.byref(t)))
        return t

    def set_tuning(self, t):
        _check(lib().ash_set_tuning(self._h, ctypes.byref(t)))

    @property
    def handle(self):
        return self._h


# ------------------------------------------------------------ geometry (Sec. 6.2)
def _cam_arrays(intrinsics, extrinsic):
    intr = (ctypes.c_float * 4)(*[float(x) for x in intrinsics])
    e = [float(x) for x in torch.as_tensor(extrinsic, dtype=torch.float32).reshape(12).tolist()]
    return intr, (ctypes.c_float * 12)(*e)


def ash_depth_to_block_keys(depth, intrinsics, extrinsic, block_edge, depth_max, keys=None, count_dev=None,
                            sync=True, stream=None):
    """Block keys of a float32 [H, W] depth image (pixel order, pixels with a
    measurement only).  sync=True returns keys[:n]; otherwise (keys, count_dev)
    with the count left in device memory."""
    _need_cuda(depth, "depth", torch.float32)
    h, w = depth.shape
    if keys is None:
        keys = torch.empty((h * w, 3), dtype=torch.int32, device=depth.device)
    if count_dev is None and not sync:
        count_dev = torch.zeros(1, dtype=torch.int64, device=depth.device)
    intr, extr = _cam_arrays(intrinsics, extrinsic)
    n = _I64(0)
    _check(lib().ash_depth_to_block_keys(_ptr(depth), w, h, intr, extr, float(block_edge), float(depth_max),
                                         _ptr(keys), _ptr(count_dev), ctypes.byref(n) if sync else None,
                                         stream if stream is not None else _stream(depth.device)))
    return keys[: n.value] if sync else (keys, count_dev)


def ash_double_map_activate(local, glob, keys, stream=None):
    """Double hash map block allocation (Sec. 6.2): returns (unique_keys [u, d],
    local_indices [u], global_indices [u]); the local map's int32 values now
    hold the global indices."""
    keys = local._keys(keys)
    n = keys.shape[0]
    uk = torch.empty((n, local.key_dim), dtype=torch.int32, device=local.device)
    li = torch.empty(n, dtype=torch.int32, device=local.device)
    gi = torch.empty(n, dtype=torch.int32, device=local.device)
    u = _I64(0)
    _check(lib().ash_double_map_activate(local.handle, glob.handle, _ptr(keys), n, _ptr(uk), _ptr(li), _ptr(gi),
                                         ctypes.byref(u), stream if stream is not None else _stream(local.device)))
    return uk[: u.value], li[: u.value], gi[: u.value]


def ash_tsdf_integrate(blocks, block_indices, depth, intrinsics, extrinsic, voxel_size, trunc, depth_max,
                       tsdf_buffer=0, weight_buffer=1, stream=None):
    """TSDF integration of one frame (Sec. 6.2, Eq. (7)-(9)) into the blocks at
    block_indices (int32 device tensor of buffer indices)."""
    _need_cuda(depth, "depth", torch.float32)
    bi = block_indices.to(torch.int32).contiguous()
    intr, extr = _cam_arrays(intrinsics, extrinsic)
    h, w = depth.shape
    _check(lib().ash_tsdf_integrate(blocks.handle, tsdf_buffer, weight_buffer, _ptr(bi), bi.numel(), _ptr(depth), w,
                                    h, intr, extr, float(voxel_size), float(trunc), float(depth_max),
                                    stream if stream is not None else _stream(blocks.device)))


def ash_tsdf_raycast(blocks, intrinsics, extrinsic, width, height, voxel_size, depth_min, step, n_steps,
                     local=None, tsdf_buffer=0, weight_buffer=1, out=None, stream=None):
    """Ray-cast depth image (float32 [height, width]; 0 where no surface)."""
    if out is None:
        out = torch.empty((height, width), dtype=torch.float32, device=blocks.device)
    intr, extr = _cam_arrays(intrinsics, extrinsic)
    _check(lib().ash_tsdf_raycast(blocks.handle, tsdf_buffer, weight_buffer, local.handle if local is not None else None,
                                  intr, extr, int(width), int(height), float(voxel_size), float(depth_min),
                                  float(step), int(n_steps), _ptr(out),
                                  stream if stream is not None else _stream(blocks.device)))
    return out


def ash_get_device_info(device=0) -> dict:
    info = DeviceInfo()
    _check(lib().ash_get_device_info(int(device), ctypes.byref(info)))
    return info.as_dict()
