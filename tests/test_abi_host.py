"""Host-side behaviour of the C ABI that needs no GPU: defaults, the tracer's
kernel names, and argument validation that rejects bad calls with
ASH_ERR_INVALID and a message before any device work (run on CPU)."""
import ctypes
import os
import shutil

import pytest

from paper_2110_00511_gb300 import ash

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2110_00511_gb300 import build
    build.build()
    return ash.lib()


def _err(status):
    assert status == ash.ASH_ERR_INVALID, status
    msg = ash.lib().ash_last_error().decode()
    assert msg, "an error must come with a message"
    return msg


def test_default_tuning_and_server_config():
    t = ash.default_tuning()
    assert (t.slots_per_bucket, t.keys_per_thread, t.find_keys_per_thread, t.warp_probe, t.auto_grow,
            t.claim_mode, t.commit_keys_per_thread, t.partition_keys) == (4, 2, 1, 0, 1, 0, 1, 0)
    assert abs(t.slots_per_capacity - 2.0) < 1e-6 and abs(t.max_used_fraction - 0.65) < 1e-6
    c = ash.ash_server_default_config()
    assert (c.n_tenants, c.key_dim, c.zero_copy) == (16, 3, 0) and abs(c.max_load - 0.7) < 1e-6


def test_tracer_names():
    L = ash.lib()
    n = L.ash_trace_kernel_kinds()
    names = [L.ash_trace_kernel_name(k).decode() for k in range(n)]
    for must in ("find", "insert_claim", "insert_commit", "erase_mark", "list_active", "tsdf_integrate",
                 "tsdf_raycast"):
        assert must in names
    assert len(set(names)) == n and L.ash_trace_kernel_name(n) == b""


def test_create_rejects_bad_arguments():
    L = ash.lib()
    out = ctypes.c_void_p()
    t = ash.default_tuning()
    assert "key_dim" in _err(L.ash_create(0, 16, 0, None, None, 0, ctypes.byref(t), None, ctypes.byref(out)))
    assert "capacity" in _err(L.ash_create(3, 0, 0, None, None, 0, ctypes.byref(t), None, ctypes.byref(out)))
    _err(L.ash_create(3, 16, 9, None, None, 0, ctypes.byref(t), None, ctypes.byref(out)))
    _err(L.ash_create(3, 16, 0, None, None, 0, ctypes.byref(t), None, None))


def test_map_calls_reject_null_map_and_bad_sizes():
    L = ash.lib()
    p = ctypes.c_void_p(0)
    _err(L.ash_find(None, p, 4, p, p, None))
    _err(L.ash_insert(None, p, None, 4, p, p, None))
    _err(L.ash_erase(None, p, 4, p, None))
    _err(L.ash_find_offsets(None, p, 4, p, 1, p, p, None))
    _err(L.ash_batch_run(None, None, 0, None))


def test_geometry_and_probe_validation():
    L = ash.lib()
    p = ctypes.c_void_p(0)
    intr = (ctypes.c_float * 4)(1, 1, 0, 0)
    extr = (ctypes.c_float * 12)(1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0)
    n = ash._I64()
    _err(L.ash_depth_to_block_keys(p, -1, 4, intr, extr, 0.1, 4.0, p, None, ctypes.byref(n), None))
    _err(L.ash_depth_to_block_keys(p, 4, 4, intr, extr, 0.0, 4.0, p, None, ctypes.byref(n), None))
    _err(L.ash_double_map_activate(None, None, p, 4, p, p, p, ctypes.byref(n), None))
    _err(L.ash_tsdf_integrate(None, 0, 1, p, 4, p, 4, 4, intr, extr, 0.01, 0.03, 4.0, None))
    _err(L.ash_tsdf_raycast(None, 0, 1, None, intr, extr, 4, 4, 0.01, 0.3, 0.01, 10, p, None))
    _err(L.ash_probe_random_atomic(p, 64, 10, 2, 0, p, 4, None))
    _err(L.ash_probe_random_read(p, 64, 10, 48, 8, 0, p, 4, None))
    _err(L.ash_probe_random_read(p, 64, 10, 32, 5, 0, p, 4, None))


def test_server_config_validation():
    L = ash.lib()
    out = ctypes.c_void_p()
    for field, bad in (("n_tenants", 0), ("key_dim", 5), ("value_row_bytes", 12), ("max_load", 0.0),
                       ("max_batch_requests", 0), ("zero_copy", 3)):
        c = ash.ash_server_default_config()
        setattr(c, field, bad)
        _err(L.ash_server_create(ctypes.byref(c), ctypes.byref(out)))


def test_erase_noalloc_binding_rejects_bad_arrays():
    """The Python route to ash_erase_noalloc checks its arrays before the
    library sees them: host tensors, wrong dtypes or shapes never reach the
    kernels (the checks run before any device work, so they hold on CPU)."""
    import torch
    k_cpu = torch.zeros((4, 3), dtype=torch.int32)
    m_cpu = torch.zeros(4, dtype=torch.bool)
    with pytest.raises(ValueError, match="CUDA"):
        ash.ash_erase_noalloc(None, k_cpu, m_cpu)
    with pytest.raises(ValueError, match="CUDA|int32"):
        ash.ash_erase_noalloc(None, k_cpu.to(torch.int64), m_cpu)
    with pytest.raises(ValueError, match="torch tensors"):
        ash.ash_erase_noalloc(None, k_cpu.numpy(), m_cpu)
