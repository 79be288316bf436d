"""Map calls with host pointers on a coherent CPU-GPU system: when the device
reports pageable memory access, keys, values and outputs may live in ordinary
host memory and the kernels read and write them in place.  Results must equal
the device-buffer calls and the oracle.  Skipped where the device lacks the
capability (a kernel must never be handed a host pointer there)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from parity import assert_op_parity, assert_same_map
from paper_2110_00511_gb300 import ash, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()
    if ash.ash_get_device_info(0)["pageable_memory_access"] != 1:
        pytest.skip("no pageable memory access on this device")


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def test_host_pointer_insert_find_erase():
    L = ash.lib()
    st = ash._stream()
    rng = np.random.default_rng(5)
    keys = rng.integers(-300, 300, size=(200_001, 3)).astype(np.int32)
    vals = rng.random(len(keys), dtype=np.float32)
    hm = ash.HashMap(3, 150_000, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, 150_000, [4])
    idx = np.empty(len(keys), np.int32)
    mask = np.empty(len(keys), np.uint8)
    varr = (ctypes.c_void_p * 1)(vals.ctypes.data)
    ash._check(L.ash_insert(hm.handle, P(keys), varr, len(keys), P(idx), P(mask), st))
    torch.cuda.synchronize()
    oi, om_ = om.insert(keys, [vals])
    assert_op_parity(hm, keys, torch.from_numpy(idx).cuda(), torch.from_numpy(mask.astype(bool)).cuda(), oi, om_)
    q = np.concatenate([keys[::2], rng.integers(-320, 320, size=(50_000, 3)).astype(np.int32)])
    fi = np.empty(len(q), np.int32)
    fm = np.empty(len(q), np.uint8)
    ash._check(L.ash_find(hm.handle, P(q), len(q), P(fi), P(fm), st))
    torch.cuda.synchronize()
    dfi, dfm = hm.find(torch.from_numpy(q).cuda())
    assert np.array_equal(fi, dfi.cpu().numpy()) and np.array_equal(fm.astype(bool), dfm.cpu().numpy())
    er = keys[rng.integers(0, len(keys), size=30_000)]
    em = np.empty(len(er), np.uint8)
    ash._check(L.ash_erase(hm.handle, P(er), len(er), P(em), st))
    torch.cuda.synchronize()
    assert np.array_equal(em, om.erase(er))
    assert_same_map(hm, om)


def test_host_pointer_quantize_and_gather():
    L = ash.lib()
    st = ash._stream()
    pts = workloads.voxel_scene_points(200_000, seed=2)
    keys_h = np.empty(pts.shape, np.int32)
    ash._check(L.ash_quantize(P(pts), pts.size, ctypes.c_float(0.005), P(keys_h), st))
    torch.cuda.synchronize()
    assert np.array_equal(keys_h, oracle.quantize(pts, 0.005))
    hm = ash.HashMap(3, len(keys_h))
    hm.activate(torch.from_numpy(keys_h).cuda())
    act = hm.active_indices().cpu().numpy()
    out = np.empty((len(act), 3), np.int32)
    ash._check(L.ash_gather_keys(hm.handle, P(act), len(act), P(out), st))
    torch.cuda.synchronize()
    assert np.array_equal(np.unique(out, axis=0), np.unique(keys_h, axis=0))
