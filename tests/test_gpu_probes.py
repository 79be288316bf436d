"""The measurement probes (random sector reads, random 64-bit CAS and the
load->CAS chain) run, stay inside their buffers and leave checkable state.

They are not part of the method; the bench uses them as the random-access
ceilings that the claim and find kernels are compared against.
"""
import numpy as np
import pytest
import torch

from paper_2110_00511_gb300 import ash

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()


def _written(buf):
    w = buf.view(torch.int64).cpu().numpy().view(np.uint64)
    return w[w != EMPTY]


@pytest.mark.parametrize("mode", [0, 1])
def test_atomic_probe_writes_distinct_op_indices(mode):
    n_buckets = 1 << 18
    whole = torch.full((n_buckets * 32 + 4096,), 255, dtype=torch.uint8, device="cuda")
    buf, guard = whole[: n_buckets * 32], whole[n_buckets * 32:]
    sink = torch.zeros(64, dtype=torch.int32, device="cuda")
    n_ops = 5000
    ash.ash_probe_random_atomic(buf, n_ops, mode, sink, seed=3)
    torch.cuda.synchronize()
    vals = _written(buf)
    # every successful CAS stored its own op index, at most once per op
    assert len(np.unique(vals)) == len(vals)
    assert vals.max() < n_ops
    # 5000 ops over 2^18 buckets: almost all land in a free slot
    assert len(vals) >= 0.98 * n_ops
    if mode == 1:
        # the chain takes the first EMPTY slot, so written slots are a prefix of each bucket
        w = buf.view(torch.int64).cpu().numpy().view(np.uint64).reshape(-1, 4)
        filled = w != EMPTY
        assert not np.any(~filled[:, :-1] & filled[:, 1:])
    assert torch.all(guard == 255)


def test_atomic_probe_rejects_bad_arguments():
    sink = torch.zeros(8, dtype=torch.int32, device="cuda")
    buf = torch.full((100,), 255, dtype=torch.uint8, device="cuda")  # not a multiple of 32 bytes
    with pytest.raises(ash.AshError):
        ash.ash_probe_random_atomic(buf, 10, 0, sink)
    good = torch.full((64,), 255, dtype=torch.uint8, device="cuda")
    with pytest.raises(ash.AshError):
        ash.ash_probe_random_atomic(good, 10, 2, sink)


def test_read_probe_runs_on_both_sector_sizes():
    buf = torch.zeros(1 << 22, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(64, dtype=torch.int32, device="cuda")
    for sector in (32, 64):
        for loads in (4, 8, 16):
            ash.ash_probe_random_read(buf, (1 << 16) + 3, sector, sink, seed=1, loads_per_thread=loads)
    torch.cuda.synchronize()
    # zero-filled input never matches the sink's trigger value
    assert torch.all(sink == 0)
