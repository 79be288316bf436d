"""Randomised differential test: random operation sequences on small maps
with random key dimensions, bucket sizes, table sizes, keys per thread and
probing modes, checked against the oracle after every operation (masks,
stored keys, values by key, size, capacity, heap permutation).  Keys come
from a small range so duplicates, re-inserts after erase, tombstones and
growth are all frequent."""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_heap_permutation, assert_op_parity, assert_same_map

from paper_2110_00511_gb300 import ash

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("seed", range(60))
def test_random_sequences(seed):
    rng = np.random.default_rng(7000 + seed)
    mode_rng_init = np.random.default_rng(9500 + seed)  # knobs drawn apart from the op sequence
    d = int(rng.choice([1, 2, 3, 4, 5, 8]))
    cap = int(rng.integers(1, 300))
    t = ash.default_tuning()
    t.slots_per_bucket = int(rng.choice([4, 8, 16]))
    t.slots_per_capacity = float(rng.choice([1.1, 1.5, 2.0, 4.0]))
    t.keys_per_thread = int(rng.choice([1, 2, 4]))
    t.warp_probe = int(rng.integers(0, 2))
    t.find_keys_per_thread = int(rng.choice([0, 1, 2, 4]))
    t.commit_keys_per_thread = int(mode_rng_init.choice([0, 1, 2, 4]))
    t.block_threads = int(rng.choice([64, 128, 256]))
    vrow = int(rng.choice([0, 4, 12]))
    shapes, dtypes, rbs = ([], [], []) if vrow == 0 else ([(vrow // 4,)], [torch.float32], [vrow])
    hm = ash.HashMap(d, cap, shapes, dtypes, tuning=t)
    om = oracle.OracleMap(d, cap, rbs)
    span = int(rng.integers(2, 40))
    # the claim protocol switches between calls (its own generator, so the
    # operation sequence of each seed does not depend on it)
    mode_rng = np.random.default_rng(9000 + seed)
    # key order (input or home-bucket ranges) switches too, from its own generator
    part_rng = np.random.default_rng(9700 + seed)
    for step in range(40):
        op = rng.choice(["insert", "activate", "find", "erase", "rehash", "reserve", "clear"],
                        p=[0.3, 0.15, 0.25, 0.2, 0.04, 0.03, 0.03])
        n = int(rng.integers(0, 400))
        keys = rng.integers(-span, span, size=(n, d)).astype(np.int32)
        if op == "activate" and vrow:
            op = "insert"
        if op in ("insert", "activate"):
            tt = hm.tuning()
            tt.claim_mode = int(mode_rng.integers(0, 3))
            hm.set_tuning(tt)
        if op in ("insert", "activate", "find"):
            tt = hm.tuning()
            tt.partition_keys = int(part_rng.integers(0, 3))
            hm.set_tuning(tt)
        if op == "insert":
            if vrow:
                vals = rng.random((n, vrow // 4), dtype=np.float32)
                gi, gm = hm.insert(dev(keys), [dev(vals)])
                oi, omask = om.insert(keys, [vals])
            else:
                gi, gm = hm.activate(dev(keys))
                oi, omask = om.activate(keys)
            assert_op_parity(hm, keys, gi, gm, oi, omask)
        elif op == "activate" and not vrow:
            # (with value buffers only insert is used: an activated key's value
            # bytes are whatever its re-used index held, which the paper leaves
            # to the user, so they are not comparable)
            gi, gm = hm.activate(dev(keys))
            oi, omask = om.activate(keys)
            assert_op_parity(hm, keys, gi, gm, oi, omask)
        elif op == "find":
            gi, gm = hm.find(dev(keys))
            oi, omask = om.find(keys)
            assert_op_parity(hm, keys, gi, gm, oi, omask, check_distinct=False)
        elif op == "erase":
            assert np.array_equal(hm.erase(dev(keys)).cpu().numpy(), om.erase(keys))
        elif op == "rehash":
            c = int(rng.integers(max(1, om.size()), 2 * om.capacity() + 2))
            hm.rehash(c)
            om.rehash(c)
        elif op == "reserve":
            c = int(rng.integers(1, 3 * om.capacity() + 2))
            hm.reserve(c)
            if c > om.capacity():
                om.rehash(c)
        else:
            hm.clear()
            om.clear()
        assert hm.size() == om.size(), f"step {step} {op}: size"
        assert hm.capacity() == om.capacity(), f"step {step} {op}: capacity"
        assert_same_map(hm, om, check_values=bool(vrow))
        assert_heap_permutation(hm)
