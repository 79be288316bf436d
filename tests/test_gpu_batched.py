"""Batched execution (one CUDA-graph launch over many maps) vs the oracle and
vs the same operations issued map by map through the plain calls.

Per map the phase order is insert -> find -> erase; the oracle applies the
same order.  Bar: bit-exact masks, stored keys and value bytes, modulo the
buffer-index permutation.
"""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_heap_permutation, assert_op_parity, assert_same_map
from paper_2110_00511_gb300 import ash, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _tuning(S):
    t = ash.default_tuning()
    t.slots_per_bucket = S
    return t


def _case(seed, d, cap):
    rng = np.random.default_rng(seed)
    n_ins = cap // 2
    ins = rng.integers(-12, 12, size=(n_ins, d)).astype(np.int32)
    vals = rng.random(n_ins, dtype=np.float32)
    fnd = rng.integers(-14, 14, size=(cap, d)).astype(np.int32)
    er = rng.integers(-12, 12, size=(cap // 4, d)).astype(np.int32)
    return ins, vals, fnd, er


def test_batch_matches_oracle_and_plain_calls():
    batch = ash.Batch(0)
    specs = [(d, S, cap) for d in (1, 2, 3, 4) for S in (4, 8, 16) for cap in (1000,)] + [(3, 4, 50_000), (2, 8, 7)]
    maps, plain, oras, data = [], [], [], []
    for i, (d, S, cap) in enumerate(specs):
        maps.append(ash.HashMap(d, cap, [(1,)], [torch.float32], tuning=_tuning(S)))
        plain.append(ash.HashMap(d, cap, [(1,)], [torch.float32], tuning=_tuning(S)))
        oras.append(oracle.OracleMap(d, cap, [4]))
        data.append(_case(100 + i, d, cap))
    for rnd in range(3):  # replays reuse the graph ring and grow some maps
        items = []
        for hm, (ins, vals, fnd, er) in zip(maps, data):
            items += [(hm, ash.ASH_OP_INSERT, dev(ins + rnd), dev(vals)), (hm, ash.ASH_OP_FIND, dev(fnd), None),
                      (hm, ash.ASH_OP_ERASE, dev(er), None)]
        outs = batch.run(items)
        torch.cuda.synchronize()
        for j, (hm, ph, om, (ins, vals, fnd, er)) in enumerate(zip(maps, plain, oras, data)):
            (gi, gm), (fi, fm), (_, em) = outs[3 * j], outs[3 * j + 1], outs[3 * j + 2]
            oi, omask = om.insert(ins + rnd, [vals])
            assert_op_parity(hm, ins + rnd, gi, gm, oi, omask)
            ofi, ofm = om.find(fnd)
            assert np.array_equal(fm.cpu().numpy(), ofm)
            kb = hm.key_buffer().cpu().numpy()
            f = fm.cpu().numpy()
            assert np.array_equal(kb[fi.cpu().numpy()[f]], fnd[f])
            oe = om.erase(er)
            assert np.array_equal(em.cpu().numpy(), oe)
            # the same ops through the plain per-map calls give the same masks
            pi, pm = ph.insert(dev(ins + rnd), [dev(vals)])
            pfi, pfm = ph.find(dev(fnd))
            pem = ph.erase(dev(er))
            assert torch.equal(pm, gm) and torch.equal(pfm, fm) and torch.equal(pem, em)
            assert_same_map(hm, om)
            assert_heap_permutation(hm)


def test_batch_workload_shape_parity():
    """The many-map workload shape (key_dim 2-4, uneven capacities, 30/60/10
    insert/find/erase), checked map by map against the oracle."""
    cases = workloads.batched_maps(n_maps=16, seed=3, log2_cap=(8, 14))
    batch = ash.Batch(0)
    maps = [ash.HashMap(c.key_dim, c.capacity, [(1,)], [torch.float32],
                        tuning=ash.ash_autotune(c.key_dim, c.capacity, c.rho)) for c in cases]
    oras = [oracle.OracleMap(c.key_dim, c.capacity, [4]) for c in cases]
    items = []
    for hm, c in zip(maps, cases):
        items += [(hm, ash.ASH_OP_INSERT, dev(c.insert_keys), dev(c.insert_values)),
                  (hm, ash.ASH_OP_FIND, dev(c.find_keys), None), (hm, ash.ASH_OP_ERASE, dev(c.erase_keys), None)]
    outs = batch.run(items)
    torch.cuda.synchronize()
    for j, (hm, om, c) in enumerate(zip(maps, oras, cases)):
        (gi, gm), (fi, fm), (_, em) = outs[3 * j], outs[3 * j + 1], outs[3 * j + 2]
        oi, omask = om.insert(c.insert_keys, [c.insert_values])
        assert_op_parity(hm, c.insert_keys, gi, gm, oi, omask)
        _, ofm = om.find(c.find_keys)
        assert np.array_equal(fm.cpu().numpy(), ofm)
        assert np.array_equal(em.cpu().numpy(), om.erase(c.erase_keys))
        assert_same_map(hm, om)


def test_batch_rejects_bad_input():
    batch = ash.Batch(0)
    hm = ash.HashMap(3, 100)
    k = dev(np.zeros((4, 3), np.int32))
    with pytest.raises(ash.AshError) as e:
        batch.run([(hm, ash.ASH_OP_FIND, k, None), (hm, ash.ASH_OP_FIND, k, None)])
    assert e.value.status == ash.ASH_ERR_INVALID
    h5 = ash.HashMap(5, 100)
    with pytest.raises(ash.AshError):
        batch.run([(h5, ash.ASH_OP_FIND, dev(np.zeros((4, 5), np.int32)), None)])
    big = ash.HashMap(3, 100, [(8, 8, 8)], [torch.float32])
    with pytest.raises(ash.AshError):
        batch.run([(big, ash.ASH_OP_INSERT, k, torch.zeros((4, 512), device="cuda"))])
    # activate on a map with values is allowed, and an empty batch is a no-op
    batch.run([(big, ash.ASH_OP_ACTIVATE, k, None)])
    batch.run([])
    torch.cuda.synchronize()
    assert big.size() == 1


def test_autotune_returns_valid_cached_tuning():
    t1 = ash.ash_autotune(3, 1 << 16, 0.5)
    t2 = ash.ash_autotune(3, 1 << 16, 0.5)
    assert t1.slots_per_bucket in (4, 8, 16) and t1.keys_per_thread in (1, 2)
    assert t1.as_dict() == t2.as_dict()
    hm = ash.HashMap(3, 1 << 16, tuning=t1)
    keys = workloads.uniform_keys(40_000, 0.5, seed=2)
    gi, gm = hm.activate(dev(keys))
    om = oracle.OracleMap(3, 1 << 16)
    oi, omask = om.activate(keys)
    assert_op_parity(hm, keys, gi, gm, oi, omask)


@pytest.mark.parametrize("S", [4, 8])
def test_batched_then_plain_inserts_with_preferred_slot_claims(S):
    """Batched inserts place keys in slot order, outside the preferred-slot
    invariant; plain inserts that follow (asked for the preferred-slot CAS,
    claim_mode 2) must fall back to the bucket-first claim until a rehash or
    clear restores the invariant, or they would store second copies of keys
    the batch placed.  Dense buckets, erase churn, checked against the oracle
    after every call."""
    rng = np.random.default_rng(60 + S)
    t = _tuning(S)
    t.slots_per_capacity = 1.1
    t.claim_mode = 2
    hm = ash.HashMap(3, 3000, [(1,)], [torch.float32], tuning=t)
    om = oracle.OracleMap(3, 3000, [4])
    batch = ash.Batch(0)
    for r in range(12):
        k = rng.integers(-9, 9, size=(1500, 3)).astype(np.int32)
        v = rng.random(1500, dtype=np.float32)
        if r % 3 == 0:
            (gi, gm), = batch.run([(hm, ash.ASH_OP_INSERT, dev(k), dev(v))])
            torch.cuda.synchronize()
        else:
            gi, gm = hm.insert(dev(k), [dev(v)])
        oi, omask = om.insert(k, [v])
        assert_op_parity(hm, k, gi, gm, oi, omask)
        e = rng.integers(-9, 9, size=(700, 3)).astype(np.int32)
        assert np.array_equal(hm.erase(dev(e)).cpu().numpy(), om.erase(e))
        if r == 7:
            hm.rehash()
            om.rehash()
        assert_same_map(hm, om)
    assert_heap_permutation(hm)
