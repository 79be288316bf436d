"""Multi-tenant serving with continuous batching: every request's result is
the same when it runs in the mix (many requests in flight, batched across
tenants) as when its tenant's requests run alone, one plain call at a time;
and the tenant maps match the oracle.  Bar: bit-exact masks, stored keys and
value bytes (indices compared through the keys they hold)."""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_same_map, gpu_state, oracle_state
from paper_2110_00511_gb300 import ash

pytestmark = pytest.mark.gpu

OPS = {"insert": ash.ASH_OP_INSERT, "find": ash.ASH_OP_FIND, "erase": ash.ASH_OP_ERASE}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()


def _trace(seed, n_req, n_tenants, size_range=(200, 30_000), span=60):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n_req):
        op = rng.choice(["insert", "find", "erase"], p=[0.4, 0.45, 0.15])
        n = int(np.exp(rng.uniform(np.log(size_range[0]), np.log(size_range[1]))))
        keys = rng.integers(-span, span, size=(n, 3)).astype(np.int32)
        vals = rng.random(n, dtype=np.float32) if op == "insert" else None
        reqs.append((int(rng.integers(0, n_tenants)), op, keys, vals))
    return reqs


def _run_alone(reqs, n_tenants, cap):
    """Each tenant's requests, in order, through plain calls on its own map."""
    maps = [ash.HashMap(3, cap, [(1,)], [torch.float32]) for _ in range(n_tenants)]
    out = []
    for t, op, keys, vals in reqs:
        k = torch.from_numpy(keys).cuda()
        if op == "insert":
            i, m = maps[t].insert(k, [torch.from_numpy(vals).cuda()])
        elif op == "find":
            i, m = maps[t].find(k)
        else:
            i, m = None, maps[t].erase(k)
        out.append((None if i is None else i.cpu().numpy(), m.cpu().numpy()))
    return maps, out


def _check_same(reqs, served, alone, server_maps, alone_maps):
    # an index stays bound to its key until a later erase on that tenant frees it
    last_erase = {}
    for j, (t, op, _, _) in enumerate(reqs):
        if op == "erase":
            last_erase[t] = j
    for j, ((t, op, keys, vals), (si, sm), (ai, am)) in enumerate(zip(reqs, served, alone)):
        assert np.array_equal(sm, am), f"request {j} ({op} on tenant {t}) differs from running alone"
        if op != "erase" and sm.any() and last_erase.get(t, -1) < j:
            kb_s = server_maps[t].key_buffer().cpu().numpy()
            assert np.array_equal(kb_s[si[sm]], keys[sm]), f"request {j}: served index holds another key"
            assert (si[~sm] == -1).all()


def _pinned(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("zero_copy", [0, 1, 2])
def test_served_results_equal_alone_and_oracle(zero_copy):
    """Staged (0), zero-copy (1: the kernels read the caller's arrays in
    place, on devices with pageable host memory access), and DMA from the
    caller's pinned arrays (2; every other request pinned, the rest copied)."""
    if zero_copy == 1 and ash.ash_get_device_info(0)["pageable_memory_access"] != 1:
        pytest.skip("no pageable memory access on this device")
    n_t = 4
    reqs = _trace(1, 80, n_t)
    if zero_copy == 2:
        reqs = [(t, op, _pinned(k), _pinned(v)) if j % 2 == 0 else (t, op, k, v)
                for j, (t, op, k, v) in enumerate(reqs)]
    srv = ash.Server(n_tenants=n_t, key_dim=3, initial_capacity=2048, value_row_bytes=4,
                     staging_bytes=64 << 20, max_load=0.7, max_batch_requests=256, zero_copy=zero_copy)
    ids = [srv.submit(t, OPS[op], keys, vals) for t, op, keys, vals in reqs]  # all in flight
    served = []
    for rid in ids:
        i, m, lat = srv.wait(rid)
        assert lat >= 0.0
        served.append((i, m))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["batches"] < len(reqs), st  # batched across tenants
    assert st["rehashes"] > 0, st  # grew past max_load
    server_maps = [ash.HashMap.wrap(srv.map_handle(t), 3, [(1,)], [torch.float32]) for t in range(n_t)]
    alone_maps, alone = _run_alone(reqs, n_t, 2048)
    _check_same(reqs, served, alone, server_maps, alone_maps)
    oras = [oracle.OracleMap(3, 2048, [4]) for _ in range(n_t)]
    for t, op, keys, vals in reqs:
        if op == "insert":
            oras[t].insert(keys, [vals])
        elif op == "erase":
            oras[t].erase(keys)
    for t in range(n_t):
        sk, _ = server_maps[t], None
        # capacities differ (the server grows at max_load 0.7), the dictionaries do not
        ok = oracle_state_equal(server_maps[t], oras[t])
        assert ok, f"tenant {t} map differs from the oracle"
    srv.close()


def oracle_state_equal(hm, om):
    from parity import gpu_state, oracle_state
    gk, gv = gpu_state(hm)
    ok, ov = oracle_state(om)
    return np.array_equal(gk, ok) and all(np.array_equal(a, b) for a, b in zip(gv, ov))


def test_admission_under_a_small_budget():
    n_t = 3
    reqs = _trace(2, 30, n_t, size_range=(1000, 200_000), span=200)
    srv = ash.Server(n_tenants=n_t, key_dim=3, initial_capacity=1 << 16, value_row_bytes=4,
                     staging_bytes=1 << 20, max_load=0.7, max_batch_requests=2)
    ids = [srv.submit(t, OPS[op], keys, vals) for t, op, keys, vals in reqs]
    served = [srv.wait(rid)[:2] for rid in ids]
    server_maps = [ash.HashMap.wrap(srv.map_handle(t), 3, [(1,)], [torch.float32]) for t in range(n_t)]
    alone_maps, alone = _run_alone(reqs, n_t, 1 << 16)
    _check_same(reqs, served, alone, server_maps, alone_maps)
    srv.close()


def test_zero_copy_refused_without_pageable_access():
    if ash.ash_get_device_info(0)["pageable_memory_access"] == 1:
        srv = ash.Server(n_tenants=1, key_dim=3, initial_capacity=1024, zero_copy=1)
        srv.close()
    else:
        with pytest.raises(ash.AshError):
            ash.Server(n_tenants=1, key_dim=3, initial_capacity=1024, zero_copy=1)
    with pytest.raises(ash.AshError):
        ash.Server(n_tenants=1, key_dim=3, initial_capacity=1024, zero_copy=3)


def test_server_rejects_bad_requests():
    srv = ash.Server(n_tenants=2, key_dim=3, initial_capacity=1024, value_row_bytes=0)
    with pytest.raises(ash.AshError):
        srv.submit(5, ash.ASH_OP_FIND, np.zeros((4, 3), np.int32))
    with pytest.raises(ash.AshError):
        srv.submit(0, 9, np.zeros((4, 3), np.int32))
    rid = srv.submit(1, ash.ASH_OP_ACTIVATE, np.arange(12, dtype=np.int32).reshape(4, 3))
    i, m, _ = srv.wait(rid)
    assert m.all()
    with pytest.raises(ash.AshError):
        srv.wait(rid)  # already collected
    srv.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_native_replay_matches_sequential_calls(mode):
    """The native replays used by the bench: one Poisson trace through the
    server (from native threads) and as sequential plain calls leaves every
    tenant's map with the same key -> value dictionary (each tenant's
    requests apply in arrival order in both), every request completes, and
    the sequential maps equal the oracle run on the same trace.  Malformed
    traces are refused before anything runs."""
    rng = np.random.default_rng(40 + mode)
    n_t, R, rows = 4, 300, 200_000
    keys = torch.from_numpy(rng.integers(-50, 50, size=(rows, 3)).astype(np.int32)).pin_memory().numpy()
    vals = torch.from_numpy(rng.random(rows, dtype=np.float32)).pin_memory().numpy()
    sizes = np.exp(rng.uniform(np.log(100), np.log(20_000), size=R)).astype(np.int64)
    trace = ash.Trace(np.cumsum(rng.exponential(1 / 20_000.0, size=R)), rng.integers(0, n_t, size=R),
                      np.array([ash.ASH_OP_INSERT, ash.ASH_OP_FIND, ash.ASH_OP_ERASE])[rng.choice(3, size=R, p=[.4, .45, .15])],
                      sizes, rng.integers(0, rows - sizes), keys, vals)
    srv = ash.Server(n_tenants=n_t, key_dim=3, initial_capacity=1 << 12, value_row_bytes=4, staging_bytes=8 << 20,
                     zero_copy=mode)
    lat, span = srv.replay(trace, threads=4)
    assert np.all(lat >= 0) and span > 0
    maps = [ash.HashMap(3, 1 << 12, [(1,)], [torch.float32]) for _ in range(n_t)]
    slat, sspan = ash.replay_sequential(maps, trace)
    assert np.all(slat >= 0) and sspan > 0
    oms = [oracle.OracleMap(3, 1 << 12, [4]) for _ in range(n_t)]
    for r in range(R):
        k = keys[trace.row[r]:trace.row[r] + trace.n[r]]
        om = oms[trace.tenant[r]]
        if trace.op[r] == ash.ASH_OP_INSERT:
            om.insert(k, [vals[trace.row[r]:trace.row[r] + trace.n[r]]])
        elif trace.op[r] == ash.ASH_OP_FIND:
            om.find(k)
        else:
            om.erase(k)
    torch.cuda.synchronize()
    for t in range(n_t):
        assert_same_map(maps[t], oms[t])
        # the server grows at load 0.7, so only its capacity may differ from the oracle's
        served = ash.HashMap.wrap(srv.map_handle(t), 3, [(1,)], [torch.float32])
        gk, gv = gpu_state(served)
        ok, ov = oracle_state(oms[t])
        assert np.array_equal(gk, ok) and all(np.array_equal(a, b) for a, b in zip(gv, ov))
        assert served.size() == oms[t].size()
    srv.close()
    bad = ash.Trace(np.array([0.0, 0.0]), np.array([0, 9]), np.array([2, 2]), np.array([10, 10]), np.array([0, 0]),
                    keys, vals)
    srv2 = ash.Server(n_tenants=n_t, key_dim=3, initial_capacity=1 << 12, value_row_bytes=4)
    with pytest.raises(ash.AshError):
        srv2.replay(bad)
    past = ash.Trace(np.array([0.0]), np.array([0]), np.array([2]), np.array([10]), np.array([rows - 5]), keys, vals)
    with pytest.raises(ash.AshError):
        ash.replay_sequential(maps, past)
    srv2.close()
