"""Pins that tie the CPU oracle to something other than itself.

Each pin takes `mutant` (0 = the oracle as built; n >= 1 = a build with one
planted mistake, see oracle/ash_oracle.cpp) and raises AssertionError when the
oracle disagrees with what the paper and the mathematics fix:
  * brute force (a linear list scan, tests/bruteforce.py) on tiny inputs with
    random operation sequences;
  * a hand-traced golden sequence (tests/golden/heap_trace.txt);
  * the map invariants: one winner per duplicate key (the first occurrence),
    the stored key at a returned index equals the query, no index handed out
    twice (active indices and h[t..c) form a permutation of 0..c-1), and
    size = t;
  * closed forms: occupancy of N uniform draws over M cells, zero hits on a
    disjoint query range, x2 growth;
  * reduction to a library routine: the activated key set equals np.unique,
    and the unique inverse agrees with find; quantisation equals numpy's
    float32 floor of the quotient, plus hand-checked boundary values.
"""
import math
import os

import numpy as np

import oracle
from bruteforce import BruteMap
from paper_2110_00511_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _tuples(keys):
    return [tuple(int(x) for x in row) for row in np.asarray(keys)]


def _rows(vals, row_bytes):
    b = np.ascontiguousarray(vals).view(np.uint8).reshape(-1, row_bytes)
    return [r.tobytes() for r in b]


def _check_permutation(om):
    heap = om.heap()
    t = om.heap_top()
    act = om.active_indices()
    assert t == om.size(), "heap top differs from the number of live entries"
    both = np.concatenate([act, heap[t:]])
    assert np.array_equal(np.sort(both), np.arange(om.capacity())), "active + free indices are not a permutation"


# ---------------------------------------------------------------- brute force
def pin_bruteforce(mutant=0, seeds=range(12)):
    for seed in seeds:
        rng = np.random.default_rng(1000 + seed)
        d = int(rng.integers(1, 5))
        cap = int(rng.integers(1, 9))
        rb = 4
        om = oracle.OracleMap(d, cap, [rb], mutant=mutant)
        bf = BruteMap(d, cap, [rb])
        for step in range(40):
            op = rng.choice(["insert", "activate", "find", "erase", "rehash", "clear"], p=[0.3, 0.15, 0.25, 0.2, 0.05, 0.05])
            n = int(rng.integers(0, 9))
            keys = rng.integers(-2, 2, size=(n, d)).astype(np.int32)
            if op == "insert":
                vals = rng.integers(-1000, 1000, size=n).astype(np.int32)
                i1, m1 = om.insert(keys, [vals])
                i2, m2 = bf.insert(_tuples(keys), [_rows(vals, rb)])
                assert list(m1) == m2 and list(i1) == i2, f"insert differs (seed {seed} step {step})"
            elif op == "activate":
                i1, m1 = om.activate(keys)
                i2, m2 = bf.activate(_tuples(keys))
                assert list(m1) == m2 and list(i1) == i2, f"activate differs (seed {seed} step {step})"
            elif op == "find":
                i1, m1 = om.find(keys)
                i2, m2 = bf.find(_tuples(keys))
                assert list(m1) == m2 and list(i1) == i2, f"find differs (seed {seed} step {step})"
            elif op == "erase":
                m1 = om.erase(keys)
                m2 = bf.erase(_tuples(keys))
                assert list(m1) == m2, f"erase differs (seed {seed} step {step})"
            elif op == "rehash":
                newc = max(len(bf.entries), int(rng.integers(1, 17)))
                om.rehash(newc)
                bf.rehash(newc)
            else:
                om.clear()
                bf.clear()
            assert om.capacity() == bf.capacity, "capacity differs"
            assert om.size() == len(bf.entries), "size differs"
            assert om.heap_top() == bf.top, "heap top differs"
            assert list(om.heap()) == bf.heap, "heap array differs"
            od = om.as_dict()
            assert od == bf.as_dict(), f"dictionary differs (seed {seed} step {step})"
            if op != "clear":
                _check_permutation(om)


# ------------------------------------------------------------- golden trace
def _parse_keys(s, d):
    return np.array([[int(x) for x in k.split(",")] for k in s.split(";")], np.int32).reshape(-1, d)


def _ints(s):
    return [int(x) for x in s.split(";")]


def pin_golden_trace(mutant=0):
    om = None
    d = None
    with open(os.path.join(GOLDEN, "heap_trace.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    for ln in lines:
        head, _, exp = ln.partition(" expect: ")
        parts = head.split()
        op = parts[0]
        args = dict(p.split("=", 1) for p in parts[1:])
        if op == "create":
            d = int(args["key_dim"])
            om = oracle.OracleMap(d, int(args["capacity"]), [4], mutant=mutant)
            continue
        expect = dict(p.split("=", 1) for p in exp.split())
        idx = mask = None
        if op in ("insert", "activate", "find", "erase"):
            keys = _parse_keys(args["keys"], d)
        if op == "insert":
            idx, mask = om.insert(keys, [np.array(_ints(args["values"]), np.int32)])
        elif op == "activate":
            idx, mask = om.activate(keys)
        elif op == "find":
            idx, mask = om.find(keys)
        elif op == "erase":
            mask = om.erase(keys)
        if "idx" in expect:
            assert list(idx) == _ints(expect["idx"]), f"golden idx: {ln}"
        if "mask" in expect:
            assert [int(m) for m in mask] == _ints(expect["mask"]), f"golden mask: {ln}"
        if "top" in expect:
            assert om.heap_top() == int(expect["top"]), f"golden top: {ln}"
        if "heap" in expect:
            assert list(om.heap()) == _ints(expect["heap"]), f"golden heap: {ln}"
        if "capacity" in expect:
            assert om.capacity() == int(expect["capacity"]), f"golden capacity: {ln}"
        if "size" in expect:
            assert om.size() == int(expect["size"]), f"golden size: {ln}"
        if "dict" in expect:
            want = {}
            for item in expect["dict"].split(";"):
                k, v = item.split(":")
                want[tuple(int(x) for x in k.split(","))] = (np.int32(int(v)).tobytes(),)
            assert om.as_dict() == want, f"golden dict: {ln}"


# ---------------------------------------------------------------- invariants
def pin_invariants(mutant=0, seed=7):
    rng = np.random.default_rng(seed)
    d = 3
    om = oracle.OracleMap(d, 1 << 12, [4], mutant=mutant)
    for step in range(12):
        n = int(rng.integers(100, 3000))
        keys = rng.integers(-8, 8, size=(n, d)).astype(np.int32)
        vals = np.arange(n, dtype=np.int32) + 100000 * step
        before = om.as_dict()
        idx, mask = om.insert(keys, [vals])
        # first occurrence of each key that was absent wins; nothing else does
        seen = set()
        for p in range(n):
            k = tuple(int(x) for x in keys[p])
            expect = (k not in before) and (k not in seen)
            seen.add(k)
            assert bool(mask[p]) == expect, "winner is not the first occurrence of an absent key"
        kb = om.key_buffer()
        assert np.array_equal(kb[idx[mask]], keys[mask]), "stored key differs from the inserted key"
        assert len(np.unique(idx[mask])) == int(mask.sum()), "an index was handed out twice"
        after = om.as_dict()
        for k, v in before.items():
            assert after[k] == v, "an existing value was overwritten"
        fi, fm = om.find(keys)
        assert fm.all() and np.array_equal(kb[fi], keys), "find does not return the stored key"
        _check_permutation(om)
        er = keys[rng.integers(0, n, size=n // 3)]
        em = om.erase(er)
        seen = set()
        for p in range(len(er)):
            k = tuple(int(x) for x in er[p])
            assert bool(em[p]) == (k not in seen), "erase winner is not the first occurrence"
            seen.add(k)
        _check_permutation(om)
        assert om.size() + (om.capacity() - om.heap_top()) == om.capacity()


# ------------------------------------------------------------ closed forms
def pin_plain_map_closed_form(mutant=0):
    case = workloads.plain_map_case(seed=0)
    n = case.insert_keys.shape[0]
    om = oracle.OracleMap(3, case.capacity, [4], mutant=mutant)
    idx, mask = om.insert(case.insert_keys, [case.insert_values])
    # occupied cells after n uniform draws over M = 128^3 cells
    M = 128 ** 3
    q = (1.0 - 1.0 / M) ** n
    mean = M * (1.0 - q)
    var = M * (M - 1) * (1.0 - 2.0 / M) ** n + M * q - (M * q) ** 2
    unique = int(mask.sum())
    assert abs(unique - mean) <= 4.0 * math.sqrt(var), f"unique count {unique} vs {mean:.1f}"
    assert om.size() == unique
    fi, fm = om.find(case.query_keys)
    fresh = (case.query_keys >= 64).all(axis=1)
    assert not fm[fresh].any(), "a key from the disjoint fresh range was found"
    assert fm[~fresh].all(), "an inserted key was not found"
    em = om.erase(case.erase_keys)
    fi2, fm2 = om.find(case.query_keys)
    erased = {tuple(int(x) for x in k) for k in case.erase_keys}
    for p in range(len(case.query_keys)):
        k = tuple(int(x) for x in case.query_keys[p])
        assert bool(fm2[p]) == (bool(fm[p]) and k not in erased), "re-find after erase is wrong"
    assert om.size() == unique - int(em.sum())


def pin_growth(mutant=0):
    om = oracle.OracleMap(2, 4, [], mutant=mutant)
    keys = np.arange(18, dtype=np.int32).reshape(9, 2)
    _, m = om.activate(keys)
    assert m.all() and om.capacity() == 16, "x2 growth from 4 for 9 keys must give 16"
    om2 = oracle.OracleMap(2, 3, [], mutant=mutant)
    om2.activate(keys[:3])
    om2.activate(keys[3:4])   # 3 + 1 > 3 -> 6
    assert om2.capacity() == 6, "x2 growth from 3 for one more key must give 6"


def pin_erase_all_and_rehash(mutant=0):
    rng = np.random.default_rng(3)
    keys = rng.integers(-50, 50, size=(5000, 3)).astype(np.int32)
    vals = rng.random(5000, dtype=np.float32)
    om = oracle.OracleMap(3, 1 << 14, [4], mutant=mutant)
    om.insert(keys, [vals])
    d0 = om.as_dict()
    om.rehash(1 << 15)
    assert om.capacity() == 1 << 15 and om.as_dict() == d0, "rehash changed the dictionary"
    om.rehash(len(d0))
    assert om.as_dict() == d0, "rehash to the exact size changed the dictionary"
    m = om.erase(keys)
    assert om.size() == 0 and om.heap_top() == 0, "erase-all left entries"
    assert int(m.sum()) == len(d0)
    _check_permutation(om)


def pin_unique_reduction(mutant=0):
    pts = workloads.voxel_scene_points(n=200_000, seed=1)
    keys = oracle.quantize(pts, 0.05, mutant=mutant)
    om = oracle.OracleMap(3, len(keys), [], mutant=mutant)
    idx, mask = om.activate(keys)
    kb = om.key_buffer()
    got = kb[om.active_indices()]
    uniq, inverse = np.unique(keys, axis=0, return_inverse=True)
    inverse = inverse.reshape(-1)
    order = np.lexsort(got.T[::-1])
    assert np.array_equal(got[order], uniq), "activated key set differs from np.unique"
    fi, fm = om.find(keys)
    assert fm.all()
    # same unique label <=> same buffer index
    first_idx = np.full(len(uniq), -1, np.int64)
    first_idx[inverse[::-1]] = fi[::-1]
    assert np.array_equal(first_idx[inverse], fi), "find disagrees with the unique inverse"
    assert len(np.unique(fi)) == len(uniq)


def pin_quantize(mutant=0):
    rng = np.random.default_rng(11)
    pts = rng.normal(scale=3.0, size=(100_000, 3)).astype(np.float32)
    for s in (0.005, 0.01, 0.048, 0.05, 1.0):
        got = oracle.quantize(pts, s, mutant=mutant)
        want = np.floor(pts / np.float32(s)).astype(np.int32)
        assert np.array_equal(got, want), f"quantisation differs from numpy float32 at s={s}"
    with open(os.path.join(GOLDEN, "quantize_cases.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            p, s, k = ln.split()
            got = oracle.quantize(np.array([np.float32(p)], np.float32), np.float32(s), mutant=mutant)
            assert int(got[0]) == int(k), f"quantize({p}, {s}) = {got[0]}, hand value {k}"


ALL_PINS = [pin_bruteforce, pin_golden_trace, pin_invariants, pin_plain_map_closed_form,
            pin_growth, pin_erase_all_and_rehash, pin_unique_reduction, pin_quantize]
