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


# ------------------------------------------------------ double hash map (Sec. 6.2)
def pin_double_map(mutant=0, seeds=range(6)):
    """Against plain Python dicts on tiny frames: the distinct new keys in
    first-occurrence order, the global key set, and local value -> a global
    index that holds the same key."""
    for seed in seeds:
        rng = np.random.default_rng(500 + seed)
        local = oracle.OracleMap(3, 4, [4], mutant=mutant)
        glob = oracle.OracleMap(3, 4, [], mutant=mutant)
        global_keys = set()
        for frame in range(5):
            if frame % 2 == 1:
                local.clear()
            local_before = set(local.as_dict().keys())
            keys = rng.integers(-3, 3, size=(int(rng.integers(0, 30)), 3)).astype(np.int32)
            uk, li, gi = oracle.double_map_activate(local, glob, keys)
            want, seen = [], set(local_before)
            for k in _tuples(keys):
                if k not in seen:
                    seen.add(k)
                    want.append(k)
            assert _tuples(uk) == want, "distinct new keys differ from the first occurrences"
            global_keys |= set(want)
            assert set(glob.as_dict().keys()) == global_keys, "global key set differs from the union of frames"
            gkb = glob.key_buffer()
            lkb = local.key_buffer()
            lv = local.value_buffer(0).view(np.int32).reshape(-1)
            for i in local.active_indices():
                assert tuple(gkb[lv[i]]) == tuple(lkb[i]), "local value does not point at the same key in global"
            assert np.array_equal(lkb[li], uk) and np.array_equal(gkb[gi], uk)
            _check_permutation(local)
            _check_permutation(glob)


# ------------------------------------------------------ TSDF integration (Sec. 6.2)
ELL = 8
S = 1.0 / 64.0          # voxel edge (dyadic: every lattice coordinate is exact in float32)
MU = 4.0 / 64.0         # truncation
INTR = (100.0, 100.0, 32.0, 24.0)   # fx, fy, cx, cy for a 64 x 48 image


def _blocks(kx, ky, kz):
    g = np.stack(np.meshgrid(kx, ky, kz, indexing="ij"), axis=-1).reshape(-1, 3)
    return g.astype(np.int32)


def _tsdf_map(keys, mutant, f64=True, values=None):
    rb = (8 if f64 else 4) * ELL ** 3
    om = oracle.OracleMap(3, max(1, len(keys)), [rb, rb], mutant=mutant)
    dt = np.float64 if f64 else np.float32
    v = values if values is not None else (np.zeros((len(keys), ELL ** 3), dt), np.zeros((len(keys), ELL ** 3), dt))
    idx, mask = om.insert(keys, list(v))
    assert mask.all()
    return om, idx


def _voxels(om, idx):
    d = om.value_buffer(0).view(np.float64).reshape(-1, ELL ** 3)[idx]
    w = om.value_buffer(1).view(np.float64).reshape(-1, ELL ** 3)[idx]
    return d, w


def _lattice_world(keys):
    """[n, ell^3, 3] world positions of the voxel lattice points, x fastest."""
    v = np.stack(np.meshgrid(np.arange(ELL), np.arange(ELL), np.arange(ELL), indexing="ij"), axis=-1)
    v = v.transpose(2, 1, 0, 3).reshape(-1, 3)  # slot (vz * ell + vy) * ell + vx holds (vx, vy, vz)
    return (keys[:, None, :].astype(np.float64) * ELL + v[None]) * S


def pin_tsdf_plane_closed_form(mutant=0):
    """Fronto-parallel planes seen from the identity pose, all values dyadic:
    after frames at depths Z_j each voxel holds the batch weighted mean of
    Eq. (8) of clamp(Z_j - z, -mu, mu) over the frames with Z_j - z >= -mu,
    and its weight counts those frames."""
    keys = _blocks([-1, 0], [-1, 0], [7, 8])
    om, idx = _tsdf_map(keys, mutant)
    extr = np.hstack([np.eye(3), np.zeros((3, 1))])
    depths = [1.0, 1.0 + 2 * S, 1.0 - S, 1.0 + 3 * S]
    psi_sum = np.zeros((len(keys), ELL ** 3))
    w_sum = np.zeros((len(keys), ELL ** 3))
    z = _lattice_world(keys)[..., 2]
    for zd in depths:
        img = np.full((48, 64), zd, np.float32)
        oracle.tsdf_integrate(om, idx, img, INTR, extr, S, MU, 10.0, ell=ELL)
        sdf = zd - z
        upd = sdf >= -MU
        psi_sum += np.where(upd, np.minimum(sdf, MU), 0.0)
        w_sum += upd
    d, w = _voxels(om, idx)
    assert np.array_equal(w, w_sum), "weights differ from the count of updating frames"
    want = np.where(w_sum > 0, psi_sum / np.maximum(w_sum, 1), 0.0)
    assert np.allclose(d, want, rtol=0, atol=1e-12), "running mean differs from the batch mean of Eq. (8)"


def pin_tsdf_rotated_pose_and_shift(mutant=0):
    """A camera turned 90 degrees about y and moved, and the same scene moved
    by whole blocks with the camera: exact arithmetic (permutation rotation,
    dyadic translation) gives the closed form Z - zc, and the shifted copy
    gives bit-identical voxels."""
    R = np.array([[0.0, 0.0, -1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])   # world x -> camera z
    t = np.array([0.25, -0.125, -0.5])
    keys = _blocks([8, 9], [-1, 0], [-1, 0])
    zd = 0.5 + 3 * S + S / 2
    img = np.full((48, 64), zd, np.float32)
    img[:, 40:48] = 0.0                                    # a hole: no depth there
    om, idx = _tsdf_map(keys, mutant)
    oracle.tsdf_integrate(om, idx, img, INTR, np.hstack([R, t[:, None]]), S, MU, 10.0, ell=ELL)
    d, w = _voxels(om, idx)
    xw = _lattice_world(keys)
    xc = xw @ R.T + t
    uf = INTR[0] * xc[..., 0] / xc[..., 2] + INTR[2] + 0.5
    vf = INTR[1] * xc[..., 1] / xc[..., 2] + INTR[3] + 0.5
    u, v = np.floor(uf), np.floor(vf)
    sdf = zd - xc[..., 2]
    inside = (xc[..., 2] > 0) & (u >= 0) & (u < 64) & ~((u >= 40) & (u < 48)) & (v >= 0) & (v < 48) & (sdf >= -MU)
    # pixel decisions taken in float32 may differ from float64 within rounding of a pixel edge
    sure = (np.abs(uf - np.round(uf)) > 1e-4) & (np.abs(vf - np.round(vf)) > 1e-4)
    assert inside[sure].any() and (~inside[sure]).any()
    assert np.array_equal(w[sure], inside[sure].astype(np.float64)), "updated voxel set differs from the closed form"
    both = sure & inside
    assert np.allclose(d[both], np.minimum(sdf[both], MU), rtol=0, atol=1e-6), "values differ from Z - zc"
    shift = np.array([3, -2, 5], np.int32)                  # whole blocks
    om2, idx2 = _tsdf_map(keys + shift, mutant)
    t2 = t - R @ (shift.astype(np.float64) * ELL * S)
    oracle.tsdf_integrate(om2, idx2, img, INTR, np.hstack([R, t2[:, None]]), S, MU, 10.0, ell=ELL)
    d2, w2 = _voxels(om2, idx2)
    assert np.array_equal(d2, d) and np.array_equal(w2, w), "moving scene and camera together changed the voxels"


def pin_tsdf_skips(mutant=0):
    """Blocks behind the camera, outside the image, and far behind the
    surface are left alone."""
    keys = np.array([[0, 0, -4], [60, 0, 8], [0, 0, 20], [0, 0, 8]], np.int32)
    om, idx = _tsdf_map(keys, mutant)
    img = np.full((48, 64), 1.0, np.float32)
    oracle.tsdf_integrate(om, idx, img, INTR, np.hstack([np.eye(3), np.zeros((3, 1))]), S, MU, 10.0, ell=ELL)
    _, w = _voxels(om, idx)
    assert not w[:3].any(), "a voxel behind the camera, outside the image or far behind the surface was updated"
    assert w[3].any()


# ------------------------------------------------------ ray casting (Sec. 6.2)
def _plane_volume(z0, kx, ky, kz):
    keys = _blocks(kx, ky, kz)
    z = _lattice_world(keys)[..., 2]
    d = np.clip(z0 - z, -MU, MU).astype(np.float32)
    return keys, (d, np.ones_like(d))


def pin_raycast_plane_exact(mutant=0):
    """Identity pose, a volume holding d = Z0 - z on the lattice, samples on
    the lattice in z: every ray that stays inside the volume meets the
    surface at exactly Z0 (linear interpolation of a linear function)."""
    z0 = 1.0 + S / 4
    keys, vals = _plane_volume(z0, range(-4, 4), range(-4, 4), range(6, 10))
    om, _ = _tsdf_map(keys, mutant, f64=False, values=vals)
    extr = np.hstack([np.eye(3), np.zeros((3, 1))])
    t0 = 52 * S                                            # samples on the lattice in z
    n_steps = 26
    depth = oracle.tsdf_raycast(om, INTR, extr, 64, 48, S, t0, S, n_steps, ell=ELL, value_bytes=4)
    assert np.all(depth == z0), "plane depth differs from Z0"
    # rays of a camera looking away from the plane find nothing
    back = np.hstack([np.diag([1.0, -1.0, -1.0]), np.zeros((3, 1))])
    assert not oracle.tsdf_raycast(om, INTR, back, 64, 48, S, t0, S, n_steps, ell=ELL, value_bytes=4).any()


def pin_raycast_sphere(mutant=0):
    """A sphere's truncated signed distance on the lattice, seen from a
    rotated and translated camera, against the textbook ray-sphere
    intersection.  Each sample reads the nearest lattice point, at most
    sqrt(3)/2 voxels away, and the distance is 1-Lipschitz, so where the ray
    meets the surface at incidence cosine cos > 1/2 the hit depth is within
    (sqrt(3)/2) s / cos + step of the true one.  Rays that pass the sphere
    by more than two voxels return 0."""
    c = np.array([0.1, -0.05, 1.0])
    r = 0.25
    keys = _blocks(range(-6, 6), range(-6, 6), range(0, 12))
    xw = _lattice_world(keys)
    d = np.clip(np.linalg.norm(xw - c, axis=-1) - r, -MU, MU).astype(np.float32)
    om, _ = _tsdf_map(keys, mutant, f64=False, values=(d, np.ones_like(d)))
    ang = 0.3
    R = np.array([[math.cos(ang), 0, -math.sin(ang)], [0, 1, 0], [math.sin(ang), 0, math.cos(ang)]])
    cam = np.array([-0.2, 0.02, 0.05])                     # camera centre in the world
    t = -R @ cam
    step = S / 2
    n_steps = int(round((1.5 - 0.2) / step)) + 1
    depth = oracle.tsdf_raycast(om, INTR, np.hstack([R, t[:, None]]), 64, 48, S, 0.2, step, n_steps, ell=ELL,
                                value_bytes=4)
    py, px = np.mgrid[0:48, 0:64]
    dc = np.stack([(px - INTR[2]) / INTR[0], (py - INTR[3]) / INTR[1], np.ones_like(px, dtype=np.float64)], -1)
    dw = dc.reshape(-1, 3) @ R                              # R^T applied to each direction
    oc = cam - c
    a = np.einsum("ij,ij->i", dw, dw)
    b = 2 * dw @ oc
    disc = b * b - 4 * a * (oc @ oc - r * r)
    hit = disc > 0
    tt = np.where(hit, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), 0.0)
    normal = (cam + tt[:, None] * dw - c) / r
    cos = np.abs(np.einsum("ij,ij->i", dw / np.sqrt(a)[:, None], normal))
    steep = hit & (cos > 0.5)
    assert steep.sum() > 1000
    bound = (math.sqrt(3) / 2) * S / cos[steep] + step
    assert np.all(np.abs(depth[steep] - tt[steep]) <= bound), "hit depth differs from the ray-sphere intersection"
    miss_dist = np.sqrt(np.maximum(oc @ oc - b * b / (4 * a), 0))
    far = ~hit & (miss_dist > r + 2 * S)
    assert far.sum() > 100 and not depth[far].any(), "a ray that misses the sphere returned a depth"


ALL_PINS += [pin_double_map, pin_tsdf_plane_closed_form, pin_tsdf_rotated_pose_and_shift, pin_tsdf_skips,
             pin_raycast_plane_exact, pin_raycast_sphere]


def pin_depth_to_block_keys(mutant=0):
    """Unprojection closed forms: identity pose over a fronto-parallel plane
    (every key's z is floor(Z0 / edge), x and y follow the pixel ray), and a
    camera turned to look along world +x from a dyadic position (key x is
    floor((pos_x + D) / edge)); pixels without depth or beyond depth_max
    are dropped and the rest keep pixel order."""
    edge = ELL * S
    z0 = 1.0 + S / 2
    img = np.full((48, 64), z0, np.float32)
    img[5, 7] = 0.0
    img[6, 9] = 20.0
    keys = oracle.depth_to_block_keys(img, INTR, np.hstack([np.eye(3), np.zeros((3, 1))]), edge, 10.0,
                                      mutant=mutant)
    assert keys.shape == (48 * 64 - 2, 3), "pixels without depth were not dropped"
    assert np.all(keys[:, 2] == math.floor(z0 / edge))
    py, px = np.mgrid[0:48, 0:64]
    valid = (img > 0) & (img <= 10.0)
    xs = (px[valid] - INTR[2]) / INTR[0] * z0 / edge
    ys = (py[valid] - INTR[3]) / INTR[1] * z0 / edge
    sure = (np.abs(xs - np.round(xs)) > 1e-4) & (np.abs(ys - np.round(ys)) > 1e-4)
    assert np.array_equal(keys[sure, 0], np.floor(xs[sure]).astype(np.int32)), "x keys differ from the pixel rays"
    assert np.array_equal(keys[sure, 1], np.floor(ys[sure]).astype(np.int32)), "y keys differ from the pixel rays (order?)"
    R = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0]])   # camera z = world x, camera y = -world z
    pos = np.array([2.0, 1.5, 0.75])
    d = np.random.default_rng(3).uniform(0.5, 3.0, size=(48, 64)).astype(np.float32)
    k2 = oracle.depth_to_block_keys(d, INTR, np.hstack([R, (-R @ pos)[:, None]]), edge, 10.0, mutant=mutant)
    want = np.floor((pos[0] + d.reshape(-1).astype(np.float64)) / edge)
    near = np.abs((pos[0] + d.reshape(-1)) / edge - np.round((pos[0] + d.reshape(-1)) / edge)) < 1e-4
    assert np.array_equal(k2[~near, 0], want[~near].astype(np.int32)), "key x differs from floor((pos_x + D) / edge)"


ALL_PINS.append(pin_depth_to_block_keys)
