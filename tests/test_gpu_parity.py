"""CUDA map vs the CPU oracle, element by element, through the C ABI.

Bar: bit-exact for masks and stored keys, byte-exact for value rows, modulo
the buffer-index permutation the paper leaves unspecified (see parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_heap_permutation, assert_op_parity, assert_same_map, value_rows_for
from paper_2110_00511_gb300 import ash, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()
    torch.cuda.init()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def tuning(**kw):
    t = ash.default_tuning()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def _rows(a, rb):
    return np.ascontiguousarray(a).view(np.uint8).reshape(-1, rb)


# ------------------------------------------------------------ plain map
def test_plain_map_sequence():
    """Insert 100k keys in [-64,64)^3 with float values, find half-hit
    queries, erase 25%, re-find (the plain single-map workload)."""
    case = workloads.plain_map_case(seed=0)
    hm = ash.HashMap(3, case.capacity, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, case.capacity, [4])
    k = dev(case.insert_keys)
    gi, gm = hm.insert(k, [dev(case.insert_values)])
    oi, omask = om.insert(case.insert_keys, [case.insert_values])
    assert_op_parity(hm, case.insert_keys, gi, gm, oi, omask)
    assert_same_map(hm, om)
    gi, gm = hm.find(dev(case.query_keys))
    oi, omask = om.find(case.query_keys)
    assert_op_parity(hm, case.query_keys, gi, gm, oi, omask, check_distinct=False)
    hit = gm.cpu().numpy()
    assert np.array_equal(value_rows_for(hm, 0, gi[gm]), om.value_buffer(0)[oi[hit]])
    ge = hm.erase(dev(case.erase_keys))
    oe = om.erase(case.erase_keys)
    assert np.array_equal(ge.cpu().numpy(), oe)
    gi, gm = hm.find(dev(case.query_keys))
    oi, omask = om.find(case.query_keys)
    assert_op_parity(hm, case.query_keys, gi, gm, oi, omask, check_distinct=False)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


# ------------------------------------------------------ dims x bucket sizes
@pytest.mark.parametrize("d", range(1, 9))
@pytest.mark.parametrize("S", [4, 8, 16])
def test_dims_and_bucket_sizes(d, S):
    rng = np.random.default_rng(100 * d + S)
    n = 5003  # ragged: not a multiple of any block size
    keys = rng.integers(-6, 6, size=(n, d)).astype(np.int32)
    vals = rng.integers(-2**31, 2**31 - 1, size=n, dtype=np.int64).astype(np.int32)
    hm = ash.HashMap(d, 4096, [(1,)], [torch.int32], tuning=tuning(slots_per_bucket=S))
    om = oracle.OracleMap(d, 4096, [4])
    gi, gm = hm.insert(dev(keys), [dev(vals)])
    oi, omask = om.insert(keys, [vals])
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    gi, gm = hm.activate(dev(keys[::-1].copy()))
    oi, omask = om.activate(keys[::-1].copy())
    assert_op_parity(hm, keys[::-1].copy(), gi, gm, oi, omask)
    er = keys[rng.integers(0, n, size=n // 2)]
    assert np.array_equal(hm.erase(dev(er)).cpu().numpy(), om.erase(er))
    q = rng.integers(-7, 7, size=(n, d)).astype(np.int32)
    gi, gm = hm.find(dev(q))
    oi, omask = om.find(q)
    assert_op_parity(hm, q, gi, gm, oi, omask, check_distinct=False)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


# ------------------------------------------------------------ race stress
@pytest.mark.parametrize("claim_mode", [1, 2])
def test_duplicate_race_stress(claim_mode):
    """1M keys drawn from 1000 distinct triples (the heavy-duplicate setting
    where Sec. 4.4.2 reports torn-copy races): exactly one winner per key, the
    first occurrence, with its own value; repeated on fresh maps, under both
    claim protocols (bucket load first; preferred-slot CAS first)."""
    rng = np.random.default_rng(5)
    distinct = rng.integers(-2**30, 2**30, size=(1000, 3)).astype(np.int32)
    for rep in range(5):
        keys = distinct[rng.integers(0, 1000, size=1_000_000)]
        vals = np.arange(1_000_000, dtype=np.int32)
        hm = ash.HashMap(3, 1_000_000, [(1,)], [torch.int32], tuning=tuning(claim_mode=claim_mode))
        gi, gm = hm.insert(dev(keys), [dev(vals)])
        _, first = np.unique(keys, axis=0, return_index=True)
        want = np.zeros(len(keys), bool)
        want[first] = True
        assert np.array_equal(gm.cpu().numpy(), want), f"winners are not the first occurrences (rep {rep})"
        stored = hm.value_buffer(0)[gi[gm].long()].cpu().numpy().ravel()
        assert np.array_equal(np.sort(stored), np.sort(first.astype(np.int32)))
        kb = hm.key_buffer().cpu().numpy()
        assert np.array_equal(kb[gi[gm].cpu().numpy()], keys[gm.cpu().numpy()])
        assert hm.size() == 1000


def test_erase_duplicates_first_occurrence():
    rng = np.random.default_rng(6)
    keys = rng.integers(-20, 20, size=(50_000, 3)).astype(np.int32)
    hm = ash.HashMap(3, 100_000)
    om = oracle.OracleMap(3, 100_000)
    hm.activate(dev(keys))
    om.activate(keys)
    er = rng.integers(-25, 25, size=(80_000, 3)).astype(np.int32)
    assert np.array_equal(hm.erase(dev(er)).cpu().numpy(), om.erase(er))
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


# --------------------------------------------------------- growth / rehash
def test_auto_growth_matches_oracle():
    rng = np.random.default_rng(7)
    hm = ash.HashMap(3, 1000, [(2,)], [torch.float32])
    om = oracle.OracleMap(3, 1000, [8])
    for step in range(6):
        n = int(rng.integers(500, 4000))
        keys = rng.integers(-2**20, 2**20, size=(n, 3)).astype(np.int32)
        vals = rng.random((n, 2), dtype=np.float32)
        gi, gm = hm.insert(dev(keys), [dev(vals)])
        oi, omask = om.insert(keys, [vals])
        assert_op_parity(hm, keys, gi, gm, oi, omask)
        assert hm.capacity() == om.capacity()
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


def test_rehash_preserves_indices_and_compacts():
    rng = np.random.default_rng(8)
    keys = rng.integers(-500, 500, size=(30_000, 3)).astype(np.int32)
    vals = rng.random(30_000, dtype=np.float32)
    hm = ash.HashMap(3, 40_000, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, 40_000, [4])
    hm.insert(dev(keys), [dev(vals)])
    om.insert(keys, [vals])
    hm.erase(dev(keys[:5000]))
    om.erase(keys[:5000])
    q = dev(keys)
    before_i, before_m = hm.find(q)
    hm.rehash(100_000)
    om.rehash(100_000)
    after_i, after_m = hm.find(q)
    assert torch.equal(before_m, after_m) and torch.equal(before_i, after_i), "growth must keep buffer indices"
    assert_same_map(hm, om)
    assert_heap_permutation(hm)
    live = om.size()
    hm.rehash(live)
    om.rehash(live)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)
    gi, gm = hm.find(q)
    oi, omask = om.find(keys)
    assert_op_parity(hm, keys, gi, gm, oi, omask, check_distinct=False)
    # inserting after a compaction keeps working
    more = rng.integers(600, 700, size=(1000, 3)).astype(np.int32)
    mv = rng.random(1000, dtype=np.float32)
    gi, gm = hm.insert(dev(more), [dev(mv)])
    oi, omask = om.insert(more, [mv])
    assert_op_parity(hm, more, gi, gm, oi, omask)
    assert_same_map(hm, om)


def test_reserve_async_keeps_map_and_indices():
    """Growth with no host synchronisation (the live count stays on the
    device) keeps every key, value and buffer index; later ops still match."""
    rng = np.random.default_rng(21)
    keys = rng.integers(-300, 300, size=(40_000, 3)).astype(np.int32)
    vals = rng.random(40_000, dtype=np.float32)
    hm = ash.HashMap(3, 50_000, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, 50_000, [4])
    hm.insert(dev(keys), [dev(vals)])
    om.insert(keys, [vals])
    hm.erase(dev(keys[:7000]))
    om.erase(keys[:7000])
    q = dev(keys)
    bi, bm = hm.find(q)
    hm.reserve_async(200_000)
    ai, am = hm.find(q)  # same stream, after the growth
    assert torch.equal(bi, ai) and torch.equal(bm, am)
    assert hm.capacity() == 200_000
    om.rehash(200_000)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)
    more = rng.integers(300, 400, size=(30_000, 3)).astype(np.int32)
    mv = rng.random(30_000, dtype=np.float32)
    gi, gm = hm.insert(dev(more), [dev(mv)])
    oi, omask = om.insert(more, [mv])
    assert_op_parity(hm, more, gi, gm, oi, omask)
    assert_same_map(hm, om)


def test_clear_and_reuse():
    rng = np.random.default_rng(9)
    keys = rng.integers(-50, 50, size=(20_000, 2)).astype(np.int32)
    hm = ash.HashMap(2, 30_000)
    om = oracle.OracleMap(2, 30_000)
    for _ in range(3):
        gi, gm = hm.activate(dev(keys))
        oi, omask = om.activate(keys)
        assert_op_parity(hm, keys, gi, gm, oi, omask)
        hm.clear()
        om.clear()
        assert hm.size() == 0
        assert_heap_permutation(hm)


# ----------------------------------------------------------------- values
def test_tsdf_block_values():
    """Voxel-block values (Sec. 6.2 setup): tsdf float32[8,8,8] and weight
    float16[8,8,8] rows, copied by the warp-per-row scatter kernel."""
    rng = np.random.default_rng(10)
    n = 20_000
    keys = rng.integers(-40, 40, size=(n, 3)).astype(np.int32)
    tsdf = rng.standard_normal((n, 8, 8, 8)).astype(np.float32)
    w = rng.standard_normal((n, 8, 8, 8)).astype(np.float16)
    hm = ash.HashMap(3, 1 << 15, [(8, 8, 8), (8, 8, 8)], [torch.float32, torch.float16])
    om = oracle.OracleMap(3, 1 << 15, [2048, 1024])
    gi, gm = hm.insert(dev(keys), [dev(tsdf), dev(w)])
    oi, omask = om.insert(keys, [tsdf, w])
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert_same_map(hm, om)


def test_value_dtypes_and_odd_row_sizes():
    rng = np.random.default_rng(11)
    n = 9_001
    keys = rng.integers(-30, 30, size=(n, 4)).astype(np.int32)
    v0 = rng.integers(0, 255, size=(n, 3)).astype(np.uint8)          # 3-byte rows
    v1 = rng.standard_normal((n, 5)).astype(np.float16)              # 10-byte rows
    v2 = rng.integers(-2**62, 2**62, size=(n, 1), dtype=np.int64)     # 8-byte rows
    v3 = rng.standard_normal((n, 3)).astype(np.float64)              # 24-byte rows
    hm = ash.HashMap(4, 1 << 14, [(3,), (5,), (1,), (3,)], [torch.uint8, torch.float16, torch.int64, torch.float64])
    om = oracle.OracleMap(4, 1 << 14, [3, 10, 8, 24])
    gi, gm = hm.insert(dev(keys), [dev(v0), dev(v1), dev(v2), dev(v3)])
    oi, omask = om.insert(keys, [v0, v1, v2, v3])
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert_same_map(hm, om)


def test_bfloat16_values():
    rng = np.random.default_rng(12)
    n = 4_000
    keys = rng.integers(-20, 20, size=(n, 3)).astype(np.int32)
    v = torch.randn(n, 4, dtype=torch.bfloat16, generator=torch.Generator().manual_seed(0))
    hm = ash.HashMap(3, 1 << 13, [(4,)], [torch.bfloat16])
    om = oracle.OracleMap(3, 1 << 13, [8])
    gi, gm = hm.insert(dev(keys), [v.cuda()])
    oi, omask = om.insert(keys, [v.view(torch.int16).numpy()])
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert_same_map(hm, om)


# ------------------------------------------------------------ quantisation
def test_quantize_bit_exact():
    rng = np.random.default_rng(13)
    pts = rng.normal(scale=5.0, size=(1_000_003, 3)).astype(np.float32)
    pts[:5] = np.array([[0.5, -0.5, -0.0], [-1e-7, 9.999, 2.5], [-2.5, 0.0025, -0.0025],
                        [1.0, -1.0, 0.1], [-0.1, 0.0049999, 0.005]], np.float32)
    for cell in (0.005, 0.048, 0.05, 0.25, 1.0):
        g = ash.ash_quantize(dev(pts), cell).cpu().numpy()
        o = oracle.quantize(pts, cell)
        assert np.array_equal(g, o), f"quantisation differs at cell {cell}"
    # unaligned view takes the scalar path
    flat = dev(pts).reshape(-1)[1:]
    g = ash.ash_quantize(flat, 0.01).cpu().numpy()
    assert np.array_equal(g, oracle.quantize(pts.reshape(-1)[1:], 0.01))


# ----------------------------------------------------------- voxelization
def test_voxelization_scene():
    """Point-cloud voxelization (Sec. 6.1): 4M points, 5 mm voxels; insert
    keys with point-index values, find every point's voxel, list the unique
    voxels.  Compared with the oracle and with np.unique."""
    pts = workloads.voxel_scene_points(n=4_000_000, seed=0)
    n = pts.shape[0]
    okeys = oracle.quantize(pts, 0.005)
    gkeys = ash.ash_quantize(dev(pts), 0.005)
    assert np.array_equal(gkeys.cpu().numpy(), okeys)
    vals = np.arange(n, dtype=np.int32)
    hm = ash.HashMap(3, n, [(1,)], [torch.int32])
    om = oracle.OracleMap(3, n, [4])
    gi, gm = hm.insert(gkeys.reshape(n, 3), [dev(vals)])
    oi, omask = om.insert(okeys, [vals])
    assert_op_parity(hm, okeys, gi, gm, oi, omask)
    fi, fm = hm.find(gkeys.reshape(n, 3))
    ofi, ofm = om.find(okeys)
    assert_op_parity(hm, okeys, fi, fm, ofi, ofm, check_distinct=False)
    assert_same_map(hm, om)
    act = hm.active_indices()
    uniq = hm.gather_keys(act).cpu().numpy()
    want = np.unique(okeys, axis=0)
    assert np.array_equal(uniq[np.lexsort(uniq.T[::-1])], want)


@pytest.mark.parametrize("voxel", [0.01, 0.02, 0.05])
def test_voxelization_voxel_sizes_full_size(voxel):
    """The voxelization step at the paper's larger voxel sizes (Sec. 6.1), on
    the full 4M-point scene, where many points share a voxel (about 15 per
    voxel at 50 mm): the activated key set is np.unique of the keys, the
    winners are exactly the first occurrences, every point finds the index
    its voxel's first point received, and at 50 mm the insert with point-id
    values matches the oracle entry for entry."""
    pts = workloads.voxel_scene_points(n=4_000_000, seed=0)
    n = pts.shape[0]
    okeys = oracle.quantize(pts, voxel)
    gkeys = ash.ash_quantize(dev(pts), voxel).reshape(n, 3)
    assert np.array_equal(gkeys.cpu().numpy(), okeys)
    want, first, inverse = np.unique(okeys, axis=0, return_index=True, return_inverse=True)
    inverse = inverse.reshape(-1)
    hm = ash.HashMap(3, n, [(1,)], [torch.int32])
    gi, gm = hm.insert(gkeys, [torch.arange(n, dtype=torch.int32, device="cuda")])
    wmask = np.zeros(n, bool)
    wmask[first] = True
    assert np.array_equal(gm.cpu().numpy(), wmask)
    assert hm.size() == len(want)
    act = hm.active_indices()
    uniq = hm.gather_keys(act).cpu().numpy()
    assert np.array_equal(uniq[np.lexsort(uniq.T[::-1])], want)
    fi, fm = hm.find(gkeys)
    assert bool(fm.all())
    gi_np = gi.cpu().numpy()
    assert np.array_equal(fi.cpu().numpy(), gi_np[first[inverse]])
    # the stored value of each voxel is its first point's id
    v = hm.value_buffer(0)[fi.long()].reshape(-1).cpu().numpy()
    assert np.array_equal(v, first[inverse].astype(np.int32))
    if voxel == 0.05:
        om = oracle.OracleMap(3, n, [4])
        oi, omask = om.insert(okeys, [np.arange(n, dtype=np.int32)])
        assert_op_parity(hm, okeys, gi, gm, oi, omask)
        assert_same_map(hm, om)
    assert_heap_permutation(hm)


@pytest.mark.parametrize("rho", [0.1, 0.5, 1.0])
def test_uniqueness_sweep_1e6(rho):
    keys = workloads.uniform_keys(1_000_000, rho, seed=3)
    hm = ash.HashMap(3, len(keys))
    om = oracle.OracleMap(3, len(keys))
    gi, gm = hm.activate(dev(keys))
    oi, omask = om.activate(keys)
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    fi, fm = hm.find(dev(keys))
    ofi, ofm = om.find(keys)
    assert_op_parity(hm, keys, fi, fm, ofi, ofm, check_distinct=False)
    assert hm.size() == om.size()


def test_uniqueness_sweep_1e7_properties():
    """The full-size sweep point timed by the bench (10^7 keys): properties
    that hold at any size, checked against np.unique rather than the oracle:
    winners are exactly the first occurrences, and every position finds the
    index its key's first occurrence received."""
    keys = workloads.uniform_keys(10_000_000, 0.5, seed=4)
    hm = ash.HashMap(3, len(keys))
    gi, gm = hm.activate(dev(keys))
    _, first, inverse = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    inverse = inverse.reshape(-1)
    want = np.zeros(len(keys), bool)
    want[first] = True
    assert np.array_equal(gm.cpu().numpy(), want)
    fi, fm = hm.find(dev(keys))
    assert bool(fm.all())
    gi_np = gi.cpu().numpy()
    assert np.array_equal(fi.cpu().numpy(), gi_np[first[inverse]])
    kb = hm.key_buffer()
    assert torch.equal(kb[fi.long()], dev(keys))
    assert hm.size() == len(first)
    assert_heap_permutation(hm)


# --------------------------------------------------------------- TSDF frames
def test_tsdf_frames_and_neighbourhood():
    """Voxel-block activation over synthetic depth frames (Sec. 6.2, reduced
    to 6 frames at 1/4 resolution), then the 27-neighbourhood find of every
    active block (the radius search of Sec. 6.2)."""
    hm = ash.HashMap(3, 1 << 16)
    om = oracle.OracleMap(3, 1 << 16)
    for keys in workloads.tsdf_block_frames(n_frames=6, seed=1, stride=4):
        gi, gm = hm.activate(dev(keys))
        oi, omask = om.activate(keys)
        assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert_same_map(hm, om)
    act = hm.active_indices()
    blocks = hm.gather_keys(act).cpu().numpy()
    offs = workloads.radius_offsets(1)
    q = (blocks[:, None, :] + offs[None, :, :]).reshape(-1, 3).astype(np.int32)
    gi, gm = hm.find(dev(q))
    oi, omask = om.find(q)
    assert_op_parity(hm, q, gi, gm, oi, omask, check_distinct=False)
    assert gm.reshape(-1, 27)[:, 13].all(), "every block must find itself"


# ------------------------------------------------------------------ edges
def test_edge_cases():
    hm = ash.HashMap(3, 64, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, 64, [4])
    empty = torch.empty((0, 3), dtype=torch.int32, device="cuda")
    gi, gm = hm.insert(empty, [torch.empty(0, device="cuda")])
    assert gi.numel() == 0 and hm.size() == 0
    gi, gm = hm.find(empty)
    assert gm.numel() == 0
    assert hm.erase(empty).numel() == 0
    gi, gm = hm.find(dev(np.zeros((5, 3), np.int32)))
    assert not gm.any() and (gi == -1).all()
    assert not hm.erase(dev(np.zeros((5, 3), np.int32))).any()
    ext = np.array([[-2**31, 2**31 - 1, 0], [2**31 - 1, -2**31, -1], [0, 0, 0], [-1, -1, -1],
                    [-2**31, -2**31, -2**31], [2**31 - 1] * 3, [0, 0, 0]], np.int32)
    v = np.arange(len(ext), dtype=np.float32)
    gi, gm = hm.insert(dev(ext), [dev(v)])
    oi, omask = om.insert(ext, [v])
    assert_op_parity(hm, ext, gi, gm, oi, omask)
    assert_same_map(hm, om)
    for n in (1, 31, 33, 255, 257, 1025):
        rng = np.random.default_rng(n)
        k = rng.integers(-3, 3, size=(n, 3)).astype(np.int32)
        vv = rng.random(n, dtype=np.float32)
        gi, gm = hm.insert(dev(k), [dev(vv)])
        oi, omask = om.insert(k, [vv])
        assert_op_parity(hm, k, gi, gm, oi, omask)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


@pytest.mark.parametrize("field,value", [("claim_mode", 3), ("claim_mode", -1), ("commit_keys_per_thread", 3),
                                         ("keys_per_thread", 0), ("find_keys_per_thread", 5),
                                         ("partition_keys", 3), ("partition_keys", -1)])
def test_tuning_validation(field, value):
    """Out-of-range tuning fields are refused at create and at set_tuning,
    and a refused set_tuning leaves the map's tuning as it was."""
    with pytest.raises(ash.AshError) as e:
        ash.HashMap(3, 64, tuning=tuning(**{field: value}))
    assert e.value.status == ash.ASH_ERR_INVALID
    hm = ash.HashMap(3, 64)
    before = hm.tuning().as_dict()
    with pytest.raises(ash.AshError) as e:
        hm.set_tuning(tuning(**{field: value}))
    assert e.value.status == ash.ASH_ERR_INVALID
    assert hm.tuning().as_dict() == before


def test_capacity_error_without_growth():
    t = tuning(auto_grow=0)
    hm = ash.HashMap(3, 100, tuning=t)
    keys = dev(np.arange(600, dtype=np.int32).reshape(200, 3))
    gi, gm = hm.activate(keys)
    with pytest.raises(ash.AshError) as e:
        hm.sync_status()
    assert e.value.status == ash.ASH_ERR_CAPACITY
    assert int(gm.sum()) == 100 and hm.size() == 100
    assert (gi[~gm] == -1).all()
    assert_heap_permutation(hm)
    hm.sync_status()  # status was cleared


def test_table_full_reported_not_trapped():
    t = tuning(max_probes=1, slots_per_bucket=4, slots_per_capacity=1.05, auto_grow=0)
    hm = ash.HashMap(2, 4096, tuning=t)
    keys = dev(np.random.default_rng(1).integers(-2**20, 2**20, size=(4096, 2)).astype(np.int32))
    gi, gm = hm.activate(keys)
    with pytest.raises(ash.AshError) as e:
        hm.sync_status()
    assert e.value.status == ash.ASH_ERR_TABLE_FULL
    fi, fm = hm.find(keys)
    assert torch.equal(fm, gm), "keys that failed must not be findable; inserted ones must be"
    assert_heap_permutation(hm)


def test_churn_with_tombstones():
    """Insert/erase cycles on a small table: tombstones accumulate and the
    used-slot bound triggers table rebuilds; results stay identical."""
    rng = np.random.default_rng(14)
    hm = ash.HashMap(3, 1024, [(1,)], [torch.int32], tuning=tuning(slots_per_bucket=4))
    om = oracle.OracleMap(3, 1024, [4])
    for r in range(40):
        k = rng.integers(-15, 15, size=(700, 3)).astype(np.int32)
        v = rng.integers(0, 1000, size=700).astype(np.int32)
        gi, gm = hm.insert(dev(k), [dev(v)])
        oi, omask = om.insert(k, [v])
        assert_op_parity(hm, k, gi, gm, oi, omask)
        e = rng.integers(-15, 15, size=(900, 3)).astype(np.int32)
        assert np.array_equal(hm.erase(dev(e)).cpu().numpy(), om.erase(e))
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


@pytest.mark.parametrize("S", [4, 8])
def test_claim_protocols_mixed_on_dense_buckets(S):
    """Both claim protocols on one map with dense buckets (1.1 slots per unit
    of capacity) under insert/erase churn, the protocol switching between
    calls: erase must leave a tombstone where another live key of the bucket
    prefers the freed slot, or a later preferred-slot CAS would store a second
    copy of that key.  Checked against the oracle after every call."""
    rng = np.random.default_rng(40 + S)
    t = tuning(slots_per_bucket=S, slots_per_capacity=1.1)
    hm = ash.HashMap(3, 6000, [(1,)], [torch.int32], tuning=t)
    om = oracle.OracleMap(3, 6000, [4])
    for r in range(30):
        tt = hm.tuning()
        tt.claim_mode = int(rng.integers(0, 3))
        hm.set_tuning(tt)
        k = rng.integers(-11, 11, size=(2500, 3)).astype(np.int32)
        v = rng.integers(0, 1 << 20, size=2500).astype(np.int32)
        gi, gm = hm.insert(dev(k), [dev(v)])
        oi, omask = om.insert(k, [v])
        assert_op_parity(hm, k, gi, gm, oi, omask)
        e = rng.integers(-11, 11, size=(1500, 3)).astype(np.int32)
        assert np.array_equal(hm.erase(dev(e)).cpu().numpy(), om.erase(e))
        f = rng.integers(-12, 12, size=(3000, 3)).astype(np.int32)
        fi, fm = hm.find(dev(f))
        ofi, ofm = om.find(f)
        assert_op_parity(hm, f, fi, fm, ofi, ofm, check_distinct=False)
        assert hm.size() == om.size()
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


def test_side_stream_and_gather():
    rng = np.random.default_rng(15)
    keys = rng.integers(-100, 100, size=(50_000, 3)).astype(np.int32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        hm = ash.HashMap(3, 60_000)
        gi, gm = hm.activate(dev(keys))
        g = hm.gather_keys(gi[gm])
    s.synchronize()
    assert np.array_equal(g.cpu().numpy(), keys[gm.cpu().numpy()])
    neg = hm.gather_keys(torch.tensor([-1, -5], dtype=torch.int32, device="cuda"))
    assert (neg == 0).all()


def test_torch_allocator_hook():
    ash.use_torch_allocator(True)
    try:
        rng = np.random.default_rng(16)
        keys = rng.integers(-100, 100, size=(30_000, 3)).astype(np.int32)
        hm = ash.HashMap(3, 1000)
        om = oracle.OracleMap(3, 1000)
        gi, gm = hm.activate(dev(keys))
        oi, omask = om.activate(keys)
        assert_op_parity(hm, keys, gi, gm, oi, omask)
        assert_same_map(hm, om)
        del hm
    finally:
        ash.use_torch_allocator(False)


# ------------------------------------------------------ neighbours / export
@pytest.mark.parametrize("d,radius", [(3, 1), (3, 2), (2, 1), (4, 1), (3, 0)])
def test_find_neighbors_matches_materialised_queries(d, radius):
    """Radius neighbour query (Sec. 6.2): the fused kernel equals the oracle's
    find over the materialised keys q + offset, offsets row-major."""
    rng = np.random.default_rng(31 + d + radius)
    keys = rng.integers(-20, 20, size=(6000, d)).astype(np.int32)
    hm = ash.HashMap(d, 8192)
    om = oracle.OracleMap(d, 8192)
    hm.activate(dev(keys))
    om.activate(keys)
    q = rng.integers(-22, 22, size=(1001, d)).astype(np.int32)
    q[:3] = np.array([[2**31 - 1] * d, [-2**31] * d, [0] * d], np.int32)  # int32 wrap-around at the edges
    gi, gm = hm.find_neighbors(dev(q), radius)
    offs = workloads.radius_offsets(radius, d)
    mq = (q[:, None, :].astype(np.int64) + offs[None, :, :]).astype(np.int64)
    mq = ((mq + 2**31) % 2**32 - 2**31).astype(np.int32).reshape(-1, d)
    oi, omask = om.find(mq)
    assert gi.shape == (len(q), len(offs))
    assert_op_parity(hm, mq, gi.reshape(-1), gm.reshape(-1), oi, omask, check_distinct=False)


def test_gather_values_and_export_roundtrip():
    rng = np.random.default_rng(41)
    keys = rng.integers(-100, 100, size=(20_000, 3)).astype(np.int32)
    v0 = rng.standard_normal((20_000, 8, 8, 8)).astype(np.float32)
    v1 = rng.integers(0, 255, size=(20_000, 3)).astype(np.uint8)
    hm = ash.HashMap(3, 1 << 15, [(8, 8, 8), (3,)], [torch.float32, torch.uint8])
    om = oracle.OracleMap(3, 1 << 15, [2048, 3])
    hm.insert(dev(keys), [dev(v0), dev(v1)])
    om.insert(keys, [v0, v1])
    act = hm.active_indices()
    g0 = hm.gather_values(act, 0)
    assert torch.equal(g0, hm.value_buffer(0)[act.long()])
    bad = hm.gather_values(torch.tensor([-1, 1 << 20], dtype=torch.int32, device="cuda"), 1)
    assert (bad == 0).all()
    state = hm.export()
    hm2 = ash.HashMap.from_export(state)
    assert_same_map(hm2, om)


def test_async_listing_and_count_gathers():
    """Listing with the live count left on the device, and gathers bounded by
    that device count, equal the synchronising forms."""
    rng = np.random.default_rng(51)
    keys = rng.integers(-60, 60, size=(50_000, 3)).astype(np.int32)
    vals = rng.random(50_000, dtype=np.float32)
    hm = ash.HashMap(3, 60_000, [(1,)], [torch.float32])
    hm.insert(dev(keys), [dev(vals)])
    hm.erase(dev(keys[:9000]))
    act_sync = hm.active_indices()
    act, cnt = hm.active_indices_async()
    n = int(cnt.item())
    assert n == act_sync.numel() == hm.size()
    assert torch.equal(torch.sort(act[:n]).values, torch.sort(act_sync).values)
    g = hm.gather_keys_count(act, cnt)
    assert torch.equal(g[:n], hm.gather_keys(act[:n]))
    out = torch.full((act.numel(), 1), -1.0, device="cuda")
    from paper_2110_00511_gb300.ash import lib, _ptr, _stream, _check
    _check(lib().ash_gather_values_count(hm.handle, 0, _ptr(act), act.numel(), _ptr(cnt), _ptr(out), _stream()))
    assert torch.equal(out[:n], hm.gather_values(act[:n]))
    assert bool((out[n:] == -1.0).all()), "rows past the device count must not be written"


def test_set_intersection_with_a_hash_set():
    """Set intersection through a hash set (no value buffers, Sec. 4.7):
    activate A, find B; B's hits are exactly the rows of B that occur in A."""
    rng = np.random.default_rng(61)
    a = rng.integers(-50, 50, size=(200_000, 3)).astype(np.int32)
    b = rng.integers(-60, 60, size=(300_001, 3)).astype(np.int32)
    hs = ash.HashMap(3, len(a))
    om = oracle.OracleMap(3, len(a))
    hs.activate(dev(a))
    om.activate(a)
    fi, fm = hs.find(dev(b))
    ofi, ofm = om.find(b)
    assert_op_parity(hs, b, fi, fm, ofi, ofm, check_distinct=False)
    pack = lambda x: (x.astype(np.int64) + 64) @ np.array([1 << 16, 1 << 8, 1], np.int64)  # noqa: E731
    assert np.array_equal(fm.cpu().numpy().astype(bool), np.isin(pack(b), pack(a)))


@pytest.mark.parametrize("table", ["radius1", "cube", "ring", "random"])
def test_find_offsets_tables(table):
    """Neighbour tables (1-radius, 1-cube, 1-ring, and an arbitrary table with
    extreme offsets) equal the oracle's find over the materialised keys."""
    d = 3
    rng = np.random.default_rng(71)
    keys = rng.integers(-16, 16, size=(7000, d)).astype(np.int32)
    hm = ash.HashMap(d, 8192)
    om = oracle.OracleMap(d, 8192)
    hm.activate(dev(keys))
    om.activate(keys)
    offs = {"radius1": workloads.radius_offsets(1, d), "cube": workloads.cube_offsets(d),
            "ring": workloads.ring_offsets(d),
            "random": np.concatenate([rng.integers(-3, 4, size=(47, d)),
                                      np.array([[2**31 - 1, 0, 0], [-2**31, 5, -5], [0, 0, 0]])]).astype(np.int32)}[table]
    q = rng.integers(-18, 18, size=(2049, d)).astype(np.int32)
    q[:2] = np.array([[2**31 - 1] * d, [-2**31] * d], np.int32)
    gi, gm = hm.find_offsets(dev(q), dev(offs))
    mq = (q[:, None, :].astype(np.int64) + offs[None, :, :].astype(np.int64))
    mq = ((mq + 2**31) % 2**32 - 2**31).astype(np.int32).reshape(-1, d)
    oi, omask = om.find(mq)
    assert gi.shape == (len(q), len(offs))
    assert_op_parity(hm, mq, gi.reshape(-1), gm.reshape(-1), oi, omask, check_distinct=False)
    if table == "radius1":
        ri, rm = hm.find_neighbors(dev(q), 1)
        assert torch.equal(ri, gi) and torch.equal(rm, gm)


@pytest.mark.parametrize("S", [4, 8, 16])
@pytest.mark.parametrize("d", [1, 3, 5, 8])
def test_warp_cooperative_find(d, S):
    """Warp-cooperative probing (lane groups, ballots) returns exactly what
    the thread-per-key find returns, and both equal the oracle, on hits,
    misses, ragged n and a long probe chain (load close to the rebuild
    threshold)."""
    rng = np.random.default_rng(81 + d + S)
    cap = 40_000
    t = ash.default_tuning()
    t.slots_per_bucket = S
    t.slots_per_capacity = 1.2  # high load: probe chains cross buckets
    hm = ash.HashMap(d, cap, tuning=t)
    om = oracle.OracleMap(d, cap)
    keys = rng.integers(-40, 40, size=(33_333, d)).astype(np.int32)
    hm.activate(dev(keys))
    om.activate(keys)
    q = np.concatenate([keys[::3], rng.integers(-45, 45, size=(20_001, d)).astype(np.int32)])
    oi, om_ = om.find(q)
    t.warp_probe = 0
    hm.set_tuning(t)
    ti, tm = hm.find(dev(q))
    t.warp_probe = 1
    hm.set_tuning(t)
    wi, wm = hm.find(dev(q))
    assert torch.equal(ti, wi) and torch.equal(tm, wm)
    assert_op_parity(hm, q, wi, wm, oi, om_, check_distinct=False)


@pytest.mark.parametrize("two_streams", [False, True])
def test_repeated_batches_near_capacity(two_streams):
    """Many insert / erase batches on one map that hovers near its capacity:
    the host's bound on the live count is tightened from asynchronous
    control-block snapshots (one stream) or by synchronising (two streams);
    either way growth follows the oracle's rule exactly and the map equals
    the oracle's."""
    rng = np.random.default_rng(91 + two_streams)
    pool = rng.integers(-10_000, 10_000, size=(9_000, 3)).astype(np.int32)
    pool = np.unique(pool, axis=0)
    hm = ash.HashMap(3, 10_000, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, 10_000, [4])
    side = torch.cuda.Stream()
    for r in range(120):
        ins = pool[rng.integers(0, len(pool), size=700)]
        vals = rng.random(700, dtype=np.float32)
        if two_streams and r % 3 == 1:
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                gi, gm = hm.insert(dev(ins), [dev(vals)])
            torch.cuda.current_stream().wait_stream(side)
        else:
            gi, gm = hm.insert(dev(ins), [dev(vals)])
        oi, omask = om.insert(ins, [vals])
        assert_op_parity(hm, ins, gi, gm, oi, omask)
        er = pool[rng.integers(0, len(pool), size=350)]
        assert np.array_equal(hm.erase(dev(er)).cpu().numpy(), om.erase(er))
        if r % 20 == 19:
            assert hm.capacity() == om.capacity()
            assert_same_map(hm, om)
    assert hm.capacity() == om.capacity()
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


@pytest.mark.parametrize("d", [1, 3, 5])
def test_partitioned_keys_match_oracle(d):
    """Calls whose keys are first put in home-bucket range order (forced,
    16+ ranges) equal the oracle: activate into a fresh map, find of hits and
    misses, activate over existing keys, erase, find again.  Each input row
    keeps its own output; the lowest position of equal keys wins."""
    rng = np.random.default_rng(31 + d)
    hm = ash.HashMap(d, 120_000, tuning=tuning(partition_keys=2))
    om = oracle.OracleMap(d, 120_000, [])
    a = rng.integers(-40, 40, size=(150_001, d)).astype(np.int32)
    gi, gm = hm.activate(dev(a))
    oi, omask = om.activate(a)
    assert_op_parity(hm, a, gi, gm, oi, omask)
    q = rng.integers(-45, 45, size=(70_003, d)).astype(np.int32)
    gi, gm = hm.find(dev(q))
    oi, omask = om.find(q)
    assert_op_parity(hm, q, gi, gm, oi, omask, check_distinct=False)
    b = rng.integers(-50, 50, size=(90_017, d)).astype(np.int32)
    gi, gm = hm.activate(dev(b))
    oi, omask = om.activate(b)
    assert_op_parity(hm, b, gi, gm, oi, omask)
    er = b[rng.integers(0, len(b), size=30_000)]
    assert np.array_equal(hm.erase(dev(er)).cpu().numpy(), om.erase(er))
    gi, gm = hm.find(dev(q))
    oi, omask = om.find(q)
    assert_op_parity(hm, q, gi, gm, oi, omask, check_distinct=False)
    assert_same_map(hm, om)
    assert_heap_permutation(hm)


@pytest.mark.parametrize("n", [1, 31, 32_767, 32_768, 32_769, 100_000])
def test_partitioned_ragged_sizes(n):
    """Ranged calls at sizes around one partition block (32768 keys): the
    same masks as calls in input order, and each index names its key."""
    rng = np.random.default_rng(n)
    keys = rng.integers(-2**20, 2**20, size=(n, 3)).astype(np.int32)
    keys[n // 2:] = keys[: n - n // 2]  # duplicates, later positions lose
    outs = []
    for part in (1, 2):
        hm = ash.HashMap(3, n, tuning=tuning(partition_keys=part))
        gi, gm = hm.activate(dev(keys))
        fi, fm = hm.find(dev(keys))
        om = oracle.OracleMap(3, n, [])
        oi, omask = om.activate(keys)
        assert_op_parity(hm, keys, gi, gm, oi, omask)
        assert fm.all() and torch.equal(hm.key_buffer()[fi.long()].cpu(), torch.from_numpy(keys))
        outs.append(gm.cpu())
    assert torch.equal(outs[0], outs[1])


def test_partitioned_first_occurrence_heavy_duplicates():
    """10^6 keys from 1000 distinct triples, ranged: exactly the first
    occurrence of each key wins (Sec. 4.4.2's heavy-duplicate setting)."""
    rng = np.random.default_rng(15)
    distinct = rng.integers(-2**30, 2**30, size=(1000, 3)).astype(np.int32)
    keys = distinct[rng.integers(0, 1000, size=1_000_000)]
    hm = ash.HashMap(3, 1_000_000, tuning=tuning(partition_keys=2))
    gi, gm = hm.activate(dev(keys))
    _, first = np.unique(keys, axis=0, return_index=True)
    want = np.zeros(len(keys), bool)
    want[first] = True
    assert np.array_equal(gm.cpu().numpy(), want)
    assert hm.size() == 1000


_REFUSING_ALLOCATOR = []  # the callbacks outlive every map that uses them


def test_partitioned_call_without_scratch_uses_input_order():
    """A ranged call whose stream-ordered scratch cannot be had (the map's
    allocator refuses it) runs its keys in input order instead, with the
    same results: activate and find against the oracle."""
    import ctypes
    refuse = {"above": None}

    def _alloc(nbytes, device, stream, ctx):
        if refuse["above"] is not None and nbytes > refuse["above"]:
            return 0
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:
            return 0

    def _free(ptr, device, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ash._ALLOC_FN(_alloc), ash._FREE_FN(_free)
    _REFUSING_ALLOCATOR.extend([a, f, refuse])
    L = ash.lib()
    ash._check(L.ash_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
    try:
        hm = ash.HashMap(3, 150_001, tuning=tuning(partition_keys=2))
    finally:
        ash._check(L.ash_set_allocator(None, None, None))  # maps keep the allocator they were created with
    rng = np.random.default_rng(41)
    keys = rng.integers(-30, 30, size=(150_001, 3)).astype(np.int32)
    kd = dev(keys)

    def partition_launches(fn):  # (fn's result, traced partitions)
        ash.ash_trace_reset()
        ash.ash_trace_enable(True)
        out = fn()
        torch.cuda.synchronize()
        ash.ash_trace_enable(False)
        return out, ash.ash_trace_collect()["partition_keys"][1]

    refuse["above"] = 1 << 20  # the call's scratch is about 3 MB
    (gi, gm), n_act = partition_launches(lambda: hm.activate(kd))
    (fi, fm), n_find = partition_launches(lambda: hm.find(kd))
    refuse["above"] = None
    assert n_act == 0 and n_find == 0, "a call whose scratch was refused still partitioned"
    om = oracle.OracleMap(3, 150_001, [])
    oi, omask = om.activate(keys)
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert bool(fm.all()) and torch.equal(hm.key_buffer()[fi.long()].cpu(), torch.from_numpy(keys))
    # with the scratch available the same find is ranged (one traced
    # partition: count, scan, scatter)
    (fi2, fm2), n_find2 = partition_launches(lambda: hm.find(kd))
    assert n_find2 == 1 and torch.equal(fi2, fi) and torch.equal(fm2, fm)
    assert_same_map(hm, om)
    del hm


def test_partitioned_at_full_size():
    """2x10^7 uniform keys at uniqueness 0.5 into capacity 2x10^7 (the
    table, 320 MB, is more than twice L2, so the default tuning ranges the
    keys): an activate, then a find in a fresh random order: one winner per
    distinct key, the first occurrence; every key found at its winner's
    index."""
    from bench import device_uniform_keys
    n = 20_000_000
    keys = device_uniform_keys(n, 0.5, 3, torch.device("cuda", 0))
    hm = ash.HashMap(3, n)
    gi, gm = hm.activate(keys)
    perm = torch.randperm(n, device=keys.device)
    fi_p, fm_p = hm.find(keys[perm].contiguous())
    fi = torch.empty_like(fi_p)
    fm = torch.empty_like(fm_p)
    fi[perm] = fi_p
    fm[perm] = fm_p
    assert bool(fm.all())
    n_unique = torch.unique(keys, dim=0).shape[0]
    assert int(gm.sum()) == n_unique == hm.size()
    # the winner of each index is the lowest position holding its key
    pos = torch.arange(n, device=keys.device)
    first = torch.full((hm.capacity(),), n, dtype=torch.int64, device=keys.device)
    first.scatter_reduce_(0, fi.long(), pos, reduce="amin")
    assert torch.equal(gm, first[fi.long()] == pos)
    assert torch.equal(gi[gm], fi[gm])
    assert torch.equal(hm.key_buffer()[fi.long()], keys)


def test_commit_snapshot_avoids_host_sync():
    """The insert's commit publishes the control block when the bound on the
    live count passes half the capacity (Sec. 4.5 growth check without a
    synchronisation): 6000 keys with 3000 distinct ones, then 6000 keys with
    3000 new distinct ones into capacity 10^4.  The loose bound (12000) would
    force a synchronising read; the landed snapshot (3000 + 6000) does not.
    Results equal the oracle's and the capacity stays."""
    rng = np.random.default_rng(17)
    pool = np.unique(rng.integers(-50_000, 50_000, size=(7_000, 3)).astype(np.int32), axis=0)[:6_000]
    a, b = pool[:3_000], pool[3_000:]
    hm = ash.HashMap(3, 10_000)
    om = oracle.OracleMap(3, 10_000, [])
    runs = []
    for part in (a, b):
        keys = np.concatenate([part, part[rng.permutation(len(part))]])
        runs.append((keys, hm.activate(dev(keys))))
        torch.cuda.synchronize()  # the snapshot has landed
    st = hm.stats()  # its own read is the one synchronising read
    assert st["host_syncs"] == 1, st
    for keys, (gi, gm) in runs:
        oi, omask = om.activate(keys)
        assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert hm.capacity() == om.capacity() == 10_000
    assert_same_map(hm, om)


@pytest.mark.parametrize("d,cell", [(3, 0.005), (3, 0.048), (2, 0.01), (1, 0.25)])
def test_point_input_ops(d, cell):
    """insert / activate / find on float32 points quantised in the kernels
    equal the same operations on ash_quantize's keys, and the oracle
    (quantisation of Sec. 6.1 + the map operations)."""
    rng = np.random.default_rng(97 + d)
    pts3 = workloads.voxel_scene_points(150_001, seed=d)
    pts = np.ascontiguousarray(pts3[:, :d]) if d < 3 else pts3
    pts = pts * np.float32(-1.0 if d == 2 else 1.0)  # negative coordinates too
    keys = oracle.quantize(pts, cell)
    ids = np.arange(len(pts), dtype=np.int32)
    hm = ash.HashMap(d, len(pts) // 3, [(1,)], [torch.int32])   # grows
    om = oracle.OracleMap(d, len(pts) // 3, [4])
    gi, gm = hm.insert_points(dev(pts), cell, [dev(ids)])
    oi, omask = om.insert(keys, [ids])
    assert_op_parity(hm, keys, gi, gm, oi, omask)
    assert hm.capacity() == om.capacity()
    q = np.concatenate([pts[::2], (pts[:5000] + np.float32(1000.0))])
    fi, fm = hm.find_points(dev(q), cell)
    ofi, ofm = om.find(oracle.quantize(q, cell))
    assert_op_parity(hm, oracle.quantize(q, cell), fi, fm, ofi, ofm, check_distinct=False)
    ki, km = hm.find(ash.ash_quantize(dev(q), cell))
    assert torch.equal(ki, fi) and torch.equal(km, fm)
    assert_same_map(hm, om)
    hs = ash.HashMap(d, 1000)
    ai, am = hs.activate_points(dev(pts), cell)
    os_ = oracle.OracleMap(d, 1000)
    aoi, aom = os_.activate(keys)
    assert_op_parity(hs, keys, ai, am, aoi, aom)
    assert_same_map(hs, os_)



def test_erase_churn_keeps_tombstones_bounded():
    """Insert/erase churn on a table larger than the tombstone floor: erased
    slots in full buckets stay tombstones, and the map rebuilds its table
    (same capacity, same indices) once the known tombstones pass a quarter of
    its live entries, so they never pile up; the map still equals the oracle
    and its stats add up (live = size, used >= live)."""
    rng = np.random.default_rng(77)
    pool = np.unique(rng.integers(-(1 << 12), 1 << 12, size=(400_000, 3)).astype(np.int32), axis=0)
    cap = 1 << 18
    hm = ash.HashMap(3, cap, [(1,)], [torch.float32])
    om = oracle.OracleMap(3, cap, [4])
    worst = 0.0
    for r in range(40):
        a = int(rng.integers(0, len(pool) - 60_000))
        ins = pool[a:a + 60_000]
        vals = rng.random(len(ins), dtype=np.float32)
        gi, gm = hm.insert(dev(ins), [dev(vals)])
        oi, omask = om.insert(ins, [vals])
        assert_op_parity(hm, ins, gi, gm, oi, omask)
        b = int(rng.integers(0, len(pool) - 50_000))
        er = pool[b:b + 50_000]
        assert np.array_equal(hm.erase(dev(er)).cpu().numpy(), om.erase(er))
        st = hm.stats()
        assert st["live"] == om.size() and st["used_slots"] >= st["live"]
        assert st["capacity"] == om.capacity() and st["table_slots"] >= 2 * st["capacity"]
        if r >= 2:
            worst = max(worst, (st["used_slots"] - st["live"]) / max(1, st["live"]))
    st = hm.stats()
    assert st["rebuilds"] > 0, st
    # the bound acts on landed snapshots, so allow the tombstones of a few
    # batches on top of a quarter of the live entries
    assert worst < 1.0, worst
    assert_same_map(hm, om)
    assert_heap_permutation(hm)
