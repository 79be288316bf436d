"""The voxel-block pipeline of Sec. 6.2 on the GPU against the oracle:
depth -> block keys (bit-exact, pixel order), the double hash map block
allocation (bit-exact key sets, first-occurrence order, index chaining), TSDF
integration (decisions bit-exact: identical updated-voxel sets and weights;
values within the float32 bound derived below) and ray casting (identical hit
sets; depths within the float32 bound derived below).

Tolerances.  Integration: each float32 update d := (w d + Psi) / (w + 1)
rounds three times (product, sum, quotient, each a relative 2^-24), the
inputs Psi are bit-identical on both sides, and |w d + Psi| / (w + 1) <= mu,
so after w updates |d_gpu - d_oracle| <= 3 w 2^-24 mu; the tests allow
4 w 2^-24 mu.  Ray casting: the crossing t_{i-1} + step * r with
r = d_{i-1} / (d_{i-1} - d_i) in [0, 1] rounds four times, so the error is at
most (3 step + t) 2^-24; the tests allow 4 (step + t) 2^-24.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2110_00511_gb300 import ash, workloads

pytestmark = pytest.mark.gpu

SMALL = workloads.Camera(width=160, height=120, fx=131.25, fy=131.25, cx=79.5, cy=59.5)
FULL = workloads.Camera()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2110_00511_gb300 import build
    build.build()
    ash.lib()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def intr(cam):
    return (cam.fx, cam.fy, cam.cx, cam.cy)


def _frames(n, cam, seed=0, holes=0.03):
    """Depth frames of the analytic room along the camera path, with a few
    pixels without depth and a few beyond depth_max."""
    scene = workloads.room_scene(seed)
    out = []
    for j, ex in enumerate(workloads.camera_path(n, seed)):
        d = workloads.render_depth(scene, ex, cam, noise=0.002, seed=seed * 1000 + j)
        rng = np.random.default_rng(seed * 1000 + j)
        d[rng.random(d.shape) < holes] = 0.0
        d[rng.random(d.shape) < holes / 3] = 9.0
        out.append((d, ex))
    return scene, out


# ------------------------------------------------------------ depth -> keys
@pytest.mark.parametrize("edge", [0.048, 0.16])
def test_depth_to_block_keys_bit_exact(edge):
    _, frames = _frames(3, FULL)
    for d, ex in frames:
        want = oracle.depth_to_block_keys(d, intr(FULL), ex, edge, 4.0)
        got = ash.ash_depth_to_block_keys(dev(d), intr(FULL), ex, edge, 4.0)
        assert np.array_equal(got.cpu().numpy(), want)
        keys, cnt = ash.ash_depth_to_block_keys(dev(d), intr(FULL), ex, edge, 4.0, sync=False)
        assert int(cnt.item()) == len(want)
        assert np.array_equal(keys[: len(want)].cpu().numpy(), want)


def test_depth_to_block_keys_edges():
    # all pixels invalid, one pixel, an empty image
    z = torch.zeros((4, 5), dtype=torch.float32, device="cuda")
    assert ash.ash_depth_to_block_keys(z, (1, 1, 2, 2), np.hstack([np.eye(3), np.zeros((3, 1))]), 0.1, 4.0).shape[0] == 0
    one = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
    one[1, 2] = 1.0
    k = ash.ash_depth_to_block_keys(one, (1, 1, 1, 1), np.hstack([np.eye(3), np.zeros((3, 1))]), 0.5, 4.0)
    assert k.cpu().numpy().tolist() == [[2, 0, 2]]
    e = torch.zeros((0, 7), dtype=torch.float32, device="cuda")
    assert ash.ash_depth_to_block_keys(e, (1, 1, 1, 1), np.hstack([np.eye(3), np.zeros((3, 1))]), 0.5, 4.0).shape[0] == 0
    with pytest.raises(ash.AshError):
        ash.ash_depth_to_block_keys(one, (1, 1, 1, 1), np.hstack([np.eye(3), np.zeros((3, 1))]), 0.0, 4.0)


# ------------------------------------------------------------ double hash map
def _assert_chained(local, glob):
    """Every live local entry's value is a global index holding the same key."""
    act = local.active_indices().long()
    lk = local.key_buffer()[act]
    gi = local.value_buffer(0)[act].reshape(-1).long()
    assert torch.equal(glob.key_buffer()[gi], lk)


def _keyset(hm):
    return {tuple(r) for r in hm.gather_keys(hm.active_indices()).cpu().numpy().tolist()}


@pytest.mark.parametrize("clear_local", [True, False])
def test_double_map_activate_matches_oracle(clear_local):
    _, frames = _frames(6, FULL, seed=1)
    edge = 0.048
    local = ash.HashMap(3, 20_000, [(1,)], [torch.int32])
    glob = ash.HashMap(3, 1000)                 # grows several times
    olocal = oracle.OracleMap(3, 20_000, [4])
    oglob = oracle.OracleMap(3, 1000)
    for d, ex in frames:
        keys = oracle.depth_to_block_keys(d, intr(FULL), ex, edge, 4.0)
        if clear_local:
            local.clear()
            olocal.clear()
        uk, li, gi = ash.ash_double_map_activate(local, glob, dev(keys))
        ouk, oli, ogi = oracle.double_map_activate(olocal, oglob, keys)
        assert np.array_equal(uk.cpu().numpy(), ouk), "distinct new keys (first-occurrence order) differ"
        assert torch.equal(local.key_buffer()[li.long()], uk)
        assert torch.equal(glob.key_buffer()[gi.long()], uk)
        assert local.size() == olocal.size() and glob.size() == oglob.size()
        assert glob.capacity() == oglob.capacity() and local.capacity() == olocal.capacity()
        assert _keyset(glob) == set(oglob.as_dict().keys())
        assert _keyset(local) == set(olocal.as_dict().keys())
        _assert_chained(local, glob)


def test_double_map_rejects_bad_maps():
    a = ash.HashMap(3, 100)
    b = ash.HashMap(3, 100)
    k = dev(np.zeros((4, 3), np.int32))
    with pytest.raises(ash.AshError):
        ash.ash_double_map_activate(a, b, k)     # local without an int32 value
    loc = ash.HashMap(3, 100, [(1,)], [torch.int32])
    with pytest.raises(ash.AshError):
        ash.ash_double_map_activate(loc, loc, k)
    with pytest.raises(ash.AshError):
        ash.ash_double_map_activate(loc, ash.HashMap(2, 100), dev(np.zeros((4, 3), np.int32)))
    uk, li, gi = ash.ash_double_map_activate(loc, b, dev(np.zeros((0, 3), np.int32)))
    assert uk.shape[0] == 0


# ------------------------------------------------------------ integration
def _integrate_pipeline(cam, frames, voxel, trunc, cap_global, ell=8):
    """GPU: depth -> keys -> double map -> integrate; oracle: the same steps."""
    edge = voxel * ell
    local = ash.HashMap(3, 50_000, [(1,)], [torch.int32])
    vol = ash.HashMap(3, cap_global, [(ell, ell, ell), (ell, ell, ell)], [torch.float32, torch.float32])
    olocal = oracle.OracleMap(3, 50_000, [4])
    ovol = oracle.OracleMap(3, cap_global, [8 * ell ** 3, 8 * ell ** 3])
    for d, ex in frames:
        dd = dev(d)
        keys = ash.ash_depth_to_block_keys(dd, intr(cam), ex, edge, 4.0)
        local.clear()
        _, _, gi = ash.ash_double_map_activate(local, vol, keys)
        ash.ash_tsdf_integrate(vol, gi, dd, intr(cam), ex, voxel, trunc, 4.0)
        okeys = oracle.depth_to_block_keys(d, intr(cam), ex, edge, 4.0)
        olocal.clear()
        _, _, ogi = oracle.double_map_activate(olocal, ovol, okeys)
        oracle.tsdf_integrate(ovol, ogi, d, intr(cam), ex, voxel, trunc, 4.0, ell=ell)
    return vol, ovol


def _compare_volumes(vol, ovol, trunc, ell=8):
    act = vol.active_indices()
    keys = vol.gather_keys(act).cpu().numpy()
    assert len(keys) == ovol.size() == vol.size()
    okb = ovol.key_buffer()
    oidx = {tuple(okb[i].tolist()): int(i) for i in ovol.active_indices()}
    assert set(oidx) == {tuple(k) for k in keys.tolist()}, "block key sets differ"
    oi = np.array([oidx[tuple(k)] for k in keys.tolist()])
    g_d = vol.value_buffer(0)[act.long()].reshape(len(keys), -1).cpu().numpy().astype(np.float64)
    g_w = vol.value_buffer(1)[act.long()].reshape(len(keys), -1).cpu().numpy().astype(np.float64)
    o_d = ovol.value_buffer(0).view(np.float64).reshape(-1, ell ** 3)[oi]
    o_w = ovol.value_buffer(1).view(np.float64).reshape(-1, ell ** 3)[oi]
    assert np.array_equal(g_w, o_w), "updated-voxel sets or weights differ"
    tol = 4 * o_w * 2.0 ** -24 * trunc
    bad = np.abs(g_d - o_d) > tol
    assert not bad.any(), f"{bad.sum()} voxels outside the float32 bound, worst {np.abs(g_d - o_d).max()}"
    return g_w


def test_tsdf_integrate_matches_oracle():
    voxel, trunc = 0.02, 0.06
    _, frames = _frames(5, SMALL, seed=2)
    vol, ovol = _integrate_pipeline(SMALL, frames, voxel, trunc, 4096)
    w = _compare_volumes(vol, ovol, trunc)
    assert (w > 0).mean() > 0.05 and w.max() >= 2


def test_tsdf_integrate_ell16_and_index_edges():
    voxel, trunc = 0.01, 0.03
    _, frames = _frames(2, SMALL, seed=3)
    vol, ovol = _integrate_pipeline(SMALL, frames, voxel, trunc, 1024, ell=16)
    _compare_volumes(vol, ovol, trunc, ell=16)
    # out-of-range block indices are skipped; an empty list is a no-op
    before = vol.value_buffer(1).clone()
    d, ex = frames[0]
    ash.ash_tsdf_integrate(vol, torch.tensor([-1, 1 << 30], dtype=torch.int32, device="cuda"), dev(d), intr(SMALL), ex,
                           voxel, trunc, 4.0)
    ash.ash_tsdf_integrate(vol, torch.zeros(0, dtype=torch.int32, device="cuda"), dev(d), intr(SMALL), ex, voxel,
                           trunc, 4.0)
    assert torch.equal(before, vol.value_buffer(1))
    with pytest.raises(ash.AshError):
        bad = ash.HashMap(3, 10, [(8, 8, 8)], [torch.float16])
        ash.ash_tsdf_integrate(bad, torch.zeros(1, dtype=torch.int32, device="cuda"), dev(d), intr(SMALL), ex, voxel,
                               trunc, 4.0, tsdf_buffer=0, weight_buffer=0)


# ------------------------------------------------------------ ray casting
def _room_volume(voxel, trunc, seed=0):
    scene = workloads.room_scene(seed)
    keys, d, w = workloads.room_tsdf_blocks(scene, voxel, trunc)
    vol = ash.HashMap(3, len(keys), [(8, 8, 8), (8, 8, 8)], [torch.float32, torch.float32])
    vol.insert(dev(keys), [dev(d.reshape(-1, 8, 8, 8)), dev(w.reshape(-1, 8, 8, 8))])
    ovol = oracle.OracleMap(3, len(keys), [4 * 512, 4 * 512])
    ovol.insert(keys, [d, w])
    return scene, keys, d, w, vol, ovol


def _assert_depths(got, want, step):
    got = got.reshape(-1).astype(np.float64)
    assert np.array_equal(got > 0, want > 0), f"hit sets differ at {(np.flatnonzero((got > 0) != (want > 0)))[:10]}"
    tol = 4 * (step + want) * 2.0 ** -24
    assert np.all(np.abs(got - want) <= tol), f"worst depth error {np.abs(got - want).max()}"


def test_tsdf_raycast_matches_oracle():
    voxel, trunc = 0.04, 0.12
    _, _, _, _, vol, ovol = _room_volume(voxel, trunc)
    step = voxel / 2
    n_steps = int((4.0 - 0.3) / step)
    hits = 0
    for ex in workloads.camera_path(4, seed=5):
        got = ash.ash_tsdf_raycast(vol, intr(SMALL), ex, SMALL.width, SMALL.height, voxel, 0.3, step, n_steps)
        want = oracle.tsdf_raycast(ovol, intr(SMALL), ex, SMALL.width, SMALL.height, voxel, 0.3, step, n_steps,
                                   value_bytes=4)
        _assert_depths(got.cpu().numpy(), want, step)
        hits += (want > 0).sum()
    assert hits > 0.5 * 4 * SMALL.width * SMALL.height


def test_tsdf_raycast_through_local_map():
    """Ray casting through the frame's local map (the double-hash-map speed-up
    of Sec. 6.2) equals the oracle's ray casting over the blocks the local map
    holds."""
    voxel, trunc = 0.04, 0.12
    _, keys, d, w, vol, ovol = _room_volume(voxel, trunc, seed=1)
    cam = SMALL
    ex = workloads.camera_path(3, seed=1)[1]
    depth = workloads.render_depth(workloads.room_scene(1), ex, cam)
    bkeys = oracle.depth_to_block_keys(depth, intr(cam), ex, voxel * 8, 4.0)
    local = ash.HashMap(3, 10_000, [(1,)], [torch.int32])
    ash.ash_double_map_activate(local, vol, dev(bkeys))
    olocal = oracle.OracleMap(3, 10_000, [4])
    oracle.double_map_activate(olocal, ovol, bkeys)
    # the oracle's view through the local map: the local keys with the volume's rows
    lkeys = np.array(sorted(olocal.as_dict().keys()), np.int32)
    _, gmask = ovol.find(lkeys)
    assert gmask.all()
    gidx, _ = ovol.find(lkeys)
    sub = oracle.OracleMap(3, len(lkeys), [4 * 512, 4 * 512])
    sub.insert(lkeys, [ovol.value_buffer(0)[gidx], ovol.value_buffer(1)[gidx]])
    step = voxel / 2
    n_steps = int((4.0 - 0.3) / step)
    got = ash.ash_tsdf_raycast(vol, intr(cam), ex, cam.width, cam.height, voxel, 0.3, step, n_steps, local=local)
    want = oracle.tsdf_raycast(sub, intr(cam), ex, cam.width, cam.height, voxel, 0.3, step, n_steps, value_bytes=4)
    _assert_depths(got.cpu().numpy(), want, step)
    full = ash.ash_tsdf_raycast(vol, intr(cam), ex, cam.width, cam.height, voxel, 0.3, step, n_steps)
    # the local view loses at most some hits (blocks outside the frame's frustum)
    assert ((got > 0) & (full == 0)).sum() == 0


def test_tsdf_raycast_recovers_rendered_depth():
    """End to end on the room: integrate 4 frames, ray-cast from a frame's
    pose; where both have a depth, the ray-cast one is within 3 voxels."""
    voxel, trunc = 0.02, 0.06
    _, frames = _frames(4, SMALL, seed=6, holes=0.0)
    vol, _ = _integrate_pipeline(SMALL, frames, voxel, trunc, 8192)
    d, ex = frames[-1]
    got = ash.ash_tsdf_raycast(vol, intr(SMALL), ex, SMALL.width, SMALL.height, voxel, 0.3, voxel / 2,
                               int(3.7 / (voxel / 2))).cpu().numpy()
    both = (got > 0) & (d > 0) & (d < 3.9)
    assert both.mean() > 0.5
    err = np.abs(got[both] - d[both])
    assert np.median(err) < voxel and np.percentile(err, 95) < 3 * voxel


# ------------------------------------------------------------ full size
@pytest.mark.slow
def test_full_frame_pipeline_sampled():
    """640 x 480 frames, 6 mm voxels in 8^3 blocks: keys and double-map sets
    bit-exact per frame, weights exact and values within the bound on a
    sample of blocks, ray-cast depth within the bound on sampled pixels."""
    voxel, trunc, ell = 0.006, 0.018, 8
    _, frames = _frames(3, FULL, seed=7)
    local = ash.HashMap(3, 400_000, [(1,)], [torch.int32])
    vol = ash.HashMap(3, 1 << 17, [(8, 8, 8), (8, 8, 8)], [torch.float32, torch.float32])
    olocal = oracle.OracleMap(3, 400_000, [4])
    ovol = oracle.OracleMap(3, 1 << 17, [8 * 512, 8 * 512])
    for d, ex in frames:
        dd = dev(d)
        keys = ash.ash_depth_to_block_keys(dd, intr(FULL), ex, voxel * ell, 4.0)
        okeys = oracle.depth_to_block_keys(d, intr(FULL), ex, voxel * ell, 4.0)
        assert np.array_equal(keys.cpu().numpy(), okeys)
        local.clear()
        olocal.clear()
        uk, _, gi = ash.ash_double_map_activate(local, vol, keys)
        ouk, _, ogi = oracle.double_map_activate(olocal, ovol, okeys)
        assert np.array_equal(uk.cpu().numpy(), ouk)
        ash.ash_tsdf_integrate(vol, gi, dd, intr(FULL), ex, voxel, trunc, 4.0)
        oracle.tsdf_integrate(ovol, ogi, d, intr(FULL), ex, voxel, trunc, 4.0)
    _compare_volumes(vol, ovol, trunc)
    rng = np.random.default_rng(0)
    pix = rng.choice(FULL.width * FULL.height, 3000, replace=False)
    d, ex = frames[1]
    step = voxel
    n_steps = int((4.0 - 0.3) / step)
    got = ash.ash_tsdf_raycast(vol, intr(FULL), ex, FULL.width, FULL.height, voxel, 0.3, step, n_steps)
    ovol32 = oracle.OracleMap(3, 1 << 17, [4 * 512, 4 * 512])   # the oracle's own volume, rounded to float32
    act = ovol.active_indices()
    okb = ovol.key_buffer()[act]
    ovol32.insert(okb, [ovol.value_buffer(0).view(np.float64).reshape(-1, 512)[act].astype(np.float32),
                        ovol.value_buffer(1).view(np.float64).reshape(-1, 512)[act].astype(np.float32)])
    want = oracle.tsdf_raycast(ovol32, intr(FULL), ex, FULL.width, FULL.height, voxel, 0.3, step, n_steps,
                               pixels=pix, value_bytes=4)
    g = got.reshape(-1)[torch.from_numpy(pix).cuda()].cpu().numpy().astype(np.float64)
    # the two volumes differ by float32 rounding of the running mean, so a
    # sample whose value sits within that bound of zero may flip its sign:
    # compare hits found by both and allow the rare disagreement
    both = (g > 0) & (want > 0)
    assert both.mean() > 0.5 and ((g > 0) != (want > 0)).mean() < 0.01
    assert np.median(np.abs(g[both] - want[both])) < 1e-5
