"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs (numpy PCG64 via default_rng).  It holds none of
the hashing method's arithmetic and imports nothing else from this package, so
both the CUDA path's tests and the CPU oracle can consume the same arrays.

Workload shapes:
  * plain map (Sec. 5.1 setup, 3-D int32 keys, float values);
  * uniform keys at a chosen uniqueness ratio rho (the rho of Sec. 5.1/5.2);
  * a synthetic point-cloud scene for voxelization (Sec. 6.1 setup): spheres
    plus the three walls of a 10 m cube, Gaussian noise;
  * TSDF-shaped voxel-block keys from synthetic depth frames (Sec. 6.2):
    pinhole unprojection of smooth depth fields along a slow trajectory;
  * depth frames of a static analytic room (walls + spheres) rendered along a
    camera path, and the room's truncated signed distance sampled on voxel
    blocks (inputs for TSDF integration and ray casting, Sec. 6.2);
  * a many-map batch and a Poisson serving trace.
The paper's real scans are not available; these generators stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------- plain map
@dataclass
class PlainMapCase:
    insert_keys: np.ndarray      # int32 [N, 3]
    insert_values: np.ndarray    # float32 [N]
    query_keys: np.ndarray       # int32 [Q, 3]
    erase_keys: np.ndarray       # int32 [E, 3]
    capacity: int


def plain_map_case(seed: int = 0, n: int = 100_000, capacity: int = 1 << 18,
                   lo: int = -64, hi: int = 64) -> PlainMapCase:
    """Insert n keys uniform in [lo, hi)^3 with float32 values U(0,1); query n
    keys, half drawn from the inserted rows and half fresh from [hi, 2hi)^3;
    erase a random 25% of the inserted rows (duplicates included)."""
    rng = np.random.default_rng(seed)
    keys = rng.integers(lo, hi, size=(n, 3), dtype=np.int64).astype(np.int32)
    values = rng.random(n, dtype=np.float32)
    half = n // 2
    hit_rows = rng.integers(0, n, size=half)
    fresh = rng.integers(hi, 2 * hi, size=(n - half, 3), dtype=np.int64).astype(np.int32)
    queries = np.concatenate([keys[hit_rows], fresh], axis=0)
    queries = queries[rng.permutation(n)]
    erase_rows = rng.permutation(n)[: n // 4]
    return PlainMapCase(keys, values, np.ascontiguousarray(queries), np.ascontiguousarray(keys[erase_rows]), capacity)


# ---------------------------------------------------------- uniform / rho sweep
def _distinct_keys(rng, u: int, key_dim: int, lo: int, hi: int) -> np.ndarray:
    """u distinct int32 keys drawn uniformly from [lo, hi)^key_dim."""
    span = hi - lo
    bits = max(1, math.ceil(math.log2(span)))
    if bits * key_dim > 63:
        raise ValueError("key range too wide for distinctness packing")
    got = np.empty((0, key_dim), np.int64)
    need = u
    while need > 0:
        draw = rng.integers(lo, hi, size=(int(need * 1.05) + 16, key_dim), dtype=np.int64)
        allk = np.concatenate([got, draw], axis=0)
        packed = np.zeros(allk.shape[0], np.int64)
        for j in range(key_dim):
            packed = (packed << bits) | (allk[:, j] - lo)
        _, first = np.unique(packed, return_index=True)
        first.sort()
        got = allk[first]
        need = u - got.shape[0]
    got = got[:u]
    return got[rng.permutation(u)].astype(np.int32)


def uniform_keys(n: int, rho: float, seed: int = 0, key_dim: int = 3,
                 lo: int = -(1 << 20), hi: int = 1 << 20) -> np.ndarray:
    """n int32 keys with round(rho*n) distinct values: each distinct key appears
    once among the first positions, the rest are uniform picks among them, and
    the whole array is shuffled."""
    rng = np.random.default_rng(seed)
    u = max(1, min(n, int(round(rho * n))))
    distinct = _distinct_keys(rng, u, key_dim, lo, hi)
    if u < n:
        extra = distinct[rng.integers(0, u, size=n - u)]
        keys = np.concatenate([distinct, extra], axis=0)
    else:
        keys = distinct
    return np.ascontiguousarray(keys[rng.permutation(n)])


# ------------------------------------------------------------- voxelization
def voxel_scene_points(n: int = 4_000_000, seed: int = 0, n_spheres: int = 32,
                       room: float = 10.0, noise: float = 0.002) -> np.ndarray:
    """float32 [n, 3] points on 32 spheres (centres U[0,room]^3, radii
    U(0.2,1.5) m) and the planes x=0, y=0, z=0 of the room cube, sampled in
    proportion to surface area, plus isotropic Gaussian noise."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, room, size=(n_spheres, 3))
    radii = rng.uniform(0.2, 1.5, size=n_spheres)
    areas = np.concatenate([4.0 * np.pi * radii ** 2, np.full(3, room * room)])
    counts = rng.multinomial(n, areas / areas.sum())
    parts = []
    for s in range(n_spheres):
        m = counts[s]
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        parts.append(centres[s] + radii[s] * d)
    for axis in range(3):
        m = counts[n_spheres + axis]
        p = rng.uniform(0.0, room, size=(m, 3))
        p[:, axis] = 0.0
        parts.append(p)
    pts = np.concatenate(parts, axis=0)
    pts += rng.normal(scale=noise, size=pts.shape)
    pts = pts[rng.permutation(n)]
    return np.ascontiguousarray(pts.astype(np.float32))


# --------------------------------------------------------------- TSDF blocks
@dataclass
class Camera:
    width: int = 640
    height: int = 480
    fx: float = 525.0
    fy: float = 525.0
    cx: float = 319.5
    cy: float = 239.5


def _rotation(yaw: float, pitch: float) -> np.ndarray:
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    rz = np.array([[cy_, -sy_, 0.0], [sy_, cy_, 0.0], [0.0, 0.0, 1.0]])
    rx = np.array([[1.0, 0.0, 0.0], [0.0, cp, -sp], [0.0, sp, cp]])
    # camera looks along +z of its frame; tilt it to look horizontally first
    to_horizontal = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]])
    return rz @ rx @ to_horizontal


def tsdf_block_frames(n_frames: int = 200, seed: int = 0, voxel: float = 0.006, block: int = 8,
                      cam: Camera | None = None, stride: int = 1, orbit: float = 0.4, turn: float = 0.25,
                      drift: float = 0.01):
    """Yields int32 [H*W/stride^2, 3] voxel-block keys, one array per frame.

    Depth per frame is a smooth random field (a sum of 8 low-frequency
    sinusoids, phases drifting by `drift` rad per frame) mapped into
    [0.5, 4] m.  The camera moves slowly inside a 10 m room (an orbit of
    `orbit` m while turning through `turn` of a full revolution), so blocks are
    revisited.  Block edge is voxel * block (48 mm for the 6 mm / 8^3 setting
    of Sec. 6.2)."""
    cam = cam or Camera()
    rng = np.random.default_rng(seed)
    edge = voxel * block
    v, u = np.mgrid[0:cam.height:stride, 0:cam.width:stride]
    u = u.astype(np.float64).ravel()
    v = v.astype(np.float64).ravel()
    freqs = rng.uniform(0.5, 3.0, size=(8, 2))
    phases0 = rng.uniform(0.0, 2 * np.pi, size=8)
    amps = rng.uniform(0.5, 1.0, size=8)
    centre = np.array([5.0, 5.0, 1.5])
    for f in range(n_frames):
        t = f / max(1, n_frames)
        phases = phases0 + drift * f
        field_ = np.zeros_like(u)
        for j in range(8):
            field_ += amps[j] * np.sin(2 * np.pi * (freqs[j, 0] * u / cam.width + freqs[j, 1] * v / cam.height) + phases[j])
        field_ = (field_ - field_.min()) / max(1e-9, field_.max() - field_.min())
        depth = 0.5 + 3.5 * field_
        pos = centre + np.array([orbit * math.cos(2 * np.pi * t), orbit * math.sin(2 * np.pi * t),
                                 0.1 * math.sin(4 * np.pi * t)])
        rot = _rotation(2 * np.pi * turn * t + 0.05 * math.sin(6 * np.pi * t), 0.05 * math.sin(2 * np.pi * t))
        xc = (u - cam.cx) * depth / cam.fx
        yc = (v - cam.cy) * depth / cam.fy
        pc = np.stack([xc, yc, depth], axis=1)
        pw = pc @ rot.T + pos
        keys = np.floor(pw / edge).astype(np.int32)
        yield np.ascontiguousarray(keys)


@dataclass
class RoomScene:
    """A closed room [0, size]^3 with spheres (centre xyz, radius) inside."""
    size: float
    spheres: np.ndarray   # float64 [k, 4]


def room_scene(seed: int = 0, size: float = 5.0, n_spheres: int = 12) -> RoomScene:
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.8, size - 0.8, size=(n_spheres, 3))
    r = rng.uniform(0.15, 0.5, size=(n_spheres, 1))
    return RoomScene(size=size, spheres=np.hstack([c, r]))


def camera_path(n_frames: int, seed: int = 0, size: float = 5.0, orbit: float = 0.6, turn: float = 0.5):
    """World-to-camera extrinsics [R | t] (float32 3x4) along a slow orbit
    around the room's centre, turning through `turn` of a revolution."""
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0, 2 * np.pi)
    out = []
    for f in range(n_frames):
        a = f / max(1, n_frames)
        pos = np.array([size / 2 + orbit * math.cos(2 * np.pi * a + phase),
                        size / 2 + orbit * math.sin(2 * np.pi * a + phase), 1.5 + 0.1 * math.sin(4 * np.pi * a)])
        r_cw = _rotation(2 * np.pi * turn * a + phase, 0.15 * math.sin(2 * np.pi * a))
        r = r_cw.T
        out.append(np.hstack([r, (-r @ pos)[:, None]]).astype(np.float32))
    return out


def render_depth(scene: RoomScene, extrinsic: np.ndarray, cam: Camera | None = None, noise: float = 0.0,
                 seed: int = 0) -> np.ndarray:
    """float32 [H, W] depth (distance along the optical axis) of the room seen
    through a pinhole camera with world-to-camera `extrinsic`; Gaussian noise
    of `noise` m if nonzero."""
    cam = cam or Camera()
    e = np.asarray(extrinsic, np.float64)
    r, t = e[:, :3], e[:, 3]
    pos = -r.T @ t
    v, u = np.mgrid[0:cam.height, 0:cam.width]
    dc = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones(u.shape)], -1).reshape(-1, 3)
    dw = dc @ r                                   # camera -> world directions (camera z component 1)
    best = np.full(dw.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        for axis in range(3):
            for wall in (0.0, scene.size):
                tt = (wall - pos[axis]) / dw[:, axis]
                best = np.where((tt > 0) & (tt < best), tt, best)
    oc = pos[None, :] - scene.spheres[:, :3]      # [k, 3]
    a = np.einsum("ij,ij->i", dw, dw)
    for k in range(len(scene.spheres)):
        b = 2 * dw @ oc[k]
        cc = oc[k] @ oc[k] - scene.spheres[k, 3] ** 2
        disc = b * b - 4 * a * cc
        tt = np.where(disc > 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.inf)
        best = np.where((tt > 0) & (tt < best), tt, best)
    depth = np.where(np.isfinite(best), best, 0.0)
    if noise > 0:
        depth = depth + np.random.default_rng(seed).normal(scale=noise, size=depth.shape)
    return depth.reshape(cam.height, cam.width).astype(np.float32)


def room_sdf(scene: RoomScene, x: np.ndarray) -> np.ndarray:
    """Signed distance to the room's surfaces, positive in free space."""
    d = np.minimum(np.min(x, axis=-1), np.min(scene.size - x, axis=-1))
    for c in scene.spheres:
        d = np.minimum(d, np.linalg.norm(x - c[:3], axis=-1) - c[3])
    return d


def block_lattice(keys: np.ndarray, voxel: float, ell: int = 8) -> np.ndarray:
    """[n, ell^3, 3] world positions (K * ell + v) * voxel of the voxels of
    blocks `keys`, voxel slot (vz * ell + vy) * ell + vx."""
    g = np.stack(np.meshgrid(np.arange(ell), np.arange(ell), np.arange(ell), indexing="ij"), -1)
    g = g.transpose(2, 1, 0, 3).reshape(-1, 3)
    return (keys[:, None, :].astype(np.float64) * ell + g[None]) * voxel


def room_tsdf_blocks(scene: RoomScene, voxel: float, trunc: float, ell: int = 8, band: int = 1):
    """Voxel blocks within `band` blocks of a surface of the room and their
    truncated signed distance clamp(sdf, -trunc, trunc) with weight 1
    (float32 [n, ell^3] each), keys int32 [n, 3]."""
    edge = voxel * ell
    n = int(math.ceil(scene.size / edge))
    k = np.stack(np.meshgrid(np.arange(-1, n + 1), np.arange(-1, n + 1), np.arange(-1, n + 1), indexing="ij"),
                 -1).reshape(-1, 3)
    centre = (k + 0.5) * edge
    near = np.abs(room_sdf(scene, centre)) < (band + 0.87) * edge
    keys = k[near].astype(np.int32)
    x = block_lattice(keys, voxel, ell)
    d = np.clip(room_sdf(scene, x), -trunc, trunc).astype(np.float32)
    return np.ascontiguousarray(keys), np.ascontiguousarray(d), np.ones_like(d)


def radius_offsets(r: int = 1, key_dim: int = 3) -> np.ndarray:
    """All integer offsets in [-r, r]^key_dim (27 for r = 1 in 3-D)."""
    axes = [np.arange(-r, r + 1)] * key_dim
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, key_dim)
    return grid.astype(np.int32)


def cube_offsets(key_dim: int = 3) -> np.ndarray:
    """The 2^key_dim grid points of the cell whose lowest corner is the key
    (the 1-cube table), first coordinate slowest."""
    axes = [np.arange(0, 2)] * key_dim
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, key_dim)
    return grid.astype(np.int32)


def ring_offsets(key_dim: int = 3) -> np.ndarray:
    """The 2*key_dim face neighbours (the 1-ring table): -e_0, +e_0, -e_1, ..."""
    out = np.zeros((2 * key_dim, key_dim), np.int32)
    for j in range(key_dim):
        out[2 * j, j] = -1
        out[2 * j + 1, j] = 1
    return out


# ----------------------------------------------------------------- batched
@dataclass
class MapBatch:
    key_dim: int
    capacity: int
    insert_keys: np.ndarray
    insert_values: np.ndarray
    find_keys: np.ndarray
    erase_keys: np.ndarray
    rho: float


def batched_maps(n_maps: int = 64, seed: int = 0, log2_cap=(10, 21), mix=(0.3, 0.6, 0.1)) -> list:
    """n_maps independent maps: key_dim in {2,3,4}, capacity log-uniform in
    [2^lo, 2^hi], a batch of capacity/2 ops split insert/find/erase by `mix`,
    uniqueness rho ~ U(0.2, 1.0).  Finds draw half from the inserted keys."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_maps):
        d = int(rng.integers(2, 5))
        cap = int(round(2 ** rng.uniform(*log2_cap)))
        n_ops = max(3, cap // 2)
        n_ins = max(1, int(n_ops * mix[0]))
        n_find = max(1, int(n_ops * mix[1]))
        n_er = max(1, n_ops - n_ins - n_find)
        rho = float(rng.uniform(0.2, 1.0))
        ins = uniform_keys(n_ins, rho, seed=seed * 1000 + m, key_dim=d, lo=-(1 << 12), hi=1 << 12)
        vals = rng.random(n_ins, dtype=np.float32)
        fnd = np.concatenate([ins[rng.integers(0, n_ins, size=n_find // 2)],
                              rng.integers(-(1 << 12), 1 << 12, size=(n_find - n_find // 2, d)).astype(np.int32)])
        fnd = fnd[rng.permutation(n_find)]
        er = ins[rng.integers(0, n_ins, size=n_er)]
        out.append(MapBatch(d, cap, ins, vals, np.ascontiguousarray(fnd), np.ascontiguousarray(er), rho))
    return out


# ----------------------------------------------------------------- serving
@dataclass
class Request:
    rid: int
    tenant: int
    arrival_s: float
    op: str               # "insert" | "find" | "erase"
    keys: np.ndarray      # int32 [n, 3]
    values: np.ndarray | None = field(default=None)


def serving_trace(n_requests: int, rate_hz: float, seed: int = 0, n_tenants: int = 16,
                  size_range=(1_000, 1_000_000), mix=(0.3, 0.6, 0.1), key_span: int = 1 << 16) -> list:
    """Poisson arrivals at rate_hz over n_tenants; request sizes log-uniform in
    size_range; op types drawn by `mix` (insert, find, erase)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    ops = np.array(["insert", "find", "erase"])[rng.choice(3, size=n_requests, p=np.array(mix) / sum(mix))]
    lo, hi = math.log(size_range[0]), math.log(size_range[1])
    reqs = []
    for r in range(n_requests):
        n = int(round(math.exp(rng.uniform(lo, hi))))
        keys = rng.integers(-key_span, key_span, size=(n, 3), dtype=np.int64).astype(np.int32)
        vals = rng.random(n, dtype=np.float32) if ops[r] == "insert" else None
        reqs.append(Request(r, int(rng.integers(0, n_tenants)), float(t[r]), str(ops[r]), keys, vals))
    return reqs
