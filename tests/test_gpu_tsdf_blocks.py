"""Voxel-block map at full size (the TSDF setting of Sec. 6.2): 200 synthetic
640x480 depth frames at 6 mm voxels / 8^3 blocks, capacity 2^20, value
buffers tsdf float32[8,8,8] and weight float16[8,8,8].  Blocks are allocated
with the double-hash-map pattern of Sec. 6.2: a per-frame local map removes
duplicates (activate), the global map activates the surviving keys, and a
find links the local entries to global indices.  After all frames, the
27-neighbourhood of every active block is found.  Compared with the oracle
(first-occurrence unique keys per frame activated in the same order)."""
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


def test_tsdf_blocks_full_size():
    cap = 1 << 20
    gmap = ash.HashMap(3, cap, [(8, 8, 8), (8, 8, 8)], [torch.float32, torch.float16])
    om = oracle.OracleMap(3, cap, [2048, 1024])
    n_frames = 200
    for f, keys in enumerate(workloads.tsdf_block_frames(n_frames=n_frames, seed=0)):
        k = torch.from_numpy(keys).cuda()
        local = ash.HashMap(3, keys.shape[0])
        li, lm = local.activate(k)
        uk = k[lm]                       # unique block keys of this frame, first-occurrence order
        gi, gm = gmap.activate(uk)
        fi, fm = gmap.find(uk)
        assert bool(fm.all())
        # oracle: the same first-occurrence order
        _, first = np.unique(keys, axis=0, return_index=True)
        ok = keys[np.sort(first)]
        assert np.array_equal(uk.cpu().numpy(), ok), f"frame {f}: local dedup differs"
        oi, omask = om.activate(ok)
        assert_op_parity(gmap, ok, gi, gm, oi, omask)
        if f % 50 == 0:
            assert gmap.size() == om.size()
    assert gmap.capacity() == om.capacity() == cap, "the live blocks must fit the 2^20 capacity"
    assert gmap.size() < 0.7 * cap
    assert_same_map(gmap, om)  # value rows all zero: activate writes no value bytes
    act = gmap.active_indices()
    blocks = gmap.gather_keys(act).cpu().numpy()
    offs = workloads.radius_offsets(1)
    q = (blocks[:, None, :] + offs[None, :, :]).reshape(-1, 3).astype(np.int32)
    gi, gm = gmap.find(torch.from_numpy(q).cuda())
    oi, omask = om.find(q)
    assert_op_parity(gmap, q, gi, gm, oi, omask, check_distinct=False)
