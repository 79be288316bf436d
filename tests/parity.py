"""Comparison rules between the CUDA map and the CPU oracle.

Buffer indices are a permutation the paper leaves unspecified, so results are
compared modulo that permutation:
  * masks equal bitwise;
  * every GPU index with mask 1 stores the queried key (kB(i) = k, Eq. (4));
  * indices with mask 0 are -1; indices handed out in one batch are distinct;
  * the maps {kB(i) -> vB_j(i)} over the live entries are equal, value rows
    compared as raw bytes (float bits, not ==);
  * live counts are equal, and the GPU heap keeps active + free a permutation.
"""
import numpy as np
import torch


def _sorted_rows(keys, values):
    order = np.lexsort(keys.T[::-1]) if keys.shape[0] else np.arange(0)
    return keys[order], [v[order] for v in values]


def gpu_state(hm):
    """(keys [n,d] int32, [value rows as uint8 [n, rb]]) of the live entries, sorted by key."""
    act = hm.active_indices().long()
    kb = hm.key_buffer()[act].cpu().numpy()
    vals = []
    for j in range(len(hm.value_shapes)):
        buf = hm.value_buffer(j)
        rb = buf[0].numel() * buf.element_size()
        v = buf[act].contiguous()
        vals.append(v.view(torch.uint8).reshape(act.numel(), rb).cpu().numpy())
    return _sorted_rows(kb, vals)


def oracle_state(om):
    act = om.active_indices()
    kb = om.key_buffer()[act]
    vals = [om.value_buffer(j)[act] for j in range(len(om.row_bytes))]
    return _sorted_rows(kb, vals)


def assert_same_map(hm, om, check_values=True):
    gk, gv = gpu_state(hm)
    ok, ov = oracle_state(om)
    assert gk.shape == ok.shape, f"live count differs: gpu {gk.shape[0]} vs oracle {ok.shape[0]}"
    assert np.array_equal(gk, ok), "live key sets differ"
    if check_values:
        for j, (a, b) in enumerate(zip(gv, ov)):
            assert np.array_equal(a, b), f"value buffer {j} differs (bitwise)"
    assert hm.size() == om.size()
    assert hm.capacity() == om.capacity(), f"capacity differs: gpu {hm.capacity()} vs oracle {om.capacity()}"


def assert_op_parity(hm, keys_np, g_idx, g_mask, o_idx, o_mask, check_distinct=True):
    gm = g_mask.cpu().numpy().astype(bool)
    gi = g_idx.cpu().numpy()
    assert np.array_equal(gm, np.asarray(o_mask, bool)), f"masks differ at {np.flatnonzero(gm != o_mask)[:10]}"
    assert (gi[~gm] == -1).all(), "an index with mask 0 is not -1"
    if gm.any():
        kb = hm.key_buffer().cpu().numpy()
        assert np.array_equal(kb[gi[gm]], keys_np[gm]), "kB at a returned index differs from the key"
        if check_distinct:
            assert len(np.unique(gi[gm])) == int(gm.sum()), "an index was handed out twice"


def assert_heap_permutation(hm):
    h, t = hm.heap()
    act = hm.active_indices().cpu().numpy()
    assert t == act.shape[0] == hm.size(), "heap top differs from the live count"
    free = h[t:].cpu().numpy()
    both = np.sort(np.concatenate([act, free]))
    assert np.array_equal(both, np.arange(hm.capacity())), "active + free indices are not a permutation"


def value_rows_for(hm, j, idx):
    buf = hm.value_buffer(j)
    rb = buf[0].numel() * buf.element_size()
    v = buf[idx.long()].contiguous()
    return v.view(torch.uint8).reshape(idx.numel(), rb).cpu().numpy()
