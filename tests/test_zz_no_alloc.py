"""The allocation-free erase entry point (ash_erase_noalloc).

It serves callers that cannot let a library allocate device memory: hosts
whose device memory is fully budgeted by their own allocator, and loops where
a first-time allocation (which may synchronise the device) is not acceptable.
It must give exactly what ash_erase gives, call after call, while using its
fixed device array instead of map-owned scratch.

This file is collected last (tests/test_zz_*), so a run that stops at the
first failure has already run every other test.  It also passes alone in a
fresh process: the fixture builds and loads the library itself.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ash_mod():
    from paper_2110_00511_gb300 import ash, build
    build.build()
    ash.lib()
    return ash


def _twin_maps(ash_mod, keys, vals):
    a = ash_mod.HashMap(3, 1 << 18, [(1,)], [torch.float32])
    b = ash_mod.HashMap(3, 1 << 18, [(1,)], [torch.float32])
    a.insert(keys, [vals])
    b.insert(keys, [vals])
    return a, b


def _live(hm):
    act = hm.active_indices().long()
    k = hm.key_buffer()[act].cpu().numpy()
    v = hm.value_buffer(0)[act].cpu().numpy().view(np.uint32)
    order = np.lexsort(k.T[::-1])
    return k[order], v[order]


def test_noalloc_erase_matches_erase_two_calls(ash_mod):
    rng = np.random.default_rng(2024)
    keys = torch.from_numpy(rng.integers(-40, 40, size=(150_000, 3)).astype(np.int32)).cuda()
    vals = torch.from_numpy(rng.random(150_000, dtype=np.float32)).cuda()
    a, b = _twin_maps(ash_mod, keys, vals)
    for call in range(2):  # two calls in a row share (and reuse) the fixed array
        er = torch.from_numpy(rng.integers(-45, 45, size=(200_000, 3)).astype(np.int32)).cuda()
        ma = a.erase(er)
        mb = torch.empty(er.shape[0], dtype=torch.bool, device="cuda")
        ash_mod.ash_erase_noalloc(b.handle, er, mb)
        torch.cuda.synchronize()
        assert torch.equal(ma, mb), f"masks differ from ash_erase on call {call}"
        assert a.size() == b.size()
        ka, va = _live(a)
        kb, vb = _live(b)
        assert np.array_equal(ka, kb) and np.array_equal(va, vb), f"maps differ after call {call}"


def test_noalloc_erase_at_the_limit_and_beyond(ash_mod):
    n = ash_mod.ASH_ERASE_NOALLOC_MAX_KEYS
    rng = np.random.default_rng(7)
    keys = torch.from_numpy(rng.integers(-64, 64, size=(n, 3)).astype(np.int32)).cuda()
    vals = torch.zeros(n, dtype=torch.float32, device="cuda")
    a, b = _twin_maps(ash_mod, keys[: 1 << 17], vals[: 1 << 17])
    ma = a.erase(keys)
    mb = torch.empty(n, dtype=torch.bool, device="cuda")
    ash_mod.ash_erase_noalloc(b.handle, keys, mb)
    assert torch.equal(ma, mb)
    too_many = torch.zeros((n + 1, 3), dtype=torch.int32, device="cuda")
    out = torch.empty(n + 1, dtype=torch.bool, device="cuda")
    with pytest.raises(ash_mod.AshError) as e:
        ash_mod.ash_erase_noalloc(b.handle, too_many, out)
    assert e.value.status == ash_mod.ASH_ERR_INVALID
    assert "ASH_ERASE_NOALLOC_MAX_KEYS" in str(e.value)


def test_noalloc_erase_binding_checks_outputs(ash_mod):
    """Short or mistyped output arrays are refused before any kernel runs,
    and the map-level method gives the same masks as HashMap.erase."""
    keys = torch.zeros((8, 3), dtype=torch.int32, device="cuda")
    a, b = _twin_maps(ash_mod, keys, torch.zeros(8, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError, match="at least n"):
        ash_mod.ash_erase_noalloc(b.handle, keys, torch.empty(7, dtype=torch.bool, device="cuda"))
    with pytest.raises(ValueError, match="bool or uint8"):
        ash_mod.ash_erase_noalloc(b.handle, keys, torch.empty(8, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError, match="key_dim"):
        ash_mod.ash_erase_noalloc(b.handle, torch.zeros((8, 2), dtype=torch.int32, device="cuda"),
                                  torch.empty(8, dtype=torch.bool, device="cuda"))
    assert torch.equal(a.erase(keys), b.erase_noalloc(keys))
    assert a.size() == b.size() == 0
