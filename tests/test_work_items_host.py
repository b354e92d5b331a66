"""The step kernels' work items, packed on the host (lbm_debug_pack_work_items), on the
geometries the benchmarks use and on random solids: every fluid cell once, each item's
cells increasing and contiguous from lane 0 with padding after them, a box segment whose 32
cells are all fluid as an item of its own, the other items confined to partly solid
segments and to a span of 449 cells (the entries' 13-bit link offsets)."""
import numpy as np
import pytest

import oracle
from paper_1508_02960_gb300 import capi
from paper_1508_02960_gb300 import inputs as I

SPAN = 449


def _solid(name):
    rng = np.random.default_rng(17)
    if name == "sphere_r60":
        g = I.centred_sphere(128, 60.0)
        return oracle.voxelize(g.shape, g.spheres)
    if name == "pack":
        g = I.random_pack(64, 6, 5.0, 9.0, 7)
        return oracle.voxelize(g.shape, g.spheres)
    if name == "slab_x":
        s = np.zeros((32, 32, 128), np.uint8)
        s[:, :, 36:91] = 1
        return s
    if name == "random30":
        return (rng.uniform(size=(24, 20, 40)) < 0.3).astype(np.uint8)
    if name == "sparse_fluid":  # isolated fluid cells far apart
        s = np.ones((16, 16, 96), np.uint8)
        s.reshape(-1)[::211] = 0
        return s
    raise KeyError(name)


@pytest.mark.parametrize("name", ["sphere_r60", "pack", "slab_x", "random30", "sparse_fluid"])
def test_work_items(name):
    solid = np.asarray(_solid(name)).reshape(-1)
    cells = np.flatnonzero(solid == 0)
    items = capi.pack_work_items(cells)
    live = items >= 0
    n_live = live.sum(axis=1)
    # lanes 0 .. n-1 live, the rest padding; every item holds a cell
    assert np.all(n_live >= 1)
    assert np.array_equal(live, np.arange(32)[None, :] < n_live[:, None])
    # every fluid cell exactly once
    got = np.sort(items[live])
    assert np.array_equal(got, cells)
    seg_of = items // 32
    full = n_live == 32
    for it, n in zip(items, n_live):
        c = it[:n]
        assert np.all(np.diff(c) > 0)
        assert c[-1] - c[0] < SPAN
    # each all-fluid box segment is one item, aligned
    n_seg = (solid.size + 31) // 32
    padded = np.ones(n_seg * 32, np.uint8)
    padded[:solid.size] = solid
    seg_fluid = (padded.reshape(n_seg, 32) == 0).sum(axis=1)
    full_segs = np.flatnonzero(seg_fluid == 32)
    aligned = full & (items[:, 0] % 32 == 0) & (items[:, 31] == items[:, 0] + 31)
    assert np.array_equal(np.sort(items[aligned, 0] // 32), full_segs)
    # the other items hold cells of partly solid segments only
    other = ~aligned
    assert np.all(seg_fluid[seg_of[other][live[other]]] < 32)
    # no more items than full segments plus the other cells in groups of 32 and one item
    # more for each span limit reached, at least the cells in groups of 32
    assert len(items) >= (len(cells) + 31) // 32
    if name == "sphere_r60":
        assert len(items) <= (len(cells) + 31) // 32 + 200


def test_work_items_reject_bad_input():
    L = capi.lib()
    n = capi.ctypes.c_int64(0)
    bad = np.array([5, 3, 9], np.uint32)
    p = bad.ctypes.data_as(capi.ctypes.POINTER(capi.ctypes.c_uint32))
    assert L.lbm_debug_pack_work_items(p, 3, None, 0, capi.ctypes.byref(n)) == capi.ERR_ARG
    assert "increasing" in capi.last_error()
    ok = np.array([1, 2, 3], np.uint32)
    p = ok.ctypes.data_as(capi.ctypes.POINTER(capi.ctypes.c_uint32))
    out = np.zeros(16, np.uint32)            # too small for one item
    assert L.lbm_debug_pack_work_items(p, 3, out.ctypes.data_as(capi.ctypes.POINTER(capi.ctypes.c_uint32)), 16,
                                       capi.ctypes.byref(n)) == capi.ERR_ARG
    assert n.value == 1
    assert L.lbm_debug_pack_work_items(None, 3, None, 0, capi.ctypes.byref(n)) == capi.ERR_ARG
