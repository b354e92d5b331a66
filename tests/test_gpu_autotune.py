"""The step-kernel autotuner (block_cells = LBM_BLOCK_AUTO): a measured choice between the
tile kernel and the TMA brick kernel, cached in the process and in LBM_AUTOTUNE_CACHE.

The two kernels give bit-identical states, so an autotuned context must match one with
the kernel given explicitly, whatever was chosen.
"""
import os

import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


FACES = I.Geometry(64, 20, 16, np.array([[61.3, 9.6, 8.7, 6.2], [20.0, 3.0, 14.5, 4.1]]))


def _kw(capi, g, **extra):
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.62, delta_rho=3e-4, collision=capi.TRT, wall=capi.CLI,
              storage=capi.F32)
    kw.update(extra)
    return kw


def _lines(path):
    with open(path) as f:
        return [ln.rstrip("\n").split("\t") for ln in f if ln.strip()]


def test_measured_cached_and_forced(capi, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(cache))
    # SBB walls: a key no other test tunes, so the first creation measures
    kw = _kw(capi, FACES, wall=capi.SBB, block_cells=capi.BLOCK_AUTO)
    with capi.Context(**kw) as ctx:
        info = ctx.info()
    assert info["autotune"] == 1 and info["block_cells"] in (128, 256)
    assert info["tune_ms_tiles"] > 0 and info["tune_ms_bricks"] > 0
    chosen = 256 if info["tune_ms_bricks"] < info["tune_ms_tiles"] else 128
    assert info["block_cells"] == chosen
    rows = _lines(cache)
    assert len(rows) == 1 and rows[0][0].startswith("64x20x16 fluid=") and int(rows[0][1]) == chosen

    with capi.Context(**kw) as ctx:                      # the process cache answers
        info2 = ctx.info()
    assert info2["autotune"] == 2 and info2["block_cells"] == chosen
    assert len(_lines(cache)) == 1

    other = 384 - chosen                                 # a file entry overrides the process cache
    forced = tmp_path / "forced.txt"
    forced.write_text(f"{rows[0][0]}\t{other}\t1.0\t2.0\n")
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(forced))
    with capi.Context(**kw) as ctx:
        info3 = ctx.info()
    assert info3["autotune"] == 2 and info3["block_cells"] == other
    assert info3["tune_ms_tiles"] == 1.0 and info3["tune_ms_bricks"] == 2.0


@pytest.mark.parametrize("case", ["AA", "ragged"])
def test_tiles_only_where_bricks_cannot_run(capi, monkeypatch, case):
    monkeypatch.delenv("LBM_AUTOTUNE_CACHE", raising=False)
    if case == "AA":
        kw = _kw(capi, FACES, layout=capi.LAYOUT_AA, block_cells=capi.BLOCK_AUTO)
    else:
        g = I.centred_sphere(24, 7.0)                     # nx = 24: no bricks
        kw = _kw(capi, g, block_cells=capi.BLOCK_AUTO)
    with capi.Context(**kw) as ctx:
        info = ctx.info()
    assert info["autotune"] in (1, 2) and info["block_cells"] == 128
    assert info["tune_ms_tiles"] > 0 and info["tune_ms_bricks"] == 0


def test_autotuned_state_equals_given_kernel(capi, orc, monkeypatch):
    monkeypatch.delenv("LBM_AUTOTUNE_CACHE", raising=False)
    solid = orc.voxelize(FACES.shape, FACES.spheres)
    _, w, _ = orc.lattice()
    f0 = w[:, None, None, None] * (1.0 + 1e-3 * I.noise((19,) + solid.shape, 5))
    f0[:, solid == 1] = 0.0
    out = []
    for block in (capi.BLOCK_AUTO, 128):
        with capi.Context(**_kw(capi, FACES, block_cells=block)) as ctx:
            ctx.set_populations(f0)
            ctx.step(17)
            out.append((ctx.get_populations(), ctx.observables()["U_sup"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
