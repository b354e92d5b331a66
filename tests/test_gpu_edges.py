"""Degenerate geometries against the oracle, as flag fields with SBB walls:

* boxes one to three cells thick, where every neighbour is a periodic image of the cell
  itself or of its one neighbour, so every x-face fix-up and periodic wrap is exercised
  on every lane;
* a box with no solid cell;
* a one-cell fluid gap between two wall planes (every pull across z hits a wall);
* a box with no fluid cell, which must step without error and stay empty.

Both layouts; FP64 to 1e-12 and FP32 to 1e-5 per population after a fixed step count.
"""
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


def _box(nz, ny, nx, walls=()):
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    for z in walls:
        solid[z] = 1
    return solid


GEOMS = {
    "1x6x5": _box(5, 6, 1),
    "2x2x2": _box(2, 2, 2),
    "3x1x7": _box(7, 1, 3),
    "gap_1": _box(3, 4, 5, walls=(0, 2)),       # one fluid plane between two wall planes
    "channel": _box(6, 3, 9, walls=(0,)),
}


def _perturbed(orc, solid, seed):
    _, w, _ = orc.lattice()
    f = w[:, None, None, None] * (1.0 + 1e-3 * I.noise((19,) + solid.shape, seed))
    f[:, solid == 1] = 0.0
    return f


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("layout", ["AB", "AA"])
@pytest.mark.parametrize("storage", ["F64", "F32"])
@pytest.mark.parametrize("coll", ["TRT", "MRT"])
def test_degenerate_boxes_match_oracle(capi, orc, geom, layout, storage, coll):
    solid = GEOMS[geom]
    nz, ny, nx = solid.shape
    f0 = _perturbed(orc, solid, 5)
    kw = dict(tau=0.62, delta_rho=3e-4, magic_lambda=0.21, collision=getattr(capi, coll), wall=capi.SBB)
    n = 13
    with capi.Context(flags=solid, shape=solid.shape, storage=getattr(capi, storage),
                      layout=getattr(capi, "LAYOUT_" + layout), **kw) as ctx:
        assert ctx.info()["n_fluid"] == int((solid == 0).sum())
        ctx.set_populations(f0)
        ctx.step(n)
        f = ctx.get_populations()
        obs = ctx.observables()
    fref, sums, _ = orc.run(solid, f0, n, **kw)
    fluid = solid == 0
    err = np.abs(f - fref)[:, fluid].max() / np.abs(fref)[:, fluid].max()
    assert err <= (1e-12 if storage == "F64" else 1e-5), err
    assert np.all(f[:, solid == 1] == 0.0)
    assert obs["U_sup"] == pytest.approx(sums[1] / solid.size, rel=1e-9 if storage == "F64" else 1e-3, abs=1e-15)


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_box_without_fluid(capi, layout):
    solid = np.ones((4, 5, 6), dtype=np.uint8)
    with capi.Context(flags=solid, shape=solid.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                      wall=capi.SBB, storage=capi.F32, layout=getattr(capi, "LAYOUT_" + layout)) as ctx:
        assert ctx.info()["n_fluid"] == 0
        ctx.init_equilibrium()
        ctx.step(7)
        obs = ctx.observables()
        assert obs["n_fluid"] == 0 and obs["U_sup"] == 0.0 and obs["porosity"] == 0.0
        assert np.all(ctx.get_populations() == 0.0)
