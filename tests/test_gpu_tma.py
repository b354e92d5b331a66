"""The TMA brick kernel against the tile kernel: the same cells, the same arithmetic, so the
states must agree bit for bit after any number of steps (the reducing step runs the tile
kernel in both, so the observables agree too).  Every storage format, collision operator
and wall rule family, on boxes whose spheres cross the periodic faces (wrapped pulls read
directly) and a box of many spheres (partly solid bricks).  The oracle comparisons of the
other GPU tests run the default tile kernel, so the bricks are checked against the oracle
through this equality.
"""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GEOMS = {
    # sphere crossing the x, y and z faces
    "faces": I.Geometry(64, 20, 16, np.array([[61.3, 9.6, 8.7, 6.2], [20.0, 3.0, 14.5, 4.1]])),
    "pack": I.random_pack(32, 6, 3.0, 6.0, 11),
}


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


def _run(capi, g, block, f0, steps, **kw):
    with capi.Context(spheres=g.spheres, shape=g.shape, block_cells=block, **kw) as ctx:
        info = ctx.info()
        ctx.set_populations(f0)
        out = []
        for n in steps:
            ctx.step(n)
            o = ctx.observables()
            out.append((ctx.get_populations(), [o["U_sup"], o["F_x"], o["F_y"], o["F_z"], o["mass"]]))
    return info, out


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("storage", ["F64", "F32", "F16DEV", "BF16DEV"])
@pytest.mark.parametrize("coll,wall", [("TRT", "CLI"), ("SRT", "SBB"), ("MRT", "CLI"), ("TRT", "QIBB"),
                                       ("TRT", "IEBB")])
def test_bricks_equal_tiles_bitwise(capi, orc, geom, storage, coll, wall):
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    _, w, _ = orc.lattice()
    f0 = w[:, None, None, None] * (1.0 + 1e-3 * I.noise((19,) + solid.shape, 21))
    f0[:, solid == 1] = 0.0
    kw = dict(tau=0.62, delta_rho=3e-4, magic_lambda=3 / 16, collision=getattr(capi, coll),
              wall=getattr(capi, wall), storage=getattr(capi, storage))
    steps = (1, 6, 25)
    it, tiles = _run(capi, g, 128, f0, steps, **kw)
    ib, bricks = _run(capi, g, 256, f0, steps, **kw)
    assert it["block_cells"] == 128 and ib["block_cells"] == 256
    for (a, oa), (b, ob) in zip(tiles, bricks):
        assert np.array_equal(a, b)
        assert oa == ob


def test_kernel_choice(capi):
    g = GEOMS["faces"]
    with capi.Context(spheres=g.spheres, shape=g.shape, tau=0.7) as ctx:
        assert ctx.info()["block_cells"] == 128                       # default: tiles of fluid cells
    with capi.Context(spheres=g.spheres, shape=g.shape, tau=0.7, block_cells=256) as ctx:
        assert ctx.info()["block_cells"] == 256
    g2 = I.centred_sphere(24, 7.0)
    with pytest.raises(capi.LBMError):                                # nx = 24: no bricks
        capi.Context(spheres=g2.spheres, shape=g2.shape, tau=0.7, block_cells=256)
    with pytest.raises(capi.LBMError):                                # AA: no bricks
        capi.Context(spheres=g.spheres, shape=g.shape, tau=0.7, layout=capi.LAYOUT_AA, block_cells=256)
