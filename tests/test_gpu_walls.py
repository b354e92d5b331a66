"""Interpolated wall rules LIBB, QIBB, IEBB and MR (Sec. 2.2.1) on the GPU against the
FP64 oracle, element by element, from a seeded perturbed state: every collision operator,
FP64 and FP32 storage, a ragged box and a box whose sphere crosses the periodic faces
(links whose x_f2 and x_f3 lie across the x faces, and one-cell gaps that exercise the
fallbacks).  The drag of the last step is compared too, and a thin slit (every link falls
back) and a batch mixing rules are checked against running alone.
"""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RAGGED = I.Geometry(24, 20, 18, np.array([[11.3, 9.6, 8.7, 6.2]]))
STAGED = I.Geometry(64, 20, 18, np.array([[61.3, 9.6, 8.7, 6.2], [20.0, 3.0, 16.5, 4.1]]))
# two spheres 1.6 cells apart: x_f2 / x_f3 solid on some links (fallbacks)
GAPPY = I.Geometry(32, 24, 20, np.array([[10.0, 12.0, 10.0, 5.2], [22.0, 12.0, 10.0, 5.2]]))
GEOMS = {"ragged": RAGGED, "staged": STAGED, "gappy": GAPPY}


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


def _perturbed(orc, solid, seed, amp=1e-3):
    _, w, _ = orc.lattice()
    f = w[:, None, None, None] * (1.0 + amp * I.noise((19,) + solid.shape, seed))
    f[:, solid == 1] = 0.0
    return f


def _rel(a, b, solid):
    m = solid == 0
    return float(np.max(np.abs(a[:, m] - b[:, m]) / np.abs(b[:, m])))


@pytest.mark.parametrize("geom", sorted(GEOMS))
@pytest.mark.parametrize("storage", ["F64", "F32"])
@pytest.mark.parametrize("coll", ["SRT", "TRT", "MRT"])
@pytest.mark.parametrize("wall", ["LIBB", "QIBB", "IEBB", "MR"])
def test_interpolated_wall_parity(capi, orc, geom, storage, coll, wall):
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    f0 = _perturbed(orc, solid, 13)
    kw = dict(tau=0.66, delta_rho=3e-4, magic_lambda=3 / 16, collision=getattr(capi, coll),
              wall=getattr(capi, wall))
    n = 31
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, storage), **kw) as ctx:
        ctx.set_populations(f0)
        ctx.step(n)
        f = ctx.get_populations()
        o = ctx.observables()
    Fref = np.zeros(3)
    fref, sums, _ = orc.run(solid, f0, n, q=q, force=Fref, **kw)
    tol = 1e-12 if storage == "F64" else 1e-5
    assert _rel(f, fref, solid) <= tol
    assert o["U_sup"] == pytest.approx(sums[1] / g.n_cells, rel=1e-9 if storage == "F64" else 1e-3, abs=0)
    F = np.array([o["F_x"], o["F_y"], o["F_z"]])
    ftol = 1e-9 if storage == "F64" else 2e-4
    assert np.abs(F - Fref).max() <= ftol * np.abs(Fref).max() + 1e-13, (F, Fref)


def test_fallback_slit_every_rule_is_bounce_back(capi, orc):
    """One fluid row: every link's x_f2 is solid; with q < 1/2 every rule is SBB."""
    e, _, _ = orc.lattice()
    s = I.slit_channel(1, nx=32, nz=4)
    q = np.full((19,) + s.shape, np.nan)
    for k in range(19):
        if e[k, 1] != 0:
            q[k, :, 1, :] = 0.3
    f0 = _perturbed(orc, s, 3)
    out = {}
    for wall in ("SBB", "CLI", "LIBB", "QIBB", "IEBB", "MR"):
        with capi.Context(flags=s, q=q, shape=s.shape, storage=capi.F64, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                          wall=getattr(capi, wall)) as ctx:
            ctx.set_populations(f0)
            ctx.step(4)
            out[wall] = ctx.get_populations()
    for wall in ("CLI", "LIBB", "QIBB", "IEBB", "MR"):
        assert np.array_equal(out[wall], out["SBB"]), wall


def test_batch_mixing_rules_equals_alone(capi):
    geoms = [I.centred_sphere(24, 8.0), I.centred_sphere(32, 11.0), I.centred_sphere(28, 9.5)]
    walls = [capi.QIBB, capi.CLI, capi.IEBB]
    keep = [capi.make_desc(spheres=gg.spheres, shape=gg.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                           wall=w, storage=capi.F32) for gg, w in zip(geoms, walls)]
    descs = [d for d, _ in keep]
    b = capi.Batch(descs)
    b.init_equilibrium()
    b.step(40)
    mix = [(b.get_populations(i), b.observables(i)) for i in range(len(descs))]
    b.close()
    for i, d in enumerate(descs):
        with capi.Context(desc=d) as ctx:
            ctx.init_equilibrium()
            ctx.step(40)
            assert np.array_equal(ctx.get_populations(), mix[i][0])
            o = ctx.observables()
            assert o["U_sup"] == mix[i][1]["U_sup"] and o["F_x"] == mix[i][1]["F_x"]
