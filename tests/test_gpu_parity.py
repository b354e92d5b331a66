"""GPU path vs FP64 CPU oracle, element by element, on the same seeded inputs.

Every call goes through the C ABI (ctypes binding).  Tolerances: FP64 storage 1e-12
relative per population, FP32 storage 1e-5 relative per population; FP16/BF16
deviation storage one unit in the last place of the stored format per step (the FP32
collision error is far below that unit).

Velocity sums: u is a difference of populations ~0.05 that cancel to ~1e-5, so a
population rounding of ~1e-17 is ~1e-12 of u on either side (the oracle works on full
f, the GPU on deviations f - w).  U and K are therefore compared at 1e-9 relative in
FP64 (the permeability requirement is 1e-3).
"""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

import half_bounds as HB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


def _fluid(solid):
    return solid == 0


def rel_err(a, b, solid):
    m = _fluid(solid)
    return float(np.max(np.abs(a[:, m] - b[:, m]) / np.abs(b[:, m])))


RAGGED = I.Geometry(24, 20, 18, np.array([[11.3, 9.6, 8.7, 6.2]]))   # rows of 24: direct loads
# rows a multiple of 32 (bulk-copy staged loads), ragged y/z, sphere crossing the periodic faces
STAGED = I.Geometry(64, 20, 18, np.array([[61.3, 9.6, 8.7, 6.2], [20.0, 3.0, 16.5, 4.1]]))
GEOMS = {"ragged": RAGGED, "staged": STAGED}


# ---------------------------------------------------------------------------------------
# Geometry: flags bit-exact, q to 1e-12
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("geom", [
    I.centred_sphere(32, 12.0),
    RAGGED,
    I.Geometry(20, 16, 12, np.array([[0.3, 15.2, 6.0, 5.1], [10.0, 8.0, 6.0, 3.3]])),  # periodic images
    I.random_pack(48, 6, 4.0, 7.0, 7),
])
def test_geometry_parity(capi, orc, geom):
    with capi.Context(spheres=geom.spheres, shape=geom.shape, wall=capi.CLI) as ctx:
        flags = ctx.get_flags()
        q = ctx.get_wall_distances()
        info = ctx.info()
    solid = orc.voxelize(geom.shape, geom.spheres)
    qref = orc.wall_distances(solid, geom.spheres)
    assert np.array_equal(flags, solid)
    assert np.array_equal(np.isfinite(q), np.isfinite(qref))
    fin = np.isfinite(qref)
    assert np.abs(q[fin] - qref[fin]).max() <= 1e-12
    assert info["n_fluid"] == int((solid == 0).sum())
    assert info["n_links"] == int(fin.sum())


def test_geometry_from_flags_and_q(capi, orc):
    geom = RAGGED
    solid = orc.voxelize(geom.shape, geom.spheres)
    qref = orc.wall_distances(solid, geom.spheres)
    with capi.Context(flags=solid, q=np.nan_to_num(qref, nan=0.5), shape=geom.shape, wall=capi.CLI) as ctx:
        assert np.array_equal(ctx.get_flags(), solid)
        q = ctx.get_wall_distances()
    fin = np.isfinite(qref)
    assert np.array_equal(np.isfinite(q), fin)
    assert np.abs(q[fin] - qref[fin]).max() == 0.0


# ---------------------------------------------------------------------------------------
# The reference workload: 32^3, r = 12, TRT Lambda 3/16, SBB, FP64, 2000 steps
# ---------------------------------------------------------------------------------------
def test_reference_32_fp64_2000_steps(capi, orc):
    cfg = I.config_reference_32()
    g = cfg["geometry"]
    kw = dict(tau=cfg["tau"], delta_rho=cfg["delta_rho"], magic_lambda=cfg["magic_lambda"],
              collision=capi.TRT, wall=capi.SBB)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, **kw) as ctx:
        ctx.init_equilibrium()
        ctx.step(cfg["steps"])
        f = ctx.get_populations()
        obs = ctx.observables()
    solid = orc.voxelize(g.shape, g.spheres)
    fref, sums, _ = orc.run(solid, orc.init_rest(solid), cfg["steps"], **kw)
    assert rel_err(f, fref, solid) <= 1e-12
    U = sums[1] / g.n_cells
    assert obs["U_sup"] == pytest.approx(U, rel=1e-9, abs=0)
    K = orc.observables(U, cfg["tau"], cfg["delta_rho"], g.nx, g.d_p)[1]
    assert obs["K"] == pytest.approx(K, rel=1e-9, abs=0)
    # the oracle sums ~5e5 full populations (its rounding ~1e-13); the GPU sums deviations
    assert obs["mass"] == pytest.approx(sums[0], rel=1e-11, abs=0)
    assert np.all(f[:, solid == 1] == 0.0)


# ---------------------------------------------------------------------------------------
# Operator x wall x storage x layout on a ragged box, from a seeded perturbed state
# ---------------------------------------------------------------------------------------
def _perturbed_state(orc, solid, amp, seed):
    _, w, _ = orc.lattice()
    xi = I.noise((19,) + solid.shape, seed)
    f = w[:, None, None, None] * (1.0 + amp * xi)
    f[:, solid == 1] = 0.0
    return f


@pytest.mark.parametrize("geom", ["ragged", "staged"])
@pytest.mark.parametrize("layout", ["AB", "AA"])
@pytest.mark.parametrize("storage", ["F64", "F32"])
@pytest.mark.parametrize("coll", ["SRT", "TRT", "MRT"])
@pytest.mark.parametrize("wall", ["SBB", "CLI"])
def test_step_parity_matrix(capi, orc, geom, layout, storage, coll, wall):
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    f0 = _perturbed_state(orc, solid, 1e-3, 11)
    kw = dict(tau=0.62, delta_rho=3e-4, magic_lambda=0.21, collision=getattr(capi, coll),
              wall=getattr(capi, wall))
    st = getattr(capi, storage)
    n = 41
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=st,
                      layout=getattr(capi, "LAYOUT_" + layout), **kw) as ctx:
        ctx.set_populations(f0)
        ctx.step(n)
        f = ctx.get_populations()
        obs = ctx.observables()
    Fref = np.zeros(3)
    fref, sums, _ = orc.run(solid, f0, n, q=q, force=Fref, **kw)
    tol = 1e-12 if storage == "F64" else 1e-5
    assert rel_err(f, fref, solid) <= tol
    assert obs["U_sup"] == pytest.approx(sums[1] / g.n_cells, rel=1e-9 if storage == "F64" else 1e-3, abs=0)
    # drag of the last step (momentum exchange): the GPU sums deviations, the oracle full
    # populations whose constant part cancels to ~1e-15 over the links
    F = np.array([obs["F_x"], obs["F_y"], obs["F_z"]])
    ftol = 1e-9 if storage == "F64" else 2e-4
    assert np.abs(F - Fref).max() <= ftol * np.abs(Fref).max() + 1e-13, (F, Fref)


@pytest.mark.parametrize("geom", ["ragged", "staged"])
@pytest.mark.parametrize("storage", ["F64", "F32", "F16DEV", "BF16DEV"])
@pytest.mark.parametrize("wall", ["SBB", "CLI"])
def test_aa_matches_ab_bitwise(capi, orc, geom, storage, wall):
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    f0 = _perturbed_state(orc, solid, 1e-3, 5)
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.7, delta_rho=2e-4, collision=capi.TRT,
              wall=getattr(capi, wall), storage=getattr(capi, storage))
    out = {}
    for lay in ("AB", "AA"):
        with capi.Context(layout=getattr(capi, "LAYOUT_" + lay), **kw) as ctx:
            ctx.set_populations(f0)
            res = []
            for n in (1, 1, 5, 12):
                ctx.step(n)
                o = ctx.observables()
                res.append((ctx.get_populations(), [o["F_x"], o["F_y"], o["F_z"], o["U_sup"]]))
            out[lay] = res
    for (a, oa), (b, ob) in zip(out["AB"], out["AA"]):
        assert np.array_equal(a, b)
        assert oa == ob


# ---------------------------------------------------------------------------------------
# Reduced-precision storage: within one unit in the last place of the format per step
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("geom", ["ragged", "staged"])
@pytest.mark.parametrize("fmt", ["F16DEV", "BF16DEV"])
@pytest.mark.parametrize("layout", ["AB", "AA"])
@pytest.mark.parametrize("coll", ["TRT", "MRT"])
@pytest.mark.parametrize("wall", ["SBB", "CLI"])
def test_half_storage_one_step(capi, orc, geom, fmt, layout, coll, wall):
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    _, w, _ = orc.lattice()
    s = 20
    dev, ulp = HB.storable(fmt, I.noise((19,) + solid.shape, 3) * 2e-4, s)
    f0 = w[:, None, None, None] + dev
    f0[:, solid == 1] = 0.0
    kw = dict(tau=0.66, delta_rho=2e-4, collision=getattr(capi, coll), wall=getattr(capi, wall))
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, fmt),
                      layout=getattr(capi, "LAYOUT_" + layout), dev_scale_log2=s if fmt == "F16DEV" else 0,
                      **kw) as ctx:
        ctx.set_populations(f0)
        assert np.abs(ctx.get_populations() - f0).max() < 1e-17       # import is exact
        ctx.step(1)
        f = ctx.get_populations()
    fref, _, _ = orc.run(solid, f0, 1, q=q, **kw)
    # from an imported state only CLI's own-cell part is rounded once more (SBB's is exact)
    HB.check_step(orc, solid, w, f, fref, f0, ulp, walls=(wall == "CLI"))


@pytest.mark.parametrize("geom", ["ragged", "staged"])
@pytest.mark.parametrize("fmt", ["F16DEV", "BF16DEV"])
@pytest.mark.parametrize("layout", ["AB", "AA"])
@pytest.mark.parametrize("coll", ["TRT", "MRT"])
@pytest.mark.parametrize("wall", ["SBB", "CLI"])
def test_half_storage_step_by_step(capi, orc, geom, fmt, layout, coll, wall):
    """Six consecutive steps (each AA step kind three times), each compared with one oracle
    step from the GPU's own exported state before it: the per-step bound holds at every step
    and in both in-place phases, without the growth a multi-step comparison would need."""
    g = GEOMS[geom]
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    _, w, _ = orc.lattice()
    s = 20
    dev, ulp = HB.storable(fmt, I.noise((19,) + solid.shape, 8) * 2e-4, s)
    f0 = w[:, None, None, None] + dev
    f0[:, solid == 1] = 0.0
    kw = dict(tau=0.66, delta_rho=2e-4, collision=getattr(capi, coll), wall=getattr(capi, wall))
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, fmt),
                      layout=getattr(capi, "LAYOUT_" + layout), dev_scale_log2=s if fmt == "F16DEV" else 0,
                      **kw) as ctx:
        ctx.set_populations(f0)
        prev = f0
        for i in range(6):
            ctx.step(1)
            f = ctx.get_populations()
            fref, _, _ = orc.run(solid, prev, 1, q=q, **kw)
            HB.check_step(orc, solid, w, f, fref, prev, ulp, walls=(i > 0 or wall == "CLI"))
            prev = f


# ---------------------------------------------------------------------------------------
# Exported fields and reductions
# ---------------------------------------------------------------------------------------
def test_velocity_and_moment_sums(capi, orc):
    g = RAGGED
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    kw = dict(tau=0.7, delta_rho=1e-4, collision=capi.TRT, wall=capi.CLI)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, **kw) as ctx:
        ctx.init_equilibrium()
        ctx.step(30)
        u = ctx.get_velocity()
        sums_state = ctx.moment_sums()
        obs = ctx.observables()
    _, sums, uref = orc.run(solid, orc.init_rest(solid), 30, q=q, want_u=True, **kw)
    scale = np.abs(uref).max()
    assert np.abs(u - uref).max() <= 1e-10 * scale
    assert sums_state[1] == pytest.approx(sums[1], rel=1e-9, abs=0)
    assert obs["U_sup"] == pytest.approx(sums[1] / g.n_cells, rel=1e-9, abs=0)


def test_mass_conservation_sbb(capi, orc):
    g = I.centred_sphere(32, 12.0)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, tau=0.8, delta_rho=1e-4,
                      collision=capi.TRT, wall=capi.SBB) as ctx:
        ctx.init_equilibrium()
        m0 = ctx.observables()["mass"]
        ctx.step(500)
        o = ctx.observables()
    assert abs(o["mass"] / m0 - 1) < 1e-13
    assert o["U_sup"] > 0


@pytest.mark.parametrize("geom", ["ragged", "staged"])
def test_checkpoint_restart_bitwise(capi, orc, tmp_path, geom):
    g = GEOMS[geom]
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
              wall=capi.CLI, storage=capi.F32)
    for lay in (capi.LAYOUT_AB, capi.LAYOUT_AA):
        with capi.Context(layout=lay, **kw) as a:
            a.init_equilibrium()
            a.step(37)
            a.save(str(tmp_path / "c.bin"))
            a.step(20)
            fa = a.get_populations()
        with capi.Context(layout=lay, **kw) as b:
            b.load(str(tmp_path / "c.bin"))
            assert b.info()["steps"] == 37
            b.step(20)
            fb = b.get_populations()
        assert np.array_equal(fa, fb)


def test_divergence_is_reported(capi):
    g = I.centred_sphere(16, 5.0)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F32, tau=0.5001, delta_rho=0.5,
                      collision=capi.SRT, wall=capi.SBB) as ctx:
        ctx.init_equilibrium()
        st, done = ctx.run_to_convergence(1e-8, 50, 5000)
        assert st == capi.ERR_DIVERGED
        assert done < 5000


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_batch_alone_vs_mix_bitwise(capi, layout):
    geoms = [I.centred_sphere(24, 8.0), RAGGED, I.centred_sphere(40, 15.0), STAGED, I.centred_sphere(64, 20.0)]
    descs_keep = [capi.make_desc(spheres=gg.spheres, shape=gg.shape, tau=0.6 + 0.05 * i, delta_rho=1e-4 * (i + 1),
                                 collision=capi.TRT, wall=capi.CLI, storage=capi.F16DEV,
                                 layout=getattr(capi, "LAYOUT_" + layout))
                  for i, gg in enumerate(geoms)]
    descs = [d for d, _ in descs_keep]
    b = capi.Batch(descs)
    b.init_equilibrium()
    b.step(160)                                   # the first 48 steps time the block shapes
    info = b.info()
    assert info["step_warps"] in (2, 4, 8) and info["shape_source"] in (1, 2)
    mix = [(b.get_populations(i), b.observables(i)) for i in range(len(geoms))]
    b.close()
    for i, d in enumerate(descs):
        with capi.Context(desc=d) as ctx:
            ctx.init_equilibrium()
            ctx.step(160)
            assert np.array_equal(ctx.get_populations(), mix[i][0])
            assert ctx.observables()["U_sup"] == mix[i][1]["U_sup"]


@pytest.mark.parametrize("n_inst", [64, 66])
def test_batch_tile_map_and_tile_records_bitwise(capi, n_inst):
    """Batches of up to 64 instances find each block's instance through the launch's tile map,
    larger ones through tile records: both give every instance the state it reaches alone,
    bit for bit (small cells of three shapes, in both layouts' kernels over 50 steps)."""
    shapes = [I.centred_sphere(8, 2.5), I.Geometry(12, 8, 8, np.array([[5.5, 4.0, 4.2, 2.7]])),
              I.Geometry(9, 10, 7, np.array([[1.0, 8.5, 3.0, 3.1]]))]
    for layout in ("AB", "AA"):
        keep = [capi.make_desc(spheres=shapes[i % 3].spheres, shape=shapes[i % 3].shape, tau=0.6 + 0.003 * i,
                               delta_rho=1e-4 * (1 + i % 5), collision=capi.TRT, wall=capi.CLI, storage=capi.F32,
                               layout=getattr(capi, "LAYOUT_" + layout)) for i in range(n_inst)]
        b = capi.Batch([d for d, _ in keep])
        b.init_equilibrium()
        b.step(50)
        check = (0, 1, n_inst // 2, n_inst - 2, n_inst - 1)
        mix = {i: b.get_populations(i) for i in check}
        b.close()
        for i in check:
            with capi.Context(desc=keep[i][0]) as ctx:
                ctx.init_equilibrium()
                ctx.step(50)
                assert np.array_equal(ctx.get_populations(), mix[i]), (layout, i)


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_batch_with_an_instance_without_fluid(capi, layout):
    """An instance without a fluid cell keeps one tile of padding in every launch shape, so
    the instances after it keep their tiles: each steps as it does alone, bit for bit."""
    solid = np.ones((4, 5, 6), dtype=np.uint8)
    lay = getattr(capi, "LAYOUT_" + layout)
    keep = [capi.make_desc(flags=solid, shape=solid.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                           wall=capi.CLI, storage=capi.F32, layout=lay)]
    for i, gg in enumerate([I.centred_sphere(8, 2.5), RAGGED]):
        keep.append(capi.make_desc(spheres=gg.spheres, shape=gg.shape, tau=0.65 + 0.05 * i, delta_rho=1e-4,
                                   collision=capi.TRT, wall=capi.CLI, storage=capi.F32, layout=lay))
    b = capi.Batch([d for d, _ in keep])
    b.init_equilibrium()
    b.step(60)
    assert np.all(b.get_populations(0) == 0.0)
    mix = [b.get_populations(i) for i in (1, 2)]
    b.close()
    for j, i in enumerate((1, 2)):
        with capi.Context(desc=keep[i][0]) as ctx:
            ctx.init_equilibrium()
            ctx.step(60)
            assert np.array_equal(ctx.get_populations(), mix[j]), i


def test_aa_batch_sets_one_instance_only_in_step0_arrangement(capi, orc):
    """The instances of an in-place batch share one arrangement: one instance's state can be
    set after an even number of steps (and steps on alike), not after an odd one."""
    geoms = [I.centred_sphere(24, 8.0), RAGGED]
    keep = [capi.make_desc(spheres=gg.spheres, shape=gg.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                           wall=capi.CLI, storage=capi.F32, layout=capi.LAYOUT_AA) for gg in geoms]
    b = capi.Batch([d for d, _ in keep])
    try:
        b.init_equilibrium()
        b.step(3)
        f1 = b.get_populations(1)
        with pytest.raises(capi.LBMError) as e:
            b.set_populations(1, f1)
        assert e.value.status == capi.ERR_STATE
        b.step(1)
        f1 = b.get_populations(1)
        b.set_populations(1, f1)                  # even: allowed, and a no-op on the state
        assert np.array_equal(b.get_populations(1), f1)
        b.step(6)
        with capi.Context(desc=keep[1][0]) as ctx:
            ctx.init_equilibrium()
            ctx.step(10)
            assert np.array_equal(ctx.get_populations(), b.get_populations(1))
    finally:
        b.close()


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_block_shapes_give_the_same_state(capi, layout):
    """The online shape tuner times three block shapes on the live state (4, 2 and 8 warps per
    block): a run whose first 48 steps went through all of them equals, bit for bit, a run in
    short calls that never tunes."""
    g = STAGED
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.64, delta_rho=2e-4, collision=capi.TRT, wall=capi.CLI,
              storage=capi.F32, layout=getattr(capi, "LAYOUT_" + layout))
    with capi.Context(**kw) as a, capi.Context(**kw) as b:
        a.init_equilibrium()
        b.init_equilibrium()
        a.step(200)
        ia = a.info()
        assert ia["shape_source"] in (1, 2) and ia["step_warps"] in (2, 4, 8)
        for _ in range(5):
            b.step(40)                             # calls of at most 48 steps: no tuning here
        assert np.array_equal(a.get_populations(), b.get_populations())
        assert a.observables()["U_sup"] == b.observables()["U_sup"]
