"""Full-size checks in the launch configuration bench.py times.

128^3 (the benchmark cell) and the 256^3 precision-study geometries are compared with the
FP64 oracle element by element over a few steps from a seeded perturbed state; the 512^3
cell, too large for the oracle's host memory in a test, is checked through properties
that hold at any size (rest state, mass conservation, mirror symmetry of the flow).
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


def _perturbed(orc, solid, seed, amp=1e-3):
    _, w, _ = orc.lattice()
    f = w[:, None, None, None] * (1.0 + amp * I.noise((19,) + solid.shape, seed))
    f[:, solid == 1] = 0.0
    return f


def _rel(a, b, solid):
    m = solid == 0
    return float(np.max(np.abs(a[:, m] - b[:, m]) / np.abs(b[:, m])))


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_bench_cell_128_fp32_against_oracle(capi, orc, layout):
    g = I.centred_sphere(128, 60.0)
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    f0 = _perturbed(orc, solid, 17)
    kw = dict(tau=0.6, delta_rho=2e-5, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F32,
                      layout=getattr(capi, "LAYOUT_" + layout), **kw) as ctx:
        assert np.array_equal(ctx.get_flags(), solid)
        ctx.set_populations(f0)
        ctx.step(21)
        f = ctx.get_populations()
        o = ctx.observables()
    Fref = np.zeros(3)
    ref, _, _ = orc.run(solid, f0, 21, q=q, force=Fref, **kw)
    assert _rel(f, ref, solid) <= 1e-5
    F = np.array([o["F_x"], o["F_y"], o["F_z"]])
    assert np.abs(F - Fref).max() <= 2e-4 * np.abs(Fref).max(), (F, Fref)


@pytest.mark.parametrize("fmt", ["F16DEV", "BF16DEV"])
@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_bench_cell_128_half_storage_against_oracle(capi, orc, fmt, layout):
    """The 16-bit deviation formats on the benchmark cell (the kernels of the 512^3 BF16 AA
    configuration at a size the oracle can run): two steps, each against one oracle step
    from the GPU's exported state before it, so that both in-place step kinds run at full
    size."""
    g = I.centred_sphere(128, 60.0)
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    _, w, _ = orc.lattice()
    s = 20
    dev, ulp = HB.storable(fmt, I.noise((19,) + solid.shape, 29) * 2e-4, s)
    f0 = w[:, None, None, None] + dev
    f0[:, solid == 1] = 0.0
    del dev
    kw = dict(tau=0.6, delta_rho=2e-5, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, fmt),
                      layout=getattr(capi, "LAYOUT_" + layout), dev_scale_log2=s if fmt == "F16DEV" else 0,
                      **kw) as ctx:
        ctx.set_populations(f0)
        prev = f0
        for i in range(2):
            ctx.step(1)
            f = ctx.get_populations()
            fref, _, _ = orc.run(solid, prev, 1, q=q, **kw)
            HB.check_step(orc, solid, w, f, fref, prev, ulp, walls=True)
            prev = f


@pytest.mark.parametrize("which", ["sphere", "pack40"])
def test_precision_geometries_256_against_oracle(capi, orc, which):
    g = I.centred_sphere(256, 120.0) if which == "sphere" else I.random_pack(256, 40, 18.0, 30.0, 20150811)
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    kw = dict(tau=0.6, delta_rho=2e-5, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F32, **kw) as ctx:
        assert np.array_equal(ctx.get_flags(), solid)
        qg = ctx.get_wall_distances()
        fin = np.isfinite(q)
        assert np.array_equal(np.isfinite(qg), fin)
        assert np.abs(qg[fin] - q[fin]).max() <= 1e-12
        del qg
        f0 = _perturbed(orc, solid, 23)
        ctx.set_populations(f0)
        ctx.step(3)
        f = ctx.get_populations()
    ref, _, _ = orc.run(solid, f0, 3, q=q, **kw)
    assert _rel(f, ref, solid) <= 1e-5


@pytest.mark.parametrize("storage", ["BF16DEV", "F32"])
def test_turbulent_cell_512_properties(capi, storage):
    g = I.centred_sphere(512, 240.0)
    # rest state: no drive, fluid at rest, stays exactly at rest
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, storage), layout=capi.LAYOUT_AA,
                      tau=0.505, delta_rho=0.0, collision=capi.TRT, wall=capi.CLI) as ctx:
        ctx.init_equilibrium()
        ctx.step(3)
        assert np.all(ctx.moment_sums() == 0.0)
        info = ctx.info()
        assert info["n_fluid"] == 512 ** 3 - int((ctx.get_flags() == 1).sum())
    # driven flow with SBB walls: mass conserved, flow along +x, mirror symmetric in y and z
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, storage), layout=capi.LAYOUT_AA,
                      tau=0.51, delta_rho=1e-3, collision=capi.TRT, wall=capi.SBB) as ctx:
        ctx.init_equilibrium()
        ctx.step(40)
        o = ctx.observables()
        s = ctx.moment_sums()
        assert o["status"] == capi.OK and o["U_sup"] > 0
        # 16-bit storage rounds every population every step: mass to its resolution
        tol = 1e-9 if storage == "F32" else 1e-6
        assert abs(s[0]) <= tol * o["n_fluid"]
        assert abs(s[2]) <= 1e-3 * abs(s[1]) and abs(s[3]) <= 1e-3 * abs(s[1])


def test_time_average_and_perturbed_start(capi):
    g = I.centred_sphere(64, 24.0)
    kw = dict(spheres=g.spheres, shape=g.shape, storage=capi.F32, tau=0.52, delta_rho=2e-4,
              collision=capi.TRT, wall=capi.CLI, perturb_u=0.01)
    with capi.Context(seed=5, **kw) as a, capi.Context(seed=5, **kw) as b, capi.Context(seed=6, **kw) as c:
        for ctx in (a, b, c):
            ctx.init_equilibrium()
        ua, ub, uc = a.get_velocity(), b.get_velocity(), c.get_velocity()
        fluid = a.get_flags() == 0
        assert np.array_equal(ua, ub) and not np.array_equal(ua, uc)       # seeded, deterministic
        assert np.abs(ua[:, fluid]).max() <= 0.01 * (1 + 1e-6)
        assert np.abs(ua[:, fluid]).max() > 0.009
        assert abs(ua[:, fluid].mean()) < 1e-4                             # centred perturbation
        assert abs(a.moment_sums()[0]) < 1e-6 * fluid.sum()                # rho = rho0 everywhere
        # the average of 4 samples of 50 steps equals the mean of the 4 sampled U values
        us, fs = [], []
        for _ in range(4):
            b.step(50)
            o = b.observables()
            us.append(o["U_sup"])
            fs.append(o["F_x"])
        avg = a.average(4, 50)
        assert avg["status"] == capi.OK and avg["steps"] == 200
        assert avg["U_sup"] == pytest.approx(np.mean(us), rel=1e-12, abs=0)
        assert avg["F_x"] == pytest.approx(np.mean(fs), rel=1e-12, abs=0)
