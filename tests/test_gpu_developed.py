"""Developed-flow time average (Sec. 4) through lbm_run_developed on the GPU.

A Stokes flow past the simple cubic array is steady: once developed, its time average is
the steady state itself, so U, K and the drag must agree with run_to_convergence, and
K* = K_app / K_D = 1 when K_D is that steady permeability.  The spin-up and averaging
schedule (flow-through time T = nx / U_sup, windows of one T sampled samples_per_ft
times) is replayed through the step / observables calls and must give the same average
bit for bit.
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


def _ctx(capi, **kw):
    g = I.centred_sphere(30, 9.0)    # r = 0.3 L (solid fraction chi = 0.6 read as 2r/L)
    base = dict(spheres=g.spheres, shape=g.shape, storage=capi.F64, tau=0.8, delta_rho=2e-5,
                magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    base.update(kw)
    return capi.Context(**base)


def test_steady_flow_average_is_the_steady_state(capi):
    # delta_rho large enough for short flow-through times, Re_p ~ 1: still a steady flow
    with _ctx(capi, delta_rho=2e-3) as c:
        c.init_equilibrium()
        st, _ = c.run_to_convergence(1e-12, 200, 400000)
        assert st == capi.OK
        ref = c.observables()
    with _ctx(capi, delta_rho=2e-3) as c:
        c.init_equilibrium()
        r = c.run_developed(min_spinup_ft=2, max_spinup_ft=2000, drag_tol=1e-11, average_ft=3, samples_per_ft=4,
                            K_darcy=ref["K"])
    assert r["status"] == capi.OK and r["developed"] == 1
    a = r["avg"]
    assert a["U_sup"] == pytest.approx(ref["U_sup"], rel=1e-9, abs=0)
    assert a["K_star"] == pytest.approx(1.0, rel=1e-9, abs=0)
    assert a["F_x"] == pytest.approx(ref["F_x"], rel=1e-9, abs=0)
    assert r["flow_through_steps"] == pytest.approx(30 / ref["U_sup"], rel=1e-9)
    assert r["average_ft"] == pytest.approx(3.0, rel=0.02)
    assert r["drag_change"] < 1e-11


def test_schedule_replayed_through_step_calls(capi):
    opts = dict(min_spinup_ft=1.5, max_spinup_ft=4.0, drag_tol=1e-30, average_ft=2.0, samples_per_ft=3)
    with _ctx(capi, storage=capi.F32, delta_rho=1e-4, tau=0.6) as c:
        c.init_equilibrium()
        r = c.run_developed(**opts)
    assert r["status"] == capi.OK and r["developed"] == 0        # tolerance never met
    with _ctx(capi, storage=capi.F32, delta_rho=1e-4, tau=0.6) as c:
        c.init_equilibrium()
        nx, ncell = 30, 30 ** 3
        c.step(nx)
        T = nx / abs(c.observables()["U_sup"])
        spin_ft, steps = nx / T, nx
        while True:
            sub = max(1, int(np.floor(T / opts["samples_per_ft"] + 0.5)))
            for _ in range(opts["samples_per_ft"]):
                c.step(sub)
            steps += sub * opts["samples_per_ft"]
            spin_ft += sub * opts["samples_per_ft"] / T
            T = nx / abs(c.observables()["U_sup"])
            if spin_ft >= opts["max_spinup_ft"]:
                break
        assert r["spinup_steps"] == steps
        sub = max(1, int(np.floor(T / opts["samples_per_ft"] + 0.5)))
        n = int(np.floor(opts["average_ft"] * opts["samples_per_ft"] + 0.5))
        sums = []
        for _ in range(n):
            c.step(sub)
            sums.append(c.observables()["U_sup"] * ncell)
        U = sum(sums) / n / ncell
    assert r["average_steps"] == n * sub
    assert r["avg"]["U_sup"] == pytest.approx(U, rel=1e-13, abs=0)   # U_sup * ncell round trip


def test_bad_options_and_flow_at_rest(capi):
    with _ctx(capi) as c:
        c.init_equilibrium()
        with pytest.raises(capi.LBMError):
            c.run_developed(samples_per_ft=0)
        with pytest.raises(capi.LBMError):
            c.run_developed(average_ft=0.0)
    with _ctx(capi, delta_rho=0.0) as c:
        c.init_equilibrium()
        with pytest.raises(capi.LBMError):
            c.run_developed()


def test_time_average_against_oracle(capi, orc):
    """lbm_average against the oracle's windowed average of U_sup and the drag (the same
    sampling schedule), FP64, from a seeded perturbed state."""
    g = I.Geometry(24, 20, 18, np.array([[11.3, 9.6, 8.7, 6.2]]))
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    _, w, _ = orc.lattice()
    f0 = w[:, None, None, None] * (1.0 + 1e-3 * I.noise((19,) + solid.shape, 13))
    f0[:, solid == 1] = 0.0
    kw = dict(tau=0.7, delta_rho=2e-4, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, **kw) as ctx:
        ctx.set_populations(f0)
        ctx.step(30)
        avg = ctx.average(6, 25)
    f, _, _ = orc.run(solid, f0, 30, q=q, **kw)
    _, U, F = orc.time_average(solid, f, 6, 25, q=q, **kw)
    assert avg["status"] == capi.OK and avg["steps"] == 30 + 150
    assert avg["U_sup"] == pytest.approx(U, rel=1e-9, abs=0)
    Fg = np.array([avg["F_x"], avg["F_y"], avg["F_z"]])
    assert np.abs(Fg - F).max() <= 1e-9 * np.abs(F).max() + 1e-15


def test_developed_average_against_oracle(capi, orc):
    """lbm_run_developed against the oracle's developed-flow average (the spin-up windows of
    one flow-through time, the drag test, the averaging schedule), FP64: the same spin-up and
    averaging step counts, U_sup and drag to 1e-9."""
    g = I.centred_sphere(16, 5.0)
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    kw = dict(tau=0.7, delta_rho=4e-3, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI)
    opts = dict(min_spinup_ft=2.0, max_spinup_ft=12.0, drag_tol=1e-4, average_ft=3.0, samples_per_ft=4,
                max_steps=200000)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, **kw) as ctx:
        ctx.init_equilibrium()
        r = ctx.run_developed(**opts)
    o = orc.developed_average(solid, orc.init_rest(solid), q=q, **opts, **kw)
    assert r["status"] == capi.OK and o["status"] == "ok"
    assert r["developed"] == int(o["developed"])
    assert r["spinup_steps"] == o["spinup_steps"] and r["average_steps"] == o["average_steps"]
    assert r["spinup_ft"] == pytest.approx(o["spinup_ft"], rel=1e-9)
    assert r["avg"]["U_sup"] == pytest.approx(o["U_sup"], rel=1e-9, abs=0)
    Fg = np.array([r["avg"]["F_x"], r["avg"]["F_y"], r["avg"]["F_z"]])
    assert np.abs(Fg - o["F"]).max() <= 1e-9 * np.abs(o["F"]).max() + 1e-15
