"""Storage formats against the FP64 oracle in permeability (the mixed-precision study's
requirement: at most 1e-3 relative in the Darcy regime).

The 32^3 simple-cubic cell (one sphere of r = 12, porosity 0.78), TRT with Lambda = 3/16
and CLI walls, tau = 0.8 and a pressure drop for Re_p ~ 1.  The oracle runs from rest until
the volume-averaged velocity changes by less than 1e-10 relative between checks 200 steps
apart; each GPU format runs the same steps from rest, then averages U over ten further
windows of 100 steps (lbm_average: the stochastically rounded 16-bit formats fluctuate at the
level of their last unit), and K = mu U / (delta_p / L_x) (Eq. Darcy) is compared with the
oracle's."""
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


@pytest.fixture(scope="module")
def oracle_state(orc):
    g = I.centred_sphere(32, 12.0)
    solid = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(solid, g.spheres)
    kw = dict(tau=0.8, delta_rho=2e-3, magic_lambda=3 / 16, collision=orc.TRT, wall=orc.CLI)
    f = orc.init_rest(solid)
    U_old, n = None, 0
    while n < 20000:
        f, sums, _ = orc.run(solid, f, 200, q=q, **kw)
        n += 200
        U = sums[1] / g.n_cells
        if U_old is not None and abs(U - U_old) < 1e-10 * abs(U):
            break
        U_old = U
    assert n < 20000, "oracle did not reach its steady state"
    obs = orc.observables(U, kw["tau"], kw["delta_rho"], g.nx, g.d_p)
    return g, kw, n, obs


@pytest.mark.parametrize("storage,tol", [("F64", 1e-9), ("F32", 1e-3), ("F16DEV", 1e-3), ("BF16DEV", 1e-3)])
@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_permeability_per_format_against_oracle(capi, oracle_state, storage, tol, layout):
    g, kw, n, obs = oracle_state
    K_ref, Re_p = obs[1], obs[2]
    assert 0.5 < Re_p < 2.0                                # the Re_p ~ 1 point
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=getattr(capi, storage),
                      layout=getattr(capi, "LAYOUT_" + layout), tau=kw["tau"], delta_rho=kw["delta_rho"],
                      magic_lambda=kw["magic_lambda"], collision=capi.TRT, wall=capi.CLI) as ctx:
        ctx.init_equilibrium()
        ctx.step(n)
        avg = ctx.average(10, 100)
    assert avg["status"] == capi.OK
    assert abs(avg["K"] / K_ref - 1.0) <= tol, (storage, avg["K"], K_ref)
