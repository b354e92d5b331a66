"""Drag force F_D (momentum exchange, Sec. 3) and drag coefficients on the GPU.

Element-by-element parity of F_D with the oracle runs inside the operator matrix of
test_gpu_parity.py and the 128^3 check of test_gpu_fullsize.py.  Here: the momentum
balance at the benchmark size in the benchmark's launch configuration (a property that
holds at any size), the dilute-array Stokes drag, and the host formulas of C_D and C_D,A.
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


def _shift_input(solid, delta_rho):
    """Momentum the periodic pressure shift adds in one step (fluid-to-fluid pulls across
    the x boundary, +-w_k delta_rho), from the flag field alone."""
    e = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                  [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
    w = np.where((e ** 2).sum(1) == 0, 1 / 3, np.where((e ** 2).sum(1) == 1, 1 / 18, 1 / 36))
    fluid = solid == 0
    S = np.zeros(3)
    for k in range(19):
        if e[k, 0] == 0:
            continue
        src = np.roll(fluid, shift=(e[k, 2], e[k, 1], e[k, 0]), axis=(0, 1, 2))
        xcol = 0 if e[k, 0] == 1 else fluid.shape[2] - 1
        n = int((fluid[:, :, xcol] & src[:, :, xcol]).sum())
        S += n * w[k] * delta_rho * e[k, 0] * e[k]
    return S


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_momentum_balance_bench_cell(capi, layout):
    """128^3, r = 60, TRT/CLI, FP32, the benchmark's launch configuration: the drag of a
    step equals the momentum the pressure shift adds minus the fluid's momentum gain,
    F = P(t) + S - P(t+1), P = rho0 * sum of u over fluid cells."""
    g = I.centred_sphere(128, 60.0)
    dr = 2e-5
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F32, layout=getattr(capi, "LAYOUT_" + layout),
                      tau=0.6, delta_rho=dr, magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI) as ctx:
        S = _shift_input(ctx.get_flags(), dr)
        ctx.init_equilibrium()
        # the first pair of steps: the drive has not yet reached the sphere (4 cells from
        # the x faces), so the walls see the rest state and F = 0 exactly
        for n in (1, 7, 120):
            ctx.step(n)
            P0 = ctx.moment_sums()[1:4]
            ctx.step(1)
            o = ctx.observables()
            P1 = ctx.moment_sums()[1:4]
            F = np.array([o["F_x"], o["F_y"], o["F_z"]])
            # FP32 arithmetic on deviations ~1e-5 over 1.2e6 cells: well inside 1e-4 of S
            assert np.abs(F - (P0 + S - P1)).max() <= 1e-4 * S[0], (F, P0 + S - P1)
            assert F[0] == 0.0 if n == 1 else F[0] > 0.01 * S[0]


def test_dilute_array_stokes_drag(capi):
    """One sphere of r = 6 in a 48^3 periodic cell (solid fraction 0.0082): C_D of the
    converged Stokes flow against the dilute simple-cubic-array series
    1/(1 - 1.7601 c^(1/3) + c - 1.5593 c^2) (Hasimoto 1959; Sangani & Acrivos 1982)."""
    L, r, tau, dr = 48, 6.0, 1.5, 1e-6
    g = I.centred_sphere(L, r)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, tau=tau, delta_rho=dr,
                      magic_lambda=3 / 16, collision=capi.TRT, wall=capi.CLI) as ctx:
        ctx.init_equilibrium()
        st, _ = ctx.run_to_convergence(1e-9, 500, 200000)
        assert st == capi.OK
        o = ctx.observables()
    assert o["F_x"] == pytest.approx(dr / 3.0 * L * L, rel=1e-6)        # steady: F balances dp A
    assert abs(o["F_y"]) <= 1e-9 * o["F_x"] and abs(o["F_z"]) <= 1e-9 * o["F_x"]
    c = 4.0 / 3.0 * np.pi * r ** 3 / L ** 3
    cd_series = 1.0 / (1.0 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)
    assert o["C_D"] == pytest.approx(cd_series, rel=0.01)


def test_drag_coefficients_host_formulas(capi, orc):
    g = I.random_pack(40, 5, 3.0, 6.0, 3)
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F32, tau=0.7, delta_rho=1e-4,
                      collision=capi.TRT, wall=capi.CLI) as ctx:
        ctx.init_equilibrium()
        o0 = ctx.observables()               # no step yet: no drag
        assert np.isnan(o0["F_x"]) and np.isnan(o0["C_D"])
        ctx.step(30)
        o = ctx.observables()
    rs = sum(s[3] for s in g.spheres)
    area = sum(np.pi * s[3] ** 2 for s in g.spheres)
    cd, cda = orc.drag_coefficients(o["F_x"], o["U_sup"], 0.7, r_sum=rs, area_sum=area)
    assert o["C_D"] == pytest.approx(cd, rel=1e-12, abs=0)
    assert o["C_D_A"] == pytest.approx(cda, rel=1e-12, abs=0)
