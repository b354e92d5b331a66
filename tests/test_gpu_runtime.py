"""GPU tests of the runtime around the step: convergence to the oracle's steady state,
observables, the serving loop (admission by memory footprint, continuous batching,
results identical to the same point run alone) and error paths of the server."""
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


def _oracle_steady_U(orc, geom, tol, chunk, max_steps, **kw):
    s = orc.voxelize(geom.shape, geom.spheres)
    q = orc.wall_distances(s, geom.spheres)
    f = orc.init_rest(s)
    U_old, n = None, 0
    while n < max_steps:
        f, sums, _ = orc.run(s, f, chunk, q=q, **kw)
        n += chunk
        U = sums[1] / geom.n_cells
        if U_old is not None and abs(U - U_old) < tol * abs(U):
            return U, n
        U_old = U
    raise AssertionError("oracle did not converge")


@pytest.mark.parametrize("wall", ["SBB", "CLI"])
def test_run_to_convergence_matches_oracle_steady_state(capi, orc, wall):
    g = I.centred_sphere(16, 6.0)
    kw = dict(tau=0.8, delta_rho=1e-5, magic_lambda=3 / 16, collision=capi.TRT, wall=getattr(capi, wall))
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, **kw) as ctx:
        ctx.init_equilibrium()
        st, steps = ctx.run_to_convergence(1e-10, 200, 40000)
        assert st == capi.OK
        obs = ctx.observables()
    U, n = _oracle_steady_U(orc, g, 1e-10, 200, 40000, **kw)
    assert steps == n                        # same check points, same decision
    assert obs["U_sup"] == pytest.approx(U, rel=1e-9, abs=0)
    K = orc.observables(U, 0.8, 1e-5, 16, 12.0)[1]
    assert obs["K"] == pytest.approx(K, rel=1e-9, abs=0)
    assert obs["Re_p"] == pytest.approx(U * 12.0 / ((0.8 - 0.5) / 3), rel=1e-12)


def _point(capi, L, r, tau, dr, layout="AB"):
    g = I.centred_sphere(L, r)
    return capi.make_desc(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=dr, collision=capi.TRT,
                          wall=capi.CLI, storage=capi.F32, layout=getattr(capi, "LAYOUT_" + layout))


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_server_results_equal_alone_and_continuous_batching(capi, layout):
    """Points are built by the admission thread while others step; in-place (AA) points join
    their group at chunk boundaries (even step counts).  Each result equals the same point
    run alone through a context, bit for bit."""
    import time
    pts = [(24, 8.0, 0.7, 1e-4), (32, 11.0, 0.6, 5e-5), (40, 13.0, 0.8, 2e-4), (24, 9.5, 0.9, 1e-4),
           (32, 10.0, 0.75, 1e-4), (40, 16.0, 0.65, 3e-5)]
    keep = [_point(capi, *p, layout=layout) for p in pts]
    # budget for about three points at a time: the rest queue and are admitted as others retire
    foot = 2 * 19 * 4 * 40 ** 3 + 2 * 2 ** 20
    srv = capi.Server(hbm_budget_bytes=3 * foot, check_interval=100, max_resident=8)
    try:
        ids = []
        for i, (d, _) in enumerate(keep):
            ids.append(srv.submit(d, 1e-6, 30000))
            if i == 2:
                time.sleep(0.2)                         # later arrivals join a running batch
        srv.drain(600.0)
        res = [srv.poll(i) for i in ids]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["completed"] == len(pts) and stats["failed"] == 0
    assert stats["mlups"] > 0
    lat = np.array([r[2] for r in res])
    assert np.all(lat > 0)
    for (st, obs, _), (d, _) in zip(res, keep):
        assert st == capi.OK
        with capi.Context(desc=d) as ctx:
            ctx.init_equilibrium()
            st2, steps = ctx.run_to_convergence(1e-6, 100, 30000)
            o = ctx.observables()
        assert st2 == capi.OK
        assert obs["steps"] == steps
        assert obs["U_sup"] == o["U_sup"] and obs["K"] == o["K"]


def test_server_rejects_point_over_budget(capi):
    d, keep = _point(capi, 64, 20.0, 0.7, 1e-4)
    srv = capi.Server(hbm_budget_bytes=1 << 20, check_interval=100)
    try:
        with pytest.raises(capi.LBMError) as e:
            srv.submit(d, 1e-6, 1000)
        assert e.value.status == capi.ERR_NO_MEMORY
    finally:
        srv.close()


def test_server_reports_not_converged(capi):
    d, keep = _point(capi, 24, 8.0, 0.7, 1e-4)
    srv = capi.Server(hbm_budget_bytes=1 << 30, check_interval=100)
    try:
        rid = srv.submit(d, 1e-14, 300)
        srv.drain(120.0)
        st, obs, lat = srv.poll(rid)
        assert st == capi.ERR_NOT_CONVERGED and obs["steps"] == 300
    finally:
        srv.close()
