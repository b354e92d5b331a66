"""Failure paths exercised from the host, without faulting the GPU.

* Every device allocation a context makes is failed in turn (lbm_debug_fail_alloc_after):
  creation must report LBM_ERR_NO_MEMORY, release what it had taken (the free device memory
  returns to where it was) and leave the library usable.
* A resident request that fails to build (injected out-of-memory) is reported and the
  server keeps serving the others.
* Requests are cancelled while queued and while resident.
* A flow driven past stability is reported as diverged (the divergence flag).
"""
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
    yield C
    C.debug_fail_alloc_after(-1)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("storage,layout,wall", [("F32", "AB", "CLI"), ("F64", "AA", "CLI"),
                                                  ("BF16DEV", "AB", "QIBB")])
def test_every_allocation_failure_is_clean(capi, storage, layout, wall):
    g = I.random_pack(32, 5, 3.0, 6.0, 2)
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.7, delta_rho=1e-4, storage=getattr(capi, storage),
              layout=getattr(capi, "LAYOUT_" + layout), wall=getattr(capi, wall), collision=capi.TRT)
    with capi.Context(**kw) as ctx:       # warm-up: first-use allocations of the runtime
        ctx.init_equilibrium()
        ctx.step(3)
    before = _free_bytes()
    failures = 0
    for n in range(200):
        capi.debug_fail_alloc_after(n)
        try:
            with capi.Context(**kw) as ctx:
                ctx.init_equilibrium()
                ctx.step(3)
                ctx.observables()
            break                                # n allocations suffice: all paths covered
        except capi.LBMError as e:
            assert e.status == capi.ERR_NO_MEMORY, e
            failures += 1
        finally:
            capi.debug_fail_alloc_after(-1)
    assert 5 <= failures < 200
    after = _free_bytes()
    assert after >= before - (8 << 20)           # nothing leaked beyond allocator granularity
    with capi.Context(**kw) as ctx:              # and the library still works
        ctx.init_equilibrium()
        ctx.step(10)
        assert ctx.observables()["U_sup"] > 0


def _point(capi, L, r):
    g = I.centred_sphere(L, r)
    return capi.make_desc(spheres=g.spheres, shape=g.shape, tau=0.7, delta_rho=1e-4, collision=capi.TRT,
                          wall=capi.CLI, storage=capi.F32)


def _wait(srv, rid, limit=60.0):
    import time
    t0 = time.time()
    while True:
        r = srv.poll(rid)
        if r is not None:
            return r
        assert time.time() - t0 < limit
        time.sleep(0.05)


def test_server_cancel_queued_and_resident(capi):
    import time
    keep = [_point(capi, 32, 10.0) for _ in range(4)]
    foot = 2 * 19 * 4 * 32 ** 3 + 2 * 2 ** 20
    srv = capi.Server(hbm_budget_bytes=2 * foot, check_interval=50, max_resident=2)
    try:
        ids = [srv.submit(d, 1e-14, 10 ** 7) for d, _ in keep]  # tol never met: they run until cancelled
        time.sleep(0.5)
        s = srv.stats()
        assert s["resident"] == 2 and s["queued"] == 2
        assert srv.cancel(ids[3]) == capi.OK                     # queued behind the budget
        st3, _, _ = _wait(srv, ids[3])
        assert st3 == capi.ERR_CANCELLED
        assert srv.cancel(ids[0]) == capi.OK                     # resident: retired after its chunk
        assert srv.cancel(ids[1]) == capi.OK
        st0, obs0, _ = _wait(srv, ids[0])
        assert st0 == capi.ERR_CANCELLED and obs0["steps"] > 0
        assert _wait(srv, ids[1])[0] == capi.ERR_CANCELLED
        assert srv.cancel(ids[3]) == capi.ERR_STATE              # already finished
        assert srv.cancel(ids[2]) == capi.OK                     # admitted once memory freed
        assert _wait(srv, ids[2])[0] == capi.ERR_CANCELLED
        srv.drain(60.0)
        stats = srv.stats()
        assert stats["cancelled"] == 4 and stats["failed"] == 0 and stats["resident"] == 0
    finally:
        srv.close()


def test_server_failed_admission_keeps_serving(capi):
    srv = capi.Server(hbm_budget_bytes=1 << 30, check_interval=50, max_resident=4)
    try:
        d1, k1 = _point(capi, 32, 10.0)
        capi.debug_fail_alloc_after(0)                           # its device memory cannot be had
        r1 = srv.submit(d1, 1e-6, 5000)
        st1, _, _ = _wait(srv, r1)
        capi.debug_fail_alloc_after(-1)
        assert st1 == capi.ERR_NO_MEMORY
        d2, k2 = _point(capi, 32, 10.0)
        r2 = srv.submit(d2, 1e-6, 20000)
        st2, obs2, _ = _wait(srv, r2, 120.0)
        assert st2 in (capi.OK, capi.ERR_NOT_CONVERGED) and obs2["U_sup"] > 0
        stats = srv.stats()
        ok2 = st2 == capi.OK                                     # NOT_CONVERGED counts as failed
        assert stats["completed"] == int(ok2) and stats["failed"] == 1 + int(not ok2)
    finally:
        capi.debug_fail_alloc_after(-1)
        srv.close()


def test_divergence_reported(capi):
    g = I.centred_sphere(32, 10.0)
    with capi.Context(spheres=g.spheres, shape=g.shape, tau=0.5001, delta_rho=0.5, collision=capi.SRT,
                      wall=capi.SBB, storage=capi.F32) as ctx:
        ctx.init_equilibrium()
        st, steps = ctx.run_to_convergence(1e-8, 50, 20000)
        assert st == capi.ERR_DIVERGED and steps <= 20000
