"""The fluid-cell state transfer (lbm_get_state / lbm_set_state): the stored values, bit for
bit, in the storage type, for the fluid cells in cell order.

* The values are the stored deviations: they agree with the FP64 export
  (lbm_get_populations_f64) minus w_k rho0, exactly up to that export's own FP64 addition.
* set_state(get_state()) leaves the state unchanged, in both layouts and at either AA phase.
* Two contexts loaded with the same state step on bit for bit alike (a complete state: the
  A-B wall terms are rebuilt from it), for every storage format and for an interpolated wall.
* A buffer of the wrong size is refused.
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


GEOM = I.Geometry(30, 18, 14, np.array([[28.3, 9.6, 8.7, 5.2], [12.0, 3.0, 12.5, 4.1]]))  # ragged, faces


def _ctx(capi, storage, layout, wall):
    return capi.Context(spheres=GEOM.spheres, shape=GEOM.shape, tau=0.62, delta_rho=3e-4, collision=capi.TRT,
                        wall=getattr(capi, wall), storage=getattr(capi, storage),
                        layout=getattr(capi, "LAYOUT_" + layout))


def _decode(capi, storage, s, scale_log2):
    if storage == "F16DEV":
        return s.view(np.float16).astype(np.float64) * 2.0 ** -scale_log2
    if storage == "BF16DEV":
        return (s.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return s.astype(np.float64)


CASES = [("F64", "AB", "CLI"), ("F32", "AB", "CLI"), ("F32", "AA", "CLI"), ("F16DEV", "AB", "CLI"),
         ("BF16DEV", "AA", "SBB"), ("F32", "AB", "QIBB")]


@pytest.mark.parametrize("storage,layout,wall", CASES)
def test_state_values_and_round_trip(capi, orc, storage, layout, wall):
    _, w, _ = orc.lattice()
    with _ctx(capi, storage, layout, wall) as ctx:
        ctx.init_equilibrium()
        ctx.step(7)                                      # odd: AA state in its shifted arrangement
        info = ctx.info()
        s = ctx.get_state()
        assert s.shape == (19, info["n_fluid"]) and s.dtype == ctx.state_dtype()
        fluid = ctx.get_flags().reshape(-1) == 0
        f = ctx.get_populations().reshape(19, -1)[:, fluid]
        g = _decode(capi, storage, s, info["dev_scale_log2"])
        assert np.all(np.isfinite(g)) and np.abs(g).max() > 0
        np.testing.assert_allclose(g, f - w[:, None], rtol=0, atol=1e-15)
        ctx.set_state(s)                                 # a no-op on the fluid state
        assert np.array_equal(ctx.get_state(), s)


@pytest.mark.parametrize("storage,layout,wall", CASES)
def test_loaded_contexts_step_alike(capi, storage, layout, wall):
    with _ctx(capi, storage, layout, wall) as a:
        a.init_equilibrium()
        a.step(9)
        s = a.get_state()
        a.set_state(s)
        with _ctx(capi, storage, layout, wall) as b:
            b.set_state(s)
            for n in (1, 12):
                a.step(n)
                b.step(n)
                oa, ob = a.observables(), b.observables()
                assert np.array_equal(a.get_state(), b.get_state())
                assert oa["U_sup"] == ob["U_sup"] and oa["F_x"] == ob["F_x"]


def test_pinned_buffers_and_size_check(capi):
    import torch
    with _ctx(capi, "F32", "AB", "CLI") as ctx:
        ctx.init_equilibrium()
        ctx.step(5)
        nf = ctx.info()["n_fluid"]
        pinned = torch.empty((19, nf), dtype=torch.float32, pin_memory=True).numpy()
        ctx.get_state(pinned)
        assert np.array_equal(pinned, ctx.get_state())
        ctx.set_state(pinned)
        assert capi.lib().lbm_set_state(ctx.handle, pinned.ctypes.data, pinned.nbytes - 4) == capi.ERR_ARG
        assert capi.lib().lbm_get_state(ctx.handle, pinned.ctypes.data, pinned.nbytes + 4) == capi.ERR_ARG


@pytest.mark.parametrize("layout", ["AB", "AA"])
def test_staged_states_apply_in_order(capi, layout):
    """Two states staged ahead are applied in order; each applied state steps exactly as the
    same state set with set_state; a third stage and an apply with nothing staged are refused."""
    with _ctx(capi, "F32", layout, "CLI") as a:
        a.init_equilibrium()
        a.step(5)
        s1 = a.get_state()
        a.step(7)
        s2 = a.get_state()
    with _ctx(capi, "F32", layout, "CLI") as b, _ctx(capi, "F32", layout, "CLI") as c:
        b.stage_state(s1)
        b.stage_state(s2)
        with pytest.raises(capi.LBMError) as e:
            b.stage_state(s1)
        assert e.value.status == capi.ERR_STATE
        b.apply_staged_state()
        b.step(3)
        c.set_state(s1)
        c.step(3)
        assert np.array_equal(b.get_state(), c.get_state())
        assert b.observables()["U_sup"] == c.observables()["U_sup"]
        b.apply_staged_state()
        assert np.array_equal(b.get_state(), s2)
        with pytest.raises(capi.LBMError) as e:
            b.apply_staged_state()
        assert e.value.status == capi.ERR_STATE
        b.stage_state(s1)                                  # the buffers are reused in turn
        b.apply_staged_state()
        assert np.array_equal(b.get_state(), s1)
