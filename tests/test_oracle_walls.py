"""Pins of the oracle's interpolated wall rules LIBB, QIBB, IEBB, MR (Sec. 2.2.1, Eqs.
LIBB, QIBB, fstar, IEBB, MR) against what the mathematics fixes:

* every rule leaves the fluid at rest at rest (its coefficients sum to one);
* at q = 1/2 LIBB, QIBB and IEBB reduce exactly to simple bounce-back;
* where a node the rule reads is solid, the rule falls back (reading O16): in a one-row
  channel every rule (q < 1/2) is SBB, in a two-row channel (x_f3 solid) QIBB (q < 1/2)
  is LIBB and MR is CLI;
* in a plane channel whose walls sit at q = 0.25 and 0.75 from the fluid nodes, every
  rule converges to the Poiseuille profile of the true width at second order (error ~4x
  smaller per refinement), SBB only at first order;
* the flow past a centred sphere keeps its mirror symmetries.
"""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I
from test_oracle_pins import _channel_profile

NEW_WALLS = {"LIBB": 2, "QIBB": 3, "IEBB": 4, "MR": 5}


@pytest.mark.parametrize("wall", sorted(NEW_WALLS))
@pytest.mark.parametrize("coll", [0, 1, 2])
def test_rest_state_preserved(orc, wall, coll):
    g = I.centred_sphere(12, 4.2)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    f0 = orc.init_rest(s)
    f, sums, _ = orc.run(s, f0, 20, q=q, collision=coll, wall=NEW_WALLS[wall], tau=0.7, delta_rho=0.0)
    # the interpolation weights sum to one up to rounding (~1e-16 a link, ~1e-15 summed)
    assert np.abs(f - f0).max() < 1e-15
    assert np.abs(sums[1:]).max() < 1e-13


@pytest.mark.parametrize("wall", ["LIBB", "QIBB", "IEBB"])
def test_half_way_wall_is_bounce_back(orc, wall):
    g = I.centred_sphere(14, 4.6)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    qh = np.where(np.isfinite(q), 0.5, np.nan)
    f0 = orc.init_rest(s)
    a, _, _ = orc.run(s, f0, 40, q=qh, wall=NEW_WALLS[wall], tau=0.7, delta_rho=1e-4, collision=1)
    b, _, _ = orc.run(s, f0, 40, q=q, wall=0, tau=0.7, delta_rho=1e-4, collision=1)
    assert np.array_equal(a, b)
    c, _, _ = orc.run(s, f0, 40, q=q, wall=NEW_WALLS[wall], tau=0.7, delta_rho=1e-4, collision=1)
    assert np.abs(c - b).max() > 1e-8


def _slit(orc, N, q_all):
    e, _, _ = orc.lattice()
    s = I.slit_channel(N, nx=4, nz=3)
    q = np.full((19,) + s.shape, np.nan)
    for k in range(19):
        if e[k, 1] == -1:
            q[k, :, 1, :] = q_all
        if e[k, 1] == 1:
            q[k, :, N, :] = q_all
    return s, q


def _perturbed(orc, s, seed):
    _, w, _ = orc.lattice()
    f = w[:, None, None, None] * (1.0 + 2e-3 * I.noise((19,) + s.shape, seed))
    f[:, s == 1] = 0.0
    return f


def test_fallbacks_in_narrow_channels(orc):
    kw = dict(tau=0.7, delta_rho=1e-4, collision=1)
    # one fluid row: x_f2 is solid for every link, every rule with q < 1/2 is SBB
    s, q = _slit(orc, 1, 0.3)
    f0 = _perturbed(orc, s, 4)
    sbb, _, _ = orc.run(s, f0, 5, q=q, wall=0, **kw)
    for wall in (1, 2, 3, 4, 5):
        f, _, _ = orc.run(s, f0, 5, q=q, wall=wall, **kw)
        assert np.array_equal(f, sbb), wall
    # two fluid rows: x_f3 is solid; QIBB (q < 1/2) is LIBB, MR is CLI
    for qv in (0.3, 0.7):
        s, q = _slit(orc, 2, qv)
        f0 = _perturbed(orc, s, 5)
        res = {w: orc.run(s, f0, 5, q=q, wall=w, **kw)[0] for w in (1, 2, 3, 5)}
        assert np.array_equal(res[5], res[1])
        if qv < 0.5:
            assert np.array_equal(res[3], res[2])
        else:
            assert np.abs(res[3] - res[2]).max() > 1e-10
        assert np.abs(res[2] - res[1]).max() > 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("delta", [0.25, 0.75])
def test_second_order_off_lattice_wall(orc, delta):
    err = {}
    for name, wall in list(NEW_WALLS.items()) + [("SBB", 0)]:
        err[name] = np.array([np.abs(ux - ua).max() / ua.max()
                              for ux, ua, _ in (_channel_profile(orc, N, delta, wall=wall) for N in (8, 16, 32))])
    for name in NEW_WALLS:
        e = err[name]
        assert (e[:-1] / e[1:] > 3.5).all(), (name, e)       # ~4x per refinement
        assert (e < err["SBB"] / 4).all(), (name, e)
    assert (err["SBB"][:-1] / err["SBB"][1:] < 2.5).all()


@pytest.mark.parametrize("wall", sorted(NEW_WALLS))
def test_symmetry_centred_sphere(orc, wall):
    g = I.centred_sphere(16, 5.5)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    _, _, u = orc.run(s, orc.init_rest(s), 120, q=q, wall=NEW_WALLS[wall], collision=1, tau=0.7,
                      delta_rho=1e-5, want_u=True)
    tol = 1e-9 * np.abs(u[0]).max()
    assert np.abs(u[0] - u[0][:, ::-1, :]).max() < tol
    assert np.abs(u[1] + u[1][:, ::-1, :]).max() < tol
    assert np.abs(u[2] + u[2][::-1, :, :]).max() < tol
    assert np.abs(u[0] - u[0].transpose(1, 0, 2)).max() < tol
    assert u[0].sum() > 0
