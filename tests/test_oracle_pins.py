"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form, an
invariant, a special case that reduces to a simpler operator, an independent
numerical method (bisection), or a qualitative finding the paper states.  Each pin is
chosen so that a plausible slip in the oracle (a dropped term, a wrong sign, a wrong
opposite index, a transposed operand) fails it.
"""
import os

import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------------
# Lattice and equilibrium (Sec. 2: D3Q19, Eq. equilibrium, Eq. Macro)
# ----------------------------------------------------------------------------------
def test_lattice_isotropy(orc):
    e, w, opp = orc.lattice()
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15                       # weights normalised to unity
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    m2 = np.einsum("k,ka,kb->ab", w, e, e)
    assert np.abs(m2 - d / 3.0).max() < 1e-15               # c_s^2 = 1/3
    m3 = np.einsum("k,ka,kb,kc->abc", w, e, e, e)
    assert np.abs(m3).max() < 1e-15
    m4 = np.einsum("k,ka,kb,kc,kd->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(m4 - iso).max() < 1e-15                   # fourth-order isotropy
    assert len({tuple(v) for v in e}) == 19
    assert (e[opp] == -e).all() and (opp[opp] == np.arange(19)).all()


def test_equilibrium_moments(orc):
    rng = np.random.default_rng(1)
    e, w, _ = orc.lattice()
    for _ in range(20):
        rho = 1.0 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        rho0 = 1.0 + 0.2 * rng.random()
        feq = orc.equilibrium(rho, u, rho0)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.abs(e.T @ feq - rho0 * u).max() < 1e-15
        # incompressible second moment: rho/3 delta + rho0 u u
        m2 = np.einsum("k,ka,kb->ab", feq, e, e)
        assert np.abs(m2 - (rho / 3.0 * np.eye(3) + rho0 * np.outer(u, u))).max() < 1e-14


def test_pressure_shift_is_equilibrium_difference(orc):
    """Eqs. PeriodicFunkown -> Periodicfunkown: with the incompressible equilibrium,
    f^eq(rho_L, u) - f^eq(rho_R, u) = w_k delta_rho exactly (f^eq is affine in rho)."""
    _, w, _ = orc.lattice()
    u = np.array([0.03, -0.01, 0.02])
    for dr in (1e-5, 1e-3, 0.1):
        diff = orc.equilibrium(1.0 + dr, u) - orc.equilibrium(1.0, u)
        assert np.abs(diff - w * dr).max() < 1e-15


def test_golden_table1_lambda():
    rows = np.loadtxt(os.path.join(HERE, "golden", "table1_lambda.txt"))
    for lo, hi, _, lam in rows:
        for re in (hi, 0.5 * (lo + hi)):
            assert I.table1_lambda(re) == pytest.approx(lam, rel=1e-12)


# ----------------------------------------------------------------------------------
# Collision operators (Sec. 2.1, Eqs. SRT, MRT, TRT)
# ----------------------------------------------------------------------------------
def _near_eq(orc, rng, amp=1e-3):
    feq = orc.equilibrium(1.0 + 0.01 * rng.standard_normal(), 0.02 * rng.standard_normal(3))
    return feq + amp * rng.standard_normal(19) / 36.0


@pytest.mark.parametrize("coll", [0, 1, 2])
def test_collision_conserves_mass_momentum(orc, coll):
    rng = np.random.default_rng(2 + coll)
    e, _, _ = orc.lattice()
    for _ in range(10):
        f = _near_eq(orc, rng)
        ft = orc.collide(f, collision=coll, tau=0.7, magic_lambda=0.2)
        assert abs(ft.sum() - f.sum()) < 1e-15
        assert np.abs(e.T @ (ft - f)).max() < 1e-16
        feq = orc.equilibrium(1.02, [0.01, 0.02, -0.03])
        assert np.abs(orc.collide(feq, collision=coll, tau=0.7) - feq).max() < 1e-16


def test_trt_eigenrates(orc):
    """Symmetric non-conserved perturbations decay by (1 - omega+), antisymmetric ones by
    (1 - omega-), with omega+ = 1/tau and (1/omega+ - 1/2)(1/omega- - 1/2) = Lambda."""
    tau, lam = 0.83, 0.11
    wp = 1.0 / tau
    wm = 1.0 / (0.5 + lam / (tau - 0.5))
    feq = orc.equilibrium(1.0, [0.0, 0.0, 0.0])
    sym = np.zeros(19); sym[[1, 2]] = 1; sym[[3, 4]] = -1                  # no mass, no momentum
    anti = np.zeros(19); anti[7] = 1; anti[8] = -1; anti[1] = -1; anti[2] = 1; anti[3] = -1; anti[4] = 1
    for pert, rate in ((sym, wp), (anti, wm)):
        f = feq + 1e-4 * pert
        ft = orc.collide(f, collision=1, tau=tau, magic_lambda=lam)
        assert np.abs((ft - feq) - (1.0 - rate) * 1e-4 * pert).max() < 2e-16
    lam_back = (1 / wp - 0.5) * (1 / wm - 0.5)
    assert lam_back == pytest.approx(lam, rel=1e-14)


def test_mrt_matrix_structure(orc):
    """Gram-Schmidt rows are mutually orthogonal; row 0 is the mass, rows 3/5/7 are
    the momentum components; every row is either even or odd under k -> k-bar."""
    e, _, opp = orc.lattice()
    M = orc.mrt_matrix()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    assert np.abs(M[0] - 1.0).max() < 1e-15
    for row, a in ((3, 0), (5, 1), (7, 2)):
        assert np.abs(M[row] - e[:, a]).max() < 1e-15
    parity = []
    for i in range(19):
        if np.abs(M[i] - M[i, opp]).max() < 1e-12:
            parity.append(+1)
        else:
            assert np.abs(M[i] + M[i, opp]).max() < 1e-12
            parity.append(-1)
    assert parity.count(+1) == 10 and parity.count(-1) == 9


def test_mrt_reduces_to_srt_and_trt(orc):
    """SRT is the special case of MRT with equal rates (Sec. 2.1); TRT is MRT with
    omega+ on the even modes and omega- on the odd modes (Eq. TRT)."""
    rng = np.random.default_rng(7)
    _, _, opp = orc.lattice()
    M = orc.mrt_matrix()
    even = np.array([np.abs(M[i] - M[i, opp]).max() < 1e-12 for i in range(19)])
    tau, lam = 0.9, 0.3
    wp, wm = 1 / tau, 1.0 / (0.5 + lam / (tau - 0.5))
    for _ in range(10):
        f = _near_eq(orc, rng, 1e-2)
        srt = orc.collide(f, collision=0, tau=tau)
        mrt = orc.collide(f, collision=2, tau=tau, mrt_s=np.full(19, 1 / tau))
        assert np.abs(srt - mrt).max() < 1e-14
        trt = orc.collide(f, collision=1, tau=tau, magic_lambda=lam)
        mrt = orc.collide(f, collision=2, tau=tau, mrt_s=np.where(even, wp, wm))
        assert np.abs(trt - mrt).max() < 1e-14


def test_mrt_rates_rules(orc):
    """Pan's kinetic rate s_zeta = 8(2-s_nu)/(8-s_nu) makes (1/s_nu-1/2)(1/s_zeta-1/2)
    = 3/16 for every viscosity; the energy modes keep the ratio 4.6 (Sec. 2.1)."""
    for tau in (0.51, 0.6, 0.8, 1.3):
        s = orc.mrt_rates(tau, 4.6)
        snu = 1 / tau
        assert s[0] == s[3] == s[5] == s[7] == 0.0
        for i in (9, 11, 13, 14, 15):
            assert s[i] == snu
        for i in (4, 6, 8, 10, 12, 16, 17, 18):
            assert (1 / snu - 0.5) * (1 / s[i] - 0.5) == pytest.approx(3 / 16, rel=1e-13)
        for i in (1, 2):
            assert (1 / snu - 0.5) / (1 / s[i] - 0.5) == pytest.approx(4.6, rel=1e-13)


# ----------------------------------------------------------------------------------
# Geometry: voxeliser and wall distance q (Sec. 2.2.1, Sec. 3)
# ----------------------------------------------------------------------------------
def test_voxel_sphere_volume_and_symmetry(orc):
    for L, r in ((32, 12.0), (24, 7.3)):
        g = I.centred_sphere(L, r)
        s = orc.voxelize(g.shape, g.spheres).astype(bool)
        vol = 4.0 / 3.0 * np.pi * r ** 3
        assert abs(s.sum() - vol) < 4 * np.pi * r ** 2 * 0.1    # staircase error ~ surface
        assert (s == s[::-1]).all() and (s == s[:, ::-1]).all() and (s == s[:, :, ::-1]).all()
        assert (s == s.transpose(1, 0, 2)).all() and (s == s.transpose(2, 1, 0)).all()


def test_voxel_periodic_images(orc):
    """A sphere centred at a corner appears in all eight corners of the periodic box."""
    g = I.Geometry(16, 16, 16, np.array([[0.0, 0.0, 0.0, 3.0]]))
    s = orc.voxelize(g.shape, g.spheres).astype(bool)
    for z in (0, -1):
        for y in (0, -1):
            for x in (0, -1):
                assert s[z, y, x]
    assert not s[8, 8, 8]
    assert (s == s[::-1, ::-1, ::-1]).all()          # mirror about the corner: i -> L-1-i


def test_voxel_far_centres_refused(orc):
    """Centres more than 64 box lengths out are refused (the periodic fold would loop);
    centres a few box lengths out are folded to the same voxels as their image in the box."""
    with pytest.raises(ValueError):
        orc.voxelize((8, 8, 8), [[1e17, 4.0, 4.0, 2.0]])
    with pytest.raises(ValueError):
        orc.wall_distances(np.zeros((8, 8, 8), np.uint8), [[4.0, -600.0, 4.0, 2.0]])
    a = orc.voxelize((8, 8, 8), [[4.25, 3.5, 4.75, 2.6]])
    b = orc.voxelize((8, 8, 8), [[4.25 + 24.0, 3.5 - 16.0, 4.75 + 8.0, 2.6]])
    assert a.sum() > 0 and np.array_equal(a, b)


def test_wall_distance_against_bisection(orc):
    """q of each cut link equals the first crossing of the segment x_f1 -> x_b with the
    sphere, found here by bisection (an independent method)."""
    e, _, _ = orc.lattice()
    rng = np.random.default_rng(3)
    g = I.Geometry(20, 18, 22, np.array([[9.3, 8.7, 11.1, 5.6]]))
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    cut = np.argwhere(np.isfinite(q))
    assert len(cut) > 100
    c = g.spheres[0, :3]
    r = g.spheres[0, 3]
    for k, z, y, x in cut[rng.choice(len(cut), 200, replace=False)]:
        assert s[z, y, x] == 0
        p = np.array([x + 0.5, y + 0.5, z + 0.5])
        d = e[k].astype(float)
        lo, hi = 0.0, 1.0
        assert np.linalg.norm(p - c) > r and np.linalg.norm(p + d - c) <= r
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if np.linalg.norm(p + mid * d - c) > r:
                lo = mid
            else:
                hi = mid
        assert q[k, z, y, x] == pytest.approx(0.5 * (lo + hi), abs=1e-12)
    # every link into a solid cell is cut, and no other link is
    for k in range(1, 19):
        nb = np.roll(s, shift=(-e[k, 2], -e[k, 1], -e[k, 0]), axis=(0, 1, 2))
        assert (np.isfinite(q[k]) == ((s == 0) & (nb == 1))).all()


# ----------------------------------------------------------------------------------
# Whole-step invariants (Sec. 2: stream then collide; Sec. 2.2 boundaries)
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("coll,wall", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_rest_state_preserved(orc, coll, wall):
    g = I.centred_sphere(12, 4.2)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    f0 = orc.init_rest(s)
    f, sums, _ = orc.run(s, f0, 30, q=q, collision=coll, wall=wall, tau=0.7, delta_rho=0.0)
    assert np.abs(f - f0).max() < 1e-15
    assert np.abs(sums[1:]).max() < 1e-15


@pytest.mark.parametrize("coll", [0, 1, 2])
def test_mass_conservation_sbb_and_flow_direction(orc, coll):
    """The shift +w dr on one crossing and -w dr on the opposite crossing, with SBB
    walls, conserves the total mass; the flow runs from the high-density left to the
    right (+x)."""
    g = I.centred_sphere(16, 5.5)
    s = orc.voxelize(g.shape, g.spheres)
    f0 = orc.init_rest(s)
    f, sums, _ = orc.run(s, f0, 400, collision=coll, wall=0, tau=0.8, delta_rho=1e-4)
    assert abs(f.sum() / f0.sum() - 1.0) < 1e-13
    assert abs(sums[0] / f0.sum() - 1.0) < 1e-13
    assert sums[1] > 0
    assert abs(sums[2]) < 1e-12 * sums[1] and abs(sums[3]) < 1e-12 * sums[1]


def _channel_profile(orc, N, delta, wall, coll=1, lam=3 / 16, tau=0.8):
    """Plane channel: fluid rows 1..N, wall planes at distance delta from the first and
    last fluid centres, flow driven by the periodic pressure drop."""
    e, _, _ = orc.lattice()
    nx = 4
    s = I.slit_channel(N, nx=nx)
    q = np.full((19,) + s.shape, np.nan)
    for k in range(19):
        if e[k, 1] == -1:
            q[k, 0, 1, :] = delta
        if e[k, 1] == 1:
            q[k, 0, N, :] = delta
    dr, nu = 1e-5, (tau - 0.5) / 3
    steps = int(3.0 * N * N / nu) + 2000
    f, _, u = orc.run(s, orc.init_rest(s), steps, q=q, collision=coll, wall=wall, tau=tau,
                      delta_rho=dr, magic_lambda=lam, want_u=True)
    G = dr / (3 * nx)                           # pressure gradient (delta p / L)
    H = N - 1 + 2 * delta
    eta = np.arange(1, N + 1) - 1 + delta
    ua = G / (2 * nu) * eta * (H - eta)         # Poiseuille profile
    return u[0, 0, 1:, 0], ua, u


def test_poiseuille_magic_three_sixteenths(orc):
    """Lambda = 3/16 places bounce-back walls exactly half-way for Poiseuille flow
    (Sec. 2.1), here driven by the periodic pressure drop (Sec. 2.2.2)."""
    ux, ua, u = _channel_profile(orc, 16, 0.5, wall=0)
    assert np.abs(ux / ua - 1).max() < 1e-9
    assert np.abs(u[0, 0, 1:, :] - ux[:, None]).max() < 1e-15          # uniform along x
    assert np.abs(u[1:]).max() < 1e-15                                  # no cross flow
    ux, ua, _ = _channel_profile(orc, 16, 0.5, wall=0, coll=2)          # MRT, Pan rates
    assert np.abs(ux / ua - 1).max() < 1e-9
    for kw in (dict(lam=0.25), dict(coll=0)):                           # controls
        ux, ua, _ = _channel_profile(orc, 16, 0.5, wall=0, **kw)
        assert np.abs(ux / ua - 1).max() > 1e-3


@pytest.mark.parametrize("N,tau", [(8, 0.8), (16, 0.8), (8, 1.3)])
def test_permeability_slit_channel_closed_form(orc, N, tau):
    """Permeability of a plane channel from the observables (Eq. Darcy, K = mu U / (dp/L_x),
    U the volume-averaged velocity of Sec. 1), against the closed form.  TRT with Lambda =
    3/16 and bounce-back walls gives the exact Poiseuille profile u = G/(2 nu) eta (N - eta)
    on the N fluid rows, eta = j - 1/2 (Sec. 2.1); summed over the rows, Sum eta (N - eta) =
    N (2 N^2 + 1) / 12, and averaged over the box of N + 1 rows (one solid row):
        K = N (2 N^2 + 1) / (24 (N + 1)) = N (N^2 + 1/2) / (12 (N + 1)),
    independent of tau.  The box is 4 x (N + 1) x 3, so that an average over the wrong
    volume, a gradient over L_y or L_z instead of L_x, dp = delta_rho instead of
    delta_rho / 3, or a viscosity off by a factor each miss it."""
    nx, nz = 4, 3
    s = I.slit_channel(N, nx=nx, nz=nz)
    ny = s.shape[1]
    dr = 1e-5
    nu = (tau - 0.5) / 3
    steps = int(3.0 * N * N / nu) + 2000
    _, sums, _ = orc.run(s, orc.init_rest(s), steps, collision=1, wall=0, tau=tau, delta_rho=dr,
                         magic_lambda=3 / 16)
    U_sup = sums[1] / (nx * ny * nz)
    K = orc.observables(U_sup, tau, dr, nx, 1.0)[1]
    K_exact = N * (N * N + 0.5) / (12.0 * (N + 1))
    assert K == pytest.approx(K_exact, rel=1e-9, abs=0)


def test_cli_half_equals_sbb(orc):
    """With q = 1/2 the CLI coefficient (1-2q)/(1+2q) vanishes and CLI is SBB (Eq. CLI)."""
    g = I.centred_sphere(14, 4.6)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    qh = np.where(np.isfinite(q), 0.5, np.nan)
    f0 = orc.init_rest(s)
    a, _, _ = orc.run(s, f0, 60, q=qh, wall=1, tau=0.7, delta_rho=1e-4)
    b, _, _ = orc.run(s, f0, 60, q=q, wall=0, tau=0.7, delta_rho=1e-4)
    assert np.array_equal(a, b)
    c, _, _ = orc.run(s, f0, 60, q=q, wall=1, tau=0.7, delta_rho=1e-4)
    assert np.abs(c - b).max() > 1e-8


def test_cli_second_order_off_lattice_wall(orc):
    """A channel whose walls sit at q = 0.25 and 0.75 from the fluid nodes: CLI
    converges to the Poiseuille profile of the true width at second order, SBB (wall
    fixed half-way) only at first order (Sec. 3.1: interpolated walls are second order)."""
    for delta in (0.25, 0.75):
        err = {}
        for wall in (0, 1):
            err[wall] = []
            for N in (8, 16, 32):
                ux, ua, _ = _channel_profile(orc, N, delta, wall=wall)
                err[wall].append(np.abs(ux - ua).max() / ua.max())
        cli, sbb = np.array(err[1]), np.array(err[0])
        assert (cli < sbb / 5).all()
        assert (cli[:-1] / cli[1:] > 3.5).all()          # ~4x per refinement
        assert (sbb[:-1] / sbb[1:] < 2.5).all()          # ~2x per refinement


def test_symmetry_centred_sphere(orc):
    """Flow past a centred sphere: u_x even and u_y odd in y, u_z odd in z, y <-> z
    interchange symmetry (Sec. 4, symmetric Stokes flow)."""
    g = I.centred_sphere(16, 5.5)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    for wall, coll in ((0, 1), (1, 1), (1, 2)):
        _, _, u = orc.run(s, orc.init_rest(s), 150, q=q, wall=wall, collision=coll, tau=0.7,
                          delta_rho=1e-5, want_u=True)
        scale = np.abs(u[0]).max()
        # rounding of f ~ 0.05 at 1e-17 is ~1e-12 of u ~ 3e-5; an index slip is O(1)
        tol = 1e-9 * scale
        # mirror about the box centre: cell j -> L-1-j
        assert np.abs(u[0] - u[0][:, ::-1, :]).max() < tol
        assert np.abs(u[1] + u[1][:, ::-1, :]).max() < tol
        assert np.abs(u[2] + u[2][::-1, :, :]).max() < tol
        assert np.abs(u[0] - u[0].transpose(1, 0, 2)).max() < tol
        assert np.abs(u[1] - u[2].transpose(1, 0, 2)).max() < tol


def _steady_K(orc, geom, tau, coll, wall, lam=3 / 16, dr=1e-6, tol=1e-9, chunk=200,
              max_steps=40000):
    s = orc.voxelize(geom.shape, geom.spheres)
    q = orc.wall_distances(s, geom.spheres)
    f = orc.init_rest(s)
    U_old, n = None, 0
    while n < max_steps:
        f, sums, _ = orc.run(s, f, chunk, q=q, tau=tau, delta_rho=dr, collision=coll,
                             wall=wall, magic_lambda=lam)
        n += chunk
        U = sums[1] / geom.n_cells
        if U_old is not None and abs(U - U_old) < tol * abs(U):
            break
        U_old = U
    return orc.observables(U, tau, dr, geom.nx, geom.d_p)


@pytest.mark.slow
def test_permeability_viscosity_independence(orc):
    """Sec. 3.2: with TRT at fixed Lambda the Stokes permeability does not depend on the
    viscosity; with SRT it does."""
    g = I.centred_sphere(16, 6.0)
    K = {c: [_steady_K(orc, g, tau, c, 0)[1] for tau in (0.6, 1.0)] for c in (0, 1)}
    assert abs(K[1][0] / K[1][1] - 1) < 1e-4
    assert abs(K[0][0] / K[0][1] - 1) > 1e-2


@pytest.mark.slow
def test_darcy_regime_linearity_and_observable_identity(orc):
    """In the Darcy regime K_app equals K_D (Eq. AppPer plateau); the friction-factor
    form satisfies F_K - 1/Re_K = C_F (Eqs. Forchheimer and frictionFactor)."""
    g = I.centred_sphere(16, 6.0)
    o6 = _steady_K(orc, g, 0.8, 1, 1, dr=1e-6)
    o5 = _steady_K(orc, g, 0.8, 1, 1, dr=1e-5)
    assert abs(o5[1] / o6[1] - 1) < 1e-3
    K_D = o6[1]
    for U in (1e-4, 3e-3, 0.05):
        U_, K, Re_p, beta, C_F, F_K, Re_K = orc.observables(U, 0.8, 1e-3, 16, 12.0, K_D)
        assert F_K - 1 / Re_K == pytest.approx(C_F, rel=1e-10, abs=1e-14)
        assert C_F == pytest.approx(beta * np.sqrt(K_D), rel=1e-14)


@pytest.mark.slow
def test_sbb_cli_agree_under_refinement(orc):
    """Sec. 3.1: interpolated walls reach a grid-independent permeability sooner than
    SBB; both converge to the same value as r grows at fixed r/L."""
    kl2 = {}
    for wall in (0, 1):
        kl2[wall] = [_steady_K(orc, I.centred_sphere(L, 0.375 * L), 1.0, 1, wall)[1] / L ** 2
                     for L in (16, 24)]
    cli, sbb = np.array(kl2[1]), np.array(kl2[0])
    assert abs(cli[1] / cli[0] - 1) < 1e-2
    assert abs(cli[1] / cli[0] - 1) < abs(sbb[1] / sbb[0] - 1)
    assert (np.abs(sbb / cli - 1) < 0.06).all()


def test_time_averages_of_a_steady_flow(orc):
    """The oracle's time averages (Sec. 4: averages of the developed flow) pinned by a steady
    Stokes flow: once the flow no longer changes, the windowed average of U_sup and of the
    drag equals the steady value, and the developed-flow procedure finds the drag converged
    and averages round(average_ft * samples_per_ft) samples of round(T / samples_per_ft)
    steps, T = nx / U_sup."""
    g = I.centred_sphere(12, 3.5)
    s = orc.voxelize(g.shape, g.spheres)
    q = orc.wall_distances(s, g.spheres)
    kw = dict(q=q, tau=0.8, delta_rho=2e-3, magic_lambda=3 / 16, collision=1, wall=1)
    f, U_old = orc.init_rest(s), None
    for _ in range(200):
        F = np.zeros(3)
        f, sums, _ = orc.run(s, f, 100, force=F, **kw)
        U = sums[1] / g.n_cells
        if U_old is not None and abs(U - U_old) < 1e-13 * abs(U):
            break
        U_old = U
    _, U_avg, F_avg = orc.time_average(s, f, 5, 40, **kw)
    assert U_avg == pytest.approx(U, rel=1e-12, abs=0)
    assert np.allclose(F_avg, F, rtol=1e-10, atol=1e-12 * abs(F[0]))     # F_y, F_z: rounding only
    o = orc.developed_average(s, f, min_spinup_ft=1.0, max_spinup_ft=50.0, drag_tol=1e-9, average_ft=2.0,
                              samples_per_ft=3, max_steps=10 ** 6, **kw)
    assert o["status"] == "ok" and o["developed"]
    T = 12 / abs(U)
    assert o["average_steps"] == 6 * int(np.floor(T / 3 + 0.5))
    assert o["U_sup"] == pytest.approx(U, rel=1e-12, abs=0)
    assert np.allclose(o["F"], F, rtol=1e-10, atol=1e-12 * abs(F[0]))
