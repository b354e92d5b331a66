"""FP64 CPU oracle for the sphere-pack LBM hot path (arXiv:1508.02960).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module; the product library never does.  The C
source (``oracle.c``) is compiled with gcc into ``oracle/_build/liboracle.so``.

Array conventions (same as the C source): scalar fields are ``[nz][ny][nx]`` and
population fields ``[19][nz][ny][nx]`` in C order, i.e. the cell index is
``x + nx*(y + ny*z)``.  Spheres are ``(n, 4)`` arrays of ``(cx, cy, cz, r)`` in lattice
units, with cell ``(i, j, k)`` centred at ``(i+0.5, j+0.5, k+0.5)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
SRT, TRT, MRT = 0, 1, 2
SBB, CLI, LIBB, QIBB, IEBB, MR = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile oracle.c (C99, -O2, no FMA contraction, OpenMP) if needed."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in oracle.c."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("collision", ctypes.c_int), ("wall", ctypes.c_int),
        ("tau", ctypes.c_double), ("delta_rho", ctypes.c_double), ("rho0", ctypes.c_double),
        ("magic_lambda", ctypes.c_double), ("mrt_ratio", ctypes.c_double),
        ("mrt_s", ctypes.POINTER(ctypes.c_double)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_lattice.argtypes = [ip, dp, ip]
            lib.orc_equilibrium.argtypes = [ctypes.c_double, dp, ctypes.c_double, dp]
            lib.orc_mrt_matrix.argtypes = [dp]
            lib.orc_mrt_rates.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            lib.orc_collide.argtypes = [ctypes.POINTER(Params), dp, dp]
            lib.orc_voxelize.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int, u8p]
            lib.orc_voxelize.restype = ctypes.c_int
            lib.orc_wall_distances.argtypes = [ctypes.c_int] * 3 + [u8p, dp, ctypes.c_int, dp]
            lib.orc_wall_distances.restype = ctypes.c_int
            lib.orc_run.argtypes = [ctypes.POINTER(Params), u8p, dp, dp, ctypes.c_int, dp, dp, dp]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_init_rest.argtypes = [ctypes.c_int] * 3 + [u8p, ctypes.c_double, dp]
            lib.orc_observables.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_double,
                                                                    ctypes.c_double, dp]
            lib.orc_drag_coefficients.argtypes = [ctypes.c_double] * 6 + [dp]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def lattice():
    """Return (e[19,3] int, w[19] float64, opp[19] int) of the oracle's D3Q19 lattice."""
    lib = _load()
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib.orc_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                    opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e, w, opp


def equilibrium(rho: float, u, rho0: float = 1.0) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    _load().orc_equilibrium(float(rho), _dp(u), float(rho0), _dp(out))
    return out


def mrt_matrix() -> np.ndarray:
    m = np.zeros((Q, Q))
    _load().orc_mrt_matrix(_dp(m))
    return m


def mrt_rates(tau: float, ratio: float = 4.6) -> np.ndarray:
    s = np.zeros(Q)
    _load().orc_mrt_rates(float(tau), float(ratio), _dp(s))
    return s


def make_params(shape, *, collision=TRT, wall=SBB, tau=0.8, delta_rho=0.0, rho0=1.0,
                magic_lambda=3.0 / 16.0, mrt_ratio=4.6, mrt_s=None):
    """shape = (nz, ny, nx).  Returns (Params, keepalive) -- keep both alive."""
    nz, ny, nx = shape
    keep = None
    p = Params(nx=nx, ny=ny, nz=nz, collision=collision, wall=wall, tau=tau,
               delta_rho=delta_rho, rho0=rho0, magic_lambda=magic_lambda,
               mrt_ratio=mrt_ratio, mrt_s=None)
    if mrt_s is not None:
        keep = np.ascontiguousarray(mrt_s, dtype=np.float64)
        p.mrt_s = _dp(keep)
    return p, keep


def collide(f, **kw) -> np.ndarray:
    """Collide one node's 19 populations (Eqs. SRT/TRT/MRT)."""
    p, keep = make_params((1, 1, 1), **kw)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(Q)
    _load().orc_collide(ctypes.byref(p), _dp(f), _dp(out))
    return out


def voxelize(shape, spheres) -> np.ndarray:
    """Solid flags uint8 [nz,ny,nx] (1 = solid) of a periodic box holding the spheres."""
    nz, ny, nx = shape
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    rc = _load().orc_voxelize(nx, ny, nz, _dp(sph), sph.shape[0], _u8(solid))
    if rc != 0:
        raise ValueError("orc_voxelize failed")
    return solid


def wall_distances(solid, spheres) -> np.ndarray:
    """q[19,nz,ny,nx]: wall distance of each cut link (fluid cell, direction into the wall)."""
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = solid.shape
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    q = np.zeros((Q, nz, ny, nx))
    rc = _load().orc_wall_distances(nx, ny, nz, _u8(solid), _dp(sph), sph.shape[0], _dp(q))
    if rc != 0:
        raise ValueError("orc_wall_distances failed")
    return q


def init_rest(solid, rho0: float = 1.0) -> np.ndarray:
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = solid.shape
    f = np.zeros((Q, nz, ny, nx))
    _load().orc_init_rest(nx, ny, nz, _u8(solid), float(rho0), _dp(f))
    return f


def run(solid, f, nsteps: int, *, q=None, want_u: bool = False, force=None, **kw):
    """Advance f (post-collision, [19,nz,ny,nx]) by nsteps.  Returns (f, sums, u|None).

    sums = [sum rho, sum u_x, sum u_y, sum u_z] over fluid cells of the last step's
    streamed moments.  force: optional float64 array of 3 that receives the momentum
    exchanged with the solid during the last step (the drag F_D of Sec. 3)."""
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    p, keep = make_params(solid.shape, **kw)
    qq = None
    if q is not None:
        qq = np.ascontiguousarray(q, dtype=np.float64)
    sums = np.zeros(4)
    u = np.zeros((3,) + solid.shape) if want_u else None
    if force is not None and (not isinstance(force, np.ndarray) or force.dtype != np.float64
                              or force.shape != (3,) or not force.flags.c_contiguous):
        raise ValueError("force must be a contiguous float64 array of 3")
    rc = _load().orc_run(ctypes.byref(p), _u8(solid), _dp(qq) if qq is not None else None,
                         _dp(f), int(nsteps), _dp(sums), _dp(u) if u is not None else None,
                         _dp(force) if force is not None else None)
    if rc != 0:
        raise ValueError(f"orc_run failed ({rc})")
    return f, sums, u


def drag_coefficients(F_D, U, tau, r_sum, area_sum, rho0=1.0):
    """[C_D, C_D_A]: F_D / (6 pi mu U r) (Eq. AnalyticForce, r = sum of radii) and
    F_D / (rho0 A U^2) (Sec. 4, A = sum of frontal areas pi r^2)."""
    out = np.zeros(2)
    _load().orc_drag_coefficients(float(F_D), float(U), float(tau), float(rho0), float(r_sum),
                                  float(area_sum), _dp(out))
    return out


def observables(U, tau, delta_rho, lx, d_p, K_D=0.0, rho0=1.0):
    """[U, K, Re_p, beta, C_F, F_K, Re_K] in lattice units (Eqs. Darcy, Forchheimer,
    frictionFactor)."""
    out = np.zeros(7)
    _load().orc_observables(float(U), float(tau), float(delta_rho), float(rho0), int(lx),
                            float(d_p), float(K_D), _dp(out))
    return out


def barree_conway(re, m, a, E, F):
    """Barree-Conway apparent permeability (Eq. AppPer) normalised by K_D (Eq.
    normalizedPermeability): K* = m + (1 - m) / (1 + Re_T^F)^E with Re_T = a Re,
    m = K_min / K_D."""
    re = np.asarray(re, dtype=np.float64)
    return m + (1.0 - m) / (1.0 + (a * re) ** F) ** E


def fit_barree_conway(re, kstar, init=None):
    """Least-squares fit of barree_conway to (re, kstar) with scipy's Levenberg-Marquardt
    least_squares (a library routine), over (logit m, ln a, ln E, ln F) so that 0 < m < 1
    and a, E, F > 0.  Returns ([m, a, E, F], rms)."""
    from scipy.optimize import least_squares
    re = np.asarray(re, dtype=np.float64)
    kstar = np.asarray(kstar, dtype=np.float64)
    if init is None:
        init = [min(0.9, max(0.01, 0.9 * kstar.min())), 1.0 / np.median(re), 1.0, 1.0]
    x0 = np.array([np.log(init[0] / (1.0 - init[0])), np.log(init[1]), np.log(init[2]), np.log(init[3])])

    def m_of(x0):
        return 1.0 / (1.0 + np.exp(-x0))

    def res(x):
        return barree_conway(re, m_of(x[0]), np.exp(x[1]), np.exp(x[2]), np.exp(x[3])) - kstar

    sol = least_squares(res, x0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    p = np.array([m_of(sol.x[0]), np.exp(sol.x[1]), np.exp(sol.x[2]), np.exp(sol.x[3])])
    return p, float(np.sqrt(np.mean(sol.fun ** 2)))



def time_average(solid, f, n_samples: int, interval: int, *, q=None, **kw):
    """Time average of the volume-averaged velocity and of the drag (Sec. 4: the flow is
    averaged over a period of the developed flow; the drag of the resolution study is
    time-averaged): advance n_samples * interval steps, take U_sup = sum u_x / (nx ny nz) and
    the drag F_D of the last step of every interval, average both in FP64.
    Returns (f, U_mean, F_mean[3])."""
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    ncell = solid.size
    U_sum, F_sum = 0.0, np.zeros(3)
    for _ in range(int(n_samples)):
        F = np.zeros(3)
        f, sums, _ = run(solid, f, int(interval), q=q, force=F, **kw)
        U_sum += sums[1] / ncell
        F_sum += F
    return f, U_sum / n_samples, F_sum / n_samples


def developed_average(solid, f, *, min_spinup_ft, max_spinup_ft, drag_tol, average_ft, samples_per_ft,
                      max_steps, q=None, **kw):
    """Developed-flow average (Sec. 4: averaging starts once the drag on the spheres has
    converged, then covers a number of flow-through times), in the reading that a
    flow-through time is T = nx / U_sup of the latest sample:
      1. one sample of nx steps gives the first T;
      2. spin-up in windows of one T, each sampled samples_per_ft times (sub-intervals of
         round(T / samples_per_ft) steps); the window's mean drag F_x is compared with the
         previous window's; T is renewed after every window; the flow is developed when at
         least min_spinup_ft flow-through times have passed and the relative change is below
         drag_tol; the spin-up ends undeveloped after max_spinup_ft flow-through times;
      3. the average: round(average_ft * samples_per_ft) samples, round(T / samples_per_ft)
         steps apart, of U_sup and the drag, averaged in FP64.
    Returns a dict with the averaged U_sup and F, the spin-up and averaging step counts and
    whether the drag converged; max_steps caps the whole run (status 'capped')."""
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = solid.shape
    ncell = solid.size
    state = {"f": f, "total": 0, "U": 0.0, "F": np.zeros(3)}

    def sample(n):
        F = np.zeros(3)
        state["f"], sums, _ = run(solid, state["f"], int(n), q=q, force=F, **kw)
        state["total"] += int(n)
        state["U"] = sums[1] / ncell
        state["F"] = F

    def rnd(x):  # nearest integer, halves away from zero (x > 0 here)
        return int(np.floor(x + 0.5))

    def flow_through():
        if not (abs(state["U"]) > 0):
            raise ValueError("no flow: U_sup is 0")
        return max(1.0, nx / abs(state["U"]))

    sample(max(1, nx))
    T = flow_through()
    spin_ft = state["total"] / T
    spin_steps = state["total"]
    prev, change, developed = None, 1.0, False
    while True:
        sub = max(1, rnd(T / samples_per_ft))
        if state["total"] + sub * samples_per_ft > max_steps:
            return dict(status="capped", spinup_steps=spin_steps, spinup_ft=spin_ft, drag_change=change,
                        f=state["f"])
        wsum = 0.0
        for _ in range(samples_per_ft):
            sample(sub)
            wsum += state["F"][0]
        spin_steps += sub * samples_per_ft
        spin_ft += sub * samples_per_ft / T
        W = wsum / samples_per_ft
        change = 1.0 if prev is None else abs(W - prev) / max(abs(W), 1e-300)
        prev = W
        T = flow_through()
        if spin_ft >= min_spinup_ft and change < drag_tol:
            developed = True
            break
        if spin_ft >= max_spinup_ft:
            break
    sub = max(1, rnd(T / samples_per_ft))
    n_samples = max(1, rnd(average_ft * samples_per_ft))
    U_sum, F_sum, done = 0.0, np.zeros(3), 0
    status = "ok"
    for _ in range(n_samples):
        if state["total"] + sub > max_steps:
            status = "capped"
            break
        sample(sub)
        U_sum += state["U"]
        F_sum += state["F"]
        done += 1
    return dict(status=status, developed=developed, spinup_steps=spin_steps, spinup_ft=spin_ft,
                drag_change=change, average_steps=done * sub, U_sup=U_sum / max(done, 1),
                F=F_sum / max(done, 1), f=state["f"])
