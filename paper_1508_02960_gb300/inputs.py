"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds geometry and parameter recipes only (sphere lists, box sizes,
relaxation times, pressure drops, noise arrays); it contains none of the lattice
Boltzmann arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper's geometry is a simple-cubic array of equal spheres (one sphere per periodic
cell, Sec. 3) and a settled random bed (Sec. 5).  Random numbers come from SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
doubles from its top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator: a Weyl sequence with step 0x9e3779b97f4a7c15 followed by
    the variant-13 MurmurHash3 finaliser."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()


@dataclass
class Geometry:
    """A periodic box (nx, ny, nz) holding spheres (n, 4) = (cx, cy, cz, r)."""
    nx: int
    ny: int
    nz: int
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def d_p(self) -> float:
        """Volume-mean sphere diameter (the particle diameter of Re_p)."""
        if len(self.spheres) == 0:
            return 0.0
        r = self.spheres[:, 3]
        return 2.0 * float(np.cbrt(np.mean(r ** 3)))


def centred_sphere(L: int, r: float, *, ny: int | None = None, nz: int | None = None,
                   shift=(0.0, 0.0, 0.0)) -> Geometry:
    """Simple-cubic pack cell: one sphere of radius r centred in an L^3 periodic box
    (optionally displaced by ``shift`` cells, as in the paper's displacement study)."""
    ny = L if ny is None else ny
    nz = L if nz is None else nz
    c = np.array([[L / 2 + shift[0], ny / 2 + shift[1], nz / 2 + shift[2], float(r)]])
    return Geometry(L, ny, nz, c)


def random_pack(L: int, n: int, r_min: float, r_max: float, seed: int, *, gap: float = 1.0,
                max_tries: int = 1_000_000) -> Geometry:
    """Random sequential addition of n non-overlapping spheres in an L^3 periodic box.

    For each sphere: radius uniform in [r_min, r_max] drawn before the centre, centre
    uniform in [0, L)^3; a candidate is rejected when its minimum-image distance to an
    accepted sphere is below r1 + r2 + gap (gap = 1 keeps a fluid cell in every gap)."""
    rng = SplitMix64(seed)
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_pack: packing jammed")
        r = rng.uniform_range(r_min, r_max)
        c = np.array([rng.uniform() * L, rng.uniform() * L, rng.uniform() * L])
        ok = True
        for s in out:
            d = c - s[:3]
            d -= L * np.round(d / L)
            if math.sqrt(float(d @ d)) < r + s[3] + gap:
                ok = False
                break
        if ok:
            out.append(np.array([c[0], c[1], c[2], r]))
    return Geometry(L, L, L, np.array(out))


def slit_channel(n_fluid: int, nx: int = 4, nz: int = 1):
    """Flag field uint8 [nz, ny, nx] of a plane channel: one solid row at y = 0 and
    n_fluid fluid rows above it (periodic in y, so the solid row bounds both sides)."""
    ny = n_fluid + 1
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[:, 0, :] = 1
    return flags


def noise(shape, seed: int) -> np.ndarray:
    """Seeded uniform noise in [-1, 1) of the given shape (numpy PCG64 stream)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


# Re_p ranges and magic parameter of Table 1 (Sec. 4): (upper bound of Re_p, Lambda).
TABLE1_LAMBDA = ((0.01, 1.0 / 4.0), (198.0, 3.0 / 16.0), (509.0, 1.0 / 12.0),
                 (1008.0, 1e-5), (1617.0, 1e-5), (5813.0, 6e-6))


def table1_lambda(re_p: float) -> float:
    """Magic parameter Lambda for a target Re_p, from the paper's Table 1."""
    for hi, lam in TABLE1_LAMBDA:
        if re_p <= hi:
            return lam
    return TABLE1_LAMBDA[-1][1]


@dataclass
class SweepPoint:
    """One independent sphere cell of the batched Reynolds-number / porosity sweep."""
    L: int
    r: float
    re_p: float
    tau: float
    magic_lambda: float

    @property
    def geometry(self) -> Geometry:
        return centred_sphere(self.L, self.r)


def sweep_points(n: int = 64, seed: int = 20150811, *, edges=(48, 64, 96, 128, 160),
                 r_frac=(0.30, 0.49), re_p=(1e-4, 500.0), u_max: float = 0.1) -> list:
    """Seeded sweep of n simple-cubic cells: edge from ``edges``, r = U[r_frac]*L,
    target Re_p log-uniform in ``re_p``, tau uniform in [0.51, min(1, tau_max)] where
    tau_max keeps the lattice velocity of the target Re_p below u_max."""
    rng = SplitMix64(seed)
    pts = []
    for _ in range(n):
        L = int(edges[int(rng.uniform() * len(edges)) % len(edges)])
        r = rng.uniform_range(*r_frac) * L
        lo, hi = math.log(re_p[0]), math.log(re_p[1])
        rp = math.exp(rng.uniform_range(lo, hi))
        d_p = 2.0 * r
        tau_max = 0.5 + 3.0 * u_max * d_p / rp
        tau = rng.uniform_range(0.51, max(0.51, min(1.0, tau_max)))
        pts.append(SweepPoint(L, r, rp, tau, table1_lambda(rp)))
    return pts


# The workloads (sizes follow the benchmark configurations of this project).
def config_reference_32() -> dict:
    """32^3 cell, sphere r = 12, TRT Lambda = 3/16, SBB, FP64, delta_rho = 1e-5,
    tau = 0.8, rest start, 2000 steps."""
    return dict(geometry=centred_sphere(32, 12.0), tau=0.8, delta_rho=1e-5,
                magic_lambda=3.0 / 16.0, steps=2000)


def config_cell_128() -> dict:
    """128^3 cell, sphere r = 60, CLI walls, FP32, tau = 0.6."""
    return dict(geometry=centred_sphere(128, 60.0), tau=0.6)


def config_precision_256() -> dict:
    """256^3 cell with r = 120, and a 40-sphere random pack (r in [18, 30])."""
    return dict(geometry=centred_sphere(256, 120.0),
                pack=random_pack(256, 40, 18.0, 30.0, 20150811))


def config_turbulent_512() -> dict:
    """512^3 cell, sphere r = 240, AA layout, BF16-deviation storage."""
    return dict(geometry=centred_sphere(512, 240.0), tau=0.505)
