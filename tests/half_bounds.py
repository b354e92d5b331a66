"""Error bounds of the 16-bit deviation formats against the FP64 oracle, shared by the GPU
parity tests (not a test module).

A step of the GPU path reads stored 16-bit deviations g = f - w rho0, collides in FP32 and
stores the results with stochastic rounding: each stored value lies within one unit in the
last place (ulp) of the format of the exact result, plus the FP32 collision error (a few
dozen roundings of operands up to max|g|).  Wall links add one more rounding: the own-cell
part of a cut link's rule waits one step in a solid slot (A-B) or in the slot the next
step's pull reads (AA), stored in the format, and the collision spreads its error over the
cell's outputs; it is computed from the unrounded post-collision values, so against an
oracle step taken from the exported (rounded) state it differs by up to an ulp of each
value it combines."""
import numpy as np


def round_bf16(x):
    """Round-to-nearest-even of float64 values to bfloat16 (through float32)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def ulp_bf16(x):
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-38)))
    return 2.0 ** (e - 7)


def ulp_f16(x):
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -14)))
    return 2.0 ** (e - 10)


def storable(fmt, xi, scale_log2):
    """Deviations xi made exactly storable in the format, and the format's ulp function (in
    deviation units)."""
    if fmt == "F16DEV":
        sc = 2.0 ** scale_log2
        return np.float16(xi * sc).astype(np.float64) / sc, (lambda v: ulp_f16(v * sc) / sc)
    return round_bf16(xi), ulp_bf16


def wall_cells(orc, solid):
    """Fluid cells with at least one solid pull source."""
    e, _, _ = orc.lattice()
    wc = np.zeros(solid.shape, bool)
    for k in range(1, 19):
        wc |= np.roll(solid, shift=(e[k, 2], e[k, 1], e[k, 0]), axis=(0, 1, 2)) == 1
    return wc & (solid == 0)


def check_step(orc, solid, w, f_gpu, f_ref, f_prev, ulp, walls):
    """Assert one GPU step f_gpu against the oracle step f_ref taken from the same state f_prev
    (all FP64 [19, nz, ny, nx]); walls: include the wall-link allowance."""
    m = solid == 0
    g_gpu = (f_gpu - w[:, None, None, None])[:, m]
    g_ref = (f_ref - w[:, None, None, None])[:, m]
    err = np.abs(g_gpu - g_ref)
    floor = 64 * 2.0 ** -24 * np.abs(g_ref).max()
    bound = ulp(g_ref) * 1.0001 + floor
    if walls:
        amax = np.abs(f_prev - w[:, None, None, None]).max(axis=0)
        bound = bound + np.where(wall_cells(orc, solid), 4 * ulp(2 * amax), 0.0)[m][None, :]
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float((err / bound).max()))
