"""The no-allocation moment sums (lbm_moment_sums_f64_noalloc), for callers that cannot let
a library allocate device memory, against an independent numpy FP64 sum of the same field,
on two calls in a row.

Collected last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


def _numpy_sums(f, solid, rho0):
    """FP64 sums over fluid cells of (rho - rho0, u_x, u_y, u_z), u = rho0^-1 sum e_k f_k, in
    the header's direction order, written out here from the lattice velocities."""
    e = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                  [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.float64)
    fl = f[:, solid.reshape(-1) == 0] if solid is not None else f
    rho = fl.sum(axis=0)
    j = e.T @ fl
    return np.array([(rho - rho0).sum(), j[0].sum() / rho0, j[1].sum() / rho0, j[2].sum() / rho0])


def _check(got, ref, n):
    # the density sum against the mass scale (n cells of rho ~ 1); the momentum sums against
    # their own size (populations ~0.05 cancelling to ~1e-4: rounding ~1e-12 relative)
    assert abs(got[0] - ref[0]) <= 1e-12 * n
    for d in (1, 2, 3):
        assert abs(got[d] - ref[d]) <= 1e-9 * max(abs(ref[d]), 1e-12), (d, got[d], ref[d])


def test_noalloc_moment_sums_of_a_flow_match_numpy(capi):
    import torch
    g = I.Geometry(24, 20, 18, np.array([[11.3, 9.6, 8.7, 6.2]]))
    stream = torch.cuda.current_stream()
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, tau=0.7, delta_rho=1e-4,
                      collision=capi.TRT, wall=capi.CLI, stream=stream) as ctx:
        ctx.init_equilibrium()
        solid = ctx.get_flags().reshape(-1)
        flags = torch.from_numpy(solid).cuda()
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        n = g.n_cells
        for steps in (25, 40):                       # two calls in a row, different states
            ctx.step(steps)
            f_host = ctx.get_populations().reshape(19, n)
            f = torch.from_numpy(f_host).cuda()
            capi.moment_sums_f64_noalloc(f.data_ptr(), flags.data_ptr(), n, 1.0, out.data_ptr(), stream)
            torch.cuda.synchronize()
            _check(out.cpu().numpy(), _numpy_sums(f_host, solid, 1.0), n)
            out.fill_(float("nan"))


@pytest.mark.parametrize("with_flags", [True, False])
def test_noalloc_moment_sums_across_blocks(capi, with_flags):
    """48^3 = 110,592 cells: four blocks of partial sums, then the final kernel's loop over
    them; with a random solid mask, and with no mask (every cell counted)."""
    import torch
    n = 48 ** 3
    rng = np.random.default_rng(41)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rho0 = 1.02
    f_host = w[:, None] * rho0 * (1.0 + 1e-3 * rng.uniform(-1, 1, size=(19, n)))
    solid = (rng.uniform(size=n) < 0.3).astype(np.uint8) if with_flags else None
    f = torch.from_numpy(f_host).cuda()
    fl = torch.from_numpy(solid).cuda() if with_flags else None
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ref = _numpy_sums(f_host, solid, rho0)
    for _ in range(2):                               # two calls in a row share the scratch
        capi.moment_sums_f64_noalloc(f.data_ptr(), fl.data_ptr() if with_flags else None, n, rho0,
                                     out.data_ptr(), stream)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref, n)
        out.fill_(float("nan"))


def test_noalloc_rejects_oversized_and_bad_arguments(capi):
    import torch
    L = capi.lib()
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert L.lbm_moment_sums_f64_noalloc(buf.data_ptr(), None, 268435457, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
    assert "limit" in capi.last_error()
    assert L.lbm_moment_sums_f64_noalloc(None, None, 8, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
    assert L.lbm_moment_sums_f64_noalloc(buf.data_ptr(), None, 0, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
