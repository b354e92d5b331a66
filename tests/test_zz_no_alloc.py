"""The no-allocation moment sums (for callers that cannot let the library allocate device
memory) agree with the context's own moment sums, on two calls in a row.

Collected last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1508_02960_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_moment_sums_match_context():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi
    capi.lib(build_if_missing=True)
    g = I.Geometry(24, 20, 18, np.array([[11.3, 9.6, 8.7, 6.2]]))
    stream = torch.cuda.current_stream()
    with capi.Context(spheres=g.spheres, shape=g.shape, storage=capi.F64, tau=0.7, delta_rho=1e-4,
                      collision=capi.TRT, wall=capi.CLI, stream=stream) as ctx:
        ctx.init_equilibrium()
        flags = torch.from_numpy(ctx.get_flags().reshape(-1)).cuda()
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        n = g.n_cells
        for steps in (25, 40):                       # two calls in a row, different states
            ctx.step(steps)
            ref = ctx.moment_sums()                  # the context's own reduction
            f = torch.from_numpy(ctx.get_populations().reshape(19, n)).cuda()
            capi.moment_sums_f64_noalloc(f.data_ptr(), flags.data_ptr(), n, 1.0, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            # u is a difference of populations ~0.05 cancelling to ~1e-5: both sums carry
            # ~1e-12 relative rounding; the density sum is compared against the mass scale
            assert abs(got[0] - ref[0]) <= 1e-9 * n
            for d in (1, 2, 3):
                assert abs(got[d] - ref[d]) <= 1e-9 * max(abs(ref[d]), 1e-9)
            out.fill_(float("nan"))


def test_noalloc_rejects_oversized_and_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi
    L = capi.lib(build_if_missing=True)
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert L.lbm_moment_sums_f64_noalloc(buf.data_ptr(), None, 268435457, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
    assert "limit" in capi.last_error()
    assert L.lbm_moment_sums_f64_noalloc(None, None, 8, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
    assert L.lbm_moment_sums_f64_noalloc(buf.data_ptr(), None, 0, 1.0, buf.data_ptr(), None) == capi.ERR_ARG
