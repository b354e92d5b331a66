"""The bounds-checked build (LBM_CHECKED; library variant "checked").

Every index the step kernels use is tested against the extent of its array there.  A
violation skips the access and is reported as LBM_ERR_BOUNDS at the next reduction.
The checked library runs in child processes (a process loads one library variant):

* a planted out-of-range cell index (lbm_debug_corrupt_worklist, which exists only in the
  checked build) is reported, and the access it would have made is skipped;
* the parity tests against the oracle pass unchanged with every check compiled in, so no
  correct run trips a check;
* the default build reports no checked features and refuses to plant the index.

The population buffers of every build carry NaN canaries in their padding, so a kernel
that read there would turn the parity tests' results non-finite.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1508_02960_gb300 import capi as C
    C.lib(build_if_missing=True)
    return C


@pytest.fixture(scope="module")
def checked_lib():
    from paper_1508_02960_gb300 import build as B
    return B.build(variant="checked")


def _child(code: str, timeout: float = 600.0):
    env = dict(os.environ, LBM_GB300_VARIANT="checked")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r.stdout


def test_default_build_has_no_checks(capi):
    from paper_1508_02960_gb300 import inputs as I
    assert capi.build_flags() & capi.BUILD_CHECKED == 0
    g = I.centred_sphere(16, 5.0)
    with capi.Context(spheres=g.spheres, shape=g.shape, tau=0.7, storage=capi.F32) as ctx:
        with pytest.raises(capi.LBMError) as e:
            capi.debug_corrupt_worklist(ctx)
        assert e.value.status == capi.ERR_STATE


CORRUPT = r"""
from paper_1508_02960_gb300 import capi as C, inputs as I
C.lib(build_if_missing=True)
assert C.build_flags() & C.BUILD_CHECKED, "not the checked build"
for storage, layout, wall in [(C.F32, C.LAYOUT_AB, C.CLI), (C.F64, C.LAYOUT_AA, C.CLI),
                              (C.BF16DEV, C.LAYOUT_AB, C.QIBB)]:
    g = I.centred_sphere(32, 10.0)
    kw = dict(spheres=g.spheres, shape=g.shape, tau=0.7, delta_rho=1e-4, storage=storage, layout=layout,
              wall=wall, collision=C.TRT)
    with C.Context(**kw) as ctx:                  # clean run: no check fires
        ctx.init_equilibrium()
        ctx.step(20)
        assert ctx.observables()["U_sup"] > 0
    with C.Context(**kw) as ctx:                  # planted index: reported, not dereferenced
        ctx.init_equilibrium()
        ctx.step(2)
        ctx.observables()
        C.debug_corrupt_worklist(ctx)
        ctx.step(3)
        try:
            ctx.observables()
            raise SystemExit("the out-of-range cell was not reported")
        except C.LBMError as e:
            assert e.status == C.ERR_BOUNDS, e
    with C.Context(**kw) as ctx:                  # and the library goes on working
        ctx.init_equilibrium()
        ctx.step(5)
        assert ctx.observables()["U_sup"] > 0
print("ok")
"""


def test_planted_index_is_reported(capi, checked_lib):
    assert "ok" in _child(CORRUPT)


def test_parity_suite_under_checked_build(capi, checked_lib):
    """The step-kernel parity tests against the oracle, every wall rule and the TMA bricks,
    rerun with the checked library: any check that fired would fail them (ERR_BOUNDS)."""
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_walls.py", "tests/test_gpu_tma.py"]
    out = _child("import sys, pytest; sys.exit(pytest.main(['-q', '-x', '-m', 'gpu', '-p', 'no:cacheprovider'] + "
                 + repr(files) + "))", timeout=1800.0)
    assert " passed" in out and " failed" not in out
