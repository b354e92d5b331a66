"""Host-side checks of the C ABI: the library loads, exports every function the header
declares, the ctypes structures match the C layout, and argument validation fails
cleanly before any GPU call.  No GPU compute is issued here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import torch

from paper_1508_02960_gb300 import build as B
from paper_1508_02960_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_gb300.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return capi.lib()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^LBM_API[^(]*?\b(lbm_\w+)\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported_and_bound(L):
    names = declared_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(L, n), n
        assert n in capi.PROTOTYPES, f"{n} missing from the binding"
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("lbm_")}
    assert exported == set(names)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lbm_gb300.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_desc), sizeof(lbm_obs), sizeof(lbm_info),
         sizeof(lbm_server_opts), sizeof(lbm_server_stats), sizeof(lbm_sphere));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(lbm_desc, tau), offsetof(lbm_desc, collision),
         offsetof(lbm_desc, d_p), offsetof(lbm_desc, seed), offsetof(lbm_info, block_cells));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_develop_opts), sizeof(lbm_develop_result),
         offsetof(lbm_develop_result, developed), offsetof(lbm_obs, K_star), offsetof(lbm_develop_opts, max_steps),
         offsetof(lbm_info, autotune), offsetof(lbm_info, tune_ms_bricks), offsetof(lbm_info, step_warps),
         offsetof(lbm_info, shape_ms));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:3]
    sizes = [int(v) for v in a.split()]
    offs = [int(v) for v in b.split()]
    assert sizes == [ctypes.sizeof(capi.Desc), ctypes.sizeof(capi.Obs), ctypes.sizeof(capi.Info),
                     ctypes.sizeof(capi.ServerOpts), ctypes.sizeof(capi.ServerStats), ctypes.sizeof(capi.Sphere)]
    assert offs == [capi.Desc.tau.offset, capi.Desc.collision.offset, capi.Desc.d_p.offset,
                    capi.Desc.seed.offset, capi.Info.block_cells.offset]
    assert [int(v) for v in c.split()] == [ctypes.sizeof(capi.DevelopOpts), ctypes.sizeof(capi.DevelopResult),
                                           capi.DevelopResult.developed.offset, capi.Obs.K_star.offset,
                                           capi.DevelopOpts.max_steps.offset, capi.Info.autotune.offset,
                                           capi.Info.tune_ms_bricks.offset, capi.Info.step_warps.offset,
                                           capi.Info.shape_ms.offset]


@pytest.mark.parametrize("bad", [
    dict(tau=0.5), dict(tau=float("nan")), dict(nx=0), dict(collision=7), dict(wall=6), dict(wall=-1),
    dict(wall=2, layout=1), dict(wall=5, layout=1), dict(wall=4, tau=2.0), dict(storage=9),
    dict(layout=3), dict(block_cells=100), dict(block_cells=64), dict(block_cells=2048), dict(block_cells=512),
    dict(block_cells=-2), dict(nx=1024, ny=1024, nz=1024), dict(perturb_u=0.5),
    dict(spheres=[[1, 1, 1, -2.0]]), dict(dev_scale_log2=99), dict(magic_lambda=-1.0),
    # centres far outside the box (the device folds them in one box length at a time)
    dict(spheres=[[1e17, 1, 1, 2.0]]), dict(spheres=[[4, -600.0, 4, 2.0]]), dict(spheres=[[4, 4, 1e10, 2.0]]),
])
def test_invalid_descriptor_rejected_before_gpu(L, bad):
    kw = dict(nx=8, ny=8, nz=8, tau=0.8)
    kw.update(bad)
    d, keep = capi.make_desc(**kw)
    h = ctypes.c_void_p()
    st = L.lbm_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == capi.ERR_ARG
    assert h.value is None
    assert capi.last_error()


def test_batch_rejects_mixed_formats(L):
    d1, k1 = capi.make_desc(nx=8, ny=8, nz=8, storage=capi.F32)
    d2, k2 = capi.make_desc(nx=8, ny=8, nz=8, storage=capi.F64)
    arr = (capi.Desc * 2)(d1, d2)
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(arr, 2, None, ctypes.byref(h)) == capi.ERR_ARG
    d3, k3 = capi.make_desc(nx=8, ny=8, nz=8, storage=capi.F32, layout=capi.LAYOUT_AA)
    arr = (capi.Desc * 2)(d1, d3)                  # one layout per batch
    assert L.lbm_batch_create(arr, 2, None, ctypes.byref(h)) == capi.ERR_ARG


def test_null_arguments(L):
    h = ctypes.c_void_p()
    assert L.lbm_create(None, None, ctypes.byref(h)) == capi.ERR_ARG
    assert L.lbm_step(None, 1) == capi.ERR_ARG
    assert L.lbm_observables(None, 0.0, None) == capi.ERR_ARG
    buf = ctypes.create_string_buffer(16)
    assert L.lbm_get_state(None, buf, 16) == capi.ERR_ARG
    assert L.lbm_set_state(None, buf, 16) == capi.ERR_ARG
    assert L.lbm_stage_state(None, buf, 16) == capi.ERR_ARG
    assert L.lbm_apply_staged_state(None) == capi.ERR_ARG
    assert L.lbm_debug_corrupt_worklist(None) == capi.ERR_ARG
    assert L.lbm_server_cancel(None, 0) == capi.ERR_ARG
    assert L.lbm_build_flags() & capi.BUILD_CHECKED == 0       # the default build
    L.lbm_destroy(None)
    L.lbm_batch_destroy(None)
    L.lbm_server_destroy(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_valid_descriptor_without_gpu_reports_cuda_error(L):
    d, keep = capi.make_desc(nx=8, ny=8, nz=8, tau=0.8)
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(d), None, ctypes.byref(h)) == capi.ERR_CUDA
    assert h.value is None


def test_delta_rho_for_re_p_inverts_forchheimer(L):
    """Feeding the returned delta_rho back into Eq. Forchheimer gives the target Re_p."""
    for re_p, tau, d_p, lx, K, C_F in ((1e-3, 0.6, 120.0, 128, 40.0, 0.0), (10.0, 0.55, 60.0, 64, 9.0, 0.0078),
                                       (500.0, 0.51, 90.0, 96, 20.0, 0.023)):
        dr = capi.delta_rho_for_re_p(re_p, tau, d_p, lx, K, C_F)
        nu = (tau - 0.5) / 3
        gradP = dr / 3 / lx
        # solve mu U / K + C_F / sqrt(K) U^2 = gradP for U
        a, b, c = C_F / np.sqrt(K), nu / K, -gradP
        U = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a) if a > 0 else -c / b
        assert U * d_p / nu == pytest.approx(re_p, rel=1e-10)
