"""ctypes binding of the C ABI in ``include/lbm_gb300.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/liblbm_gb300.so``; this module
declares the structures and prototypes, converts numpy arrays to pointers and turns
non-zero status codes into :class:`LBMError`.  There is no fallback: if the library is
missing or cannot be loaded, :func:`lib` raises.

Device memory is owned by the library.  A CUDA stream handle (``int`` or a
``torch.cuda.Stream``) may be passed at creation; work is queued on it.
"""
from __future__ import annotations

import collections
import ctypes
import os
import threading

import numpy as np

from . import build as _build

Q = 19
SRT, TRT, MRT = 0, 1, 2
SBB, CLI, LIBB, QIBB, IEBB, MR = 0, 1, 2, 3, 4, 5
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
LAYOUT_AB, LAYOUT_AA = 0, 1
DEV_SCALE_AUTO = -1000
BLOCK_AUTO = -1

STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_NO_MEMORY", -3: "LBM_ERR_CUDA",
          -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_NOT_CONVERGED", -6: "LBM_ERR_TIMEOUT",
          -7: "LBM_ERR_STATE", -8: "LBM_ERR_IO", -9: "LBM_ERR_CANCELLED", -10: "LBM_ERR_BOUNDS"}
OK, ERR_ARG, ERR_NO_MEMORY, ERR_CUDA, ERR_DIVERGED, ERR_NOT_CONVERGED, ERR_TIMEOUT, \
    ERR_STATE, ERR_IO, ERR_CANCELLED, ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10
BUILD_CHECKED = 1

STORAGE_BYTES = {F64: 8, F32: 4, F16DEV: 2, BF16DEV: 2}


class LBMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Sphere(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("r", ctypes.c_double)]


class Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("n_spheres", ctypes.c_int32),
        ("spheres", ctypes.POINTER(Sphere)),
        ("flags", ctypes.POINTER(ctypes.c_uint8)),
        ("q", ctypes.POINTER(ctypes.c_double)),
        ("tau", ctypes.c_double), ("delta_rho", ctypes.c_double), ("rho0", ctypes.c_double),
        ("magic_lambda", ctypes.c_double), ("mrt_energy_ratio", ctypes.c_double),
        ("mrt_rates", ctypes.POINTER(ctypes.c_double)),
        ("collision", ctypes.c_int32), ("wall", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("layout", ctypes.c_int32), ("dev_scale_log2", ctypes.c_int32),
        ("block_cells", ctypes.c_int32),
        ("d_p", ctypes.c_double), ("perturb_u", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


class Obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("U_sup", "U_int", "mass", "porosity", "K", "K_app", "Re_p", "Re_K", "beta",
                 "C_F", "F_K", "u_max", "F_x", "F_y", "F_z", "C_D", "C_D_A", "K_star")] + \
               [("steps", ctypes.c_int64), ("n_fluid", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class DevelopOpts(ctypes.Structure):
    _fields_ = [("min_spinup_ft", ctypes.c_double), ("max_spinup_ft", ctypes.c_double),
                ("drag_tol", ctypes.c_double), ("average_ft", ctypes.c_double),
                ("samples_per_ft", ctypes.c_int32), ("reserved", ctypes.c_int32), ("max_steps", ctypes.c_int64)]


class DevelopResult(ctypes.Structure):
    _fields_ = [("avg", Obs), ("flow_through_steps", ctypes.c_double), ("spinup_ft", ctypes.c_double),
                ("average_ft", ctypes.c_double), ("drag_change", ctypes.c_double),
                ("spinup_steps", ctypes.c_int64), ("average_steps", ctypes.c_int64),
                ("developed", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n not in ("avg", "reserved")}
        d["avg"] = self.avg.as_dict()
        return d


class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_cells", "n_fluid", "n_boundary", "n_links", "n_links_cli",
                 "bytes_populations", "bytes_geometry", "kernel_launches")] + \
               [(n, ctypes.c_int32) for n in
                ("block_cells", "storage", "layout", "collision", "wall", "dev_scale_log2")] + \
               [("steps", ctypes.c_int64), ("autotune", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("tune_ms_tiles", ctypes.c_double), ("tune_ms_bricks", ctypes.c_double),
                ("step_warps", ctypes.c_int32), ("shape_source", ctypes.c_int32),
                ("shape_ms", ctypes.c_double * 3)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "pad_"}
        d["shape_ms"] = list(d["shape_ms"])
        return d


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("check_interval", ctypes.c_int32),
                ("max_resident", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "resident", "queued",
                                              "cancelled")] + \
               [(n, ctypes.c_double) for n in ("fluid_updates", "busy_seconds", "mlups")] + \
               [("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_st = ctypes.c_int

PROTOTYPES = {
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_version": (ctypes.c_char_p, []),
    "lbm_create": (_st, [ctypes.POINTER(Desc), _vp, ctypes.POINTER(_vp)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_init_equilibrium": (_st, [_vp]),
    "lbm_step": (_st, [_vp, ctypes.c_int64]),
    "lbm_run_to_convergence": (_st, [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64)]),
    "lbm_observables": (_st, [_vp, ctypes.c_double, ctypes.POINTER(Obs)]),
    "lbm_moment_sums": (_st, [_vp, _dp]),
    "lbm_average": (_st, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(Obs)]),
    "lbm_run_developed": (_st, [_vp, ctypes.POINTER(DevelopOpts), ctypes.c_double, ctypes.POINTER(DevelopResult)]),
    "lbm_fit_barree_conway": (_st, [_dp, _dp, ctypes.c_int32, _dp, _dp, _dp]),
    "lbm_get_populations_f64": (_st, [_vp, _dp]),
    "lbm_set_populations_f64": (_st, [_vp, _dp]),
    "lbm_get_state": (_st, [_vp, _vp, ctypes.c_size_t]),
    "lbm_set_state": (_st, [_vp, _vp, ctypes.c_size_t]),
    "lbm_stage_state": (_st, [_vp, _vp, ctypes.c_size_t]),
    "lbm_apply_staged_state": (_st, [_vp]),
    "lbm_get_velocity_f64": (_st, [_vp, _dp]),
    "lbm_get_flags": (_st, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
    "lbm_get_wall_distances": (_st, [_vp, _dp]),
    "lbm_get_info": (_st, [_vp, ctypes.POINTER(Info)]),
    "lbm_synchronize": (_st, [_vp]),
    "lbm_moment_sums_f64_noalloc": (_st, [_vp, _vp, ctypes.c_int64, ctypes.c_double, _vp, _vp]),
    "lbm_save": (_st, [_vp, ctypes.c_char_p]),
    "lbm_load": (_st, [_vp, ctypes.c_char_p]),
    "lbm_delta_rho_for_re_p": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double]),
    "lbm_batch_create": (_st, [ctypes.POINTER(Desc), ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm_batch_init_equilibrium": (_st, [_vp]),
    "lbm_batch_step": (_st, [_vp, ctypes.c_int64]),
    "lbm_batch_observables": (_st, [_vp, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(Obs)]),
    "lbm_batch_get_populations_f64": (_st, [_vp, ctypes.c_int32, _dp]),
    "lbm_batch_set_populations_f64": (_st, [_vp, ctypes.c_int32, _dp]),
    "lbm_batch_get_info": (_st, [_vp, ctypes.POINTER(Info)]),
    "lbm_server_create": (_st, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)]),
    "lbm_server_submit": (_st, [_vp, ctypes.POINTER(Desc), ctypes.c_double, ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_int64)]),
    "lbm_server_poll": (_st, [_vp, ctypes.c_int64, ctypes.POINTER(Obs), _dp]),
    "lbm_server_drain": (_st, [_vp, ctypes.c_double]),
    "lbm_server_get_stats": (_st, [_vp, ctypes.POINTER(ServerStats)]),
    "lbm_server_cancel": (_st, [_vp, ctypes.c_int64]),
    "lbm_debug_fail_alloc_after": (None, [ctypes.c_int64]),
    "lbm_build_flags": (ctypes.c_uint, []),
    "lbm_debug_corrupt_worklist": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_debug_pack_work_items": (_st, [ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "lbm_server_destroy": (None, [_vp]),
}


def library_variant() -> str:
    """The library variant this process loads: LBM_GB300_VARIANT ("" = the default build,
    "checked" = the bounds-checked build)."""
    return os.environ.get("LBM_GB300_VARIANT", "")


def library_path() -> str:
    return _build.lib_path(library_variant())


def lib(build_if_missing: bool = False):
    """Load the CUDA library (raises if it is missing and build_if_missing is False)."""
    global _lib
    with _lock:
        if _lib is None:
            variant = library_variant()
            path = _build.lib_path(variant)
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
                _build.build(variant=variant)
            L = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().lbm_last_error().decode()


def check(status: int, where: str) -> int:
    if status != OK:
        raise LBMError(status, where, last_error())
    return status


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def make_desc(shape=None, *, nx=None, ny=None, nz=None, spheres=None, flags=None, q=None, tau=0.8,
              delta_rho=0.0, rho0=1.0, magic_lambda=3.0 / 16.0, mrt_energy_ratio=4.6, mrt_rates=None,
              collision=TRT, wall=SBB, storage=F64, layout=LAYOUT_AB, dev_scale_log2=DEV_SCALE_AUTO,
              block_cells=0, d_p=0.0, perturb_u=0.0, seed=0):
    """Build a Desc.  Returns (desc, keepalive): keep both alive until the call returns.

    shape = (nz, ny, nx) or nx/ny/nz keywords; spheres (n, 4) array of (cx, cy, cz, r);
    flags uint8 [nz, ny, nx]; q [19, nz, ny, nx] float64."""
    if shape is not None:
        nz, ny, nx = shape
    keep = []
    d = Desc(nx=nx, ny=ny, nz=nz, tau=tau, delta_rho=delta_rho, rho0=rho0, magic_lambda=magic_lambda,
             mrt_energy_ratio=mrt_energy_ratio, collision=collision, wall=wall, storage=storage,
             layout=layout, dev_scale_log2=dev_scale_log2, block_cells=block_cells, d_p=d_p,
             perturb_u=perturb_u, seed=seed)
    if spheres is not None and len(spheres):
        sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
        keep.append(sp)
        d.n_spheres = sp.shape[0]
        d.spheres = sp.ctypes.data_as(ctypes.POINTER(Sphere))
    if flags is not None:
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        assert fl.size == nx * ny * nz
        keep.append(fl)
        d.flags = fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if q is not None:
        qq = np.ascontiguousarray(q, dtype=np.float64)
        assert qq.size == Q * nx * ny * nz
        keep.append(qq)
        d.q = qq.ctypes.data_as(_dp)
    if mrt_rates is not None:
        mr = np.ascontiguousarray(mrt_rates, dtype=np.float64)
        assert mr.size == Q
        keep.append(mr)
        d.mrt_rates = mr.ctypes.data_as(_dp)
    return d, keep


def _f64(a):
    return a.ctypes.data_as(_dp)


class Context:
    """One periodic cell on the GPU (wraps lbm_ctx)."""

    def __init__(self, desc: Desc | None = None, stream=None, **kw):
        keep = None
        if desc is None:
            desc, keep = make_desc(**kw)
        self._keep = keep
        self.shape = (desc.nz, desc.ny, desc.nx)
        self.storage = desc.storage
        h = _vp()
        check(lib().lbm_create(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(h)), "lbm_create")
        self._h = h
        self._staged = collections.deque()   # host arrays of states staged, not yet applied
        self._applied = []                   # applied; their copies may still be queued

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_destroy(self._h)  # waits for the context's copies
            self._h = None
        self._staged = collections.deque()
        self._applied = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def n_cells(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def init_equilibrium(self):
        check(lib().lbm_init_equilibrium(self._h), "lbm_init_equilibrium")

    def step(self, n: int):
        check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def run_to_convergence(self, tol: float, check_interval: int, max_steps: int):
        done = ctypes.c_int64(0)
        st = lib().lbm_run_to_convergence(self._h, float(tol), int(check_interval), int(max_steps),
                                          ctypes.byref(done))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            check(st, "lbm_run_to_convergence")
        return st, int(done.value)

    def observables(self, K_darcy: float = 0.0) -> dict:
        o = Obs()
        st = lib().lbm_observables(self._h, float(K_darcy), ctypes.byref(o))
        self._applied = []  # the stream has synchronised: applied states' copies are done
        if st not in (OK, ERR_DIVERGED):
            check(st, "lbm_observables")
        d = o.as_dict()
        d["status"] = st
        return d

    def average(self, n_samples: int, sample_interval: int, K_darcy: float = 0.0) -> dict:
        """Time-averaged observables over n_samples * sample_interval further steps."""
        o = Obs()
        st = lib().lbm_average(self._h, int(n_samples), int(sample_interval), float(K_darcy), ctypes.byref(o))
        if st not in (OK, ERR_DIVERGED):
            check(st, "lbm_average")
        d = o.as_dict()
        d["status"] = st
        return d

    def run_developed(self, *, min_spinup_ft=5.0, max_spinup_ft=200.0, drag_tol=1e-4, average_ft=100.0,
                      samples_per_ft=10, max_steps=10 ** 9, K_darcy: float = 0.0) -> dict:
        """Spin up until the drag converges, then time-average (lbm_run_developed)."""
        o = DevelopOpts(min_spinup_ft=float(min_spinup_ft), max_spinup_ft=float(max_spinup_ft),
                        drag_tol=float(drag_tol), average_ft=float(average_ft), samples_per_ft=int(samples_per_ft),
                        max_steps=int(max_steps))
        r = DevelopResult()
        st = lib().lbm_run_developed(self._h, ctypes.byref(o), float(K_darcy), ctypes.byref(r))
        if st not in (OK, ERR_NOT_CONVERGED, ERR_DIVERGED):
            check(st, "lbm_run_developed")
        d = r.as_dict()
        d["status"] = st
        return d

    def moment_sums(self) -> np.ndarray:
        s = np.zeros(4)
        check(lib().lbm_moment_sums(self._h, _f64(s)), "lbm_moment_sums")
        return s

    def get_populations(self, out=None) -> np.ndarray:
        f = out if out is not None else np.empty((Q,) + self.shape)
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.size == Q * self.n_cells
        check(lib().lbm_get_populations_f64(self._h, _f64(f)), "lbm_get_populations_f64")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == Q * self.n_cells
        check(lib().lbm_set_populations_f64(self._h, _f64(f)), "lbm_set_populations_f64")

    def state_dtype(self):
        """numpy dtype of the stored state (16-bit formats as their raw uint16 patterns)."""
        return {F64: np.float64, F32: np.float32, F16DEV: np.uint16, BF16DEV: np.uint16}[self.storage]

    def get_state(self, out=None) -> np.ndarray:
        """The stored fluid-cell state, bit for bit: [19][n_fluid] in the storage type
        (lbm_get_state).  out: an optional C-contiguous array of that shape and dtype
        (e.g. a pinned buffer)."""
        nf = self.info()["n_fluid"]
        s = out if out is not None else np.empty((Q, nf), dtype=self.state_dtype())
        assert s.dtype == self.state_dtype() and s.flags.c_contiguous and s.size == Q * nf
        check(lib().lbm_get_state(self._h, s.ctypes.data, s.nbytes), "lbm_get_state")
        return s

    def set_state(self, s):
        """Set the fluid-cell state from get_state's layout (lbm_set_state)."""
        s = np.ascontiguousarray(s)
        assert s.dtype == self.state_dtype()
        check(lib().lbm_set_state(self._h, s.ctypes.data, s.nbytes), "lbm_set_state")

    def stage_state(self, s):
        """Start copying a state (get_state's layout) into a staging buffer and return
        (lbm_stage_state).  s must stay unchanged until the apply_staged_state that
        consumes it has returned; the context keeps a reference to it until then, so a
        temporary (e.g. a pinned buffer's view) is not freed under the copy.  Returns s."""
        assert s.dtype == self.state_dtype() and s.flags.c_contiguous
        check(lib().lbm_stage_state(self._h, s.ctypes.data, s.nbytes), "lbm_stage_state")
        self._staged.append(s)
        return s

    def apply_staged_state(self):
        """Make the oldest staged state current, queued on the stream (lbm_apply_staged_state)."""
        check(lib().lbm_apply_staged_state(self._h), "lbm_apply_staged_state")
        # the scatter is queued behind the copy, so the host array is no longer read once
        # the stream passes this point; the reference goes when the stream next syncs
        self._applied.append(self._staged.popleft())

    def get_velocity(self) -> np.ndarray:
        u = np.empty((3,) + self.shape)
        check(lib().lbm_get_velocity_f64(self._h, _f64(u)), "lbm_get_velocity_f64")
        return u

    def get_flags(self) -> np.ndarray:
        fl = np.empty(self.shape, dtype=np.uint8)
        check(lib().lbm_get_flags(self._h, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "lbm_get_flags")
        return fl

    def get_wall_distances(self) -> np.ndarray:
        q = np.empty((Q,) + self.shape)
        check(lib().lbm_get_wall_distances(self._h, _f64(q)), "lbm_get_wall_distances")
        return q

    def info(self) -> dict:
        i = Info()
        check(lib().lbm_get_info(self._h, ctypes.byref(i)), "lbm_get_info")
        return i.as_dict()

    def synchronize(self):
        check(lib().lbm_synchronize(self._h), "lbm_synchronize")
        self._applied = []

    def save(self, path: str):
        check(lib().lbm_save(self._h, path.encode()), "lbm_save")

    def load(self, path: str):
        check(lib().lbm_load(self._h, path.encode()), "lbm_load")


class Batch:
    """Many independent periodic cells advanced by one launch per step (wraps lbm_batch)."""

    def __init__(self, descs, stream=None):
        arr = (Desc * len(descs))(*descs)
        self.shapes = [(d.nz, d.ny, d.nx) for d in descs]
        h = _vp()
        check(lib().lbm_batch_create(arr, len(descs), _stream_handle(stream), ctypes.byref(h)),
              "lbm_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self):
        check(lib().lbm_batch_init_equilibrium(self._h), "lbm_batch_init_equilibrium")

    def step(self, n: int):
        check(lib().lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def observables(self, i: int, K_darcy: float = 0.0) -> dict:
        o = Obs()
        st = lib().lbm_batch_observables(self._h, int(i), float(K_darcy), ctypes.byref(o))
        if st not in (OK, ERR_DIVERGED):
            check(st, "lbm_batch_observables")
        d = o.as_dict()
        d["status"] = st
        return d

    def get_populations(self, i: int) -> np.ndarray:
        f = np.empty((Q,) + self.shapes[i])
        check(lib().lbm_batch_get_populations_f64(self._h, int(i), _f64(f)), "lbm_batch_get_populations_f64")
        return f

    def set_populations(self, i: int, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        check(lib().lbm_batch_set_populations_f64(self._h, int(i), _f64(f)), "lbm_batch_set_populations_f64")

    def info(self) -> dict:
        x = Info()
        check(lib().lbm_batch_get_info(self._h, ctypes.byref(x)), "lbm_batch_get_info")
        return x.as_dict()


class Server:
    """Memory-admitted continuous-batching request loop (wraps lbm_server)."""

    def __init__(self, hbm_budget_bytes: int, check_interval: int = 200, max_resident: int = 256):
        o = ServerOpts(hbm_budget_bytes=int(hbm_budget_bytes), check_interval=check_interval,
                       max_resident=max_resident)
        h = _vp()
        check(lib().lbm_server_create(ctypes.byref(o), ctypes.byref(h)), "lbm_server_create")
        self._h = h

    def submit(self, desc: Desc, tol: float, max_steps: int) -> int:
        rid = ctypes.c_int64(0)
        check(lib().lbm_server_submit(self._h, ctypes.byref(desc), float(tol), int(max_steps),
                                      ctypes.byref(rid)), "lbm_server_submit")
        return int(rid.value)

    def poll(self, rid: int):
        """Returns None while running, else (status, obs dict, latency_s)."""
        o = Obs()
        lat = ctypes.c_double(0.0)
        st = lib().lbm_server_poll(self._h, int(rid), ctypes.byref(o), ctypes.byref(lat))
        if st == ERR_STATE:
            return None
        if st == ERR_ARG:
            check(st, "lbm_server_poll")
        return st, o.as_dict(), lat.value

    def drain(self, timeout_s: float = 0.0):
        check(lib().lbm_server_drain(self._h, float(timeout_s)), "lbm_server_drain")

    def cancel(self, rid: int) -> int:
        """Cancel a request (lbm_server_cancel); returns the status (OK, or ERR_STATE if it
        had already finished)."""
        st = lib().lbm_server_cancel(self._h, int(rid))
        if st not in (OK, ERR_STATE):
            check(st, "lbm_server_cancel")
        return st

    def stats(self) -> dict:
        s = ServerStats()
        check(lib().lbm_server_get_stats(self._h, ctypes.byref(s)), "lbm_server_get_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moment_sums_f64_noalloc(f_dev_ptr: int, solid_dev_ptr: int | None, n_cells: int, rho0: float,
                            sums_dev_ptr: int, stream=None) -> None:
    """Moment sums of a device FP64 population field without any allocation inside the
    library (lbm_moment_sums_f64_noalloc); pointers are device addresses (e.g.
    tensor.data_ptr()).  Queued on the stream; does not wait."""
    check(lib().lbm_moment_sums_f64_noalloc(f_dev_ptr, solid_dev_ptr, int(n_cells), float(rho0), sums_dev_ptr,
                                            _stream_handle(stream)), "lbm_moment_sums_f64_noalloc")


def pack_work_items(cells) -> np.ndarray:
    """The step kernels' work items for the fluid cells `cells` (increasing linear indices),
    as lbm_debug_pack_work_items packs them: an int64 array [n_items, 32] of cell indices,
    -1 for padding.  Host code."""
    c = np.ascontiguousarray(cells, dtype=np.uint32)
    n = ctypes.c_int64(0)
    p = c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    st = lib().lbm_debug_pack_work_items(p, int(c.size), None, 0, ctypes.byref(n))
    if st != ERR_ARG or n.value < 0:
        check(st, "lbm_debug_pack_work_items")
    out = np.empty(32 * n.value, dtype=np.uint32)
    check(lib().lbm_debug_pack_work_items(p, int(c.size), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                          int(out.size), ctypes.byref(n)), "lbm_debug_pack_work_items")
    items = out.reshape(-1, 32).astype(np.int64)
    items[items == 0xFFFFFFFF] = -1
    return items


def debug_fail_alloc_after(n: int):
    """Host-side fault injection (lbm_debug_fail_alloc_after): device allocations after the
    next n fail as out of memory; n < 0 disables."""
    lib().lbm_debug_fail_alloc_after(int(n))


def build_flags() -> int:
    """Features the loaded library was compiled with (lbm_build_flags; BUILD_CHECKED)."""
    return int(lib().lbm_build_flags())


def debug_corrupt_worklist(ctx: "Context"):
    """Checked build only: plant an out-of-range cell index in the context's work list
    (lbm_debug_corrupt_worklist); the next reduction reports ERR_BOUNDS."""
    check(lib().lbm_debug_corrupt_worklist(ctx.handle), "lbm_debug_corrupt_worklist")


def fit_barree_conway(re, kstar, init=None):
    """Least-squares Barree-Conway fit K*(Re) = m + (1-m)/(1 + (a Re)^F)^E (lbm_fit_barree_conway).
    Returns ([m, a, E, F], rms)."""
    r = np.ascontiguousarray(re, dtype=np.float64)
    k = np.ascontiguousarray(kstar, dtype=np.float64)
    if r.shape != k.shape or r.ndim != 1:
        raise ValueError("re and kstar must be 1-D arrays of one length")
    out = np.zeros(4)
    rms = ctypes.c_double(0.0)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.float64)
    check(lib().lbm_fit_barree_conway(_f64(r), _f64(k), int(r.size), _f64(ini) if ini is not None else None,
                                      _f64(out), ctypes.byref(rms)), "lbm_fit_barree_conway")
    return out, rms.value


def delta_rho_for_re_p(re_p, tau, d_p, lx, K_D, C_F=0.0, rho0=1.0) -> float:
    return float(lib().lbm_delta_rho_for_re_p(float(re_p), float(tau), float(d_p), int(lx), float(K_D),
                                              float(C_F), float(rho0)))
