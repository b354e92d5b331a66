"""Benchmark of the fused D3Q19 sphere-pack step on GB300.

One benchmark step = one pass of the whole hot path over the workload: TIME_STEPS fused
stream-collide time steps (pull streaming, periodic pressure shift, CLI walls, TRT
collision, store) and the FP64 volume-averaged velocity reduction of the last of them.  The
device-resident number queues its benchmark steps back to back; the end-to-end number
also copies each step's input state in and its sums out, and evaluates the observables on
the host.  The metric is fluid-cell million lattice updates per second (MLUPS) and the
fraction of the HBM roofline the step kernel reaches (19 reads + 19 writes of the stored
format per fluid-cell update).

Workload (default): 128^3 periodic simple-cubic cell, sphere radius 60 (porosity 0.569),
TRT with Lambda = 3/16, CLI walls with analytic q, FP32 storage, in-place AA layout
(159 MB of populations; the A-B layout on the same cell is timed beside it), tau = 0.6,
pressure drop for Re_p ~ 1.  Synthetic, seeded.  The touched state (fluid populations,
91 MB, plus wall slots) is below the 126 MB L2, so every benchmark step is preceded by a
write of 256 MB that flushes L2; within a benchmark step the state stays resident as it
does in any run.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 it runs under torchrun, one independent replica per GPU (the single-cell
path has no exchange step), barrier + max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TIME_STEPS = 1000          # fused time steps per benchmark step (one FP64 reduction each)
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    # name: (L, r, storage, layout, collision, wall, tau, delta_rho)
    "cell128_trt_cli_f32_ab": (128, 60.0, "F32", "AB", "TRT", "CLI", 0.6, 2.0e-5),
    "cell128_trt_cli_f32_aa": (128, 60.0, "F32", "AA", "TRT", "CLI", 0.6, 2.0e-5),
    # a dilute cell (porosity 0.98): the same kernel with few wall lanes
    "cell128_r20_trt_cli_f32_aa": (128, 20.0, "F32", "AA", "TRT", "CLI", 0.6, 2.0e-5),
    "cell128_srt_cli_f32_ab": (128, 60.0, "F32", "AB", "SRT", "CLI", 0.6, 2.0e-5),
    "cell128_mrt_cli_f32_ab": (128, 60.0, "F32", "AB", "MRT", "CLI", 0.6, 2.0e-5),
    "cell256_trt_cli_f16_ab": (256, 120.0, "F16DEV", "AB", "TRT", "CLI", 0.6, 2.0e-5),
    "cell256_trt_cli_bf16_ab": (256, 120.0, "BF16DEV", "AB", "TRT", "CLI", 0.6, 2.0e-5),
    "cell512_trt_cli_bf16_aa": (512, 240.0, "BF16DEV", "AA", "TRT", "CLI", 0.505, 1.0e-3),
    "cell512_trt_cli_f32_aa": (512, 240.0, "F32", "AA", "TRT", "CLI", 0.505, 1.0e-3),
}
# the 128^3 cell's headline runs the in-place AA kernel (the faster of the two there); the
# same line reports the A-B kernel on the same cell under "other_layout"
DEFAULT_WORKLOAD = "cell128_trt_cli_f32_aa"
BYTES = {"F64": 8, "F32": 4, "F16DEV": 2, "BF16DEV": 2}
DTYPE = {"F64": "f64", "F32": "f32", "F16DEV": "f32 (f16 storage)", "BF16DEV": "f32 (bf16 storage)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha() -> str:
    """Short hash of the step-kernel sources, recorded beside the ncu counters."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1508_02960_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("lbm_step.cuh", "lbm_device.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per step-kernel launch from the committed ncu summary of this workload,
    or None when there is none or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for ln in fh:
            if ":" in ln and ln.split(":")[0].strip() in ("kernel_source_sha", "dram_bytes_per_launch"):
                k, v = ln.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("kernel_source_sha") != kernel_source_sha():
        return None
    try:
        return int(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_profile(args):
    """Build the workload's context and run a few steps (the command ncu wraps)."""
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I
    L, r, storage, layout, coll, wall, tau, dr = WORKLOADS[args.workload]
    g = I.centred_sphere(L, r)
    ctx = capi.Context(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=dr, magic_lambda=3 / 16,
                       collision=getattr(capi, coll), wall=getattr(capi, wall), storage=getattr(capi, storage),
                       layout=getattr(capi, "LAYOUT_" + layout), stream=torch.cuda.current_stream())
    ctx.init_equilibrium()
    ctx.step(args.profile_steps)
    print(json.dumps({"workload": args.workload, "steps": args.profile_steps,
                      "U_sup": ctx.observables()["U_sup"]}))
    ctx.close()


def study_precision(args):
    """Error of every storage format against the FP64 oracle in permeability (Eq. Darcy),
    Forchheimer beta (Eq. Forchheimer) and friction factor F_K (Eq. frictionFactor), on the
    precision workloads at the 64^3 downsample (the 256^3 sphere r = 120 and the 40-sphere
    pack, scaled).  The oracle's steady states (Darcy K_D, Re_p ~ 1, Re_p ~ 100; TRT, Lambda
    = 3/16, CLI walls) were computed once by tests/golden/make_precision_reference.py, which
    calls only the oracle; they are read here, not recomputed.  Each GPU format runs the
    oracle's step count from rest, then averages U over ten windows of 100 steps
    (lbm_average; the stochastically rounded 16-bit formats fluctuate at the level of their
    last unit).  beta and F_K use each side's own K_D."""
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    path = os.path.join(ROOT, "tests", "golden", f"precision_reference_{args.study_size}.json")
    with open(path) as fh:
        ref = json.load(fh)
    L = ref["L"]
    summary = {}
    for gname, grec in ref["geometries"].items():
        spheres = np.array(grec["spheres"])
        shape = (L, L, L)
        for fmt in ("F64", "F32", "F16DEV", "BF16DEV"):
            for layout in ("AB", "AA"):
                res = {}
                for pname in ("darcy", "re1", "re100"):
                    pt = grec["points"][pname]
                    with capi.Context(spheres=spheres, shape=shape, tau=pt["tau"], delta_rho=pt["delta_rho"],
                                      magic_lambda=ref["magic_lambda"], collision=capi.TRT, wall=capi.CLI,
                                      storage=getattr(capi, fmt), layout=getattr(capi, "LAYOUT_" + layout),
                                      stream=torch.cuda.current_stream()) as ctx:
                        ctx.init_equilibrium()
                        t0 = time.perf_counter()
                        ctx.step(pt["steps"])
                        K_D = res["darcy"]["K"] if pname != "darcy" else 0.0
                        avg = ctx.average(10, 100, K_D)
                        dt = time.perf_counter() - t0
                        res[pname] = {"K": avg["K"], "U_sup": avg["U_sup"], "Re_p": avg["Re_p"], "beta": avg["beta"],
                                      "C_F": avg["C_F"], "F_K": avg["F_K"], "status": capi.STATUS.get(avg["status"]),
                                      "mlups_incl_host": ctx.info()["n_fluid"] * (pt["steps"] + 1000) / dt / 1e6}
                rec = {"study": "precision", "geometry": gname, "L": L, "format": fmt, "layout": layout,
                       "reference": "FP64 oracle steady states (tests/golden/precision_reference_%d.json)" % L}
                for pname in ("darcy", "re1", "re100"):
                    o, g = grec["points"][pname], res[pname]
                    rec[pname] = {"Re_p": g["Re_p"], "K": g["K"], "K_rel_err": abs(g["K"] / o["K"] - 1.0),
                                  "oracle_converged": o["converged"], "status": g["status"]}
                    if pname != "darcy":
                        for q in ("beta", "F_K"):
                            rec[pname][q] = g[q]
                            rec[pname][q + "_rel_err"] = abs(g[q] / o[q] - 1.0)
                print(json.dumps(rec), flush=True)
                worst = max(rec[p]["K_rel_err"] for p in ("darcy", "re1"))
                summary.setdefault(fmt, {})[f"{gname}_{layout}"] = {
                    "K_rel_err_darcy_max": worst, "K_rel_err_re100": rec["re100"]["K_rel_err"],
                    "beta_rel_err_re100": rec["re100"]["beta_rel_err"], "F_K_rel_err_re100": rec["re100"]["F_K_rel_err"]}
    print(json.dumps({"study": "precision_summary", "L": L,
                      "criterion": "permeability error at most 1e-3 relative against the FP64 oracle in the "
                                   "Darcy regime (Re_p <= 1)", "formats": summary}), flush=True)


def study_sweep(args):
    """The batched Reynolds-number / porosity sweep served through the memory-admitted
    request loop: 64 seeded simple-cubic cells, FP16-deviation storage."""
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I
    pts = I.sweep_points(args.sweep_points)
    # Darcy permeability estimate per point: a short FP32 run at a Stokes pressure drop
    descs, keep = [], []
    for p in pts:
        g = p.geometry
        d, k = capi.make_desc(spheres=g.spheres, shape=g.shape, tau=p.tau, delta_rho=1e-6, collision=capi.TRT,
                              wall=capi.CLI, storage=capi.F32, magic_lambda=p.magic_lambda)
        descs.append(d)
        keep.append(k)
    b = capi.Batch(descs)
    b.init_equilibrium()
    b.step(2000)
    K_est = [b.observables(i)["K"] for i in range(len(pts))]
    b.close()
    sub = []
    for p, K in zip(pts, K_est):
        g = p.geometry
        dr = capi.delta_rho_for_re_p(p.re_p, p.tau, g.d_p, p.L, K, 0.0078)
        d, k = capi.make_desc(spheres=g.spheres, shape=g.shape, tau=p.tau, delta_rho=dr, collision=capi.TRT,
                              wall=capi.CLI, storage=capi.F16DEV, magic_lambda=p.magic_lambda,
                              layout=getattr(capi, "LAYOUT_" + args.sweep_layout))
        sub.append((d, k, p))
    buffers = 2 if args.sweep_layout == "AB" else 1
    total_bytes = sum(buffers * 19 * 2 * p.L ** 3 for p in pts)
    srv = capi.Server(hbm_budget_bytes=int(args.sweep_budget_gb * 2 ** 30), check_interval=200, max_resident=256)
    t0 = time.perf_counter()
    ids = [srv.submit(d, 1e-6, args.study_max_steps) for d, _, _ in sub]
    srv.drain(3600.0)
    wall = time.perf_counter() - t0
    res = [srv.poll(i) for i in ids]
    stats = srv.stats()
    srv.close()
    lat = np.array([r[2] for r in res])
    conv = sum(1 for r in res if r[0] == capi.OK)
    # the same point alone: identical result expected
    checks = []
    for j in (0, len(sub) // 2, len(sub) - 1):
        d, _, p = sub[j]
        ctx = capi.Context(desc=d)
        ctx.init_equilibrium()
        st, steps = ctx.run_to_convergence(1e-6, 200, args.study_max_steps)
        o = ctx.observables()
        ctx.close()
        checks.append({"point": j, "L": p.L, "steps_alone": steps, "steps_mix": res[j][1]["steps"],
                       "U_alone": o["U_sup"], "U_mix": res[j][1]["U_sup"],
                       "identical": o["U_sup"] == res[j][1]["U_sup"] and steps == res[j][1]["steps"]})
    print(json.dumps({"study": "sweep", "layout": args.sweep_layout, "storage": "F16DEV",
                      "points": len(pts), "cells_total": int(sum(p.L ** 3 for p in pts)),
                      "population_bytes_total": total_bytes, "budget_gb": args.sweep_budget_gb,
                      "wall_s": wall, "aggregate_mlups": stats["mlups"], "busy_s": stats["busy_seconds"],
                      "fluid_updates": stats["fluid_updates"], "converged": conv, "capped": len(pts) - conv,
                      "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                      "kernel_launches": stats["kernel_launches"], "alone_vs_mix": checks}), flush=True)


def study_drag(args):
    """Drag studies of Sec. 3 on the simple cubic array: one sphere of radius r = 0.3 L in an
    L^3 periodic cell (reading O12), Stokes flow (delta_rho = 1e-6), FP64 storage, run to a
    steady state (|dU|/U < 1e-10 between checks 500 steps apart).
    E1 grid convergence (Fig. 3): C_D (momentum-exchange drag, Eq. AnalyticForce) for
       L = 10, 15, .., 60 (r = 3 .. 18), every collision operator x every wall rule, tau = 0.8,
       Lambda = 3/16; error against the Richardson extrapolation (second order) of TRT-CLI on
       the two finest lattices -- C_D,ref of the series the paper cites is not printed there.
    E3 viscosity dependence (Fig. 5): K at r = 16.5 (L = 55) for nu = 0.029 .. 0.45,
       relative to the same scheme's K at nu = 1/6."""
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I

    def steady(L, r, coll, wall, tau):
        g = I.centred_sphere(L, r)
        with capi.Context(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=1e-6, magic_lambda=3 / 16,
                          collision=getattr(capi, coll), wall=getattr(capi, wall), storage=capi.F64,
                          stream=torch.cuda.current_stream()) as ctx:
            ctx.init_equilibrium()
            st, steps = ctx.run_to_convergence(1e-10, 500, max(args.study_max_steps, 200000))
            o = ctx.observables()
        return o, capi.STATUS.get(st, st), steps

    schemes = [(c, w) for c in ("SRT", "TRT", "MRT") for w in ("SBB", "CLI", "LIBB", "QIBB", "IEBB", "MR")]
    t0 = time.perf_counter()
    e1 = {}
    Ls = list(range(10, 61, 5))
    for coll, wall in schemes:
        for L in Ls:
            o, st, steps = steady(L, 0.3 * L, coll, wall, 0.8)
            e1[(coll, wall, L)] = dict(C_D=o["C_D"], K=o["K"], F_x=o["F_x"], status=st, steps=steps)
    c1, c2 = e1[("TRT", "CLI", Ls[-2])]["C_D"], e1[("TRT", "CLI", Ls[-1])]["C_D"]
    ratio = (Ls[-1] / Ls[-2]) ** 2
    cd_ext = c2 + (c2 - c1) / (ratio - 1.0)
    rows = []
    for (coll, wall, L), v in e1.items():
        rows.append(dict(scheme=f"{coll}-{wall}", L=L, r=0.3 * L, C_D=v["C_D"], err=abs(v["C_D"] / cd_ext - 1.0),
                         status=v["status"], steps=v["steps"]))
    indep = {}
    for coll, wall in schemes:
        errs = [(L, abs(e1[(coll, wall, L)]["C_D"] / cd_ext - 1.0)) for L in Ls]
        ok = None
        for i, (L, _) in enumerate(errs):
            if all(e < 0.01 for _, e in errs[i:]):
                ok = 0.3 * L
                break
        indep[f"{coll}-{wall}"] = ok
    print(json.dumps({"study": "drag_grid_convergence", "C_D_extrapolated": cd_ext, "tau": 0.8,
                      "grid_independent_r": indep, "rows": rows}), flush=True)

    nus = [0.029, 0.05, 0.1, 1 / 6, 0.25, 0.35, 0.45]
    e3 = []
    for coll, wall in schemes:
        Ks = {}
        for nu in nus:
            o, st, steps = steady(55, 16.5, coll, wall, 0.5 + 3.0 * nu)
            Ks[nu] = (o["K"], st, steps)
        k0 = Ks[1 / 6][0]
        for nu in nus:
            e3.append(dict(scheme=f"{coll}-{wall}", nu=nu, K=Ks[nu][0], K_rel=Ks[nu][0] / k0, status=Ks[nu][1],
                           steps=Ks[nu][2]))
    spread = {}
    for coll, wall in schemes:
        rel = [r["K_rel"] for r in e3 if r["scheme"] == f"{coll}-{wall}"]
        spread[f"{coll}-{wall}"] = max(rel) - min(rel)
    print(json.dumps({"study": "drag_viscosity", "r": 16.5, "L": 55, "K_rel_spread": spread, "rows": e3,
                      "wall_s": time.perf_counter() - t0}), flush=True)


def study_geometry(args):
    """The same step kernel (FP32, AA, TRT, SBB walls, tau = 0.6) on 128^3 cells whose solid
    is shaped to separate what the geometry costs: the r = 60 and r = 20 spheres, a slab of
    55 solid planes (z), of 55 solid rows in every plane (y), of 55 solid cells in every row
    (x; porosity 0.57, as the r = 60 sphere), and no solid at all.  Per geometry: MLUPS and
    the fraction of the copy bandwidth (best of 10 windows of 100 steps)."""
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I

    L = 128
    stream = torch.cuda.current_stream()
    peak, _ = load_peaks()

    def slab(axis):
        f = np.zeros((L, L, L), np.uint8)  # [z][y][x]
        sl = [slice(None)] * 3
        sl[axis] = slice(36, 91)
        f[tuple(sl)] = 1
        return f

    cases = [("sphere_r60", dict(spheres=I.centred_sphere(L, 60.0).spheres)),
             ("sphere_r20", dict(spheres=I.centred_sphere(L, 20.0).spheres)),
             ("slab_z", dict(flags=slab(0))), ("slab_y", dict(flags=slab(1))), ("slab_x", dict(flags=slab(2))),
             ("empty", dict(flags=np.zeros((L, L, L), np.uint8)))]
    rows = []
    for name, geo in cases:
        with capi.Context(shape=(L, L, L), tau=0.6, delta_rho=2e-5, magic_lambda=3 / 16, collision=capi.TRT,
                          wall=capi.SBB, storage=capi.F32, layout=capi.LAYOUT_AA, stream=stream, **geo) as ctx:
            nf = ctx.info()["n_fluid"]
            ctx.init_equilibrium()
            for _ in range(3):
                ctx.step(100)
                ctx.observables()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            best = None
            for _ in range(10):
                e0.record(stream)
                ctx.step(100)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 100
                best = ms if best is None else min(best, ms)
            rec = {"study": "geometry_point", "geometry": name, "n_fluid": nf, "us_per_step": best * 1e3,
                   "mlups": nf / (best * 1e3), "roofline_frac": 38 * 4 * nf / (best * 1e-3) / 1e9 / peak}
            rows.append(rec)
            print(json.dumps(rec), flush=True)
    print(json.dumps({"study": "geometry", "storage": "F32", "layout": "AA", "collision": "TRT", "wall": "SBB",
                      "rows": rows}), flush=True)


def study_kstar(args):
    """Apparent permeability and Forchheimer coefficient over Re_p (Sec. 4) on the simple
    cubic array (one sphere of r = 0.3 L, reading O12), TRT-CLI, FP32 storage, Lambda of
    Table 1 by Re_p, the mean velocity held near 0.05 by the viscosity (tau >= 0.503): K_D
    from a Stokes run, then for each Re_p a developed-flow time average (lbm_run_developed:
    spin-up until the window drag changes < 1e-3 between flow-through times or 200
    flow-through times have passed, then 30 flow-through times averaged (2 for the steady
    Re_p = 1 flow) -- the paper spins up
    400-600 and averages 100-150, at far higher resolution), K* = K_app / K_D (Eq.
    normalizedPermeability), C_F (Eq. Forchheimer), F_K and Re_K (Eq. frictionFactor), and
    the Barree-Conway fit (Eq. AppPer) of K*(Re_p) over the points that finished."""
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I
    L = args.study_size
    r = 0.3 * L
    g = I.centred_sphere(L, r)
    d_p = 2 * r
    t0 = time.perf_counter()

    def ctx(tau, dr, lam):
        return capi.Context(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=dr, magic_lambda=lam,
                            collision=capi.TRT, wall=capi.CLI, storage=capi.F32, stream=torch.cuda.current_stream())

    with ctx(0.8, 1e-6, 3 / 16) as c:
        c.init_equilibrium()
        st, n_darcy = c.run_to_convergence(1e-10, 500, 4000000)
        K_D = c.observables()["K"]
    rows = []
    for re_t in (1.0, 5.0, 10.0, 20.0, 50.0, 80.0, 120.0, 200.0, 300.0, 500.0, 800.0, 1000.0):
        lam = I.table1_lambda(re_t)
        tau = min(1.0, max(0.503, 0.5 + 3.0 * 0.05 * d_p / re_t))   # U near 0.05 where tau allows
        dr = capi.delta_rho_for_re_p(re_t, tau, d_p, L, K_D, 0.0078 if re_t > 1 else 0.0)
        t1 = time.perf_counter()
        with ctx(tau, dr, lam) as c:
            c.init_equilibrium()
            res = c.run_developed(min_spinup_ft=3, max_spinup_ft=200, drag_tol=1e-3,
                                  average_ft=2 if re_t < 5 else 30, samples_per_ft=10, max_steps=2_000_000,
                                  K_darcy=K_D)
        a = res["avg"]
        rows.append(dict(re_target=re_t, Re_p=a["Re_p"], tau=tau, Lambda=lam, delta_rho=dr, K_star=a["K_star"],
                         C_F=a["C_F"], F_K=a["F_K"], Re_K=a["Re_K"], U=a["U_sup"], developed=res["developed"],
                         spinup_ft=res["spinup_ft"], average_ft=res["average_ft"], drag_change=res["drag_change"],
                         steps=res["spinup_steps"] + res["average_steps"], status=capi.STATUS.get(res["status"]),
                         seconds=time.perf_counter() - t1))
        print(json.dumps({"study": "kstar_point", **rows[-1]}), flush=True)
    ok = [x for x in rows if x["status"] == "LBM_OK" and np.isfinite(x["K_star"]) and x["Re_p"] > 0]
    fit = None
    if len(ok) >= 4:
        p, rms = capi.fit_barree_conway([x["Re_p"] for x in ok], [x["K_star"] for x in ok])
        fit = dict(m=p[0], a=p[1], E=p[2], F=p[3], rms=rms, points=len(ok))
    print(json.dumps({"study": "kstar", "L": L, "r": r, "K_D": K_D, "darcy_steps": n_darcy, "rows": rows,
                      "barree_conway": fit, "wall_s": time.perf_counter() - t0}), flush=True)


def dist_setup(n_gpus: int):
    import torch
    rank, world, local = 0, 1, 0
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        local = int(os.environ.get("LOCAL_RANK", 0))
        if world > 1:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", init_method="env://")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_over_ranks(units: float, seconds: float, world: int, device: str = "cuda"):
    """Whole-job figures of independent replicas: (sum of units over ranks, max of the timed
    seconds over ranks).  world <= 1: the local values."""
    if world <= 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(t.item()), float(m.item())


def cpu_baseline(workload: str, target_s: float = 10.0, one_core_s: float = 5.0) -> dict:
    """The FP64 oracle (as it stands) timed on this host's cores on a bounded sample of the
    same workload: the same geometry and operators for as many steps as fit ~target_s with
    every core, then again on one core for ~one_core_s."""
    import numpy as np

    import oracle
    from paper_1508_02960_gb300 import inputs as I
    L, r, storage, layout, coll, wall, tau, dr = WORKLOADS[workload]
    g = I.centred_sphere(L, r)
    solid = oracle.voxelize(g.shape, g.spheres)
    q = oracle.wall_distances(solid, g.spheres)
    f = oracle.init_rest(solid)
    kw = dict(q=q, tau=tau, delta_rho=dr, collision=getattr(oracle, coll), wall=getattr(oracle, wall))
    nf = int((solid == 0).sum())
    t0 = time.perf_counter()
    f, _, _ = oracle.run(solid, f, 1, **kw)
    t1 = time.perf_counter() - t0
    steps = max(1, min(200, int(target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    f, _, _ = oracle.run(solid, f, steps, **kw)
    dt = time.perf_counter() - t0
    cores = oracle.max_threads()
    # the same oracle on one core
    oracle.set_threads(1)
    t0 = time.perf_counter()
    f, _, _ = oracle.run(solid, f, 1, **kw)
    t1c = time.perf_counter() - t0
    steps1 = max(1, min(50, int(one_core_s / max(t1c, 1e-3))))
    t0 = time.perf_counter()
    f, _, _ = oracle.run(solid, f, steps1, **kw)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    del f
    return {"value": nf * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{L}^3 r={r:g} {coll}/{wall} FP64 oracle, {steps} time steps from rest "
                      f"({nf} fluid cells), OpenMP over z", "seconds": round(dt, 3),
            "one_core": {"value": nf * steps1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                         "sample": f"{steps1} further time steps of the same run", "seconds": round(dt1, 3)}}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, each benchmark step a bounded
    sample (a few time steps) of the same workload."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1508_02960_gb300 import inputs as I
    oracle.build()
    L, r, storage, layout, coll, wall, tau, dr = WORKLOADS[args.workload]
    g = I.centred_sphere(L, r)
    solid = oracle.voxelize(g.shape, g.spheres)
    q = oracle.wall_distances(solid, g.spheres)
    f = oracle.init_rest(solid)
    nf = int((solid == 0).sum())
    kw = dict(q=q, tau=tau, delta_rho=dr, collision=getattr(oracle, coll), wall=getattr(oracle, wall))
    t0 = time.perf_counter()
    f, _, _ = oracle.run(solid, f, 1, **kw)
    t1 = time.perf_counter() - t0
    # size each sample so that the whole run stays within about two minutes
    per = max(1, min(TIME_STEPS, int(100.0 / max(args.steps + args.warmup, 1) / max(t1, 1e-3))))
    for _ in range(args.warmup):
        f, _, _ = oracle.run(solid, f, per, **kw)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, sums, _ = oracle.run(solid, f, per, **kw)
    dt = time.perf_counter() - t0
    value = nf * per * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "D3Q19 fluid MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells": L ** 3, "fluid_cells": nf,
                   "time_steps_per_step": per, "note": "FP64 CPU oracle, bounded sample per step"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{per} time steps of {L}^3 per benchmark step"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def other_layout(workload: str):
    """The same cell with the other population layout, when it is a bench workload."""
    for a, b in (("_aa", "_ab"), ("_ab", "_aa")):
        if workload.endswith(a) and workload[: -len(a)] + b in WORKLOADS:
            return workload[: -len(a)] + b
    return None


def time_device(workload, args, stream):
    """Device-resident timing of a workload (warm-up, then args.steps graph launches of
    TIME_STEPS steps, each after an L2 flush, with CUDA events on the launching stream); the
    same procedure as the headline's timed region."""
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I

    L, r, storage, layout, coll, wall, tau, dr = WORKLOADS[workload]
    g = I.centred_sphere(L, r)
    with capi.Context(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=dr, magic_lambda=3 / 16,
                      collision=getattr(capi, coll), wall=getattr(capi, wall), storage=getattr(capi, storage),
                      layout=getattr(capi, "LAYOUT_" + layout), block_cells=args.block, stream=stream) as ctx:
        nf = ctx.info()["n_fluid"]
        ctx.init_equilibrium()
        for _ in range(args.warmup + 2):
            ctx.step(TIME_STEPS)
            ctx.observables()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        flush.fill_(-1.0)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            flush.fill_(float(i))
            ctx.step(TIME_STEPS)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    value = nf * TIME_STEPS * args.steps / (ms * 1e-3) / 1e6
    peak, _ = load_peaks()
    achieved = 38.0 * BYTES[storage] * nf * TIME_STEPS * args.steps / (ms * 1e-3) / 1e9
    return {"workload": workload, "layout": layout, "value": value, "unit": "MLUPS",
            "ms_per_step": ms / args.steps, "roofline_frac": achieved / peak}


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1508_02960_gb300 import capi
    from paper_1508_02960_gb300 import inputs as I

    capi.lib()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    L, r, storage, layout, coll, wall, tau, dr = WORKLOADS[args.workload]
    g = I.centred_sphere(L, r)
    es = BYTES[storage]
    ctx = capi.Context(spheres=g.spheres, shape=g.shape, tau=tau, delta_rho=dr, magic_lambda=3 / 16,
                       collision=getattr(capi, coll), wall=getattr(capi, wall), storage=getattr(capi, storage),
                       layout=getattr(capi, "LAYOUT_" + layout), block_cells=args.block, stream=stream)
    info = ctx.info()
    nf = info["n_fluid"]
    ctx.init_equilibrium()
    ctx.step(2 * TIME_STEPS)
    ctx.observables()

    # ---- device-resident timing -------------------------------------------------------
    for _ in range(args.warmup):
        ctx.step(TIME_STEPS)
        ctx.observables()
    launches0 = ctx.info()["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush.fill_(-1.0)                         # first touch of fresh device memory, outside the timing
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    # every step is queued without a host round trip in between, so that no host-side delay
    # (the clock sampler's driver queries, Python) leaves the GPU idle inside the timed
    # region; each step still ends with its reduction, whose sums stay on the device here
    # (the end-to-end number below reads them back every step)
    for i in range(args.steps):
        flush.fill_(float(i))                 # 256 MB write: nothing of the state left in L2
        ev[i][0].record(stream)
        ctx.step(TIME_STEPS)                  # graph: TIME_STEPS fused steps + reduction
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    obs = ctx.observables()                   # FP64 sums of the last step, convergence quantities
    info_t = ctx.info()
    launches = info_t["kernel_launches"] - launches0
    total_ms = t_start.elapsed_time(t_end)
    graph_ms = [a.elapsed_time(b) for a, b in ev]
    updates = float(nf) * TIME_STEPS * args.steps
    all_updates, total_s = aggregate_over_ranks(updates, total_ms * 1e-3, world)
    total_ms = total_s * 1e3
    value = all_updates / total_s / 1e6

    # per-launch duration of the step kernel inside the timed region
    kernel_ms = statistics.mean(graph_ms) / TIME_STEPS
    alg_bytes = 38.0 * es * nf
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9

    # ---- end-to-end through the C ABI with host buffers ---------------------------------
    # each step's input: the fluid-cell state in the storage type (19 values per fluid
    # cell), copied from pinned host memory; the copy of the next step's input is started
    # before this step's work (lbm_stage_state) and overlaps it, the step itself begins by
    # making its staged input current (lbm_apply_staged_state)
    tdt = {"F64": torch.float64, "F32": torch.float32, "F16DEV": torch.int16, "BF16DEV": torch.int16}[storage]
    s_host = torch.empty((19, nf), dtype=tdt, pin_memory=True).numpy().view(ctx.state_dtype())
    ctx.get_state(s_host)

    def e2e_steps(n):
        ctx.stage_state(s_host)               # H2D of the first step's input
        for i in range(n):
            ctx.apply_staged_state()          # this step's input becomes the state
            if i + 1 < n:
                ctx.stage_state(s_host)       # H2D of the next step's input, during this step
            ctx.step(TIME_STEPS)
            ctx.observables()                 # D2H of the step's result

    e2e_steps(2)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps(args.steps)
    torch.cuda.synchronize()
    all_updates, e2e_s = aggregate_over_ranks(updates, time.perf_counter() - t0, world)
    e2e_value = all_updates / e2e_s / 1e6

    traffic = profiled_traffic(args.workload)
    companion = None
    if world == 1 and other_layout(args.workload):
        companion = time_device(other_layout(args.workload), args, stream)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(args.workload)
        line = {
            "metric": "D3Q19 fluid MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[storage],
            "data": "synthetic",
            "config": {"workload": args.workload, "cells": L ** 3, "fluid_cells": nf, "sphere_radius": r,
                       "storage": storage, "layout": layout, "collision": coll, "wall": wall, "tau": tau,
                       "delta_rho": dr, "time_steps_per_step": TIME_STEPS, "block_cells": info["block_cells"],
                       "step_shape": {"warps": info_t["step_warps"], "source": info_t["shape_source"],
                                      "ms_candidates": [round(x, 5) for x in info_t["shape_ms"]]},
                       "l2": "L2 flushed before every benchmark step (256 MB write); populations %.0f MB, "
                             "%.0f MB of them touched per time step" % (info["bytes_populations"] / 1e6,
                                                                          38.0 * es * nf / 2e6),
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                         "kernel": "step_kernel", "kernel_ms": kernel_ms,
                         "alg_bytes_per_launch": alg_bytes},
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": int(s_host.nbytes),
                    "d2h_bytes_per_step": 72,  # 8 FP64 sums, the status and error words
                    "input": "fluid-cell state in the storage type from pinned memory; the next "
                             "step's copy overlaps this step (lbm_stage_state / lbm_apply_staged_state)"},
            "gpu_launches": int(launches),
            "clocks": clk,
            "observables": {"U_sup": obs["U_sup"], "K": obs["K"], "Re_p": obs["Re_p"]},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if companion is not None:
            line["other_layout"] = companion
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--block", type=int, default=0, help="cells per thread block (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only build the workload and run this many steps (for ncu), no timing")
    ap.add_argument("--study", choices=["precision", "sweep", "drag", "kstar", "geometry"], default=None,
                    help="run a study instead of the benchmark (JSON lines)")
    ap.add_argument("--study-size", type=int, default=64)
    ap.add_argument("--study-max-steps", type=int, default=60000)
    ap.add_argument("--sweep-points", type=int, default=64)
    ap.add_argument("--sweep-budget-gb", type=float, default=6.0)
    ap.add_argument("--sweep-layout", choices=["AB", "AA"], default="AB")
    args = ap.parse_args()
    if args.profile_steps > 0:
        run_profile(args)
        return
    if args.study == "precision":
        study_precision(args)
        return
    if args.study == "sweep":
        study_sweep(args)
        return
    if args.study == "drag":
        study_drag(args)
        return
    if args.study == "kstar":
        study_kstar(args)
        return
    if args.study == "geometry":
        study_geometry(args)
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", 0))
        run_reference(args, rank, int(os.environ.get("WORLD_SIZE", 1)))
        return
    rank, world, local = dist_setup(args.gpus)
    run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
