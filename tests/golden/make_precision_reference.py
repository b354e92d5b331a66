"""Writes precision_reference_64.json: the FP64 oracle's steady states of the mixed-precision
study's workloads, against which the storage formats' permeability, Forchheimer beta and
friction factor are measured.

Workloads (the precision configuration's 256^3 geometries at the 64^3 downsample, geometry
regenerated at that scale): one sphere of r = 120 L/256 centred in an L^3 periodic box, and
the seeded 40-sphere random pack (radii in [18, 30] at 256^3) scaled by L/256; TRT with
Lambda = 3/16 and CLI walls (Sec. 2.1, Sec. 2.2.1), pressure drop across x (Sec. 2.2.2).
Three points per geometry:
  darcy   Stokes flow, tau = 0.8, delta_rho = 1e-6: the Darcy permeability K_D (Eq. Darcy);
  re1     Re_p ~ 1, tau = 0.8, delta_rho from Eq. Darcy with K_D;
  re100   Re_p ~ 100, mean velocity ~ 0.05 (tau = 1/2 + 3 U d_p / Re_p), delta_rho from Eq.
          Forchheimer with K_D and C_F = 0.0078 (the paper's laminar value, Sec. 4).
Each runs from rest in chunks of 200 steps until |U_n - U_{n-1}| < 1e-10 |U_n| between
chunks, or for at most MAX_STEPS steps (recorded as not converged).  Observables by the
oracle's own formulas (Eqs. Darcy, Forchheimer, frictionFactor).

This script calls only the oracle and the seeded input recipes; it is the only writer of the
JSON file.  Run: python tests/golden/make_precision_reference.py [L] [threads]
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1508_02960_gb300 import inputs as I  # noqa: E402

MAX_STEPS = 60000
CHUNK = 200
TOL = 1e-10
C_F_PRIOR = 0.0078
LAMBDA = 3.0 / 16.0


def geometries(L):
    pack = I.random_pack(256, 40, 18.0, 30.0, 20150811)
    return {"sphere": I.centred_sphere(L, 120.0 * L / 256.0),
            "pack40": I.Geometry(L, L, L, pack.spheres * (L / 256.0))}


def steady(solid, q, L, tau, dr):
    f = oracle.init_rest(solid)
    U_old, n = None, 0
    kw = dict(q=q, tau=tau, delta_rho=dr, collision=oracle.TRT, wall=oracle.CLI, magic_lambda=LAMBDA)
    while n < MAX_STEPS:
        f, sums, _ = oracle.run(solid, f, CHUNK, **kw)
        n += CHUNK
        U = sums[1] / L ** 3
        if U_old is not None and abs(U - U_old) < TOL * abs(U):
            return U, n, True
        U_old = U
    return U, n, False


def main():
    L = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    if len(sys.argv) > 2:
        oracle.set_threads(int(sys.argv[2]))
    out = {"description": __doc__.strip().split("\n\n")[0], "L": L, "magic_lambda": LAMBDA, "wall": "CLI",
           "collision": "TRT", "chunk": CHUNK, "tol": TOL, "max_steps": MAX_STEPS, "geometries": {}}
    for name, g in geometries(L).items():
        t0 = time.time()
        solid = oracle.voxelize(g.shape, g.spheres)
        q = oracle.wall_distances(solid, g.spheres)
        d_p = g.d_p
        rec = {"spheres": g.spheres.tolist(), "d_p": d_p, "n_fluid": int((solid == 0).sum()), "points": {}}
        # Darcy permeability
        tau, dr = 0.8, 1e-6
        U, n, conv = steady(solid, q, L, tau, dr)
        K_D = oracle.observables(U, tau, dr, L, d_p)[1]
        rec["points"]["darcy"] = dict(tau=tau, delta_rho=dr, steps=n, converged=conv, U_sup=U, K=K_D,
                                      Re_p=oracle.observables(U, tau, dr, L, d_p)[2])
        for pname, re_p in (("re1", 1.0), ("re100", 100.0)):
            if re_p <= 1.0:
                tau = 0.8
                nu = (tau - 0.5) / 3.0
                U_t = re_p * nu / d_p
                gradP = nu * U_t / K_D
            else:
                U_t = 0.05
                tau = 0.5 + 3.0 * U_t * d_p / re_p
                nu = (tau - 0.5) / 3.0
                gradP = nu * U_t / K_D + C_F_PRIOR / math.sqrt(K_D) * U_t * U_t
            dr = 3.0 * L * gradP
            U, n, conv = steady(solid, q, L, tau, dr)
            o = oracle.observables(U, tau, dr, L, d_p, K_D)
            rec["points"][pname] = dict(tau=tau, delta_rho=dr, steps=n, converged=conv, U_sup=U, K=o[1],
                                        Re_p=o[2], beta=o[3], C_F=o[4], F_K=o[5], Re_K=o[6])
            print(name, pname, rec["points"][pname], flush=True)
        rec["oracle_seconds"] = round(time.time() - t0, 1)
        out["geometries"][name] = rec
        print(name, "done", rec["oracle_seconds"], "s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"precision_reference_{L}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
