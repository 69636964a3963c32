"""Writes cavity_c1_hweno_solve.json: the oracle's steady solve of the lid-driven
cavity workload with the compact scheme, for the GPU test that runs the same
solve through the C ABI (tests/test_gpu_steady_cavity.py).

Workload: unit cube, 8 x 8 x 8 hexahedra split into 3,072 tetrahedra, interior
vertices jittered by up to 10 % of h, cells permuted (inputs.cavity_mesh(8));
lid y = 1 moving along +x at speed 1, Mach 0.15, Re 100, Pr 0.72, isothermal
no-slip walls (Sec. 5.1); compact HWENO reconstruction with nonlinear weights,
GMRES with Krylov dimension 10, 3 restarts, 2 Jacobi sweeps, CFL 10 (Sec. 5),
from rest, Algorithm 1 until the L1 density residual has dropped to 1e-8 of its
largest value. Stored: the step count, the whole residual history, the state
(Q and the cell-averaged gradients G) of 256 seeded cells, and norms of the
final state. Only the oracle computes anything here.

Run from the repository root: python tests/golden/make_cavity_c1_solve.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O                                   # noqa: E402
from paper_2304_09485_gb300 import inputs as I       # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity_c1_hweno_solve.json")
DROP, MAX_STEPS = 1e-8, 4000
SETTINGS = dict(scheme=1, weights=0, Pr=0.72, cfl=10.0, krylov_dim=10, restarts=3, jacobi_sweeps=2)


def main():
    m = I.cavity_mesh(8)
    cond = I.cavity_conditions(0.15, 100.0)
    om = O.OracleMesh(m)
    Q0 = I.state_from_conditions(m.n_tet, cond)
    G0 = np.zeros((m.n_tet, 15))
    p = O.make_params(**SETTINGS, **cond)
    t0 = time.time()
    Q, G, hist, conv = om.solve_steady(p, Q0, G0, drop=DROP, max_steps=MAX_STEPS)
    cells = np.sort(np.random.default_rng(I.BASE_SEED + 800).choice(m.n_tet, 256, replace=False))
    out = {
        "_about": __doc__.split("\n\n")[0] + " Written by tests/golden/make_cavity_c1_solve.py (oracle only).",
        "settings": {**SETTINGS, "Mach": 0.15, "Re": 100.0, "lid_speed": 1.0, "drop": DROP, "max_steps": MAX_STEPS,
                     "mesh": "inputs.cavity_mesh(8)", "weno_eps": p.weno_eps},
        "converged": bool(conv), "steps": int(len(hist) - 1), "hist": [float(h) for h in hist],
        "cells": cells.tolist(), "Q": Q[cells].tolist(), "G": G[cells].tolist(),
        "Q_norm": float(np.linalg.norm(Q)), "G_norm": float(np.linalg.norm(G)),
        "oracle_seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"{'converged' if conv else 'NOT converged'} after {len(hist) - 1} steps, "
          f"final drop {hist[-1] / hist.max():.3e}, {time.time() - t0:.0f} s -> {OUT}")


if __name__ == "__main__":
    main()
