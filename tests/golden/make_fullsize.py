"""Writes the oracle's solutions of the two full-size benchmark workloads.

Run from the repository root:  python tests/golden/make_fullsize.py [elastance|mobility|all]

It calls only the FP64 oracle (`oracle/`) on the seeded synthetic inputs of
`synth/`; nothing here touches the CUDA library.  Outputs (text, one value per
row, 17 significant digits):

  stars100_M25600_elastance.txt   100 star curves x 256 nodes (M = 25,600),
      charges from the generator (seed 1000): the conductor potentials phi_i of
      the dense Nystrom system of eq. ModRep2 (Section 3) solved by LU.
  ellipses400_M51200_mobility.txt 400 ellipses x 128 nodes (M = 51,200, 2M
      unknowns), forces and torques from the generator (seed 2000): the rigid
      motions (v_x, v_y, omega) of eq. ModRep2Stokes (Section 4); the dense
      matrix (84 GB) does not fit host memory, so the oracle solves the same
      system by block-Jacobi-preconditioned GMRES on row-blocked operator
      applications with FP64 refinement down to a true relative residual of
      1e-13 (oracle.stokes.solve_gmres).

Each file records a fingerprint of its inputs (node count, sums of the node
coordinates and of the loads) so that a test can tell a changed generator from
a wrong solver.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import laplace, stokes  # noqa: E402


def fingerprint(g: dict, load: np.ndarray) -> list[str]:
    return [f"M {g['x'].size}", f"N {g['body_start'].size - 1}",
            f"sum_x {float(np.sum(g['x'])):.17e}", f"sum_y {float(np.sum(g['y'])):.17e}",
            f"sum_load {float(np.sum(np.abs(load))):.17e}"]


def elastance() -> None:
    g = synth.star_grid(seed=1000)
    t0 = time.perf_counter()
    res = laplace.solve(g, g["q"])
    dt = time.perf_counter() - t0
    lines = ["# Oracle potentials phi_i of the 100-star elastance workload (M = 25,600).",
             "# Written by tests/golden/make_fullsize.py: oracle.laplace.solve (dense Nystrom",
             "# matrix of eq. ModRep2, LU with partial pivoting, FP64), charges q = g['q'] of",
             "# synth.star_grid(seed=1000).  Rows: phi_i, i = 0..99.",
             f"# oracle wall time {dt:.1f} s"]
    lines += fingerprint(g, g["q"])
    lines += [f"{v:.17e}" for v in res["phi"]]
    with open(os.path.join(HERE, "stars100_M25600_elastance.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"elastance: {dt:.1f} s")


def mobility() -> None:
    g = synth.ellipse_suspension(seed=2000)
    FT = g["FT"]
    t0 = time.perf_counter()
    res = stokes.solve_gmres(g, FT, tol=1e-13, workers=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    lines = ["# Oracle rigid motions (v_x, v_y, omega) of the 400-ellipse mobility workload",
             "# (M = 51,200).  Written by tests/golden/make_fullsize.py: oracle.stokes.solve_gmres",
             "# (eq. ModRep2Stokes, FP64, block-Jacobi-preconditioned GMRES with FP64",
             "# refinement), loads FT = g['FT'] of synth.ellipse_suspension(seed=2000).",
             f"# true relative residual {res['rel_residual']:.3e} after {res['matvecs']} operator",
             f"# applications; oracle wall time {dt:.1f} s.  Rows: vx vy omega per body.",
             f"rel_residual {res['rel_residual']:.6e}"]
    lines += fingerprint(g, FT.reshape(-1))
    lines += [f"{a:.17e} {b:.17e} {c:.17e}" for a, b, c in res["UW"]]
    with open(os.path.join(HERE, "ellipses400_M51200_mobility.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"mobility: {dt:.1f} s, residual {res['rel_residual']:.3e}, {res['matvecs']} applications")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    if which in ("elastance", "all"):
        elastance()
    if which in ("mobility", "all"):
        mobility()
