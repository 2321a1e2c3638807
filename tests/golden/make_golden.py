"""Write the stored expected values of tests/golden/ by calling only oracle/.

The paper prints no worked-example values for the HEX8 weak-form path (its
results are figures or whole-pipeline scalars on geometry that is not
available), so the fixtures here are regression values of the oracle itself,
taken after the oracle passed its pins (tests/test_oracle_*.py).  Run:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import solve as osolve  # noqa: E402
from paper_2212_00964_gb300 import inputs  # noqa: E402


def c0_samples():
    w = inputs.c0()
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(w.kind, w.E, w.nu)
    f = oracle.traction(m, *w.traction)
    u = osolve.linear_solve(m, mat, w.mask, w.u_bar, f)
    nodes = [728, 720, 364, 80]  # far corner, far edge, centre, near face
    return {"compliance": float(f @ u), "nodes": nodes, "u": u.reshape(-1, 3)[nodes]}


def nh_samples():
    w = inputs.c1(n=4, n_steps=10)
    m = oracle.mesh(w.nx, w.ny, w.nz)
    u = osolve.newton_solve(m, oracle.Material(w.kind, w.E, w.nu), w.mask, w.u_bar, n_steps=w.n_steps)
    R = oracle.residual(m, oracle.Material(w.kind, w.E, w.nu), u)
    face = inputs.face_nodes(w.nx, w.ny, w.nz, "x1")
    return {"reaction_x": float(R[3 * face].sum()), "u_centre": u.reshape(-1, 3)[62]}


def main():
    a = c0_samples()
    with open(os.path.join(HERE, "c0_le_8cube.txt"), "w") as fh:
        fh.write("# c0: LE 8^3, E=70e3, nu=0.3, x=0 clamped, traction (0,0,-100) on x=1\n")
        fh.write("# oracle linear solve (written by tests/golden/make_golden.py)\n")
        fh.write(f"compliance {a['compliance']:.17e}\n")
        for n, v in zip(a["nodes"], a["u"]):
            fh.write(f"u {n} {v[0]:.17e} {v[1]:.17e} {v[2]:.17e}\n")
    b = nh_samples()
    with open(os.path.join(HERE, "nh_4cube_10steps.txt"), "w") as fh:
        fh.write("# Neo-Hookean 4^3 (c1 recipe), 10 load steps: oracle Newton (make_golden.py)\n")
        fh.write(f"reaction_x {b['reaction_x']:.17e}\n")
        v = b["u_centre"]
        fh.write(f"u 62 {v[0]:.17e} {v[1]:.17e} {v[2]:.17e}\n")


if __name__ == "__main__":
    main()
