"""Writes tests/golden/*.txt from the oracle alone (O-dense).

The paper prints no worked numerical example, so the stored values here are
the dense definition G = A^{-1}, G< = G Sigma< G^H (Sec. 1) evaluated by
``oracle/`` on the 16x16 workload (5-point, t = 1, V ~ U[-0.5, 0.5] seed 1105,
E = 1 + 1e-6 i, f_L = 1, f_R = 0), plus the clean-wire open-mode count.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import dense, problem  # noqa: E402


def main():
    mesh = W.c1()
    E = W.c1_energies()[0]
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E, 1.0, 0.0)
    dG, dGl, J, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    out = os.path.join(HERE, "c1_16x16_dense.txt")
    with open(out, "w") as f:
        f.write("# O-dense, 16x16 5-point, seed 1105, E=1+1e-6i, fL=1, fR=0\n")
        f.write("# node  Re(G_nn)  Im(G_nn)  Im(G<_nn)\n")
        for k in range(mesh.n):
            f.write(f"{k} {dG[k].real:.17e} {dG[k].imag:.17e} {dGl[k].imag:.17e}\n")
    out = os.path.join(HERE, "c1_16x16_bond_current.txt")
    with open(out, "w") as f:
        f.write("# O-dense bond currents J_{i->j}, bond order of oracle.dense.bond_list\n")
        for k in range(len(J)):
            f.write(f"{J[k].real:.17e}\n")


if __name__ == "__main__":
    main()
