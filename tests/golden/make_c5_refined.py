"""Write c5_refined_samples.txt: diag G and diag G< of the 256x1024 9-point
mesh (t = 1, t' = 0.2, V ~ U[-1, 1], seed 1109) at 8 evenly spaced points of
its energy grid linspace(0.1, 7.9, 512) + 1e-6i, on sampled nodes, from the
refined definition of G = A^{-1} and G< = G Sigma< G^dagger (Sec. 1;
oracle/refined.py), with f_L = 1, f_R = 0.

Nodes per energy: the nodes where |diag G| and |diag G<| of O-find peak, and
30 nodes evenly spaced over the mesh.  Each energy also records, from O-find
(the FIND oracle, Sec. 2-3), max_i |diag G_i| and max_i |diag G<_i| over the
whole mesh (the normalisers of the normwise error) and O-find's own error on
the sampled nodes against the refined values.

Calls only oracle/ and workloads.py.  Run from the repository root:
    python tests/golden/make_c5_refined.py
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W                          # noqa: E402
from oracle import find as ofind, problem, refined   # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c5_refined_samples.txt")
ENERGY_INDEX = np.linspace(0, 511, 8).astype(int)


def main():
    mesh = W.c5()
    P = problem.MeshProblem.from_mesh(mesh)
    Es = W.c5_energies()
    lines = [
        "# diag G and diag G< of the 256x1024 9-point mesh (t=1, t'=0.2, V~U[-1,1] seed 1109),",
        "# f_L=1, f_R=0, closed-form leads; G = A^{-1} and G< = G Sigma< G^dagger (Sec. 1)",
        "# evaluated on sampled nodes by banded LU + iterative refinement with an",
        "# extended-precision residual (oracle/refined.py).  Written by",
        "# tests/golden/make_c5_refined.py.",
        "# norm <energy index> <Re E> <Im E> <max|diagG|> <max|diagG<|> <O-find err G> <O-find err G<> <last correction>",
        "# node <energy index> <node> <Re G> <Im G> <Re G<> <Im G<>",
    ]
    for ei in ENERGY_INDEX:
        E = Es[ei]
        t = time.time()
        fG, fGl, _, _ = ofind.find_outputs(P, E, leaf=8, bonds=False)
        spread = np.linspace(0, mesh.n - 1, 30).astype(int)
        nodes = np.unique(np.concatenate([[np.abs(fG).argmax(), np.abs(fGl).argmax()], spread]))
        G, Gl, hist = refined.sampled_outputs(P, E, nodes)
        G = G.astype(np.complex128)
        Gl = Gl.astype(np.complex128)
        mG, mGl = np.abs(fG).max(), np.abs(fGl).max()
        eG = np.abs(fG[nodes] - G).max() / mG
        eGl = np.abs(fGl[nodes] - Gl).max() / mGl
        lines.append(f"norm {ei} {E.real:.17e} {E.imag:.17e} {mG:.17e} {mGl:.17e} "
                     f"{eG:.3e} {eGl:.3e} {hist[:, -1].max():.3e}")
        for k, nd in enumerate(nodes):
            lines.append(f"node {ei} {nd} {G[k].real:.17e} {G[k].imag:.17e} "
                         f"{Gl[k].real:.17e} {Gl[k].imag:.17e}")
        print(f"E[{ei}] = {E:.4f}: O-find err G {eG:.2e}, G< {eGl:.2e} ({time.time() - t:.0f} s)",
              flush=True)
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
