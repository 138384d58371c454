"""Accuracy of the two FP64 FIND oracles on the 256x1024 9-point mesh against
the refined definition of G and G< (c5_refined_samples.txt): the LU-based
elimination (O-find, whose errors the golden file records) and the symmetric
LDL^T elimination (FindOracle(symmetric=True), Sec. 4.2).  Prints one line per
sampled energy: max error over the sampled nodes / max over the mesh, for
diag G and diag G<.  About ten minutes per energy on one host (the LDL^T
factors are post-processed in Python); pass energy indices to run a subset.

Calls only oracle/ and workloads.py.  Run from the repository root:
    python tests/golden/symmetric_accuracy.py [energy index ...]
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W                       # noqa: E402
from oracle import find as ofind, problem   # noqa: E402
from test_oracle_refined import read_golden  # noqa: E402


def main(which):
    norms, rows = read_golden()
    P = problem.MeshProblem.from_mesh(W.c5())
    for ei in sorted(norms):
        if which and ei not in which:
            continue
        nm = norms[ei]
        G, Gl, _, _ = ofind.find_outputs(P, nm["E"], leaf=8, bonds=False, symmetric=True)
        sel = [(n, g, gl) for e, n, g, gl in rows if e == ei]
        nodes = np.array([x[0] for x in sel])
        eG = np.abs(G[nodes] - np.array([x[1] for x in sel])).max() / nm["maxG"]
        eGl = np.abs(Gl[nodes] - np.array([x[2] for x in sel])).max() / nm["maxGl"]
        print(f"E = {nm['E'].real:.3f}: LU-based {nm['ofind_G']:.1e} / {nm['ofind_Gl']:.1e}, "
              f"LDL^T {eG:.1e} / {eGl:.1e}", flush=True)


if __name__ == "__main__":
    main({int(a) for a in sys.argv[1:]})
