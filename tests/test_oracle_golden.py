"""The oracle still reproduces its stored 16x16 values (tests/golden)."""
import os

import numpy as np

import workloads as W
from oracle import dense, find, problem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_c1():
    d = np.loadtxt(os.path.join(GOLD, "c1_16x16_dense.txt"))
    j = np.loadtxt(os.path.join(GOLD, "c1_16x16_bond_current.txt"))
    return d[:, 1] + 1j * d[:, 2], 1j * d[:, 3], j


def test_golden_c1_reproduced_by_find():
    gG, gGl, gJ = load_c1()
    mesh = W.c1()
    P = problem.MeshProblem.from_mesh(mesh)
    fG, fGl, (fJ, _), _ = find.find_outputs(P, W.c1_energies()[0], leaf=4)
    assert np.abs(fG - gG).max() <= 1e-11 * np.abs(gG).max()
    assert np.abs(fGl - gGl).max() <= 1e-11 * np.abs(gGl).max()
    assert np.abs(fJ.real - gJ).max() <= 1e-11 * np.abs(gJ).max()
