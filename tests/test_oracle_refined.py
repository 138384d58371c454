"""Pins of O-refined (oracle/refined.py): sampled entries of G = A^{-1} and
G< = G Sigma< G^dagger by banded LU with extended-precision refinement.

* equal to the dense inverse on random non-symmetric, non-Hermitian A and
  Sigma (a transposed solve or an unconjugated factor fails this);
* equal to O-dense on meshes with both leads, f_L, f_R and node-diagonal
  Sigma<;
* equal to the clean-wire closed forms on a long 9-point wire;
* on an ill-conditioned system, equal to an arbitrary-precision inverse
  (mpmath) well below the error of the unrefined double-precision solve;
* the committed 256x1024 samples (tests/golden/c5_refined_samples.txt) hold
  the closed-form property Re diag G< = 0 and Im diag G <= 0 <= Im diag G<.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import dense, problem, refined
from test_oracle_dense import clean_wire_diag
from test_oracle_find import general_system

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c5_refined_samples.txt")


def rel(a, b):
    return float(np.abs(np.asarray(a, np.complex128) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nx,ny,stencil,seed", [(6, 9, 5, 21), (7, 8, 9, 22), (10, 5, 9, 23)])
def test_refined_equals_dense_inverse_on_general_systems(nx, ny, stencil, seed):
    A, S = general_system(nx, ny, stencil, seed)
    assert np.abs(A - A.T).max() > 0.1
    G = np.linalg.inv(A.toarray())
    Gl = G @ S.toarray() @ G.conj().T
    nodes = np.arange(nx * ny)
    Y, hist = refined.BandedInverse(A).rows(nodes)
    assert rel(Y[nodes, nodes], np.diag(G)) <= 1e-13
    # a whole row, not only its diagonal entry
    assert rel(Y[:, 3], G[3]) <= 1e-13
    assert rel(refined.lesser_diagonal(Y, nodes, S), np.diag(Gl)) <= 1e-13
    assert hist[:, -1].max() <= 1e-17


@pytest.mark.parametrize("mesh,E,fL,fR,dl", [
    (W.c1(), 1.0 + 1e-6j, 1.0, 0.0, None),
    (W.Mesh(10, 13, 9, 1.0, 0.2, -1, 1, 4), 5.5 + 1e-6j, 0.7, 0.2, 0.05j),
])
def test_refined_equals_dense_on_meshes(mesh, E, fL, fR, dl):
    P = problem.MeshProblem.from_mesh(mesh)
    diag_lesser = None if dl is None else np.full(mesh.n, dl)
    A, Sl = P.assemble(E, fL, fR, diag_lesser=diag_lesser)
    dG, dGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    nodes = np.arange(0, mesh.n, 3)
    G, Gl, _ = refined.sampled_outputs(P, E, nodes, fL, fR, diag_lesser)
    assert rel(G, dG[nodes]) <= 1e-12
    assert rel(Gl, dGl[nodes]) <= 1e-12


@pytest.mark.parametrize("E", [2.1 + 1e-6j, 6.9 + 1e-6j])
def test_refined_clean_wire_closed_form(E):
    mesh = W.Mesh(12, 400, 9, 1.0, 0.2, 0.0, 0.0, 1)
    P = problem.MeshProblem.from_mesh(mesh)
    nodes = np.array([0, 5, 11, 12 * 57 + 3, 12 * 200 + 6, 12 * 399 + 11])
    G, Gl, _ = refined.sampled_outputs(P, E, nodes)
    rG, rGl = clean_wire_diag(mesh, E)
    assert rel(G, rG[nodes]) <= 1e-12
    assert rel(Gl, rGl[nodes]) <= 1e-12


def test_refinement_beats_the_plain_solve_on_an_ill_conditioned_system():
    # a hard dependency: this is the only pin of the refinement itself, so a
    # missing mpmath must fail the suite, not skip the pin
    import mpmath
    # a closed 5x6 box (no leads) at E = an eigenvalue of H + 1e-7 i: A is
    # close to singular (cond ~ 1e8), so a plain double solve keeps only
    # about 8 digits
    mesh = W.Mesh(5, 6, 9, 1.0, 0.2, -1.0, 1.0, 31)
    P = problem.MeshProblem.from_mesh(mesh)
    lam = np.linalg.eigvalsh(P.H.toarray())[11]
    E = lam + 1e-7j
    zero = np.zeros((mesh.nx, mesh.nx), np.complex128)
    A, _ = P.assemble(E, sigL=zero, sigR=zero)
    n = mesh.n
    mpmath.mp.dps = 40
    Am = mpmath.matrix(n, n)
    Ad = A.toarray()
    for i in range(n):
        for j in range(n):
            if Ad[i, j] != 0:
                Am[i, j] = mpmath.mpc(Ad[i, j].real, Ad[i, j].imag)
    Gm = Am ** -1
    exact = np.array([complex(Gm[i, i]) for i in range(n)])
    inv = refined.BandedInverse(A)
    nodes = np.arange(n)
    plain = np.array([inv._solve_t(np.eye(n, dtype=np.complex128)[:, [i]])[i, 0] for i in nodes])
    Y, _ = inv.rows(nodes, sweeps=4)
    assert rel(plain, exact) > 1e-12                      # the case is hard in double
    assert rel(Y[nodes, nodes], exact) <= 1e-3 * rel(plain, exact)


def read_golden():
    norms, rows = {}, []
    with open(GOLD) as fh:
        for line in fh:
            if line.startswith("norm"):
                p = line.split()
                norms[int(p[1])] = dict(E=complex(float(p[2]), float(p[3])), maxG=float(p[4]),
                                        maxGl=float(p[5]), ofind_G=float(p[6]), ofind_Gl=float(p[7]))
            elif line.startswith("node"):
                p = line.split()
                rows.append((int(p[1]), int(p[2]), complex(float(p[3]), float(p[4])),
                             complex(float(p[5]), float(p[6]))))
    return norms, rows


def test_c5_refined_samples_are_physical():
    norms, rows = read_golden()
    assert len(norms) == 8 and len(rows) >= 8 * 30
    Es = W.c5_energies()
    for ei, nm in norms.items():
        assert nm["E"] == Es[ei]
        # O-find (the FIND oracle in FP64) agrees with the refined
        # definition to its own rounding: between 1e-13 and 1e-9 on this
        # mesh, depending on the energy (the conditioning of A); a mistake in
        # either would show far above that
        assert nm["ofind_G"] <= 5e-9 and nm["ofind_Gl"] <= 5e-9
    for ei, node, G, Gl in rows:
        assert G.imag <= 0.0 <= Gl.imag
        assert abs(Gl.real) <= 1e-12 * norms[ei]["maxGl"]
