"""Pins of the symmetric elimination of O-find (oracle/find.py,
eliminate_symmetric; Sec. 4.2): M(S,S) = L D L^T with Bunch-Kaufman
pivoting, U = M(B,B) - W^T D^{-1} W with W = L^{-1} M(S,B).

* on meshes with closed-form leads (A = A^T) it equals the dense definition
  and the LU-based elimination, for diag G, diag G< and bond currents;
* one elimination equals the LU form on random complex symmetric blocks,
  including a block whose diagonal is zero (no pivot-free LDL^T exists);
* U stays complex symmetric (Property 1);
* a non-symmetric A is refused;
* using conjugate transposes (an LDL^H, right only for Hermitian A) instead
  of plain transposes is caught.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, find, problem


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("mesh,E,leaf", [
    (W.c1(), 1.0 + 1e-6j, 4),
    (W.Mesh(12, 9, 9, 1.0, 0.2, -1.0, 1.0, 12), 3.1 + 1e-6j, 4),
    (W.Mesh(7, 19, 9, 1.0, 0.2, -1.0, 1.0, 13), 6.7 + 1e-6j, 3),
])
def test_symmetric_find_equals_dense_and_lu_find(mesh, E, leaf):
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()   # symmetric to rounding
    dG, dGl, dJ, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    sG, sGl, (sJ, _), _ = find.find_outputs(P, E, leaf=leaf, symmetric=True)
    lG, lGl, (lJ, _), _ = find.find_outputs(P, E, leaf=leaf)
    for got in ((sG, dG), (sGl, dGl), (sJ, dJ.real)):
        assert rel(*got) <= 1e-11
    assert rel(sG, lG) <= 1e-12 and rel(sGl, lGl) <= 1e-12


def _sym_block(rng, n, zero_diag_s=0):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    M = X + X.T
    if zero_diag_s:
        M[np.arange(zero_diag_s), np.arange(zero_diag_s)] = 0.0
    S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return M, S - S.conj().T


@pytest.mark.parametrize("n,s,zero_diag", [(9, 5, 0), (14, 8, 0), (12, 6, 6), (7, 4, 4)])
def test_one_elimination_equals_the_lu_form(n, s, zero_diag):
    rng = np.random.default_rng(100 + n + zero_diag)
    M, Sg = _sym_block(rng, n, zero_diag)
    U1, R1 = find.eliminate(M, Sg, s)
    U2, R2 = find.eliminate_symmetric(M, Sg, s)
    assert rel(U2, U1) <= 1e-12 and rel(R2, R1) <= 1e-12
    assert np.abs(U2 - U2.T).max() <= 1e-12 * np.abs(U2).max()


def test_nonsymmetric_A_is_refused():
    from test_oracle_find import general_system
    A, S = general_system(6, 9, 5, 21)
    with pytest.raises(ValueError):
        find.FindOracle(A, S, 6, 9, problem.find_pattern(6, 9, 5), 3, symmetric=True)


@pytest.mark.filterwarnings(r"ignore:scipy\.linalg\.ldl")
def test_hermitian_transpose_mistake_is_caught(monkeypatch):
    from scipy.linalg import ldl, solve_triangular

    def ldlh(M, Sg, s):
        # LDL^H with conjugate transposes: right for Hermitian blocks only
        MSS, MSB, MBB = M[:s, :s], M[:s, s:], M[s:, s:]
        lu, d, perm = ldl(MSS, lower=True, hermitian=True)
        W = solve_triangular(lu[perm], MSB[perm], lower=True, unit_diagonal=True)
        DW = np.linalg.solve(d, W)
        U = MBB - W.conj().T @ DW
        Lt = np.empty_like(DW)
        Lt[perm] = solve_triangular(lu[perm].conj().T, DW, lower=False, unit_diagonal=True)
        L = Lt.conj().T
        LH = L.conj().T
        R = Sg[s:, s:] - L @ Sg[:s, s:] - Sg[s:, :s] @ LH + L @ Sg[:s, :s] @ LH
        return U, R

    mesh = W.Mesh(12, 9, 9, 1.0, 0.2, -1.0, 1.0, 12)
    E = 3.1 + 1e-6j
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E)
    dG, dGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    monkeypatch.setattr(find, "eliminate_symmetric", ldlh)
    fG, fGl, _, _ = find.find_outputs(P, E, leaf=4, bonds=False, symmetric=True)
    assert max(rel(fG, dG), rel(fGl, dGl)) > 1e-6
