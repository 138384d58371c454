"""The symmetric LDL^T elimination (Sec. 4.2; Bunch-Kaufman
diagonal pivoting, U = M(B,B) - W^T D^-1 W) against

* the dense definition (G = A^-1, G< = G Sigma< G^H, bond currents) and the
  symmetric FIND oracle (FindOracle(symmetric=True)) on a 5-point and a
  9-point mesh, 1e-10 normwise per energy;
* the LU elimination of the same path (ldl=False), 1e-10;
* the mixed paths with FIND_FLAG_LDL (ldl=True; float-float or FP64
  factorisation, float-float solves) on the 9-point mesh: dense definition
  and their default LU form, 1e-7;
* a mesh whose every diagonal entry is planted on the host at 0.05i (onsite
  V_n = Re E - onsite0), so that |a_kk| < alpha |a_rk| at the first step of
  every elimination and the factorisation must take 2x2 pivots: dense
  definition, 1e-10 (FP64) and 1e-7 (mixed paths);
* a call that passes Sigma_L and Sigma_R (not known to be symmetric) takes the
  LU elimination: bitwise equal to a handle built with ldl=False.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, find as ofind, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1104_0623_gb300 import build
    build.build()
    import paper_1104_0623_gb300 as F
    return F


def rel(x, r):
    return np.abs(x - r).max() / np.abs(r).max()


def gpu(F, mesh, Es, V=None, precision="fp64", **kw):
    import torch
    f = F.Find.from_mesh(mesh, V=V, leaf=8, max_batch=len(Es), precision=precision, **kw)
    out = [x.cpu().numpy() for x in f.solve_lesser(torch.tensor(Es, dtype=torch.complex128, device="cuda"))]
    f.close()
    return out


MESHES = [W.c1(), W.Mesh(24, 40, 9, 1.0, 0.2, -1.0, 1.0, 1109)]


def test_mixed_paths_ldl_against_dense(F):
    mesh = MESHES[1]
    Es = W.c5_energies()[[0, 73, 219, 365, 511]]
    P = problem.MeshProblem.from_mesh(mesh)
    for precision in ("mixed", "mixed_ff"):
        G, Gl, J = gpu(F, mesh, Es, precision=precision, ldl=True)
        Glu, Gllu, _ = gpu(F, mesh, Es, precision=precision)
        for k, E in enumerate(Es):
            A, Sl = P.assemble(E, 1.0, 0.0)
            rG, rGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
            assert rel(G[k], rG) <= 1e-7 and rel(Gl[k], rGl) <= 1e-7, (precision, k, rel(G[k], rG))
            assert rel(G[k], Glu[k]) <= 1e-7 and rel(Gl[k], Gllu[k]) <= 1e-7


@pytest.mark.parametrize("mesh", MESHES, ids=["16x16-5pt", "24x40-9pt"])
def test_ldl_against_dense_and_symmetric_oracle(F, mesh):
    Es = W.c5_energies()[[0, 73, 219, 365, 511]] if mesh.stencil == 9 else W.c2_energies()[[0, 21, 42, 63]]
    G, Gl, J = gpu(F, mesh, Es)
    Glu, Gllu, Jlu = gpu(F, mesh, Es, ldl=False)
    P = problem.MeshProblem.from_mesh(mesh)
    for k, E in enumerate(Es):
        A, Sl = P.assemble(E, 1.0, 0.0)
        rG, rGl, rJ, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
        assert rel(G[k], rG) <= 1e-10 and rel(Gl[k], rGl) <= 1e-10, (k, rel(G[k], rG), rel(Gl[k], rGl))
        assert rel(J[k], rJ.real) <= 1e-10, (k, rel(J[k], rJ.real))
        sG, sGl, _, _ = ofind.find_outputs(P, E, leaf=8, bonds=False, symmetric=True)
        assert rel(G[k], sG) <= 1e-10 and rel(Gl[k], sGl) <= 1e-10
        assert rel(G[k], Glu[k]) <= 1e-10 and rel(Gl[k], Gllu[k]) <= 1e-10


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("mixed_ff", 1e-7), ("mixed", 1e-7)])
def test_ldl_two_by_two_pivots_on_a_planted_diagonal(F, precision, bar):
    mesh = W.Mesh(16, 24, 5, 1.0, 0.0, 0.0, 0.0, 1105)
    E = 0.3 + 0.05j
    V = np.full(mesh.n, E.real - mesh.onsite0)  # every A_nn = 0.05i before the lead terms
    G, Gl, J = gpu(F, mesh, np.array([E]), V=V, precision=precision, ldl=True)
    P = problem.MeshProblem.from_mesh(mesh, V=V)
    A, Sl = P.assemble(E, 1.0, 0.0)
    inner = [i for i in range(mesh.n) if 0 < i // mesh.nx < mesh.ny - 1]
    assert np.allclose(A.diagonal()[inner], 0.05j)
    rG, rGl, rJ, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    assert rel(G[0], rG) <= bar and rel(Gl[0], rGl) <= bar, (rel(G[0], rG), rel(Gl[0], rGl))
    assert rel(J[0], rJ.real) <= bar


def test_given_sigma_takes_the_lu_elimination(F):
    import torch
    mesh = MESHES[1]
    Es = W.c5_energies()[[10, 300]]
    P = problem.MeshProblem.from_mesh(mesh)
    sig = np.stack([P.lead_sigmas(E)[0] for E in Es])  # the closed form, passed as data
    out = []
    for ldl in (True, False):
        f = F.Find.from_mesh(mesh, leaf=8, max_batch=2, precision="fp64", ldl=ldl)
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.complex128, device="cuda")
        out.append([x.cpu().numpy() for x in f.solve_lesser(t(Es), sigmaL=t(sig), sigmaR=t(sig))])
        f.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
