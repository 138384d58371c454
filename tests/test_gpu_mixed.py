"""Mixed paths.  FIND_MIXED: below the top FP64 levels the Schur update U,
the solves for L, the Sigma update and the leaf G< products run in
float-float (about 48 significant bits); LU and leaf inversion in FP64.
FIND_MIXED_FF: the LU and the leaf inversion in float-float as well.  The
complex64 Sigma update (opt-in) is checked against its own looser bar.
Bar: 1e-5 normwise per energy against the FP64 oracle for diag G and diag G<
(diag G, fed only by float-float and FP64 steps, is held to 1e-9)."""

import numpy as np
import pytest

import workloads as W
from oracle import dense, find as ofind, problem

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1104_0623_gb300 import build
    build.build()
    import paper_1104_0623_gb300 as F
    return F


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def solve(F, mesh, Es, precision, leaf=8, top=2, max_batch=0, c64=0):
    import torch
    f = F.Find.from_mesh(mesh, leaf=leaf, precision=precision, fp64_top_levels=top,
                         max_batch=max_batch, sigma_c64_depth=c64)
    out = [x.cpu().numpy() for x in f.solve_lesser(torch.tensor(Es, dtype=torch.complex128,
                                                                 device="cuda"))]
    f.close()
    return out


@pytest.mark.parametrize("precision", ["mixed", "mixed_ff"])
def test_c2_mixed_all_energies_within_1e5(F, precision):
    mesh, Es = W.c2(), W.c2_energies()
    G, Gl, J = solve(F, mesh, Es, precision, leaf=5)
    P = problem.MeshProblem.from_mesh(mesh)
    worst = 0.0
    for k in range(0, 64, 4):
        A, Sl = P.assemble(Es[k])
        rG, rGl, rJ, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
        worst = max(worst, rel(Gl[k], rGl), rel(J[k], rJ.real))
        assert rel(G[k], rG) <= 1e-9
    assert worst <= TOL_MIXED, worst
    assert worst <= 1e-7, worst  # float-float paths measured near 1e-9


# Float-float paths: the stated bar is 1e-5; they were measured near 1e-9 on
# this mesh (and on 256x1024), so 1e-7 guards against a regression.  With the
# opt-in complex64 Sigma update from depth 3 down, one energy reached 1e-5 on
# this mesh; it is held to 3e-5.
@pytest.mark.parametrize("precision,top,c64,tol", [("mixed", 2, 0, 1e-7), ("mixed", 0, 0, 1e-7),
                                                   ("mixed_ff", 2, 0, 1e-7), ("mixed", 2, 3, 3e-5)])
def test_mixed_9pt_mesh_against_oracle_find(F, precision, top, c64, tol):
    mesh = W.Mesh(64, 128, 9, 1.0, 0.2, -1.0, 1.0, 1109)
    Es = W.c5_energies()[[0, 100, 300, 400, 511]]
    G, Gl, J = solve(F, mesh, Es, precision, top=top, c64=c64)
    P = problem.MeshProblem.from_mesh(mesh)
    for k, E in enumerate(Es):
        rG, rGl, _, _ = ofind.find_outputs(P, E, leaf=8, bonds=False)
        assert rel(G[k], rG) <= 1e-9
        assert rel(Gl[k], rGl) <= min(tol, TOL_MIXED * 3), (E, rel(Gl[k], rGl))


@pytest.mark.parametrize("precision", ["mixed", "mixed_ff"])
def test_mixed_alone_and_in_batch_are_bitwise_equal(F, precision):
    mesh = W.Mesh(24, 40, 9, 1.0, 0.2, -1.0, 1.0, 81)
    Es = W.energy_grid(0.2, 7.8, 6)
    both = solve(F, mesh, Es, precision, leaf=5, max_batch=6)
    for k in (1, 5):
        alone = solve(F, mesh, Es[k:k + 1], precision, leaf=5, max_batch=1)
        for a, b in zip(alone, both):
            assert np.array_equal(a[0], b[k])
