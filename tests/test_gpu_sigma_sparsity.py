"""Sigma< sparsity (Sec. 4.3): the upward merges of clusters with no contact
node skip their Sigma update (Eq. 7 with Sigma_M = 0 gives R = 0).

The leaves with no contact node likewise run their G< products over the
nonzero block R_Cbar of Sigma_K only.  A node-diagonal Sigma< that is
identically zero gives the same problem but makes the library run every
Sigma update in full, so on the FP64 path the two calls must agree bitwise
(the skipped terms are exact zeros); on the mixed path the shorter leaf
products may take the CUDA-core GEMM instead of the tensor cores, so there
both are held to the path's tolerance.  Both are checked against the dense
definition too.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, problem

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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed_ff", 1e-7)])
@pytest.mark.parametrize("mesh", [W.Mesh(24, 40, 9, 1.0, 0.2, -1.0, 1.0, 1109),
                                  W.Mesh(16, 64, 5, 1.0, 0.0, -0.5, 0.5, 1107)],
                         ids=["24x40-9pt", "16x64-5pt"])
def test_skipped_sigma_updates_match_the_full_pass(F, mesh, precision, tol):
    import torch
    Es = W.c5_energies()[[5, 130, 260, 400]]
    E = torch.tensor(Es, dtype=torch.complex128, device="cuda")
    zeros = torch.zeros((len(Es), mesh.n), dtype=torch.complex128, device="cuda")
    f = F.Find.from_mesh(mesh, leaf=4, max_batch=len(Es), precision=precision)
    sparse = [x.cpu().numpy() for x in f.solve_lesser(E, 1.0, 0.3)]
    full = [x.cpu().numpy() for x in f.solve_lesser(E, 1.0, 0.3, sigma_lesser_diag=zeros)]
    again = [x.cpu().numpy() for x in f.solve_lesser(E, 1.0, 0.3)]  # dense tables serve it too
    f.close()
    for a, b, c in zip(sparse, full, again):
        if precision == "fp64":
            np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(a, c)
        else:
            assert rel(a, b) <= tol and rel(a, c) <= tol
    P = problem.MeshProblem.from_mesh(mesh)
    for k, En in enumerate(Es):
        A, Sl = P.assemble(En, 1.0, 0.3)
        rG, rGl, rJ, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
        assert rel(sparse[0][k], rG) <= tol and rel(sparse[1][k], rGl) <= tol, (k, rel(sparse[1][k], rGl))
