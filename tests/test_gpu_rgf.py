"""The recursive Green's function baseline (find_rgf_solve_lesser) against the
dense definition (G = A^-1, G< = G Sigma< G^H), and against FIND.

RGF is the O(Nx^3 Ny) comparison method of the paper (Sec. 1, Sec. 5); the
library runs it on the GPU so that the FIND/RGF crossover can be measured on
the same device with the same kernels.
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


@pytest.mark.parametrize("mesh,fl,fr", [(W.c1(), 1.0, 0.0),
                                       (W.Mesh(24, 40, 9, 1.0, 0.2, -1.0, 1.0, 1109), 1.0, 0.3),
                                       (W.Mesh(7, 5, 5, 1.0, 0.0, -0.5, 0.5, 77), 0.2, 1.0)],
                         ids=["16x16-5pt", "24x40-9pt", "7x5-5pt"])
def test_rgf_against_dense(F, mesh, fl, fr):
    import torch
    Es = W.c5_energies()[[0, 73, 219, 365, 511]] if mesh.stencil == 9 else W.c2_energies()[[0, 21, 63]]
    f = F.Find.from_mesh(mesh, leaf=8, max_batch=len(Es))
    G, Gl = (x.cpu().numpy() for x in f.solve_rgf(torch.tensor(Es, dtype=torch.complex128, device="cuda"),
                                                   fl, fr))
    hG, hGl = f.solve_rgf(np.ascontiguousarray(Es), fl, fr)  # host buffers
    f.close()
    assert np.array_equal(hG, G) and np.array_equal(hGl, Gl)
    P = problem.MeshProblem.from_mesh(mesh)
    for k, E in enumerate(Es):
        A, Sl = P.assemble(E, fl, fr)
        rG, rGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
        assert rel(G[k], rG) <= 1e-10 and rel(Gl[k], rGl) <= 1e-10, (k, rel(G[k], rG), rel(Gl[k], rGl))


def test_rgf_equals_find_fp64_on_a_wider_mesh(F):
    import torch
    mesh = W.Mesh(64, 128, 5, 1.0, 0.0, -0.5, 0.5, 1107)
    Es = torch.tensor(W.c3_energies()[::8], dtype=torch.complex128, device="cuda")
    f = F.Find.from_mesh(mesh, leaf=8, max_batch=len(Es))
    rG, rGl = (x.cpu().numpy() for x in f.solve_rgf(Es))
    G, Gl, _ = f.solve_lesser(Es, bonds=False)
    G, Gl = G.cpu().numpy(), Gl.cpu().numpy()
    f.close()
    for k in range(len(Es)):
        assert rel(rG[k], G[k]) <= 1e-10 and rel(rGl[k], Gl[k]) <= 1e-10, (k, rel(rG[k], G[k]))
