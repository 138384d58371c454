"""The tensor-core products (digit planes on tcgen05, see include/find.h) in the
FIND passes, against the dense definition G = A^-1, G< = G Sigma< G^H.

* the mixed paths run their Schur and leaf products on the tensor cores by
  default: the profiler must show tensor-core launches, and the results must
  hold the mixed bar on a 64x128 9-point mesh at five grid energies;
* the FP64 path runs them only when asked (tc_slices): with 10 planes it must
  stay within 1e-10 of the dense definition on the same mesh;
* FIND_FLAG_NO_TC removes every tensor-core launch and reproduces the
  CUDA-core results bitwise.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, problem

pytestmark = pytest.mark.gpu

MESH = W.Mesh(64, 128, 9, 1.0, 0.2, -1.0, 1.0, 1109)
EIDX = [0, 100, 300, 400, 511]


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1104_0623_gb300 import build
    build.build()
    import paper_1104_0623_gb300 as F
    return F


@pytest.fixture(scope="module")
def ref():
    P = problem.MeshProblem.from_mesh(MESH)
    out = []
    for E in W.c5_energies()[EIDX]:
        A, Sl = P.assemble(E, 1.0, 0.0)
        rG, rGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, MESH.nx, MESH.ny, MESH.stencil)
        out.append((rG, rGl))
    return out


def run(F, **kw):
    import torch
    f = F.Find.from_mesh(MESH, leaf=8, max_batch=len(EIDX), **kw)
    f.profile(True)
    Es = torch.tensor(W.c5_energies()[EIDX], dtype=torch.complex128, device="cuda")
    G, Gl, J = (x.cpu().numpy() for x in f.solve_lesser(Es))
    prof = {p["name"]: p for p in f.profile_read()}
    f.close()
    return G, Gl, J, prof


def rel(x, r):
    return np.abs(x - r).max() / np.abs(r).max()


@pytest.mark.parametrize("precision", ["mixed", "mixed_ff"])
def test_mixed_paths_use_tensor_cores(F, ref, precision):
    G, Gl, _, prof = run(F, precision=precision)
    assert prof["tcgemm"]["launches"] > 0 and prof["tcsplit"]["launches"] > 0
    # the tensor cores take the large products: 36 % of this small mesh's
    # product flops (the rest are leaf and low-level products below the
    # 128 x 128 tiles); a routing mistake that sent them all to the CUDA
    # cores would leave 0
    assert prof["tcgemm"]["flops"] > 0.25 * sum(p["flops"] for k, p in prof.items()
                                                if "gemm" in k)
    for k, (rG, rGl) in enumerate(ref):
        assert rel(G[k], rG) <= 1e-7 and rel(Gl[k], rGl) <= 1e-7, (k, rel(G[k], rG), rel(Gl[k], rGl))


def test_fp64_path_on_tensor_cores_when_asked(F, ref):
    G, Gl, _, prof = run(F, precision="fp64")
    assert prof["tcgemm"]["launches"] == 0  # FP64 products stay on the CUDA cores by default
    G10, Gl10, _, prof10 = run(F, precision="fp64", tc_slices=10)
    assert prof10["tcgemm"]["launches"] > 0
    for k, (rG, rGl) in enumerate(ref):
        assert rel(G10[k], rG) <= 1e-10 and rel(Gl10[k], rGl) <= 1e-10, (k, rel(G10[k], rG))


def test_no_tc_flag_is_the_cuda_core_path(F):
    G, Gl, J, prof = run(F, precision="mixed_ff", tensor_cores=False)
    assert prof["tcgemm"]["launches"] == 0 and prof["tcsplit"]["launches"] == 0
    G2, Gl2, J2, _ = run(F, precision="mixed_ff", tensor_cores=False, tc_slices_mixed=11)
    assert np.array_equal(G, G2) and np.array_equal(Gl, Gl2) and np.array_equal(J, J2)
