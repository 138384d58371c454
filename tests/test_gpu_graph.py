"""FIND_FLAG_GRAPH: passes captured into CUDA graphs and replayed give the
same results, bitwise, as the same passes launched one by one: closed-form
and explicit lead Sigma, diag and lesser solves, several passes per call
(each pass offset its own graph), concurrent energy groups (forked streams
inside the graph), host buffers, new energies on a replayed graph, and the
singular-pivot report."""

import time

import numpy as np
import pytest

import workloads as W
from oracle import problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1104_0623_gb300 import build
    build.build()
    import paper_1104_0623_gb300 as F
    return F


def tcplx(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.complex128), device="cuda")


def run(F, mesh, Es, graph, calls, **kw):
    """Results of a list of solve calls on one handle."""
    f = F.Find.from_mesh(mesh, graph=graph, **kw)
    out = []
    for c in calls:
        out.append([None if x is None else (x.cpu().numpy() if hasattr(x, "cpu") else np.array(x))
                    for x in c(f)])
    f.close()
    return out


def same(a, b):
    for ra, rb in zip(a, b):
        for x, y in zip(ra, rb):
            assert (x is None) == (y is None)
            if x is not None:
                assert np.array_equal(x, y)


def test_graph_replay_is_bitwise_equal_to_eager(F):
    mesh = W.Mesh(24, 40, 9, 1.0, 0.2, -1.0, 1.0, 91)
    E1 = W.energy_grid(0.3, 7.7, 6)
    E2 = W.energy_grid(0.5, 7.1, 6)
    P = problem.MeshProblem.from_mesh(mesh)
    sig = np.stack([P.lead_sigmas(E)[0] for E in E1])
    calls = [
        lambda f: f.solve_lesser(tcplx(E1)),
        lambda f: f.solve_lesser(tcplx(E2)),                     # replay with new energies
        lambda f: f.solve_lesser(tcplx(E1)),
        lambda f: (f.solve_diag(tcplx(E2)),),
        lambda f: f.solve_lesser(tcplx(E1), 1.0, 0.3, sigmaL=tcplx(sig), sigmaR=tcplx(sig)),
        lambda f: f.solve_lesser(tcplx(E1), 1.0, 1.0,
                                 sigma_lesser_diag=tcplx(np.full(mesh.n, 2e-6j)), bonds=False),
        lambda f: f.solve_lesser(np.ascontiguousarray(E2)),      # host buffers
    ]
    for kw in ({"leaf": 5, "max_batch": 6, "precision": "fp64"},
               {"leaf": 5, "max_batch": 6, "precision": "mixed_ff", "energy_group": 2},
               {"leaf": 5, "max_batch": 4, "precision": "mixed"}):  # 6 energies = 2 passes
        eager = run(F, mesh, E1, False, calls, **kw)
        graph = run(F, mesh, E1, True, calls, **kw)
        same(eager, graph)


def test_graph_reports_the_singular_energy(F):
    mesh = W.Mesh(1, 3, 5, 1.0, 0.0, 0.0, 0.0, 1)
    E = np.array([0.5 + 0.0j, 0.7 + 0.0j])
    sR = (E - 4.0).reshape(2, 1, 1).copy()
    sR[0] = 0.1  # energy 0 is regular, energy 1 is singular
    f = F.Find.from_mesh(mesh, leaf=1, graph=True)
    for _ in range(2):  # captured, then replayed
        with pytest.raises(F.FindError) as ei:
            f.solve_diag(tcplx(E), sigmaR=tcplx(sR))
        assert ei.value.code == 3 and "energy index 1" in str(ei.value)
    f.close()


def test_graph_replay_time(F):
    # not a bar, a record: launch overhead on a small mesh, eager vs replayed
    import torch
    mesh = W.Mesh(48, 96, 9, 1.0, 0.2, -1.0, 1.0, 92)
    E = tcplx(W.energy_grid(0.3, 7.7, 8))
    res = {}
    for graph in (False, True):
        f = F.Find.from_mesh(mesh, leaf=8, max_batch=8, precision="mixed_ff", graph=graph)
        for _ in range(3):
            f.solve_lesser(E)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(20):
            f.solve_lesser(E)
        torch.cuda.synchronize()
        res[graph] = (time.perf_counter() - t) / 20
        f.close()
    print(f"48x96, 8 energies: eager {1e3 * res[False]:.2f} ms, graph {1e3 * res[True]:.2f} ms per call")
