"""Serving loop on the GPU: requests of different meshes run concurrently and
each result equals the same request solved alone."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_1104_0623_gb300 import build
    build.build()
    import paper_1104_0623_gb300 as F
    return F


@pytest.mark.parametrize("graph_max_nodes", [0, 1 << 30], ids=["eager", "graph-replay"])
def test_each_result_is_the_same_alone_and_in_the_mix(F, graph_max_nodes):
    # with graph_max_nodes, every chunk runs as a captured CUDA graph
    # (FIND_FLAG_GRAPH), replayed on the worker streams: the same bits as the
    # eager launches of a handle solving the request alone
    from paper_1104_0623_gb300.serve import GpuBackend, Request, Server, summarize
    meshes = [W.Mesh(24, 40, 5, seed=91), W.Mesh(32, 33, 5, seed=92), W.Mesh(17, 60, 5, seed=93)]
    reqs = [Request(k, 0.01 * k, meshes[k % 3], W.energy_grid(0.2, 3.8, 6 + 5 * k)) for k in range(6)]
    srv = Server(GpuBackend(precision="mixed", chunk=8, graph_max_nodes=graph_max_nodes), slots=3, chunk=8)
    res = srv.run(reqs)
    if graph_max_nodes:  # a second stream replays the graphs the first captured
        res = srv.run(reqs)
    assert srv.max_active >= 2
    for r, req in zip(res, reqs):
        f = F.Find.from_mesh(req.mesh, leaf=8, precision="mixed", max_batch=8)
        G, Gl, _ = f.solve_lesser(np.ascontiguousarray(req.energies), bonds=False)
        f.close()
        assert np.array_equal(r.diagG, G) and np.array_equal(r.diagGl, Gl)
    s = summarize(res)
    assert s["energy_points"] == sum(len(q.energies) for q in reqs)
    srv.close()
