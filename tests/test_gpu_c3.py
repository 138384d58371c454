"""Ragged batch: nine 5-point meshes Nx in {64, 96, 128} x Ny in {128, 256,
512} (V ~ U[-0.5, 0.5], seeds 1107..1115), 32 energies each in
linspace(0.2, 3.8) + 1e-6i, solved together on the mixed float-float path
with knobs chosen by the autotuner, against

* the FP64 path on every energy (bar 1e-5 normwise per energy);
* on two energies per mesh, the refined definition of G and G< on sampled
  nodes (oracle/refined.py) for the FP64 path, and the FP64 FIND oracle
  (O-find) on every node for the mixed path (bar 1e-5).  FP64 bar: 1e-10
  against the refined values (the FP64 path eliminates by LDL^T; the
  LU-based O-find itself reaches ~1e-10 at 96x512 at some energies);
* the same meshes solved one at a time (each result is the same alone and in
  the ragged batch: bitwise, since an energy's arithmetic does not depend on
  what shares the device).
"""

import numpy as np
import pytest

import workloads as W
from oracle import find as ofind, problem, refined

pytestmark = pytest.mark.gpu


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


def test_c3_ragged_batch_autotuned(F, tmp_path):
    import torch

    from paper_1104_0623_gb300 import serve, tune
    meshes, Es = W.c3(), W.c3_energies()
    tuner = tune.Tuner(cache_path=str(tmp_path / "tune.json"), repeats=1, sample=8, budget_s=4.0)
    backend = serve.GpuBackend(precision="mixed_ff", chunk=16, tuner=tuner)
    mixed = serve.solve_ragged([(m, Es) for m in meshes], backend, slots=4, chunk=16)
    assert len(tuner.cache) == len(meshes)
    for key, entry in tuner.log:
        print(f"tuned {key.split(':')[0]}: {entry['params']} "
              f"{1e3 * entry['seconds_per_energy']:.2f} ms/E (defaults "
              f"{1e3 * entry['default_seconds_per_energy']:.2f}), {entry['candidates']} candidates")
    for k, mesh in enumerate(meshes):
        params = tuner.tune(mesh, Es[:16], "mixed_ff", 16)
        f = F.Find.from_mesh(mesh, max_batch=32, precision="fp64")
        G64, Gl64, _ = f.solve_lesser(np.ascontiguousarray(Es), bonds=False)
        f.close()
        for e in range(len(Es)):
            assert rel(mixed[k][0][e], G64[e]) <= 1e-5, (mesh.nx, mesh.ny, e)
            assert rel(mixed[k][1][e], Gl64[e]) <= 1e-5, (mesh.nx, mesh.ny, e)
        # alone, with the tuned knobs, in the same 16-energy chunks
        g = F.Find.from_mesh(mesh, max_batch=16, precision="mixed_ff", **params)
        for lo in (0, 16):
            aG, aGl, _ = g.solve_lesser(np.ascontiguousarray(Es[lo:lo + 16]), bonds=False)
            assert np.array_equal(aG, mixed[k][0][lo:lo + 16])
            assert np.array_equal(aGl, mixed[k][1][lo:lo + 16])
        g.close()
        P = problem.MeshProblem.from_mesh(mesh)
        for e in (5, 26):
            oG, oGl, _, _ = ofind.find_outputs(P, Es[e], leaf=8, bonds=False)
            assert rel(mixed[k][0][e], oG) <= 1e-5 and rel(mixed[k][1][e], oGl) <= 1e-5
            nodes = np.unique(np.concatenate([[np.abs(oG).argmax(), np.abs(oGl).argmax()],
                                              np.linspace(0, mesh.n - 1, 18).astype(int)]))
            xG, xGl, _ = refined.sampled_outputs(P, Es[e], nodes)
            xG, xGl = xG.astype(np.complex128), xGl.astype(np.complex128)
            mG, mGl = np.abs(oG).max(), np.abs(oGl).max()

            def err(g, gl):
                return max(np.abs(g[nodes] - xG).max() / mG, np.abs(gl[nodes] - xGl).max() / mGl)
            assert err(G64[e], Gl64[e]) <= 1e-10, (mesh.nx, mesh.ny, e, err(G64[e], Gl64[e]))
    torch.cuda.synchronize()
