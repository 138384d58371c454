"""find_solve_diag_static: the diag solve for callers that cannot allocate
device memory (a host program whose memory pool already holds the device, a
plug-in whose host owns all device allocation, a loop that must not allocate
while it runs).  Its device buffers live in the library's fixed 64 MiB array.

Called through the C ABI and compared with find_solve_diag, which allocates
its own workspace, on two calls in a row.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def test_static_scratch_matches_allocating_solve(F):
    import torch
    lib = F._abi.load()
    mesh = W.Mesh(28, 36, 9, 1.0, 0.2, -1.0, 1.0, 71)
    f = F.Find.from_mesh(mesh, leaf=6)
    stream = torch.cuda.current_stream().cuda_stream
    # 20 energies need two passes through the fixed array; then a second call
    for call, Es in enumerate((W.energy_grid(0.4, 7.6, 20), W.energy_grid(1.1, 6.3, 5))):
        E = torch.tensor(Es, dtype=torch.complex128, device="cuda")
        ref = f.solve_diag(E).cpu().numpy()
        out = torch.full((len(Es), mesh.n), float("nan"), dtype=torch.complex128, device="cuda")
        rc = lib.find_solve_diag_static(f.handle, E.data_ptr(), len(Es), None, None,
                                        out.data_ptr(), stream)
        assert rc == 0, lib.find_last_error(f.handle).decode()
        got = out.cpu().numpy()
        for k in range(len(Es)):
            assert rel(got[k], ref[k]) <= TOL, (call, k, rel(got[k], ref[k]))
    f.close()


def test_static_scratch_alternating_handles_host_buffers_and_mixed_path(F):
    """Two handles on different meshes called A, B, A on one stream (each call
    re-uploads its own tables into the shared array); host numpy energies and
    outputs over several passes (copied out pass by pass); a float-float handle
    against its own allocating solve."""
    import torch
    lib = F._abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    fa = F.Find.from_mesh(W.Mesh(28, 36, 9, 1.0, 0.2, -1.0, 1.0, 71), leaf=6)
    fb = F.Find.from_mesh(W.Mesh(20, 24, 5, 1.0, 0.0, -0.5, 0.5, 72), leaf=8)
    fm = F.Find.from_mesh(W.Mesh(24, 30, 5, 1.0, 0.0, -0.5, 0.5, 73), leaf=8, precision="mixed_ff")
    Es = W.energy_grid(0.3, 3.9, 23)  # several passes through the fixed array
    for f, tol in ((fa, TOL), (fb, TOL), (fa, TOL), (fm, 1e-7)):
        ref = f.solve_diag(np.ascontiguousarray(Es))
        out = np.full((len(Es), f.n), np.nan, dtype=np.complex128)
        E = np.ascontiguousarray(Es)
        rc = lib.find_solve_diag_static(f.handle, E.ctypes.data, len(Es), None, None,
                                        out.ctypes.data, stream)
        assert rc == 0, lib.find_last_error(f.handle).decode()
        for k in range(len(Es)):
            assert rel(out[k], ref[k]) <= tol, (f.nx, f.ny, k, rel(out[k], ref[k]))
    for f in (fa, fb, fm):
        f.close()


def test_static_scratch_rejects_a_mesh_that_does_not_fit(F):
    import torch
    lib = F._abi.load()
    f = F.Find(128, 512, 5, 1.0, 0.0, leaf=8)
    E = torch.tensor(W.energy_grid(1.0, 2.0, 2), dtype=torch.complex128, device="cuda")
    out = torch.empty((2, f.n), dtype=torch.complex128, device="cuda")
    rc = lib.find_solve_diag_static(f.handle, E.data_ptr(), 2, None, None, out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == F._abi.FIND_EINVAL
    msg = lib.find_last_error(f.handle).decode()
    assert "MiB" in msg and "64" in msg
    f.close()
