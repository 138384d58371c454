"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Error metric (per energy, normwise): max_i |x_i - ref_i| / max_i |ref_i| for
diag G, diag G< and the bond currents J.  The FP64 path must hold 1e-10.
Inputs are seeded synthetic meshes (workloads.py).
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import dense, find as ofind, problem

pytestmark = pytest.mark.gpu

TOL = 1e-10
GOLD = os.path.join(os.path.dirname(__file__), "golden")


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


def tcplx(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.complex128), device="cuda")


def gpu_lesser(F, mesh, Es, leaf=8, fL=1.0, fR=0.0, sigL=None, sigR=None, dles=None,
               bonds=True, max_batch=0, V=None):
    f = F.Find.from_mesh(mesh, V=V, leaf=leaf, max_batch=max_batch)
    out = f.solve_lesser(tcplx(Es), fL, fR,
                         None if sigL is None else tcplx(sigL), None if sigR is None else tcplx(sigR),
                         None if dles is None else tcplx(dles), bonds=bonds)
    res = [None if x is None else x.cpu().numpy() for x in out]
    f.close()
    return res


def dense_ref(mesh, E, fL=1.0, fR=0.0, sigL=None, sigR=None, dles=None, V=None):
    P = problem.MeshProblem.from_mesh(mesh, V=V)
    A, Sl = P.assemble(E, fL, fR, sigL, sigR, dles)
    dG, dGl, J, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    return dG, dGl, J.real


def check(got, ref, tol=TOL, bonds=True):
    gG, gGl, gJ = got
    rG, rGl, rJ = ref
    assert rel(gG, rG) <= tol, ("diagG", rel(gG, rG))
    assert rel(gGl, rGl) <= tol, ("diagGl", rel(gGl, rGl))
    if bonds:
        assert rel(gJ, rJ) <= tol, ("J", rel(gJ, rJ))


@pytest.mark.parametrize("leaf", [4, 8])
def test_c1_16x16_against_golden(F, leaf):
    d = np.loadtxt(os.path.join(GOLD, "c1_16x16_dense.txt"))
    gJ = np.loadtxt(os.path.join(GOLD, "c1_16x16_bond_current.txt"))
    ref = (d[:, 1] + 1j * d[:, 2], 1j * d[:, 3], gJ)
    G, Gl, J = gpu_lesser(F, W.c1(), W.c1_energies(), leaf=leaf)
    check((G[0], Gl[0], J[0]), ref)


def test_c2_40x40_64_energies_one_batch(F):
    mesh, Es = W.c2(), W.c2_energies()
    G, Gl, J = gpu_lesser(F, mesh, Es, leaf=5, max_batch=64)
    for k in range(0, 64, 3):
        check((G[k], Gl[k], J[k]), dense_ref(mesh, Es[k]))


@pytest.mark.parametrize("mesh,E,leaf", [
    (W.Mesh(13, 17, 9, 1.0, 0.2, -1.0, 1.0, 51), 2.3 + 1e-6j, 3),
    (W.Mesh(37, 21, 9, 1.0, 0.2, -1.0, 1.0, 52), 5.1 + 1e-6j, 4),
    (W.Mesh(40, 61, 9, 1.0, 0.2, -1.0, 1.0, 53), 1.7 + 1e-6j, 5),
    (W.Mesh(70, 33, 5, 1.0, 0.0, -0.5, 0.5, 54), 0.9 + 1e-6j, 8),
])
def test_ragged_meshes(F, mesh, E, leaf):
    G, Gl, J = gpu_lesser(F, mesh, np.array([E]), leaf=leaf)
    check((G[0], Gl[0], J[0]), dense_ref(mesh, E))


def test_diag_path_equals_lesser_diag(F):
    mesh = W.Mesh(24, 30, 9, 1.0, 0.2, -1.0, 1.0, 55)
    Es = W.energy_grid(0.5, 7.5, 5)
    f = F.Find.from_mesh(mesh, leaf=4)
    g1 = f.solve_diag(tcplx(Es)).cpu().numpy()
    g2 = f.solve_lesser(tcplx(Es))[0].cpu().numpy()
    f.close()
    assert np.array_equal(g1, g2)
    for k in range(5):
        assert rel(g1[k], dense_ref(mesh, Es[k])[0]) <= TOL


def test_user_given_nonsymmetric_lead_sigma(F):
    # Sigma_L, Sigma_R neither symmetric nor equal: A != A^T, so any transposed
    # block in the kernels shows up.
    mesh = W.Mesh(9, 14, 9, 1.0, 0.2, -1.0, 1.0, 56)
    rng = np.random.default_rng(7)
    E = np.array([1.9 + 1e-6j, 4.4 + 1e-6j])
    nx = mesh.nx
    sL = rng.uniform(-0.5, 0.5, (2, nx, nx)) + 1j * rng.uniform(-0.6, 0.0, (2, nx, nx))
    sR = rng.uniform(-0.5, 0.5, (2, nx, nx)) + 1j * rng.uniform(-0.6, 0.0, (2, nx, nx))
    G, Gl, J = gpu_lesser(F, mesh, E, leaf=3, fL=0.7, fR=0.2, sigL=sL, sigR=sR)
    for k in range(2):
        check((G[k], Gl[k], J[k]), dense_ref(mesh, E[k], 0.7, 0.2, sL[k], sR[k]))


def test_eta_identity(F):
    # Sigma< = i (Gamma_L + Gamma_R + 2 eta I)  =>  diag G< = -2 i Im diag G
    mesh = W.Mesh(31, 45, 9, 1.0, 0.2, -1.0, 1.0, 57)
    Es = W.energy_grid(0.3, 7.7, 4)
    d = np.full(mesh.n, 2j * 1e-6)
    G, Gl, _ = gpu_lesser(F, mesh, Es, leaf=4, fL=1.0, fR=1.0, dles=d, bonds=False)
    for k in range(4):
        assert rel(Gl[k], -2j * G[k].imag) <= 1e-9


def test_per_energy_node_diagonal_sigma_lesser(F):
    mesh = W.Mesh(11, 12, 5, 1.0, 0.0, -0.5, 0.5, 58)
    Es = W.energy_grid(0.4, 3.6, 3)
    rng = np.random.default_rng(3)
    d = 1j * rng.uniform(0.0, 0.1, (3, mesh.n))
    G, Gl, J = gpu_lesser(F, mesh, Es, leaf=4, dles=d)
    for k in range(3):
        check((G[k], Gl[k], J[k]), dense_ref(mesh, Es[k], dles=d[k]))


def test_host_pointers_match_device_pointers(F):
    mesh = W.Mesh(20, 26, 9, 1.0, 0.2, -1.0, 1.0, 59)
    Es = W.energy_grid(1.0, 6.0, 3)
    f = F.Find.from_mesh(mesh, leaf=4)
    hG, hGl, hJ = f.solve_lesser(np.ascontiguousarray(Es))
    dG, dGl, dJ = (x.cpu().numpy() for x in f.solve_lesser(tcplx(Es)))
    f.close()
    assert isinstance(hG, np.ndarray)
    assert np.array_equal(hG, dG) and np.array_equal(hGl, dGl) and np.array_equal(hJ, dJ)


def test_alone_and_in_batch_are_bitwise_equal(F):
    mesh = W.Mesh(24, 40, 5, 1.0, 0.0, -0.5, 0.5, 60)
    Es = W.energy_grid(0.2, 3.8, 6)
    both = gpu_lesser(F, mesh, Es, leaf=5, max_batch=6)
    for k in (0, 4):
        alone = gpu_lesser(F, mesh, Es[k:k + 1], leaf=5, max_batch=1)
        for a, b in zip(alone, both):
            assert np.array_equal(a[0], b[k])


def test_chunked_batches_match_single_batch(F):
    mesh = W.Mesh(16, 22, 9, 1.0, 0.2, -1.0, 1.0, 61)
    Es = W.energy_grid(0.5, 7.5, 7)
    a = gpu_lesser(F, mesh, Es, leaf=4, max_batch=7)
    b = gpu_lesser(F, mesh, Es, leaf=4, max_batch=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("mesh,leaf", [
    (W.Mesh(3, 4, 9, 1.0, 0.2, -1.0, 1.0, 62), 8),    # the root is the only leaf
    (W.Mesh(1, 23, 5, 1.0, 0.0, -0.5, 0.5, 63), 2),   # a 1D chain
    (W.Mesh(9, 2, 9, 1.0, 0.2, -1.0, 1.0, 64), 2),    # only the two contact columns
])
def test_degenerate_meshes(F, mesh, leaf):
    E = np.array([1.3 + 1e-6j])
    G, Gl, J = gpu_lesser(F, mesh, E, leaf=leaf)
    check((G[0], Gl[0], J[0]), dense_ref(mesh, E[0]))


def test_exact_zero_pivot_is_reported(F):
    # 1D chain of 3 nodes, leaf 1: node 2 is eliminated alone from the upward
    # merge of [1,3).  Sigma_R chosen so that A(2,2) = 0 exactly.
    mesh = W.Mesh(1, 3, 5, 1.0, 0.0, 0.0, 0.0, 1)
    E = np.array([0.5 + 0.0j, 0.7 + 0.0j])
    sR = (E - 4.0).reshape(2, 1, 1).copy()
    sR[0] = 0.1  # energy 0 is regular, energy 1 is singular
    f = F.Find.from_mesh(mesh, leaf=1)
    with pytest.raises(F.FindError) as ei:
        f.solve_diag(tcplx(E), sigmaR=tcplx(sR))
    assert ei.value.code == 3 and "energy index 1" in str(ei.value)
    f.close()


def test_current_continuity_on_gpu(F):
    mesh = W.Mesh(30, 50, 9, 1.0, 0.2, -1.0, 1.0, 65)
    E = np.array([2.6 + 1e-6j])
    G, Gl, J = gpu_lesser(F, mesh, E, leaf=6)
    bi, bj = dense.bond_list(mesh.nx, mesh.ny, mesh.stencil)
    out = np.zeros(mesh.n)
    np.add.at(out, bi, J[0])
    np.add.at(out, bj, -J[0])
    y = np.arange(mesh.n) // mesh.nx
    inner = (y > 0) & (y < mesh.ny - 1)
    expect = (2j * 1e-6 * Gl[0]).real
    assert np.abs(out[inner] - expect[inner]).max() <= 1e-9 * np.abs(J[0]).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed_ff"])
def test_symmetric_updates_match_full_updates(F, precision):
    # closed-form leads: A = A^T, so U is computed on one triangle and R
    # (anti-Hermitian) too; passing the same Sigma explicitly computes every
    # entry.  Both must agree to rounding and with the dense definition.
    import torch
    mesh = W.Mesh(30, 44, 9, 1.0, 0.2, -1.0, 1.0, 66)
    Es = W.energy_grid(0.7, 7.3, 3)
    P = problem.MeshProblem.from_mesh(mesh)
    sig = np.stack([P.lead_sigmas(E)[0] for E in Es])
    f = F.Find.from_mesh(mesh, leaf=5, precision=precision, sym_u=True)
    a = [x.cpu().numpy() for x in f.solve_lesser(tcplx(Es))]
    b = [x.cpu().numpy() for x in f.solve_lesser(tcplx(Es), sigmaL=tcplx(sig), sigmaR=tcplx(sig))]
    f.close()
    # computing one triangle of U moves results by rounding only (measured
    # 7e-12 on a 64x128 mesh): both forms are held to the path's bar
    tol = 1e-10 if precision == "fp64" else 1e-5
    for k in range(3):
        for name, x, y in zip(("diagG", "diagGl", "J"), a, b):
            assert rel(x[k], y[k]) <= tol, (name, k, rel(x[k], y[k]))
        check((a[0][k], a[1][k], a[2][k]), dense_ref(mesh, Es[k]), tol=tol)
