"""Pins of the problem assembly and of O-dense against closed forms and
identities that hold independently of any implementation.

* clean wire (V = 0): device plus leads is a perfect infinite wire, so
  diag G and diag G< have mode-sum closed forms;
* the eta identity: with Sigma<_test = i (Gamma_L + Gamma_R + 2 eta I),
  G<_test = G^H - G exactly, so diag G<_test = -2 i Im diag G;
* current continuity at every node off the contact columns;
* Landauer: the current through any cut is Tr[Gamma_L G Gamma_R G^H] (f_L = 1,
  f_R = 0) up to O(eta) leakage, and equals the number of open modes in a
  clean wire (5 open modes at E = 1 for nx = 16, counted by hand:
  |E - 4 + 2 cos(m pi/17)| < 2  <=>  m <= 5);
* symmetry: A = A^T gives G = G^T; Re diag G< = 0, Im diag G <= 0 <= Im diag G<.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, problem


def clean_wire_diag(mesh, E):
    nx = mesh.nx
    phi, _ = problem.transverse_modes(nx)
    eps, tau = problem.mode_energies(nx, mesh.t, mesh.tp, mesh.onsite0, mesh.stencil)
    sig = problem.mode_self_energy(E, eps, tau)
    g00 = 1.0 / (E - eps - 2.0 * sig)
    gam = -2.0 * sig.imag
    lam2 = np.abs(sig / tau) ** 2
    G = np.empty((mesh.ny, nx), np.complex128)
    Gl = np.empty((mesh.ny, nx), np.complex128)
    for y in range(mesh.ny):
        G[y] = (phi ** 2) @ g00
        Gl[y] = 1j * (phi ** 2) @ (gam * np.abs(g00) ** 2 * lam2 ** y)
    return G.reshape(-1), Gl.reshape(-1)


@pytest.mark.parametrize("mesh,E", [
    (W.Mesh(16, 16, 5, 1.0, 0.0, 0.0, 0.0, 1), 1.0 + 1e-6j),
    (W.Mesh(9, 14, 9, 1.0, 0.2, 0.0, 0.0, 1), 3.3 + 1e-6j),
    (W.Mesh(6, 20, 9, 1.0, 0.2, 0.0, 0.0, 1), 6.4 + 1e-6j),
])
def test_clean_wire_closed_form(mesh, E):
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E, 1.0, 0.0)
    dG, dGl, _, _, _ = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    rG, rGl = clean_wire_diag(mesh, E)
    assert np.abs(dG - rG).max() <= 1e-9 * np.abs(rG).max()
    assert np.abs(dGl - rGl).max() <= 1e-9 * np.abs(rGl).max()


def _eta_identity(mesh, E):
    P = problem.MeshProblem.from_mesh(mesh)
    eta = E.imag
    A, Sl = P.assemble(E, 1.0, 1.0, diag_lesser=np.full(mesh.n, 2j * eta))
    G = dense.dense_green(A)
    Gl = dense.dense_lesser(G, Sl)
    return G, Gl


@pytest.mark.parametrize("mesh,E", [(W.c1(), 1.0 + 1e-6j), (W.Mesh(10, 13, 9, 1.0, 0.2, -1, 1, 4), 5.5 + 1e-6j)])
def test_eta_identity(mesh, E):
    G, Gl = _eta_identity(mesh, E)
    assert np.abs(Gl - (G.conj().T - G)).max() <= 1e-9 * np.abs(G).max()
    assert np.abs(np.diag(Gl) + 2j * np.diag(G).imag).max() <= 1e-9 * np.abs(np.diag(G)).max()


def _dense(mesh, E, fL=1.0, fR=0.0):
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E, fL, fR)
    return P, A, Sl, dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)


@pytest.mark.parametrize("mesh,E", [(W.c1(), 1.0 + 1e-6j), (W.Mesh(8, 11, 9, 1.0, 0.2, -1, 1, 5), 2.2 + 1e-6j)])
def test_current_continuity(mesh, E):
    P, A, Sl, (dG, dGl, J, G, Gl) = _dense(mesh, E)
    assert np.abs(J.imag).max() <= 1e-12 * np.abs(J).max()
    bi, bj = dense.bond_list(mesh.nx, mesh.ny, mesh.stencil)
    out = np.zeros(mesh.n)
    np.add.at(out, bi, J.real)
    np.add.at(out, bj, -J.real)
    y = np.arange(mesh.n) // mesh.nx
    inner = (y > 0) & (y < mesh.ny - 1)
    expect = (2j * E.imag * dGl).real
    assert np.abs(out[inner] - expect[inner]).max() <= 1e-9 * np.abs(J).max()


def _cut_currents(mesh, J):
    bi, bj = dense.bond_list(mesh.nx, mesh.ny, mesh.stencil)
    yi, yj = bi // mesh.nx, bj // mesh.nx
    return np.array([J.real[(yi == k) & (yj == k + 1)].sum() for k in range(mesh.ny - 1)])


def test_landauer_clean_wire_counts_open_modes():
    mesh = W.Mesh(16, 16, 5, 1.0, 0.0, 0.0, 0.0, 1)
    P, A, Sl, (dG, dGl, J, G, Gl) = _dense(mesh, 1.0 + 1e-6j)
    cut = _cut_currents(mesh, J)
    assert np.abs(cut - 5.0).max() < 1e-3


@pytest.mark.parametrize("mesh,E", [(W.c1(), 1.0 + 1e-6j), (W.Mesh(9, 12, 9, 1.0, 0.2, -1, 1, 6), 4.1 + 1e-6j)])
def test_landauer_transmission(mesh, E):
    P, A, Sl, (dG, dGl, J, G, Gl) = _dense(mesh, E)
    sL, sR = P.lead_sigmas(E)
    left, right = problem.contact_nodes(mesh.nx, mesh.ny)
    gL, gR = problem.broadening(sL), problem.broadening(sR)
    Glr = G[np.ix_(left, right)]
    T = np.trace(gL @ Glr @ gR @ Glr.conj().T).real
    cut = _cut_currents(mesh, J)
    assert T > 0
    assert np.abs(cut - T).max() <= 1e-4 * max(T, 1.0)


def test_symmetry_and_signs():
    mesh = W.Mesh(10, 12, 9, 1.0, 0.2, -1, 1, 3)
    P, A, Sl, (dG, dGl, J, G, Gl) = _dense(mesh, 1.7 + 1e-6j)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(G - G.T).max() <= 1e-10 * np.abs(G).max()
    assert np.abs(Gl + Gl.conj().T).max() <= 1e-10 * np.abs(Gl).max()
    assert np.abs(dGl.real).max() <= 1e-10 * np.abs(dGl).max()
    assert dG.imag.max() <= 0
    assert dGl.imag.min() >= 0


def test_bond_list_counts():
    i, j = dense.bond_list(5, 7, 5)
    assert len(i) == 5 * 6 + 4 * 7
    i, j = dense.bond_list(5, 7, 9)
    assert len(i) == 5 * 6 + 4 * 7 + 2 * 4 * 6
    xi, yi, xj, yj = i % 5, i // 5, j % 5, j // 5
    assert np.all(np.maximum(abs(xi - xj), abs(yi - yj)) == 1)
    assert len(set(zip(i.tolist(), j.tolist()))) == len(i)
