"""Pins of O-find (oracle/find.py).

* brute force: O-find equals the dense definition (Theorem 1, Sec. 2.2) on
  small meshes, 5- and 9-point, for diag G, diag G< and bond currents;
* a random NON-symmetric, non-Hermitian A and Sigma on the FIND pattern, so a
  transposed or unconjugated operand cannot hide behind A = A^T;
* tree independence: leaf sizes and the tie rule do not change the result;
* Property 1 (symmetry preservation): every U_g is complex symmetric, and
  with anti-Hermitian Sigma< every R_g is anti-Hermitian;
* a bond reached from two leaves gives the same current from both;
* planted mistakes in the elimination step are caught by these pins.
"""

import numpy as np
import pytest

import workloads as W
from oracle import dense, find, problem


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _both(mesh, E, leaf=8, tie="y", bonds=True):
    P = problem.MeshProblem.from_mesh(mesh)
    A, Sl = P.assemble(E)
    d = dense.dense_outputs(A, Sl, P.H, mesh.nx, mesh.ny, mesh.stencil)
    f = find.find_outputs(P, E, leaf=leaf, tie=tie, bonds=bonds)
    return d, f


@pytest.mark.parametrize("mesh,E,leaf", [
    (W.Mesh(8, 8, 5, 1.0, 0.0, -0.5, 0.5, 11), 1.0 + 1e-6j, 4),
    (W.c1(), 1.0 + 1e-6j, 4),
    (W.c1(), 1.0 + 1e-6j, 8),
    (W.Mesh(12, 9, 9, 1.0, 0.2, -1.0, 1.0, 12), 3.1 + 1e-6j, 4),
    (W.Mesh(7, 19, 9, 1.0, 0.2, -1.0, 1.0, 13), 6.7 + 1e-6j, 3),
    (W.Mesh(21, 6, 5, 1.0, 0.0, -0.5, 0.5, 14), 2.5 + 1e-6j, 5),
])
def test_find_equals_dense(mesh, E, leaf):
    (dG, dGl, J, _, _), (fG, fGl, (fJ, fJalt), _) = _both(mesh, E, leaf)
    assert rel(fG, dG) <= 1e-11
    assert rel(fGl, dGl) <= 1e-11
    assert rel(fJ, J) <= 1e-11
    both = ~np.isnan(fJalt)
    assert both.any()
    assert np.abs(fJalt[both] - fJ[both]).max() <= 1e-11 * np.abs(J).max()


def test_find_equals_dense_c2_subset():
    mesh = W.c2()
    Es = W.c2_energies()[[0, 21, 42, 63]]
    for E in Es:
        (dG, dGl, _, _, _), (fG, fGl, _, _) = _both(mesh, E, 5, bonds=False)
        assert rel(fG, dG) <= 1e-10
        assert rel(fGl, dGl) <= 1e-10


def test_find_single_leaf_root():
    mesh = W.Mesh(3, 4, 9, 1.0, 0.2, -1, 1, 15)
    (dG, dGl, J, _, _), (fG, fGl, (fJ, _), _) = _both(mesh, 0.9 + 1e-6j, 8)
    assert rel(fG, dG) <= 1e-12 and rel(fGl, dGl) <= 1e-12 and rel(fJ, J) <= 1e-12


def general_system(nx, ny, stencil, seed):
    """Random complex A and Sigma on the FIND pattern, neither symmetric nor
    (anti-)Hermitian."""
    diag, off, lead, sig, lead_sig = W.random_general_system(nx, ny, stencil, seed)
    n = nx * ny
    offs = problem.stencil_offsets(9)
    rows, cols, av, sv = [np.arange(n)], [np.arange(n)], [diag], [sig[:, 8]]
    x = np.arange(n) % nx
    y = np.arange(n) // nx
    for k, (dx, dy, kind) in enumerate(offs):
        if stencil == 5 and kind == 1:
            continue
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        rows.append(np.nonzero(ok)[0])
        cols.append(((y + dy) * nx + x + dx)[ok])
        av.append(off[ok, k])
        sv.append(sig[ok, k])
    import scipy.sparse as sp
    A = sp.csr_matrix((np.concatenate(av), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    S = sp.csr_matrix((np.concatenate(sv), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    left, right = problem.contact_nodes(nx, ny)
    A = (A + problem.embed(n, left, lead[0]) + problem.embed(n, right, lead[1])).tocsr()
    S = (S + problem.embed(n, left, lead_sig[0]) + problem.embed(n, right, lead_sig[1])).tocsr()
    return A, S


@pytest.mark.parametrize("nx,ny,stencil,leaf,seed", [(6, 9, 5, 3, 21), (7, 8, 9, 4, 22), (10, 5, 9, 2, 23)])
def test_find_general_nonsymmetric(nx, ny, stencil, leaf, seed):
    A, S = general_system(nx, ny, stencil, seed)
    assert np.abs(A - A.T).max() > 0.1
    G = np.linalg.inv(A.toarray())
    Gl = G @ S.toarray() @ G.conj().T
    f = find.FindOracle(A, S, nx, ny, problem.find_pattern(nx, ny, stencil), leaf)
    bi, bj = dense.bond_list(nx, ny, stencil)
    fG, fGl, (gji, gij, _, _) = f.run(bonds=(bi, bj))
    assert rel(fG, np.diag(G)) <= 1e-11
    assert rel(fGl, np.diag(Gl)) <= 1e-11
    assert rel(gji, Gl[bj, bi]) <= 1e-11
    assert rel(gij, Gl[bi, bj]) <= 1e-11


def test_tree_independence():
    mesh = W.Mesh(12, 10, 9, 1.0, 0.2, -1.0, 1.0, 31)
    P = problem.MeshProblem.from_mesh(mesh)
    E = 2.9 + 1e-6j
    ref = find.find_outputs(P, E, leaf=8, tie="y")
    for leaf, tie in [(2, "y"), (4, "x"), (5, "y"), (16, "x")]:
        got = find.find_outputs(P, E, leaf=leaf, tie=tie)
        assert rel(got[0], ref[0]) <= 1e-11
        assert rel(got[1], ref[1]) <= 1e-11
        assert rel(got[2][0], ref[2][0]) <= 1e-11


def test_symmetry_preservation():
    mesh = W.Mesh(12, 14, 9, 1.0, 0.2, -1.0, 1.0, 32)
    P = problem.MeshProblem.from_mesh(mesh)
    _, _, _, f = find.find_outputs(P, 1.3 + 1e-6j, leaf=4, bonds=False)
    for store in (f.U, f.Ubar):
        for U in store.values():
            assert np.abs(U - U.T).max() <= 1e-10 * np.abs(U).max()
    for store in (f.R, f.Rbar):
        for R in store.values():
            if np.abs(R).max() > 0:
                assert np.abs(R + R.conj().T).max() <= 1e-10 * np.abs(R).max()


def test_sigma_update_vanishes_away_from_the_contacts():
    # Sec. 4.3 (Sigma< sparsity): Sigma< lives on the contact columns only,
    # so the upward R of a cluster with no contact node is exactly zero and
    # the library skips its Eq. (7) products; every cluster touching a
    # biased contact has R != 0, and every complement cluster too.
    mesh = W.Mesh(12, 24, 9, 1.0, 0.2, -1.0, 1.0, 33)
    P = problem.MeshProblem.from_mesh(mesh)
    _, _, _, f = find.find_outputs(P, 2.1 + 1e-6j, fL=1.0, fR=0.4, leaf=4, bonds=False)
    zero = nonzero = 0
    for c, R in f.R.items():
        C = f.tree[c]
        if C.y0 > 0 and C.y1 < mesh.ny:
            assert not np.any(R), c
            zero += 1
        else:
            assert np.abs(R).max() > 0, c
            nonzero += 1
    assert zero > nonzero > 0
    assert all(np.abs(R).max() > 0 for R in f.Rbar.values())


def test_set_rules():
    # B_C lies in C, Bbar_C outside C; S_C = (B_C1 u B_C2) \ B_C contains no
    # node with a neighbour outside C; leaves tile the mesh.
    nx, ny = 13, 17
    tree = find.build_tree(nx, ny, 4)
    Pm = problem.find_pattern(nx, ny, 9)
    B, Bbar = find.boundary_sets(tree, Pm, nx)
    cover = np.zeros(nx * ny, int)
    for k, c in enumerate(tree):
        assert np.all(c.contains(B[k], nx))
        assert not np.any(c.contains(Bbar[k], nx))
        if not c.children:
            cover[c.nodes] += 1
            assert c.x1 - c.x0 <= 4 and c.y1 - c.y0 <= 4
        else:
            c1, c2 = c.children
            S = np.setdiff1d(np.union1d(B[c1], B[c2]), B[k])
            nb = Pm[S].indices
            assert np.all(c.contains(nb, nx))
    assert np.all(cover == 1)


# ---- planted mistakes: each broken elimination must fail the brute-force pin

def _broken(kind):
    def elim(M, Sg, s):
        if s == 0:
            return M.copy(), Sg.copy()
        MSS, MSB, MBS, MBB = M[:s, :s], M[:s, s:], M[s:, :s], M[s:, s:]
        L = np.linalg.solve(MSS.T, MBS.T).T
        if kind == "L_from_wrong_side":
            L = np.linalg.solve(MSS, MBS.T).T
        U = MBB - L @ MSB
        if kind == "U_transposed_operand":
            U = MBB - L @ MBS.T
        LH = L.conj().T
        if kind == "LH_not_conjugated":
            LH = L.T
        t2 = L @ Sg[:s, s:]
        t3 = Sg[s:, :s] @ LH
        t4 = L @ Sg[:s, :s] @ LH
        if kind == "drop_LSL":
            t4 = 0 * t4
        if kind == "sign_t2":
            t2 = -t2
        if kind == "swap_SB_BS":
            t2 = L @ Sg[s:, :s].T
        return U, Sg[s:, s:] - t2 - t3 + t4
    return elim


@pytest.mark.parametrize("kind", ["L_from_wrong_side", "U_transposed_operand", "LH_not_conjugated",
                                  "drop_LSL", "sign_t2", "swap_SB_BS"])
def test_planted_mistakes_are_caught(kind, monkeypatch):
    nx, ny, stencil = 7, 8, 9
    A, S = general_system(nx, ny, stencil, 41)
    G = np.linalg.inv(A.toarray())
    Gl = G @ S.toarray() @ G.conj().T
    monkeypatch.setattr(find, "eliminate", _broken(kind))
    f = find.FindOracle(A, S, nx, ny, problem.find_pattern(nx, ny, stencil), 3)
    fG, fGl, _ = f.run()
    err = max(rel(fG, np.diag(G)), rel(fGl, np.diag(Gl)))
    assert err > 1e-6
