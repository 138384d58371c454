"""Plain FIND on the CPU (O-find): upward pass, downward pass, leaf extraction.

TEST INFRASTRUCTURE ONLY (see ``oracle/problem.py``).

The steps follow the paper in its own order and notation:

* Sec. 2.1 / 2.2 -- cluster tree, boundary set B_C (nodes of C with a
  neighbour outside C), private inner set S_C = (B_C1 u B_C2) \\ B_C.
* Eq. (13)  L = A(B,S) A(S,S)^{-1}
* Eq. (2)   U = A(B,B) - L A(S,B)              (major update)
* Eq. (7)   R = S(B,B) - L S(S,B) - S(B,S) L^H + L S(S,S) L^H   (Sigma update)
* Upward pass (Sec. 2.2, Sec. 3.1), children before parents: a leaf starts
  from A(C,C) and Sigma(C,C); a merge assembles [U_C1 A(B1,B2); A(B2,B1) U_C2]
  (original couplings off the diagonal blocks, Corollary 1) and the same for
  Sigma with R_C1, R_C2; the root is not eliminated.
* Downward pass (Sec. 2.2), parents before children: for C with parent D and
  sibling D1, assemble over B_Dbar u B_D1 from (U_Dbar, U_D1) and (R_Dbar,
  R_D1); when D is the root, Dbar is empty and the blocks of D1 alone are
  used (the reading taken: U_Cbar from U_D1 and R_Cbar from R_D1).
* Leaf extraction, Sec. 3.2: for each leaf C,
    Eq. (8)   G(C,C) = [A(C,C) - A(C,Bb) U_Cbar^{-1} A(Bb,C)]^{-1}
    Eq. (5)   G<(C,C) = U_nn^{-1} R_nn U_nn^{-H}, where U_nn, R_nn come from
              one more elimination (Eqs. 13, 2, 7) of Bb from the bordered
              system over Bb u C (so U_nn^{-1} = G(C,C));
    Eqs. (9)-(10) G(Bb,C), G(C,Bb), and the block inverse for G(Bb,Bb)
              ("nodes farther away"), from which the bordered G< over Bb u C
              is G_K Sigma_K G_K^H with Sigma_K = [R_Cbar S(Bb,C); S(C,Bb) S(C,C)].
    Bond currents use the neighbour entries of that bordered G<.

Optionally (symmetric=True, Sec. 4.2) the eliminations use the symmetric
factorisation M(S,S) = L D L^T with Bunch-Kaufman pivoting instead of the LU
(eliminate_symmetric); A must equal A^T.

Readings taken where the paper is silent: the tree bisects the longer side
(ties split y; the first half gets floor(len/2)) until both sides are <= leaf;
B sets are computed on the structural graph of A, which includes the dense
contact-column couplings of the lead self-energies.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Cluster:
    __slots__ = ("x0", "x1", "y0", "y1", "parent", "children", "depth", "nodes")

    def __init__(self, x0, x1, y0, y1, parent, depth, nx):
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.parent = parent
        self.depth = depth
        self.children = []
        self.nodes = np.add.outer(np.arange(y0, y1) * nx, np.arange(x0, x1)).reshape(-1)

    def contains(self, nodes, nx):
        x = nodes % nx
        y = nodes // nx
        return (x >= self.x0) & (x < self.x1) & (y >= self.y0) & (y < self.y1)


def build_tree(nx: int, ny: int, leaf: int, tie: str = "y"):
    """Recursive bisection; cluster 0 is the root (the whole mesh)."""
    tree = []

    def make(x0, x1, y0, y1, parent, depth):
        idx = len(tree)
        c = Cluster(x0, x1, y0, y1, parent, depth, nx)
        tree.append(c)
        wx, wy = x1 - x0, y1 - y0
        if wx <= leaf and wy <= leaf:
            return idx
        split_y = wy > wx or (wy == wx and tie == "y")
        if split_y:
            h = wy // 2
            kids = [(x0, x1, y0, y0 + h), (x0, x1, y0 + h, y1)]
        else:
            h = wx // 2
            kids = [(x0, x0 + h, y0, y1), (x0 + h, x1, y0, y1)]
        c.children = [make(*k, idx, depth + 1) for k in kids]
        return idx

    make(0, nx, 0, ny, -1, 0)
    return tree


def _neighbours(P: sp.csr_matrix, nodes: np.ndarray):
    starts = P.indptr[nodes]
    counts = P.indptr[nodes + 1] - starts
    src = np.repeat(nodes, counts)
    base = np.repeat(starts - (np.cumsum(counts) - counts), counts)
    nbr = P.indices[base + np.arange(counts.sum())]
    return src, nbr


def boundary_sets(tree, P: sp.csr_matrix, nx: int):
    """B_C (inside C, touching outside) and B_Cbar (outside C, touching C)."""
    B, Bbar = [], []
    for c in tree:
        src, nbr = _neighbours(P, c.nodes)
        out = ~c.contains(nbr, nx)
        B.append(np.unique(src[out]))
        Bbar.append(np.unique(nbr[out]))
    return B, Bbar


def eliminate(M: np.ndarray, Sg: np.ndarray, s: int):
    """Eliminate the first s indices of an [S, B]-ordered block pair.

    Eq. (13): L = M(B,S) M(S,S)^{-1}   (LAPACK solve, partial pivoting)
    Eq. (2):  U = M(B,B) - L M(S,B)
    Eq. (7):  R = Sg(B,B) - L Sg(S,B) - Sg(B,S) L^H + L Sg(S,S) L^H
    """
    if s == 0:
        return M.copy(), Sg.copy()
    MSS, MSB, MBS, MBB = M[:s, :s], M[:s, s:], M[s:, :s], M[s:, s:]
    L = np.linalg.solve(MSS.T, MBS.T).T
    U = MBB - L @ MSB
    LH = L.conj().T
    R = Sg[s:, s:] - L @ Sg[:s, s:] - Sg[s:, :s] @ LH + L @ Sg[:s, :s] @ LH
    return U, R


def eliminate_symmetric(M: np.ndarray, Sg: np.ndarray, s: int):
    """The same elimination for complex symmetric M (A = A^T), by the
    symmetric factorisation of Sec. 4.2 (optimisation for symmetry):

        M(S,S) = Lf D Lf^T       (LDL^T with Bunch-Kaufman diagonal pivoting:
                                   D has 1x1 and 2x2 blocks; Lf is lower
                                   triangular up to the pivot permutation)
        W = Lf^{-1} M(S,B)
        U = M(B,B) - W^T D^{-1} W                     (Eq. 2, as in Sec. 4.2)
        L = M(B,S) M(S,S)^{-1} = (Lf^{-T} D^{-1} W)^T (Eq. 13; M(B,S) = M(S,B)^T)
        R as in Eq. (7).

    Plain transposes throughout (complex symmetric, not Hermitian)."""
    if s == 0:
        return M.copy(), Sg.copy()
    from scipy.linalg import ldl, solve_triangular
    MSS, MSB, MBB = M[:s, :s], M[:s, s:], M[s:, s:]
    lu, d, perm = ldl(MSS, lower=True, hermitian=False)
    W = solve_triangular(lu[perm], MSB[perm], lower=True, unit_diagonal=True)
    DW = np.linalg.solve(d, W)
    U = MBB - W.T @ DW
    # L^T = Lf^{-T} D^{-1} W with Lf = lu, whose rows perm form a unit lower
    # triangle T: Lf^{-T} = P^T T^{-T} applied as a solve with T^T, unpermuted
    Lt = np.empty_like(DW)
    Lt[perm] = solve_triangular(lu[perm].T, DW, lower=False, unit_diagonal=True)
    L = Lt.T
    LH = L.conj().T
    R = Sg[s:, s:] - L @ Sg[:s, s:] - Sg[s:, :s] @ LH + L @ Sg[:s, :s] @ LH
    return U, R


def _reorder(nodes: np.ndarray, keep: np.ndarray):
    """Permutation of ``nodes`` into [S, keep]: S = nodes not kept (in their
    given order), followed by the kept nodes in the order of ``keep``."""
    is_keep = np.isin(nodes, keep)
    s_pos = np.nonzero(~is_keep)[0]
    order = np.argsort(nodes, kind="stable")
    k_pos = order[np.searchsorted(nodes[order], keep)]
    if not np.array_equal(nodes[k_pos], keep):
        raise AssertionError("kept set is not a subset of the merged set")
    return np.concatenate([s_pos, k_pos]), len(s_pos)


class FindOracle:
    """FIND for one matrix A and one Sigma (any values on the FIND pattern)."""

    def __init__(self, A, Sl, nx: int, ny: int, pattern=None, leaf: int = 8,
                 tie: str = "y", symmetric: bool = False):
        self.A = sp.csr_matrix(A, dtype=np.complex128)
        # symmetric: eliminate with the LDL^T form (eliminate_symmetric),
        # which reads one triangle of each block and M(S,B) for M(B,S), i.e.
        # uses the symmetric part of A; A must equal A^T up to rounding (the
        # closed-form lead Sigma = Phi diag(sigma) Phi^T is symmetric only to
        # the last bit).  Property 1 keeps every U symmetric.
        self.symmetric = symmetric
        if symmetric and abs(self.A - self.A.T).max() > 1e-13 * abs(self.A).max():
            raise ValueError("the symmetric elimination needs A = A^T")
        self.Sl = sp.csr_matrix(Sl, dtype=np.complex128)
        self.A.sum_duplicates()
        self.Sl.sum_duplicates()
        self.nx, self.ny = nx, ny
        self._colpos = np.full(nx * ny, -1, np.int64)
        if pattern is None:
            pattern = self.A.copy()
            pattern.data = np.abs(pattern.data)
            pattern = (pattern + pattern.T).tocsr()
            pattern.setdiag(0)
            pattern.eliminate_zeros()
        self.tree = build_tree(nx, ny, leaf, tie)
        self.B, self.Bbar = boundary_sets(self.tree, sp.csr_matrix(pattern), nx)
        self.U, self.R, self.Ubar, self.Rbar = {}, {}, {}, {}

    # -- blocks of the original matrices: Mat(rows, cols) as a dense array,
    # read straight from the CSR rows through a column-position map
    def _block(self, Mat, rows, cols):
        pos = self._colpos
        pos[cols] = np.arange(len(cols))
        starts = Mat.indptr[rows]
        counts = Mat.indptr[rows + 1] - starts
        flat = np.repeat(starts - (np.cumsum(counts) - counts), counts) + np.arange(counts.sum())
        r = np.repeat(np.arange(len(rows)), counts)
        c = pos[Mat.indices[flat]]
        keep = c >= 0
        out = np.zeros((len(rows), len(cols)), np.complex128)
        out[r[keep], c[keep]] = Mat.data[flat[keep]]
        pos[cols] = -1
        return out

    def _a(self, rows, cols):
        return self._block(self.A, rows, cols)

    def _s(self, rows, cols):
        return self._block(self.Sl, rows, cols)

    def _merge(self, n1, n2, U1, U2, R1, R2):
        M = np.block([[U1, self._a(n1, n2)], [self._a(n2, n1), U2]])
        Sg = np.block([[R1, self._s(n1, n2)], [self._s(n2, n1), R2]])
        return np.concatenate([n1, n2]), M, Sg

    def _eliminate_onto(self, nodes, M, Sg, keep):
        perm, s = _reorder(nodes, keep)
        elim = eliminate_symmetric if self.symmetric else eliminate
        return elim(M[np.ix_(perm, perm)], Sg[np.ix_(perm, perm)], s)

    def _postorder(self):
        """Cluster indices, children before parents (the root last)."""
        order, stack = [], [(0, False)]
        while stack:
            c, expanded = stack.pop()
            if expanded or not self.tree[c].children:
                order.append(c)
                continue
            stack.append((c, True))
            for ch in reversed(self.tree[c].children):
                stack.append((ch, False))
        return order

    def upward_pass(self):
        """U_C and R_C for every cluster but the root (Sec. 2.2, Sec. 3.1),
        children before parents.  A leaf's block is A(C,C) with Sigma<(C,C);
        a parent's is the block over B_C1 u B_C2 assembled from its
        children's U and R and the original couplings between the two sets
        (Corollary 1); eliminating its private inner set S_C leaves U_C on
        B_C (Eqs. 13, 2) and R_C (Eq. 7)."""
        for c in self._postorder():
            if c == 0:
                continue
            C = self.tree[c]
            if C.children:
                c1, c2 = C.children
                nodes, M, Sg = self._merge(self.B[c1], self.B[c2], self.U[c1], self.U[c2],
                                           self.R[c1], self.R[c2])
            else:
                nodes = C.nodes
                M, Sg = self._a(nodes, nodes), self._s(nodes, nodes)
            self.U[c], self.R[c] = self._eliminate_onto(nodes, M, Sg, self.B[c])

    def downward_pass(self):
        """U and R of every complement cluster Cbar (the mesh outside C,
        eliminated onto B_Cbar), parents before children (Sec. 2.2): for C
        with parent D and sibling D1 the block over B_Dbar u B_D1 comes from
        (U_Dbar, U_D1) and (R_Dbar, R_D1) with the original couplings; for the
        root's children Dbar is empty and the block is D1's own U and R."""
        for c in reversed(self._postorder()):
            if c == 0:
                continue
            d = self.tree[c].parent
            D = self.tree[d]
            d1 = D.children[1] if D.children[0] == c else D.children[0]
            if d == 0:
                nodes, M, Sg = self.B[d1], self.U[d1], self.R[d1]
            else:
                nodes, M, Sg = self._merge(self.Bbar[d], self.B[d1], self.Ubar[d], self.U[d1],
                                           self.Rbar[d], self.R[d1])
            self.Ubar[c], self.Rbar[c] = self._eliminate_onto(nodes, M, Sg, self.Bbar[c])

    # -- leaf extraction (Sec. 3.2, Eqs. 8-10)
    def leaf(self, c: int, bordered: bool):
        C = self.tree[c]
        nodes = C.nodes
        A_CC = self._a(nodes, nodes)
        S_CC = self._s(nodes, nodes)
        if c == 0:
            G_CC = np.linalg.inv(A_CC)
            Gl_CC = G_CC @ S_CC @ G_CC.conj().T
            return G_CC, Gl_CC, nodes, Gl_CC
        Bb, Ub, Rb = self.Bbar[c], self.Ubar[c], self.Rbar[c]
        A_CB, A_BC = self._a(nodes, Bb), self._a(Bb, nodes)
        S_CB, S_BC = self._s(nodes, Bb), self._s(Bb, nodes)
        Ui = np.linalg.inv(Ub)
        G_CC = np.linalg.inv(A_CC - A_CB @ Ui @ A_BC)                    # Eq. (8)
        Lp = A_CB @ Ui                                                   # Eq. (13), S = Bb
        R_nn = S_CC - Lp @ S_BC - S_CB @ Lp.conj().T + Lp @ Rb @ Lp.conj().T   # Eq. (7)
        Gl_CC = G_CC @ R_nn @ G_CC.conj().T                              # Eq. (5)
        if not bordered:
            return G_CC, Gl_CC, None, None
        G_BC = -Ui @ A_BC @ G_CC                                         # Eq. (9)
        G_CB = -G_CC @ A_CB @ Ui                                         # Eq. (10)
        G_BB = Ui - G_BC @ A_CB @ Ui                                     # block inverse
        GK = np.block([[G_BB, G_BC], [G_CB, G_CC]])
        SK = np.block([[Rb, S_BC], [S_CB, S_CC]])
        GlK = GK @ SK @ GK.conj().T
        return G_CC, Gl_CC, np.concatenate([Bb, nodes]), GlK

    def run(self, H=None, bonds=None):
        """Both passes and every leaf: returns diag G, diag G<, and optionally the bond
        entries (G<_ji, G<_ij) for bonds i -> j, taken from the leaf holding
        i, plus the same pair taken from the leaf holding j (NaN when both
        ends share a leaf)."""
        n = self.nx * self.ny
        self.upward_pass()
        self.downward_pass()
        diagG = np.zeros(n, np.complex128)
        diagGl = np.zeros(n, np.complex128)
        leaves = [k for k, c in enumerate(self.tree) if not c.children]
        want = bonds is not None
        if want:
            bi, bj = bonds
            leaf_of = np.empty(n, np.int64)
            for k in leaves:
                leaf_of[self.tree[k].nodes] = k
            li, lj = leaf_of[bi], leaf_of[bj]
            gl_ji = np.full(len(bi), np.nan + 0j)
            gl_ij = np.full(len(bi), np.nan + 0j)
            alt_ji = np.full(len(bi), np.nan + 0j)
            alt_ij = np.full(len(bi), np.nan + 0j)
            pos = np.full(n, -1, np.int64)
        for k in leaves:
            nodes = self.tree[k].nodes
            G_CC, Gl_CC, knodes, GlK = self.leaf(k, want)
            diagG[nodes] = np.diag(G_CC)
            diagGl[nodes] = np.diag(Gl_CC)
            if want:
                pos[knodes] = np.arange(len(knodes))
                sel = np.nonzero(li == k)[0]
                pi, pj = pos[bi[sel]], pos[bj[sel]]
                gl_ji[sel] = GlK[pj, pi]
                gl_ij[sel] = GlK[pi, pj]
                sel = np.nonzero((lj == k) & (li != k))[0]
                pi, pj = pos[bi[sel]], pos[bj[sel]]
                alt_ji[sel] = GlK[pj, pi]
                alt_ij[sel] = GlK[pi, pj]
                pos[knodes] = -1
        if want:
            return diagG, diagGl, (gl_ji, gl_ij, alt_ji, alt_ij)
        return diagG, diagGl, None


def find_outputs(problem, E, fL=1.0, fR=0.0, leaf=8, tie="y", bonds=True,
                 sigL=None, sigR=None, diag_lesser=None, symmetric=False):
    """diag G, diag G< and bond currents J of a MeshProblem at energy E."""
    from .dense import bond_list, bond_current_from

    A, Sl = problem.assemble(E, fL, fR, sigL, sigR, diag_lesser)
    f = FindOracle(A, Sl, problem.nx, problem.ny, problem.pattern, leaf, tie, symmetric)
    if not bonds:
        dG, dGl, _ = f.run()
        return dG, dGl, None, f
    bi, bj = bond_list(problem.nx, problem.ny, problem.stencil)
    dG, dGl, (gji, gij, aji, aij) = f.run(bonds=(bi, bj))
    J = bond_current_from(problem.H, gji, gij, bi, bj)
    J_alt = bond_current_from(problem.H, aji, aij, bi, bj)
    return dG, dGl, (J, J_alt), f
