"""Sampled entries of G and G< to nearly full double precision (O-refined).

TEST INFRASTRUCTURE ONLY (see ``oracle/problem.py``).

Sec. 1 of the paper defines the outputs as entries of G = A^{-1} and of
G< = G Sigma< G^dagger.  For a mesh too large for a dense inverse this module
writes those definitions out for a chosen set of nodes i:

  * row i of G solves A^T y = e_i (row i of A^{-1} is column i of A^{-T});
  * G_ii = y_i and G<_ii = sum_{k,l} y_k Sigma<_kl conj(y_l) over the
    nonzeros of Sigma<.

A is banded in the node order n = y * nx + x (bandwidth nx + 1 for the
9-point stencil, the contact blocks lie inside the band), so the solve is
LAPACK's banded LU with partial pivoting (zgbtrf / zgbtrs), a library step.
Its result carries an error of about cond(A) * eps, the same order as any
other double-precision evaluation; to get below that, each solution is
improved by classical iterative refinement (Wilkinson): the residual
r = e_i - A^T y is formed in extended precision (numpy longdouble: 64-bit
significand on x86, 113-bit on aarch64), the correction solves A^T d = r
with the same factors, and y += d is kept in extended precision.  While
cond(A) * eps_double < 1 each sweep multiplies the error by about
cond(A) * eps_double, so a few sweeps leave an error of order
cond(A) * eps_extended, far below what separates two double-precision
implementations.  The quadratic form for G< is also accumulated in extended
precision.

This module does not follow FIND: it is the plain definition, used to decide
which of two double-precision evaluations (O-find, the GPU path) is closer to
the exact value where they disagree.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import lapack

XC = np.clongdouble     # extended-precision complex used for residuals and sums


def band_widths(A) -> tuple:
    """(kl, ku): lower and upper bandwidth of the sparse matrix A."""
    C = sp.coo_matrix(A)
    d = C.row.astype(np.int64) - C.col.astype(np.int64)
    return int(max(d.max(), 0)), int(max(-d.min(), 0))


class BandedInverse:
    """Banded LU of A, kept for solves with A^T and refinement."""

    def __init__(self, A):
        C = sp.coo_matrix(A)
        n = C.shape[0]
        kl, ku = band_widths(C)
        ab = np.zeros((2 * kl + ku + 1, n), np.complex128)
        ab[kl + ku + C.row - C.col, C.col] = C.data
        lu, piv, info = lapack.zgbtrf(ab, kl, ku, overwrite_ab=True)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrf: info = {info}")
        self.n, self.kl, self.ku, self.lu, self.piv = n, kl, ku, lu, piv
        AT = sp.csr_matrix(C.T)
        AT.sort_indices()
        self.at_ptr = AT.indptr
        self.at_col = AT.indices
        self.at_val = AT.data.astype(XC)

    def _solve_t(self, b: np.ndarray) -> np.ndarray:
        x, info = lapack.zgbtrs(self.lu, self.kl, self.ku, np.asfortranarray(b), self.piv, trans=1)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrs: info = {info}")
        return x

    def residual_t(self, b: np.ndarray, y: np.ndarray) -> np.ndarray:
        """b - A^T y in extended precision (b, y of shape (n, m))."""
        prod = self.at_val[:, None] * y[self.at_col, :]
        return b.astype(XC) - np.add.reduceat(prod, self.at_ptr[:-1], axis=0)

    def rows(self, nodes, sweeps: int = 3, group: int = 8):
        """Rows `nodes` of G = A^{-1}, refined; returns (Y, history) with
        Y[:, k] = row nodes[k] of G in extended precision and history the
        max relative size of each correction."""
        nodes = np.asarray(nodes)
        Y = np.empty((self.n, len(nodes)), XC)
        hist = []
        for g0 in range(0, len(nodes), group):
            cols = nodes[g0:g0 + group]
            b = np.zeros((self.n, len(cols)), np.complex128)
            b[cols, np.arange(len(cols))] = 1.0
            y = self._solve_t(b).astype(XC)
            h = []
            for _ in range(sweeps):
                r = self.residual_t(b, y)
                d = self._solve_t(r.astype(np.complex128))
                y += d.astype(XC)
                h.append(float(np.abs(d).max() / np.abs(y).max()))
            Y[:, g0:g0 + group] = y
            hist.append(h)
        return Y, np.array(hist)


def lesser_diagonal(Y: np.ndarray, nodes, Sl) -> np.ndarray:
    """G<_ii = sum_{k,l} G_ik Sigma<_kl conj(G_il) for i in nodes, with the
    rows G_i. given as the columns of Y; summed in extended precision over
    the nonzeros of Sigma<."""
    S = sp.coo_matrix(Sl)
    val = S.data.astype(XC)
    out = np.empty(len(nodes), XC)
    for k in range(len(nodes)):
        y = Y[:, k]
        out[k] = np.sum(y[S.row] * val * np.conj(y[S.col]))
    return out


def sampled_outputs(problem, E, nodes, fL=1.0, fR=0.0, diag_lesser=None, sweeps=3):
    """diag G and diag G< at `nodes` (extended precision) and the refinement
    history, for a MeshProblem at energy E."""
    A, Sl = problem.assemble(E, fL, fR, diag_lesser=diag_lesser)
    inv = BandedInverse(A)
    Y, hist = inv.rows(nodes, sweeps=sweeps)
    nodes = np.asarray(nodes)
    G = Y[nodes, np.arange(len(nodes))]
    Gl = lesser_diagonal(Y, nodes, Sl)
    return G, Gl, hist
