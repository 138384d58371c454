"""Dense definition of the outputs (O-dense).

TEST INFRASTRUCTURE ONLY (see ``oracle/problem.py``).

Sec. 1 of the paper defines G = A^{-1} and G< = G Sigma< G^dagger; FIND
reaches these values exactly up to rounding (Theorem 1, Sec. 2.2).  This
module writes the definitions out with a dense LAPACK inverse, so it is only
usable while n = nx * ny is a few thousand.

Bond currents (Sec. 3.2 asks for the neighbour entries of G<): for every
stencil bond i -> j,
    J_{i->j} = H_ij G<_ji - G<_ij H_ji
which is real for Hermitian H and anti-Hermitian G<.  The bond list order is
fixed by ``bond_list``.
"""

from __future__ import annotations

import numpy as np


def dense_green(A) -> np.ndarray:
    """G = A^{-1} (LAPACK LU with partial pivoting)."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    return np.linalg.inv(Ad)


def dense_lesser(G: np.ndarray, Sl) -> np.ndarray:
    """G< = G Sigma< G^dagger."""
    Sd = Sl.toarray() if hasattr(Sl, "toarray") else np.asarray(Sl)
    return G @ Sd @ G.conj().T


def bond_list(nx: int, ny: int, stencil: int):
    """Ordered bonds (i, j): every bond is listed once, from i to j.

    Blocks, in this order:
      y-bonds   (x, y) -> (x, y+1)      index y*nx + x,       y < ny-1
      x-bonds   (x, y) -> (x+1, y)      index y*(nx-1) + x,   x < nx-1
      9-point only:
      d+ bonds  (x, y) -> (x+1, y+1)    index y*(nx-1) + x
      d- bonds  (x+1, y) -> (x, y+1)    index y*(nx-1) + x
    """
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny - 1))
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    src = [ys * nx + xs]
    dst = [(ys + 1) * nx + xs]
    xs, ys = np.meshgrid(np.arange(nx - 1), np.arange(ny))
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    src.append(ys * nx + xs)
    dst.append(ys * nx + xs + 1)
    if stencil == 9:
        xs, ys = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
        xs, ys = xs.reshape(-1), ys.reshape(-1)
        src.append(ys * nx + xs)
        dst.append((ys + 1) * nx + xs + 1)
        src.append(ys * nx + xs + 1)
        dst.append((ys + 1) * nx + xs)
    return np.concatenate(src), np.concatenate(dst)


def bond_current_from(H, gl_ji: np.ndarray, gl_ij: np.ndarray, i: np.ndarray,
                      j: np.ndarray) -> np.ndarray:
    """J_{i->j} = H_ij G<_ji - G<_ij H_ji, for given entries of G<."""
    Hd = H.tocsr()
    hij = np.asarray(Hd[i, j]).reshape(-1)
    hji = np.asarray(Hd[j, i]).reshape(-1)
    return hij * gl_ji - gl_ij * hji


def dense_outputs(A, Sl, H, nx, ny, stencil):
    """diag G, diag G<, and the (complex-valued) bond currents J."""
    G = dense_green(A)
    Gl = dense_lesser(G, Sl)
    i, j = bond_list(nx, ny, stencil)
    J = bond_current_from(H, Gl[j, i], Gl[i, j], i, j)
    return np.diag(G).copy(), np.diag(Gl).copy(), J, G, Gl
