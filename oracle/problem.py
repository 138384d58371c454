"""Problem assembly for the FIND oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path; the two meet only in ``workloads.py`` (seeded
random inputs, no arithmetic of the method).

Plain float64/complex128 numpy + scipy.sparse, written for clarity.

What is assembled (Sec. 1 of the paper, the NEGF definitions):
    A   = (E + i eta) I - H - Sigma_L - Sigma_R        (E carries eta)
    G   = A^{-1}
    G<  = G Sigma< G^dagger,  Sigma< = i (f_L Gamma_L + f_R Gamma_R) [+ diag]
    Gamma = i (Sigma - Sigma^dagger)

Readings the paper leaves open (it takes Sigma as given):
  * H is the finite-difference stencil: onsite0 + V_n on the diagonal, -t to
    the 4 nearest neighbours, -t' to the 4 diagonal neighbours (9-point).
  * node n = y * nx + x; the leads attach to the columns y = 0 and
    y = ny - 1, each a semi-infinite continuation of the clean stencil
    (V = 0 in the leads, same t, t').
  * Sigma of a lead is the sine-mode closed form Phi diag(sigma_m) Phi^T,
    where sigma_m is the retarded root of
        sigma^2 - (E - eps_m) sigma + tau_m^2 = 0,   |sigma_m| < |tau_m|,
    eps_m = onsite0 - 2 t cos(theta_m), tau_m = -t - 2 t' cos(theta_m),
    theta_m = m pi / (nx + 1).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------- lead modes

def transverse_modes(nx: int):
    """Orthonormal sine modes of an nx-site chain with hard walls.

    Returns (phi, theta) with phi[x, m-1] = sqrt(2/(nx+1)) sin(m pi (x+1)/(nx+1))
    and theta[m-1] = m pi / (nx+1), m = 1..nx.
    """
    x = np.arange(nx, dtype=np.float64)
    m = np.arange(1, nx + 1, dtype=np.float64)
    theta = m * np.pi / (nx + 1)
    phi = np.sqrt(2.0 / (nx + 1)) * np.sin(np.outer(x + 1.0, m) * np.pi / (nx + 1))
    return phi, theta


def mode_energies(nx: int, t: float, tp: float, onsite0: float, stencil: int):
    """Per-mode onsite eps_m and inter-slice hopping tau_m of the lead."""
    _, theta = transverse_modes(nx)
    eps = onsite0 - 2.0 * t * np.cos(theta)
    if stencil == 9:
        tau = -t - 2.0 * tp * np.cos(theta)
    else:
        tau = np.full(nx, -t, dtype=np.float64)
    return eps, tau


def mode_self_energy(E: complex, eps: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Retarded surface self-energy of each mode chain.

    sigma solves sigma^2 - (E - eps) sigma + tau^2 = 0; the two roots multiply
    to tau^2, and the decaying (retarded, Im E > 0) root is the one with
    |sigma| < |tau|.
    """
    w = np.asarray(E, dtype=np.complex128) - eps
    d = np.sqrt(w * w - 4.0 * tau * tau + 0j)
    r1 = 0.5 * (w + d)
    r2 = 0.5 * (w - d)
    return np.where(np.abs(r1) < np.abs(r2), r1, r2)


def lead_self_energy(E: complex, nx: int, t: float, tp: float, onsite0: float,
                     stencil: int) -> np.ndarray:
    """Dense nx x nx retarded self-energy of one semi-infinite lead."""
    phi, _ = transverse_modes(nx)
    eps, tau = mode_energies(nx, t, tp, onsite0, stencil)
    sig = mode_self_energy(E, eps, tau)
    return (phi * sig[None, :]) @ phi.T


# ---------------------------------------------------------------- the mesh

def stencil_offsets(stencil: int):
    """Neighbour offsets (dx, dy, kind); kind 0 = nearest (-t), 1 = diagonal (-t')."""
    offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
    if stencil == 9:
        offs += [(1, 1, 1), (-1, -1, 1), (1, -1, 1), (-1, 1, 1)]
    return offs


def hamiltonian(nx: int, ny: int, stencil: int, t: float, tp: float,
                onsite0: float, V: np.ndarray) -> sp.csr_matrix:
    """Real symmetric tight-binding H of the device (no leads)."""
    n = nx * ny
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny))
    xs = xs.reshape(-1)
    ys = ys.reshape(-1)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [onsite0 + np.asarray(V, dtype=np.float64).reshape(-1)]
    for dx, dy, kind in stencil_offsets(stencil):
        x2 = xs + dx
        y2 = ys + dy
        ok = (x2 >= 0) & (x2 < nx) & (y2 >= 0) & (y2 < ny)
        rows.append((ys * nx + xs)[ok])
        cols.append((y2 * nx + x2)[ok])
        vals.append(np.full(int(ok.sum()), -(t if kind == 0 else tp)))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def contact_nodes(nx: int, ny: int):
    """Node indices of the left (y = 0) and right (y = ny - 1) contact columns."""
    left = np.arange(nx)
    right = (ny - 1) * nx + np.arange(nx)
    return left, right


def embed(n: int, nodes: np.ndarray, block: np.ndarray) -> sp.csr_matrix:
    """n x n sparse matrix holding the dense block on rows/cols ``nodes``."""
    k = len(nodes)
    r = np.repeat(nodes, k)
    c = np.tile(nodes, k)
    return sp.csr_matrix((np.asarray(block).reshape(-1), (r, c)), shape=(n, n))


def system_matrix(E: complex, H: sp.csr_matrix, sigL: np.ndarray, sigR: np.ndarray,
                  nx: int, ny: int) -> sp.csr_matrix:
    """A = E I - H - Sigma_L - Sigma_R (E complex, eta included)."""
    n = nx * ny
    left, right = contact_nodes(nx, ny)
    A = sp.identity(n, dtype=np.complex128, format="csr") * complex(E) - H.astype(np.complex128)
    A = A - embed(n, left, sigL) - embed(n, right, sigR)
    return A.tocsr()


def broadening(sig: np.ndarray) -> np.ndarray:
    """Gamma = i (Sigma - Sigma^dagger)."""
    return 1j * (sig - sig.conj().T)


def sigma_lesser(sigL: np.ndarray, sigR: np.ndarray, fL: float, fR: float,
                 nx: int, ny: int, diag=None) -> sp.csr_matrix:
    """Sigma< = i (f_L Gamma_L + f_R Gamma_R) on the contact columns, plus an
    optional node-diagonal part ``diag`` (length nx*ny, complex)."""
    n = nx * ny
    left, right = contact_nodes(nx, ny)
    S = embed(n, left, 1j * fL * broadening(sigL)) + embed(n, right, 1j * fR * broadening(sigR))
    if diag is not None:
        S = S + sp.diags(np.asarray(diag, dtype=np.complex128), format="csr")
    return S.tocsr()


def find_pattern(nx: int, ny: int, stencil: int) -> sp.csr_matrix:
    """Structural nonzero graph of A (off-diagonal): stencil bonds plus the
    dense coupling of every pair of nodes inside each contact column."""
    H = hamiltonian(nx, ny, stencil, 1.0, 1.0, 0.0, np.zeros(nx * ny))
    n = nx * ny
    left, right = contact_nodes(nx, ny)
    ones = np.ones((nx, nx))
    P = (abs(H) + embed(n, left, ones) + embed(n, right, ones)).tocsr()
    P.setdiag(0)
    P.eliminate_zeros()
    P.data[:] = 1.0
    return P


class MeshProblem:
    """The assembled problem of one mesh at one energy (oracle side)."""

    def __init__(self, nx, ny, stencil, t, tp, onsite0, V):
        if ny < 2:
            raise ValueError("need ny >= 2: the two contact columns must differ")
        self.nx, self.ny, self.stencil = nx, ny, stencil
        self.t, self.tp, self.onsite0 = t, tp, onsite0
        self.V = np.asarray(V, dtype=np.float64).reshape(-1)
        self.H = hamiltonian(nx, ny, stencil, t, tp, onsite0, self.V)
        self.pattern = find_pattern(nx, ny, stencil)

    @classmethod
    def from_mesh(cls, mesh, V=None):
        return cls(mesh.nx, mesh.ny, mesh.stencil, mesh.t, mesh.tp, mesh.onsite0,
                   mesh.potential() if V is None else V)

    def lead_sigmas(self, E):
        s = lead_self_energy(E, self.nx, self.t, self.tp, self.onsite0, self.stencil)
        return s, s.copy()

    def assemble(self, E, fL=1.0, fR=0.0, sigL=None, sigR=None, diag_lesser=None):
        """Return (A, Sigma<) as sparse complex matrices."""
        if sigL is None or sigR is None:
            dl, dr = self.lead_sigmas(E)
            sigL = dl if sigL is None else sigL
            sigR = dr if sigR is None else sigR
        A = system_matrix(E, self.H, sigL, sigR, self.nx, self.ny)
        S = sigma_lesser(sigL, sigR, fL, fR, self.nx, self.ny, diag_lesser)
        return A, S
