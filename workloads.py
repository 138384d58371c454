"""Seeded synthetic workloads for the FIND selected-inversion path.

This module is shared by the CPU oracle (``oracle/``) and the CUDA path
(``paper_1104_0623_gb300``).  It only draws random numbers and lays out
energy grids and mesh descriptions; it holds none of the method's
arithmetic (no Hamiltonian, no self-energy, no elimination).

The paper benchmarks on synthetic 2D Cartesian meshes (Sec. 1, Sec. 5);
the workloads below restate those meshes with seeded disorder:

* ``c1``  16x16, 5-point, V ~ U[-0.5, 0.5], one energy 1.0 + 1e-6 i
* ``c2``  40x40, 5-point, 64 energies in [0.2, 3.8] + 1e-6 i
* ``c3``  nine meshes Nx in {64, 96, 128} x Ny in {128, 256, 512}, 32 energies
* ``c4``  serving stream: Poisson arrivals, Nx ~ U{32..256}, Ny ~ U{32..1024}
* ``c5``  256x1024, 9-point (t' = 0.2 t), V ~ U[-1, 1], 512 energies in
          [0.1, 7.9] + 1e-6 i

Potentials are laid out in node order n = y * Nx + x (x transverse,
y transport).  Config k draws its potential from seed 1104 + k.
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

ETA = 1e-6


@dataclasses.dataclass(frozen=True)
class Mesh:
    """One device: mesh size, stencil, hoppings and the disorder draw."""

    nx: int
    ny: int
    stencil: int = 5
    t: float = 1.0
    tp: float = 0.0
    v_lo: float = -0.5
    v_hi: float = 0.5
    seed: int = 1105

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def onsite0(self) -> float:
        """Clean onsite energy: 4t (5-point) or 4t + 4t' (9-point)."""
        return 4.0 * self.t + (4.0 * self.tp if self.stencil == 9 else 0.0)

    def potential(self) -> np.ndarray:
        """Disorder V_n, float64, length nx*ny in node order y*nx + x."""
        rng = np.random.default_rng(self.seed)
        return rng.uniform(self.v_lo, self.v_hi, size=(self.ny, self.nx)).reshape(-1)

    def clean(self) -> "Mesh":
        """The same mesh with V = 0 (used by the clean-wire closed form)."""
        return dataclasses.replace(self, v_lo=0.0, v_hi=0.0)


def energy_grid(lo: float, hi: float, count: int, eta: float = ETA) -> np.ndarray:
    """Inclusive uniform grid lo..hi with a fixed positive imaginary part."""
    if count == 1:
        return np.array([complex(lo, eta)])
    return np.linspace(lo, hi, count) + 1j * eta


def c1() -> Mesh:
    return Mesh(16, 16, 5, 1.0, 0.0, -0.5, 0.5, 1105)


def c1_energies() -> np.ndarray:
    return np.array([1.0 + 1j * ETA])


def c2() -> Mesh:
    return Mesh(40, 40, 5, 1.0, 0.0, -0.5, 0.5, 1106)


def c2_energies() -> np.ndarray:
    return energy_grid(0.2, 3.8, 64)


def c3() -> List[Mesh]:
    out = []
    k = 0
    for nx in (64, 96, 128):
        for ny in (128, 256, 512):
            out.append(Mesh(nx, ny, 5, 1.0, 0.0, -0.5, 0.5, 1107 + k))
            k += 1
    return out


def c3_energies() -> np.ndarray:
    return energy_grid(0.2, 3.8, 32)


def c5() -> Mesh:
    return Mesh(256, 1024, 9, 1.0, 0.2, -1.0, 1.0, 1109)


def c5_energies() -> np.ndarray:
    return energy_grid(0.1, 7.9, 512)


def c5_bench_energies() -> np.ndarray:
    """The 512 c5 grid energies, then the 511 midpoints between neighbours:
    1023 distinct energies in [0.1, 7.9] + 1e-6i, so that a benchmark timing
    more than 512 energy points never repeats one."""
    g = c5_energies()
    return np.concatenate([g, 0.5 * (g[:-1] + g[1:])])


@dataclasses.dataclass(frozen=True)
class Request:
    """One serving request: a mesh and its energy grid, with an arrival time."""

    arrival_s: float
    mesh: Mesh
    energies: np.ndarray


def serving_stream(count: int, rate_hz: float, seed: int = 2011,
                   nx_range=(32, 256), ny_range=(32, 1024),
                   ne_range=(8, 128)) -> List[Request]:
    """Poisson arrivals with uniformly drawn mesh sizes and energy counts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate_hz)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        ne = int(rng.integers(ne_range[0], ne_range[1] + 1))
        mesh = Mesh(nx, ny, 5, 1.0, 0.0, -0.5, 0.5, seed * 100003 + k)
        out.append(Request(t, mesh, energy_grid(0.2, 3.8, ne)))
    return out


def random_general_system(nx: int, ny: int, stencil: int, seed: int):
    """Random complex values on the FIND sparsity pattern, NOT symmetric.

    Returns (diag, offdiag_fn seed material) as plain random arrays; the
    caller places them on its own pattern.  Used to exercise the oracle's
    elimination on a matrix that is neither symmetric nor Hermitian, so a
    transposed operand cannot hide behind A = A^T.
    """
    rng = np.random.default_rng(seed)
    n = nx * ny
    diag = rng.uniform(3.0, 5.0, n) + 1j * rng.uniform(0.5, 1.0, n)
    # one value per ordered neighbour slot (8 slots cover the 9-point stencil)
    off = rng.uniform(-1.0, 1.0, (n, 8)) + 1j * rng.uniform(-0.3, 0.3, (n, 8))
    lead = (rng.uniform(-0.5, 0.5, (2, nx, nx)) + 1j * rng.uniform(-0.5, 0.0, (2, nx, nx)))
    sig = (rng.uniform(-1.0, 1.0, (n, 9)) + 1j * rng.uniform(-1.0, 1.0, (n, 9)))
    lead_sig = (rng.uniform(-1.0, 1.0, (2, nx, nx)) + 1j * rng.uniform(-1.0, 1.0, (2, nx, nx)))
    return diag, off, lead, sig, lead_sig
