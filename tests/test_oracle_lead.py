"""Pins of the lead self-energy (oracle/problem.py) against independent facts.

* the defining quadratic of each mode and the retarded-root conditions;
* a Lopez-Sancho decimation of the semi-infinite lead in real space, which
  uses no transverse modes at all (it catches a wrong mode normalisation,
  a wrong tau for the 9-point stencil, or a transposed Phi);
* the 1D limit nx = 1, where Sigma is the textbook chain value.
"""

import numpy as np
import pytest

from oracle import problem


def decimation_surface_sigma(E, h, tau, tol=1e-14, maxit=200):
    """Sigma = tau g_s tau for a semi-infinite stack of slices (slice
    Hamiltonian h, inter-slice coupling tau), by renormalisation decimation."""
    n = h.shape[0]
    I = np.eye(n)
    eps_s = h.astype(np.complex128).copy()
    eps = h.astype(np.complex128).copy()
    a = tau.astype(np.complex128).copy()
    b = tau.T.astype(np.complex128).copy()
    for _ in range(maxit):
        gi = np.linalg.inv(E * I - eps)
        agb = a @ gi @ b
        bga = b @ gi @ a
        eps_s = eps_s + agb
        eps = eps + agb + bga
        a = a @ gi @ a
        b = b @ gi @ b
        if np.abs(a).max() < tol and np.abs(b).max() < tol:
            break
    gs = np.linalg.inv(E * I - eps_s)
    return tau.T @ gs @ tau


def slice_matrices(nx, t, tp, onsite0, stencil):
    h = np.diag(np.full(nx, onsite0)) - t * (np.eye(nx, k=1) + np.eye(nx, k=-1))
    tau = -t * np.eye(nx)
    if stencil == 9:
        tau = tau - tp * (np.eye(nx, k=1) + np.eye(nx, k=-1))
    return h, tau


@pytest.mark.parametrize("stencil,tp,onsite0", [(5, 0.0, 4.0), (9, 0.2, 4.8)])
@pytest.mark.parametrize("E", [0.3 + 1e-3j, 1.0 + 1e-3j, 2.7 + 1e-2j, 6.1 + 1e-3j, 9.0 + 1e-6j, -0.5 + 1e-6j])
def test_sigma_matches_real_space_decimation(stencil, tp, onsite0, E):
    nx = 7
    h, tau = slice_matrices(nx, 1.0, tp, onsite0, stencil)
    ref = decimation_surface_sigma(E, h, tau)
    got = problem.lead_self_energy(E, nx, 1.0, tp, onsite0, stencil)
    assert np.abs(got - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("stencil,tp,onsite0", [(5, 0.0, 4.0), (9, 0.2, 4.8)])
def test_mode_roots_are_retarded(stencil, tp, onsite0):
    nx = 33
    eps, tau = problem.mode_energies(nx, 1.0, tp, onsite0, stencil)
    for Er in np.linspace(-1.0, 9.0, 41):
        E = Er + 1e-6j
        s = problem.mode_self_energy(E, eps, tau)
        resid = s * s - (E - eps) * s + tau * tau
        assert np.abs(resid).max() < 1e-12 * max(1.0, np.abs(E - eps).max() ** 2)
        assert np.all(np.abs(s) < np.abs(tau) * (1 + 1e-12))
        assert np.all(s.imag <= 1e-15)


def test_one_dimensional_chain_limit():
    # nx = 1: eps = onsite0 - 2t cos(pi/2) = onsite0, tau = -t; inside the band
    # sigma = (w - i sqrt(4t^2 - w^2)) / 2 with w = E - onsite0.
    E = 4.5 + 0j
    s = problem.lead_self_energy(E + 1e-9j, 1, 1.0, 0.0, 4.0, 5)[0, 0]
    w = 0.5
    ref = 0.5 * (w - 1j * np.sqrt(4.0 - w * w))
    assert abs(s - ref) < 1e-8


def test_modes_are_orthonormal_eigenvectors():
    nx = 11
    phi, theta = problem.transverse_modes(nx)
    assert np.allclose(phi.T @ phi, np.eye(nx), atol=1e-13)
    h, _ = slice_matrices(nx, 1.0, 0.0, 4.0, 5)
    assert np.allclose(h @ phi, phi * (4.0 - 2.0 * np.cos(theta)), atol=1e-12)
