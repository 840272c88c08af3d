"""Mie series for the field inside a homogeneous sphere under a plane wave.

Solver-level pin of the body operator (Sec. II.A, Eq. vie): a homogeneous
lossy sphere in vacuum, illuminated by E_inc = x_hat exp(-i k0 z) (time
convention exp(+i omega t), as everywhere in this package), has the interior
field of the classical Lorenz-Mie solution.  The expansion follows Bohren and
Huffman, "Absorption and Scattering of Light by Small Particles" (1983),
Sec. 4.4: internal coefficients c_n, d_n and the vector spherical harmonics
M_o1n, N_e1n with spherical Bessel radial functions j_n(m k0 r), written in
their exp(-i omega t) convention and conjugated at the end (a real incident
amplitude makes the exp(+i omega t) phasor the complex conjugate).

Pinned by: the m -> 1 limit (the expansion must return the incident plane
wave) and the quasi-static limit 3 / (eps_c + 2) (tests/test_oracle_mie.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn

from . import physics


def _n_max(x):
    # Wiscombe's truncation with a margin for the interior series
    return int(np.ceil(abs(x) + 4.0 * abs(x) ** (1.0 / 3.0) + 2.0)) + 4


def _psi(n, z):
    """Riccati-Bessel psi_n(z) = z j_n(z) and its derivative (complex z)."""
    jn = spherical_jn(n, z)
    djn = spherical_jn(n, z, derivative=True)
    return z * jn, jn + z * djn


def _xi(n, x):
    """x h_n^(1)(x) and its derivative (real x)."""
    h = spherical_jn(n, x) + 1j * spherical_yn(n, x)
    dh = spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True)
    return x * h, h + x * dh


def interior_coefficients(x, m, n_max=None):
    """c_n, d_n (n = 1..n_max) of the internal field for size parameter x = k0 a
    and relative refractive index m (Bohren-Huffman convention, mu = mu1 = 1)."""
    n_max = n_max or _n_max(m * x)
    n = np.arange(1, n_max + 1)
    jx = spherical_jn(n, x)
    hx = jx + 1j * spherical_yn(n, x)
    psi_x, dpsi_x = _psi(n, x)
    xi_x, dxi_x = _xi(n, x)
    jmx = spherical_jn(n, m * x)
    psi_mx, dpsi_mx = _psi(n, m * x)
    # c_n = [j_n(x) xi'(x) - h_n(x) psi'(x)] / [j_n(mx) xi'(x) - h_n(x) (mx j_n(mx))']
    c = (jx * dxi_x - hx * dpsi_x) / (jmx * dxi_x - hx * dpsi_mx)
    # d_n = [m j_n(x) xi'(x) - m h_n(x) psi'(x)] / [m^2 j_n(mx) xi'(x) - h_n(x) (mx j_n(mx))']
    d = (m * jx * dxi_x - m * hx * dpsi_x) / (m * m * jmx * dxi_x - hx * dpsi_mx)
    return c, d


def _pi_tau(n_max, mu):
    """Angular functions pi_n = P_n^1 / sin(theta), tau_n = d P_n^1 / d theta."""
    pi = np.zeros((n_max + 1,) + mu.shape)
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, n_max + 1):
        pi[n] = (2 * n - 1) / (n - 1) * mu * pi[n - 1] - n / (n - 1) * pi[n - 2]
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi, tau


def interior_field(points, radius, eps_r, sigma, freq_hz, n_max=None):
    """Total electric field (V/m, unit incident amplitude) at interior points
    (P x 3, metres, sphere centred at the origin) for E_inc = x_hat exp(-i k0 z).
    Returns P x 3 complex Cartesian components (exp(+i omega t) phasors)."""
    omega, k0 = physics.omega_k0(freq_hz)
    eps_bh = eps_r + 1j * sigma / (omega * physics.EPS0)    # exp(-i omega t) form
    m = np.sqrt(eps_bh)
    x = k0 * radius
    c, d = interior_coefficients(x, m, n_max)
    nm = c.size
    P = np.asarray(points, float)
    r = np.linalg.norm(P, axis=1)
    r = np.where(r == 0, 1e-30, r)
    theta = np.arccos(np.clip(P[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(P[:, 1], P[:, 0])
    mu = np.cos(theta)
    st = np.sin(theta)
    pi, tau = _pi_tau(nm, mu)
    rho = m * k0 * r
    Er = np.zeros(r.shape, complex)
    Et = np.zeros(r.shape, complex)
    Ep = np.zeros(r.shape, complex)
    cphi, sphi = np.cos(phi), np.sin(phi)
    for n in range(1, nm + 1):
        En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
        zn = spherical_jn(n, rho)
        dz = (zn + rho * spherical_jn(n, rho, derivative=True)) / rho     # (rho z_n)' / rho
        # M_o1n and N_e1n with radial function j_n(rho)
        M_t = cphi * pi[n] * zn
        M_p = -sphi * tau[n] * zn
        N_r = cphi * n * (n + 1) * st * pi[n] * zn / rho
        N_t = cphi * tau[n] * dz
        N_p = -sphi * pi[n] * dz
        cn, dn = c[n - 1], d[n - 1]
        Er += En * (-1j * dn * N_r)
        Et += En * (cn * M_t - 1j * dn * N_t)
        Ep += En * (cn * M_p - 1j * dn * N_p)
    # spherical -> Cartesian
    ct = mu
    Ex = Er * st * cphi + Et * ct * cphi - Ep * sphi
    Ey = Er * st * sphi + Et * ct * sphi + Ep * cphi
    Ez = Er * ct - Et * st
    return np.conj(np.stack([Ex, Ey, Ez], -1))


def plane_wave(points, freq_hz):
    """E_inc = x_hat exp(-i k0 z) at the points (P x 3)."""
    _, k0 = physics.omega_k0(freq_hz)
    P = np.asarray(points, float)
    E = np.zeros((P.shape[0], 3), complex)
    E[:, 0] = np.exp(-1j * k0 * P[:, 2])
    return E


def body_rhs(grid, eps_r, sigma, freq_hz):
    """Right-hand side of the body equations for the plane wave:
    i omega eps0 h^3 E_inc at material voxels (component-major), zero elsewhere."""
    omega, _ = physics.omega_k0(freq_hz)
    chi = physics.chi(eps_r, sigma, freq_hz)
    E = plane_wave(grid.centres(), freq_hz)
    b = (1j * omega * physics.EPS0 * grid.h ** 3) * E
    b[chi == 0] = 0
    return b.T.reshape(-1)


def body_field(x, eps_r, sigma, freq_hz):
    """Electric field E = j / (i omega eps0 chi) from the body unknowns
    (component-major), nv x 3; zero at vacuum voxels."""
    omega, _ = physics.omega_k0(freq_hz)
    chi = physics.chi(eps_r, sigma, freq_hz)
    nv = chi.size
    J = np.asarray(x).reshape(3, nv).T
    E = np.zeros_like(J)
    m = chi != 0
    E[m] = J[m] / (1j * omega * physics.EPS0 * chi[m][:, None])
    return E
