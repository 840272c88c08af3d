"""Physical constants, susceptibility and the dyadic Green's function.

Sec. II.A of the paper: equivalent currents (Eq. 1), the free-space Green's
function g = exp(-i k0 R) / (4 pi R) and the dyad built from it.  The paper
prints the dyad with an extra 1/(4 pi) in front although g already carries it;
the oracle keeps a single 1/(4 pi), inside g.

Time convention exp(+i omega t) (consistent with g and with j_b = i omega eps0
chi e_b of Eq. 1).  Conductivity enters through the complex permittivity
eps_rc = eps_r - i sigma / (omega eps0) (the paper writes chi = eps_r - 1 and
never names sigma).

The operator used everywhere in the oracle is
    Gop J (r) = k0^2 \\int g J + grad \\int g div' J  =  \\int (k0^2 I + grad grad) g J,
so that the scattered field is E = Gop J / (i omega eps0).
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C0 * C0)


def omega_k0(freq_hz: float):
    w = 2.0 * np.pi * freq_hz
    return w, w / C0


def chi(eps_r, sigma, freq_hz):
    """Complex electric susceptibility chi = eps_r - 1 - i sigma / (omega eps0)."""
    w, _ = omega_k0(freq_hz)
    return np.asarray(eps_r, np.float64) - 1.0 - 1j * np.asarray(sigma, np.float64) / (w * EPS0)


def g_scalar(R, k0):
    """g(R) = exp(-i k0 R) / (4 pi R)."""
    return np.exp(-1j * k0 * R) / (4.0 * np.pi * R)


def grad_g(Rvec, k0):
    """Gradient of g(|r - r'|) with respect to r, for Rvec = r - r' (..., 3)."""
    R = np.sqrt(np.sum(Rvec * Rvec, -1))
    g = g_scalar(R, k0)
    return (-(1.0 + 1j * k0 * R) * g / (R * R))[..., None] * Rvec


def dyad(Rvec, k0):
    """(k0^2 I + grad grad) g evaluated at R = r - r' != 0, shape (..., 3, 3).

    Written from the second derivatives of g(R):
      d_a d_b g = g/R^2 [ (3 + 3 i k R - k^2 R^2) Rh_a Rh_b - (1 + i k R) delta_ab ].
    """
    Rvec = np.asarray(Rvec, np.float64)
    R = np.sqrt(np.sum(Rvec * Rvec, -1))
    Rh = Rvec / R[..., None]
    g = g_scalar(R, k0)
    kR = k0 * R
    a = (g / (R * R)) * (kR * kR - 1.0 - 1j * kR)
    b = (g / (R * R)) * (3.0 + 3.0j * kR - kR * kR)
    eye = np.eye(3)
    return a[..., None, None] * eye + b[..., None, None] * (Rh[..., :, None] * Rh[..., None, :])


def self_term(k0, h):
    """Self term of the PWC voxel operator: the field at the centre of the
    equal-volume sphere (radius a = (3/(4 pi))^(1/3) h) carrying a unit uniform
    current, in units of 1/(i omega eps0):
        (2/3)(1 + i k0 a) exp(-i k0 a) - 1.
    The -1 is the static depolarisation -1/3 minus the 2/3 of the sphere's
    principal-value integral at k0 = 0."""
    a = (3.0 / (4.0 * np.pi)) ** (1.0 / 3.0) * h
    return (2.0 / 3.0) * (1.0 + 1j * k0 * a) * np.exp(-1j * k0 * a) - 1.0


def voxel_kernel(d_idx, h, k0):
    """T(Delta) for integer voxel offsets d_idx (..., 3): h^3 * dyad(h d) for
    d != 0 and self_term * I for d = 0.  Shape (..., 3, 3)."""
    d = np.asarray(d_idx, np.float64)
    zero = np.all(d == 0, -1)
    Rvec = h * np.where(zero[..., None], 1.0, d)  # placeholder for d = 0
    T = (h ** 3) * dyad(Rvec, k0)
    T = np.where(zero[..., None, None], self_term(k0, h) * np.eye(3), T)
    return T
