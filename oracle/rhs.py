"""Plane-wave right-hand side of the hybrid system (Sec. II.A; Eq. (hvsie)).

Test infrastructure only (see oracle/__init__.py).

With Z = D - K and the E-field testing used throughout (K = <test, Gop basis>,
Gop J = (k0^2 + grad div) \\int g J, so that the scattered field is
E_s = Gop J / (i omega eps0), time convention exp(+i omega t)):

  * a conductor row m states <f_m, E_inc + E_s> = 0, i.e.
        (Z j)_m = i omega eps0 \\int f_m . E_inc dS
    (the delta-gap port excitation i omega eps0 V l_m is the special case of an
    impressed field V delta(edge) across the port edge);
  * a body row (voxel p, component a) states J / (i omega eps0 chi) = E_inc + E_s
    tested over the voxel, i.e. (Z j)_{p,a} = i omega eps0 h^3 E_inc,a(r_p) on
    material voxels and 0 on vacuum voxels (identity rows, zero input).

E_inc(r) = e0 exp(-i k0 k_hat . r) with real polarisation e0 orthogonal to
k_hat.  The surface integrals use the 6-point Dunavant rule on each triangle
(degree 4; E_inc varies on the scale of a wavelength, the triangles on the
scale of a centimetre).

Pinned by (tests/test_oracle_rhs.py): the uniform-field limit, where the
integral of an RWG function has the closed form (l/2)[(c+ - v+) - (c- - v-)];
a 64-times-refined quadrature of the same integrals at 298 MHz; and the body
part of the Mie check (oracle.mie.body_rhs) for k_hat = z, e0 = x.
"""
from __future__ import annotations

import numpy as np

from . import physics
from . import rwg as R
from . import volume


def incident(points, k_hat, e0, k0):
    """E_inc at the points (P x 3): e0 exp(-i k0 k_hat . r)."""
    P = np.asarray(points, np.float64)
    kh = np.asarray(k_hat, np.float64)
    kh = kh / np.linalg.norm(kh)
    ph = np.exp(-1j * k0 * (P @ kh))
    return ph[:, None] * np.asarray(e0, np.float64)[None, :]


def tested_incident(rw, k_hat, e0, k0, rule=R.TRI6):
    """\\int f_m . E_inc dS for every RWG m of rw (length m)."""
    out = np.zeros(rw.m, np.complex128)
    for t_arr, s, v_arr in ((rw.tplus, 1.0, rw.vplus), (rw.tminus, -1.0, rw.vminus)):
        q, wq = R.tri_points(rw, t_arr, rule)            # (m, Q, 3), weights x area
        E = incident(q.reshape(-1, 3), k_hat, e0, k0).reshape(q.shape)
        f = (s * rw.length / (2 * rw.area[t_arr]))[:, None, None] * (q - rw.xyz[v_arr][:, None, :])
        out += np.einsum("mq,mqd,mqd->m", wq, f, E)
    return out


def planewave(prob, k_hat, e0):
    """The full right-hand side [v_f; v_n; v_b] (length N) of a Problem."""
    omega, k0 = physics.omega_k0(prob.freq_hz)
    s = 1j * omega * physics.EPS0
    parts = []
    if prob.shield is not None:
        parts.append(s * tested_incident(R.build(prob.shield), k_hat, e0, k0))
    if prob.coil is not None:
        parts.append(s * tested_incident(R.build(prob.coil), k_hat, e0, k0))
    g = prob.grid
    chi = physics.chi(prob.eps_r, prob.sigma, prob.freq_hz)
    E = incident(g.centres(), k_hat, e0, k0) * (s * g.h ** 3)
    E[~volume.material_mask(chi)] = 0
    parts.append(E.T.reshape(-1))
    return np.concatenate(parts)
