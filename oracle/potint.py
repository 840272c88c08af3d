"""Analytic potential integrals over a flat triangle, for singularity extraction.

For a triangle T' with unit normal n and an observation point r:
    I0(r) = \\int_T' 1 / |r - r'| dS',
    I1(r) = \\int_T' (r' - r) / |r - r'| dS'.
Closed forms after Wilton et al. (IEEE TAP 1984) and Graglia (IEEE TAP 1993),
re-derived here: with d = n . (r - r1) and rho the projection of r on the plane,
for every edge (a -> b, counter-clockwise about n) with unit direction l and
outward in-plane normal u = l x n,
    s+ = (b - rho) . l,  s- = (a - rho) . l,  t = (a - rho) . u,
    R0^2 = t^2 + d^2,    R+- = |b|a - r|,     f = ln((R+ + s+) / (R- + s-)),
    I0  = sum t f - |d| sum [atan(t s+ / (R0^2 + |d| R+)) - atan(t s- / (R0^2 + |d| R-))],
    I1  = (1/2) sum u (R0^2 f + s+ R+ - s- R-)  -  d n I0.
Pinned against brute-force adaptive quadrature (tests/test_oracle_surface.py).
"""
from __future__ import annotations

import numpy as np


def integrals(r, P, n):
    """r: (..., q, 3) observation points; P: (..., 3, 3) triangle vertices (rows);
    n: (..., 3) unit normal consistent with the vertex order.  Batched over the
    leading dimensions.  Returns I0 (..., q) and I1 (..., q, 3)."""
    r = np.asarray(r, np.float64)
    P = np.asarray(P, np.float64)
    n = np.asarray(n, np.float64)
    if P.ndim == 2:
        r = np.atleast_2d(r)
        I0, I1 = integrals(r[None], P[None], n[None])
        return I0[0], I1[0]
    nn = n[..., None, :]
    d = np.sum((r - P[..., None, 0, :]) * nn, -1)
    rho = r - d[..., None] * nn
    ad = np.abs(d)
    I0 = np.zeros(d.shape)
    Iv = np.zeros(r.shape)
    for k in range(3):
        a = P[..., None, k, :]
        b = P[..., None, (k + 1) % 3, :]
        L = b - a
        l = L / np.linalg.norm(L, axis=-1, keepdims=True)
        u = np.cross(l, nn)
        sp = np.sum((b - rho) * l, -1)
        sm = np.sum((a - rho) * l, -1)
        t = np.sum((a - rho) * u, -1)
        R0sq = t * t + d * d
        Rp = np.linalg.norm(b - r, axis=-1)
        Rm = np.linalg.norm(a - r, axis=-1)
        # ln((R+ + s+)/(R- + s-)); for a point that projects behind the edge
        # start (s+ + s- < 0) use the equal ratio (R- - s-)/(R+ - s+), which
        # avoids the cancellation in R- + s-.
        fwd = sp + sm >= 0
        f = np.where(fwd,
                     np.log(np.maximum(Rp + sp, 1e-300) / np.maximum(Rm + sm, 1e-300)),
                     np.log(np.maximum(Rm - sm, 1e-300) / np.maximum(Rp - sp, 1e-300)))
        I0 += t * f
        I0 -= ad * (np.arctan2(t * sp, R0sq + ad * Rp) - np.arctan2(t * sm, R0sq + ad * Rm))
        Iv += 0.5 * (R0sq * f + sp * Rp - sm * Rm)[..., None] * u
    I1 = Iv - (d * I0)[..., None] * nn
    return I0, I1
