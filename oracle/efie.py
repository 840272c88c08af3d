"""Galerkin EFIE matrix of RWG functions (Eq. sie, Eq. disc_sie).

The oracle computes K_mn = <f_m, Gop f_n> with the mixed-potential form
    K_mn = k0^2 \\int\\int f_m . f_n g  -  \\int\\int (div f_m)(div' f_n) g,
and the surface blocks of the system are Z_cc = -K (so that the whole system is
Z = D - K with D the body diagonal; see oracle.hybrid).

Quadrature per triangle pair (T, T'), by centroid distance d and the longer of
the two triangle diameters D (a definition shared with the CUDA library's own,
separately written, assembly):
  * near  (T, T' share a vertex, or d < 2 D): singularity extraction - outer
    7-point rule; inner smooth part (g - 1/(4 pi R)) with the 7-point rule and
    the 1/R part with the analytic integrals of oracle.potint; the result is
    averaged with the same rule applied with T and T' swapped, which makes the
    matrix exactly symmetric (reciprocity);
  * mid   (d < 6 D): 6-point x 6-point;
  * far   (otherwise): centroid x centroid.
Pinned by: symmetry, the low-frequency loop inductance (tests).
"""
from __future__ import annotations

import numpy as np

from . import rwg as R
from . import potint

NEAR_FACTOR = 2.0
MID_FACTOR = 6.0


def _gs(Rd, k0):
    """g - 1/(4 pi R), written without cancellation; limit -i k0 / (4 pi) at R = 0."""
    out = np.empty(Rd.shape, np.complex128)
    z = Rd == 0
    Rz = np.where(z, 1.0, Rd)
    s = np.sin(0.5 * k0 * Rz)
    val = (-2.0 * s * s - 1j * np.sin(k0 * Rz)) / (4.0 * np.pi * Rz)
    out[...] = np.where(z, -1j * k0 / (4.0 * np.pi), val)
    return out


def _g(Rd, k0):
    return np.exp(-1j * k0 * Rd) / (4.0 * np.pi * Rd)


def tier(rwA, rwB, tA, tB, same_mesh):
    """0 = near (singular extraction), 1 = mid, 2 = far, for triangle pairs."""
    d = np.linalg.norm(rwA.centroid[tA] - rwB.centroid[tB], axis=-1)
    D = np.maximum(rwA.diam[tA], rwB.diam[tB])
    t = np.where(d < NEAR_FACTOR * D, 0, np.where(d < MID_FACTOR * D, 1, 2))
    if same_mesh:
        va = rwA.tri[tA]
        vb = rwB.tri[tB]
        share = (va[..., :, None] == vb[..., None, :]).any((-1, -2))
        t = np.where(share, 0, t)
    return t


def _moments_regular(rwA, rwB, tA, tB, rule, k0):
    """Moments A0 = \\int\\int g, A1 = \\int\\int (r - cA) g, B1 = \\int\\int (r' - cB) g,
    C = \\int\\int (r - cA).(r' - cB) g for triangle pairs (tA[i], tB[i])."""
    pa, wa = R.tri_points(rwA, tA, rule)
    pb, wb = R.tri_points(rwB, tB, rule)
    la = pa - rwA.centroid[tA][:, None, :]
    lb = pb - rwB.centroid[tB][:, None, :]
    Rv = pa[:, :, None, :] - pb[:, None, :, :]
    Rd = np.sqrt(np.sum(Rv * Rv, -1))
    G = _g(Rd, k0) * wa[:, :, None] * wb[:, None, :]
    A0 = G.sum((1, 2))
    A1 = np.einsum("kij,kid->kd", G, la)
    B1 = np.einsum("kij,kjd->kd", G, lb)
    C = np.einsum("kij,kid,kjd->k", G, la, lb)
    return A0, A1, B1, C


def _moments_singular_dir(rwA, rwB, tA, tB, k0):
    """One direction of the singular moments: outer 7-point rule on T (of A),
    inner 7-point rule on g - 1/(4 pi R) plus the analytic 1/R integrals on T'."""
    pa, wa = R.tri_points(rwA, tA, R.TRI7)          # (k, 7, 3), (k, 7)
    pb, wb = R.tri_points(rwB, tB, R.TRI7)
    ca, cb = rwA.centroid[tA], rwB.centroid[tB]
    Rv = pa[:, :, None, :] - pb[:, None, :, :]
    Rd = np.sqrt(np.sum(Rv * Rv, -1))
    Gs = _gs(Rd, k0) * wb[:, None, :]
    J0 = Gs.sum(2)
    J1 = np.einsum("kij,kjd->kid", Gs, pb - cb[:, None, :])
    P = rwB.xyz[rwB.tri[tB]]
    I0, I1 = potint.integrals(pa, P, rwB.normal[tB])
    J0 = J0 + I0 / (4 * np.pi)
    J1 = J1 + (I1 + (pa - cb[:, None, :]) * I0[..., None]) / (4 * np.pi)
    la = pa - ca[:, None, :]
    A0 = np.sum(wa * J0, 1)
    A1 = np.einsum("ki,kid->kd", wa * J0, la)
    B1 = np.einsum("ki,kid->kd", wa, J1)
    C = np.einsum("ki,kid,kid->k", wa, la, J1)
    return A0, A1, B1, C


def _moments_singular(rwA, rwB, tA, tB, k0):
    """Singular-pair moments, averaged over both directions so that the
    Galerkin matrix is exactly symmetric: the transposed direction swaps the
    roles of A1 and B1."""
    a0, a1, b1, c = _moments_singular_dir(rwA, rwB, tA, tB, k0)
    a0t, a1t, b1t, ct = _moments_singular_dir(rwB, rwA, tB, tA, k0)
    return 0.5 * (a0 + a0t), 0.5 * (a1 + b1t), 0.5 * (b1 + a1t), 0.5 * (c + ct)


def tri_pair_moments(rwA, rwB, tA, tB, k0, same_mesh):
    tA = np.asarray(tA, np.int64).ravel()
    tB = np.asarray(tB, np.int64).ravel()
    tr = tier(rwA, rwB, tA, tB, same_mesh)
    A0 = np.zeros(tA.size, np.complex128)
    A1 = np.zeros((tA.size, 3), np.complex128)
    B1 = np.zeros((tA.size, 3), np.complex128)
    C = np.zeros(tA.size, np.complex128)
    for lvl, rule in ((1, R.TRI6), (2, R.TRI1)):
        s = np.nonzero(tr == lvl)[0]
        for c0 in range(0, s.size, 20000):
            ss = s[c0:c0 + 20000]
            a0, a1, b1, cc = _moments_regular(rwA, rwB, tA[ss], tB[ss], rule, k0)
            A0[ss], A1[ss], B1[ss], C[ss] = a0, a1, b1, cc
    s = np.nonzero(tr == 0)[0]
    for c0 in range(0, s.size, 20000):
        ss = s[c0:c0 + 20000]
        a0, a1, b1, cc = _moments_singular(rwA, rwB, tA[ss], tB[ss], k0)
        A0[ss], A1[ss], B1[ss], C[ss] = a0, a1, b1, cc
    return A0, A1, B1, C


def K_block(rwA, rwB, rows, cols, k0, same_mesh):
    """K[rows, cols] with K_mn = <f_m, Gop f_n> (test RWG m of rwA, basis n of rwB).
    Moments are computed once per distinct triangle pair."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    ua, inva = np.unique(np.concatenate([rwA.tplus[rows], rwA.tminus[rows]]),
                         return_inverse=True)
    ub, invb = np.unique(np.concatenate([rwB.tplus[cols], rwB.tminus[cols]]),
                         return_inverse=True)
    ta = np.repeat(ua, ub.size)
    tb = np.tile(ub, ua.size)
    A0, A1, B1, C = tri_pair_moments(rwA, rwB, ta, tb, k0, same_mesh)
    shp = (ua.size, ub.size)
    A0, C = A0.reshape(shp), C.reshape(shp)
    A1, B1 = A1.reshape(shp + (3,)), B1.reshape(shp + (3,))
    nr, nc = rows.size, cols.size
    K = np.zeros((nr, nc), np.complex128)
    halvesA = ((rwA.tplus, 1.0, rwA.vplus, inva[:nr]), (rwA.tminus, -1.0, rwA.vminus, inva[nr:]))
    halvesB = ((rwB.tplus, 1.0, rwB.vplus, invb[:nc]), (rwB.tminus, -1.0, rwB.vminus, invb[nc:]))
    for ta_arr, sa, va_arr, ia in halvesA:
        for tb_arr, sb, vb_arr, ib in halvesB:
            a0 = A0[ia][:, ib]
            c = C[ia][:, ib]
            a1 = A1[ia][:, ib]
            b1 = B1[ia][:, ib]
            va = (rwA.xyz[va_arr[rows]] - rwA.centroid[ta_arr[rows]])[:, None, :]
            vb = (rwB.xyz[vb_arr[cols]] - rwB.centroid[tb_arr[cols]])[None, :, :]
            vv = c - np.sum(vb * a1, -1) - np.sum(va * b1, -1) + np.sum(va * vb, -1) * a0
            la, lb = rwA.length[rows][:, None], rwB.length[cols][None, :]
            Aa, Ab = rwA.area[ta_arr[rows]][:, None], rwB.area[tb_arr[cols]][None, :]
            K += sa * sb * (la * lb / (4 * Aa * Ab)) * (k0 * k0 * vv - 4.0 * a0)
    return K


def K_dense(rwA, rwB, k0, same_mesh):
    return K_block(rwA, rwB, np.arange(rwA.m), np.arange(rwB.m), k0, same_mesh)
