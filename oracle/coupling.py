"""Body-surface coupling matrix Z_cb (Sec. II.B, Eq. nvsie; Sec. II.C).

Entry (body voxel p, field component a; RWG n), Petrov-Galerkin:
    K[(p,a), n] = \\int_{V_p} [Gop f_n](r)_a dV,
    Gop f_n (r) = k0^2 \\int g(r, r') f_n(r') dS' + \\int (div' f_n) grad_r g(r, r') dS',
and Z_cb = -K.  Quadrature (Sec. IV.C): "near" coupling (coil <-> body, the
pFFT precorrection and the dense reference) with 8 volume points (2x2x2 Gauss)
and 6 surface points per triangle; "far" coupling (shield/bore <-> body, the
entries that the TT approximates) with 1 volume point (voxel centre) and 1
surface point (centroid).
Pinned by: Gop f_n against a finite-difference curl-curl of the vector
potential (tests/test_oracle_surface.py); the near entries against a 10^3-point
Gauss voxel rule on a refined triangle rule, whose difference falls like
(h/d)^4 with distance, the order of a product rule exact for cubics; and
reciprocity: the voxel-tested field of f_n equals the RWG-tested field of the
voxel's uniform current computed from the dyadic Green's function
(tests/test_oracle_coupling.py).  The far (1 x 1 point) entries, which the TT
approximates, are pinned against the same high-order reference: within 1e-3 at
5 voxel widths and 3e-4 beyond 10 (tests/test_oracle_coupling.py).
"""
from __future__ import annotations

import numpy as np

from . import physics
from . import rwg as R


def gop_rwg(rw, cols, pts, rule, k0):
    """[Gop f_n](r) for RWG n in cols and points pts (P, 3); returns (P, N, 3)."""
    cols = np.asarray(cols, np.int64)
    pts = np.asarray(pts, np.float64)
    out = np.zeros((pts.shape[0], cols.size, 3), np.complex128)
    for t_arr, s, v_arr in ((rw.tplus, 1.0, rw.vplus), (rw.tminus, -1.0, rw.vminus)):
        t = t_arr[cols]
        q, wq = R.tri_points(rw, t, rule)                 # (N, Q, 3), (N, Q)
        v = rw.xyz[v_arr[cols]]                           # (N, 3)
        l = rw.length[cols]
        A = rw.area[t]
        Rv = pts[:, None, None, :] - q[None, :, :, :]     # (P, N, Q, 3)
        Rd = np.sqrt(np.sum(Rv * Rv, -1))
        g = physics.g_scalar(Rd, k0) * wq[None]           # (P, N, Q)
        vec = (q - v[:, None, :])                         # (N, Q, 3)
        term1 = k0 * k0 * (s * l / (2 * A))[None, :, None] * np.einsum("pnq,nqd->pnd", g, vec)
        dg = (-(1.0 + 1j * k0 * Rd) / (Rd * Rd))[..., None] * Rv   # grad g / g
        term2 = (s * l / A)[None, :, None] * np.einsum("pnq,pnqd->pnd", g, dg)
        out += term1 + term2
    return out


def K_block(grid, voxels, rw, cols, k0, near=True, chunk=64):
    """K[(a, voxels), cols] as an array (3, len(voxels), len(cols))."""
    voxels = np.asarray(voxels, np.int64)
    cols = np.asarray(cols, np.int64)
    n1, n2, _ = grid.n
    ijk = np.stack([voxels % n1, (voxels // n1) % n2, voxels // (n1 * n2)], -1)
    cen = np.asarray(grid.origin)[None, :] + grid.h * ijk
    h3 = grid.h ** 3
    out = np.zeros((3, voxels.size, cols.size), np.complex128)
    if near:
        xi, wv = R.HEX8
        rule = R.TRI6
    else:
        xi, wv = np.zeros((1, 3)), np.ones(1)
        rule = R.TRI1
    for c0 in range(0, voxels.size, chunk):
        sl = slice(c0, c0 + chunk)
        acc = np.zeros((cen[sl].shape[0], cols.size, 3), np.complex128)
        for x, w in zip(xi, wv):
            acc += w * gop_rwg(rw, cols, cen[sl] + grid.h * x[None, :], rule, k0)
        out[:, sl, :] = h3 * np.transpose(acc, (2, 0, 1))
    return out
