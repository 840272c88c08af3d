"""Precorrected FFT (pFFT) coupling of the near coil to the voxel grid.

Sec. II.C (extended voxel domain enclosing coil and body; each triangle pair
projected onto an expansion domain of voxels) and Sec. III (the 2 x 2 near
sub-system Z^pFFT handled as one block-Toeplitz VIE on the extended grid).  The
paper cites Phillips-White and Guryev et al. for the projection rule; the
reading taken here:

* stencil: RWG n (centre c_n = mean of its two triangle centroids) owns the
  s x s x s voxels around the voxel nearest c_n;
* projection: 3 s^3 complex voxel currents w_n whose point-dipole fields
  h^3 Gop(r - r_q) w_q reproduce the field Gop f_n of the RWG function at N_c
  collocation points on a sphere (Fibonacci lattice,
  N_c = 6 s^3) around the stencil centre, by Tikhonov-regularised least squares
  (lambda = reg * sigma_max(A)).  The sphere radius is rfac * s * h / 2 with
  rfac = 2 by default: a 3^3 stencil then reproduces the field to ~2e-3 beyond
  4 voxels and a 5^3 stencil (the paper's choice) to ~1e-6 beyond 6 voxels;
* interpolation: by reciprocity (Galerkin symmetry) the transpose P^T;
* precorrection: on near pairs (body voxel within Chebyshev distance `near` of
  the stencil centre) S = K_direct - (K_grid P), and for the coil-coil block the
  dense correction C_nn = K_nn - P^T K_grid P (exact coil-coil interaction).
Parity: the projection is pinned by its fitting residual and by the coupling
accuracy against direct (8 x 6-point) coupling (tests/test_oracle_surface.py).
"""
from __future__ import annotations

import numpy as np

from . import physics, coupling, volume


def fibonacci_sphere(N):
    k = np.arange(N)
    z = 1.0 - (2.0 * k + 1.0) / N
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = k * np.pi * (3.0 - np.sqrt(5.0))
    return np.stack([rr * np.cos(ph), rr * np.sin(ph), z], -1)


def stencil_offsets(s):
    """(s^3, 3) local voxel offsets, x fastest, centred on 0."""
    r = np.arange(s) - (s - 1) // 2
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)


def stencil_centres(ext_grid, rw, cols, s):
    """Integer index of the stencil centre voxel for each RWG in cols."""
    cols = np.asarray(cols, np.int64)
    c = 0.5 * (rw.centroid[rw.tplus[cols]] + rw.centroid[rw.tminus[cols]])
    ic = np.rint((c - np.asarray(ext_grid.origin)[None, :]) / ext_grid.h).astype(np.int64)
    half = (s - 1) // 2
    if np.any(ic - half < 0) or np.any(ic + half >= np.asarray(ext_grid.n)[None, :]):
        raise ValueError("pFFT stencil leaves the extended grid")
    return ic


RFAC = 2.0


def fit_matrix(s, h, k0, rfac=RFAC):
    """A[(a, c), (b, q)] = h^3 Gop_ab(r_c - r_q) for collocation c and stencil voxel q."""
    Nc = 6 * s ** 3
    rc = rfac * s * h / 2.0 * fibonacci_sphere(Nc)
    rq = h * stencil_offsets(s)
    D = physics.dyad(rc[:, None, :] - rq[None, :, :], k0) * h ** 3   # (Nc, s3, 3, 3)
    A = np.transpose(D, (2, 0, 3, 1)).reshape(3 * Nc, 3 * s ** 3)
    return A, rc


def projector(s, h, k0, reg, rfac=RFAC):
    """Tikhonov pseudo-inverse  V diag(sig / (sig^2 + lam^2)) U^H."""
    A, rc = fit_matrix(s, h, k0, rfac)
    U, sig, Vh = np.linalg.svd(A, full_matrices=False)
    lam = reg * sig[0]
    f = sig / (sig * sig + lam * lam)
    return (Vh.conj().T * f[None, :]) @ U.conj().T, A, rc


def projection(ext_grid, rw, cols, s, k0, reg=1e-10, rfac=RFAC):
    """P weights (len(cols), 3 s^3) ordered (b, q) and stencil base indices
    (len(cols), 3) (the lowest corner of each stencil)."""
    cols = np.asarray(cols, np.int64)
    Pi, A, rc = projector(s, ext_grid.h, k0, reg, rfac)
    ic = stencil_centres(ext_grid, rw, cols, s)
    ctr = np.asarray(ext_grid.origin)[None, :] + ext_grid.h * ic
    W = np.zeros((cols.size, 3 * s ** 3), np.complex128)
    for j, n in enumerate(cols):
        pts = ctr[j][None, :] + rc
        e = coupling.gop_rwg(rw, [n], pts, coupling.R.TRI6, k0)[:, 0, :]   # (Nc, 3)
        W[j] = Pi @ e.T.reshape(-1)
    return W, ic - (s - 1) // 2


def scatter(ext_grid, W, base, s, xn):
    """g = P x_n on the extended grid: (3 * nv_ext, p)."""
    n1, n2, n3 = ext_grid.n
    nv = ext_grid.nv
    xn = np.asarray(xn).reshape(W.shape[0], -1)
    g = np.zeros((3 * nv, xn.shape[1]), np.complex128)
    off = stencil_offsets(s) + (s - 1) // 2
    for j in range(W.shape[0]):
        ijk = base[j][None, :] + off
        vox = ijk[:, 0] + n1 * (ijk[:, 1] + n2 * ijk[:, 2])
        for b in range(3):
            g[b * nv + vox] += W[j, b * s ** 3:(b + 1) * s ** 3, None] * xn[j][None, :]
    return g


def gather(ext_grid, W, base, s, c):
    """P^T c for grid vectors c (3 * nv_ext, p); returns (len(W), p)."""
    n1, n2, n3 = ext_grid.n
    nv = ext_grid.nv
    c = np.asarray(c).reshape(3 * nv, -1)
    out = np.zeros((W.shape[0], c.shape[1]), np.complex128)
    off = stencil_offsets(s) + (s - 1) // 2
    for j in range(W.shape[0]):
        ijk = base[j][None, :] + off
        vox = ijk[:, 0] + n1 * (ijk[:, 1] + n2 * ijk[:, 2])
        for b in range(3):
            out[j] += W[j, b * s ** 3:(b + 1) * s ** 3] @ c[b * nv + vox]
    return out


def grid_times_P(ext_grid, W, base, s, k0, targets_ext, cols_local):
    """(K_grid P)[(a, target voxels), cols] by direct summation with the voxel
    kernel T (self term included).  Returns (3, len(targets), len(cols))."""
    n1, n2, _ = ext_grid.n
    t = np.asarray(targets_ext, np.int64)
    tijk = np.stack([t % n1, (t // n1) % n2, t // (n1 * n2)], -1)
    off = stencil_offsets(s) + (s - 1) // 2
    out = np.zeros((3, t.size, len(cols_local)), np.complex128)
    for k, j in enumerate(cols_local):
        qijk = base[j][None, :] + off                      # (s3, 3)
        T = physics.voxel_kernel(tijk[:, None, :] - qijk[None, :, :], ext_grid.h, k0)
        w = W[j].reshape(3, -1)                            # (b, q)
        out[:, :, k] = np.einsum("tqab,bq->at", T, w)
    return out


def near_pairs(body_grid, ext_offset, ext_ic, material, near):
    """For each RWG, the material body voxels within Chebyshev distance `near`
    of its stencil centre."""
    n1, n2, n3 = body_grid.n
    out = []
    off = np.asarray(ext_offset)
    for j in range(ext_ic.shape[0]):
        lo = np.maximum(ext_ic[j] - off - near, 0)
        hi = np.minimum(ext_ic[j] - off + near, np.asarray(body_grid.n) - 1)
        if np.any(hi < lo):
            out.append(np.zeros(0, np.int64))
            continue
        r = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        Z, Y, X = np.meshgrid(r[2], r[1], r[0], indexing="ij")
        vox = (X + n1 * (Y + n2 * Z)).ravel()
        out.append(vox[material[vox]])
    return out
