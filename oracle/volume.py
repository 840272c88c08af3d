"""Body operator Z_bb for piecewise-constant (PWC, q = 3) voxel currents.

Sec. II.B: the discretised current-based VIE (Eq. vie, Eq. disc_vie) on a uniform
voxel grid, whose matrix is multilevel block-Toeplitz so that only generating
columns are assembled and products go through the FFT.

Reading of the paper (its Z_bb discretisation is delegated to MARIE): with the
Galerkin PWC basis and the E-field-tested, unscaled form the body block is
    Z_bb[(p,a),(q,b)] = h^3 [ delta_pq delta_ab / chi_p  -  T_ab(p - q) ],
    T(Delta) = h^3 (k0^2 I + grad grad) g (h Delta)   for Delta != 0,
    T(0)     = self_term(k0, h) I                      (equal-volume sphere),
on voxels that hold material (chi != 0).  Vacuum voxels carry identity rows and
columns (their unknown is zero).  This form is complex-symmetric.

Vector layout: component-major, x[a * nv + voxel], voxel = i1 + n1 (i2 + n2 i3).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import physics

# the 6 unique components of the symmetric 3x3 kernel
PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def material_mask(chi):
    return np.asarray(chi) != 0


def dense_Zbb(grid, chi, k0):
    """Dense Z_bb restricted to material voxels, by brute force over all voxel
    pairs with the closed-form dyad (no Toeplitz structure used).

    Returns (Z, idx) where idx are the material voxel indices and Z has the
    unknown order (a, material voxel).  Pinned by: symmetry, Clausius-Mossotti
    limit, Mie series (tests/test_oracle_volume.py)."""
    chi = np.asarray(chi)
    idx = np.nonzero(material_mask(chi))[0]
    n1, n2, n3 = grid.n
    i1 = idx % n1
    i2 = (idx // n1) % n2
    i3 = idx // (n1 * n2)
    ijk = np.stack([i1, i2, i3], -1)
    d = ijk[:, None, :] - ijk[None, :, :]
    T = physics.voxel_kernel(d, grid.h, k0)          # (m, m, 3, 3)
    m = idx.size
    h3 = grid.h ** 3
    Z = np.zeros((3 * m, 3 * m), np.complex128)
    for a in range(3):
        for b in range(3):
            blk = -h3 * T[:, :, a, b]
            if a == b:
                blk = blk + np.diag(h3 / chi[idx])
            Z[a * m:(a + 1) * m, b * m:(b + 1) * m] = blk
    return Z, idx


def dense_matvec(grid, chi, k0, x):
    """y = Z_bb x with the dense brute-force matrix (vacuum rows: identity)."""
    Z, idx = dense_Zbb(grid, chi, k0)
    nv = grid.nv
    x = np.asarray(x, np.complex128).reshape(3 * nv, -1)
    y = x.copy()
    m = idx.size
    sel = np.concatenate([a * nv + idx for a in range(3)])
    y[sel] = Z @ x[sel]
    return y


def embedded_kernel(n, h, k0, L=None):
    """Circulant embedding of the generating columns of the Toeplitz blocks.

    For each axis, position k in [0, L) holds offset k (k < n), offset k - L
    (k > L - n) and zero otherwise (for L = 2n only k = n is zero).  Returns the
    6 unique components, shape (6, L1, L2, L3), evaluated directly at every
    (positive and negative) offset."""
    n = tuple(int(v) for v in n)
    L = tuple(2 * v for v in n) if L is None else tuple(int(v) for v in L)
    offs = []
    valid = []
    for ni, Li in zip(n, L):
        k = np.arange(Li)
        d = np.where(k < ni, k, k - Li)
        ok = (k < ni) | (k > Li - ni)
        offs.append(d)
        valid.append(ok)
    D = np.stack(np.meshgrid(*offs, indexing="ij"), -1)
    V = valid[0][:, None, None] & valid[1][None, :, None] & valid[2][None, None, :]
    T = physics.voxel_kernel(D, h, k0)
    out = np.zeros((6,) + L, np.complex128)
    for c, (a, b) in enumerate(PAIRS):
        out[c] = np.where(V, T[..., a, b], 0.0)
    return out


def kernel_spectra(n, h, k0, L=None):
    """FFT of the embedded kernel: (6, L1, L2, L3)."""
    return sfft.fftn(embedded_kernel(n, h, k0, L), axes=(1, 2, 3))


def conv(spec, n, x):
    """c_a = sum_b T_ab * x_b (aperiodic 3D convolution over the grid) via the
    circulant embedding: zero-pad, FFT, multiply by the symmetric 3x3 spectra,
    inverse FFT, truncate.  x: (3 * nv, p) component-major; returns same shape."""
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    L = spec.shape[1:]
    x = np.asarray(x, np.complex128).reshape(3 * nv, -1)
    p = x.shape[1]
    y = np.zeros((3 * nv, p), np.complex128)
    comp = {}
    for c, (a, b) in enumerate(PAIRS):
        comp[(a, b)] = c
        comp[(b, a)] = c
    for j in range(p):
        xh = []
        for b in range(3):
            xb = x[b * nv:(b + 1) * nv, j].reshape((n1, n2, n3), order="F")
            xh.append(sfft.fftn(xb, s=L))
        for a in range(3):
            acc = sum(spec[comp[(a, b)]] * xh[b] for b in range(3))
            ya = sfft.ifftn(acc)[:n1, :n2, :n3]
            y[a * nv:(a + 1) * nv, j] = ya.reshape(-1, order="F")
    return y


def fft_matvec(grid, chi, k0, x, spec=None):
    """y = Z_bb x through the FFT convolution (vacuum rows: identity)."""
    nv = grid.nv
    chi = np.asarray(chi)
    M = material_mask(chi)
    M3 = np.tile(M, 3)
    x = np.asarray(x, np.complex128).reshape(3 * nv, -1)
    if spec is None:
        spec = kernel_spectra(grid.n, grid.h, k0)
    xm = np.where(M3[:, None], x, 0.0)
    c = conv(spec, grid.n, xm)
    h3 = grid.h ** 3
    invchi = np.zeros(nv, np.complex128)
    invchi[M] = 1.0 / chi[M]
    d = np.tile(invchi, 3)[:, None]
    y = np.where(M3[:, None], h3 * (d * x - c), x)
    return y


def rows_matvec(grid, chi, k0, x, rows, chunk=1 << 20):
    """Selected rows of y = Z_bb x by direct summation over every material
    voxel (the definition, no FFT): for row r = a * nv + p,
        y_r = h^3 x_r / chi_p - h^3 sum_{q, b} T_ab(p - q) x_{b, q}   (p material),
        y_r = x_r                                                    (p vacuum).
    Used where the FFT oracle does not fit the host (grids of ~10^7 voxels).
    x: (3 nv, k); returns (len(rows), k).  Pinned by dense_matvec
    (tests/test_oracle_volume.py)."""
    chi = np.asarray(chi)
    nv = grid.nv
    n1, n2, _ = grid.n
    x = np.asarray(x, np.complex128).reshape(3 * nv, -1)
    M = material_mask(chi)
    idx = np.nonzero(M)[0]
    qi = np.stack([idx % n1, (idx // n1) % n2, idx // (n1 * n2)], -1)
    xs = [x[b * nv + idx] for b in range(3)]          # (m, k) per component
    h3 = grid.h ** 3
    out = np.zeros((len(rows), x.shape[1]), np.complex128)
    for i, r in enumerate(rows):
        a, p = divmod(int(r), nv)
        if not M[p]:
            out[i] = x[r]
            continue
        pi = np.array([p % n1, (p // n1) % n2, p // (n1 * n2)])
        acc = np.zeros(x.shape[1], np.complex128)
        for c0 in range(0, idx.size, chunk):
            sl = slice(c0, c0 + chunk)
            T = physics.voxel_kernel(pi[None, :] - qi[sl], grid.h, k0)     # (c, 3, 3)
            for b in range(3):
                acc += T[:, a, b] @ xs[b][sl]
        out[i] = h3 * (x[r] / chi[p] - acc)
    return out
