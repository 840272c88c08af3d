"""Tucker (HOSVD) compression of the Green generators of the body block
(Sec. II.A: the defining columns of the block-Toeplitz Z_bb, reshaped into
n1 x n2 x n3 tensors per pair of components, compressed by the Tucker
decomposition; the hot path would decompress them on the fly).

Test infrastructure only (see oracle/__init__.py).

The generator of component pair (a, b) at non-negative offsets Delta is the
octant tensor T_ab[d1, d2, d3] = T_ab(d1 h, d2 h, d3 h), d_i in [0, n_i).  The
dyad (k0^2 delta_ab + d_a d_b) g(|r|) is even in every offset for a = b and, for
a != b, odd in the offsets along axes a and b and even in the third, so the other
octants follow from parity signs.  HOSVD (De Lathauwer, De Moor, Vandewalle 2000):
the factor of mode k holds the leading left singular vectors of the mode-k
unfolding, truncated so that the discarded squared singular values are at most
tol^2 ||T||^2 / 3 per mode; the core is T multiplied by the conjugate
transposed factors.  The truncation error is then at most tol ||T|| (the squared
error is bounded by the sum of the discarded squared singular values of the
three modes).

Pinned by (tests/test_oracle_tucker.py): exact reconstruction at full rank; the
error bound; multilinear rank (1, 1, 1) for a separable tensor; the parity
re-embedding of the exact octants against the direct evaluation at every offset
(oracle.volume.embedded_kernel); and the body matvec with the compressed
generators against the uncompressed one.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import physics, volume


def _unfold(T, k):
    return np.moveaxis(T, k, 0).reshape(T.shape[k], -1)


def hosvd(T, tol):
    """Truncated HOSVD of a 3-way tensor: (core, [U1, U2, U3]), ||T - T^|| <= tol ||T||."""
    T = np.asarray(T, np.complex128)
    nrm2 = float(np.vdot(T, T).real)
    budget = tol * tol * nrm2 / 3.0
    U = []
    for k in range(3):
        u, s, _ = np.linalg.svd(_unfold(T, k), full_matrices=False)
        tail = np.cumsum((s ** 2)[::-1])[::-1]          # tail[r] = sum_{i >= r} s_i^2
        r = len(s)
        while r > 1 and tail[r - 1] <= budget:
            r -= 1
        U.append(u[:, :r])
    core = T
    for k in range(3):
        core = np.moveaxis(np.tensordot(U[k].conj().T, np.moveaxis(core, k, 0), axes=1), 0, k)
    return core, U


def reconstruct(core, U):
    T = core
    for k in range(3):
        T = np.moveaxis(np.tensordot(U[k], np.moveaxis(T, k, 0), axes=1), 0, k)
    return T


def generator_octants(n, h, k0):
    """The 6 unique component pairs (oracle.volume.PAIRS order) at offsets
    [0, n_i) per axis: shape (6, n1, n2, n3)."""
    D = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), -1)
    T = physics.voxel_kernel(D, h, k0)
    return np.stack([T[..., a, b] for a, b in volume.PAIRS])


def embed_octants(G, n, L=None):
    """Circulant embedding (the layout of oracle.volume.embedded_kernel) of the
    octant tensors G (6, n1, n2, n3), the negative offsets filled by parity."""
    n = tuple(int(v) for v in n)
    L = tuple(2 * v for v in n) if L is None else tuple(int(v) for v in L)
    out = np.zeros((6,) + L, np.complex128)
    idx, sgn = [], []
    for ni, Li in zip(n, L):
        k = np.arange(Li)
        d = np.where(k < ni, k, k - Li)
        ok = (k < ni) | (k > Li - ni)
        idx.append((np.abs(d), ok))
        sgn.append(np.where(d < 0, -1.0, 1.0))
    for c, (a, b) in enumerate(volume.PAIRS):
        s = np.ones(L)
        for ax in range(3):
            if (a == ax) != (b == ax):     # odd in this axis
                shape = [1, 1, 1]
                shape[ax] = L[ax]
                s = s * sgn[ax].reshape(shape)
        V = idx[0][1][:, None, None] & idx[1][1][None, :, None] & idx[2][1][None, None, :]
        vals = G[c][np.ix_(idx[0][0] % n[0], idx[1][0] % n[1], idx[2][0] % n[2])]
        out[c] = np.where(V, s * vals, 0.0)
    return out


def compressed_spectra(n, h, k0, tol, L=None):
    """Spectra of the generators after Tucker compression at tol (per component)
    and the multilinear ranks: ((6, L1, L2, L3), [(r1, r2, r3)] * 6)."""
    G = generator_octants(n, h, k0)
    Gc = np.empty_like(G)
    ranks = []
    for c in range(6):
        core, U = hosvd(G[c], tol)
        Gc[c] = reconstruct(core, U)
        ranks.append(core.shape)
    return sfft.fftn(embed_octants(Gc, n, L), axes=(1, 2, 3)), ranks
