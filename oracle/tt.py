"""Tensor train: TT-SVD, reconstruction and the TT matvecs of the paper.

Eq. (TT) / Eq. (ass_TT): a 4D tensor Z(i1, i2, i3, i4) is represented by cores
G1 (n1 x r1), G2 (r1 x n2 x r2), G3 (r2 x n3 x r3), G4 (r3 x n4).  TT-SVD
(Sec. II.D, Oseledets 2011) by sequential truncated SVDs of the unfoldings with
per-step threshold tol ||Z||_F / sqrt(d - 1).

Eq. (mvp): y = G4 x; y = G3 y (G3 reshaped (r2 n3) x r3); Y = G2 Y (Y: r2 x n3,
G2 reshaped (r1 n2) x r2); Y = G1 Y (Y: r1 x n2 n3); y = vec(Y) (n1 n2 n3).
Eq. (tmvp): the transposed chain j^T G1, G2, G3, G4 with the reshapes implied by
the column-major order of Eq. (mvp).  All reshapes are column-major.
Pinned by reconstruction against the dense tensor (tests).
"""
from __future__ import annotations

import numpy as np


def tt_svd(A, tol):
    A = np.asarray(A, np.complex128)
    dims = A.shape
    d = len(dims)
    delta = tol * np.linalg.norm(A.ravel()) / np.sqrt(d - 1)
    cores = []
    r = 1
    C = A.reshape(dims, order="F")
    W = C.reshape((r * dims[0], -1), order="F")
    for k in range(d - 1):
        W = W.reshape((r * dims[k], -1), order="F")
        U, s, Vh = np.linalg.svd(W, full_matrices=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]   # tail[i] = ||s[i:]||
        rk = int(np.sum(tail > delta))
        rk = max(rk, 1)
        cores.append(U[:, :rk].reshape((r, dims[k], rk), order="F"))
        W = s[:rk, None] * Vh[:rk]
        r = rk
    cores.append(W.reshape((r, dims[-1], 1), order="F"))
    G1 = cores[0][0]                      # (n1, r1)
    G4 = cores[-1][:, :, 0]               # (r3, n4)
    return [G1] + cores[1:-1] + [G4]


def tt_full(cores):
    """Dense tensor of Eq. (TT), contracted one core at a time."""
    G1, G2, G3, G4 = cores
    T = np.tensordot(G1, G2, axes=(1, 0))        # (n1, n2, r2)
    T = np.tensordot(T, G3, axes=(2, 0))         # (n1, n2, n3, r3)
    return np.tensordot(T, G4, axes=(3, 0))      # (n1, n2, n3, n4)


def tt_matvec(cores, x):
    """Eq. (mvp) step by step; x (n4, p) -> y (n1 n2 n3, p)."""
    G1, G2, G3, G4 = cores
    n1, r1 = G1.shape
    _, n2, r2 = G2.shape
    _, n3, r3 = G3.shape
    x = np.asarray(x).reshape(G4.shape[1], -1)
    out = []
    for j in range(x.shape[1]):
        y = G4 @ x[:, j]                                  # r3
        y = G3.reshape((r2 * n3, r3), order="F") @ y      # r2 n3
        Y = y.reshape((r2, n3), order="F")
        Y = G2.reshape((r1 * n2, r2), order="F") @ Y      # (r1 n2) x n3
        Y = Y.reshape((r1, n2 * n3), order="F")
        Y = G1 @ Y                                        # n1 x (n2 n3)
        out.append(Y.reshape(-1, order="F"))
    return np.stack(out, 1)


def tt_rmatvec(cores, jb):
    """Eq. (tmvp) for one component: (jb^T Z)^T with jb (n1 n2 n3, p) -> (n4, p)."""
    G1, G2, G3, G4 = cores
    n1, r1 = G1.shape
    _, n2, r2 = G2.shape
    _, n3, r3 = G3.shape
    jb = np.asarray(jb).reshape(n1 * n2 * n3, -1)
    out = []
    for j in range(jb.shape[1]):
        Y = jb[:, j].reshape((n1, n2 * n3), order="F").T   # (n2 n3) x n1
        Y = Y @ G1                                           # (n2 n3) x r1
        # rows i2 + n2 i3, columns j1 -> (n3) x (r1 n2) with column j1 + r1 i2
        Y = Y.reshape((n2, n3, r1), order="F").transpose(1, 2, 0).reshape((n3, r1 * n2), order="F")
        Y = Y @ G2.reshape((r1 * n2, r2), order="F")        # n3 x r2
        y = Y.T.reshape(-1, order="F")                      # 1 x (r2 n3): j2 + r2 i3
        y = y @ G3.reshape((r2 * n3, r3), order="F")        # r3
        y = y @ G4                                          # n4
        out.append(y)
    return np.stack(out, 1)
