"""Adaptive cross approximation with partial pivoting (Sec. III, U V^* = ACA(Z_cc^fn)).

Follows Zhao, Vouvakis and Lee (IEEE TEMC 2005): starting from row 0, take the
residual row, pivot on its largest entry, take the residual column there, and
pick the next row at the largest entry of that column among unused rows.  Stop
when ||u_k|| ||v_k|| <= tol ||Z_k||_F, with ||Z_k||_F updated recursively.
Returns U (m x k) and V (n x k) with Z ~= U V^H (the paper's U V^*).
Pinned by exact-rank matrices and by the error on a dense block (tests).
"""
from __future__ import annotations

import numpy as np


def aca(get_row, get_col, m, n, tol, max_rank=None):
    max_rank = min(m, n) if max_rank is None else max_rank
    us, vs = [], []                      # Z ~= sum_k u_k v_k^T
    used_r = np.zeros(m, bool)
    used_c = np.zeros(n, bool)
    i = 0
    norm2 = 0.0
    for _ in range(max_rank):
        used_r[i] = True
        row = np.array(get_row(i), np.complex128)
        for u, v in zip(us, vs):
            row -= u[i] * v
        row_m = np.where(used_c, 0.0, np.abs(row))
        j = int(np.argmax(row_m))
        if row_m[j] == 0.0:
            free = np.nonzero(~used_r)[0]
            if free.size == 0:
                break
            i = int(free[0])
            continue
        used_c[j] = True
        v = row / row[j]
        u = np.array(get_col(j), np.complex128)
        for uu, vv in zip(us, vs):
            u -= vv[j] * uu
        nu, nv = np.linalg.norm(u), np.linalg.norm(v)
        cross = 0.0
        for uu, vv in zip(us, vs):
            cross += 2.0 * np.real(np.vdot(uu, u) * np.vdot(vv, v))
        norm2 += cross + (nu * nv) ** 2
        us.append(u)
        vs.append(v)
        if nu * nv <= tol * np.sqrt(max(norm2, 0.0)):
            break
        col_m = np.where(used_r, 0.0, np.abs(u))
        i = int(np.argmax(col_m))
        if col_m[i] == 0.0:
            break
    if not us:
        return np.zeros((m, 0), np.complex128), np.zeros((n, 0), np.complex128)
    U = np.stack(us, 1)
    V = np.conj(np.stack(vs, 1))
    return U, V


def aca_dense(Z, tol, max_rank=None):
    return aca(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, max_rank)
