"""GMRES(m) and flexible GMRES (Sec. III.A; Saad and Schultz 1986; Saad 1993).

Plain restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations,
x0 = 0, stopping when the relative residual ||b - A x|| / ||b|| <= tol; the true
residual is recomputed at every restart.  The flexible variant stores the
preconditioned directions z_j = M(v_j) (right preconditioning that may change
between iterations).  Pinned against LU solves (tests).
"""
from __future__ import annotations

import numpy as np


def gmres(A, b, tol=1e-6, restart=50, maxit=10000, M=None, x0=None):
    """Solve A x = b for one right-hand side.  A, M: callables on vectors.
    Returns x, info dict (iterations, relative residual history)."""
    b = np.asarray(b, np.complex128).ravel()
    n = b.size
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    bn = np.linalg.norm(b)
    hist = []
    if bn == 0:
        return np.zeros(n, np.complex128), {"iters": 0, "relres": 0.0, "hist": hist}
    it = 0
    est_last = 1.0
    r = b - A(x) if np.any(x) else b.copy()
    beta = np.linalg.norm(r)
    hist.append(beta / bn)
    while it < maxit and beta / bn > tol:
        V = np.zeros((restart + 1, n), np.complex128)
        Zs = np.zeros((restart, n), np.complex128) if M is not None else None
        H = np.zeros((restart + 1, restart), np.complex128)
        cs = np.zeros(restart, np.complex128)
        sn = np.zeros(restart, np.complex128)
        g = np.zeros(restart + 1, np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            zj = M(V[j]) if M is not None else V[j]
            if M is not None:
                Zs[j] = zj
            w = A(zj)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            # previous rotations G_i = [[conj(c), conj(s)], [-s, c]] (unitary)
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.sqrt(abs(H[j, j]) ** 2 + abs(H[j + 1, j]) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = H[j, j] / den
                sn[j] = H[j + 1, j] / den
            H[j, j] = np.conj(cs[j]) * H[j, j] + np.conj(sn[j]) * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= tol or it >= maxit:
                break
        est_last = abs(g[k]) / bn
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        basis = Zs[:k] if M is not None else V[:k]
        x = x + basis.T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bn
    return x, {"iters": it, "relres": beta / bn, "hist": hist,
               "est": est_last if it else beta / bn}
