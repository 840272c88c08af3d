"""Pins of the oracle's TT (Eq. TT, mvp, tmvp), ACA and GMRES against exact
constructions and LU."""
import numpy as np

from oracle import tt, aca, gmres


def _rand_tt(rng, n, r):
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    return [c(n[0], r[0]), c(r[0], n[1], r[1]), c(r[1], n[2], r[2]), c(r[2], n[3])]


def test_tt_svd_exact_ranks():
    rng = np.random.default_rng(0)
    G = _rand_tt(rng, (6, 5, 7, 9), (2, 3, 4))
    A = tt.tt_full(G)
    C = tt.tt_svd(A, 1e-12)
    assert [c.shape for c in C] == [(6, 2), (2, 5, 3), (3, 7, 4), (4, 9)]
    assert np.linalg.norm(tt.tt_full(C) - A) / np.linalg.norm(A) < 1e-13


def test_tt_svd_error_bound():
    """Truncated TT-SVD error <= tol ||A||_F (quasi-optimality bound)."""
    i = np.arange(10)
    A = 1.0 / (i[:, None, None, None] + i[None, :, None, None] + i[None, None, :, None]
               + i[None, None, None, :] + 1.0) + 0j
    for tol in (1e-3, 1e-6):
        C = tt.tt_svd(A, tol)
        assert np.linalg.norm(tt.tt_full(C) - A) <= tol * np.linalg.norm(A) * 1.0001


def test_tt_matvec_and_transpose_vs_dense():
    rng = np.random.default_rng(1)
    G = _rand_tt(rng, (4, 6, 5, 11), (3, 4, 2))
    A = tt.tt_full(G)
    Am = A.reshape((4 * 6 * 5, 11), order="F")   # rows i1 + n1 (i2 + n2 i3)
    x = rng.standard_normal((11, 3)) + 1j * rng.standard_normal((11, 3))
    assert np.linalg.norm(tt.tt_matvec(G, x) - Am @ x) < 1e-12 * np.linalg.norm(Am @ x)
    jb = rng.standard_normal((120, 2)) + 1j * rng.standard_normal((120, 2))
    assert np.linalg.norm(tt.tt_rmatvec(G, jb) - Am.T @ jb) < 1e-12 * np.linalg.norm(Am.T @ jb)


def test_aca_exact_rank():
    rng = np.random.default_rng(2)
    Z = (rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))) @ \
        (rng.standard_normal((5, 30)) + 1j * rng.standard_normal((5, 30)))
    U, V = aca.aca_dense(Z, 1e-12)
    assert U.shape[1] <= 6
    assert np.linalg.norm(U @ V.conj().T - Z) / np.linalg.norm(Z) < 1e-12


def test_aca_smooth_kernel():
    x = np.linspace(0, 1, 60)
    y = np.linspace(3, 4, 50)
    Z = 1.0 / np.abs(x[:, None] - y[None, :]) + 0j
    U, V = aca.aca_dense(Z, 1e-8)
    assert np.linalg.norm(U @ V.conj().T - Z) / np.linalg.norm(Z) < 1e-7
    assert U.shape[1] < 15


def test_gmres_vs_lu():
    rng = np.random.default_rng(3)
    n = 80
    A = 3 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    x, info = gmres.gmres(lambda v: A @ v, b, 1e-10, restart=15)
    assert info["relres"] <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    Mi = np.linalg.inv(A + 0.2 * np.eye(n))
    x2, info2 = gmres.gmres(lambda v: A @ v, b, 1e-10, restart=15, M=lambda v: Mi @ v)
    assert info2["relres"] <= 1e-10 and info2["iters"] < info["iters"]
    assert np.linalg.norm(x2 - xs) / np.linalg.norm(xs) < 1e-9


def test_gmres_estimate_equals_true_residual_nonnormal_complex():
    """Without restarts GMRES is exact in n steps, and its Givens residual
    estimate equals the true residual at every step (complex, non-normal,
    indefinite matrix: a wrong rotation convention fails this)."""
    rng = np.random.default_rng(4)
    n = 40
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) + \
        np.diag(np.exp(2j * np.pi * rng.random(n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, b, 1e-12, restart=n, maxit=n)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 1e-10
    # estimate after k steps equals the true residual of the k-step solution
    for k in (5, 17, 29):
        xk, ik = gmres.gmres(lambda v: A @ v, b, 1e-30, restart=k, maxit=k)
        true = np.linalg.norm(A @ xk - b) / np.linalg.norm(b)
        assert abs(ik["est"] - true) <= 1e-9 * true


def test_fgmres_with_a_changing_preconditioner():
    """Flexible GMRES (Saad 1993) keeps z_j = M_j(v_j): with a preconditioner that
    changes at every call it still converges to the LU solution, and its
    unrestarted residual after k steps is the minimum over x0 + span(z_0..z_k-1)
    (checked by a direct least-squares solve over the same directions)."""
    rng = np.random.default_rng(5)
    n = 60
    A = 2 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    Mi = np.linalg.inv(A)
    calls = []

    def M(v):   # a different, noisy approximate inverse at every call
        k = len(calls)
        E = np.random.default_rng(100 + k).standard_normal((n, n)) * 0.05 / np.sqrt(n)
        z = (Mi + E) @ v
        calls.append(z.copy())
        return z

    x, info = gmres.gmres(lambda v: A @ v, b, 1e-10, restart=20, M=M)
    assert info["relres"] <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    # minimal-residual property of one cycle of k steps
    calls.clear()
    k = 6
    xk, ik = gmres.gmres(lambda v: A @ v, b, 1e-30, restart=k, maxit=k, M=M)
    Z = np.array(calls[:k]).T                          # the k directions used
    y, *_ = np.linalg.lstsq(A @ Z, b, rcond=None)
    best = np.linalg.norm(A @ (Z @ y) - b)
    assert abs(np.linalg.norm(A @ xk - b) - best) <= 1e-10 * np.linalg.norm(b)
