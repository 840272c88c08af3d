"""GPU GMRES (Sec. III.A) with the oracle's operator parts: plain FP64 and
FP32-inner / FP64-refined solves, each checked by the oracle's own matvec;
error statuses from host-side injections.  The small sphere + loop + closed
shield problem (N = 832) is used because restarted GMRES converges on it with a
300-vector restart; the larger workloads need far longer Krylov spaces."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import hybrid, gmres as ogmres, rwg, physics
from tests.conftest import oracle_parts_to_abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    import __graft_entry__ as ge
    prob = ge._tiny_problem()
    return prob, hybrid.build_parts(prob)


@pytest.fixture(scope="module")
def ctx(tiny):
    from paper_2206_12409_gb300 import vsie as V
    prob, P = tiny
    parts, keep = oracle_parts_to_abi(P)
    g = prob.grid
    c = V.vsie_create(V.make_grid(g.n, g.h, g.origin), prob.eps_r, prob.sigma, prob.freq_hz,
                      V.make_options(ext_n=prob.ext_n, ext_offset=prob.ext_offset, max_rhs=4),
                      parts)
    yield c
    V.vsie_destroy(c)


def _rhs(prob, P):
    """Coil port RHS (delta gap, 1 V) plus a plane-wave-like body excitation,
    two columns."""
    w, _ = physics.omega_k0(prob.freq_hz)
    rc = rwg.build(prob.coil)
    b = np.zeros((P.N, 2), np.complex128)
    e = rc.ports[0]
    b[P.m_f + e, 0] = 1j * w * physics.EPS0 * rc.length[e]
    M = P.chi != 0
    nb = P.body.nv
    b[P.m_f + P.m_n:P.m_f + P.m_n + nb, 1] = np.where(M, 1j * w * physics.EPS0 * P.body.h ** 3, 0)
    return b


def _solve(ctx, b, tol, mode, check=True, **kw):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    N, p = b.shape
    B = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    X = torch.zeros_like(B)
    o = V.vsie_solve_opts()
    o.mode = mode
    for k, v in kw.items():
        setattr(o, k, v)
    st, info = V.vsie_solve(ctx, p, B.data_ptr(), N, X.data_ptr(), N, tol, o, check=check)
    torch.cuda.synchronize()
    return st, info, X.cpu().numpy().T.copy()


def test_plain_fp64_gmres(ctx, tiny):
    from paper_2206_12409_gb300 import vsie as V
    prob, P = tiny
    b = _rhs(prob, P)
    st, info, x = _solve(ctx, b, 1e-10, 0, restart=300, maxit=3000)
    assert st == V.VSIE_OK
    r = b - hybrid.matvec(P, x)
    for c in range(2):
        rel = np.linalg.norm(r[:, c]) / np.linalg.norm(b[:, c])
        assert rel <= 1.05e-10, rel
        assert info.relres[c] <= 1e-10
    # against the oracle's own GMRES solution
    xo, io = ogmres.gmres(lambda v: hybrid.matvec(P, v)[:, 0], b[:, 0], 1e-11, restart=300)
    assert np.linalg.norm(x[:, 0] - xo) <= 1e-7 * np.linalg.norm(xo)


def test_mixed_refined_reaches_fp64_residual(ctx, tiny):
    from paper_2206_12409_gb300 import vsie as V
    prob, P = tiny
    b = _rhs(prob, P)
    st, info, x = _solve(ctx, b, 1e-6, 1, restart=300, maxit=3000, inner_tol=1e-4)
    assert st == V.VSIE_OK
    assert info.matvecs32 > 0 and info.outer >= 1
    r = b - hybrid.matvec(P, x)
    for c in range(2):
        assert np.linalg.norm(r[:, c]) / np.linalg.norm(b[:, c]) <= 1.05e-6


def test_refined_solution_matches_fp64_solution(ctx, tiny):
    """Both solved to 1e-10: refined and plain FP64 solutions agree to 1e-6."""
    prob, P = tiny
    b = _rhs(prob, P)
    _, _, x0 = _solve(ctx, b, 1e-10, 0, restart=300, maxit=3000)
    _, info, x1 = _solve(ctx, b, 1e-10, 1, restart=300, maxit=3000, inner_tol=1e-4)
    for c in range(2):
        assert np.linalg.norm(x1[:, c] - x0[:, c]) <= 1e-6 * np.linalg.norm(x0[:, c])


def test_enoconv_returns_last_iterate(ctx, tiny):
    from paper_2206_12409_gb300 import vsie as V
    prob, P = tiny
    b = _rhs(prob, P)[:, :1]
    st, info, x = _solve(ctx, b, 1e-12, 0, restart=5, maxit=5)
    assert st == V.VSIE_ENOCONV
    r = b - hybrid.matvec(P, x)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert 0 < rel < 1 and abs(rel - info.relres[0]) <= 1e-8


def test_nan_rhs_is_breakdown(ctx, tiny):
    from paper_2206_12409_gb300 import vsie as V
    b = np.zeros((tiny[1].N, 1), np.complex128)
    b[3, 0] = np.nan
    st, _, _ = _solve(ctx, b, 1e-6, 0, check=False)
    assert st == V.VSIE_EBREAKDOWN


def test_rhs_ports_from_setup(sphere_loop_shield):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    prob = sphere_loop_shield
    c = V.setup_problem(prob, max_rhs=2)
    try:
        N, mf, mn, nb = V.vsie_sizes(c)
        B = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
        V.vsie_rhs_ports(c, [0], 1.0, B.data_ptr(), N)
        torch.cuda.synchronize()
        b = B.cpu().numpy()[0]
        w, _ = physics.omega_k0(prob.freq_hz)
        rc = rwg.build(prob.coil)
        e = rc.ports[0]
        assert np.count_nonzero(b) == 1
        assert abs(b[mf + e] - 1j * w * physics.EPS0 * rc.length[e]) <= 1e-15
    finally:
        V.vsie_destroy(c)
