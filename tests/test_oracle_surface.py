"""Pins of the oracle's surface parts: analytic potential integrals, the EFIE
(Sec. II.B), body-surface coupling, pFFT (Sec. II.C/III) and the hybrid
operator (Eq. hvsie_disc) against the uncompressed dense operator."""
import numpy as np
import pytest
from scipy import integrate

from paper_2206_12409_gb300 import inputs as I
from oracle import physics, rwg, potint, efie, coupling, pfft, hybrid


def _brute_potint(r, P):
    e1, e2 = P[1] - P[0], P[2] - P[0]
    A2 = np.linalg.norm(np.cross(e1, e2))
    lim = lambda u: 1 - u
    I0 = integrate.dblquad(lambda v, u: A2 / np.linalg.norm(r - P[0] - u * e1 - v * e2),
                           0, 1, 0, lim, epsabs=1e-13, epsrel=1e-12)[0]
    I1 = [integrate.dblquad(lambda v, u, k=k: A2 * (P[0] + u * e1 + v * e2 - r)[k]
                            / np.linalg.norm(r - P[0] - u * e1 - v * e2),
                            0, 1, 0, lim, epsabs=1e-13, epsrel=1e-12)[0] for k in range(3)]
    return I0, np.array(I1)


@pytest.mark.parametrize("r", [(0.3, 0.3, 0.5), (2.0, -1.0, 0.3), (1.5, 1.5, 0.0),
                               (-0.5, 0.2, 0.0), (0.4, 0.3, 0.01), (0.35, 0.3, 0.0)])
def test_potential_integrals_vs_adaptive_quadrature(r):
    P = np.array([[0.0, 0, 0], [1.0, 0.2, 0], [0.3, 0.9, 0]])
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    r = np.asarray(r)
    a0, a1 = potint.integrals(r[None], P, n)
    b0, b1 = _brute_potint(r, P)
    assert abs(a0[0] - b0) < 1e-9 * abs(b0)
    assert np.abs(a1[0] - b1).max() < 1e-9 * np.abs(b1).max()


def test_rwg_topology(sphere_loop_shield):
    rs = rwg.build(sphere_loop_shield.shield)
    rc = rwg.build(sphere_loop_shield.coil)
    assert rs.m == 1536 and rc.m == 256
    # divergence integrates to zero over each RWG: A+ (l/A+) - A- (l/A-) = 0
    assert rc.ports.tolist() == [int(np.nonzero((rc.edges == [0, 128]).all(1))[0][0])]


def test_efie_symmetric(sphere_loop_shield):
    _, k0 = physics.omega_k0(298e6)
    rc = rwg.build(sphere_loop_shield.coil)
    K = efie.K_dense(rc, rc, k0, True)
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()


def test_loop_inductance_and_radiation_resistance():
    """Low-frequency strip loop: X = omega mu0 R (ln(8R/a) - 2) with a = w/4
    (within 5%), and R_rad = 20 pi^2 (C/lambda)^4 (within 3%)."""
    f = 10e6
    m = I.loop_strip(40e-3, 2e-3, 128)
    r = rwg.build(m)
    w, k0 = physics.omega_k0(f)
    Z = -efie.K_dense(r, r, k0, True)
    b = rwg.rhs_ports(r, w, physics.EPS0)
    j = np.linalg.solve(Z, b)
    Zin = 1.0 / (j[r.ports[0], 0] * r.length[r.ports[0]])
    L = physics.MU0 * 0.04 * (np.log(8 * 0.04 / 0.5e-3) - 2)
    assert abs(Zin.imag / (w * L) - 1) < 0.05
    Rrad = 20 * np.pi ** 2 * (2 * np.pi * 0.04 * f / physics.C0) ** 4
    assert abs(Zin.real / Rrad - 1) < 0.03


def test_gop_rwg_matches_potentials_fd():
    """Gop f = k0^2 A + grad(phi) with A = \\int g f, phi = \\int g div f; the
    gradient by central differences of the same-rule scalar potential."""
    m = I.loop_strip(40e-3, 2e-3, 32)
    r = rwg.build(m)
    k0 = 6.24
    pts = np.array([[0.0, 0.0, 0.02], [0.05, 0.01, -0.01]])
    E = coupling.gop_rwg(r, [3], pts, rwg.TRI6, k0)[:, 0, :]

    def pot(x):
        A = np.zeros(3, complex)
        phi = 0j
        for t, s, v in rwg.halves(r, 3):
            q, wq = rwg.tri_points(r, t, rwg.TRI6)
            q, wq = q[0], wq[0]
            g = physics.g_scalar(np.linalg.norm(x - q, axis=1), k0) * wq
            A += s * r.length[3] / (2 * r.area[t]) * (g[:, None] * (q - r.xyz[v])).sum(0)
            phi += s * r.length[3] / r.area[t] * g.sum()
        return A, phi
    for p, e in zip(pts, E):
        A, _ = pot(p)
        grad = np.array([(pot(p + d)[1] - pot(p - d)[1]) / 2e-6 for d in np.eye(3) * 1e-6])
        ref = k0 ** 2 * A + grad
        assert np.abs(e - ref).max() < 1e-6 * np.abs(ref).max()


def test_pfft_projection_reproduces_field():
    """Projected stencil currents reproduce the RWG field away from the
    stencil: 3^3 to 5e-3 beyond 4 voxels, 5^3 to 2e-4."""
    p = I.problem_sphere_loop_shield(ext_n=(22, 22, 12))
    _, k0 = physics.omega_k0(p.freq_hz)
    rc = rwg.build(p.coil)
    eg = p.ext_grid
    cols = np.arange(0, 256, 32)
    for s, tol in ((3, 5e-3), (5, 2e-4)):
        W, base = pfft.projection(eg, rc, cols, s, k0)
        for j, n in enumerate(cols):
            ctr = np.asarray(eg.origin) + eg.h * (base[j] + (s - 1) // 2)
            tp = ctr + 4 * eg.h * pfft.fibonacci_sphere(40)
            et = coupling.gop_rwg(rc, [n], tp, rwg.TRI6, k0)[:, 0, :]
            rq = ctr + eg.h * pfft.stencil_offsets(s)
            D = physics.dyad(tp[:, None, :] - rq[None], k0) * eg.h ** 3
            ef = np.einsum("tqab,bq->ta", D, W[j].reshape(3, -1))
            assert np.linalg.norm(ef - et) / np.linalg.norm(et) < tol


def _blocks_err(prob, P, Z, idx):
    mf, mn = P.m_f, P.m_n
    M3 = np.tile(P.chi != 0, 3)
    x0 = I.random_vectors(P.N, 1)
    x0[mf + mn:][~M3] = 0
    errs = {}
    for name, sl in (("f", slice(0, mf)), ("n", slice(mf, mf + mn)), ("b", slice(mf + mn, None))):
        x = np.zeros_like(x0)
        x[sl] = x0[sl]
        yh = hybrid.matvec(P, x)
        yd = hybrid.dense_matvec(prob, Z, idx, x)
        for nm, s2 in (("f", slice(0, mf)), ("n", slice(mf, mf + mn)), ("b", slice(mf + mn, None))):
            errs[name + nm] = np.linalg.norm(yh[s2] - yd[s2]) / np.linalg.norm(yd[s2])
    return errs


def test_hybrid_matches_dense_blocks(sphere_loop_shield, hybrid_parts, dense_reference):
    """Exact blocks to 1e-13; TT blocks within the TT tolerance (1e-6); ACA
    exact at this size (full rank); pFFT coupling with the 3^3 stencil ~1e-3."""
    Z, idx = dense_reference
    e = _blocks_err(sphere_loop_shield, hybrid_parts, Z, idx)
    for k in ("ff", "nn", "bb", "fn", "nf"):
        assert e[k] < 1e-12, (k, e[k])
    assert e["fb"] < 2e-6 and e["bf"] < 2e-6
    assert e["nb"] < 2e-3 and e["bn"] < 2e-3


def test_dense_reference_symmetric(dense_reference):
    Z, _ = dense_reference
    assert np.abs(Z - Z.T).max() <= 1e-12 * np.abs(Z).max()


def test_hybrid_reciprocity(hybrid_parts):
    """u^T (Z v) = v^T (Z u) for the compressed operator (TT and its transpose,
    P and P^T, U V^H and conj(V) U^T are consistent)."""
    P = hybrid_parts
    M3 = np.tile(P.chi != 0, 3)
    u = I.random_vectors(P.N, 1, seed=1)
    v = I.random_vectors(P.N, 1, seed=2)
    u[P.m_f + P.m_n:][~M3] = 0
    v[P.m_f + P.m_n:][~M3] = 0
    a = (u.T @ hybrid.matvec(P, v))[0, 0]
    b = (v.T @ hybrid.matvec(P, u))[0, 0]
    assert abs(a - b) <= 1e-12 * abs(a)


def test_pfft_coupling_with_5_stencil_meets_1e4(dense_reference):
    """With the 5^3 projection stencil the pFFT coil-body coupling products
    (both directions, precorrection included) are within 1e-4 of the dense
    direct coupling; the exact blocks stay exact."""
    from oracle import hybrid
    import dataclasses
    prob = dataclasses.replace(I.problem_sphere_loop_shield(), stencil=5)
    P = hybrid.build_parts(prob)
    Z, idx = dense_reference
    e = _blocks_err(prob, P, Z, idx)
    assert e["nb"] < 1e-4 and e["bn"] < 1e-4, (e["nb"], e["bn"])
    for k in ("ff", "nn", "bb", "fn", "nf"):
        assert e[k] < 1e-12, (k, e[k])
