"""Pins of the oracle's body operator (Sec. II.B) against brute force, symmetry
and closed-form physics."""
import numpy as np
import pytest
from scipy import integrate

from paper_2206_12409_gb300 import inputs as I
from oracle import physics, volume


@pytest.mark.parametrize("n", [(4, 4, 4), (7, 6, 5), (3, 8, 5), (12, 12, 12)])
def test_fft_matches_dense_brute_force(n):
    """Toeplitz/FFT product == dense brute-force product (all voxels material)."""
    g, er, sg = I.sphere_phantom(n, 5e-3, 1.0, 50.0, 0.6)
    chi = physics.chi(er, sg, 298e6)
    _, k0 = physics.omega_k0(298e6)
    x = I.random_vectors(3 * g.nv, 2)
    yd = volume.dense_matvec(g, chi, k0, x)
    yf = volume.fft_matvec(g, chi, k0, x)
    assert np.linalg.norm(yd - yf) / np.linalg.norm(yd) < 1e-13


def test_fft_matches_dense_heterogeneous():
    g, er, sg = I.sphere_phantom((9, 8, 7), 5e-3, 16e-3, 50.0, 0.6)
    chi = physics.chi(er, sg, 298e6)
    _, k0 = physics.omega_k0(298e6)
    x = I.random_vectors(3 * g.nv, 1)
    M3 = np.tile(chi != 0, 3)
    yd = volume.dense_matvec(g, chi, k0, x)
    yf = volume.fft_matvec(g, chi, k0, x)
    assert np.linalg.norm((yd - yf)[M3]) / np.linalg.norm(yd[M3]) < 1e-13
    assert np.array_equal(yf[~M3], x[~M3])


def test_complex_symmetry():
    g, er, sg = I.sphere_phantom((7, 7, 7), 5e-3, 15e-3, 50.0, 0.6)
    chi = physics.chi(er, sg, 298e6)
    _, k0 = physics.omega_k0(298e6)
    Z, _ = volume.dense_Zbb(g, chi, k0)
    assert np.abs(Z - Z.T).max() <= 1e-12 * np.abs(Z).max()


def test_self_term_is_sphere_quadrature():
    """Self term = field at the centre of the equal-volume sphere carrying unit
    uniform x-current: principal-value volume integral of the dyad plus the
    -1/3 depolarisation, by 2D adaptive quadrature (phi done in closed form)."""
    k0, h = 6.24, 5e-3
    a = (3 / (4 * np.pi)) ** (1 / 3) * h

    def f(th, r, part):
        g = np.exp(-1j * k0 * r) / (4 * np.pi * r)
        A = g / r ** 2 * (k0 ** 2 * r ** 2 - 1 - 1j * k0 * r)
        B = g / r ** 2 * (3 + 3j * k0 * r - k0 ** 2 * r ** 2)
        v = (A + B * np.sin(th) ** 2 / 2) * 2 * np.pi * r ** 2 * np.sin(th)
        return v.real if part == 0 else v.imag
    re = integrate.dblquad(f, 0, a, 0, np.pi, args=(0,), epsabs=1e-13)[0]
    im = integrate.dblquad(f, 0, a, 0, np.pi, args=(1,), epsabs=1e-13)[0]
    ref = re + 1j * im - 1.0 / 3.0
    assert abs(physics.self_term(k0, h) - ref) < 1e-9


def test_static_limit_self_term():
    assert abs(physics.self_term(1e-9, 1e-3) + 1.0 / 3.0) < 1e-12


def test_dyad_matches_finite_difference():
    """(k0^2 I + grad grad) g against central differences of g."""
    k0 = 6.0
    r = np.array([0.011, -0.007, 0.004])
    D = physics.dyad(r, k0)
    e = 1e-5
    H = np.zeros((3, 3), complex)
    for a in range(3):
        for b in range(3):
            ea, eb = np.eye(3)[a] * e, np.eye(3)[b] * e
            gg = lambda v: physics.g_scalar(np.linalg.norm(v), k0)
            H[a, b] = (gg(r + ea + eb) - gg(r + ea - eb) - gg(r - ea + eb) + gg(r - ea - eb)) / (4 * e * e)
    ref = k0 ** 2 * physics.g_scalar(np.linalg.norm(r), k0) * np.eye(3) + H
    assert np.abs(D - ref).max() < 1e-5 * np.abs(D).max()


def test_clausius_mossotti_limit_converges():
    """Small dielectric sphere at low frequency: interior field -> 3 E0 / (eps_r + 2).
    The staircased sphere approaches it under refinement (within 10%)."""
    errs = []
    for n, rad in [(9, 4.0), (13, 6.0)]:
        h = 1e-3
        g, er, sg = I.sphere_phantom((n, n, n), h, rad * h, 50.0, 0.0)
        f = 1e5
        chi = physics.chi(er, sg, f)
        w, k0 = physics.omega_k0(f)
        Z, idx = volume.dense_Zbb(g, chi, k0)
        m = idx.size
        b = np.zeros(3 * m, complex)
        b[:m] = 1j * w * physics.EPS0 * h ** 3
        j = np.linalg.solve(Z, b)
        E = j[:m] / (1j * w * physics.EPS0 * chi[idx])
        errs.append(abs(E.mean() - 3 / 52) / (3 / 52))
    assert errs[0] < 0.10 and errs[1] < errs[0]


def test_rows_matvec_equals_dense():
    """The direct-sum rows (used for sampled checks on grids the FFT oracle does
    not fit) equal the brute-force dense matvec, vacuum rows included."""
    from oracle import volume, physics
    from paper_2206_12409_gb300 import inputs as I
    g, er, sg = I.sphere_phantom((7, 6, 5), 5e-3, 14e-3, 50.0, 0.6)
    chi = physics.chi(er, sg, 298e6)
    _, k0 = physics.omega_k0(298e6)
    x = I.random_vectors(3 * g.nv, 2, seed=5)
    yd = volume.dense_matvec(g, chi, k0, x)
    rows = np.array([0, 17, g.nv + 44, 2 * g.nv + 101, 3 * g.nv - 1, int(np.argmax(chi != 0))])
    yr = volume.rows_matvec(g, chi, k0, x, rows, chunk=37)
    assert np.max(np.abs(yr - yd[rows])) <= 1e-13 * np.max(np.abs(yd))
