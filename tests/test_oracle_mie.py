"""Mie-series pins (oracle/mie.py) and the solver-level check of the oracle's
body operator: a homogeneous sphere under a plane wave, solved through the
FFT body operator, against the Lorenz-Mie interior field."""
import numpy as np
import pytest
from scipy.sparse.linalg import LinearOperator, gmres

from oracle import mie, physics, volume
from paper_2206_12409_gb300 import inputs as I


def test_unit_index_returns_plane_wave():
    # m = 1: c_n = d_n = 1 and the internal expansion is the incident wave's
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.05, 0.05, (64, 3))
    E = mie.interior_field(P, 0.1, 1.0, 0.0, 1e9)
    assert np.abs(E - mie.plane_wave(P, 1e9)).max() < 1e-10


def test_quasi_static_limit():
    # k0 a -> 0, lossless: uniform interior field 3 / (eps + 2) x_hat (the
    # induced magnetic-dipole field is of relative order k0 r (eps + 2) / 3,
    # about 1e-5 here)
    rng = np.random.default_rng(2)
    P = rng.uniform(-5e-4, 5e-4, (32, 3))
    E = mie.interior_field(P, 1e-3, 50.0, 0.0, 100e3)
    ref = 3.0 / 52.0
    assert np.abs(E[:, 0] - ref).max() / ref < 1e-4
    assert np.abs(E[:, 1:]).max() / ref < 1e-4


def test_series_truncation_converged():
    rng = np.random.default_rng(3)
    P = rng.uniform(-0.012, 0.012, (32, 3))
    a = mie.interior_field(P, 25e-3, 50.0, 0.6, 298e6)
    b = mie.interior_field(P, 25e-3, 50.0, 0.6, 298e6, n_max=40)
    assert np.abs(a - b).max() / np.abs(b).max() < 1e-12


def _vie_vs_mie(N, eps, sig, f=298e6, R=25e-3):
    """Sphere of diameter N voxels; returns (error over all material voxels,
    error over voxels within 0.6 of the equal-volume radius)."""
    h = 2 * R / N
    g, er, sg = I.sphere_phantom(n=(N + 2,) * 3, h=h, radius=R, eps_r=eps, sigma=sig)
    chi = physics.chi(er, sg, f)
    _, k0 = physics.omega_k0(f)
    b = mie.body_rhs(g, er, sg, f)
    spec = volume.kernel_spectra(g.n, g.h, k0)
    A = LinearOperator((3 * g.nv,) * 2, dtype=complex,
                       matvec=lambda v: volume.fft_matvec(g, chi, k0, v, spec).ravel())
    x, info = gmres(A, b, rtol=1e-10, restart=200, maxiter=3000)
    assert info == 0
    E = mie.body_field(x, er, sg, f)
    inside = chi != 0
    req = (3 * inside.sum() * h ** 3 / (4 * np.pi)) ** (1 / 3)   # equal-volume sphere
    C = g.centres()[inside]
    Em = mie.interior_field(C, req, eps, sig, f)
    core = np.linalg.norm(C, axis=1) < 0.6 * req
    e_all = np.linalg.norm(E[inside] - Em) / np.linalg.norm(Em)
    e_core = np.linalg.norm(E[inside][core] - Em[core]) / np.linalg.norm(Em[core])
    return e_all, e_core


def test_body_operator_converges_to_mie_low_contrast():
    e8 = _vie_vs_mie(8, 2.0, 0.0)
    e16 = _vie_vs_mie(16, 2.0, 0.0)
    assert e8[1] < 0.02 and e16[1] < 0.008 and e16[1] < 0.6 * e8[1]
    assert e16[0] < 0.06


def test_body_operator_converges_to_mie_moderate_contrast():
    # eps_r = 10, sigma = 0.3 S/m: the one-point discretisation converges slowly
    # near the surface, so the core field is what is compared
    e8 = _vie_vs_mie(8, 10.0, 0.3)
    e16 = _vie_vs_mie(16, 10.0, 0.3)
    assert e16[1] < 0.25 and e16[1] < 0.6 * e8[1]
