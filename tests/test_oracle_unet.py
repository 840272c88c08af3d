"""Pins of the oracle U-Net (oracle/unet.py): convolution against SciPy's
correlation and a brute-force loop, every gradient against central finite
differences, pooling/upsampling adjointness, and one Adam step by hand."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import unet


def test_conv3d_matches_correlate_and_brute_force():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv3d(x, w, b)
    for o in range(4):
        ref = b[o] + sum(correlate(x[i], w[o, i], mode="same") for i in range(3))
        assert np.abs(y[o] - ref).max() < 1e-12
    # brute force at a few points
    for (o, z, yy, xx) in [(0, 0, 0, 0), (3, 4, 5, 6), (2, 2, 3, 1)]:
        s = b[o]
        for i in range(3):
            for kz in range(3):
                for ky in range(3):
                    for kx in range(3):
                        zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                        if 0 <= zz < 5 and 0 <= y2 < 6 and 0 <= x2 < 7:
                            s += w[o, i, kz, ky, kx] * x[i, zz, y2, x2]
        assert abs(y[o, z, yy, xx] - s) < 1e-12


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((3, 4, 4, 5))
    dx, dw, db = unet.conv3d_backward(x, w, dy)
    f = lambda x_, w_, b_: np.sum(dy * unet.conv3d(x_, w_, b_))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 3, 2, 4), (0, 2, 1, 1)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0, 0), (2, 1, 2, 1, 0), (1, 0, 1, 1, 1)]:
        e = np.zeros_like(w); e[idx] = h
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * h) - dw[idx]) < 1e-6
    e = np.zeros_like(b); e[1] = h
    assert abs((f(x, w, b + e) - f(x, w, b - e)) / (2 * h) - db[1]) < 1e-6


def test_pool_up_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 8))
    y = rng.standard_normal((2, 2, 3, 4))
    assert abs(np.sum(unet.pool(x) * y) - np.sum(x * unet.pool_backward(y))) < 1e-12
    assert abs(np.sum(unet.up(y) * x) - np.sum(y * unet.up_backward(x))) < 1e-12


@pytest.fixture(scope="module")
def small_net():
    rng = np.random.default_rng(3)
    P = unet.init_params(4)
    for k in P:
        if k.endswith(".b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    x = rng.standard_normal((8, 8, 8, 8))
    return P, x


def test_unet_gradients_finite_differences(small_net):
    P, x = small_net
    rng = np.random.default_rng(5)
    y, tape = unet.forward(P, x)
    assert y.shape == (6, 8, 8, 8)
    dy = rng.standard_normal(y.shape)
    G, gx = unet.backward(P, tape, dy)
    f = lambda P_, x_: np.sum(dy * unet.forward(P_, x_)[0])
    h = 1e-6
    # one weight and one bias of every layer, central differences
    for name, ci, co, k in unet.LAYERS:
        for key, idx in ((name + ".w", tuple(int(rng.integers(s)) for s in P[name + ".w"].shape)),
                         (name + ".b", (int(rng.integers(co)),))):
            Pp = dict(P); Pm = dict(P)
            Pp[key] = P[key].copy(); Pp[key][idx] += h
            Pm[key] = P[key].copy(); Pm[key][idx] -= h
            fd = (f(Pp, x) - f(Pm, x)) / (2 * h)
            assert abs(fd - G[key][idx]) <= 1e-5 * max(1.0, abs(fd)), (key, fd, G[key][idx])
    for idx in [(0, 0, 0, 0), (7, 3, 4, 5)]:
        e = np.zeros_like(x); e[idx] = h
        fd = (f(P, x + e) - f(P, x - e)) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-5 * max(1.0, abs(fd))


def test_adam_first_step_is_signed_lr():
    # at t = 1 the bias-corrected moments give a step of lr * g / (|g| + eps)
    P = {"a": np.array([1.0, -2.0, 0.5])}
    G = {"a": np.array([0.3, -4.0, 0.0])}
    M = {"a": np.zeros(3)}
    V = {"a": np.zeros(3)}
    unet.adam_step(P, G, M, V, 1, lr=0.01)
    ref = np.array([1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8), 0.5])
    assert np.abs(P["a"] - ref).max() < 1e-15


def test_preconditioner_application_pins():
    """The oracle's learned-preconditioner application: with an all-zero network
    it is the inverse of the body block's diagonal (taken from the brute-force
    dense Z_bb) and the identity on vacuum voxels; for any network it is
    positively homogeneous, M(a v) = a M(v) for a > 0 (the input is normalised
    by its RMS and the correction rescaled by it)."""
    from oracle import physics, volume
    from paper_2206_12409_gb300 import inputs as I
    g, er, sg = I.sphere_phantom(n=(6, 6, 6), h=8e-3, radius=20e-3, eps_r=30.0, sigma=0.4)
    f = 298e6
    chi = physics.chi(er, sg, f)
    _, k0 = physics.omega_k0(f)
    Z, idx = volume.dense_Zbb(g, chi, k0)
    m = idx.size
    rng = np.random.default_rng(9)
    v = rng.standard_normal(3 * g.nv) + 1j * rng.standard_normal(3 * g.nv)
    P0 = {k: 0 * w for k, w in unet.init_params(0).items()}
    z0 = unet.apply_preconditioner(P0, g, er, sg, f, v).reshape(3, g.nv)
    vv = v.reshape(3, g.nv)
    vac = chi == 0
    assert np.allclose(z0[:, vac], vv[:, vac], rtol=0, atol=1e-15)
    for a in range(3):
        diag = np.diag(Z)[a * m:(a + 1) * m]
        assert np.allclose(z0[a, idx], vv[a, idx] / diag, rtol=1e-12, atol=0)
    P = unet.init_params(3)
    z1 = unet.apply_preconditioner(P, g, er, sg, f, v)
    z2 = unet.apply_preconditioner(P, g, er, sg, f, 7.5 * v)
    assert np.linalg.norm(z2 - 7.5 * z1) <= 1e-12 * np.linalg.norm(z2)
    # the network's correction is present on material voxels only
    assert np.linalg.norm((z1.reshape(3, g.nv) - z0)[:, vac]) == 0.0
    assert np.linalg.norm((z1.reshape(3, g.nv) - z0)[:, ~vac]) > 0.0
