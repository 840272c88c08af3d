"""Learned right preconditioner for the body block: a small 3D U-Net.

This part is not in the paper.  The paper names only the Calderon-type idea of
preconditioning the coupled system (Sec. VI).  The network is this package's
FP64 reference for the GPU network: a plain, slow restatement of the forward
pass, its gradients (reverse-mode, written out layer by layer) and one Adam
step, in NumPy.

Architecture (4 levels, 16/32/64/64 channels, 3x3x3 convolutions, zero "same"
padding, ReLU, 2x2x2 average pooling, nearest x2 upsampling, skips concatenated
after the upsampled tensor):

    e1a 8->16, e1b 16->16 (skip s1) | pool | e2a 16->32, e2b 32->32 (s2) | pool |
    e3a 32->64, e3b 64->64 (s3) | pool | ba 64->64, bb 64->64 | up, cat s3 |
    d3a 128->64, d3b 64->64 | up, cat s2 | d2a 96->32, d2b 32->32 | up, cat s1 |
    d1a 48->16, d1b 16->16 | head 1x1x1 16->6 (linear)

Tensors are (C, D, H, W) with the body grid's i1 as W (fastest), i2 as H,
i3 as D.  Weights are (Cout, Cin, k, k, k), biases (Cout,).

Input channels: the six real parts (re, im of components x, y, z) of the
Jacobi-scaled residual u = D^-1 r divided by its RMS s, then (eps_r - 1) / 50
and sigma (S/m).  Output y (6 channels): the correction, so that the
preconditioner returns e = u + s y (y = 0 is the Jacobi preconditioner).

Pinned by: a 3x3x3 convolution against scipy.signal.correlate and a brute-force
loop, and every gradient against central finite differences
(tests/test_oracle_unet.py).
"""
from __future__ import annotations

import numpy as np

LAYERS = (
    ("e1a", 8, 16, 3), ("e1b", 16, 16, 3),
    ("e2a", 16, 32, 3), ("e2b", 32, 32, 3),
    ("e3a", 32, 64, 3), ("e3b", 64, 64, 3),
    ("ba", 64, 64, 3), ("bb", 64, 64, 3),
    ("d3a", 128, 64, 3), ("d3b", 64, 64, 3),
    ("d2a", 96, 32, 3), ("d2b", 32, 32, 3),
    ("d1a", 48, 16, 3), ("d1b", 16, 16, 3),
    ("head", 16, 6, 1),
)


def conv3d(x, w, b):
    """y[o] = b[o] + sum_i sum_t w[o, i, t] x[i, shifted by t - k//2] (zero outside)."""
    C, D, H, W = x.shape
    O, I, k = w.shape[0], w.shape[1], w.shape[2]
    r = k // 2
    xp = np.zeros((C, D + 2 * r, H + 2 * r, W + 2 * r), x.dtype)
    xp[:, r:r + D, r:r + H, r:r + W] = x
    y = np.broadcast_to(b[:, None, None, None], (O, D, H, W)).astype(np.result_type(x, w)).copy()
    for kz in range(k):
        for ky in range(k):
            for kx in range(k):
                patch = xp[:, kz:kz + D, ky:ky + H, kx:kx + W]          # (I, D, H, W)
                y += np.tensordot(w[:, :, kz, ky, kx], patch, axes=(1, 0))
    return y


def conv3d_backward(x, w, dy):
    """Gradients of sum(dy * conv3d(x, w, b)) with respect to x, w and b."""
    C, D, H, W = x.shape
    k = w.shape[2]
    r = k // 2
    xp = np.zeros((C, D + 2 * r, H + 2 * r, W + 2 * r), x.dtype)
    xp[:, r:r + D, r:r + H, r:r + W] = x
    dxp = np.zeros_like(xp, dtype=np.result_type(dy, w))
    dw = np.zeros(w.shape, np.result_type(dy, x))
    for kz in range(k):
        for ky in range(k):
            for kx in range(k):
                patch = xp[:, kz:kz + D, ky:ky + H, kx:kx + W]
                dw[:, :, kz, ky, kx] = np.tensordot(dy, patch, axes=((1, 2, 3), (1, 2, 3)))
                dxp[:, kz:kz + D, ky:ky + H, kx:kx + W] += np.tensordot(w[:, :, kz, ky, kx], dy,
                                                                        axes=(0, 0))
    db = dy.sum(axis=(1, 2, 3))
    return dxp[:, r:r + D, r:r + H, r:r + W], dw, db


def pool(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_backward(dy):
    C, D, H, W = dy.shape
    return dy.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def init_params(seed=0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, k in LAYERS:
        P[name + ".w"] = rng.standard_normal((co, ci, k, k, k)) * np.sqrt(2.0 / (ci * k ** 3))
        P[name + ".b"] = np.zeros(co)
    return P


def forward(P, x):
    """Returns (y, tape) where tape holds what backward needs."""
    t = {}

    def cr(name, a):
        z = conv3d(a, P[name + ".w"], P[name + ".b"])
        t[name] = (a, z)
        return np.maximum(z, 0.0)

    a = cr("e1a", x)
    s1 = cr("e1b", a)
    a = cr("e2a", pool(s1))
    s2 = cr("e2b", a)
    a = cr("e3a", pool(s2))
    s3 = cr("e3b", a)
    a = cr("ba", pool(s3))
    a = cr("bb", a)
    a = cr("d3a", np.concatenate([up(a), s3]))
    a = cr("d3b", a)
    a = cr("d2a", np.concatenate([up(a), s2]))
    a = cr("d2b", a)
    a = cr("d1a", np.concatenate([up(a), s1]))
    a = cr("d1b", a)
    y = conv3d(a, P["head.w"], P["head.b"])
    t["head"] = (a, y)
    return y, t


def backward(P, tape, dy):
    """Gradients of sum(dy * forward(P, x)) with respect to every parameter and x."""
    G = {}

    def cb(name, g, relu=True):
        a, z = tape[name]
        if relu:
            g = g * (z > 0)
        da, dw, db = conv3d_backward(a, P[name + ".w"], g)
        G[name + ".w"] = dw
        G[name + ".b"] = db
        return da

    g = cb("head", dy, relu=False)
    g = cb("d1b", g)
    g = cb("d1a", g)
    gu, gs1 = g[:32], g[32:]
    g = cb("d2b", up_backward(gu))
    g = cb("d2a", g)
    gu, gs2 = g[:64], g[64:]
    g = cb("d3b", up_backward(gu))
    g = cb("d3a", g)
    gu, gs3 = g[:64], g[64:]
    g = cb("bb", up_backward(gu))
    g = cb("ba", g)
    g = cb("e3b", pool_backward(g) + gs3)
    g = cb("e3a", g)
    g = cb("e2b", pool_backward(g) + gs2)
    g = cb("e2a", g)
    g = cb("e1b", pool_backward(g) + gs1)
    gx = cb("e1a", g)
    return G, gx


def loss_and_grad(P, x, target):
    """Mean squared error over all output entries and its gradients."""
    y, tape = forward(P, x)
    diff = y - target
    L = float(np.mean(diff * diff))
    G, _ = backward(P, tape, 2.0 * diff / diff.size)
    return L, G


def adam_step(P, G, M, V, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) in place; t counts from 1."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def apply_preconditioner(P, grid, eps_r, sigma, freq_hz, v_body):
    """The learned right preconditioner on the body block (the application step of
    the network inside flexible GMRES), for one body vector v (component-major,
    3 n_v complex):
        u = D^-1 v    with D the diagonal of Z_bb: h^3 (1/chi - T(0)) on material
                      voxels, 1 on vacuum voxels (identity rows),
        s = RMS(u)    over all 3 n_v entries,
        y = net([Re u_a / s, Im u_a / s (a = x, y, z); (eps_r - 1) / 50; sigma])
                      on the grid padded to multiples of 8 (zeros outside),
        z_a = u_a + s (y_2a + i y_2a+1)   on material voxels,  z_a = u_a  on vacuum.
    Pinned through unet.forward (see the tests of this module) and the definition
    of the body diagonal in volume.dense_Zbb."""
    from . import physics
    n1, n2, n3 = grid.n
    nv = n1 * n2 * n3
    chi = physics.chi(eps_r, sigma, freq_hz)
    _, k0 = physics.omega_k0(freq_hz)
    mat = chi != 0
    d = np.ones(nv, np.complex128)
    d[mat] = 1.0 / (grid.h ** 3 * (1.0 / chi[mat] - physics.self_term(k0, grid.h)))
    u = np.asarray(v_body, np.complex128).reshape(3, nv) * d[None, :]
    s = np.sqrt(np.sum(np.abs(u) ** 2) / (3 * nv))
    pad = lambda n: (n + 7) // 8 * 8
    D, H, W = pad(n3), pad(n2), pad(n1)
    x = np.zeros((8, D, H, W))
    cube = lambda f: f.reshape(n3, n2, n1)          # voxel i1 + n1 (i2 + n2 i3) -> [i3, i2, i1]
    for a in range(3):
        x[2 * a, :n3, :n2, :n1] = cube(u[a].real) / s
        x[2 * a + 1, :n3, :n2, :n1] = cube(u[a].imag) / s
    x[6, :n3, :n2, :n1] = cube((np.asarray(eps_r, float) - 1.0) / 50.0)
    x[7, :n3, :n2, :n1] = cube(np.asarray(sigma, float))
    y, _ = forward(P, x)
    z = u.copy()
    for a in range(3):
        corr = (y[2 * a, :n3, :n2, :n1] + 1j * y[2 * a + 1, :n3, :n2, :n1]).reshape(nv)
        z[a, mat] += s * corr[mat]
    return z.reshape(-1)
