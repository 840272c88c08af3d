"""Hybrid-VSIE operator parts and matvec (Sec. III, Eq. hvsie and Eq. hvsie_disc).

Unknowns are ordered [j_f; j_n; j_b] (far surface RWG, near surface RWG, body
voxel currents component-major over the body grid), Eq. (hvsie).  With
K_ij = <f_i, Gop f_j> the system is Z = D - K (D = h^3 / chi on material voxels,
identity rows/columns on vacuum voxels).  The hybrid representation of
Eq. (hvsie_disc):

  * Z_ff                      dense (far-far Galerkin block);
  * U V^H ~= Z_cc^fn          ACA of the near-far block (m_n x m_f); its
                              transpose conj(V) U^T in the far rows;
  * TT(Z_cb^{f,chi})          one TT per component chi over (n1, n2, n3, m_f) of
                              the unmasked far coupling (1 x 1 point), applied
                              by Eq. (mvp) and its transpose by Eq. (tmvp);
  * Z^pFFT                    body + near coil on the extended grid: the FFT
                              convolution c = K_grid (E_b M x_b + P x_n) with
                              K_grid = h^3 T* (voxel Galerkin testing), the
                              precorrection matrix (Z form) on near pairs and the
                              dense coil block  Znn~ = -(K_nn - P^T K_grid P).

Matvec, for material body rows (vacuum rows return x):
  y_b = h^3 x_b / chi - E_b^T c + Pre x_n + TT(x_f)
  y_n = -P^T c + Znn~ x_n + Pre^T (M x_b) + U V^H x_f
  y_f = Z_ff x_f + conj(V) U^T x_n + TT^T(M x_b)

`dense_operator` assembles the same system without compression (direct 8 x 6
point near coupling, 1 x 1 far coupling, dense volume block): the reference the
hybrid approximates.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import physics, volume, rwg, efie, coupling, pfft, aca, tt


@dataclass
class Parts:
    body: object          # inputs.Grid
    ext: object           # inputs.Grid (extended pFFT grid)
    ext_offset: tuple
    chi: np.ndarray       # (n_b,) complex susceptibility on the body grid
    k0: float
    omega: float
    s: int
    W: np.ndarray         # (m_n, 3 s^3) projection weights, (b, q) order
    base: np.ndarray      # (m_n, 3) stencil lowest-corner indices on the ext grid
    pre: object           # scipy.sparse (3 n_b, m_n), Z form (= -S)
    Znn: np.ndarray       # (m_n, m_n) Z form (= -(K_nn - P^T K_grid P))
    U: np.ndarray         # (m_n, k)
    V: np.ndarray         # (m_f, k)
    Zff: np.ndarray       # (m_f, m_f)
    tt: list              # 3 lists of 4 cores (Z form)
    spec: np.ndarray      # (6, L1, L2, L3) ext-grid kernel spectra

    @property
    def m_f(self):
        return self.Zff.shape[0]

    @property
    def m_n(self):
        return self.W.shape[0]

    @property
    def N(self):
        return self.m_f + self.m_n + 3 * self.body.nv


def body_to_ext_index(body, ext_n, offset):
    n1, n2, n3 = body.n
    v = np.arange(body.nv)
    i1, i2, i3 = v % n1, (v // n1) % n2, v // (n1 * n2)
    e1, e2, _ = ext_n
    return (i1 + offset[0]) + e1 * ((i2 + offset[1]) + e2 * (i3 + offset[2]))


def build_parts(prob, near=None, rfac=pfft.RFAC, s=None):
    """All compressed parts for a Problem (coil and shield required)."""
    omega, k0 = physics.omega_k0(prob.freq_hz)
    body = prob.grid
    ext = prob.ext_grid
    s = prob.stencil if s is None else s
    near = s + 1 if near is None else near
    chi = physics.chi(prob.eps_r, prob.sigma, prob.freq_hz)
    mat = volume.material_mask(chi)
    rwn = rwg.build(prob.coil)
    rwf = rwg.build(prob.shield)
    spec = volume.kernel_spectra(ext.n, ext.h, k0)
    # projection
    W, base = pfft.projection(ext, rwn, np.arange(rwn.m), s, k0, rfac=rfac)
    ic = base + (s - 1) // 2
    # precorrection on near (material voxel, RWG) pairs
    lists = pfft.near_pairs(body, prob.ext_offset, ic, mat, near)
    b2e = body_to_ext_index(body, ext.n, prob.ext_offset)
    h3 = body.h ** 3
    rows, cols, vals = [], [], []
    nb = body.nv
    for n, vox in enumerate(lists):
        if vox.size == 0:
            continue
        Kd = coupling.K_block(body, vox, rwn, [n], k0, near=True)[:, :, 0]   # (3, v)
        Kg = h3 * pfft.grid_times_P(ext, W, base, s, k0, b2e[vox], [n])[:, :, 0]
        S = Kd - Kg
        for a in range(3):
            rows.append(a * nb + vox)
            cols.append(np.full(vox.size, n))
            vals.append(-S[a])
    if rows:
        pre = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                            shape=(3 * nb, rwn.m))
    else:
        pre = sp.csr_matrix((3 * nb, rwn.m), dtype=np.complex128)
    # coil block with the grid part folded out
    Knn = efie.K_dense(rwn, rwn, k0, True)
    gP = pfft.scatter(ext, W, base, s, np.eye(rwn.m))
    PtKP = pfft.gather(ext, W, base, s, h3 * volume.conv(spec, ext.n, gP))
    Znn = -(Knn - PtKP)
    # near-far ACA and far-far dense
    Kfn = efie.K_dense(rwn, rwf, k0, False)       # (m_n, m_f)
    U, V = aca.aca_dense(-Kfn, prob.aca_tol)
    Zff = -efie.K_dense(rwf, rwf, k0, True)
    # TT of the far coupling per component
    Kbf = coupling.K_block(body, np.arange(nb), rwf, np.arange(rwf.m), k0, near=False)
    cores = []
    for a in range(3):
        T = (-Kbf[a]).reshape(tuple(body.n) + (rwf.m,), order="F")
        cores.append(tt.tt_svd(T, prob.tt_tol))
    return Parts(body, ext, tuple(prob.ext_offset), chi, k0, omega, s, W, base, pre,
                 Znn, U, V, Zff, cores, spec)


def matvec(P: Parts, x):
    x = np.asarray(x, np.complex128).reshape(P.N, -1)
    mf, mn, nb = P.m_f, P.m_n, P.body.nv
    xf, xn, xb = x[:mf], x[mf:mf + mn], x[mf + mn:]
    mat = volume.material_mask(P.chi)
    M3 = np.tile(mat, 3)[:, None]
    xbm = np.where(M3, xb, 0.0)
    nve = P.ext.nv
    b2e = body_to_ext_index(P.body, P.ext.n, P.ext_offset)
    g = pfft.scatter(P.ext, P.W, P.base, P.s, xn)
    for a in range(3):
        g[a * nve + b2e] += xbm[a * nb:(a + 1) * nb]
    h3 = P.body.h ** 3
    c = h3 * volume.conv(P.spec, P.ext.n, g)
    cb = np.concatenate([c[a * nve + b2e] for a in range(3)], 0)
    invchi = np.zeros(nb, np.complex128)
    invchi[mat] = 1.0 / P.chi[mat]
    ttf = np.concatenate([tt.tt_matvec(P.tt[a], xf) for a in range(3)], 0)
    yb = h3 * np.tile(invchi, 3)[:, None] * xb - cb + P.pre @ xn + ttf
    yb = np.where(M3, yb, xb)
    yn = -pfft.gather(P.ext, P.W, P.base, P.s, c) + P.Znn @ xn + P.pre.T @ xbm \
        + P.U @ (P.V.conj().T @ xf)
    ttb = sum(tt.tt_rmatvec(P.tt[a], xbm[a * nb:(a + 1) * nb]) for a in range(3))
    yf = P.Zff @ xf + P.V.conj() @ (P.U.T @ xn) + ttb
    return np.concatenate([yf, yn, yb], 0)


def dense_operator(prob):
    """Uncompressed reference Z on [j_f; j_n; j_b(material voxels)] and the
    material voxel index list."""
    omega, k0 = physics.omega_k0(prob.freq_hz)
    body = prob.grid
    chi = physics.chi(prob.eps_r, prob.sigma, prob.freq_hz)
    rwn = rwg.build(prob.coil)
    rwf = rwg.build(prob.shield)
    Zbb, idx = volume.dense_Zbb(body, chi, k0)
    Kbn = coupling.K_block(body, idx, rwn, np.arange(rwn.m), k0, near=True)
    Kbf = coupling.K_block(body, idx, rwf, np.arange(rwf.m), k0, near=False)
    Kbn = Kbn.reshape(3 * idx.size, rwn.m)
    Kbf = Kbf.reshape(3 * idx.size, rwf.m)
    Knn = efie.K_dense(rwn, rwn, k0, True)
    Knf = efie.K_dense(rwn, rwf, k0, False)
    Kff = efie.K_dense(rwf, rwf, k0, True)
    Z = np.block([[-Kff, -Knf.T, -Kbf.T],
                  [-Knf, -Knn, -Kbn.T],
                  [-Kbf, -Kbn, Zbb]])
    return Z, idx


def dense_matvec(prob, Z, idx, x):
    x = np.asarray(x, np.complex128)
    x = x.reshape(x.shape[0], -1)
    mf = rwg.build(prob.shield).m
    mn = rwg.build(prob.coil).m
    nb = prob.grid.nv
    sel = np.concatenate([np.arange(mf + mn)] + [mf + mn + a * nb + idx for a in range(3)])
    y = x.copy()
    y[sel] = Z @ x[sel]
    return y
