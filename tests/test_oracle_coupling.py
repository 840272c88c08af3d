"""Direct pins of the oracle's body-surface coupling (oracle/coupling.py, Sec. II.B
Eq. (nvsie), the 8 volume points of Sec. IV.C):

  * K_block(near=True), the 2 x 2 x 2 Gauss voxel rule times the 6-point
    triangle rule, against a 10^3-point Gauss-Legendre voxel rule of the same
    field on a 64-fold refined triangle rule: the error falls like (h/d)^4 with
    the voxel-RWG distance d, the rate of a product rule exact for cubics (a
    misplaced node would fall like (h/d)^2);
  * reciprocity: the voxel-tested field of f_n (the charge form of Gop used by
    the oracle) equals the RWG-tested field of a uniform current in the voxel,
    computed instead from the dyadic Green's function (k0^2 + grad grad) g;
  * K_block(near=False), the one-point voxel and triangle rules of the far
    coupling (Sec. IV.C: 1 volume and 1 surface point for Z_bc^f), against the
    same high-order reference: within 1e-3 at 5 voxel widths and 3e-4 beyond 10
    (a dropped term or a wrong sign of the grad-div part is an O(1) error).
"""
import numpy as np
import pytest

from oracle import coupling, physics, rwg
from paper_2206_12409_gb300 import inputs as I

H = 5e-3


def _composite(rule, levels):
    bary, w = rule
    sub = [np.eye(3)]
    for _ in range(levels):
        nxt = []
        for B in sub:
            a, b, c = B
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        sub = nxt
    return np.concatenate([bary @ B for B in sub]), np.concatenate([w / len(sub)] * len(sub))


def _gauss_voxel(n):
    """n^3 Gauss-Legendre points in units of h about the centre; weights sum to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    X, Y, Z = np.meshgrid(x / 2, x / 2, x / 2, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1), np.einsum("i,j,k->ijk", w / 2, w / 2, w / 2).ravel()


@pytest.fixture(scope="module")
def setup():
    _, k0 = physics.omega_k0(298e6)
    rw = rwg.build(I.loop_strip(40e-3, 2e-3, 128))
    n = 5
    cen = 0.5 * (rw.centroid[rw.tplus[n]] + rw.centroid[rw.tminus[n]])
    return rw, n, cen, k0, _composite(rwg.TRI6, 3)


def _reference(rw, n, c, k0, fine, nq=10):
    xi, wv = _gauss_voxel(nq)
    E = coupling.gop_rwg(rw, [n], c[None, :] + H * xi, fine, k0)[:, 0, :]
    return H ** 3 * np.einsum("q,qa->a", wv, E)


def _k8(rw, n, c, k0):
    return coupling.K_block(I.Grid((1, 1, 1), H, tuple(c)), [0], rw, [n], k0, near=True)[:, 0, 0]


@pytest.mark.parametrize("direction", [(0.0, 0.0, 1.0), (1.0, 0.3, 0.2)])
def test_near_coupling_against_high_order_cubature(setup, direction):
    rw, n, cen, k0, fine = setup
    u = np.asarray(direction) / np.linalg.norm(direction)
    err = {}
    for d in (3.0, 6.0):
        c = cen + d * H * u
        ref = _reference(rw, n, c, k0, fine)
        err[d] = np.linalg.norm(_k8(rw, n, c, k0) - ref) / np.linalg.norm(ref)
    assert err[6.0] <= 2e-4 and err[3.0] <= 3e-3, err
    assert err[3.0] / err[6.0] >= 10.0, err          # (h/d)^4 decay: 16 at a factor 2


@pytest.mark.parametrize("d", [1.0, 2.0, 6.0])
def test_reciprocity_voxel_and_rwg_testing(setup, d):
    rw, n, cen, k0, fine = setup
    c = cen + d * H * np.array([1.0, 0.3, 0.2]) / np.linalg.norm([1.0, 0.3, 0.2])
    ref = _reference(rw, n, c, k0, fine)                     # int_V Gop f_n dV (charge form)
    xi, wv = _gauss_voxel(10)
    vp = c[None, :] + H * xi
    rec = np.zeros(3, complex)
    for t_arr, s, v_arr in ((rw.tplus, 1.0, rw.vplus), (rw.tminus, -1.0, rw.vminus)):
        t = t_arr[n]
        q = fine[0] @ rw.xyz[rw.tri[t]]
        wq = fine[1] * rw.area[t]
        f = s * rw.length[n] / (2 * rw.area[t]) * (q - rw.xyz[v_arr[n]])
        D = physics.dyad((q[:, None, :] - vp[None, :, :]).reshape(-1, 3), k0)
        D = D.reshape(q.shape[0], vp.shape[0], 3, 3)
        rec += H ** 3 * np.einsum("s,v,svab,sb->a", wq, wv, D, f)   # int_S f_n . E_voxel dS
    assert np.linalg.norm(rec - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,tol", [(5.0, 1e-3), (10.0, 3e-4), (20.0, 3e-4)])
def test_far_coupling_one_point_rule(setup, d, tol):
    rw, n, cen, k0, fine = setup
    u = np.array([1.0, 0.3, 0.2]) / np.linalg.norm([1.0, 0.3, 0.2])
    c = cen + d * H * u
    ref = _reference(rw, n, c, k0, fine, nq=6)
    kf = coupling.K_block(I.Grid((1, 1, 1), H, tuple(c)), [0], rw, [n], k0, near=False)[:, 0, 0]
    assert np.linalg.norm(kf - ref) <= tol * np.linalg.norm(ref)
