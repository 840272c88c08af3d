"""Pins of the oracle's plane-wave right-hand side (oracle/rhs.py) against what
the mathematics fixes: the closed form of an RWG integral in a uniform field, a
refined quadrature at 298 MHz, and the body right-hand side of the Mie check."""
import numpy as np

from oracle import mie, physics, rhs, rwg
from paper_2206_12409_gb300 import inputs as I


def _shapes():
    return [I.loop_strip(40e-3, 2e-3, 64), I.closed_cylinder(0.1, 0.2, 16, 4, 3)]


def test_uniform_field_closed_form():
    """k0 = 0: E_inc = e0 everywhere, and the integral of f_m over its support
    is (l/2)[(c+ - v+) - (c- - v-)] (c the centroids, v the free vertices)."""
    e0 = np.array([0.3, -1.1, 0.7])
    for mesh in _shapes():
        rw = rwg.build(mesh)
        got = rhs.tested_incident(rw, [0, 0, 1], e0, 0.0)
        cp, cm = rw.centroid[rw.tplus], rw.centroid[rw.tminus]
        vp, vm = rw.xyz[rw.vplus], rw.xyz[rw.vminus]
        ref = (rw.length / 2) * (((cp - vp) - (cm - vm)) @ e0)
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def _refined(rw, k_hat, e0, k0, levels):
    """The same integrals with every triangle split into 4**levels congruent
    sub-triangles, each integrated by the 6-point rule."""
    bary, w = rwg.TRI6
    sub = [np.eye(3)]
    for _ in range(levels):
        nxt = []
        for B in sub:
            a, b, c = B
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        sub = nxt
    out = np.zeros(rw.m, complex)
    for t_arr, s, v_arr in ((rw.tplus, 1.0, rw.vplus), (rw.tminus, -1.0, rw.vminus)):
        P = rw.xyz[rw.tri[t_arr]]                          # (m, 3, 3)
        for B in sub:
            q = np.einsum("qj,jk,mkd->mqd", bary, B, P)     # sub-triangle points
            E = rhs.incident(q.reshape(-1, 3), k_hat, e0, k0).reshape(q.shape)
            f = (s * rw.length / (2 * rw.area[t_arr]))[:, None, None] * (q - rw.xyz[v_arr][:, None, :])
            wq = (rw.area[t_arr] / len(sub))[:, None] * w[None, :]
            out += np.einsum("mq,mqd,mqd->m", wq, f, E)
    return out


def test_refined_quadrature_at_298mhz():
    _, k0 = physics.omega_k0(298e6)
    k_hat, e0 = np.array([0.6, 0.0, 0.8]), np.array([0.8, 0.0, -0.6])
    for mesh in _shapes():
        rw = rwg.build(mesh)
        got = rhs.tested_incident(rw, k_hat, e0, k0)
        r2, r3 = _refined(rw, k_hat, e0, k0, 2), _refined(rw, k_hat, e0, k0, 3)
        scale = np.max(np.abs(r3))
        assert np.max(np.abs(r3 - r2)) <= 1e-9 * scale      # the refinement has converged
        assert np.max(np.abs(got - r3)) <= 1e-6 * scale     # degree-4 rule on cm triangles


def test_body_part_is_the_mie_rhs():
    prob = I.problem_volume_only()
    b = rhs.planewave(prob, [0, 0, 1], [1, 0, 0])
    assert np.array_equal(b.shape, (3 * prob.grid.nv,))
    ref = mie.body_rhs(prob.grid, prob.eps_r, prob.sigma, prob.freq_hz)
    assert np.max(np.abs(b - ref)) <= 1e-15 * np.max(np.abs(ref))
