"""RWG basis functions on a triangle mesh, and quadrature rules.

Sec. II.B: coil currents are expanded in Rao-Wilton-Glisson (RWG) functions,
one per interior edge (Eq. disc_sie).  For edge m of length l shared by T+ and
T- with free vertices v+ and v-:
    f_m(r) = l / (2 A+) (r - v+)  on T+,    f_m(r) = l / (2 A-) (v- - r)  on T-,
    div f_m = +l / A+  on T+,               div f_m = -l / A-  on T-.

Conventions fixed here (the paper leaves them to MARIE): interior edges are
ordered by (smaller vertex id, larger vertex id); T+ is the adjacent triangle
with the smaller triangle index.  A port (vertex pair) drives its edge with the
reference direction T+ -> T-, and its right-hand side is i omega eps0 V l.

Quadrature rules (published tables, written out here):
  * TRI6: Dunavant degree-4, 6 points (the paper's "5 surface points" reading);
  * TRI7: Radon degree-5, 7 points (outer rule of singular pairs);
  * TRI1: centroid;
  * HEX8: 2 x 2 x 2 Gauss-Legendre in a voxel (the paper's "8 volume points").
Weights are normalised to sum to 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _sym3(a, b):
    """The 3 permutations of barycentric (a, b, b)."""
    return [(a, b, b), (b, a, b), (b, b, a)]


TRI1 = (np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0]))
TRI6 = (
    np.array(_sym3(0.108103018168070, 0.445948490915965)
             + _sym3(0.816847572980459, 0.091576213509771)),
    np.array([0.223381589678011] * 3 + [0.109951743655322] * 3),
)
TRI7 = (
    np.array([(1 / 3, 1 / 3, 1 / 3)]
             + _sym3(0.059715871789770, 0.470142064105115)
             + _sym3(0.797426985353087, 0.101286507323456)),
    np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3),
)
_gl = 1.0 / np.sqrt(3.0)
HEX8 = (
    np.array([(sx * _gl / 2, sy * _gl / 2, sz * _gl / 2)
              for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)]),  # in units of h
    np.full(8, 1.0 / 8.0),
)


@dataclass
class RWG:
    xyz: np.ndarray        # (nverts, 3)
    tri: np.ndarray        # (ntris, 3)
    edges: np.ndarray      # (m, 2) vertex ids, sorted
    tplus: np.ndarray      # (m,)
    tminus: np.ndarray     # (m,)
    vplus: np.ndarray      # (m,) free vertex of T+
    vminus: np.ndarray     # (m,) free vertex of T-
    length: np.ndarray     # (m,)
    area: np.ndarray       # (ntris,)
    centroid: np.ndarray   # (ntris, 3)
    normal: np.ndarray     # (ntris, 3) unit normals from the vertex order
    diam: np.ndarray       # (ntris,) longest edge
    ports: np.ndarray      # (nports,) edge index of each port

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])


def build(mesh) -> RWG:
    xyz = np.asarray(mesh.xyz, np.float64)
    tri = np.asarray(mesh.tri, np.int64)
    emap = {}
    for t in range(tri.shape[0]):
        for k in range(3):
            a, b = tri[t, (k + 1) % 3], tri[t, (k + 2) % 3]
            key = (min(a, b), max(a, b))
            emap.setdefault(key, []).append((t, tri[t, k]))
    keys = sorted(k for k, v in emap.items() if len(v) == 2)
    m = len(keys)
    edges = np.array(keys, np.int64).reshape(m, 2)
    tp = np.zeros(m, np.int64)
    tm = np.zeros(m, np.int64)
    vp = np.zeros(m, np.int64)
    vm = np.zeros(m, np.int64)
    for i, k in enumerate(keys):
        (t0, f0), (t1, f1) = sorted(emap[k])
        tp[i], vp[i], tm[i], vm[i] = t0, f0, t1, f1
    P = xyz[tri]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    normal = cr / (2 * area[:, None])
    cen = P.mean(1)
    el = np.stack([np.linalg.norm(P[:, 1] - P[:, 0], axis=1),
                   np.linalg.norm(P[:, 2] - P[:, 1], axis=1),
                   np.linalg.norm(P[:, 0] - P[:, 2], axis=1)], 1)
    length = np.linalg.norm(xyz[edges[:, 0]] - xyz[edges[:, 1]], axis=1)
    index = {k: i for i, k in enumerate(keys)}
    ports = np.array([index[(min(a, b), max(a, b))] for a, b in np.asarray(mesh.ports)],
                     np.int64)
    return RWG(xyz, tri, edges, tp, tm, vp, vm, length, area, cen, normal, el.max(1), ports)


def tri_points(rw: RWG, t, rule):
    """Quadrature points (len(t), q, 3) and weights times area (len(t), q)."""
    bary, w = rule
    P = rw.xyz[rw.tri[np.atleast_1d(t)]]         # (k, 3, 3)
    pts = np.einsum("qj,kjd->kqd", bary, P)
    return pts, w[None, :] * rw.area[np.atleast_1d(t)][:, None]


def halves(rw: RWG, m):
    """For RWG m, the two (triangle, sign, free vertex) triples: sign +1 on T+,
    -1 on T-, so that f = sign * l / (2 A) (r - v) and div f = sign * l / A."""
    return ((int(rw.tplus[m]), 1.0, int(rw.vplus[m])),
            (int(rw.tminus[m]), -1.0, int(rw.vminus[m])))


def rhs_ports(rw: RWG, omega, eps0, V=1.0):
    """Delta-gap right-hand sides, one column per port: i omega eps0 V l_m."""
    b = np.zeros((rw.m, rw.ports.size), np.complex128)
    for j, e in enumerate(rw.ports):
        b[e, j] = 1j * omega * eps0 * V * rw.length[e]
    return b
