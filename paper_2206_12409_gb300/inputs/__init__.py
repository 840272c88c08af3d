"""Seeded synthetic inputs for the hybrid-VSIE workloads.

This module generates *inputs only*: voxel grids with tissue maps, triangle meshes
of coils and shields, port edges and random test vectors.  It holds none of the
method's arithmetic (no Green's function, no basis functions, no quadrature), so
both the CUDA library and the CPU oracle can consume what it produces.

The workloads stand in for the paper's Billie/Duke head models and coil meshes
(Sec. IV.A-B), which are not available: a homogeneous sphere with a loop and a
closed cylindrical shield, and layered ellipsoid heads with a loop array and a
shield/bore cylinder.

Geometry is in metres.  Voxel index order is i1 fastest (i1 + n1*(i2 + n2*i3)),
matching the column-major reshapes of Eq. (mvp).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Grid", "Mesh", "Problem",
    "sphere_phantom", "layered_head_phantom",
    "loop_strip", "closed_cylinder", "open_cylinder", "loop_array_on_cylinder",
    "merge_meshes", "random_vectors", "problem_sphere_loop_shield",
    "problem_head", "problem_volume_only", "problem_coil_array_mid", "problem_head_1mm",
    "problem_two_loops",
]


@dataclass
class Grid:
    """Uniform voxel grid: n = (n1, n2, n3) voxels of edge h, voxel (0,0,0)
    centred at ``origin``."""
    n: tuple
    h: float
    origin: tuple

    @property
    def nv(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def centres(self) -> np.ndarray:
        """(nv, 3) voxel centres, i1 fastest."""
        i1, i2, i3 = np.meshgrid(np.arange(self.n[0]), np.arange(self.n[1]),
                                 np.arange(self.n[2]), indexing="ij")
        idx = np.stack([i1.ravel(order="F"), i2.ravel(order="F"),
                        i3.ravel(order="F")], -1)
        return np.asarray(self.origin)[None, :] + self.h * idx


@dataclass
class Mesh:
    """Triangle mesh: ``xyz`` (nverts, 3) float64, ``tri`` (ntris, 3) int32 and
    ``ports`` (nports, 2) int32 vertex pairs naming the port edges."""
    xyz: np.ndarray
    tri: np.ndarray
    ports: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))

    @property
    def nverts(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def ntris(self) -> int:
        return int(self.tri.shape[0])


@dataclass
class Problem:
    """A complete hybrid-VSIE workload description (inputs only)."""
    name: str
    grid: Grid                 # body grid
    eps_r: np.ndarray          # (nv,) relative permittivity, i1 fastest
    sigma: np.ndarray          # (nv,) conductivity S/m
    freq_hz: float
    coil: Mesh | None = None   # near-domain conductors (pFFT)
    shield: Mesh | None = None  # far-domain conductors (TT / dense)
    ext_n: tuple | None = None  # extended pFFT grid size (contains the body grid)
    ext_offset: tuple = (0, 0, 0)  # body grid offset inside the extended grid
    stencil: int = 3
    tt_tol: float = 1e-6
    aca_tol: float = 1e-6
    nrhs: int = 1

    @property
    def ext_grid(self) -> Grid:
        if self.ext_n is None:
            return self.grid
        o = np.asarray(self.grid.origin) - self.grid.h * np.asarray(self.ext_offset)
        return Grid(tuple(int(v) for v in self.ext_n), self.grid.h, tuple(o.tolist()))


# --------------------------------------------------------------------------- grids

def _centred_grid(n, h) -> Grid:
    n = tuple(int(v) for v in n)
    origin = tuple(-(ni - 1) * h / 2.0 for ni in n)
    return Grid(n, float(h), origin)


def sphere_phantom(n=(12, 12, 12), h=5e-3, radius=25e-3, eps_r=50.0, sigma=0.6,
                   centre=(0.0, 0.0, 0.0)):
    """Homogeneous sphere; a voxel is inside when its centre is."""
    g = _centred_grid(n, h)
    c = g.centres() - np.asarray(centre)[None, :]
    inside = np.einsum("ij,ij->i", c, c) <= radius * radius
    er = np.where(inside, eps_r, 1.0)
    sg = np.where(inside, sigma, 0.0)
    return g, er.astype(np.float64), sg.astype(np.float64)


def _real_sph_harm(lmax: int, theta: np.ndarray, phi: np.ndarray) -> list:
    """Real spherical harmonics up to degree lmax (l >= 1), orthonormal on S^2.
    Returns a list of arrays, one per (l, m)."""
    from scipy.special import lpmv
    out = []
    ct = np.cos(theta)
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) *
                             math.factorial(l - am) / math.factorial(l + am))
            p = lpmv(am, l, ct) * ((-1) ** am)  # undo Condon-Shortley phase
            if m == 0:
                out.append(norm * p)
            elif m > 0:
                out.append(math.sqrt(2.0) * norm * p * np.cos(am * phi))
            else:
                out.append(math.sqrt(2.0) * norm * p * np.sin(am * phi))
    return out


def layered_head_phantom(n=(96, 96, 112), h=2e-3, semi_axes=(80e-3, 95e-3, 110e-3),
                         shells=(5e-3, 10e-3),
                         tissues=((50.0, 0.55), (15.0, 0.07), (80.0, 2.2)),
                         rms=3e-3, lmax=6, seed=0):
    """Layered ellipsoid head: tissue 0 fills the outer shell of thickness
    shells[0], tissue 1 the next shells[1], tissue 2 the core.  All boundaries
    carry one seeded real spherical-harmonic radial displacement (degrees
    1..lmax) scaled to ``rms`` metres RMS over the sphere."""
    g = _centred_grid(n, h)
    c = g.centres()
    r = np.sqrt(np.einsum("ij,ij->i", c, c))
    rs = np.where(r > 0, r, 1.0)
    u = c / rs[:, None]
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    a, b, cc = semi_axes
    rho_e = 1.0 / np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2 + (u[:, 2] / cc) ** 2)
    rng = np.random.default_rng(seed)
    ylm = _real_sph_harm(lmax, theta, phi)
    coef = rng.standard_normal(len(ylm))
    # orthonormal basis: mean square over the sphere = sum(coef^2) / (4 pi)
    coef *= rms / math.sqrt(np.sum(coef ** 2) / (4 * math.pi))
    delta = np.zeros_like(r)
    for cf, y in zip(coef, ylm):
        delta += cf * y
    bound0 = rho_e + delta
    bound1 = bound0 - shells[0]
    bound2 = bound1 - shells[1]
    er = np.ones_like(r)
    sg = np.zeros_like(r)
    t0 = r <= bound0
    t1 = r <= bound1
    t2 = r <= bound2
    for mask, (e, s) in ((t0, tissues[0]), (t1, tissues[1]), (t2, tissues[2])):
        er = np.where(mask, e, er)
        sg = np.where(mask, s, sg)
    return g, er, sg


# --------------------------------------------------------------------------- meshes

def loop_strip(radius=40e-3, width=2e-3, n_seg=128, z=0.0):
    """Planar circular strip loop in the plane z = const, one quad across the
    strip (2 triangles per segment).  The port is the rung edge at phi = 0."""
    phi = 2 * np.pi * np.arange(n_seg) / n_seg
    ri, ro = radius - width / 2, radius + width / 2
    inner = np.stack([ri * np.cos(phi), ri * np.sin(phi), np.full(n_seg, z)], -1)
    outer = np.stack([ro * np.cos(phi), ro * np.sin(phi), np.full(n_seg, z)], -1)
    xyz = np.concatenate([inner, outer], 0)
    tri = []
    for i in range(n_seg):
        j = (i + 1) % n_seg
        tri.append((i, n_seg + i, n_seg + j))
        tri.append((i, n_seg + j, j))
    ports = np.array([[0, n_seg]], np.int32)
    return Mesh(xyz.astype(np.float64), np.asarray(tri, np.int32), ports)


def closed_cylinder(radius=0.1, length=0.2, n_theta=32, n_z=7, n_rings=5):
    """Closed cylinder about the z axis centred at the origin: side of n_theta x
    n_z quads, end caps made of a centre fan plus (n_rings - 1) annular rings of
    2*n_theta triangles each.  1024 triangles for the defaults."""
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    zs = np.linspace(-length / 2, length / 2, n_z + 1)
    verts = []
    side = np.zeros((n_z + 1, n_theta), np.int64)
    for k, z in enumerate(zs):
        for i in range(n_theta):
            side[k, i] = len(verts)
            verts.append((radius * np.cos(th[i]), radius * np.sin(th[i]), z))
    tri = []
    for k in range(n_z):
        for i in range(n_theta):
            j = (i + 1) % n_theta
            a, b, c, d = side[k, i], side[k, j], side[k + 1, j], side[k + 1, i]
            tri.append((a, b, c))
            tri.append((a, c, d))
    radii = radius * np.arange(1, n_rings) / n_rings  # inner ring radii

    def cap(z, rim, flip):
        rings = [rim]
        for rr in radii[::-1]:
            ids = []
            for i in range(n_theta):
                ids.append(len(verts))
                verts.append((rr * np.cos(th[i]), rr * np.sin(th[i]), z))
            rings.append(np.asarray(ids))
        centre = len(verts)
        verts.append((0.0, 0.0, z))
        for q in range(len(rings) - 1):
            o, inn = rings[q], rings[q + 1]
            for i in range(n_theta):
                j = (i + 1) % n_theta
                t1, t2 = (o[i], o[j], inn[j]), (o[i], inn[j], inn[i])
                tri.append(t1[::-1] if flip else t1)
                tri.append(t2[::-1] if flip else t2)
        inn = rings[-1]
        for i in range(n_theta):
            j = (i + 1) % n_theta
            t = (inn[i], inn[j], centre)
            tri.append(t[::-1] if flip else t)

    cap(zs[-1], side[n_z], False)
    cap(zs[0], side[0], True)
    return Mesh(np.asarray(verts, np.float64), np.asarray(tri, np.int32))


def open_cylinder(radius=0.33, length=1.2, n_theta=125, n_z=80):
    """Open cylinder (shield/bore) about the z axis: 2*n_theta*n_z triangles."""
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    zs = np.linspace(-length / 2, length / 2, n_z + 1)
    T, Z = np.meshgrid(th, zs)
    xyz = np.stack([radius * np.cos(T).ravel(), radius * np.sin(T).ravel(), Z.ravel()], -1)
    tri = []
    for k in range(n_z):
        for i in range(n_theta):
            j = (i + 1) % n_theta
            a, b = k * n_theta + i, k * n_theta + j
            c, d = (k + 1) * n_theta + j, (k + 1) * n_theta + i
            tri.append((a, b, c))
            tri.append((a, c, d))
    return Mesh(xyz.astype(np.float64), np.asarray(tri, np.int32))


def _rounded_rect_path(wu, hv, rc, n):
    """n points, evenly spaced in arclength, on a rounded rectangle of width wu,
    height hv and corner radius rc centred at (0, 0); returns points and unit
    outward normals in the (u, v) plane."""
    su, sv = wu - 2 * rc, hv - 2 * rc
    perim = 2 * su + 2 * sv + 2 * np.pi * rc
    s = perim * np.arange(n) / n
    pts = np.zeros((n, 2))
    nrm = np.zeros((n, 2))
    segs = [
        ("line", (-su / 2, -hv / 2), (1.0, 0.0), su, (0.0, -1.0)),
        ("arc", (su / 2, -sv / 2), -np.pi / 2, None, None),
        ("line", (wu / 2, -sv / 2), (0.0, 1.0), sv, (1.0, 0.0)),
        ("arc", (su / 2, sv / 2), 0.0, None, None),
        ("line", (su / 2, hv / 2), (-1.0, 0.0), su, (0.0, 1.0)),
        ("arc", (-su / 2, sv / 2), np.pi / 2, None, None),
        ("line", (-wu / 2, sv / 2), (0.0, -1.0), sv, (-1.0, 0.0)),
        ("arc", (-su / 2, -sv / 2), np.pi, None, None),
    ]
    lens = [sg[3] if sg[0] == "line" else np.pi * rc / 2 for sg in segs]
    starts = np.concatenate([[0.0], np.cumsum(lens)])
    for k, sk in enumerate(s):
        q = min(np.searchsorted(starts, sk, side="right") - 1, len(segs) - 1)
        t = sk - starts[q]
        sg = segs[q]
        if sg[0] == "line":
            p0, d, _, nn = np.asarray(sg[1]), np.asarray(sg[2]), sg[3], np.asarray(sg[4])
            pts[k] = p0 + t * d
            nrm[k] = nn
        else:
            cen, a0 = np.asarray(sg[1]), sg[2]
            ang = a0 + t / rc
            nrm[k] = (np.cos(ang), np.sin(ang))
            pts[k] = cen + rc * nrm[k]
    return pts, nrm


def loop_array_on_cylinder(n_loops=8, radius=0.12, height=0.1, width=3e-3,
                           gap=8e-3, corner=10e-3, n_seg=256, z0=0.0):
    """n_loops rounded-rectangle strip loops conformal to a cylinder of the
    given radius (axis z), evenly spaced in azimuth.  Each loop has n_seg
    segments of 2 triangles; its port is the rung edge of segment 0."""
    arc = 2 * np.pi * radius / n_loops - gap
    pts, nrm = _rounded_rect_path(arc, height, corner, n_seg)
    meshes = []
    for L in range(n_loops):
        phi0 = 2 * np.pi * L / n_loops
        ui = pts - nrm * width / 2
        uo = pts + nrm * width / 2

        def wrap(uv):
            ang = phi0 + uv[:, 0] / radius
            return np.stack([radius * np.cos(ang), radius * np.sin(ang), z0 + uv[:, 1]], -1)
        xyz = np.concatenate([wrap(ui), wrap(uo)], 0)
        tri = []
        for i in range(n_seg):
            j = (i + 1) % n_seg
            tri.append((i, n_seg + i, n_seg + j))
            tri.append((i, n_seg + j, j))
        meshes.append(Mesh(xyz, np.asarray(tri, np.int32),
                           np.array([[0, n_seg]], np.int32)))
    return merge_meshes(meshes)


def merge_meshes(meshes):
    xyz, tri, ports = [], [], []
    off = 0
    for m in meshes:
        xyz.append(m.xyz)
        tri.append(m.tri + off)
        ports.append(m.ports + off)
        off += m.nverts
    return Mesh(np.concatenate(xyz, 0), np.concatenate(tri, 0).astype(np.int32),
                np.concatenate(ports, 0).astype(np.int32))


# --------------------------------------------------------------------------- vectors

def random_vectors(N: int, p: int = 1, seed: int = 12409, dtype=np.complex128):
    """x ~ CN(0, 1) i.i.d., shape (N, p), column-major semantics."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((N, p)) + 1j * rng.standard_normal((N, p))) / math.sqrt(2.0)
    return x.astype(dtype)


# --------------------------------------------------------------------------- problems

def problem_volume_only(n=(12, 12, 12), h=5e-3, radius=25e-3, eps_r=50.0, sigma=0.6,
                        freq_hz=298e6):
    g, er, sg = sphere_phantom(n, h, radius, eps_r, sigma)
    return Problem("volume", g, er, sg, freq_hz)


def problem_sphere_loop_shield(n_body=(12, 12, 12), h=5e-3, freq_hz=298e6,
                               ext_n=(20, 20, 12), tt_tol=1e-6, aca_tol=1e-6,
                               loop_radius=40e-3, loop_width=2e-3, loop_seg=128,
                               shield_radius=0.1, shield_length=0.2):
    """Sphere r = 25 mm (eps_r 50, sigma 0.6) on a 12^3 5 mm grid, a 2 mm strip loop
    of radius 40 mm (256 triangles) and a closed cylinder shield r = 100 mm,
    L = 200 mm (1024 triangles)."""
    g, er, sg = sphere_phantom(n_body, h, 25e-3, 50.0, 0.6)
    coil = loop_strip(loop_radius, loop_width, loop_seg)
    shield = closed_cylinder(shield_radius, shield_length)
    off = tuple((e - b) // 2 for e, b in zip(ext_n, n_body))
    return Problem("sphere_loop_shield", g, er, sg, freq_hz, coil, shield,
                   tuple(ext_n), off, 3, tt_tol, aca_tol, 1)


def problem_head(n_body=(96, 96, 112), h=2e-3, freq_hz=298e6, ext_n=(128, 128, 112),
                 n_loops=8, loop_seg=256, shield_theta=125, shield_z=80,
                 tt_tol=1e-5, aca_tol=1e-5, seed=0, nrhs=8):
    """Head-size workload: layered ellipsoid head on a 2 mm grid, an n_loops strip
    loop array (512 triangles per loop) and a shield/bore cylinder r = 0.33 m,
    L = 1.2 m (2*shield_theta*shield_z triangles)."""
    g, er, sg = layered_head_phantom(n_body, h, seed=seed)
    coil = loop_array_on_cylinder(n_loops=n_loops, n_seg=loop_seg)
    shield = open_cylinder(0.33, 1.2, shield_theta, shield_z)
    off = tuple((e - b) // 2 for e, b in zip(ext_n, n_body))
    return Problem("head", g, er, sg, freq_hz, coil, shield, tuple(ext_n), off, 3,
                   tt_tol, aca_tol, nrhs)


def problem_coil_array_mid(n_body=(18, 18, 24), h=5e-3, freq_hz=298e6, ext_n=(26, 26, 24),
                           n_loops=4, loop_seg=128, tt_tol=1e-6, aca_tol=1e-6, seed=3, nrhs=8):
    """Mid-size workload with the structure of the head workload at a size the
    oracle assembles in about a minute: a layered ellipsoid (semi-axes
    40/40/52 mm, 5 mm and 10 mm shells, 2 mm RMS perturbation) on an 18 x 18 x 24
    grid at 5 mm; a 4-loop strip array on a 55 mm cylinder (1024 triangles, 1024
    RWG, 4 ports) close enough to the body for precorrection pairs; a closed
    cylinder shield r = 0.1 m, L = 0.2 m of 1216 triangles (1824 RWG, not a
    multiple of 256); extended grid 26 x 26 x 24 (FFT lengths 54, 54, 48)."""
    g, er, sg = layered_head_phantom(n_body, h, (40e-3, 40e-3, 52e-3), (5e-3, 10e-3),
                                     rms=2e-3, seed=seed)
    coil = loop_array_on_cylinder(n_loops=n_loops, radius=0.055, height=0.08, width=3e-3,
                                  gap=8e-3, corner=10e-3, n_seg=loop_seg)
    shield = closed_cylinder(0.1, 0.2, n_theta=32, n_z=10, n_rings=5)
    off = tuple((e - b) // 2 for e, b in zip(ext_n, n_body))
    return Problem("coil_array_mid", g, er, sg, freq_hz, coil, shield, tuple(ext_n), off, 3,
                   tt_tol, aca_tol, nrhs)


def problem_head_1mm(freq_hz=298e6, seed=0, nrhs=16):
    """Head at 1 mm: the layered ellipsoid family of problem_head on a
    192 x 192 x 224 grid (the same 192 x 192 x 224 mm box; 2.48e7 body unknowns),
    a 16-loop strip array on the 0.12 m cylinder (512 triangles per loop, 8192 in
    all, 16 ports) on the 256 x 256 x 224 extended grid, and the shield/bore
    cylinder r = 0.33 m, L = 1.2 m of 40,000 triangles (200 x 100 quads); TT and
    ACA tolerance 1e-5; one right-hand side per port."""
    return problem_head(n_body=(192, 192, 224), h=1e-3, freq_hz=freq_hz, ext_n=(256, 256, 224),
                        n_loops=16, loop_seg=256, shield_theta=200, shield_z=100, tt_tol=1e-5,
                        aca_tol=1e-5, seed=seed, nrhs=nrhs)


def problem_two_loops(freq_hz=298e6):
    """Port-network case: a 6^3 sphere at 10 mm (r = 25 mm, eps_r 50, sigma 0.6),
    two strip loops on a 40 mm cylinder (32 segments each, 2 ports) and a small
    closed cylinder shield, on a 12 x 12 x 6 extended grid; TT and ACA at 1e-6."""
    g, er, sg = sphere_phantom((6, 6, 6), 10e-3, 25e-3, 50.0, 0.6)
    coil = loop_array_on_cylinder(n_loops=2, radius=0.04, height=0.03, width=3e-3, gap=10e-3,
                                  corner=6e-3, n_seg=32)
    shield = closed_cylinder(0.1, 0.2, n_theta=8, n_z=2, n_rings=2)
    return Problem("two loops", g, er, sg, freq_hz, coil, shield, (12, 12, 6), (3, 3, 0), 3,
                   1e-6, 1e-6, 2)
