"""ctypes binding of libvsie (include/vsie.h): argument marshalling only.

Function names match the C ABI.  Device buffers are passed as integer device
pointers (for example ``tensor.data_ptr()``) with leading dimensions in complex
elements; streams as integer ``cudaStream_t`` handles (0 = default stream).
Every computation runs inside libvsie; when the library cannot be loaded the
calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvsie.so")

VSIE_OK, VSIE_EINVAL, VSIE_ENOMEM, VSIE_ECUDA, VSIE_ENOCONV, VSIE_EBREAKDOWN, \
    VSIE_ETIMEOUT, VSIE_EUNSUPPORTED = range(8)
VSIE_C128, VSIE_C64 = 0, 1
STATUS_NAMES = {0: "VSIE_OK", 1: "VSIE_EINVAL", 2: "VSIE_ENOMEM", 3: "VSIE_ECUDA",
                4: "VSIE_ENOCONV", 5: "VSIE_EBREAKDOWN", 6: "VSIE_ETIMEOUT",
                7: "VSIE_EUNSUPPORTED"}

EXPORTS = ["vsie_last_error", "vsie_version", "vsie_setup", "vsie_create", "vsie_sizes",
           "vsie_matvec", "vsie_rhs_ports", "vsie_rhs_planewave", "vsie_rhs_drive", "vsie_set_loads", "vsie_port_network",
           "vsie_solve", "vsie_save", "vsie_load",
           "vsie_get_parts", "vsie_profile", "vsie_profile_query", "vsie_volume_matvec_static",
           "vsie_net_create", "vsie_net_num_params", "vsie_net_set_params", "vsie_net_get_params",
           "vsie_net_forward", "vsie_net_backward", "vsie_net_step", "vsie_net_train",
           "vsie_net_attach", "vsie_precond_apply", "vsie_net_last_error", "vsie_net_destroy",
           "vsie_solve_batch", "vsie_destroy"]
PROFILE_GROUPS = {"fft_conv": 0, "pfft": 1, "precorrection": 2, "surface": 3, "tt": 4,
                  "krylov": 5, "precond": 6, "fft_conv_c128": 7}


class VsieError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vsie_grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("origin", C.c_double * 3)]


class vsie_mesh(C.Structure):
    _fields_ = [("nverts", C.c_int32), ("xyz", C.POINTER(C.c_double)), ("ntris", C.c_int32),
                ("tri", C.POINTER(C.c_int32)), ("nports", C.c_int32),
                ("ports", C.POINTER(C.c_int32))]


class vsie_options(C.Structure):
    _fields_ = [("ext_n", C.c_int32 * 3), ("ext_offset", C.c_int32 * 3), ("stencil", C.c_int32),
                ("near_radius", C.c_int32), ("colloc_rfac", C.c_double), ("tt_tol", C.c_double),
                ("aca_tol", C.c_double), ("max_rhs", C.c_int32), ("precisions", C.c_int32),
                ("far_hmatrix", C.c_int32), ("hm_leaf", C.c_int32), ("hm_eta", C.c_double),
                ("dense_gemm", C.c_int32), ("reserved", C.c_int32)]


class vsie_parts(C.Structure):
    _fields_ = [("m_f", C.c_int32), ("m_n", C.c_int32), ("stencil", C.c_int32),
                ("W", C.c_void_p), ("base", C.c_void_p), ("pre_nnz", C.c_int64),
                ("pre_rowptr", C.c_void_p), ("pre_col", C.c_void_p), ("pre_val", C.c_void_p),
                ("Znn", C.c_void_p), ("aca_rank", C.c_int32), ("U", C.c_void_p),
                ("V", C.c_void_p), ("Zff", C.c_void_p), ("tt_rank", (C.c_int32 * 3) * 3),
                ("tt_core", (C.c_void_p * 4) * 3)]


class vsie_solve_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("precond", C.c_int32)]


class vsie_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32 * 64), ("relres", C.c_double * 64), ("outer", C.c_int32),
                ("matvecs64", C.c_int32), ("matvecs32", C.c_int32), ("seconds", C.c_double)]


_lib = None


def load_library(path: str | None = None):
    """Load libvsie (built in-tree by paper_2206_12409_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libvsie not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.vsie_last_error.restype = C.c_char_p
    lib.vsie_last_error.argtypes = [P]
    lib.vsie_version.restype = C.c_char_p
    lib.vsie_version.argtypes = []
    lib.vsie_setup.restype = C.c_int
    lib.vsie_setup.argtypes = [C.POINTER(vsie_grid), C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(vsie_mesh), C.POINTER(vsie_mesh), C.c_double,
                               C.POINTER(vsie_options), C.POINTER(P)]
    lib.vsie_create.restype = C.c_int
    lib.vsie_create.argtypes = [C.POINTER(vsie_grid), C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.c_double, C.POINTER(vsie_options),
                                C.POINTER(vsie_parts), C.POINTER(P)]
    lib.vsie_sizes.restype = C.c_int
    lib.vsie_sizes.argtypes = [P] + [C.POINTER(C.c_int64)] * 4
    lib.vsie_matvec.restype = C.c_int
    lib.vsie_matvec.argtypes = [P, C.c_int32, P, C.c_int64, P, C.c_int64, C.c_int32, P]
    lib.vsie_rhs_ports.restype = C.c_int
    lib.vsie_rhs_ports.argtypes = [P, C.c_int32, C.POINTER(C.c_int32), C.c_double, P, C.c_int64, P]
    lib.vsie_rhs_planewave.restype = C.c_int
    lib.vsie_rhs_planewave.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double), P, P]
    lib.vsie_set_loads.restype = C.c_int
    lib.vsie_set_loads.argtypes = [P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.vsie_port_network.restype = C.c_int
    lib.vsie_port_network.argtypes = [P, C.c_int32, C.POINTER(C.c_int32), P, C.c_int64, C.c_double,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.vsie_solve.restype = C.c_int
    lib.vsie_solve.argtypes = [P, C.c_int32, P, C.c_int64, P, C.c_int64, C.c_double,
                               C.POINTER(vsie_solve_opts), C.POINTER(vsie_solve_info), P]
    lib.vsie_save.restype = C.c_int
    lib.vsie_save.argtypes = [P, C.c_char_p]
    lib.vsie_load.restype = C.c_int
    lib.vsie_load.argtypes = [C.c_char_p, C.POINTER(P)]
    lib.vsie_get_parts.restype = C.c_int
    lib.vsie_get_parts.argtypes = [P, C.POINTER(vsie_parts)]
    lib.vsie_profile.restype = C.c_int
    lib.vsie_profile.argtypes = [P, C.c_int32]
    lib.vsie_profile_query.restype = C.c_int
    lib.vsie_profile_query.argtypes = [P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_double)]
    lib.vsie_volume_matvec_static.restype = C.c_int
    lib.vsie_volume_matvec_static.argtypes = [P, C.c_int32, P, C.c_int64, P, C.c_int64, C.c_int32, P]
    lib.vsie_destroy.restype = None
    lib.vsie_destroy.argtypes = [P]
    F = C.POINTER(C.c_float)
    lib.vsie_net_create.restype = C.c_int
    lib.vsie_net_create.argtypes = [C.c_uint64, C.POINTER(P)]
    lib.vsie_net_num_params.restype = C.c_int
    lib.vsie_net_num_params.argtypes = [P, C.POINTER(C.c_int64)]
    lib.vsie_net_set_params.restype = C.c_int
    lib.vsie_net_set_params.argtypes = [P, F, C.c_int64]
    lib.vsie_net_get_params.restype = C.c_int
    lib.vsie_net_get_params.argtypes = [P, F, C.c_int64]
    lib.vsie_net_forward.restype = C.c_int
    lib.vsie_net_forward.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P]
    lib.vsie_net_backward.restype = C.c_int
    lib.vsie_net_backward.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, F, P, P]
    lib.vsie_net_step.restype = C.c_int
    lib.vsie_net_step.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_double,
                                  C.POINTER(C.c_double), P]
    lib.vsie_net_train.restype = C.c_int
    lib.vsie_net_train.argtypes = [P, P, C.c_int32, C.c_double, C.c_uint64, F, P]
    lib.vsie_solve_batch.restype = C.c_int
    lib.vsie_solve_batch.argtypes = [C.c_int32, C.POINTER(P), C.POINTER(C.c_int32), C.POINTER(P),
                                     C.POINTER(C.c_int64), C.POINTER(P), C.POINTER(C.c_int64), C.c_double,
                                     C.POINTER(vsie_solve_opts), C.POINTER(vsie_solve_info),
                                     C.POINTER(C.c_int), C.c_int32]
    lib.vsie_precond_apply.restype = C.c_int
    lib.vsie_precond_apply.argtypes = [P, C.c_int32, P, C.c_int64, P, C.c_int64, C.c_int32, P]
    lib.vsie_net_attach.restype = C.c_int
    lib.vsie_net_attach.argtypes = [P, P]
    lib.vsie_net_last_error.restype = C.c_char_p
    lib.vsie_net_last_error.argtypes = [P]
    lib.vsie_net_destroy.restype = None
    lib.vsie_net_destroy.argtypes = [P]
    _lib = lib
    return lib


def _check(st, ctx=None):
    if st != VSIE_OK:
        lib = load_library()
        msg = lib.vsie_last_error(ctx)
        raise VsieError(st, msg.decode() if msg else "")


def _dptr(a):
    return C.cast(a.ctypes.data, C.POINTER(C.c_double))


def _iptr(a):
    return C.cast(a.ctypes.data, C.POINTER(C.c_int32))


def make_grid(n, h, origin):
    g = vsie_grid()
    for i in range(3):
        g.n[i] = int(n[i])
        g.origin[i] = float(origin[i])
    g.h = float(h)
    return g


def make_mesh(xyz, tri, ports=None):
    """vsie_mesh over numpy arrays; returns (struct, keep-alive tuple)."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    ports = np.ascontiguousarray(np.zeros((0, 2)) if ports is None else ports, np.int32)
    m = vsie_mesh(xyz.shape[0], _dptr(xyz), tri.shape[0], _iptr(tri), ports.shape[0], _iptr(ports))
    return m, (xyz, tri, ports)


def make_options(ext_n=None, ext_offset=None, stencil=0, near_radius=0, colloc_rfac=0.0,
                 tt_tol=0.0, aca_tol=0.0, max_rhs=0, precisions=0, far_hmatrix=0, hm_leaf=0,
                 hm_eta=0.0, dense_gemm=0):
    o = vsie_options()
    for i in range(3):
        o.ext_n[i] = int(ext_n[i]) if ext_n is not None else 0
        o.ext_offset[i] = int(ext_offset[i]) if ext_offset is not None else 0
    o.stencil, o.near_radius, o.colloc_rfac = int(stencil), int(near_radius), float(colloc_rfac)
    o.tt_tol, o.aca_tol, o.max_rhs, o.precisions = float(tt_tol), float(aca_tol), int(max_rhs), \
        int(precisions)
    o.far_hmatrix, o.hm_leaf, o.hm_eta = int(far_hmatrix), int(hm_leaf), float(hm_eta)
    o.dense_gemm = int(dense_gemm)
    return o


def make_parts(m_f=0, m_n=0, stencil=3, W=None, base=None, pre_rowptr=None, pre_col=None,
               pre_val=None, Znn=None, U=None, V=None, Zff=None, tt=None):
    """vsie_parts over numpy arrays (complex arrays as complex128, column-major
    matrices, TT cores per component as [G1, G2, G3, G4]); returns (struct,
    keep-alive list)."""
    keep = []

    def cplx(a, order="F"):
        a = np.asarray(a, np.complex128)
        a = np.asfortranarray(a) if order == "F" else np.ascontiguousarray(a)
        keep.append(a)
        return C.c_void_p(a.ctypes.data)

    p = vsie_parts()
    p.m_f, p.m_n, p.stencil = int(m_f), int(m_n), int(stencil)
    if m_n:
        p.W = cplx(W, "C")
        b = np.ascontiguousarray(base, np.int32)
        keep.append(b)
        p.base = C.c_void_p(b.ctypes.data)
        p.Znn = cplx(Znn)
        if pre_val is not None and len(pre_val):
            rp = np.ascontiguousarray(pre_rowptr, np.int64)
            pc = np.ascontiguousarray(pre_col, np.int32)
            keep += [rp, pc]
            p.pre_nnz = int(len(pre_val))
            p.pre_rowptr = C.c_void_p(rp.ctypes.data)
            p.pre_col = C.c_void_p(pc.ctypes.data)
            p.pre_val = cplx(pre_val, "C")
    if m_f:
        p.Zff = cplx(Zff)
        if U is not None and U.shape[1] > 0 and m_n:
            p.aca_rank = int(U.shape[1])
            p.U = cplx(U)
            p.V = cplx(V)
        if tt is not None:
            for a in range(3):
                G1, G2, G3, G4 = tt[a]
                p.tt_rank[a][0], p.tt_rank[a][1], p.tt_rank[a][2] = \
                    int(G1.shape[1]), int(G2.shape[2]), int(G3.shape[2])
                for q, G in enumerate((G1, G2, G3, G4)):
                    p.tt_core[a][q] = cplx(G)
    return p, keep


def vsie_version():
    return load_library().vsie_version().decode()


def vsie_setup(grid, eps_r, sigma, coil, shield, freq_hz, opts=None):
    lib = load_library()
    er = np.ascontiguousarray(eps_r, np.float64)
    sg = np.ascontiguousarray(sigma, np.float64)
    out = C.c_void_p()
    st = lib.vsie_setup(C.byref(grid), _dptr(er), _dptr(sg),
                        C.byref(coil) if coil is not None else None,
                        C.byref(shield) if shield is not None else None, float(freq_hz),
                        C.byref(opts) if opts is not None else None, C.byref(out))
    _check(st)
    return out


def vsie_create(grid, eps_r, sigma, freq_hz, opts=None, parts=None):
    lib = load_library()
    er = np.ascontiguousarray(eps_r, np.float64)
    sg = np.ascontiguousarray(sigma, np.float64)
    out = C.c_void_p()
    st = lib.vsie_create(C.byref(grid), _dptr(er), _dptr(sg), float(freq_hz),
                         C.byref(opts) if opts is not None else None,
                         C.byref(parts) if parts is not None else None, C.byref(out))
    _check(st)
    return out


def vsie_sizes(ctx):
    lib = load_library()
    v = [C.c_int64() for _ in range(4)]
    _check(lib.vsie_sizes(ctx, *[C.byref(x) for x in v]), ctx)
    return tuple(int(x.value) for x in v)


def vsie_matvec(ctx, p, X, ldx, Y, ldy, precision, stream=0):
    lib = load_library()
    _check(lib.vsie_matvec(ctx, int(p), C.c_void_p(int(X)), int(ldx), C.c_void_p(int(Y)),
                           int(ldy), int(precision), C.c_void_p(int(stream))), ctx)


def vsie_rhs_ports(ctx, ports, V, B, ldb, stream=0):
    lib = load_library()
    pr = (C.c_int32 * len(ports))(*[int(x) for x in ports])
    _check(lib.vsie_rhs_ports(ctx, len(ports), pr, float(V), C.c_void_p(int(B)), int(ldb),
                              C.c_void_p(int(stream))), ctx)


def vsie_rhs_planewave(ctx, k_hat, e0, B, stream=0):
    """One plane-wave right-hand side column into device pointer B (N double2)."""
    lib = load_library()
    kh = (C.c_double * 3)(*[float(v) for v in k_hat])
    ev = (C.c_double * 3)(*[float(v) for v in e0])
    _check(lib.vsie_rhs_planewave(ctx, kh, ev, C.c_void_p(int(B)), C.c_void_p(int(stream))), ctx)


def vsie_rhs_drive(ctx, ports, v, B, stream=0):
    """One column B (device, N double2) with ports[i] driven by the complex voltage v[i]."""
    vv = np.asarray(v, np.complex128).ravel()
    pr = (C.c_int32 * max(len(ports), 1))(*[int(x) for x in ports])
    buf = np.ascontiguousarray(np.stack([vv.real, vv.imag], -1).ravel(), np.float64)
    _check(load_library().vsie_rhs_drive(ctx, len(ports), pr, _dptr(buf), C.c_void_p(int(B)),
                                         C.c_void_p(int(stream))), ctx)


def cp_mode_voltages(n):
    """Drive voltages of the circularly polarised mode of an n-loop array (1 V each)."""
    return np.exp(-2j * np.pi * np.arange(n) / n)


def vsie_set_loads(ctx, ports, z_load):
    """Lumped loads: z_load complex ohms in series with the listed port edges."""
    z = np.asarray(z_load, np.complex128).ravel()
    pr = (C.c_int32 * max(len(ports), 1))(*[int(x) for x in ports])
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], -1).ravel(), np.float64)
    _check(load_library().vsie_set_loads(ctx, len(ports), pr, _dptr(zz) if len(ports) else None), ctx)


def vsie_port_network(ctx, ports, X, ldx, z0=50.0):
    """Y, Z, S (numpy complex, nports x nports) from the solutions X (device)."""
    n = len(ports)
    pr = (C.c_int32 * n)(*[int(x) for x in ports])
    out = [np.zeros(2 * n * n, np.float64) for _ in range(3)]
    _check(load_library().vsie_port_network(ctx, n, pr, C.c_void_p(int(X)), int(ldx), float(z0),
                                             *[_dptr(o) for o in out]), ctx)
    return tuple(o.view(np.complex128).reshape(n, n, order="F") for o in out)


def vsie_solve(ctx, p, B, ldb, X, ldx, tol, opts=None, stream=0, check=True):
    """Returns (status, vsie_solve_info)."""
    lib = load_library()
    info = vsie_solve_info()
    st = lib.vsie_solve(ctx, int(p), C.c_void_p(int(B)), int(ldb), C.c_void_p(int(X)), int(ldx),
                        float(tol), C.byref(opts) if opts is not None else None, C.byref(info),
                        C.c_void_p(int(stream)))
    if check and st not in (VSIE_OK, VSIE_ENOCONV):
        _check(st, ctx)
    return st, info


def vsie_save(ctx, path):
    _check(load_library().vsie_save(ctx, str(path).encode()), ctx)


def vsie_load(path):
    out = C.c_void_p()
    _check(load_library().vsie_load(str(path).encode(), C.byref(out)))
    return out


def vsie_get_parts(ctx):
    p = vsie_parts()
    _check(load_library().vsie_get_parts(ctx, C.byref(p)), ctx)
    return p


def vsie_profile(ctx, enable):
    _check(load_library().vsie_profile(ctx, int(bool(enable))), ctx)


def vsie_profile_query(ctx, group):
    """Returns (ms, launches, alg_bytes) of a kernel group (-1: all launches)."""
    ms, n, b = C.c_double(), C.c_int64(), C.c_double()
    _check(load_library().vsie_profile_query(ctx, int(group), C.byref(ms), C.byref(n), C.byref(b)),
           ctx)
    return ms.value, n.value, b.value


def vsie_volume_matvec_static(ctx, p, X, ldx, Y, ldy, precision, stream=0):
    """Body operator without allocation (see include/vsie.h)."""
    lib = load_library()
    _check(lib.vsie_volume_matvec_static(ctx, int(p), C.c_void_p(int(X)), int(ldx),
                                         C.c_void_p(int(Y)), int(ldy), int(precision),
                                         C.c_void_p(int(stream))), ctx)


def vsie_destroy(ctx):
    if ctx:
        load_library().vsie_destroy(ctx)


def parts_to_numpy(ctx, body_n):
    """Copy the context's operator parts into numpy arrays (dict)."""
    p = vsie_get_parts(ctx)

    def carr(ptr, n):
        if not ptr or n == 0:
            return np.zeros(0, np.complex128)
        buf = (C.c_double * (2 * n)).from_address(ptr)
        return np.frombuffer(buf, np.float64).copy().view(np.complex128)

    def iarr(ptr, n, ct=C.c_int32, dt=np.int32):
        if not ptr or n == 0:
            return np.zeros(0, dt)
        return np.frombuffer((ct * n).from_address(ptr), dt).copy()

    n1, n2, n3 = body_n
    nb = n1 * n2 * n3
    out = {"m_f": p.m_f, "m_n": p.m_n, "stencil": p.stencil}
    s3 = p.stencil ** 3
    if p.m_n:
        out["W"] = carr(p.W, p.m_n * 3 * s3).reshape(p.m_n, 3 * s3)
        out["base"] = iarr(p.base, p.m_n * 3).reshape(p.m_n, 3)
        out["Znn"] = carr(p.Znn, p.m_n * p.m_n).reshape(p.m_n, p.m_n, order="F")
        out["pre_nnz"] = p.pre_nnz
        if p.pre_nnz:
            out["pre_rowptr"] = iarr(p.pre_rowptr, 3 * nb + 1, C.c_int64, np.int64)
            out["pre_col"] = iarr(p.pre_col, p.pre_nnz)
            out["pre_val"] = carr(p.pre_val, p.pre_nnz)
    if p.m_f:
        out["Zff"] = carr(p.Zff, p.m_f * p.m_f).reshape(p.m_f, p.m_f, order="F")
        k = p.aca_rank
        out["U"] = carr(p.U, p.m_n * k).reshape(p.m_n, k, order="F")
        out["V"] = carr(p.V, p.m_f * k).reshape(p.m_f, k, order="F")
        tt = []
        for a in range(3):
            r1, r2, r3 = p.tt_rank[a][0], p.tt_rank[a][1], p.tt_rank[a][2]
            if r1 == 0:
                tt.append(None)
                continue
            tt.append([carr(p.tt_core[a][0], n1 * r1).reshape(n1, r1, order="F"),
                       carr(p.tt_core[a][1], r1 * n2 * r2).reshape(r1, n2, r2, order="F"),
                       carr(p.tt_core[a][2], r2 * n3 * r3).reshape(r2, n3, r3, order="F"),
                       carr(p.tt_core[a][3], r3 * p.m_f).reshape(r3, p.m_f, order="F")])
        out["tt"] = tt
    return out


def setup_problem(prob, max_rhs=8, precisions=0, far_hmatrix=0, hm_leaf=0, hm_eta=0.0, dense_gemm=0):
    """vsie_setup for an inputs.Problem (geometry marshalling only)."""
    g = prob.grid
    coil = shield = None
    keep = []
    if prob.coil is not None:
        coil, k1 = make_mesh(prob.coil.xyz, prob.coil.tri, prob.coil.ports)
        keep.append(k1)
    if prob.shield is not None:
        shield, k2 = make_mesh(prob.shield.xyz, prob.shield.tri, prob.shield.ports)
        keep.append(k2)
    opts = make_options(ext_n=prob.ext_n, ext_offset=prob.ext_offset, stencil=prob.stencil,
                        tt_tol=prob.tt_tol, aca_tol=prob.aca_tol, max_rhs=max_rhs,
                        precisions=precisions, far_hmatrix=far_hmatrix, hm_leaf=hm_leaf,
                        hm_eta=hm_eta, dense_gemm=dense_gemm)
    return vsie_setup(make_grid(g.n, g.h, g.origin), prob.eps_r, prob.sigma, coil, shield,
                      prob.freq_hz, opts)


# ------------------------------------------------------------- learned preconditioner
def _check_net(st, net):
    if st != VSIE_OK:
        lib = load_library()
        msg = lib.vsie_net_last_error(net) if net else lib.vsie_last_error(None)
        raise VsieError(st, msg.decode() if msg else "")


def vsie_net_create(seed=0):
    lib = load_library()
    out = C.c_void_p()
    _check(lib.vsie_net_create(int(seed), C.byref(out)))
    return out


def vsie_net_num_params(net):
    n = C.c_int64()
    _check_net(load_library().vsie_net_num_params(net, C.byref(n)), net)
    return n.value


def vsie_net_set_params(net, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check_net(load_library().vsie_net_set_params(net, a.ctypes.data_as(C.POINTER(C.c_float)), a.size), net)


def vsie_net_get_params(net):
    a = np.empty(vsie_net_num_params(net), np.float32)
    _check_net(load_library().vsie_net_get_params(net, a.ctypes.data_as(C.POINTER(C.c_float)), a.size), net)
    return a


def vsie_net_forward(net, D, H, W, x_ptr, y_ptr, stream=0):
    _check_net(load_library().vsie_net_forward(net, int(D), int(H), int(W), C.c_void_p(int(x_ptr)),
                                               C.c_void_p(int(y_ptr)), C.c_void_p(int(stream))), net)


def vsie_net_backward(net, D, H, W, x_ptr, dy_ptr, dx_ptr=0, stream=0):
    """Returns the packed parameter gradients (host)."""
    g = np.empty(vsie_net_num_params(net), np.float32)
    _check_net(load_library().vsie_net_backward(net, int(D), int(H), int(W), C.c_void_p(int(x_ptr)),
                                                C.c_void_p(int(dy_ptr)),
                                                g.ctypes.data_as(C.POINTER(C.c_float)),
                                                C.c_void_p(int(dx_ptr)), C.c_void_p(int(stream))), net)
    return g


def vsie_net_step(net, D, H, W, x_ptr, target_ptr, lr, stream=0):
    loss = C.c_double()
    _check_net(load_library().vsie_net_step(net, int(D), int(H), int(W), C.c_void_p(int(x_ptr)),
                                            C.c_void_p(int(target_ptr)), float(lr), C.byref(loss),
                                            C.c_void_p(int(stream))), net)
    return loss.value


def vsie_net_train(ctx, net, steps, lr=1e-3, seed=0, stream=0):
    """Returns the per-step losses."""
    L = np.zeros(max(int(steps), 1), np.float32)
    _check(load_library().vsie_net_train(ctx, net, int(steps), float(lr), int(seed),
                                         L.ctypes.data_as(C.POINTER(C.c_float)), C.c_void_p(int(stream))),
           ctx)
    return L[:int(steps)]


def vsie_net_attach(ctx, net):
    _check(load_library().vsie_net_attach(ctx, net), ctx)


def vsie_net_destroy(net):
    if net:
        load_library().vsie_net_destroy(net)


def vsie_precond_apply(ctx, p, X, ldx, Y, ldy, kind, stream=0):
    """Y = M X with the FP32 preconditioner (kind 0 block, 2 learned)."""
    _check(load_library().vsie_precond_apply(ctx, int(p), C.c_void_p(int(X)), int(ldx), C.c_void_p(int(Y)),
                                             int(ldy), int(kind), C.c_void_p(int(stream))), ctx)


def vsie_solve_batch(ctxs, p, B, ldb, X, ldx, tol, opts=None, nthreads=0):
    """Concurrent solves of independent contexts; returns (status, statuses, infos)."""
    n = len(ctxs)
    lib = load_library()
    P = C.c_void_p
    ca = (P * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    pa = (C.c_int32 * n)(*[int(v) for v in p])
    ba = (P * n)(*[int(v) for v in B])
    xa = (P * n)(*[int(v) for v in X])
    lb = (C.c_int64 * n)(*[int(v) for v in ldb])
    lx = (C.c_int64 * n)(*[int(v) for v in ldx])
    infos = (vsie_solve_info * n)()
    sts = (C.c_int * n)()
    st = lib.vsie_solve_batch(n, ca, pa, ba, lb, xa, lx, float(tol),
                              C.byref(opts) if opts is not None else None, infos, sts, int(nthreads))
    return st, list(sts), list(infos)
