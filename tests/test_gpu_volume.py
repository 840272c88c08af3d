"""GPU parity of the volume operator (K1 fused FFT convolution) against the
oracle: FP64 relative error <= 1e-10, FP32 <= 2e-5, vacuum rows exact."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from oracle import physics, volume
from tests.conftest import gpu_matvec

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


def _ctx(g, er, sg, f, max_rhs=4, ext=None, off=None):
    from paper_2206_12409_gb300 import vsie as V
    return V.vsie_create(V.make_grid(g.n, g.h, g.origin), er, sg, f,
                         V.make_options(ext_n=ext, ext_offset=off, max_rhs=max_rhs))


def _check(g, er, sg, f, p=2, ext=None, off=None, ld_pad=0):
    from paper_2206_12409_gb300 import vsie as V
    chi = physics.chi(er, sg, f)
    _, k0 = physics.omega_k0(f)
    x = I.random_vectors(3 * g.nv, p)
    yo = volume.fft_matvec(g, chi, k0, x)
    M3 = np.tile(chi != 0, 3)
    ctx = _ctx(g, er, sg, f, max_rhs=max(p, 4), ext=ext, off=off)
    try:
        for prec in (V.VSIE_C128, V.VSIE_C64):
            y = gpu_matvec(ctx, x, prec, ld=3 * g.nv + ld_pad)
            err = np.linalg.norm((y - yo)[M3]) / np.linalg.norm(yo[M3])
            assert err <= TOL[prec], (prec, err)
            xv = x if prec == V.VSIE_C128 else x.astype(np.complex64).astype(np.complex128)
            assert np.array_equal(y[~M3], xv[~M3])
    finally:
        V.vsie_destroy(ctx)


@pytest.mark.parametrize("n", [(12, 12, 12), (7, 6, 5), (5, 9, 13), (3, 1, 4), (1, 1, 1)])
def test_volume_sphere(n):
    g, er, sg = I.sphere_phantom(n, 5e-3, 25e-3, 50.0, 0.6)
    _check(g, er, sg, 298e6)


def test_volume_all_material_radix_mix():
    # L = 40 (8*5), 40, 24 (8*3)
    g, er, sg = I.sphere_phantom((20, 20, 12), 5e-3, 1.0, 50.0, 0.6)
    _check(g, er, sg, 298e6, p=3, ld_pad=5)


def test_volume_radix7_and_odd_lengths():
    # L = 14 (2*7), 25 (5^2), 49 (7^2)
    g, er, sg = I.sphere_phantom((7, 13, 25), 4e-3, 1.0, 40.0, 0.3)
    _check(g, er, sg, 123e6, p=1)


def test_volume_body_inside_extended_grid():
    g, er, sg = I.sphere_phantom((6, 5, 4), 5e-3, 1.0, 50.0, 0.6)
    _check(g, er, sg, 298e6, p=2, ext=(9, 8, 7), off=(1, 2, 3))


def test_volume_head_full_size():
    """96 x 96 x 112 head phantom (2 mm), 2 RHS, against the oracle FFT product."""
    g, er, sg = I.layered_head_phantom()
    _check(g, er, sg, 298e6, p=2, ext=(128, 128, 112), off=(16, 16, 0))


# z-pass variants of the FP32 operator (the generic half-length Stockham kernels
# come first, 7 of them; then the register kernels: 7-9 k_zreg, 10 k_zreg_st with
# 8 lines per CTA, 11 k_zreg_st with 16 lines, M = 112 only)
@pytest.mark.parametrize("zv", [9, 10, 11])
def test_volume_head_z_variants(zv, monkeypatch):
    """Every register z-pass variant on the 2 mm head grid against the oracle
    (forced through VSIE_ZPASS_VARIANT; 3 RHS, so the staged kernel's loop over
    right-hand sides and its prefetch run)."""
    monkeypatch.setenv("VSIE_ZPASS_VARIANT", str(zv))
    g, er, sg = I.layered_head_phantom()
    _check(g, er, sg, 298e6, p=3, ext=(128, 128, 112), off=(16, 16, 0))
