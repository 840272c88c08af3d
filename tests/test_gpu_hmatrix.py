"""Hierarchical far-far block (include/vsie.h, far_hmatrix): the H-matrix product
against the oracle's dense Z_ff (oracle.efie, the definition of the block), the
rest of the operator unchanged against a dense-block context, and the mixed
solve on the hierarchical operator.  The low-rank blocks are ACA approximations
at aca_tol (1e-6 here), so the far rows differ from the dense product by at most
a small multiple of it, and by more than rounding (the compression is in use)."""
import numpy as np
import pytest

from paper_2206_12409_gb300 import inputs as I
from tests.conftest import gpu_matvec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm_ctx(sphere_loop_shield):
    from paper_2206_12409_gb300 import vsie as V
    ctx = V.setup_problem(sphere_loop_shield, max_rhs=4, far_hmatrix=1, hm_leaf=64)
    yield ctx
    V.vsie_destroy(ctx)


def test_hmatrix_far_block_against_oracle(hm_ctx, hybrid_parts):
    from paper_2206_12409_gb300 import vsie as V
    N, mf, mn, nb = V.vsie_sizes(hm_ctx)
    assert mf == hybrid_parts.m_f
    x = np.zeros((N, 3), complex)
    x[:mf] = I.random_vectors(mf, 3, seed=61)
    yo = hybrid_parts.Zff @ x[:mf]
    for prec, tol in ((V.VSIE_C128, 1e-5), (V.VSIE_C64, 2e-5)):
        y = gpu_matvec(hm_ctx, x, prec)
        e = np.linalg.norm(y[:mf] - yo) / np.linalg.norm(yo)
        print(f"[H-matrix far block] precision={prec} rel_err={e:.2e}")
        assert e <= tol
        if prec == V.VSIE_C128:
            assert e > 1e-13            # low-rank blocks are in use


def test_hmatrix_leaves_the_other_blocks_unchanged(hm_ctx, sphere_loop_shield):
    from paper_2206_12409_gb300 import vsie as V
    dense = V.setup_problem(sphere_loop_shield, max_rhs=4, far_hmatrix=-1)
    try:
        N, mf, mn, nb = V.vsie_sizes(hm_ctx)
        x = I.random_vectors(N, 2, seed=62)
        yh = gpu_matvec(hm_ctx, x, V.VSIE_C128)
        yd = gpu_matvec(dense, x, V.VSIE_C128)
        rest = slice(mf, None)
        assert np.linalg.norm(yh[rest] - yd[rest]) <= 1e-13 * np.linalg.norm(yd[rest])
        assert np.linalg.norm(yh[:mf] - yd[:mf]) <= 1e-5 * np.linalg.norm(yd[:mf])
    finally:
        V.vsie_destroy(dense)


def test_hmatrix_mixed_solve_and_limits(hm_ctx):
    import torch
    from paper_2206_12409_gb300 import vsie as V
    N = V.vsie_sizes(hm_ctx)[0]
    B = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
    V.vsie_rhs_ports(hm_ctx, [0], 1.0, B.data_ptr(), N)
    X = torch.zeros_like(B)
    o = V.vsie_solve_opts()
    o.mode, o.restart, o.maxit, o.inner_tol = 1, 50, 3000, 1e-3
    st, info = V.vsie_solve(hm_ctx, 1, B.data_ptr(), N, X.data_ptr(), N, 1e-6, o)
    assert st == V.VSIE_OK and info.relres[0] <= 1e-6
    o.mode = 0
    with pytest.raises(V.VsieError) as e:
        V.vsie_solve(hm_ctx, 1, B.data_ptr(), N, X.data_ptr(), N, 1e-6, o)
    assert e.value.status == V.VSIE_EUNSUPPORTED
    with pytest.raises(V.VsieError) as e:
        V.vsie_get_parts(hm_ctx)
    assert e.value.status == V.VSIE_EUNSUPPORTED
